"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/heatcg.h declares; the binding mirrors the
header's structs.  No compute call is made (no GPU here)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent


def declared_functions():
    text = (ROOT / "include" / "heatcg.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2608_11882_gb300.build import build
    lib = ctypes.CDLL(str(build()))
    names = declared_functions()
    assert "heat_create" in names and "cg_solve" in names and "heat_interior" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_struct_sizes_match_header_layout():
    from paper_2608_11882_gb300 import _native as nat
    # hs_heat_desc: 3*int32 + pad, double, uint32, int32, int32 + pad, 3 * void*
    assert ctypes.sizeof(nat.hs_heat_desc) == 64
    assert ctypes.sizeof(nat.hs_op) == 64
    assert ctypes.sizeof(nat.hs_cg_info) == 32
    assert ctypes.sizeof(nat.hs_cg_mixed_opts) == 16


def test_version_and_error_string_without_gpu():
    from paper_2608_11882_gb300 import _native as nat
    assert nat.lib.hs_version() >= 100
    assert isinstance(nat.last_error(), str)
    # argument validation happens before any CUDA call
    desc = nat.hs_heat_desc(nx=0, ny=1, nz=1, r=0.1, flags=0, dtype=0, tdepth=0, stream=None)
    h = ctypes.c_void_p()
    assert nat.lib.heat_create(ctypes.byref(h), ctypes.byref(desc)) == nat.HS_EINVAL
    assert "interior" in nat.last_error()
    desc = nat.hs_heat_desc(nx=4, ny=4, nz=4, r=0.2, flags=0, dtype=0, tdepth=0, stream=None)
    assert nat.lib.heat_create(ctypes.byref(h), ctypes.byref(desc)) == nat.HS_EUNSTABLE
    size = ctypes.c_size_t()
    desc.r = 0.1
    assert nat.lib.heat_device_bytes(ctypes.byref(desc), ctypes.byref(size)) == 0
    # two padded buffers (pitch 16, (ny+2)(nz+2) rows, 8-byte values) + the
    # 64-byte per-step state of the default FP64 arithmetic
    assert size.value == 2 * 6 * 6 * 16 * 8 + 64
    desc.flags = nat.HS_FP64_PIPE   # the FP64-pipe arithmetic keeps no per-step state
    assert nat.lib.heat_device_bytes(ctypes.byref(desc), ctypes.byref(size)) == 0
    assert size.value == 2 * 6 * 6 * 16 * 8


def test_timing_entry_points_reject_null_handles():
    from paper_2608_11882_gb300 import _native as nat
    ms, n = ctypes.c_double(), ctypes.c_int64()
    assert nat.lib.heat_time_interior(None, 1) == nat.HS_EINVAL
    assert nat.lib.heat_interior_time(None, ctypes.byref(ms), ctypes.byref(n)) == nat.HS_EINVAL
    assert "NULL handle" in nat.last_error()


def test_caller_buffer_checks_without_gpu():
    """heat_buffer_bytes gives one padded buffer; caller-owned buffers that are
    half given, misaligned or overlapping are refused before any CUDA call."""
    from paper_2608_11882_gb300 import _native as nat
    desc = nat.hs_heat_desc(nx=4, ny=4, nz=4, r=0.1, flags=0, dtype=0, tdepth=0, stream=None)
    size = ctypes.c_size_t()
    assert nat.lib.heat_buffer_bytes(ctypes.byref(desc), ctypes.byref(size)) == 0
    assert size.value == 6 * 6 * 16 * 8
    one = size.value
    h = ctypes.c_void_p()
    for b0, b1, what in ((4096, None, "both"), (4096 + 8, 1 << 20, "aligned"),
                         (1 << 20, (1 << 20) + 256, "overlap"), (1 << 20, 1 << 20, "overlap")):
        desc.dev_buf0, desc.dev_buf1 = b0, b1
        assert nat.lib.heat_create(ctypes.byref(h), ctypes.byref(desc)) == nat.HS_EINVAL
        assert what in nat.last_error()
    # caller buffers: the library allocates only the per-step state
    desc.dev_buf0, desc.dev_buf1 = 1 << 20, (1 << 20) + one
    assert nat.lib.heat_device_bytes(ctypes.byref(desc), ctypes.byref(size)) == 0
    assert size.value == 64
