"""GB300-native explicit heat stencil and CG solver (arXiv 2608.11882, Sections 4 and 7.5).

The compute path is the CUDA library ``libheatcg.so`` (C ABI in include/heatcg.h),
built in-tree by ``paper_2608_11882_gb300.build.build()``.  ``_native`` is the
ctypes binding under the C names; ``api`` adds Heat, Operator and CG.  Those
names load the library on first use and raise ImportError if it is not built:
there is no CPU fallback.
"""
_API = {"Heat", "HeatBatch", "Operator", "CG", "CGBatch", "HeatCGError", "HS_F64", "HS_F32", "HS_ALLOW_UNSTABLE",
        "HS_EXACT_ROUNDING", "HS_SCHED_FULL", "HS_FIXED64", "HS_VARKAPPA", "HS_FP64_PIPE", "HS_OP_STENCIL7", "HS_OP_CSR", "native"}

__all__ = sorted(_API)


def __getattr__(name):
    if name in _API:
        from . import api
        return getattr(api, name)
    raise AttributeError(f"module 'paper_2608_11882_gb300' has no attribute {name!r}")
