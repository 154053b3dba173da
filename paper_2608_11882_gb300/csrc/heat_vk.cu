// The paper's variable-coefficient heat problem (Section 4, Eqs. 1-4):
//     du/dt = div(kappa grad u) + f,  kappa = 0.5 + 0.45 sin(pi x) sin(pi y) sin(pi z),
//     f = 1 + cos(pi x) cos(pi y) cos(pi z),
//     u' = u + dt f + sum_d dt/(2 h_d^2) D_d(u),
//     D_x = (k[i+1] + k[i]) (u[i+1] - u[i]) - (k[i] + k[i-1]) (u[i] - u[i-1])
// (face-averaged kappa: the reading of the unprinted D that matches
// beta = dt/(2h^2)).  As in the paper's Algorithm "1-GPU Baseline", the
// coefficients and dt f are arrays resident beside u, dt f on the interior.
// Interior and Boundary kernels as for the constant-coefficient update.
//
// FP32 keeps kappa on every node of the padded box (16 bytes per update:
// the kernel is bound by HBM, where three face arrays would cost more than the
// six additions they save).  FP64 keeps the three face sums k[i+1] + k[i] of
// each node instead (constant in time, formed once at creation, bit for bit
// the sums the formula forms every step), 48 bytes per update, and forms the
// operator sums exactly in 128-bit integers on the field's fixed-point scale,
// each rounded once: 2 FP64 instructions per update on a cubic grid (one beta
// for every axis: the paper's case), 5 otherwise.  Fields outside the exact
// form's exponent range use the FP64 form, 16 FP64 instructions per update
// with the z difference u[k+1] - u[k] carried to the next plane (23 with kappa
// itself).
#include <cmath>

#include "heat_common.cuh"

namespace hcg {

constexpr int kVkBX = 32, kVkBY = 8;

// kappa on every padded node, dt f on interior nodes (zero on the boundary).
template <typename T>
__global__ void __launch_bounds__(256) k_vk_init(T* __restrict__ kap, T* __restrict__ fdt, HeatGeom g,
                                                 double dt)
{
    const double hx = 1.0 / (g.nx + 1), hy = 1.0 / (g.ny + 1), hz = 1.0 / (g.nz + 1);
    const int64_t n = (int64_t)(g.nx + 2) * (g.ny + 2) * (g.nz + 2);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(t % (g.nx + 2));
        const int64_t jk = t / (g.nx + 2);
        const int J = (int)(jk % (g.ny + 2));
        const int K = (int)(jk / (g.ny + 2));
        const int64_t c = (int64_t)K * g.plane + (int64_t)J * g.pitch + g.lead - 1 + I;
        const double x = I * hx, y = J * hy, z = K * hz;
        kap[c] = (T)(0.5 + 0.45 * sinpi(x) * sinpi(y) * sinpi(z));
        const bool interior = I >= 1 && I <= g.nx && J >= 1 && J <= g.ny && K >= 1 && K <= g.nz;
        fdt[c] = interior ? (T)(dt * (1.0 + cospi(x) * cospi(y) * cospi(z))) : (T)0;
    }
}

// FP64: the three face sums of kappa on every padded node (f*[c] = kappa at the
// node's +d neighbour + kappa at the node, zero where that neighbour lies
// outside the padded box) and dt f on the interior.  The kappa values are the
// same expression as k_vk_init's, so the sums are the bits the formula forms.
// Sets *off = 1 if a face sum lies outside [1, 2), where the exact-sum form's
// 53-bit significands would not hold it (kappa in [0.5, 1) keeps every face
// sum inside).
__global__ void __launch_bounds__(256) k_vk_init_faces(double* __restrict__ fc, double* __restrict__ fdt,
                                                       HeatGeom g, double dt, int* off)
{
    const double hx = 1.0 / (g.nx + 1), hy = 1.0 / (g.ny + 1), hz = 1.0 / (g.nz + 1);
    const int64_t n = (int64_t)(g.nx + 2) * (g.ny + 2) * (g.nz + 2);
    auto kappa = [&](int I, int J, int K) {
        return 0.5 + 0.45 * sinpi(I * hx) * sinpi(J * hy) * sinpi(K * hz);
    };
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(t % (g.nx + 2));
        const int64_t jk = t / (g.nx + 2);
        const int J = (int)(jk % (g.ny + 2));
        const int K = (int)(jk / (g.ny + 2));
        const int64_t c = (int64_t)K * g.plane + (int64_t)J * g.pitch + g.lead - 1 + I;
        const double kc = kappa(I, J, K);
        const double sx = kappa(I + 1, J, K) + kc, sy = kappa(I, J + 1, K) + kc, sz = kappa(I, J, K + 1) + kc;
        fc[c] = I <= g.nx ? sx : 0.0;
        fc[g.total + c] = J <= g.ny ? sy : 0.0;
        fc[2 * g.total + c] = K <= g.nz ? sz : 0.0;
        auto out = [](double v) { return !(v >= 1.0 && v < 2.0); };
        if ((I <= g.nx && out(sx)) || (J <= g.ny && out(sy)) || (K <= g.nz && out(sz))) atomicOr(off, 1);
        const bool interior = I >= 1 && I <= g.nx && J >= 1 && J <= g.ny && K >= 1 && K <= g.nz;
        fdt[c] = interior ? dt * (1.0 + cospi(I * hx) * cospi(J * hy) * cospi(K * hz)) : 0.0;
    }
}

// One FP64 update from the face sums: cxp = k[i+1] + k[i], cxm = k[i] + k[i-1]
// (the -x neighbour's +x face) and so on, and the z difference below the
// point, dzm = u[k] - u[k-1], carried from the plane below.
__device__ __forceinline__ double vk_point_faces(double uc, double uxm, double uxp, double uym, double uyp,
                                                 double dzp, double dzm, double cxm, double cxp, double cym,
                                                 double cyp, double czm, double czp, double f, double bx,
                                                 double by, double bz)
{
    const double dx = __fma_rn(cxp, __dsub_rn(uxp, uc), -__dmul_rn(cxm, __dsub_rn(uc, uxm)));
    const double dy = __fma_rn(cyp, __dsub_rn(uyp, uc), -__dmul_rn(cym, __dsub_rn(uc, uym)));
    const double dz = __fma_rn(czp, dzp, -__dmul_rn(czm, dzm));
    return __dadd_rn(__dadd_rn(uc, f), __fma_rn(bz, dz, __fma_rn(by, dy, __dmul_rn(bx, dx))));
}

__global__ void __launch_bounds__(kVkBX* kVkBY)
    k_vk_interior_faces(const double* __restrict__ src, double* __restrict__ dst, const double* __restrict__ fc,
                        const double* __restrict__ fdt, HeatGeom g, double bx, double by, double bz, int kbeg,
                        int kend, int kchunk)
{
    const int i = blockIdx.x * kVkBX + threadIdx.x;
    const int j = blockIdx.y * kVkBY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int k0 = kbeg + (int)blockIdx.z * kchunk;
    const int k1 = min(k0 + kchunk, kend);
    if (k0 >= k1) return;
    const int64_t P = g.plane, Y = g.pitch;
    const double* fx = fc;
    const double* fy = fc + g.total;
    const double* fz = fc + 2 * g.total;
    int64_t c = g.at(i, j, k0);
    double uc = __ldg(src + c);
    double dzm = __dsub_rn(uc, __ldg(src + c - P));
    double czm = __ldg(fz + c - P);
    for (int k = k0; k < k1; ++k) {
        const double ua = __ldg(src + c + P), cza = __ldg(fz + c);
        const double dzp = __dsub_rn(ua, uc);
        dst[c] = vk_point_faces(uc, __ldg(src + c - 1), __ldg(src + c + 1), __ldg(src + c - Y),
                                __ldg(src + c + Y), dzp, dzm, __ldg(fx + c - 1), __ldg(fx + c),
                                __ldg(fy + c - Y), __ldg(fy + c), czm, cza, __ldg(fdt + c), bx, by, bz);
        uc = ua;
        dzm = dzp;
        czm = cza;
        c += P;
    }
}

__global__ void __launch_bounds__(kVkBX* kVkBY)
    k_vk_boundary_faces(const double* __restrict__ src, double* __restrict__ dst, const double* __restrict__ fc,
                        const double* __restrict__ fdt, HeatGeom g, double bx, double by, double bz)
{
    const int i = blockIdx.x * kVkBX + threadIdx.x;
    const int j = blockIdx.y * kVkBY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int k = (blockIdx.z == 0) ? 0 : g.nz - 1;
    const int64_t P = g.plane, Y = g.pitch;
    const int64_t c = g.at(i, j, k);
    const double* fx = fc;
    const double* fy = fc + g.total;
    const double* fz = fc + 2 * g.total;
    const double uc = __ldg(src + c);
    dst[c] = vk_point_faces(uc, __ldg(src + c - 1), __ldg(src + c + 1), __ldg(src + c - Y), __ldg(src + c + Y),
                            __dsub_rn(__ldg(src + c + P), uc), __dsub_rn(uc, __ldg(src + c - P)),
                            __ldg(fx + c - 1), __ldg(fx + c), __ldg(fy + c - Y), __ldg(fy + c),
                            __ldg(fz + c - P), __ldg(fz + c), __ldg(fdt + c), bx, by, bz);
}

// ---- FP64, exact sum ------------------------------------------------------
// The operator sums D_d = c_d+ (u_d+ - u) - c_d- (u - u_d-) on the field's
// fixed-point scale: U the exact-sum integers of the u values (xsum.cuh, the
// scale 2^(1080 - e) of the field's largest exponent field e, tracked per step
// in the handle's FxState like the default FP64 arithmetic's), C the face
// sums' 53-bit significands (every face sum of kappa = 0.5 + 0.45 s, s in
// [0, 1], lies in [1, 2), so C = c 2^52 exactly; heat_create checks it), each
// product C dU exact and their sums exact in 128 bits.  On a cubic grid (one
// beta for every axis, the paper's case) the whole operator sum is rounded
// once and u' = fma(beta, D, u + dt f): two FP64 instructions per update
// instead of sixteen; otherwise each axis sum is rounded once and combined as
// the FP64 form combines them, five FP64 instructions.  The error against the
// same formula in exact arithmetic is below 6 * 2 * 1.9 * 4 * 2^-57 max|u|
// beta plus a few roundings.  Fields whose exponent lies outside
// [kVkEmaxLo, kVkEmaxHi] (all-zero or tiny fields, values near overflow, NaN,
// Inf) take the FP64 form of vk_point_faces.
constexpr int kVkEmaxLo = 120, kVkEmaxHi = 2030;

__device__ __forceinline__ unsigned long long vk_face_sig(double c)
{
    // significand of c in [1, 2), its implicit bit included
    return ((unsigned long long)__double_as_longlong(c) & 0x000fffffffffffffull) | 0x0010000000000000ull;
}

__device__ __forceinline__ bool vk_exact_ok(int emax) { return emax >= kVkEmaxLo && emax <= kVkEmaxHi; }

// u' from the exact operator sums: one sum (all axes) rounded once on a cubic
// grid, u' = fma(beta, D, u + dt f); else the three axis sums, each rounded
// once, combined as the FP64 form combines them: (u + dt f) + ((bx Dx + by Dy)
// + bz Dz).  C dU carries the scale 2^52 2^(1080 - e).
template <bool CUBIC>
__device__ __forceinline__ double vk_combine(double uc, double f, I128 dx, I128 dy, I128 dz, double bx, double by,
                                             double bz, int emax)
{
    if constexpr (CUBIC) {
        const double D = i128_to_double(i128_add(i128_add(dx, dy), dz), emax - 1132);
        return __fma_rn(bx, D, __dadd_rn(uc, f));
    } else {
        const double Dx = i128_to_double(dx, emax - 1132), Dy = i128_to_double(dy, emax - 1132),
                     Dz = i128_to_double(dz, emax - 1132);
        return __dadd_rn(__dadd_rn(uc, f), __fma_rn(bz, Dz, __fma_rn(by, Dy, __dmul_rn(bx, Dx))));
    }
}

// One update on the exact path from the seven u values (as doubles, the centre
// also as its integer), the six face sums and dt f.
template <bool CUBIC>
__device__ __forceinline__ double vk_point_exact(double uc, long long Uc, long long Uxm, long long Uxp,
                                                 long long Uym, long long Uyp, long long dzp, long long dzm,
                                                 double cxm, double cxp, double cym, double cyp, double czm,
                                                 double czp, double f, double bx, double by, double bz, int emax)
{
    const I128 dx = i128_sub(i128_mul(vk_face_sig(cxp), Uxp - Uc), i128_mul(vk_face_sig(cxm), Uc - Uxm));
    const I128 dy = i128_sub(i128_mul(vk_face_sig(cyp), Uyp - Uc), i128_mul(vk_face_sig(cym), Uc - Uym));
    const I128 dz = i128_sub(i128_mul(vk_face_sig(czp), dzp), i128_mul(vk_face_sig(czm), dzm));
    return vk_combine<CUBIC>(uc, f, dx, dy, dz, bx, by, bz, emax);
}

// Interior (planes kbeg..kend-1) of an FP64 grid: the exact sums while the
// field's exponent allows it, the FP64 form otherwise; every output joins the
// step's maximum (slot (m3 + 1) % 3).  Every thread takes two consecutive x
// points (16-byte loads of u, the face sums and dt f): four conversions per
// point and half the load instructions of one point per thread, whose loads
// left the kernel waiting on memory; three blocks per SM at 80 registers.
// The products through the face between a thread's two points and through the
// face below a plane (the face above it one plane earlier) are formed once: 9
// products for two points instead of 12, and the sums stay exact, so the
// result is the same.  Measured at 510^3: one point per thread 57 GLUP/s, two
// points 77, shared fluxes 85; staging each plane through shared memory so
// that every value is converted once (one block barrier per plane) 55, 71 with
// the staging loads issued one plane ahead.  A thread whose second point is
// the boundary node nx computes only the first.
template <bool CUBIC>
__global__ void __launch_bounds__(kVkBX* kVkBY, 3)
    k_vk_interior_xs(const double* __restrict__ src, double* __restrict__ dst, const double* __restrict__ fc,
                      const double* __restrict__ fdt, HeatGeom g, double bx, double by, double bz, int kbeg,
                      int kend, int kchunk, FxState* fx, int m3)
{
    const int i0 = (blockIdx.x * kVkBX + threadIdx.x) * 2;
    const int j = blockIdx.y * kVkBY + threadIdx.y;
    const int k0 = kbeg + (int)blockIdx.z * kchunk;
    const int k1 = min(k0 + kchunk, kend);
    const int emax = xs_emax(fx, m3);
    unsigned mx = 0;
    if (i0 < g.nx && j < g.ny && k0 < k1) {
        const bool two = i0 + 1 < g.nx;
        const int64_t P = g.plane, Y = g.pitch;
        const double* fxs = fc;
        const double* fys = fc + g.total;
        const double* fzs = fc + 2 * g.total;
        auto ld2 = [](const double* p, double (&o)[2]) {
            const double2 v = __ldg(reinterpret_cast<const double2*>(p));
            o[0] = v.x;
            o[1] = v.y;
        };
        int64_t c = g.at(i0, j, k0);
        if (vk_exact_ok(emax)) {
            // D = sum over faces of +- F, F = C (U beyond the face - U before it):
            // the face between the thread's two points and the face below the
            // plane (the face above the plane before) are each formed once
            auto fix = [emax](double v) { return xs_fix(__double_as_longlong(v), emax); };
            double uc[2], t[2], czm[2];
            long long Uc[2];
            I128 fzm[2];   // the flux through the face below plane k
            ld2(src + c, uc);
            ld2(src + c - P, t);
            ld2(fzs + c - P, czm);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                Uc[q] = fix(uc[q]);
                fzm[q] = i128_mul(vk_face_sig(czm[q]), Uc[q] - fix(t[q]));
            }
            for (int k = k0; k < k1; ++k) {
                double ua[2], ym[2], yp[2], cx[2], cym[2], cyp[2], cza[2], f[2];
                ld2(src + c + P, ua);
                ld2(src + c - Y, ym);
                ld2(src + c + Y, yp);
                ld2(fxs + c, cx);
                ld2(fys + c - Y, cym);
                ld2(fys + c, cyp);
                ld2(fzs + c, cza);
                ld2(fdt + c, f);
                const long long Uxm = fix(__ldg(src + c - 1)), Uxp = fix(__ldg(src + c + 2));
                const double cxm0 = __ldg(fxs + c - 1);
                const I128 fa = i128_mul(vk_face_sig(cxm0), Uc[0] - Uxm);   // face i0 - 1/2
                const I128 fb = i128_mul(vk_face_sig(cx[0]), Uc[1] - Uc[0]);  // face i0 + 1/2
                const I128 fcx = i128_mul(vk_face_sig(cx[1]), Uxp - Uc[1]);  // face i0 + 3/2
                long long Ua[2];
                double v[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    Ua[q] = fix(ua[q]);
                    const I128 fzp = i128_mul(vk_face_sig(cza[q]), Ua[q] - Uc[q]);
                    const I128 dx = q == 0 ? i128_sub(fb, fa) : i128_sub(fcx, fb);
                    const I128 dy = i128_sub(i128_mul(vk_face_sig(cyp[q]), fix(yp[q]) - Uc[q]),
                                             i128_mul(vk_face_sig(cym[q]), Uc[q] - fix(ym[q])));
                    const I128 dz = i128_sub(fzp, fzm[q]);
                    fzm[q] = fzp;
                    v[q] = vk_combine<CUBIC>(uc[q], f[q], dx, dy, dz, bx, by, bz, emax);
                }
                if (two) {
                    *reinterpret_cast<double2*>(dst + c) = make_double2(v[0], v[1]);
                } else {
                    dst[c] = v[0];
                    v[1] = 0.0;
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const unsigned a = xs_abs_hi(v[q]);
                    mx = a > mx ? a : mx;
                    uc[q] = ua[q];
                    Uc[q] = Ua[q];
                }
                c += P;
            }
        } else {
            // outside the exact form's range: the FP64 form, point by point
            for (int q = 0; q < (two ? 2 : 1); ++q) {
                int64_t cq = c + q;
                double u = __ldg(src + cq);
                double dzmq = __dsub_rn(u, __ldg(src + cq - P));
                double czmq = __ldg(fzs + cq - P);
                for (int k = k0; k < k1; ++k) {
                    const double ua = __ldg(src + cq + P), cza = __ldg(fzs + cq);
                    const double dzp = __dsub_rn(ua, u);
                    const double w = vk_point_faces(u, __ldg(src + cq - 1), __ldg(src + cq + 1), __ldg(src + cq - Y),
                                                    __ldg(src + cq + Y), dzp, dzmq, __ldg(fxs + cq - 1), __ldg(fxs + cq),
                                                    __ldg(fys + cq - Y), __ldg(fys + cq), czmq, cza, __ldg(fdt + cq),
                                                    bx, by, bz);
                    dst[cq] = w;
                    const unsigned a = xs_abs_hi(w);
                    mx = a > mx ? a : mx;
                    u = ua;
                    dzmq = dzp;
                    czmq = cza;
                    cq += P;
                }
            }
        }
    }
    fx_finish<kVkBX * kVkBY>((unsigned long long)mx << 32, fx, m3, 0,
                             blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0);
}

// Boundary planes 0 and nz-1 of an FP64 grid, as k_vk_interior_xs (one
// point per thread).
template <bool CUBIC>
__global__ void __launch_bounds__(kVkBX* kVkBY)
    k_vk_boundary_xs(const double* __restrict__ src, double* __restrict__ dst, const double* __restrict__ fc,
                     const double* __restrict__ fdt, HeatGeom g, double bx, double by, double bz, FxState* fx,
                     int m3)
{
    const int i = blockIdx.x * kVkBX + threadIdx.x;
    const int j = blockIdx.y * kVkBY + threadIdx.y;
    const int emax = xs_emax(fx, m3);
    unsigned mx = 0;
    if (i < g.nx && j < g.ny) {
        const int k = (blockIdx.z == 0) ? 0 : g.nz - 1;
        const int64_t P = g.plane, Y = g.pitch;
        const int64_t c = g.at(i, j, k);
        const double* fxs = fc;
        const double* fys = fc + g.total;
        const double* fzs = fc + 2 * g.total;
        const double uc = __ldg(src + c);
        double v;
        if (vk_exact_ok(emax)) {
            auto fix = [emax](double w) { return xs_fix(__double_as_longlong(w), emax); };
            const long long Uc = fix(uc);
            v = vk_point_exact<CUBIC>(uc, Uc, fix(__ldg(src + c - 1)), fix(__ldg(src + c + 1)),
                                      fix(__ldg(src + c - Y)), fix(__ldg(src + c + Y)),
                                      fix(__ldg(src + c + P)) - Uc, Uc - fix(__ldg(src + c - P)),
                                      __ldg(fxs + c - 1), __ldg(fxs + c), __ldg(fys + c - Y), __ldg(fys + c),
                                      __ldg(fzs + c - P), __ldg(fzs + c), __ldg(fdt + c), bx, by, bz, emax);
        } else {
            v = vk_point_faces(uc, __ldg(src + c - 1), __ldg(src + c + 1), __ldg(src + c - Y), __ldg(src + c + Y),
                               __dsub_rn(__ldg(src + c + P), uc), __dsub_rn(uc, __ldg(src + c - P)),
                               __ldg(fxs + c - 1), __ldg(fxs + c), __ldg(fys + c - Y), __ldg(fys + c),
                               __ldg(fzs + c - P), __ldg(fzs + c), __ldg(fdt + c), bx, by, bz);
        }
        dst[c] = v;
        mx = xs_abs_hi(v);
    }
    fx_finish<kVkBX * kVkBY>((unsigned long long)mx << 32, fx, m3, 0,
                             blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0);
}

template <typename T>
__device__ __forceinline__ T vk_point(T uc, T uxm, T uxp, T uym, T uyp, T uzm, T uzp, T kc, T kxm, T kxp,
                                      T kym, T kyp, T kzm, T kzp, T f, T bx, T by, T bz)
{
    const T dx = (kxp + kc) * (uxp - uc) - (kc + kxm) * (uc - uxm);
    const T dy = (kyp + kc) * (uyp - uc) - (kc + kym) * (uc - uym);
    const T dz = (kzp + kc) * (uzp - uc) - (kc + kzm) * (uc - uzm);
    return (uc + f) + ((bx * dx + by * dy) + bz * dz);
}

// FP32 Interior: every thread four consecutive x points (one 16-byte vector
// of u, kappa and dt f per row), so a point costs about 3.5 load instructions
// instead of 11; the update of each point is vk_point's.  A thread whose four
// points run past nx loads element by element up to the boundary node nx (u
// zero there, kappa not) and computes only its interior points.  The kernel
// waits on its loads (long-scoreboard stalls): four blocks per SM at 64
// registers, with 8-plane chunks, ran 340 GLUP/s at 510^3 against 265 with
// three blocks at 80 registers.
__global__ void __launch_bounds__(kVkBX* kVkBY, 4)
    k_vk_interior_f4(const float* __restrict__ src, float* __restrict__ dst, const float* __restrict__ kap,
                     const float* __restrict__ fdt, HeatGeom g, float bx, float by, float bz, int kbeg, int kend,
                     int kchunk)
{
    const int i0 = (blockIdx.x * kVkBX + threadIdx.x) * 4;
    const int j = blockIdx.y * kVkBY + threadIdx.y;
    if (i0 >= g.nx || j >= g.ny) return;
    const int k0 = kbeg + (int)blockIdx.z * kchunk;
    const int k1 = min(k0 + kchunk, kend);
    if (k0 >= k1) return;
    const int64_t P = g.plane, Y = g.pitch;
    const bool full = i0 + 3 < g.nx;
    const int nv = min(4, g.nx - i0);   // interior points of this thread
    auto ld4 = [&](const float* p, float (&o)[4]) {
        if (full) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(p));
            o[0] = v.x;
            o[1] = v.y;
            o[2] = v.z;
            o[3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = i0 + q <= g.nx ? __ldg(p + q) : 0.0f;
        }
    };
    int64_t c = g.at(i0, j, k0);
    float ub[4], uc[4], kb[4], kc[4];
    ld4(src + c - P, ub);
    ld4(src + c, uc);
    ld4(kap + c - P, kb);
    ld4(kap + c, kc);
    for (int k = k0; k < k1; ++k) {
        float ua[4], ka[4], uym[4], uyp[4], kym[4], kyp[4], f[4];
        ld4(src + c + P, ua);
        ld4(kap + c + P, ka);
        ld4(src + c - Y, uym);
        ld4(src + c + Y, uyp);
        ld4(kap + c - Y, kym);
        ld4(kap + c + Y, kyp);
        ld4(fdt + c, f);
        const float uL = __ldg(src + c - 1), kL = __ldg(kap + c - 1);
        const float uR = full ? __ldg(src + c + 4) : 0.0f, kR = full ? __ldg(kap + c + 4) : 0.0f;
        float o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float uxm = q == 0 ? uL : uc[q - 1], uxp = q == 3 ? uR : uc[q + 1];
            const float kxm = q == 0 ? kL : kc[q - 1], kxp = q == 3 ? kR : kc[q + 1];
            o[q] = vk_point<float>(uc[q], uxm, uxp, uym[q], uyp[q], ub[q], ua[q], kc[q], kxm, kxp, kym[q], kyp[q],
                                   kb[q], ka[q], f[q], bx, by, bz);
        }
        if (full) {
            *reinterpret_cast<float4*>(dst + c) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nv) dst[c + q] = o[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ub[q] = uc[q];
            uc[q] = ua[q];
            kb[q] = kc[q];
            kc[q] = ka[q];
        }
        c += P;
    }
}

template <typename T>
__global__ void __launch_bounds__(kVkBX* kVkBY)
    k_vk_boundary(const T* __restrict__ src, T* __restrict__ dst, const T* __restrict__ kap,
                  const T* __restrict__ fdt, HeatGeom g, T bx, T by, T bz)
{
    const int i = blockIdx.x * kVkBX + threadIdx.x;
    const int j = blockIdx.y * kVkBY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int k = (blockIdx.z == 0) ? 0 : g.nz - 1;
    const int64_t P = g.plane, Y = g.pitch;
    const int64_t c = g.at(i, j, k);
    dst[c] = vk_point<T>(__ldg(src + c), __ldg(src + c - 1), __ldg(src + c + 1), __ldg(src + c - Y),
                         __ldg(src + c + Y), __ldg(src + c - P), __ldg(src + c + P), __ldg(kap + c),
                         __ldg(kap + c - 1), __ldg(kap + c + 1), __ldg(kap + c - Y), __ldg(kap + c + Y),
                         __ldg(kap + c - P), __ldg(kap + c + P), __ldg(fdt + c), bx, by, bz);
}

int vk_init(const VkCall& c, double dt)
{
    const int64_t n = (int64_t)(c.g->nx + 2) * (c.g->ny + 2) * (c.g->nz + 2);
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)kNumSMs * 16) blocks = (int64_t)kNumSMs * 16;
    if (c.f64)
        k_vk_init_faces<<<(unsigned)blocks, 256, 0, c.stream>>>((double*)c.kap, (double*)c.fdt, *c.g, dt,
                                                                c.face_off);
    else
        k_vk_init<float><<<(unsigned)blocks, 256, 0, c.stream>>>((float*)c.kap, (float*)c.fdt, *c.g, dt);
    HS_CHECK_LAUNCH("heat: kappa/source init kernel");
    return HS_OK;
}

template <typename T>
int vk_launch_t(const VkCall& c)
{
    const HeatGeom& g = *c.g;
    dim3 block(kVkBX, kVkBY, 1);
    const T bx = (T)c.bx, by = (T)c.by, bz = (T)c.bz;
    constexpr bool kFaces = std::is_same<T, double>::value;
    if (c.part == 0) {
        if (g.nz < 3) return HS_OK;
        const int kbeg = 1, kend = g.nz - 1;
        const int nchunks = (kend - kbeg + c.kchunk - 1) / c.kchunk;
        dim3 grid((g.nx + kVkBX - 1) / kVkBX, (g.ny + kVkBY - 1) / kVkBY, nchunks);
        if constexpr (kFaces) {
            if (c.fx) {
                dim3 grid2((g.nx + 2 * kVkBX - 1) / (2 * kVkBX), grid.y, grid.z);
                auto kern = (bx == by && by == bz) ? k_vk_interior_xs<true> : k_vk_interior_xs<false>;
                kern<<<grid2, block, 0, c.stream>>>((const double*)c.src, (double*)c.dst, (const double*)c.kap,
                                                    (const double*)c.fdt, g, bx, by, bz, kbeg, kend, c.kchunk,
                                                    c.fx, c.m3);
            }
            else
                k_vk_interior_faces<<<grid, block, 0, c.stream>>>((const double*)c.src, (double*)c.dst,
                                                                  (const double*)c.kap, (const double*)c.fdt, g,
                                                                  bx, by, bz, kbeg, kend, c.kchunk);
        }
        else {
            dim3 grid4((g.nx + 4 * kVkBX - 1) / (4 * kVkBX), grid.y, grid.z);
            k_vk_interior_f4<<<grid4, block, 0, c.stream>>>((const float*)c.src, (float*)c.dst,
                                                            (const float*)c.kap, (const float*)c.fdt, g,
                                                            (float)bx, (float)by, (float)bz, kbeg, kend,
                                                            c.kchunk);
        }
        HS_CHECK_LAUNCH("heat variable-kappa interior kernel");
    } else {
        dim3 grid((g.nx + kVkBX - 1) / kVkBX, (g.ny + kVkBY - 1) / kVkBY, g.nz >= 2 ? 2 : 1);
        if constexpr (kFaces) {
            if (c.fx) {
                auto kern = (bx == by && by == bz) ? k_vk_boundary_xs<true> : k_vk_boundary_xs<false>;
                kern<<<grid, block, 0, c.stream>>>((const double*)c.src, (double*)c.dst, (const double*)c.kap,
                                                   (const double*)c.fdt, g, bx, by, bz, c.fx, c.m3);
            }
            else
                k_vk_boundary_faces<<<grid, block, 0, c.stream>>>((const double*)c.src, (double*)c.dst,
                                                                  (const double*)c.kap, (const double*)c.fdt, g,
                                                                  bx, by, bz);
        }
        else
            k_vk_boundary<T><<<grid, block, 0, c.stream>>>((const T*)c.src, (T*)c.dst, (const T*)c.kap,
                                                           (const T*)c.fdt, g, bx, by, bz);
        HS_CHECK_LAUNCH("heat variable-kappa boundary kernel");
    }
    return HS_OK;
}

int vk_launch(const VkCall& c) { return c.f64 ? vk_launch_t<double>(c) : vk_launch_t<float>(c); }

}  // namespace hcg
