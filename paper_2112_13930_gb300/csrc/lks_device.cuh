// lks_device.cuh -- device-side building blocks of the fused LKS-MHD step.
//
// Everything here works on deviations from the rest equilibrium
//   f_rest_a = f^eq_a(rho = 1, u = 0, B = (0, B0)),  g_rest_xa = 0,  g_rest_ya = W_a B0,
// so that FP32 and 16-bit storage keep the small signal (u ~ 1e-2, B_x ~ 1e-2 B0 scales)
// instead of the O(1) rest populations.  With d = f - f_rest:
//   rho - 1 = sum d, rho u = sum d e (+ F/2), B_x = sum dg_x, B_y - B0 = sum dg_y,
// because the rest populations have unit mass, no first moment and sum_a W_a = 1.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lks {

// Coefficients of one wall's closure, precomputed on the host in FP64.
//   link   : g_in,x = r * g_out,x(opposite, own node) + kx      (Eq. movingwalllinkbasedclosure)
//            f_in   = f_out(opposite, own node) +/- du          (Ladd's moving bounce-back, App. B.1)
//   moment : g_unknown,x = r * g_opposite,x - bc * (g0x + g1x + g3x) + kx
//            (Eq. momentconstraintgx / momentbasedclosureformovingwall times c a, beta = c a/(tau_m c^2),
//             r = (beta-1)/(beta+1), bc = 1/(beta+1), kx = -/+ beta/(beta+1) B0 U)
//            f: moment closure of App. A / App. B.2 with wall speed U.
template <typename C>
struct WallCoef {
    C r, bc, kx, du, U;
};

template <typename C>
struct StepParams {
    int32_t nx, ny;
    int64_t N;            // nx * ny
    C omega_f;            // 1 / tau_f
    C omega_m;            // 1 / tau_m
    C src_coef;           // 1 - 1/(2 tau_f)
    C Fx;                 // body force along x
    C B0;                 // applied field along y
    // products of the above folded on the host, so the collision needs fewer operations:
    C om1f, om1m;         // 1 - omega_f, 1 - omega_m
    C owf0, owf1, owf5;   // omega_f * w_a for |e_a|^2 = 0, 1, 2
    C owm0, owm1;         // omega_m * W_a for a = 0 and a = 1..4
    C sw0, sw1, sw5;      // (1 - 1/(2 tau_f)) * 3 Fx * w_a   (source-term prefactor)
    WallCoef<C> bot, top;
};

// Storage conversions (round to nearest even on the way down).  RO = true loads through the
// read-only (non-coherent) path, valid only when the buffer is not written during the kernel;
// RO = false is a plain coherent load for kernels that write and re-read buffers across steps.
template <typename S, typename C, bool RO = true> struct Loader;
template <bool RO> struct Loader<double, double, RO> {
    static __device__ __forceinline__ double ld(const double* p) { return RO ? __ldg(p) : *p; }
};
template <bool RO> struct Loader<float, float, RO> {
    static __device__ __forceinline__ float ld(const float* p) { return RO ? __ldg(p) : *p; }
};
template <bool RO> struct Loader<__nv_bfloat16, float, RO> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(RO ? __ldg(p) : *p); }
};
template <bool RO> struct Loader<__half, float, RO> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(RO ? __ldg(p) : *p); }
};
template <typename S, typename C> __device__ __forceinline__ C load_s(const S* p) { return Loader<S, C, true>::ld(p); }

template <typename S, typename C> __device__ __forceinline__ void store_s(S* p, C v);
template <> __device__ __forceinline__ void store_s<double, double>(double* p, double v) { *p = v; }
template <> __device__ __forceinline__ void store_s<float, float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void store_s<__nv_bfloat16, float>(__nv_bfloat16* p, float v) {
    *p = __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ void store_s<__half, float>(__half* p, float v) { *p = __float2half_rn(v); }

// 1/rho.  FP64: Newton-Raphson iteration for the reciprocal, r <- r + r (1 - rho r), started from
// the correctly rounded FP32 reciprocal (relative error <= 2^-24); two iterations square the error
// twice (<= 2^-96 before rounding), far below FP64's resolution.  FP32: the correctly rounded
// reciprocal.
__device__ __forceinline__ double recip(double rho) {
    double r = (double)__frcp_rn((float)rho);
    r = fma(r, fma(-rho, r, 1.0), r);
    r = fma(r, fma(-rho, r, 1.0), r);
    return r;
}
__device__ __forceinline__ float recip(float rho) { return __frcp_rn(rho); }

// Equilibrium deviations and the collision, for one node whose post-stream, post-closure
// populations are in f[9], gx[5], gy[5] (deviation form).  Overwrites them with the
// post-collision deviations.  Returns nothing; moments are recomputed by callers that need them.
//
// f^eq (Sec. V) with Dellar's Maxwell stress:
//   f^eq_a = w_a [rho + 3 rho e.u + 4.5 rho (e.u)^2 - 1.5 rho u^2]
//          + 4.5 w_a [ |B|^2 |e_a|^2 / 2 - (e_a . B)^2 ]
// source (Sec. V): S_a = 3 (e_a - u) . F  f^eq,hyd_a / rho
// g^eq (Eq. geqmagneticfield): g^eq_ax = W_a (B_x - 3 e_ay E), g^eq_ay = W_a (B_y + 3 e_ax E),
//   E = u_x B_y - u_y B_x.
template <typename C>
__device__ __forceinline__ void collide_node(C f[9], C gx[5], C gy[5], const StepParams<C>& p) {
    const C half = C(0.5), three = C(3), four5 = C(4.5), one5 = C(1.5);

    // a3: moments
    const C drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const C rho = C(1) + drho;
    const C jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const C jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const C inv_rho = recip(rho);
    const C ux = (jx + half * p.Fx) * inv_rho;
    const C uy = jy * inv_rho;
    const C bx = ((gx[0] + gx[1]) + (gx[2] + gx[3])) + gx[4];
    const C dby = ((gy[0] + gy[1]) + (gy[2] + gy[3])) + gy[4];
    const C by = p.B0 + dby;

    // a4-a5 for f.  Post-collision deviation:
    //   f' = (1 - w) f + w f^eq,dev + (1 - 1/(2 tau)) S
    //   f^eq,dev_a = w_a (drho + rho bm1_a) + M_a,  bm1_a = 3 eu + 4.5 eu^2 - 1.5 u^2
    //   S_a = 3 (e_ax - u_x) F_x w_a (1 + bm1_a)
    // Maxwell-stress part M_a with q = B_y^2 - B0^2 = dby (2 B0 + dby):
    //   a=1,3: 2.25 w1 (q - Bx^2)   a=2,4: -2.25 w1 (q - Bx^2)   a=5,7: -9 w5 Bx By   a=6,8: +9 w5 Bx By
    const C q = dby * (p.B0 + by);
    const C om13 = p.owf1 * (C(2.25) * (q - bx * bx));   // omega * M_1 = omega * M_3 = -omega * M_2
    const C omxy = p.owf5 * (C(9) * bx * by);            // omega * M_6 = omega * M_8 = -omega * M_5
    const C usq = one5 * (ux * ux + uy * uy);
    const C s0 = p.sw0 * (-ux);                            // source prefactors per e_x and weight
    const C s1p = p.sw1 * (C(1) - ux), s1z = p.sw1 * (-ux), s1m = p.sw1 * (C(-1) - ux);
    const C s5p = p.sw5 * (C(1) - ux), s5m = p.sw5 * (C(-1) - ux);
    const C om1 = p.om1f;
#define LKS_DIR(A, EU, OW, OMAG, SA)                                                    \
    {                                                                                   \
        const C eu = (EU);                                                              \
        const C bm1 = (three + four5 * eu) * eu - usq;                                  \
        const C ofeq = (OW) * (drho + rho * bm1) + (OMAG);                              \
        const C src = (SA) + (SA) * bm1;                                                \
        f[A] = om1 * f[A] + (ofeq + src);                                               \
    }
    LKS_DIR(0, C(0), p.owf0, C(0), s0)
    LKS_DIR(1, ux, p.owf1, om13, s1p)
    LKS_DIR(2, uy, p.owf1, -om13, s1z)
    LKS_DIR(3, -ux, p.owf1, om13, s1m)
    LKS_DIR(4, -uy, p.owf1, -om13, s1z)
    LKS_DIR(5, ux + uy, p.owf5, -omxy, s5p)
    LKS_DIR(6, uy - ux, p.owf5, omxy, s5m)
    LKS_DIR(7, -ux - uy, p.owf5, -omxy, s5m)
    LKS_DIR(8, ux - uy, p.owf5, omxy, s5p)
#undef LKS_DIR

    // a4-a5 for g (Eqs. geqmagneticfield, LKSformagneticfield): g' = (1 - w_m) g + w_m g^eq,dev with
    //   g^eq_x = W (Bx - 3 e_y E),  g^eq,dev_y = W (dBy + 3 e_x E),  E = u_x B_y - u_y B_x.
    const C om1m = p.om1m;
    const C ce = p.owm1 * (three * (ux * by - uy * bx));
    const C cb0 = p.owm0 * bx, cb1 = p.owm1 * bx;
    const C cd0 = p.owm0 * dby, cd1 = p.owm1 * dby;
    gx[0] = om1m * gx[0] + cb0;
    gx[1] = om1m * gx[1] + cb1;
    gx[2] = om1m * gx[2] + (cb1 - ce);
    gx[3] = om1m * gx[3] + cb1;
    gx[4] = om1m * gx[4] + (cb1 + ce);
    gy[0] = om1m * gy[0] + cd0;
    gy[1] = om1m * gy[1] + (cd1 + ce);
    gy[2] = om1m * gy[2] + cd1;
    gy[3] = om1m * gy[3] + (cd1 - ce);
    gy[4] = om1m * gy[4] + cd1;
}

// Moment-based closures at a wet wall node (Sec. VII, App. A, App. B.2), deviation form.
// g first (its B_x enters the Pi_20 target of f), then f.  Bottom: unknown f2, f5, f6, g2.
template <typename C>
__device__ __forceinline__ void moment_closure_bottom(C f[9], C gx[5], C gy[5], const WallCoef<C>& w, C B0) {
    const C half = C(0.5), cs2 = C(1.0 / 3.0);
    gx[2] = w.r * gx[4] - w.bc * ((gx[0] + gx[1]) + gx[3]) + w.kx;
    gy[2] = -(((gy[0] + gy[1]) + gy[3]) + gy[4]);
    const C bx = ((gx[0] + gx[1]) + (gx[2] + gx[3])) + gx[4];
    const C dby = ((gy[0] + gy[1]) + (gy[2] + gy[3])) + gy[4];
    const C drho = (f[0] + f[1]) + f[3] + C(2) * ((f[4] + f[7]) + f[8]);
    const C rho = C(1) + drho;
    const C U = w.U;
    // P - P_rest with P = rho (c^2 + U^2) + (B_y^2 - B_x^2)/2 and P_rest = c^2 + B0^2/2
    const C dP = U * U + drho * (cs2 + U * U) + dby * (B0 + half * dby) - half * bx * bx;
    const C rU = rho * U;
    f[2] = -dP + (f[1] + f[3]) + f[4] + C(2) * (f[7] + f[8]);
    f[5] = half * (dP + rU) - (f[1] + f[8]);
    f[6] = half * (dP - rU) - (f[3] + f[7]);
}

// Top: unknown f4, f7, f8, g4.
template <typename C>
__device__ __forceinline__ void moment_closure_top(C f[9], C gx[5], C gy[5], const WallCoef<C>& w, C B0) {
    const C half = C(0.5), cs2 = C(1.0 / 3.0);
    gx[4] = w.r * gx[2] - w.bc * ((gx[0] + gx[1]) + gx[3]) + w.kx;
    gy[4] = -(((gy[0] + gy[1]) + gy[2]) + gy[3]);
    const C bx = ((gx[0] + gx[1]) + (gx[2] + gx[3])) + gx[4];
    const C dby = ((gy[0] + gy[1]) + (gy[2] + gy[3])) + gy[4];
    const C drho = (f[0] + f[1]) + f[3] + C(2) * ((f[2] + f[5]) + f[6]);
    const C rho = C(1) + drho;
    const C U = w.U;
    const C dP = U * U + drho * (cs2 + U * U) + dby * (B0 + half * dby) - half * bx * bx;
    const C rU = rho * U;
    f[4] = -dP + (f[1] + f[2]) + f[3] + C(2) * (f[5] + f[6]);
    f[7] = half * (dP - rU) - (f[3] + f[6]);
    f[8] = half * (dP + rU) - (f[1] + f[5]);
}

// One node of the fused step (hot-path steps a1-a6): pull-stream from (fin, gin), wall closure,
// moments, equilibria, collision, store to (fout, gout).  n = y*nx + x of a lattice laid out as
// f[a][y][x], g[k][a][y][x].  Every element of fin/gin is read by exactly one node per step:
// interior rows pull from rows y-1 / y / y+1 (Eqs. LBMforflowfield, LKSformagneticfield);
// link-based wall rows take the unknown incoming populations from the same node's outgoing ones
// (Sec. VI, App. B.1), which nobody else reads; moment-based wall rows reconstruct them from the
// pulled ones (Sec. VII, App. A, App. B.2).
template <typename S, typename C, int CLOSURE, typename L>
__device__ __forceinline__ void step_node_with(const S* fin, const S* gin, S* fout, S* gout, const StepParams<C>& p,
                                               int64_t n) {
    const int nx = p.nx;
    const int j = (int)(n / nx);
    const int i = (int)(n - (int64_t)j * nx);
    const int64_t N = p.N;
    const int64_t rc = n - i;    // start of row j
    const int64_t rs = rc - nx;  // row j-1
    const int64_t rn = rc + nx;  // row j+1
    const int im = (i == 0) ? nx - 1 : i - 1;
    const int ip = (i == nx - 1) ? 0 : i + 1;
    const bool bottom = (j == 0);
    const bool top = (j == p.ny - 1);

    C f[9], gx[5], gy[5];
    const S* gxin = gin;
    const S* gyin = gin + 5 * N;
    // a1: pull-stream, periodic in x
    f[0] = L::ld(fin + 0 * N + rc + i);
    f[1] = L::ld(fin + 1 * N + rc + im);
    f[3] = L::ld(fin + 3 * N + rc + ip);
    gx[0] = L::ld(gxin + 0 * N + rc + i);
    gx[1] = L::ld(gxin + 1 * N + rc + im);
    gx[3] = L::ld(gxin + 3 * N + rc + ip);
    gy[0] = L::ld(gyin + 0 * N + rc + i);
    gy[1] = L::ld(gyin + 1 * N + rc + im);
    gy[3] = L::ld(gyin + 3 * N + rc + ip);
    if (!bottom) {
        f[2] = L::ld(fin + 2 * N + rs + i);
        f[5] = L::ld(fin + 5 * N + rs + im);
        f[6] = L::ld(fin + 6 * N + rs + ip);
        gx[2] = L::ld(gxin + 2 * N + rs + i);
        gy[2] = L::ld(gyin + 2 * N + rs + i);
    }
    if (!top) {
        f[4] = L::ld(fin + 4 * N + rn + i);
        f[7] = L::ld(fin + 7 * N + rn + ip);
        f[8] = L::ld(fin + 8 * N + rn + im);
        gx[4] = L::ld(gxin + 4 * N + rn + i);
        gy[4] = L::ld(gyin + 4 * N + rn + i);
    }
    // a2: wall closures
    if (CLOSURE == 0) {
        if (bottom) {
            const WallCoef<C>& w = p.bot;
            f[2] = L::ld(fin + 4 * N + rc + i);
            f[5] = L::ld(fin + 7 * N + rc + i) + w.du;
            f[6] = L::ld(fin + 8 * N + rc + i) - w.du;
            gx[2] = w.r * L::ld(gxin + 4 * N + rc + i) + w.kx;
            gy[2] = -L::ld(gyin + 4 * N + rc + i);
        }
        if (top) {
            const WallCoef<C>& w = p.top;
            f[4] = L::ld(fin + 2 * N + rc + i);
            f[7] = L::ld(fin + 5 * N + rc + i) - w.du;
            f[8] = L::ld(fin + 6 * N + rc + i) + w.du;
            gx[4] = w.r * L::ld(gxin + 2 * N + rc + i) + w.kx;
            gy[4] = -L::ld(gyin + 2 * N + rc + i);
        }
    } else {
        if (bottom) moment_closure_bottom<C>(f, gx, gy, p.bot, p.B0);
        if (top) moment_closure_top<C>(f, gx, gy, p.top, p.B0);
    }
    // a3-a5
    collide_node<C>(f, gx, gy, p);
    // a6: store
    S* gxo = gout;
    S* gyo = gout + 5 * N;
#pragma unroll
    for (int a = 0; a < 9; ++a) store_s<S, C>(fout + a * N + n, f[a]);
#pragma unroll
    for (int a = 0; a < 5; ++a) store_s<S, C>(gxo + a * N + n, gx[a]);
#pragma unroll
    for (int a = 0; a < 5; ++a) store_s<S, C>(gyo + a * N + n, gy[a]);
}

// step_node with the read-only loads (RO) or plain coherent loads.
template <typename S, typename C, int CLOSURE, bool RO>
__device__ __forceinline__ void step_node(const S* fin, const S* gin, S* fout, S* gout, const StepParams<C>& p,
                                          int64_t n) {
    step_node_with<S, C, CLOSURE, Loader<S, C, RO>>(fin, gin, fout, gout, p, n);
}

}  // namespace lks
