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

#include <type_traits>

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
    C src3;               // 3 (1 - 1/(2 tau_f))   (source prefactor when the force varies per node)
    int32_t coupling;     // 0: Maxwell stress in f^eq; 1: Lorentz force J x B in the source
    WallCoef<C> bot, top;
};

// FP16 storage holds each deviation times kHalfScale = 2^14.  The deviations of these flows span
// roughly 1e-9 .. 1e-1 (the induced field of a weakly perturbed channel sits at W B_x ~ 1e-7);
// unscaled, everything below 2^-14 = 6.1e-5 would fall into FP16's subnormals and lose its relative
// precision.  Scaled, values down to 2^-28 = 3.7e-9 keep the full 11-bit significand, and because the
// scale is a power of two the multiplications are exact: the only rounding is the store's, as before.
// |deviation| >= 4 overflows to inf, which the residual reports as non-finite (the populations of a
// stable run deviate from the rest state by well under 1).  BF16 keeps FP32's exponent range and is
// stored unscaled.
constexpr float kHalfScale = 16384.0f;
constexpr float kHalfUnscale = 1.0f / 16384.0f;

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
    static __device__ __forceinline__ float ld(const __half* p) {
        return __fmul_rn(__half2float(RO ? __ldg(p) : *p), kHalfUnscale);
    }
};
template <typename S, typename C> __device__ __forceinline__ C load_s(const S* p) { return Loader<S, C, true>::ld(p); }

template <typename S, typename C> __device__ __forceinline__ void store_s(S* p, C v);
template <> __device__ __forceinline__ void store_s<double, double>(double* p, double v) { *p = v; }
template <> __device__ __forceinline__ void store_s<float, float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void store_s<__nv_bfloat16, float>(__nv_bfloat16* p, float v) {
    *p = __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ void store_s<__half, float>(__half* p, float v) {
    *p = __float2half_rn(__fmul_rn(v, kHalfScale));
}

// Pinned floating-point operations.  Every product in the collision and the closures is written
// as an explicit fused multiply-add (ffma) or a separately rounded multiply (fmul); no plain '*'
// on floating-point values remains, so the compiler has nothing to contract and every kernel that
// inlines this code (one- and two-node, in-place, batched, cluster) performs exactly the same
// operations in the same order -- their results agree bit for bit.
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double ffma(double a, double b, double c) { return __fma_rn(a, b, c); }

// 1/rho.  FP64: Newton-Raphson iteration for the reciprocal, r <- r + r (1 - rho r), started from
// the correctly rounded FP32 reciprocal (relative error <= 2^-24); two iterations square the error
// twice (<= 2^-96 before rounding), far below FP64's resolution.  FP32: the correctly rounded
// reciprocal.
__device__ __forceinline__ double recip(double rho) {
    double r = (double)__frcp_rn((float)rho);
    r = ffma(r, ffma(-rho, r, 1.0), r);
    r = ffma(r, ffma(-rho, r, 1.0), r);
    return r;
}
__device__ __forceinline__ float recip(float rho) { return __frcp_rn(rho); }

// Two nodes at once: float2 values with the packed FP32 instructions of sm_100 and later (add, mul,
// fma on .f32x2), each half rounded exactly as the scalar float operation above, so the collision
// code below, written once, gives a node the same bits alone (float) or in a pair (float2).  A
// float operand is used in both halves.  These take part only when an operand is a float2.
__device__ __forceinline__ float2 pair_of(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pair_of(float2 a) { return a; }
template <typename... T>
struct HasPair : std::false_type {};
template <typename T0, typename... T>
struct HasPair<T0, T...>
    : std::integral_constant<bool, std::is_same<T0, float2>::value || HasPair<T...>::value> {};
template <typename... T>
using IfPair = typename std::enable_if<HasPair<T...>::value, int>::type;

template <typename A, typename B, IfPair<A, B> = 0>
__device__ __forceinline__ float2 fmul(A a, B b) { return __fmul2_rn(pair_of(a), pair_of(b)); }
template <typename A, typename B, typename D, IfPair<A, B, D> = 0>
__device__ __forceinline__ float2 ffma(A a, B b, D c) { return __ffma2_rn(pair_of(a), pair_of(b), pair_of(c)); }
template <typename A, typename B, IfPair<A, B> = 0>
__device__ __forceinline__ float2 operator+(A a, B b) { return __fadd2_rn(pair_of(a), pair_of(b)); }
// a - b as b * (-1) + a: the product is exact, so the one rounding is that of a - b
template <typename A, typename B, IfPair<A, B> = 0>
__device__ __forceinline__ float2 operator-(A a, B b) {
    return __ffma2_rn(pair_of(b), make_float2(-1.0f, -1.0f), pair_of(a));
}
__device__ __forceinline__ float2 operator-(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 operator/(float2 a, float2 b) { return make_float2(a.x / b.x, a.y / b.y); }
__device__ __forceinline__ float2 recip(float2 rho) { return make_float2(recip(rho.x), recip(rho.y)); }
// zero of a node value type
template <typename V> __device__ __forceinline__ V zero_of() { return V(0); }
template <> __device__ __forceinline__ float2 zero_of<float2>() { return make_float2(0.0f, 0.0f); }

// Equilibrium and collision of g (Eqs. geqmagneticfield, LKSformagneticfield): g' = (1 - w_m) g + w_m g^eq,dev with
//   g^eq_x = W (Bx - 3 e_y E),  g^eq,dev_y = W (dBy + 3 e_x E),  E = u_x B_y - u_y B_x.
template <typename C, typename V>
__device__ __forceinline__ void collide_g(V gx[5], V gy[5], V ux, V uy, V bx, V by, V dby, const StepParams<C>& p) {
    const auto om1m = p.om1m;
    const auto ce = fmul(p.owm1, fmul(C(3), ffma(ux, by, -fmul(uy, bx))));
    const auto cb0 = fmul(p.owm0, bx), cb1 = fmul(p.owm1, bx);
    const auto cd0 = fmul(p.owm0, dby), cd1 = fmul(p.owm1, dby);
    gx[0] = ffma(om1m, gx[0], cb0);
    gx[1] = ffma(om1m, gx[1], cb1);
    gx[2] = ffma(om1m, gx[2], cb1 - ce);
    gx[3] = ffma(om1m, gx[3], cb1);
    gx[4] = ffma(om1m, gx[4], cb1 + ce);
    gy[0] = ffma(om1m, gy[0], cd0);
    gy[1] = ffma(om1m, gy[1], cd1 + ce);
    gy[2] = ffma(om1m, gy[2], cd1);
    gy[3] = ffma(om1m, gy[3], cd1 - ce);
    gy[4] = ffma(om1m, gy[4], cd1);
}

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
template <typename C, typename V>
__device__ __forceinline__ void collide_node(V f[9], V gx[5], V gy[5], const StepParams<C>& p) {
    const auto half = C(0.5), three = C(3), four5 = C(4.5), one5 = C(1.5);

    // moments
    const auto drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const auto rho = C(1) + drho;
    const auto jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const auto jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const auto inv_rho = recip(rho);
    const auto ux = fmul(ffma(half, p.Fx, jx), inv_rho);
    const auto uy = fmul(jy, inv_rho);
    const auto bx = ((gx[0] + gx[1]) + (gx[2] + gx[3])) + gx[4];
    const auto dby = ((gy[0] + gy[1]) + (gy[2] + gy[3])) + gy[4];
    const auto by = p.B0 + dby;

    // equilibrium, source and collision of f.  Post-collision deviation:
    //   f' = (1 - w) f + w f^eq,dev + (1 - 1/(2 tau)) S
    //   f^eq,dev_a = w_a (drho + rho bm1_a) + M_a,  bm1_a = 3 eu + 4.5 eu^2 - 1.5 u^2
    //   S_a = 3 (e_ax - u_x) F_x w_a (1 + bm1_a)
    // Maxwell-stress part M_a with q = B_y^2 - B0^2 = dby (2 B0 + dby):
    //   a=1,3: 2.25 w1 (q - Bx^2)   a=2,4: -2.25 w1 (q - Bx^2)   a=5,7: -9 w5 Bx By   a=6,8: +9 w5 Bx By
    const auto q = fmul(dby, p.B0 + by);
    const auto om13 = fmul(p.owf1, fmul(C(2.25), ffma(-bx, bx, q)));   // omega * M_1 = omega * M_3 = -omega * M_2
    const auto omxy = fmul(p.owf5, fmul(fmul(C(9), bx), by));         // omega * M_6 = omega * M_8 = -omega * M_5
    const auto usq = fmul(one5, ffma(ux, ux, fmul(uy, uy)));
    const auto s0 = fmul(p.sw0, -ux);                                  // source prefactors per e_x and weight
    const auto s1p = fmul(p.sw1, C(1) - ux), s1z = fmul(p.sw1, -ux), s1m = fmul(p.sw1, C(-1) - ux);
    const auto s5p = fmul(p.sw5, C(1) - ux), s5m = fmul(p.sw5, C(-1) - ux);
    const auto om1 = p.om1f;
#define LKS_DIR(A, EU, OW, OMAG, SA)                                                    \
    {                                                                                   \
        const auto eu = (EU);                                                              \
        const auto bm1 = ffma(ffma(four5, eu, three), eu, -usq);                           \
        const auto ofeq = ffma((OW), ffma(rho, bm1, drho), (OMAG));                        \
        const auto src = ffma((SA), bm1, (SA));                                            \
        f[A] = ffma(om1, f[A], ofeq + src);                                             \
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
    collide_g(gx, gy, ux, uy, bx, by, dby, p);
}

// Moment-based closures at a wet wall node (Sec. VII, App. A, App. B.2), deviation form.
// g first (its moments enter the f closure), then f.  Bottom: unknown f2, f5, f6, g2.
//   COUPLING 0 (Maxwell stress in f^eq): Pi_10 = rho U, Pi_01 = 0,
//              Pi_20 = rho (c^2 + U^2) + (B_y^2 - B_x^2)/2 (the full equilibrium value).
//   COUPLING 1 (Lorentz force in the source): the node's velocity (Pi + F/2)/rho is (U, 0):
//              Pi_10 = rho U - F_x/2, Pi_01 = -F_y/2 with F = F_ext + J x B, J_z from the closed g
//              at u = (U, 0) (J_z = 3 omega_m (Lambda_yx - Lambda_xy + 2 U B_y)); Pi_20 = rho (c^2 + U^2).
// In both, the rest state satisfies the closure exactly, so the deviations need no constant terms.
template <typename C, int COUPLING, typename V>
__device__ __forceinline__ void wall_force_halves(const V gx[5], const V gy[5], V bx, V by, C U,
                                                  const StepParams<C>& p, V& hfx, V& hfy) {
    if (COUPLING == 1) {
        const auto jz = fmul(fmul(C(3), p.omega_m), ffma(fmul(C(2), U), by, (gx[2] - gx[4]) - (gy[1] - gy[3])));
        hfx = fmul(C(0.5), ffma(-jz, by, p.Fx));
        hfy = fmul(C(0.5), fmul(jz, bx));
    } else {
        hfx = zero_of<V>();
        hfy = zero_of<V>();
    }
}

template <typename C, int COUPLING, typename V>
__device__ __forceinline__ void moment_closure_bottom(V f[9], V gx[5], V gy[5], const WallCoef<C>& w,
                                                      const StepParams<C>& p) {
    const auto half = C(0.5), cs2 = C(1.0 / 3.0);
    const auto B0 = p.B0;
    gx[2] = ffma(w.r, gx[4], -fmul(w.bc, (gx[0] + gx[1]) + gx[3])) + w.kx;
    gy[2] = -(((gy[0] + gy[1]) + gy[3]) + gy[4]);
    const auto bx = ((gx[0] + gx[1]) + (gx[2] + gx[3])) + gx[4];
    const auto dby = ((gy[0] + gy[1]) + (gy[2] + gy[3])) + gy[4];
    const auto U = w.U;
    V hfx, hfy;
    wall_force_halves<C, COUPLING>(gx, gy, bx, B0 + dby, U, p, hfx, hfy);
    // With the Maxwell coupling the force halves are zero and left out (a constant zero in an fma
    // lets the compiler turn it into a product it may fuse with the next sum, and the one- and
    // two-node forms would then round differently).
    V drho = ffma(C(2), (f[4] + f[7]) + f[8], (f[0] + f[1]) + f[3]);
    if constexpr (COUPLING == 1) drho = drho - hfy;
    const auto rho = C(1) + drho;
    // P - P_rest
    const auto uu = fmul(U, U);
    auto dP = ffma(drho, cs2 + uu, uu);
    if (COUPLING == 0) dP = dP + ffma(-fmul(half, bx), bx, fmul(dby, ffma(half, dby, B0)));
    V rU;
    if constexpr (COUPLING == 1) rU = ffma(rho, U, -hfx);
    else rU = fmul(rho, U);
    f[2] = ((-dP + (f[1] + f[3])) + f[4]) + fmul(C(2), f[7] + f[8]);
    if constexpr (COUPLING == 1) f[2] = f[2] - hfy;
    f[5] = ffma(half, dP + rU, -(f[1] + f[8]));
    f[6] = ffma(half, dP - rU, -(f[3] + f[7]));
}

// Top: unknown f4, f7, f8, g4.
template <typename C, int COUPLING, typename V>
__device__ __forceinline__ void moment_closure_top(V f[9], V gx[5], V gy[5], const WallCoef<C>& w,
                                                   const StepParams<C>& p) {
    const auto half = C(0.5), cs2 = C(1.0 / 3.0);
    const auto B0 = p.B0;
    gx[4] = ffma(w.r, gx[2], -fmul(w.bc, (gx[0] + gx[1]) + gx[3])) + w.kx;
    gy[4] = -(((gy[0] + gy[1]) + gy[2]) + gy[3]);
    const auto bx = ((gx[0] + gx[1]) + (gx[2] + gx[3])) + gx[4];
    const auto dby = ((gy[0] + gy[1]) + (gy[2] + gy[3])) + gy[4];
    const auto U = w.U;
    V hfx, hfy;
    wall_force_halves<C, COUPLING>(gx, gy, bx, B0 + dby, U, p, hfx, hfy);
    V drho = ffma(C(2), (f[2] + f[5]) + f[6], (f[0] + f[1]) + f[3]);
    if constexpr (COUPLING == 1) drho = drho + hfy;
    const auto rho = C(1) + drho;
    const auto uu = fmul(U, U);
    auto dP = ffma(drho, cs2 + uu, uu);
    if (COUPLING == 0) dP = dP + ffma(-fmul(half, bx), bx, fmul(dby, ffma(half, dby, B0)));
    V rU;
    if constexpr (COUPLING == 1) rU = ffma(rho, U, -hfx);
    else rU = fmul(rho, U);
    f[4] = ((-dP + (f[1] + f[2])) + f[3]) + fmul(C(2), f[5] + f[6]);
    if constexpr (COUPLING == 1) f[4] = f[4] + hfy;
    f[7] = ffma(half, dP - rU, -(f[3] + f[6]));
    f[8] = ffma(half, dP + rU, -(f[1] + f[5]));
}

// Collision with the paper's own coupling (Sec. IV-V): f^eq without magnetic terms; the Lorentz
// force F_L = J x B, J_z = (Lambda^(1)_yx - Lambda^(1)_xy)/(tau_m c_sm^2), enters the source and the
// half shift of rho u.  Lambda^(1) = Lambda - Lambda^(0)(u) and u = (j + F/2)/rho depend on each
// other linearly; with k = 3 omega_m and D = Lambda_yx - Lambda_xy the exact solution is
//   J_z = k [D + 2 (B_y (j_x + F_ext/2) - B_x j_y)/rho] / (1 + k |B|^2 / rho).
template <typename C, typename V>
__device__ __forceinline__ void collide_node_lorentz(V f[9], V gx[5], V gy[5], const StepParams<C>& p) {
    const auto half = C(0.5), three = C(3), four5 = C(4.5), one5 = C(1.5);
    const auto drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const auto rho = C(1) + drho;
    const auto jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const auto jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const auto inv_rho = recip(rho);
    const auto bx = ((gx[0] + gx[1]) + (gx[2] + gx[3])) + gx[4];
    const auto dby = ((gy[0] + gy[1]) + (gy[2] + gy[3])) + gy[4];
    const auto by = p.B0 + dby;
    const auto k = fmul(three, p.omega_m);
    const auto D = (gx[2] - gx[4]) - (gy[1] - gy[3]);
    const auto jxp = ffma(half, p.Fx, jx);
    const auto num = fmul(k, ffma(fmul(C(2), inv_rho), ffma(by, jxp, -fmul(bx, jy)), D));
    const auto den = ffma(fmul(k, inv_rho), ffma(bx, bx, fmul(by, by)), C(1));
    const auto jz = num / den;
    const auto Fx = ffma(-jz, by, p.Fx), Fy = fmul(jz, bx);
    const auto ux = fmul(ffma(half, Fx, jx), inv_rho);
    const auto uy = fmul(ffma(half, Fy, jy), inv_rho);
    const auto usq = fmul(one5, ffma(ux, ux, fmul(uy, uy)));
    const auto ax = fmul(p.src3, Fx), ay = fmul(p.src3, Fy);
    // (e_x - u_x) a_x and (e_y - u_y) a_y for e = -1, 0, +1
    const auto px0 = fmul(-ux, ax), pxp = fmul(C(1) - ux, ax), pxm = fmul(C(-1) - ux, ax);
    const auto py0 = fmul(-uy, ay), pyp = fmul(C(1) - uy, ay), pym = fmul(C(-1) - uy, ay);
    const auto w0 = C(4.0 / 9.0), w1 = C(1.0 / 9.0), w5 = C(1.0 / 36.0);
    const auto om1 = p.om1f;
#define LKS_DIRL(A, EU, OW, W, PX, PY)                                                  \
    {                                                                                   \
        const auto eu = (EU);                                                              \
        const auto bm1 = ffma(ffma(four5, eu, three), eu, -usq);                           \
        const auto ofeq = fmul((OW), ffma(rho, bm1, drho));                                \
        const auto sa = fmul((W), (PX) + (PY));                                            \
        f[A] = ffma(om1, f[A], ofeq + ffma(sa, bm1, sa));                               \
    }
    LKS_DIRL(0, C(0), p.owf0, w0, px0, py0)
    LKS_DIRL(1, ux, p.owf1, w1, pxp, py0)
    LKS_DIRL(2, uy, p.owf1, w1, px0, pyp)
    LKS_DIRL(3, -ux, p.owf1, w1, pxm, py0)
    LKS_DIRL(4, -uy, p.owf1, w1, px0, pym)
    LKS_DIRL(5, ux + uy, p.owf5, w5, pxp, pyp)
    LKS_DIRL(6, uy - ux, p.owf5, w5, pxm, pyp)
    LKS_DIRL(7, -ux - uy, p.owf5, w5, pxm, pym)
    LKS_DIRL(8, ux - uy, p.owf5, w5, pxp, pym)
#undef LKS_DIRL
    collide_g(gx, gy, ux, uy, bx, by, dby, p);
}

template <typename C, int COUPLING, typename V>
__device__ __forceinline__ void collide(V f[9], V gx[5], V gy[5], const StepParams<C>& p) {
    if (COUPLING == 1)
        collide_node_lorentz<C>(f, gx, gy, p);
    else
        collide_node<C>(f, gx, gy, p);
}

// One node of the fused step: pull-stream from (fin, gin), wall closure,
// moments, equilibria, collision, store to (fout, gout).  n = y*nx + x of a lattice laid out as
// f[a][y][x], g[k][a][y][x].  Every element of fin/gin is read by exactly one node per step:
// interior rows pull from rows y-1 / y / y+1 (Eqs. LBMforflowfield, LKSformagneticfield);
// link-based wall rows take the unknown incoming populations from the same node's outgoing ones
// (Sec. VI, App. B.1), which nobody else reads; moment-based wall rows reconstruct them from the
// pulled ones (Sec. VII, App. A, App. B.2).
template <typename S, typename C, int CLOSURE, typename L, int COUPLING = 0>
__device__ __forceinline__ void step_node_with(const S* fin, const S* gin, S* fout, S* gout, const StepParams<C>& p,
                                               int64_t n, int i, int j) {
    const int nx = p.nx;
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
    // pull-stream, periodic in x
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
    // wall closures
    if (CLOSURE == 0) {
        if (bottom) {
            const WallCoef<C>& w = p.bot;
            f[2] = L::ld(fin + 4 * N + rc + i);
            f[5] = L::ld(fin + 7 * N + rc + i) + w.du;
            f[6] = L::ld(fin + 8 * N + rc + i) - w.du;
            gx[2] = ffma(w.r, L::ld(gxin + 4 * N + rc + i), w.kx);
            gy[2] = -L::ld(gyin + 4 * N + rc + i);
        }
        if (top) {
            const WallCoef<C>& w = p.top;
            f[4] = L::ld(fin + 2 * N + rc + i);
            f[7] = L::ld(fin + 5 * N + rc + i) - w.du;
            f[8] = L::ld(fin + 6 * N + rc + i) + w.du;
            gx[4] = ffma(w.r, L::ld(gxin + 2 * N + rc + i), w.kx);
            gy[4] = -L::ld(gyin + 2 * N + rc + i);
        }
    } else {
        if (bottom) moment_closure_bottom<C, COUPLING>(f, gx, gy, p.bot, p);
        if (top) moment_closure_top<C, COUPLING>(f, gx, gy, p.top, p);
    }
    // moments, equilibria, collision
    collide<C, COUPLING>(f, gx, gy, p);
    // store
    S* gxo = gout;
    S* gyo = gout + 5 * N;
#pragma unroll
    for (int a = 0; a < 9; ++a) store_s<S, C>(fout + a * N + n, f[a]);
#pragma unroll
    for (int a = 0; a < 5; ++a) store_s<S, C>(gxo + a * N + n, gx[a]);
#pragma unroll
    for (int a = 0; a < 5; ++a) store_s<S, C>(gyo + a * N + n, gy[a]);
}

// step_node with the read-only (RO) or plain coherent loads; (i, j) are n's column and row.
template <typename S, typename C, int CLOSURE, bool RO, int COUPLING = 0>
__device__ __forceinline__ void step_node(const S* fin, const S* gin, S* fout, S* gout, const StepParams<C>& p,
                                          int64_t n, int i, int j) {
    step_node_with<S, C, CLOSURE, Loader<S, C, RO>, COUPLING>(fin, gin, fout, gout, p, n, i, j);
}

// Fixed-order sum of K FP64 values over the 32 lanes of a warp: a shuffle tree with offsets 16, 8,
// 4, 2, 1, after which lane 0 holds the totals.  Every call combines the lanes in the same order, so
// the sums are bitwise reproducible.  All 32 lanes must take part.
template <int K>
__device__ __forceinline__ void warp_sum(double v[K]) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
}

// Fixed-order sum of K values per thread over a block of up to 1024 threads (a multiple of 32):
// each warp sums its lanes with warp_sum, lane 0 of every warp parks the warp's K sums in
// sh[k * 32 + warp], and thread 0 adds the warps' sums in warp order.  The totals end up in
// thread 0's v (the other threads' v hold partial sums).  sh holds 32 K doubles.  The order depends
// only on the thread index, so the result is bitwise reproducible.
template <int K>
__device__ __forceinline__ void block_sum(double v[K], double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    warp_sum<K>(v);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sh[k * 32 + warp] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = sh[k * 32];
            for (int w = 1; w < nw; ++w) t += sh[k * 32 + w];
            v[k] = t;
        }
    }
}

// Walks a thread's nodes n = first, first + stride, ... of an nx-wide lattice keeping (i, j) up
// to date with additions only (no per-node division).
struct NodeWalker {
    int64_t n;
    int i, j, di, dj, nx;
    __device__ __forceinline__ NodeWalker(int64_t first, int64_t stride, int nx_) : n(first), nx(nx_) {
        j = (int)(first / nx_);
        i = (int)(first - (int64_t)j * nx_);
        dj = (int)(stride / nx_);
        di = (int)(stride - (int64_t)dj * nx_);
    }
    __device__ __forceinline__ void next(int64_t stride) {
        n += stride;
        i += di;
        j += dj;
        if (i >= nx) {
            i -= nx;
            ++j;
        }
    }
};

}  // namespace lks
