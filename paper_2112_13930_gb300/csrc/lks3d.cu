// lks3d.cu -- the three-dimensional channel (include/lks3d.h): fused D3Q19 + 3 x D3Q7 collide-
// stream kernel with the link-based Shercliff walls, moments, residual, state conversion and the
// lks3_* C ABI.
//
// One thread per node, x fastest (grid: x blocks, y, z), pull scheme: every population of the
// source buffer is read by exactly one node per step, so a step moves 40 values in and 40 out per
// node (320 B in FP32).  Stored values are deviations from the rest equilibrium; the arithmetic
// below is the oracle's (absolute populations) rewritten for deviations:
//   d_a = f_a - f_rest_a,  f_rest_a = w_a + M_a(0, B0, 0),
//   rho = 1 + sum d,  rho u = sum d e + F/2,  B = (sum dg_x, B0 + sum dg_y, sum dg_z),
//   f'_a - f_rest_a = (1 - w) d_a + w [w_a (drho + rho bm1_a) + M_a(B) - M_a(B_rest)]
//                     + (1 - w/2) 3 (e_ax - u_x) F_x w_a (1 + bm1_a),
//   bm1_a = 3 e.u + 4.5 (e.u)^2 - 1.5 u^2,
//   M_a(B) - M_a(B_rest) = 4.5 w_a [ |e|^2 q / 2 - (e.B - e_y B0)(e.B + e_y B0) - q / 6 ],
//   q = |B|^2 - B0^2 = B_x^2 + B_z^2 + dB_y (2 B0 + dB_y),
//   g'_ai - g_rest_ai = (1 - w_m) dg_ai + w_m W_a (B_i - B_rest_i + 4 e_a.(u B_i - B u_i)).
// Rest populations of opposite directions are equal, so the bounce-back closures carry over to
// deviations unchanged, and the normal-component anti-bounce-back becomes dg_in = -dg_out.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <new>
#include <string>

#include "../../include/lks3d.h"
#include "lks_device.cuh"
#include "lks_bulk.cuh"
#include "lks_internal.h"
#include "lks_packed.cuh"
#include "lks_vec.cuh"

using lks::load_s;
using lks::store_s;

namespace {

thread_local std::string g3_last_error = "";
constexpr size_t kAlign3 = 256;
constexpr int kRedBlocks = 1024;  // residual partial sums (fixed, so the reduction order is fixed)

inline size_t align3(size_t x) { return (x + kAlign3 - 1) & ~(kAlign3 - 1); }

// D3Q19 velocity components (order of lks3d.h) as constant expressions, so that unrolled loops
// over the directions fold them; D3Q7 is the first seven directions.
__host__ __device__ constexpr int EXa(int a) {
    return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1 : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
}
__host__ __device__ constexpr int EYa(int a) {
    return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1 : (a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0;
}
__host__ __device__ constexpr int EZa(int a) {
    return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1 : (a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0;
}
__host__ __device__ inline double w19(int a) { return a == 0 ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
__host__ __device__ inline double w7(int a) { return a == 0 ? 0.25 : 0.125; }
__host__ __device__ constexpr int opp(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }

// Rest deviation offsets in FP64 (host side; passed to the conversion kernels).
double f_rest(int a, double B0) {
    const double e2 = EXa(a) * EXa(a) + EYa(a) * EYa(a) + EZa(a) * EZa(a);
    const double eB = EYa(a) * B0;
    return w19(a) + 4.5 * w19(a) * (0.5 * B0 * B0 * e2 - eB * eB - B0 * B0 / 6.0);
}

template <typename C>
struct Wall3 {
    C r, kx, du;  // tangential-component ratio, B_x moving-wall term, Ladd term for the diagonals
};

template <typename C>
struct Params3 {
    int32_t nx, ny, nz;
    int64_t N;
    C om_f, om1f, om_m, om1m;  // 1/tau_f, 1 - 1/tau_f, 1/tau_m, 1 - 1/tau_m
    C B0, Fx, hFx, twoB0;      // hFx = F/2, twoB0 = 2 B0
    C Ks[3];                   // (1 - 1/(2 tau_f)) 3 F w for |e|^2 = 0, 1, 2 (source term)
    C cB[3];                   // 4.5 w (-1) 2 B0 for |e|^2 = 0, 1, 2 (Maxwell stress, e_y = +1)
    C omW0, omW1, omW1x4;      // w_m W_0, w_m W, 4 w_m W (D3Q7)
    Wall3<C> bot, top;
    C rs_back, rs_front;       // duct: tangential-component ratios of the side walls z = -b, z = +b
};

template <typename C>
Params3<C> make_params3(const lks3_params& p, double c_bot, double c_top, double u_bot, double u_top,
                        double c_back = 0.0, double c_front = 0.0) {
    Params3<C> q;
    q.nx = p.nx;
    q.ny = p.ny;
    q.nz = p.nz;
    q.N = (int64_t)p.nx * p.ny * p.nz;
    q.om_f = (C)(1.0 / p.tau_f);
    q.om1f = (C)(1.0 - 1.0 / p.tau_f);
    q.om_m = (C)(1.0 / p.tau_m);
    q.om1m = (C)(1.0 - 1.0 / p.tau_m);
    q.B0 = (C)p.B0;
    q.Fx = (C)p.Fx;
    q.hFx = (C)(0.5 * p.Fx);
    q.twoB0 = (C)(2.0 * p.B0);
    const double src = 1.0 - 0.5 / p.tau_f;
    q.Ks[0] = (C)(src * 3.0 * p.Fx / 3.0);
    q.Ks[1] = (C)(src * 3.0 * p.Fx / 18.0);
    q.Ks[2] = (C)(src * 3.0 * p.Fx / 36.0);
    q.cB[0] = (C)0;
    q.cB[1] = (C)(-0.25 * 2.0 * p.B0);
    q.cB[2] = (C)(-0.125 * 2.0 * p.B0);
    q.omW0 = (C)(0.25 / p.tau_m);
    q.omW1 = (C)(0.125 / p.tau_m);
    q.omW1x4 = (C)(0.5 / p.tau_m);
    const double a = 0.5 * p.ny;
    auto wall = [&](double c, double U, double ey) {
        Wall3<C> w;
        double r, k;
        if (isinf(c)) {
            r = 1.0;
            k = 1.0;
        } else {
            const double th = c * a / (p.tau_m - 0.5);  // Eq. weightingfactor
            r = (th - 1.0) / (th + 1.0);
            k = th / (th + 1.0);
        }
        w.r = (C)r;
        // -(2 theta/(theta+1)) W e_y B0 U / c_sm^2 with W = 1/8, c_sm^2 = 1/4 (App. B.1)
        w.kx = (C)(-k * ey * p.B0 * U);
        w.du = (C)(6.0 * (1.0 / 36.0) * U);
        return w;
    };
    q.bot = wall(c_bot, u_bot, +1.0);
    q.top = wall(c_top, u_top, -1.0);
    // side walls (at rest): the same theta = c a/(tau_m - 1/2), with c relative to the Hartmann
    // half-width a
    q.rs_back = wall(c_back, 0.0, 0.0).r;
    q.rs_front = wall(c_front, 0.0, 0.0).r;
    return q;
}

// Slot k of a node's 40 populations: k = a (0..18) for f_a, k = 19 + 7 i + a for g_a of component
// i (x, y, z).  A slot whose direction enters the node through a wall (e_y = +1 in row 0, e_y = -1
// in row ny-1) is filled by the loaders with the node's own stored population of the opposite
// direction, to which wall_in3 adds the closure's terms.
__host__ __device__ constexpr int slot_dir3(int k) { return k < 19 ? k : (k - 19) % 7; }
__host__ __device__ constexpr int slot_plane3(int k, int a) { return k < 19 ? a : k - slot_dir3(k) + a - 19; }

// Link-based walls (Sec. VI; App. B.1): f by half-way bounce-back with Ladd's term on the
// diagonals; B_x and B_z by the weighted (anti-)bounce-back with ratio r, plus the moving-wall term
// on B_x; B_y by anti-bounce-back to B0 (deviation form: -v).  V: one node (C) or a pair (float2).
template <typename V, typename C>
__device__ __forceinline__ V wall_in3(const Params3<C>& p, bool bottom, bool top, int k, V v) {
    using namespace lks;
    typedef VecOf<V> K;
    if (bottom) {
        const Wall3<C>& w = p.bot;
        if (k == 7) return vadd(v, K::set(w.du));
        if (k == 10) return vsub(v, K::set(w.du));
        if (k == 19 + 3) return vfma(K::set(w.r), v, K::set(w.kx));
        if (k == 26 + 3) return vneg(v);
        if (k == 33 + 3) return vmul(K::set(w.r), v);
    }
    if (top) {
        const Wall3<C>& w = p.top;
        if (k == 8) return vsub(v, K::set(w.du));
        if (k == 9) return vadd(v, K::set(w.du));
        if (k == 19 + 4) return vfma(K::set(w.r), v, K::set(w.kx));
        if (k == 26 + 4) return vneg(v);
        if (k == 33 + 4) return vmul(K::set(w.r), v);
    }
    return v;
}

// Side walls of a duct (the planes z = -b below plane 0 and z = +b above plane nz-1, parallel to
// B0; at rest).  A slot entering through one holds the node's own stored population of the
// opposite direction.  f: half-way bounce-back (unchanged); B_x and B_y are tangential there: the
// weighted (anti-)bounce-back with the side wall's ratio r (for B_y around its applied value B0,
// which the deviation form absorbs: dg_in = r dg_out); B_z is normal: anti-bounce-back to 0 (-v).
template <typename V, typename C>
__device__ __forceinline__ V side_in3(const Params3<C>& p, bool back, int k, V v) {
    using namespace lks;
    typedef VecOf<V> K;
    const C r = back ? p.rs_back : p.rs_front;
    if (k >= 19 && k < 33) return vmul(K::set(r), v);
    if (k >= 33) return vneg(v);
    return v;
}

// e_a . (vx, vy, vz) for a != 0: the signed sum of the nonzero components, in the order x, y, z.
template <typename V>
__device__ __forceinline__ V edot3(int a, V vx, V vy, V vz) {
    using namespace lks;
    const int e[3] = {EXa(a), EYa(a), EZa(a)};
    const V c[3] = {vx, vy, vz};
    V r = c[0];
    bool first = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (e[d] == 0) continue;
        r = first ? (e[d] > 0 ? c[d] : vneg(c[d])) : (e[d] > 0 ? vadd(r, c[d]) : vsub(r, c[d]));
        first = false;
    }
    return r;
}

// Sum of n values as a balanced tree of additions (depth ceil(log2 n)); v is overwritten.
template <int N, typename V>
__device__ __forceinline__ V tree_sum3(V (&v)[N]) {
#pragma unroll
    for (int width = N; width > 1; width = (width + 1) / 2) {
#pragma unroll
        for (int i = 0; i < width / 2; ++i) v[i] = lks::vadd(v[2 * i], v[2 * i + 1]);
        if (width & 1) v[width / 2] = v[width - 1];
    }
    return v[0];
}

// Moments, equilibria, source and collision of one node or of a pair of nodes.  F(k) returns
// the streamed value of slot k (wall terms included), out(k, v) takes the post-collision value of
// slot k.  With the rest (rho = 1, u = 0, B = (0, B0, 0)) subtracted, per direction a of D3Q19
//   f^eq_a - f^rest_a = w_a (drho + rho b_a) + 4.5 w_a [ (|e_a|^2/2 - 1/6) q - (e_a.B)^2 + (e_a.B_rest)^2 ]
// with b_a = 3 e.u + 4.5 (e.u)^2 - 1.5 u^2 and q = |B|^2 - B0^2; the source is
// (1 - 1/(2 tau_f)) 3 w_a (e_a - u).F (1 + b_a); and per component i of B on D3Q7
//   g'_ai = (1 - w_m) g_ai + w_m W_a (dB_i + 4 e_ad E_di),  E_di = u_d B_i - B_d u_i  (E_ii = 0).
template <typename V, typename C, typename In, typename Out>
__device__ __forceinline__ void collide3(const Params3<C>& p, In F, Out out) {
    using namespace lks;
    typedef VecOf<V> K;
    V f[19];
#pragma unroll
    for (int a = 0; a < 19; ++a) f[a] = F(a);
    // Moments.  FP64 (bound by the FP64 pipe's latency and rate) sums as balanced trees; FP32 and
    // the FP32x2 pairs keep left-to-right sums, which need fewer live registers in the staged
    // kernel.  The one-node and two-node FP32 paths use the same order, so they agree bit for bit.
    constexpr bool kTree = std::is_same<C, double>::value;
    auto sum_of = [&](auto& v) -> V {
        constexpr int n = sizeof(v) / sizeof(v[0]);
        if constexpr (kTree) {
            return tree_sum3(v);
        } else {
            V r = v[0];
#pragma unroll
            for (int i = 1; i < n; ++i) r = vadd(r, v[i]);
            return r;
        }
    };
    V t19[19];
#pragma unroll
    for (int a = 0; a < 19; ++a) t19[a] = f[a];
    const V drho = sum_of(t19);
    auto jsum = [&](int d) -> V {
        V pos[5], neg[5];
        int np = 0, nn = 0;
#pragma unroll
        for (int a = 1; a < 19; ++a) {
            const int e = d == 0 ? EXa(a) : (d == 1 ? EYa(a) : EZa(a));
            if (e == 1) pos[np++] = f[a];
            if (e == -1) neg[nn++] = f[a];
        }
        return vsub(sum_of(pos), sum_of(neg));
    };
    const V jx = jsum(0), jy = jsum(1), jz = jsum(2);
    const V rho = vadd(K::set(C(1)), drho);
    const V inv = vrecip(rho);
    const V ux = vmul(vadd(jx, K::set(p.hFx)), inv), uy = vmul(jy, inv), uz = vmul(jz, inv);
    V g[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) g[k] = F(19 + k);
    V t7[3][7];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int a = 0; a < 7; ++a) t7[i][a] = g[7 * i + a];
    const V bx = sum_of(t7[0]), dby = sum_of(t7[1]), bz = sum_of(t7[2]);
    const V by = vadd(K::set(p.B0), dby);
    const V q = vfma(bx, bx, vfma(bz, bz, vmul(dby, vadd(K::set(p.twoB0), dby))));  // |B|^2 - B0^2
    const V usq = vfma(ux, ux, vfma(uy, uy, vmul(uz, uz)));
    const V nus15 = vmul(K::set(C(-1.5)), usq);
    // 4.5 w (|e|^2/2 - 1/6) q for |e|^2 = 0, 1, 2
    const V cq0 = vmul(K::set(C(-0.25)), q), cq1 = vmul(K::set(C(1.0 / 12.0)), q), cq2 = vmul(K::set(C(5.0 / 48.0)), q);
    // source prefactors K_|e|^2 (e_x - u_x) for the (|e|^2, e_x) that occur
    const V onemux = vsub(K::set(C(1)), ux), monemux = vsub(K::set(C(-1)), ux);
    const V kx0[3] = {vmul(K::set(-p.Ks[0]), ux), vmul(K::set(-p.Ks[1]), ux), vmul(K::set(-p.Ks[2]), ux)};
    const V kxp[3] = {kx0[0], vmul(K::set(p.Ks[1]), onemux), vmul(K::set(p.Ks[2]), onemux)};
    const V kxm[3] = {kx0[0], vmul(K::set(p.Ks[1]), monemux), vmul(K::set(p.Ks[2]), monemux)};
    const V om1f = K::set(p.om1f), omf = K::set(p.om_f);
#pragma unroll
    for (int a = 0; a < 19; ++a) {
        const int ex = EXa(a), ey = EYa(a);
        const int e2 = ex * ex + ey * ey + EZa(a) * EZa(a);
        V bm1, mag;
        if (a == 0) {
            bm1 = nus15;
            mag = cq0;
        } else {
            const V eu = edot3<V>(a, ux, uy, uz);
            const V eBm = edot3<V>(a, bx, dby, bz);  // e.B - e_y B0
            // b = 3 e.u + 4.5 (e.u)^2 - 1.5 u^2
            bm1 = vfma(vfma(K::set(C(4.5)), eu, K::set(C(3))), eu, nus15);
            // -4.5 w (e.B - e_y B0)(e.B + e_y B0) + 4.5 w (|e|^2/2 - 1/6) q
            const C cE = C(e2 == 1 ? -0.25 : -0.125);
            const V t = ey == 0 ? vmul(K::set(cE), eBm) : vfma(K::set(cE), eBm, K::set(ey > 0 ? p.cB[e2] : -p.cB[e2]));
            mag = vfma(t, eBm, e2 == 1 ? cq1 : cq2);
        }
        const C w = (C)w19(a);
        const V feq = vfma(K::set(w), vfma(rho, bm1, drho), mag);
        const V kxe = ex == 0 ? kx0[e2] : (ex > 0 ? kxp[e2] : kxm[e2]);
        const V sa = vfma(kxe, bm1, kxe);  // K (e_x - u_x) (1 + b)
        out(a, vfma(om1f, f[a], vfma(omf, feq, sa)));
    }
    const V o1 = K::set(p.om1m), ow0 = K::set(p.omW0), ow1 = K::set(p.omW1);
    const V u[3] = {ux, uy, uz}, B[3] = {bx, by, bz};
    auto comp = [&](int i, V dBi) {
        const int k0 = 19 + 7 * i;
        const V* gi = g + 7 * i;
        const V b1 = vmul(ow1, dBi);
        out(k0, vfma(o1, gi[0], vmul(ow0, dBi)));
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d == i) {
                out(k0 + 1 + 2 * d, vfma(o1, gi[1 + 2 * d], b1));
                out(k0 + 2 + 2 * d, vfma(o1, gi[2 + 2 * d], b1));
            } else {
                const V E = vfma(u[d], B[i], vneg(vmul(B[d], u[i])));
                out(k0 + 1 + 2 * d, vfma(o1, gi[1 + 2 * d], vfma(K::set(p.omW1x4), E, b1)));
                out(k0 + 2 + 2 * d, vfma(o1, gi[2 + 2 * d], vfma(K::set(-p.omW1x4), E, b1)));
            }
        }
    };
    comp(0, bx);
    comp(1, dby);
    comp(2, bz);
}

// The fused step of node (x, y, z).  S: storage type, C: compute type.  SIDE: the duct's walls at the
// z planes take the place of the periodic wrap in z.  Each cut link is closed on its own by the
// wall it crosses (no corner reconstruction); a link through both a y and a z wall (e_x = 0, f only)
// is closed by the y wall, whose bounce-back adds no moving-wall term when e_x = 0.
template <typename S, typename C, bool SIDE>
__device__ __forceinline__ void step3_node(const S* __restrict__ fin, const S* __restrict__ gin,
                                           S* __restrict__ fout, S* __restrict__ gout, const Params3<C>& p, int x,
                                           int y, int z) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int64_t N = p.N;
    const int64_t n = ((int64_t)z * ny + y) * nx + x;
    const bool bottom = (y == 0), top = (y == ny - 1);
    const int xs[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};  // source x for e_x = +1, 0, -1
    const int zs[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
    // source index of a pull along e: (x - e_x, y - e_y, z - e_z)
    auto src = [&](int ex, int ey, int ez) -> int64_t {
        return ((int64_t)zs[1 - ez] * ny + (y - ey)) * nx + xs[1 - ex];
    };
    const bool back = SIDE && z == 0, front = SIDE && z == nz - 1;
    // does the pull along direction a cross a wall?
    auto cut = [&](int a) {
        const int ey = EYa(a), ez = EZa(a);
        return (ey == 1 && bottom) || (ey == -1 && top) || (SIDE && ((ez == 1 && back) || (ez == -1 && front)));
    };
    C v[40];
#pragma unroll
    for (int a = 0; a < 19; ++a) {
        const int ey = EYa(a);
        if (cut(a)) continue;  // filled below
        v[a] = load_s<S, C>(fin + a * N + src(EXa(a), ey, EZa(a)));
    }
#pragma unroll
    for (int a = 0; a < 7; ++a) {
        const int ey = EYa(a);
        if (cut(a)) continue;
        const int64_t s = src(EXa(a), ey, EZa(a));
        v[19 + a] = load_s<S, C>(gin + a * N + s);
        v[26 + a] = load_s<S, C>(gin + (7 + a) * N + s);
        v[33 + a] = load_s<S, C>(gin + (14 + a) * N + s);
    }
    // wall rows: the node's own populations of the opposite directions, with the closure's terms
    if (bottom) {  // entering along e_y = +1: 3, 7, 10, 15, 17 (D3Q19); 3 (D3Q7)
#pragma unroll
        for (int k = 0; k < 40; ++k) {
            const int a = slot_dir3(k);
            if (EYa(a) != 1) continue;
            v[k] = wall_in3<C, C>(p, true, false, k, load_s<S, C>((k < 19 ? fin : gin) + slot_plane3(k, opp(a)) * N + n));
        }
    }
    if (top) {  // entering along e_y = -1: 4, 8, 9, 16, 18; 4
#pragma unroll
        for (int k = 0; k < 40; ++k) {
            const int a = slot_dir3(k);
            if (EYa(a) != -1) continue;
            v[k] = wall_in3<C, C>(p, false, true, k, load_s<S, C>((k < 19 ? fin : gin) + slot_plane3(k, opp(a)) * N + n));
        }
    }
    if (SIDE && (back || front)) {  // entering along e_z = +1 at z = 0, e_z = -1 at z = nz-1
#pragma unroll
        for (int k = 0; k < 40; ++k) {
            const int a = slot_dir3(k), ey = EYa(a), ez = EZa(a);
            if (!((ez == 1 && back) || (ez == -1 && front))) continue;
            if ((ey == 1 && bottom) || (ey == -1 && top)) continue;  // closed by the y wall above
            v[k] = side_in3<C, C>(p, ez == 1, k, load_s<S, C>((k < 19 ? fin : gin) + slot_plane3(k, opp(a)) * N + n));
        }
    }
    collide3<C, C>(p, [&](int k) -> C { return v[k]; },
                [&](int k, C val) { store_s<S, C>((k < 19 ? fout : gout) + slot_plane3(k, slot_dir3(k)) * N + n, val); });
}

// One node per thread, x fastest (grid: x blocks, y, z).
template <typename S, typename C>
__global__ void __launch_bounds__(256) step3_kernel(const S* __restrict__ fin, const S* __restrict__ gin,
                                                    S* __restrict__ fout, S* __restrict__ gout, const Params3<C> p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    step3_node<S, C, false>(fin, gin, fout, gout, p, x, blockIdx.y, blockIdx.z);
}

// The duct: one node per thread over the flattened node index n = (z ny + y) nx + x, so that a warp
// covers consecutive nodes (coalesced) whatever nx is -- a fully developed duct flow has nx = 1.
template <typename S, typename C>
__global__ void __launch_bounds__(256) step3_duct_kernel(const S* __restrict__ fin, const S* __restrict__ gin,
                                                         S* __restrict__ fout, S* __restrict__ gout,
                                                         const Params3<C> p) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const int64_t t = n / p.nx;
    const int x = (int)(n - t * p.nx);
    const int z = (int)(t / p.ny);
    const int y = (int)(t - (int64_t)z * p.ny);
    step3_node<S, C, true>(fin, gin, fout, gout, p, x, y, z);
}

// 16-bit storage staged through shared memory by the bulk-copy engine.  A task is R whole rows
// (y0 .. y0 + R' - 1, R' <= R, at one z; R nx <= kTaskNodes3).  For slot k the rows it pulls from,
// (y - e_y, z - e_z) of plane a_k, are R' consecutive rows in memory, so a producer warp fetches
// each slot with one bulk copy of R' nx elements (two where the task holds a wall row and e_y != 0:
// that row takes the node's own row of the opposite plane), one slot per lane, into one of
// kStages3 shared-memory stages, completing on the stage's `full` barrier.  The periodic x pull is
// an index wrap within the staged row.  Eight consumer warps take the task's nodes: 40 values from
// shared memory, collide3, 40 stores; each warp then arrives on the stage's `empty` barrier,
// which the producer waits for before it refills the stage, so kStages3 - 1 tasks' reads are in
// flight while one is computed.  Each consumer thread takes two x-adjacent nodes (x even) as one
// float2 (packed FP32 arithmetic), reading 32-bit words of the staged rows and storing one word
// per plane.  Each slot takes a fixed kTaskNodes3 elements of a stage, so the slot offsets are
// constants.  Rows must be 16-byte aligned: nx a multiple of 8, and nx <= kTaskNodes3.  A wait
// that runs out (kWaitNs) sets *err and ends that warp's loop; the producer then waits, within the
// same limit, for the last copies it issued to each stage before it returns.
constexpr int kTaskNodes3 = 512;                 // nodes of a task: consumer threads x 2
constexpr int kConsumerWarps3 = kTaskNodes3 / 64;
constexpr int kThreads3 = kTaskNodes3 / 2 + 32;  // consumers + the producer warp
constexpr int kStages3 = 5;
constexpr int kStageElems3 = 40 * kTaskNodes3;   // a slot takes kTaskNodes3 elements of a stage
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s

inline int rows_per_task3(int nx, int ny) { return std::max(1, std::min(ny, kTaskNodes3 / nx)); }
inline size_t staged_smem3() { return 128 + (size_t)kStages3 * kStageElems3 * 2; }

template <typename S>
__global__ void __launch_bounds__(kThreads3, 1) step3_staged_kernel(const S* __restrict__ fin, const S* __restrict__ gin,
                                                                    S* __restrict__ fout, S* __restrict__ gout,
                                                                    const Params3<float> p, int R, int* err) {
    extern __shared__ __align__(128) unsigned char sm3[];
    uint64_t* full = reinterpret_cast<uint64_t*>(sm3);
    uint64_t* empty = full + kStages3;
    S* stage0 = reinterpret_cast<S*>(sm3 + 128);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int64_t N = p.N;
    const int tpp = (ny + R - 1) / R;                 // tasks per z plane
    const int64_t ntask = (int64_t)nz * tpp;
    const int64_t G = gridDim.x, t0 = blockIdx.x;
    const int64_t nmine = t0 < ntask ? (ntask - 1 - t0) / G + 1 : 0;  // tasks t0, t0 + G, ...
    if (tid == 0) {
        for (int s = 0; s < kStages3; ++s) {
            lks::mbar_init(&full[s], 1);
            lks::mbar_init(&empty[s], kConsumerWarps3);
        }
        lks::mbar_init_fence();
    }
    __syncthreads();

    if (warp == kConsumerWarps3) {  // producer: lane l fetches slots l and l + 32
        int ex2[2], ey2[2], ez2[2];
        const S* bn[2];  // plane of the slot's own direction
        const S* bw[2];  // plane of the opposite direction (wall rows)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int k = lane + 32 * i < 40 ? lane + 32 * i : 39;
            const int a = slot_dir3(k);
            ex2[i] = EXa(a);
            ey2[i] = EYa(a);
            ez2[i] = EZa(a);
            const S* base = k < 19 ? fin : gin;
            bn[i] = base + slot_plane3(k, a) * N;
            bw[i] = base + slot_plane3(k, opp(a)) * N;
        }
        (void)ex2;
        int64_t it = 0;
        for (; it < nmine; ++it) {
            const int s = (int)(it % kStages3);
            const int64_t u = it / kStages3;
            if (u > 0 && !lks::mbar_wait_bounded(&empty[s], (uint32_t)(u - 1) & 1u, kWaitNs)) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            const int64_t t = t0 + it * G;
            const int z = (int)(t / tpp), y0 = (int)(t % tpp) * R;
            const int Rt = min(R, ny - y0);
            const uint32_t row_bytes = (uint32_t)nx * 2u;
            if (lane == 0) lks::mbar_arrive_expect_tx(&full[s], 40u * (uint32_t)Rt * row_bytes);
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int k = lane + 32 * i;
                if (k >= 40) continue;
                const int ey = ey2[i], ez = ez2[i];
                const int zsrc = ez == 1 ? (z == 0 ? nz - 1 : z - 1) : ez == -1 ? (z == nz - 1 ? 0 : z + 1) : z;
                const int64_t rsrc = (int64_t)zsrc * ny, rown = (int64_t)z * ny;
                S* dst = stage0 + s * kStageElems3 + k * kTaskNodes3;
                if (ey == 1 && y0 == 0) {  // row 0 is a wall row: own row 0, opposite plane
                    lks::bulk_g2s(dst, bw[i] + rown * nx, row_bytes, &full[s]);
                    if (Rt > 1) lks::bulk_g2s(dst + nx, bn[i] + rsrc * nx, (uint32_t)(Rt - 1) * row_bytes, &full[s]);
                } else if (ey == -1 && y0 + Rt == ny) {  // row ny - 1 is a wall row
                    if (Rt > 1) lks::bulk_g2s(dst, bn[i] + (rsrc + y0 + 1) * nx, (uint32_t)(Rt - 1) * row_bytes, &full[s]);
                    lks::bulk_g2s(dst + (size_t)(Rt - 1) * nx, bw[i] + (rown + ny - 1) * nx, row_bytes, &full[s]);
                } else {
                    lks::bulk_g2s(dst, bn[i] + (rsrc + y0 - ey) * nx, (uint32_t)Rt * row_bytes, &full[s]);
                }
            }
        }
        // no copy may be left in flight into this block's shared memory: wait for the last phase
        // issued to each stage (already complete unless a consumer gave up)
        for (int s = 0; s < kStages3; ++s) {
            if (it <= s) continue;
            const int64_t u_last = (it - 1 - s) / kStages3;
            if (!lks::mbar_wait_bounded(&full[s], (uint32_t)u_last & 1u, kWaitNs) && lane == 0) atomicExch(err, 1);
        }
        return;
    }

    // consumers: thread tid holds nodes x, x + 1 (x = 2 tid mod nx, even) of task row j = 2 tid / nx
    typedef lks::Packed<S> P;
    const int j = (2 * tid) / nx, x = 2 * tid - j * nx;
    const int nw = nx / 2, xw = x / 2;                        // words per row, the pair's word
    const int xwm = xw == 0 ? nw - 1 : xw - 1, xwp = xw == nw - 1 ? 0 : xw + 1;
    for (int64_t it = 0; it < nmine; ++it) {
        const int s = (int)(it % kStages3);
        if (!lks::mbar_wait_bounded(&full[s], (uint32_t)(it / kStages3) & 1u, kWaitNs)) {
            atomicExch(err, 1);
            break;
        }
        const int64_t t = t0 + it * G;
        const int z = (int)(t / tpp), y0 = (int)(t % tpp) * R;
        const int y = y0 + j;
        if (j < R && y < ny) {
            const bool bottom = (y == 0), top = (y == ny - 1);
            const uint32_t* st = reinterpret_cast<const uint32_t*>(stage0 + s * kStageElems3 + j * nx);
            const int64_t n = ((int64_t)z * ny + y) * nx + x;
            uint32_t* fo = reinterpret_cast<uint32_t*>(fout + n);
            uint32_t* go = reinterpret_cast<uint32_t*>(gout + n);
            // rows without a wall (all but two per z plane) take a path with no wall logic
            auto body = [&](auto walls) {
                constexpr bool W = decltype(walls)::value;
                auto in = [&](int k) -> float2 {
                    const int a = slot_dir3(k), ex = EXa(a), ey = EYa(a);
                    const bool wall = W && ((ey == 1 && bottom) || (ey == -1 && top));
                    const uint32_t* row = st + k * (kTaskNodes3 / 2);
                    uint32_t w;
                    if (wall || ex == 0)
                        w = row[xw];
                    else if (ex == 1)  // x <- x - 1 (high half of the word before), x + 1 <- x
                        w = __byte_perm(row[xwm], row[xw], 0x5432);
                    else  // x <- x + 1, x + 1 <- x + 2 (low half of the word after)
                        w = __byte_perm(row[xw], row[xwp], 0x5432);
                    const float2 v = P::pair(w);
                    return W ? wall_in3<float2, float>(p, bottom, top, k, v) : v;
                };
                collide3<float2, float>(p, in, [&](int k, float2 v) {
                    const size_t off = (size_t)slot_plane3(k, slot_dir3(k)) * (size_t)N / 2;
                    (k < 19 ? fo : go)[off] = P::pack(v.x, v.y);
                });
            };
            if (bottom || top)
                body(std::true_type{});
            else
                body(std::false_type{});
        }
        __syncwarp();
        if (lane == 0) lks::mbar_arrive(&empty[s]);
    }
}

// FP64 moments of the stored state of node n: rho = 1 + sum d, rho u = sum d e - F/2, B.
template <typename S>
__device__ void node_moments3(const S* f, const S* g, int64_t N, int64_t n, double B0, double Fx, double m[7]) {
    double drho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
    for (int a = 0; a < 19; ++a) {
        const double v = (double)load_s<S, float>(f + a * N + n);
        drho += v;
        jx += EXa(a) * v;
        jy += EYa(a) * v;
        jz += EZa(a) * v;
    }
    const double rho = 1.0 + drho;
    m[0] = rho;
    m[1] = (jx - 0.5 * Fx) / rho;
    m[2] = jy / rho;
    m[3] = jz / rho;
    double b[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int a = 0; a < 7; ++a) b[i] += (double)load_s<S, float>(g + (7 * i + a) * N + n);
    m[4] = b[0];
    m[5] = B0 + b[1];
    m[6] = b[2];
}
template <>
__device__ void node_moments3<double>(const double* f, const double* g, int64_t N, int64_t n, double B0, double Fx,
                                      double m[7]) {
    double drho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
    for (int a = 0; a < 19; ++a) {
        const double v = f[a * N + n];
        drho += v;
        jx += EXa(a) * v;
        jy += EYa(a) * v;
        jz += EZa(a) * v;
    }
    const double rho = 1.0 + drho;
    m[0] = rho;
    m[1] = (jx - 0.5 * Fx) / rho;
    m[2] = jy / rho;
    m[3] = jz / rho;
    double b[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int a = 0; a < 7; ++a) b[i] += g[(7 * i + a) * N + n];
    m[4] = b[0];
    m[5] = B0 + b[1];
    m[6] = b[2];
}

template <typename S>
__global__ void moments3_kernel(const S* f, const S* g, int64_t N, int64_t n0, int64_t M, double B0, double Fx,
                                double* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        double m[7];
        node_moments3<S>(f, g, N, n0 + i, B0, Fx, m);
#pragma unroll
        for (int k = 0; k < 7; ++k) out[k * M + i] = m[k];
    }
}

// x-z averages per row y: one block per row, fixed-order block reduction.
template <typename S>
__global__ void profiles3_kernel(const S* f, const S* g, int nx, int ny, int nz, double B0, double Fx, double* out) {
    __shared__ double red[7 * 32];
    const int y = blockIdx.x;
    const int64_t N = (int64_t)nx * ny * nz;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t k = threadIdx.x; k < (int64_t)nx * nz; k += blockDim.x) {
        const int z = (int)(k / nx), x = (int)(k - (int64_t)z * nx);
        double m[7];
        node_moments3<S>(f, g, N, ((int64_t)z * ny + y) * nx + x, B0, Fx, m);
#pragma unroll
        for (int c = 0; c < 7; ++c) acc[c] += m[c];
    }
    lks::block_sum<7>(acc, red);
    if (threadIdx.x == 0)
        for (int c = 0; c < 7; ++c) out[c * ny + y] = acc[c] / ((double)nx * nz);
}

// Residual partial sums (du^2, u^2, db^2, b^2 of u_x, B_x against the snapshot), one per block;
// the snapshot is replaced.  kRedBlocks blocks of 256 threads, fixed order.
template <typename S>
__global__ void residual3_partial(const S* f, const S* g, int64_t N, double B0, double Fx, double* snap,
                                  double* partial) {
    __shared__ double red[4 * 32];
    double acc[4] = {0, 0, 0, 0};
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        double m[7];
        node_moments3<S>(f, g, N, n, B0, Fx, m);
        const double du = m[1] - snap[n], db = m[4] - snap[N + n];
        acc[0] += du * du;
        acc[1] += m[1] * m[1];
        acc[2] += db * db;
        acc[3] += m[4] * m[4];
        snap[n] = m[1];
        snap[N + n] = m[4];
    }
    lks::block_sum<4>(acc, red);
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) partial[c * gridDim.x + blockIdx.x] = acc[c];
}

__global__ void residual3_final(const double* partial, int nb, double* out) {
    __shared__ double red[4 * 32];
    double acc[4];
    for (int c = 0; c < 4; ++c) acc[c] = (int)threadIdx.x < nb ? partial[c * nb + threadIdx.x] : 0.0;
    lks::block_sum<4>(acc, red);
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) out[c] = acc[c];
}

// Absolute FP64 populations <-> stored deviations, for the M nodes n0 .. n0+M-1 of the N-node
// state; the FP64 side holds 40 planes of M values (19 of f, then 21 of g).  rest_f: 19 FP64 rest
// values; g rest is W_a B0 for the y component and 0 otherwise.
template <typename S, typename C>
__global__ void to_abs3_kernel(const S* f, const S* g, int64_t N, int64_t n0, int64_t M, const double* rest_f,
                               double B0, double* of, double* og) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        // all loads before the first store: the FP64 planes may be host memory behind a link
        const int64_t n = n0 + i;
        C v[40];
#pragma unroll
        for (int a = 0; a < 19; ++a) v[a] = load_s<S, C>(f + a * N + n);
#pragma unroll
        for (int k = 0; k < 21; ++k) v[19 + k] = load_s<S, C>(g + k * N + n);
#pragma unroll
        for (int a = 0; a < 19; ++a) of[a * M + i] = (double)v[a] + rest_f[a];
#pragma unroll
        for (int k = 0; k < 21; ++k) og[k * M + i] = (double)v[19 + k] + (k / 7 == 1 ? w7(k % 7) * B0 : 0.0);
    }
}

template <typename S, typename C>
__global__ void from_abs3_kernel(const double* inf, const double* ing, int64_t N, int64_t n0, int64_t M,
                                 const double* rest_f, double B0, S* f, S* g) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        // all loads before the first store (see to_abs3_kernel)
        const int64_t n = n0 + i;
        double v[40];
#pragma unroll
        for (int a = 0; a < 19; ++a) v[a] = inf[a * M + i];
#pragma unroll
        for (int k = 0; k < 21; ++k) v[19 + k] = ing[k * M + i];
#pragma unroll
        for (int a = 0; a < 19; ++a) store_s<S, C>(f + a * N + n, (C)(v[a] - rest_f[a]));
#pragma unroll
        for (int k = 0; k < 21; ++k) store_s<S, C>(g + k * N + n, (C)(v[19 + k] - (k / 7 == 1 ? w7(k % 7) * B0 : 0.0)));
    }
}

}  // namespace

namespace {

const char* validate3(const lks3_params* p) {
    if (!p) return "params is NULL";
    if (p->nx < 1 || p->nz < 1) return "nx and nz must be >= 1";
    if (p->ny < 2) return "ny must be >= 2";
    if (p->ny > 65535 || p->nz > 65535) return "ny and nz must be <= 65535";
    if ((int64_t)p->nx * p->ny * p->nz > ((int64_t)1 << 30)) return "nx*ny*nz exceeds 2^30 nodes";
    if (p->storage < LKS_F64 || p->storage > LKS_F16_DEV) return "storage must be one of lks_storage";
    if (!(p->tau_f > 0.5) || !isfinite(p->tau_f)) return "tau_f must be finite and > 1/2";
    if (!(p->tau_m > 0.5) || !isfinite(p->tau_m)) return "tau_m must be finite and > 1/2";
    if (!isfinite(p->B0) || !isfinite(p->Fx)) return "B0 and Fx must be finite";
    return nullptr;
}

struct Layout3 {
    size_t f_bytes, g_bytes, off_f[2], off_g[2], off_snap, off_partial, off_out, off_prof, off_rest, off_flag, total;
};

Layout3 layout3(const lks3_params* p) {
    Layout3 L;
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    const size_t sb = p->storage == LKS_F64 ? 8 : (p->storage == LKS_F32 ? 4 : 2);
    L.f_bytes = align3(19 * N * sb);
    L.g_bytes = align3(21 * N * sb);
    size_t o = 0;
    for (int k = 0; k < 2; ++k) {
        L.off_f[k] = o;
        o += L.f_bytes;
        L.off_g[k] = o;
        o += L.g_bytes;
    }
    L.off_snap = o;
    o += align3(2 * N * sizeof(double));
    L.off_partial = o;
    o += align3(4 * kRedBlocks * sizeof(double));
    L.off_out = o;
    o += align3(4 * sizeof(double));
    L.off_prof = o;
    o += align3(7 * (size_t)p->ny * sizeof(double));
    L.off_rest = o;
    o += align3(19 * sizeof(double));
    L.off_flag = o;  // set by a staged step whose stage wait ran out
    o += align3(sizeof(int));
    L.total = o;
    return L;
}

}  // namespace

struct lks3_handle {
    lks3_params p;
    Layout3 L;
    cudaStream_t stream = nullptr;
    char* base = nullptr;
    bool owns = false;
    void* f[2] = {nullptr, nullptr};
    void* g[2] = {nullptr, nullptr};
    int cur = 0;
    double *snap = nullptr, *partial = nullptr, *dout = nullptr, *prof = nullptr, *rest = nullptr;
    int* flag = nullptr;
    bool staged = false;       // 16-bit storage with nx % 8 == 0: step3_staged_kernel
    unsigned staged_grid = 0;  // resident blocks of it on the device
    double* host4 = nullptr;  // pinned
    double* state_stage = nullptr;  // 40 * min(N, 2^20) doubles for state and moment transfers, on first use
    double c_bot = 0.0, c_top = 0.0, u_bot = 0.0, u_top = 0.0;
    bool side = false;                 // duct: walls at the z planes (lks3_set_side_walls)
    double c_back = 0.0, c_front = 0.0;
    int64_t steps = 0;
    std::string err;
};

namespace {

lks_status fail3(lks3_handle* h, lks_status s, const std::string& m) {
    if (h)
        h->err = m;
    else
        g3_last_error = m;
    return s;
}

lks_status cuda3(lks3_handle* h, cudaError_t e, const char* where) {
    return fail3(h, LKS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// After a synchronisation: LKS_ETIMEOUT if a staged step gave up waiting for its copies.
lks_status flag_check3(lks3_handle* h, const char* where) {
    if (!h->staged) return LKS_OK;
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, h->flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda3(h, e, where);
    if (v) return fail3(h, LKS_ETIMEOUT, std::string(where) + ": a staged step's shared-memory wait ran out");
    return LKS_OK;
}

unsigned grid_for(int64_t N) { return (unsigned)std::min<int64_t>((N + 255) / 256, 152 * 16); }

// Storage type S and compute type C of a handle.
#define LKS3_DISPATCH(storage, ...)      \
    do {                                 \
        if ((storage) == LKS_F64) {      \
            typedef double S;            \
            typedef double C;            \
            __VA_ARGS__;                    \
        } else if ((storage) == LKS_F32) { \
            typedef float S;             \
            typedef float C;             \
            __VA_ARGS__;                    \
        } else if ((storage) == LKS_BF16_DEV) { \
            typedef __nv_bfloat16 S;     \
            typedef float C;             \
            __VA_ARGS__;                    \
        } else {                         \
            typedef __half S;            \
            typedef float C;             \
            __VA_ARGS__;                    \
        }                                \
    } while (0)

template <typename S>
void launch_staged3(lks3_handle* h, int src) {
    const lks3_params& p = h->p;
    const int R = rows_per_task3(p.nx, p.ny);
    const int64_t ntask = (int64_t)p.nz * ((p.ny + R - 1) / R);
    const unsigned grid = (unsigned)std::min<int64_t>(ntask, h->staged_grid);
    const Params3<float> q = make_params3<float>(p, h->c_bot, h->c_top, h->u_bot, h->u_top);
    step3_staged_kernel<S><<<grid, kThreads3, staged_smem3(), h->stream>>>(
        (const S*)h->f[src], (const S*)h->g[src], (S*)h->f[src ^ 1], (S*)h->g[src ^ 1], q, R, h->flag);
}

// Opt the staged kernel of the handle's storage into its shared memory and size its grid.
cudaError_t prepare_staged3(lks3_handle* h) {
    int dev = 0, sms = 0, occ = 0;
    const size_t smem = staged_smem3();
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (h->p.storage == LKS_BF16_DEV) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step3_staged_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step3_staged_kernel<__nv_bfloat16>, kThreads3, smem);
    } else {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step3_staged_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step3_staged_kernel<__half>, kThreads3, smem);
    }
    if (e == cudaSuccess && occ < 1) e = cudaErrorInvalidConfiguration;
    h->staged_grid = (unsigned)(sms * occ);
    return e;
}

cudaError_t launch_step3(lks3_handle* h) {
    const lks3_params& p = h->p;
    const dim3 grid((p.nx + 255) / 256, p.ny, p.nz);
    const int src = h->cur;
    if (h->side) {
        const int64_t N = (int64_t)p.nx * p.ny * p.nz;
        LKS3_DISPATCH(p.storage, {
            const Params3<C> q = make_params3<C>(p, h->c_bot, h->c_top, h->u_bot, h->u_top, h->c_back, h->c_front);
            step3_duct_kernel<S, C><<<(unsigned)((N + 255) / 256), 256, 0, h->stream>>>(
                (const S*)h->f[src], (const S*)h->g[src], (S*)h->f[src ^ 1], (S*)h->g[src ^ 1], q);
        });
        return cudaGetLastError();
    }
    if (h->staged) {
        if (p.storage == LKS_BF16_DEV)
            launch_staged3<__nv_bfloat16>(h, src);
        else
            launch_staged3<__half>(h, src);
        return cudaGetLastError();
    }
    LKS3_DISPATCH(p.storage, {
        const Params3<C> q = make_params3<C>(p, h->c_bot, h->c_top, h->u_bot, h->u_top);
        step3_kernel<S, C><<<grid, 256, 0, h->stream>>>((const S*)h->f[src], (const S*)h->g[src], (S*)h->f[src ^ 1],
                                                        (S*)h->g[src ^ 1], q);
    });
    return cudaGetLastError();
}

cudaError_t launch_snapshot3(lks3_handle* h) {
    const int64_t N = (int64_t)h->p.nx * h->p.ny * h->p.nz;
    LKS3_DISPATCH(h->p.storage,
                  (residual3_partial<S><<<kRedBlocks, 256, 0, h->stream>>>((const S*)h->f[h->cur], (const S*)h->g[h->cur],
                                                                           N, h->p.B0, h->p.Fx, h->snap, h->partial)));
    return cudaGetLastError();
}

}  // namespace

extern "C" {

size_t lks3_footprint_bytes(const lks3_params* p) {
    if (validate3(p)) return 0;
    return layout3(p).total;
}

lks_status lks3_create(const lks3_params* p, lks3_handle** out) {
    if (!out) return fail3(nullptr, LKS_EINVAL, "out is NULL");
    *out = nullptr;
    if (const char* m = validate3(p)) return fail3(nullptr, LKS_EINVAL, m);
    lks3_handle* h = new (std::nothrow) lks3_handle();
    if (!h) return fail3(nullptr, LKS_ENOMEM, "host allocation of the handle failed");
    h->p = *p;
    h->L = layout3(p);
    h->stream = (cudaStream_t)p->cuda_stream;
    cudaError_t e;
    if (p->dev_buffer) {
        if (p->dev_buffer_bytes < h->L.total || ((uintptr_t)p->dev_buffer % kAlign3) != 0) {
            delete h;
            return fail3(nullptr, LKS_ENOMEM, "dev_buffer is smaller than lks3_footprint_bytes() or not 256-byte aligned");
        }
        h->base = (char*)p->dev_buffer;
    } else {
        e = cudaMalloc((void**)&h->base, h->L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return fail3(nullptr, LKS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        h->owns = true;
    }
    for (int k = 0; k < 2; ++k) {
        h->f[k] = h->base + h->L.off_f[k];
        h->g[k] = h->base + h->L.off_g[k];
    }
    h->snap = (double*)(h->base + h->L.off_snap);
    h->partial = (double*)(h->base + h->L.off_partial);
    h->dout = (double*)(h->base + h->L.off_out);
    h->prof = (double*)(h->base + h->L.off_prof);
    h->rest = (double*)(h->base + h->L.off_rest);
    h->flag = (int*)(h->base + h->L.off_flag);
    h->staged = (p->storage == LKS_BF16_DEV || p->storage == LKS_F16_DEV) && p->nx % 8 == 0 && p->nx <= kTaskNodes3;
    double rest[19];
    for (int a = 0; a < 19; ++a) rest[a] = f_rest(a, p->B0);
    e = cudaHostAlloc((void**)&h->host4, 4 * sizeof(double), cudaHostAllocDefault);
    // rest state: all deviations zero
    if (e == cudaSuccess) e = cudaMemsetAsync(h->f[0], 0, h->L.f_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->g[0], 0, h->L.g_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream);
    if (e == cudaSuccess && h->staged) e = prepare_staged3(h);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->rest, rest, sizeof(rest), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_snapshot3(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // rest[] is on this stack frame
    if (e != cudaSuccess) {
        lks3_destroy(h);
        return cuda3(nullptr, e, "lks3_create");
    }
    *out = h;
    return LKS_OK;
}

lks_status lks3_set_walls(lks3_handle* h, double c_bottom, double c_top, double u_bottom, double u_top) {
    if (!h) return fail3(nullptr, LKS_EINVAL, "handle is NULL");
    if (!(c_bottom >= 0.0) || !(c_top >= 0.0)) return fail3(h, LKS_EINVAL, "wall conductance ratios must be >= 0");
    if (!(fabs(u_bottom) < 0.3) || !(fabs(u_top) < 0.3)) return fail3(h, LKS_EINVAL, "|wall speed| must be < 0.3");
    h->c_bot = c_bottom;
    h->c_top = c_top;
    h->u_bot = u_bottom;
    h->u_top = u_top;
    return LKS_OK;
}

lks_status lks3_set_side_walls(lks3_handle* h, int32_t enable, double c_back, double c_front) {
    if (!h) return fail3(nullptr, LKS_EINVAL, "handle is NULL");
    if (enable != 0 && enable != 1) return fail3(h, LKS_EINVAL, "enable must be 0 or 1");
    if (!(c_back >= 0.0) || !(c_front >= 0.0)) return fail3(h, LKS_EINVAL, "side-wall conductance ratios must be >= 0");
    if (enable && h->p.nz < 2) return fail3(h, LKS_EINVAL, "a duct needs nz >= 2");
    h->side = enable != 0;
    h->c_back = c_back;
    h->c_front = c_front;
    return LKS_OK;
}

lks_status lks3_step(lks3_handle* h, int64_t n) {
    if (!h) return fail3(nullptr, LKS_EINVAL, "handle is NULL");
    if (n < 0) return fail3(h, LKS_EINVAL, "n must be >= 0");
    for (int64_t k = 0; k < n; ++k) {
        cudaError_t e = launch_step3(h);
        if (e != cudaSuccess) return cuda3(h, e, "3D step kernel launch");
        h->cur ^= 1;
        h->steps += 1;
    }
    return LKS_OK;
}

int64_t lks3_steps_taken(const lks3_handle* h) { return h ? h->steps : -1; }

// State transfers and per-node host moments convert kStateChunk3 nodes at a time through a staging
// buffer the handle keeps, so their device memory stays bounded (335 MB) whatever the lattice size.
constexpr int64_t kStateChunk3 = int64_t(1) << 20;

static lks_status state_stage3(lks3_handle* h, int64_t* chunk) {
    const int64_t N = (int64_t)h->p.nx * h->p.ny * h->p.nz;
    *chunk = N < kStateChunk3 ? N : kStateChunk3;
    if (!h->state_stage) {
        cudaError_t e = cudaMalloc((void**)&h->state_stage, 40 * (size_t)*chunk * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->state_stage = nullptr;
            return fail3(h, LKS_ENOMEM, "cudaMalloc of the FP64 state staging buffer failed");
        }
    }
    return LKS_OK;
}

lks_status lks3_moments(lks3_handle* h, int what, double* host_out) {
    if (!h) return fail3(nullptr, LKS_EINVAL, "handle is NULL");
    if (!host_out) return fail3(h, LKS_EINVAL, "host_out is NULL");
    const lks3_params& p = h->p;
    const int64_t N = (int64_t)p.nx * p.ny * p.nz;
    cudaError_t e;
    if (what == LKS_MOMENTS_PROFILES) {
        LKS3_DISPATCH(p.storage, (profiles3_kernel<S><<<p.ny, 256, 0, h->stream>>>(
                                     (const S*)h->f[h->cur], (const S*)h->g[h->cur], p.nx, p.ny, p.nz, p.B0, p.Fx, h->prof)));
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_out, h->prof, 7 * (size_t)p.ny * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    } else if (what == LKS_MOMENTS_NODES) {
        // page-locked host_out: written by the kernel (one chunk of N nodes); else M nodes at a time
        // through the staging buffer
        double* direct = (double*)lks::host_direct_ptr(host_out);
        int64_t M = N;
        if (!direct) {
            if (lks_status s = state_stage3(h, &M)) return s;
        }
        double* out = direct ? direct : h->state_stage;
        e = cudaSuccess;
        for (int64_t n0 = 0; n0 < N && e == cudaSuccess; n0 += M) {
            const int64_t m = N - n0 < M ? N - n0 : M;
            LKS3_DISPATCH(p.storage, (moments3_kernel<S><<<grid_for(m), 256, 0, h->stream>>>(
                                         (const S*)h->f[h->cur], (const S*)h->g[h->cur], N, n0, m, p.B0, p.Fx, out)));
            e = cudaGetLastError();
            for (int k = 0; k < 7 && e == cudaSuccess && !direct; ++k)
                e = cudaMemcpyAsync(host_out + k * N + n0, out + k * m, m * sizeof(double), cudaMemcpyDeviceToHost,
                                    h->stream);
        }
    } else {
        return fail3(h, LKS_EINVAL, "bad 'what'");
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda3(h, e, "lks3_moments");
    return flag_check3(h, "lks3_moments");
}

lks_status lks3_residual(lks3_handle* h, double* r_u, double* r_b) {
    if (!h) return fail3(nullptr, LKS_EINVAL, "handle is NULL");
    cudaError_t e = launch_snapshot3(h);
    if (e == cudaSuccess) {
        residual3_final<<<1, 1024, 0, h->stream>>>(h->partial, kRedBlocks, h->dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->host4, h->dout, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda3(h, e, "lks3_residual");
    if (lks_status fs = flag_check3(h, "lks3_residual")) return fs;
    const double* s = h->host4;
    const double ru = s[1] > 1e-30 * 1e-30 ? sqrt(s[0] / s[1]) : 0.0;
    const double rb = s[3] > 1e-30 * 1e-30 ? sqrt(s[2] / s[3]) : 0.0;
    if (r_u) *r_u = ru;
    if (r_b) *r_b = rb;
    if (!isfinite(s[0]) || !isfinite(s[1]) || !isfinite(s[2]) || !isfinite(s[3]))
        return fail3(h, LKS_EUNSTABLE, "non-finite state");
    return LKS_OK;
}

lks_status lks3_run_to_steady(lks3_handle* h, double tol, int64_t check_every, int64_t max_steps, int64_t* steps_out,
                              double* r_out) {
    if (!h) return fail3(nullptr, LKS_EINVAL, "handle is NULL");
    if (check_every < 1 || max_steps < 0 || !(tol > 0.0)) return fail3(h, LKS_EINVAL, "bad run_to_steady arguments");
    int64_t taken = 0;
    double r = INFINITY, best = INFINITY;
    int since_best = 0;
    bool stalled = false;
    const bool zero_stalls = lks::zero_residual_is_stall(h->p.storage, h->p.Fx, h->u_bot, h->u_top);
    lks_status s = LKS_OK;
    while (taken < max_steps) {
        const int64_t n = (max_steps - taken < check_every) ? max_steps - taken : check_every;
        s = lks3_step(h, n);
        if (s != LKS_OK) break;
        taken += n;
        double ru, rb;
        s = lks3_residual(h, &ru, &rb);
        if (s != LKS_OK) break;
        r = ru > rb ? ru : rb;
        if (r == 0.0 && zero_stalls) {
            stalled = true;
            break;
        }
        if (r < tol) break;
        if (r < best) {
            best = r;
            since_best = 0;
        } else if (++since_best >= lks::kStallChecks && best < lks::stall_floor(h->p.storage)) {
            stalled = true;
            break;
        }
    }
    if (steps_out) *steps_out = taken;
    if (r_out) *r_out = r;
    if (s != LKS_OK) return s;
    if (stalled)
        return fail3(h, LKS_ESTALLED,
                     r == 0.0 ? "the state stopped changing (per-step increments below the storage resolution)"
                              : "the residual stopped decreasing at the storage's rounding floor");
    if (!(r < tol)) return fail3(h, LKS_ENOTCONVERGED, "max_steps reached before the residual tolerance");
    return LKS_OK;
}

// State transfers and per-node host moments: for page-locked host arrays one chunk of N nodes whose
// FP64 planes are the caller's arrays themselves; otherwise M nodes at a time through the staging
// buffer, one copy per plane.
lks_status lks3_get_state(lks3_handle* h, double* host_f, double* host_g) {
    if (!h) return fail3(nullptr, LKS_EINVAL, "handle is NULL");
    if (!host_f || !host_g) return fail3(h, LKS_EINVAL, "host_f/host_g is NULL");
    const int64_t N = (int64_t)h->p.nx * h->p.ny * h->p.nz;
    double* df = (double*)lks::host_direct_ptr(host_f);
    double* dg = (double*)lks::host_direct_ptr(host_g);
    const bool direct = df && dg;
    int64_t M = N;
    if (!direct) {
        if (lks_status s = state_stage3(h, &M)) return s;
    }
    cudaError_t e = cudaSuccess;
    for (int64_t n0 = 0; n0 < N && e == cudaSuccess; n0 += M) {
        const int64_t m = N - n0 < M ? N - n0 : M;
        double* of = direct ? df : h->state_stage;
        double* og = direct ? dg : h->state_stage + 19 * m;
        LKS3_DISPATCH(h->p.storage, (to_abs3_kernel<S, C><<<grid_for(m), 256, 0, h->stream>>>(
                                        (const S*)h->f[h->cur], (const S*)h->g[h->cur], N, n0, m, h->rest, h->p.B0,
                                        of, og)));
        e = cudaGetLastError();
        for (int a = 0; a < 40 && e == cudaSuccess && !direct; ++a) {
            double* dst = a < 19 ? host_f + a * N + n0 : host_g + (a - 19) * N + n0;
            e = cudaMemcpyAsync(dst, h->state_stage + a * m, m * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda3(h, e, "lks3_get_state");
    return flag_check3(h, "lks3_get_state");
}

lks_status lks3_set_state(lks3_handle* h, const double* host_f, const double* host_g) {
    if (!h) return fail3(nullptr, LKS_EINVAL, "handle is NULL");
    if (!host_f || !host_g) return fail3(h, LKS_EINVAL, "host_f/host_g is NULL");
    const int64_t N = (int64_t)h->p.nx * h->p.ny * h->p.nz;
    const double* df = (const double*)lks::host_direct_ptr(host_f);
    const double* dg = (const double*)lks::host_direct_ptr(host_g);
    const bool direct = df && dg;
    int64_t M = N;
    if (!direct) {
        if (lks_status s = state_stage3(h, &M)) return s;
    }
    cudaError_t e = cudaSuccess;
    for (int64_t n0 = 0; n0 < N && e == cudaSuccess; n0 += M) {
        const int64_t m = N - n0 < M ? N - n0 : M;
        const double* sf = df;
        const double* sg = dg;
        if (!direct) {
            for (int a = 0; a < 40 && e == cudaSuccess; ++a) {
                const double* src = a < 19 ? host_f + a * N + n0 : host_g + (a - 19) * N + n0;
                e = cudaMemcpyAsync(h->state_stage + a * m, src, m * sizeof(double), cudaMemcpyHostToDevice,
                                    h->stream);
            }
            sf = h->state_stage;
            sg = h->state_stage + 19 * m;
        }
        if (e == cudaSuccess) {
            LKS3_DISPATCH(h->p.storage, (from_abs3_kernel<S, C><<<grid_for(m), 256, 0, h->stream>>>(
                                            sf, sg, N, n0, m, h->rest, h->p.B0, (S*)h->f[h->cur], (S*)h->g[h->cur])));
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = launch_snapshot3(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda3(h, e, "lks3_set_state");
    h->steps = 0;
    return LKS_OK;
}

lks_status lks3_selftest_wait_timeout(lks3_handle* h, double limit_s) {
    if (!h) return fail3(nullptr, LKS_EINVAL, "handle is NULL");
    if (!h->staged) return fail3(h, LKS_EINVAL, "lks3_selftest_wait_timeout: the handle runs no staged kernel");
    if (!(limit_s > 0.0 && limit_s <= 1.0))
        return fail3(h, LKS_EINVAL, "lks3_selftest_wait_timeout: limit not in (0, 1] s");
    cudaError_t e = lks::launch_wait_timeout_probe(h->flag, (uint64_t)(limit_s * 1e9), h->stream);
    if (e != cudaSuccess) return cuda3(h, e, "lks3_selftest_wait_timeout");
    return LKS_OK;
}

lks_status lks3_sync(lks3_handle* h) {
    if (!h) return fail3(nullptr, LKS_EINVAL, "handle is NULL");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda3(h, e, "lks3_sync");
    return flag_check3(h, "lks3_sync");
}

lks_status lks3_destroy(lks3_handle* h) {
    if (!h) return LKS_OK;
    if (h->stream || h->base) cudaStreamSynchronize(h->stream);
    if (h->state_stage) cudaFree(h->state_stage);
    if (h->owns && h->base) cudaFree(h->base);
    if (h->host4) cudaFreeHost(h->host4);
    delete h;
    return LKS_OK;
}

const char* lks3_last_error(const lks3_handle* h) { return h ? h->err.c_str() : g3_last_error.c_str(); }

}  // extern "C"
