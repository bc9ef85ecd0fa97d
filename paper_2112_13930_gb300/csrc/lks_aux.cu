// lks_aux.cu -- initial state, moments, x-averaged profiles, the steady-state residual
// reduction and the FP64 <-> storage conversions.  None of these is on the per-step path.
#include <type_traits>

#include "lks_device.cuh"
#include "lks_internal.h"

namespace lks {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double w9(int a) { return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
__device__ __forceinline__ double w5(int a) { return a == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
__device__ __forceinline__ int ex9(int a) {
    const int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    return t[a];
}
__device__ __forceinline__ int ey9(int a) {
    const int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    return t[a];
}
// Rest equilibrium f^eq(rho = 1, u = 0, B = (0, B0)): with the Maxwell stress (coupling 0) or
// without magnetic terms (coupling 1, Lorentz force in the source).
__device__ __forceinline__ double f_rest(int a, double B0, int coupling) {
    if (coupling == 1) return w9(a);
    const double m = (a == 1 || a == 3) ? 0.5 * B0 * B0 : ((a == 2 || a == 4) ? -0.5 * B0 * B0 : 0.0);
    return w9(a) * (1.0 + 4.5 * m);
}

// What the moments of a stored state depend on.
struct MomentModel {
    double B0, Fx, tau_m;
    int coupling;
};

// Storage slot of node n.  ilv = 0: the node order, n = y nx + x.  ilv = nx (16-bit storage, nx
// even): rows interleaved for the two-nodes-per-thread kernels -- 32-bit word w of a row holds
// node x = w in its lower half and x = w + nx/2 in its upper half, so slot 2 (x mod nx/2) + (x >= nx/2).
__device__ __forceinline__ int64_t slot_of(int64_t n, int ilv) {
    if (ilv == 0) return n;
    const int64_t y = n / ilv;
    const int x = (int)(n - y * ilv);
    const int h = ilv >> 1;
    return y * ilv + (x < h ? 2 * x : 2 * (x - h) + 1);
}

// SplitMix64 (Steele, Lea & Flood 2014) of seed XOR counter -> [0, 1) with 53 bits.
__device__ __forceinline__ double splitmix_unit(uint64_t seed, uint64_t counter) {
    uint64_t z = (seed ^ counter) + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

template <typename S, typename C>
__global__ void init_kernel(S* f, S* g, int64_t N, double B0, uint64_t seed, double amp, int ilv) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int64_t pn = slot_of(n, ilv);
    double ux = 0.0, uy = 0.0;
    if (amp != 0.0) {
        ux = amp * (2.0 * splitmix_unit(seed, 2ull * (uint64_t)n) - 1.0);
        uy = amp * (2.0 * splitmix_unit(seed, 2ull * (uint64_t)n + 1ull) - 1.0);
    }
    const double usq = 1.5 * (ux * ux + uy * uy);
    for (int a = 0; a < 9; ++a) {
        const double eu = ex9(a) * ux + ey9(a) * uy;
        const double b = 3.0 * eu + 4.5 * eu * eu - usq;  // rho = 1, B = rest
        store_s<S, C>(f + a * N + pn, (C)(w9(a) * b));
    }
    const double E = ux * B0;  // u_x B_y - u_y B_x at B = (0, B0)
    for (int a = 0; a < 5; ++a) {
        store_s<S, C>(g + a * N + pn, (C)(-3.0 * w5(a) * ey9(a) * E));
        store_s<S, C>(g + (5 + a) * N + pn, (C)(3.0 * w5(a) * ex9(a) * E));
    }
}

// FP64 moments of the node stored in slot n of a state: rho, u_x, u_y, B_x, B_y.
// Coupling 0: rho u = sum f~ e - F/2.  Coupling 1: the force includes J x B; the stored g carries
// (1 - 1/tau_m) Lambda^(1) of the last collision, so with k' = 3/(tau_m - 1) and
// D~ = Lambda~_yx - Lambda~_xy:  J_z = k' [D~ + 2 (B_y (j_x - F_ext/2) - B_x j_y)/rho] / (1 - k' |B|^2/rho).
//
// FP32 and 16-bit storage (C = float, Maxwell coupling): the per-node sums and u are taken in FP32,
// the type the state is held and stepped in -- the stored values carry FP32 precision at best, so
// FP64 here only cost time (these readouts were FP64-pipe bound) -- and converted to FP64 for the
// accumulation across nodes, which stays FP64.  FP64 storage and the Lorentz coupling take FP64.
template <typename S, typename C>
__device__ __forceinline__ void node_moments(const S* f, const S* g, int64_t N, int64_t n, const MomentModel& mm,
                                             double m[5]) {
    if constexpr (std::is_same<C, float>::value) {
        if (mm.coupling == 0) {
            float fv[9], gv5[10];
#pragma unroll
            for (int a = 0; a < 9; ++a) fv[a] = load_s<S, C>(f + a * N + n);
#pragma unroll
            for (int a = 0; a < 10; ++a) gv5[a] = load_s<S, C>(g + a * N + n);
            const float drho = (((fv[0] + fv[1]) + (fv[2] + fv[3])) + ((fv[4] + fv[5]) + (fv[6] + fv[7]))) + fv[8];
            const float jx = ((fv[1] - fv[3]) + (fv[5] - fv[6])) + (fv[8] - fv[7]);
            const float jy = ((fv[2] - fv[4]) + (fv[5] + fv[6])) - (fv[7] + fv[8]);
            const float bx = ((gv5[0] + gv5[1]) + (gv5[2] + gv5[3])) + gv5[4];
            const float dby = ((gv5[5] + gv5[6]) + (gv5[7] + gv5[8])) + gv5[9];
            const float rho = 1.0f + drho;
            const float inv = __frcp_rn(rho);
            m[0] = (double)rho;
            m[1] = (double)__fmul_rn(__fadd_rn(jx, -0.5f * (float)mm.Fx), inv);
            m[2] = (double)__fmul_rn(jy, inv);
            m[3] = (double)bx;
            m[4] = mm.B0 + (double)dby;
            return;
        }
    }
    double drho = 0.0, jx = 0.0, jy = 0.0, bx = 0.0, dby = 0.0;
    double gv[10];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const double v = (double)load_s<S, C>(f + a * N + n);
        drho += v;
        jx += ex9(a) * v;
        jy += ey9(a) * v;
    }
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        gv[a] = (double)load_s<S, C>(g + a * N + n);
        gv[5 + a] = (double)load_s<S, C>(g + (5 + a) * N + n);
        bx += gv[a];
        dby += gv[5 + a];
    }
    const double rho = 1.0 + drho;
    const double by = mm.B0 + dby;
    double ux = (jx - 0.5 * mm.Fx) / rho, uy = jy / rho;
    if (mm.coupling == 1) {
        const double kp = 3.0 / (mm.tau_m - 1.0);
        const double D = (gv[2] - gv[4]) - (gv[5 + 1] - gv[5 + 3]);
        const double jxp = jx - 0.5 * mm.Fx;
        const double jz = kp * (D + 2.0 * (by * jxp - bx * jy) / rho) / (1.0 - kp * (bx * bx + by * by) / rho);
        ux = (jxp + 0.5 * jz * by) / rho;
        uy = (jy - 0.5 * jz * bx) / rho;
    }
    m[0] = rho;
    m[1] = ux;
    m[2] = uy;
    m[3] = bx;
    m[4] = by;
}

// Moments of the M nodes n0 .. n0+M-1 of the N-node state: out[k*M + i] for node n0 + i.
template <typename S, typename C>
__global__ void moments_kernel(const S* f, const S* g, int64_t N, int64_t n0, int64_t M, MomentModel mm,
                               double* out, int ilv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    double m[5];
    node_moments<S, C>(f, g, N, slot_of(n0 + i, ilv), mm, m);
#pragma unroll
    for (int k = 0; k < 5; ++k) out[k * M + i] = m[k];
}

template <typename S, typename C>
__global__ void __launch_bounds__(kThreads) profiles_kernel(const S* f, const S* g, int nx, int ny, MomentModel mm,
                                                           double* out, int ilv) {
    __shared__ double sh[5 * 32];
    const int j = blockIdx.x;
    const int64_t N = (int64_t)nx * ny;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < nx; i += kThreads) {
        double m[5];
        node_moments<S, C>(f, g, N, slot_of((int64_t)j * nx + i, ilv), mm, m);
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += m[k];
    }
    block_sum<5>(acc, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 5; ++k) out[k * ny + j] = acc[k] / nx;
}

template <typename S, typename C>
__global__ void __launch_bounds__(kThreads) residual_partial_kernel(const S* f, const S* g, int64_t N,
                                                                   MomentModel mm, double* snap, double* partial,
                                                                   int ilv) {
    __shared__ double sh[4 * 32];
    double acc[4] = {0, 0, 0, 0};
    for (int64_t n = (int64_t)blockIdx.x * kThreads + threadIdx.x; n < N; n += (int64_t)gridDim.x * kThreads) {
        double m[5];
        node_moments<S, C>(f, g, N, slot_of(n, ilv), mm, m);
        const double du = m[1] - snap[n];
        const double db = m[3] - snap[N + n];
        acc[0] += du * du;
        acc[1] += m[1] * m[1];
        acc[2] += db * db;
        acc[3] += m[3] * m[3];
        snap[n] = m[1];
        snap[N + n] = m[3];
    }
    block_sum<4>(acc, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) partial[4 * blockIdx.x + k] = acc[k];
}

__global__ void __launch_bounds__(kThreads) residual_final_kernel(const double* partial, int nblk, double* out) {
    __shared__ double sh[4 * 32];
    double acc[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += kThreads)
        for (int k = 0; k < 4; ++k) acc[k] += partial[4 * b + k];
    block_sum<4>(acc, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) out[k] = acc[k];
}

template <typename S, typename C>
__global__ void snapshot_kernel(const S* f, const S* g, int64_t N, MomentModel mm, double* snap, int ilv) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double m[5];
    node_moments<S, C>(f, g, N, slot_of(n, ilv), mm, m);
    snap[n] = m[1];
    snap[N + n] = m[3];
}

template <typename S, typename C>
__global__ void to_abs_kernel(const S* f, const S* g, int64_t N, int64_t n0, int64_t M, double B0, int coupling,
                              double* fa, double* ga, int ilv) {
    // nodes n0 .. n0 + M - 1 into planes of stride M
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    // All loads before the first store: the FP64 planes may be host memory behind a link with
    // microseconds of latency, and a store the compiler cannot prove disjoint would order the loads.
    const int64_t pn = slot_of(n0 + i, ilv);
    C v[19];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = load_s<S, C>(f + a * N + pn);
#pragma unroll
    for (int a = 0; a < 10; ++a) v[9 + a] = load_s<S, C>(g + a * N + pn);
#pragma unroll
    for (int a = 0; a < 9; ++a) fa[a * M + i] = (double)v[a] + f_rest(a, B0, coupling);
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        ga[a * M + i] = (double)v[9 + a];
        ga[(5 + a) * M + i] = (double)v[14 + a] + w5(a) * B0;
    }
}

template <typename S, typename C>
__global__ void from_abs_kernel(const double* fa, const double* ga, int64_t N, int64_t n0, int64_t M, double B0,
                                int coupling, S* f, S* g, int ilv) {
    // nodes n0 .. n0 + M - 1 from planes of stride M
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    // All loads before the first store (see to_abs_kernel).
    const int64_t pn = slot_of(n0 + i, ilv);
    double v[19];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = fa[a * M + i];
#pragma unroll
    for (int a = 0; a < 10; ++a) v[9 + a] = ga[a * M + i];
#pragma unroll
    for (int a = 0; a < 9; ++a) store_s<S, C>(f + a * N + pn, (C)(v[a] - f_rest(a, B0, coupling)));
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        store_s<S, C>(g + a * N + pn, (C)v[9 + a]);
        store_s<S, C>(g + (5 + a) * N + pn, (C)(v[14 + a] - w5(a) * B0));
    }
}

inline unsigned grid_for(int64_t N) { return (unsigned)((N + kThreads - 1) / kThreads); }

}  // namespace

#define LKS_DISPATCH(storage, CALL)                          \
    do {                                                     \
        if ((storage) == 0) {                                \
            typedef double S;                                \
            typedef double C;                                \
            CALL;                                            \
        } else if ((storage) == 1) {                         \
            typedef float S;                                 \
            typedef float C;                                 \
            CALL;                                            \
        } else if ((storage) == 2) {                         \
            typedef __nv_bfloat16 S;                         \
            typedef float C;                                 \
            CALL;                                            \
        } else {                                             \
            typedef __half S;                                \
            typedef float C;                                 \
            CALL;                                            \
        }                                                    \
    } while (0)

cudaError_t launch_init(int storage, void* f, void* g, int nx, int ny, double B0, uint64_t seed, double amp,
                        cudaStream_t st, int ilv) {
    const int64_t N = (int64_t)nx * ny;
    LKS_DISPATCH(storage, (init_kernel<S, C><<<grid_for(N), kThreads, 0, st>>>((S*)f, (S*)g, N, B0, seed, amp, ilv)));
    return cudaGetLastError();
}

cudaError_t launch_moments(int storage, const void* f, const void* g, int nx, int ny, double B0, double Fx,
                           int what, double* out, cudaStream_t st, int coupling, double tau_m, int ilv) {
    const int64_t N = (int64_t)nx * ny;
    const MomentModel mm{B0, Fx, tau_m, coupling};
    if (what == 0) {
        LKS_DISPATCH(storage, (moments_kernel<S, C><<<grid_for(N), kThreads, 0, st>>>((const S*)f, (const S*)g, N,
                                                                                      0, N, mm, out, ilv)));
    } else {
        LKS_DISPATCH(storage, (profiles_kernel<S, C><<<ny, kThreads, 0, st>>>((const S*)f, (const S*)g, nx, ny, mm,
                                                                              out, ilv)));
    }
    return cudaGetLastError();
}

cudaError_t launch_node_moments(int storage, const void* f, const void* g, int64_t N, int64_t n0, int64_t M,
                                double B0, double Fx, double* out, cudaStream_t st, int coupling, double tau_m,
                                int ilv) {
    const MomentModel mm{B0, Fx, tau_m, coupling};
    LKS_DISPATCH(storage, (moments_kernel<S, C><<<grid_for(M), kThreads, 0, st>>>((const S*)f, (const S*)g, N, n0,
                                                                                  M, mm, out, ilv)));
    return cudaGetLastError();
}

int residual_blocks(int64_t N) {
    int64_t b = (N + 2047) / 2048;
    if (b < 1) b = 1;
    if (b > kResidualMaxBlocks) b = kResidualMaxBlocks;
    return (int)b;
}

cudaError_t launch_residual(int storage, const void* f, const void* g, int nx, int ny, double B0, double Fx,
                            double* snap, double* partial, double* out, cudaStream_t st, int coupling, double tau_m,
                            int ilv) {
    const int64_t N = (int64_t)nx * ny;
    const int nblk = residual_blocks(N);
    const MomentModel mm{B0, Fx, tau_m, coupling};
    LKS_DISPATCH(storage, (residual_partial_kernel<S, C><<<nblk, kThreads, 0, st>>>((const S*)f, (const S*)g, N,
                                                                                    mm, snap, partial, ilv)));
    residual_final_kernel<<<1, kThreads, 0, st>>>(partial, nblk, out);
    return cudaGetLastError();
}

cudaError_t launch_snapshot(int storage, const void* f, const void* g, int nx, int ny, double B0, double Fx,
                            double* snap, cudaStream_t st, int coupling, double tau_m, int ilv) {
    const int64_t N = (int64_t)nx * ny;
    const MomentModel mm{B0, Fx, tau_m, coupling};
    LKS_DISPATCH(storage, (snapshot_kernel<S, C><<<grid_for(N), kThreads, 0, st>>>((const S*)f, (const S*)g, N, mm,
                                                                                   snap, ilv)));
    return cudaGetLastError();
}

cudaError_t launch_to_abs(int storage, const void* f, const void* g, int64_t N, int64_t n0, int64_t M, double B0,
                          double* fabs, double* gabs, cudaStream_t st, int coupling, int ilv) {
    LKS_DISPATCH(storage, (to_abs_kernel<S, C><<<grid_for(M), kThreads, 0, st>>>((const S*)f, (const S*)g, N, n0, M,
                                                                                 B0, coupling, fabs, gabs, ilv)));
    return cudaGetLastError();
}

cudaError_t launch_from_abs(int storage, const double* fabs, const double* gabs, int64_t N, int64_t n0, int64_t M,
                            double B0, void* f, void* g, cudaStream_t st, int coupling, int ilv) {
    LKS_DISPATCH(storage, (from_abs_kernel<S, C><<<grid_for(M), kThreads, 0, st>>>(fabs, gabs, N, n0, M, B0, coupling,
                                                                                   (S*)f, (S*)g, ilv)));
    return cudaGetLastError();
}

}  // namespace lks
