// lks_batch.cu -- batched / served solver of many independent channel instances (lks_batch.h).
//
// One persistent kernel launch per lks_batch_run: every CTA is split into groups of
// threads_per_group threads; a group takes the next running instance from a work list with one
// atomicAdd (no spin-wait anywhere), advances it step after step with the same per-node update
// as the single-lattice kernel (step_node), synchronising only its own threads (a named barrier
// per group) between steps, and checks the steady-state residual every check_every steps with a
// fixed-order reduction.  An instance's state (two population buffers + residual snapshot, about
// 170 B per FP32 node) stays in L2 while its group works on it, so the per-step traffic is served
// from L2 rather than HBM.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <map>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lks_batch.h"
#include "lks_aa.cuh"
#include "lks_internal.h"

using lks::StepParams;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxGroups = 15;  // named barriers 1..15 (0 is __syncthreads)
// An instance is declared STALLED when its residual has not reached a new minimum for kStallChecks
// checks in a row while already below the rounding floor of the storage type (lks::stall_floor), or
// when the residual is exactly 0 on a driven channel stored in FP32 or 16 bits
// (lks::zero_residual_is_stall): the state stopped changing, it did not converge.
using lks::kStallChecks;
using lks::stall_floor;

inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Device-side record of one instance.
struct InstDev {
    StepParams<double> pd;
    char* f[2];
    char* g[2];
    double* snap;
    int64_t steps, check_every, max_steps;
    double tol, best_r, residual, stall_below, tau_m;
    int32_t closure, cur, state, stall;
};

// Per-slot result, same layout as lks_instance_result; pad carries the current buffer index.
struct ResultDev {
    int32_t state, cur;
    int64_t steps;
    double residual;
};

struct Ctl {
    int32_t nwork;
    int32_t pad;
    int64_t quantum;
};

__device__ __forceinline__ void group_sync(int gid, int T) {
    asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(T) : "memory");
}

template <typename C>
__device__ __forceinline__ StepParams<C> to_compute(const StepParams<double>& d) {
    StepParams<C> o;
    o.nx = d.nx;
    o.ny = d.ny;
    o.N = d.N;
    o.omega_f = (C)d.omega_f;
    o.omega_m = (C)d.omega_m;
    o.src_coef = (C)d.src_coef;
    o.Fx = (C)d.Fx;
    o.B0 = (C)d.B0;
    o.om1f = (C)d.om1f; o.om1m = (C)d.om1m;
    o.owf0 = (C)d.owf0; o.owf1 = (C)d.owf1; o.owf5 = (C)d.owf5;
    o.owm0 = (C)d.owm0; o.owm1 = (C)d.owm1;
    o.sw0 = (C)d.sw0; o.sw1 = (C)d.sw1; o.sw5 = (C)d.sw5;
    o.src3 = (C)d.src3; o.coupling = d.coupling;
    o.bot.r = (C)d.bot.r; o.bot.bc = (C)d.bot.bc; o.bot.kx = (C)d.bot.kx; o.bot.du = (C)d.bot.du; o.bot.U = (C)d.bot.U;
    o.top.r = (C)d.top.r; o.top.bc = (C)d.top.bc; o.top.kx = (C)d.top.kx; o.top.du = (C)d.top.du; o.top.U = (C)d.top.U;
    return o;
}

// u_x and B_x (FP64) of node n of a stored post-collision state, loads through L.  Maxwell
// coupling: rho u_x = sum f~ e_x - F_x/2.  Lorentz coupling: J_z is read back from the
// (1 - 1/tau_m)-scaled non-equilibrium moment of the stored g, as for lks_moments.
template <typename S, typename C, typename L, int COUPLING>
__device__ __forceinline__ void stored_ux_bx(const S* f, const S* g, int64_t N, int64_t n, const InstDev* I,
                                             double& ux, double& bx) {
    double v[9], w[10];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = (double)L::ld(f + a * N + n);
#pragma unroll
    for (int a = 0; a < 10; ++a) w[a] = (double)L::ld(g + a * N + n);
    const double drho = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
    const double jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
    const double rho = 1.0 + drho;
    const double Fx = (double)I->pd.Fx;
    bx = ((w[0] + w[1]) + (w[2] + w[3])) + w[4];
    if (COUPLING == 1) {
        const double jy = (v[2] - v[4]) + (v[5] + v[6]) - (v[7] + v[8]);
        const double by = (double)I->pd.B0 + (((w[5] + w[6]) + (w[7] + w[8])) + w[9]);
        const double kp = 3.0 / (I->tau_m - 1.0);
        const double D = (w[2] - w[4]) - (w[6] - w[8]);
        const double jxp = lks::ffma(-0.5, Fx, jx);
        const double jz = lks::fmul(kp, D + lks::fmul(2.0, lks::ffma(by, jxp, -lks::fmul(bx, jy))) / rho) /
                          (1.0 - lks::fmul(kp, lks::ffma(bx, bx, lks::fmul(by, by))) / rho);
        ux = lks::ffma(lks::fmul(0.5, jz), by, jxp) / rho;
    } else {
        ux = lks::ffma(-0.5, Fx, jx) / rho;
    }
}

template <typename S, typename C, int COUPLING, bool INPLACE>
__global__ void __launch_bounds__(512) batch_kernel(InstDev* tab, const int32_t* work, const Ctl* ctl,
                                                     int32_t* counter, ResultDev* res, int T) {
    extern __shared__ double red[];
    __shared__ int32_t pick[16];
    __shared__ int32_t flag[16];
    const int gid = threadIdx.x / T;
    const int lt = threadIdx.x - gid * T;
    double* rd = red + (size_t)gid * 4 * (T >> 5);  // 4 sums per warp of the group
    const int nwork = ctl->nwork;
    const int64_t quantum = ctl->quantum;
    for (;;) {
        if (lt == 0) pick[gid] = atomicAdd(counter, 1);
        group_sync(gid, T);
        const int w = pick[gid];
        if (w >= nwork) break;
        const int slot = work[w];
        InstDev* I = tab + slot;
        const StepParams<C> p = to_compute<C>(I->pd);
        const int64_t N = p.N;
        const int closure = I->closure;
        const int64_t check_every = I->check_every, max_steps = I->max_steps;
        int cur = I->cur;
        int64_t steps = I->steps;
        int state = LKS_INST_RUNNING;
        // residual bookkeeping lives in thread lt == 0
        double r = I->residual, best = I->best_r;
        int stall = I->stall;
        for (int64_t s = 0; s < quantum; ++s) {
            if (INPLACE) {  // one buffer: phase (steps & 1) of an in-place pair (lks_aa.cuh)
                S* fb = (S*)I->f[0];
                S* gb = (S*)I->g[0];
                if ((steps & 1) == 0) {
                    if (closure == 0) {
                        for (lks::NodeWalker w(lt, T, p.nx); w.n < N; w.next(T))
                            lks::aa_node_pull_push<S, C, 0, COUPLING>(fb, gb, p, w.n, w.i, w.j);
                    } else {
                        for (lks::NodeWalker w(lt, T, p.nx); w.n < N; w.next(T))
                            lks::aa_node_pull_push<S, C, 1, COUPLING>(fb, gb, p, w.n, w.i, w.j);
                    }
                } else {
                    if (closure == 0) {
                        for (lks::NodeWalker w(lt, T, p.nx); w.n < N; w.next(T))
                            lks::aa_node_local<S, C, 0, COUPLING>(fb, gb, p, w.n, w.j);
                    } else {
                        for (lks::NodeWalker w(lt, T, p.nx); w.n < N; w.next(T))
                            lks::aa_node_local<S, C, 1, COUPLING>(fb, gb, p, w.n, w.j);
                    }
                }
            } else {
                const S* fi = (const S*)I->f[cur];
                const S* gi = (const S*)I->g[cur];
                S* fo = (S*)I->f[cur ^ 1];
                S* go = (S*)I->g[cur ^ 1];
                if (closure == 0) {
                    for (lks::NodeWalker w(lt, T, p.nx); w.n < N; w.next(T))
                        lks::step_node<S, C, 0, false, COUPLING>(fi, gi, fo, go, p, w.n, w.i, w.j);
                } else {
                    for (lks::NodeWalker w(lt, T, p.nx); w.n < N; w.next(T))
                        lks::step_node<S, C, 1, false, COUPLING>(fi, gi, fo, go, p, w.n, w.i, w.j);
                }
                cur ^= 1;
            }
            ++steps;
            group_sync(gid, T);
            if (steps % check_every == 0 || steps >= max_steps) {
                double acc[4] = {0.0, 0.0, 0.0, 0.0};
                const S* fc = (const S*)I->f[cur];
                const S* gc = (const S*)I->g[cur];
                double* snap = I->snap;
                for (int64_t n = lt; n < N; n += T) {
                    double ux, bx;
                    stored_ux_bx<S, C, lks::Loader<S, C, false>, COUPLING>(fc, gc, N, n, I, ux, bx);
                    const double du = ux - snap[n], db = bx - snap[N + n];
                    acc[0] = lks::ffma(du, du, acc[0]);
                    acc[1] = lks::ffma(ux, ux, acc[1]);
                    acc[2] = lks::ffma(db, db, acc[2]);
                    acc[3] = lks::ffma(bx, bx, acc[3]);
                    snap[n] = ux;
                    snap[N + n] = bx;
                }
                // fixed-order reduction: shuffle tree within each warp, then lane 0 of the group
                // adds the T/32 warp sums in warp order
                lks::warp_sum<4>(acc);
                const int W = T >> 5;
                if ((lt & 31) == 0)
#pragma unroll
                    for (int k = 0; k < 4; ++k) rd[k * W + (lt >> 5)] = acc[k];
                group_sync(gid, T);
                if (lt == 0) {
                    double t[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        t[k] = rd[k * W];
                        for (int q = 1; q < W; ++q) t[k] += rd[k * W + q];
                    }
                    const double ru = t[1] > 1e-60 ? sqrt(t[0] / t[1]) : 0.0;
                    const double rb = t[3] > 1e-60 ? sqrt(t[2] / t[3]) : 0.0;
                    r = ru > rb ? ru : rb;
                    int st = LKS_INST_RUNNING;
                    if (!isfinite(r) || !isfinite(t[1]) || !isfinite(t[3])) {
                        st = LKS_INST_UNSTABLE;
                    } else if (r == 0.0 && sizeof(S) < 8 &&
                               (I->pd.Fx != 0.0 || I->pd.bot.U != 0.0 || I->pd.top.U != 0.0)) {
                        st = LKS_INST_STALLED;  // a driven channel that stopped changing (zero_residual_is_stall)
                    } else if (r < I->tol) {
                        st = LKS_INST_CONVERGED;
                    } else {
                        if (r < best) {
                            best = r;
                            stall = 0;
                        } else if (++stall >= kStallChecks && best < I->stall_below) {
                            st = LKS_INST_STALLED;
                        }
                        if (st == LKS_INST_RUNNING && steps >= max_steps) st = LKS_INST_MAX_STEPS;
                    }
                    flag[gid] = st;
                }
                group_sync(gid, T);
                state = flag[gid];
                if (state != LKS_INST_RUNNING) break;
            }
        }
        if (lt == 0) {
            I->cur = cur;
            I->steps = steps;
            I->state = state;
            I->residual = r;
            I->best_r = best;
            I->stall = stall;
            res[slot].state = state;
            res[slot].cur = cur;
            res[slot].steps = steps;
            res[slot].residual = r;
        }
        group_sync(gid, T);
    }
}

// Loads that bypass L1 (ld.global.cg): in cluster mode a node's neighbours may have been written
// by a CTA on another SM, whose stores L1 of this SM does not see.
template <typename S, typename C> struct CgLoader;
template <> struct CgLoader<double, double> {
    static __device__ __forceinline__ double ld(const double* p) { return __ldcg(p); }
};
template <> struct CgLoader<float, float> {
    static __device__ __forceinline__ float ld(const float* p) { return __ldcg(p); }
};
template <> struct CgLoader<__nv_bfloat16, float> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) {
        return __bfloat162float(__ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short*>(p))));
    }
};
template <> struct CgLoader<__half, float> {
    static __device__ __forceinline__ float ld(const __half* p) {
        return __fmul_rn(__half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short*>(p)))),
                         lks::kHalfUnscale);  // FP16 storage holds deviations times kHalfScale
    }
};

// Cluster mode: the CS CTAs of one thread-block cluster (on CS SMs) work on one instance together,
// CTA r updating nodes r*T + t, r*T + t + CS*T, ...; one cluster barrier (release/acquire at cluster
// scope) separates the steps, and the residual partials of the CTAs are summed by CTA 0 in rank
// order through distributed shared memory.  Large instances then advance CS times faster per step
// than with one CTA.
template <typename S, typename C, int COUPLING, bool INPLACE>
__global__ void __launch_bounds__(512) batch_cluster_kernel(InstDev* tab, const int32_t* work, const Ctl* ctl,
                                                             int32_t* counter, ResultDev* res, int T) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double red[];
    __shared__ int32_t pick;
    __shared__ int32_t flag;
    __shared__ double cpart[4 * 8];
    const int CS = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int lt = threadIdx.x;
    const int nwork = ctl->nwork;
    const int64_t quantum = ctl->quantum;
    int32_t* pick0 = cl.map_shared_rank(&pick, 0);
    int32_t* flag0 = cl.map_shared_rank(&flag, 0);
    double* cpart0 = cl.map_shared_rank(cpart, 0);
    const int64_t stride = (int64_t)CS * T;
    for (;;) {
        if (rank == 0 && lt == 0) pick = atomicAdd(counter, 1);
        cl.sync();
        const int w = *pick0;
        // Every CTA must have read CTA 0's shared `pick` before CTA 0 can overwrite it or exit
        // (reading the shared memory of a CTA that has exited is an invalid access).
        cl.sync();
        if (w >= nwork) break;
        const int slot = work[w];
        InstDev* I = tab + slot;
        const StepParams<C> p = to_compute<C>(I->pd);
        const int64_t N = p.N;
        const int closure = I->closure;
        const int64_t check_every = I->check_every, max_steps = I->max_steps;
        int cur = I->cur;
        int64_t steps = I->steps;
        int state = LKS_INST_RUNNING;
        double r = I->residual, best = I->best_r;
        int stall = I->stall;
        const int64_t first = (int64_t)rank * T + lt;
        for (int64_t s = 0; s < quantum; ++s) {
            if (INPLACE) {
                S* fb = (S*)I->f[0];
                S* gb = (S*)I->g[0];
                if ((steps & 1) == 0) {
                    if (closure == 0) {
                        for (lks::NodeWalker w(first, stride, p.nx); w.n < N; w.next(stride))
                            lks::aa_node_pull_push<S, C, 0, COUPLING, CgLoader<S, C>>(fb, gb, p, w.n, w.i, w.j);
                    } else {
                        for (lks::NodeWalker w(first, stride, p.nx); w.n < N; w.next(stride))
                            lks::aa_node_pull_push<S, C, 1, COUPLING, CgLoader<S, C>>(fb, gb, p, w.n, w.i, w.j);
                    }
                } else {
                    if (closure == 0) {
                        for (lks::NodeWalker w(first, stride, p.nx); w.n < N; w.next(stride))
                            lks::aa_node_local<S, C, 0, COUPLING, CgLoader<S, C>>(fb, gb, p, w.n, w.j);
                    } else {
                        for (lks::NodeWalker w(first, stride, p.nx); w.n < N; w.next(stride))
                            lks::aa_node_local<S, C, 1, COUPLING, CgLoader<S, C>>(fb, gb, p, w.n, w.j);
                    }
                }
            } else {
                const S* fi = (const S*)I->f[cur];
                const S* gi = (const S*)I->g[cur];
                S* fo = (S*)I->f[cur ^ 1];
                S* go = (S*)I->g[cur ^ 1];
                if (closure == 0) {
                    for (lks::NodeWalker w(first, stride, p.nx); w.n < N; w.next(stride))
                        lks::step_node_with<S, C, 0, CgLoader<S, C>, COUPLING>(fi, gi, fo, go, p, w.n, w.i, w.j);
                } else {
                    for (lks::NodeWalker w(first, stride, p.nx); w.n < N; w.next(stride))
                        lks::step_node_with<S, C, 1, CgLoader<S, C>, COUPLING>(fi, gi, fo, go, p, w.n, w.i, w.j);
                }
                cur ^= 1;
            }
            ++steps;
            cl.sync();
            if (steps % check_every == 0 || steps >= max_steps) {
                double acc[4] = {0.0, 0.0, 0.0, 0.0};
                const S* fc = (const S*)I->f[cur];
                const S* gc = (const S*)I->g[cur];
                double* snap = I->snap;
                for (int64_t n = first; n < N; n += stride) {
                    double ux, bx;
                    stored_ux_bx<S, C, CgLoader<S, C>, COUPLING>(fc, gc, N, n, I, ux, bx);
                    const double du = ux - snap[n], db = bx - snap[N + n];
                    acc[0] = lks::ffma(du, du, acc[0]);
                    acc[1] = lks::ffma(ux, ux, acc[1]);
                    acc[2] = lks::ffma(db, db, acc[2]);
                    acc[3] = lks::ffma(bx, bx, acc[3]);
                    snap[n] = ux;
                    snap[N + n] = bx;
                }
                lks::warp_sum<4>(acc);
                const int W = T >> 5;
                if ((lt & 31) == 0)
#pragma unroll
                    for (int k = 0; k < 4; ++k) red[k * W + (lt >> 5)] = acc[k];
                __syncthreads();
                if (lt == 0)
                    for (int k = 0; k < 4; ++k) {
                        double t = red[k * W];
                        for (int q = 1; q < W; ++q) t += red[k * W + q];
                        cpart0[4 * rank + k] = t;
                    }
                cl.sync();
                if (rank == 0 && lt == 0) {
                    double t[4] = {0.0, 0.0, 0.0, 0.0};
                    for (int q = 0; q < CS; ++q)
                        for (int k = 0; k < 4; ++k) t[k] += cpart[4 * q + k];
                    const double ru = t[1] > 1e-60 ? sqrt(t[0] / t[1]) : 0.0;
                    const double rb = t[3] > 1e-60 ? sqrt(t[2] / t[3]) : 0.0;
                    r = ru > rb ? ru : rb;
                    int st = LKS_INST_RUNNING;
                    if (!isfinite(r) || !isfinite(t[1]) || !isfinite(t[3])) {
                        st = LKS_INST_UNSTABLE;
                    } else if (r == 0.0 && sizeof(S) < 8 &&
                               (I->pd.Fx != 0.0 || I->pd.bot.U != 0.0 || I->pd.top.U != 0.0)) {
                        st = LKS_INST_STALLED;  // a driven channel that stopped changing (zero_residual_is_stall)
                    } else if (r < I->tol) {
                        st = LKS_INST_CONVERGED;
                    } else {
                        if (r < best) {
                            best = r;
                            stall = 0;
                        } else if (++stall >= kStallChecks && best < I->stall_below) {
                            st = LKS_INST_STALLED;
                        }
                        if (st == LKS_INST_RUNNING && steps >= max_steps) st = LKS_INST_MAX_STEPS;
                    }
                    flag = st;
                }
                cl.sync();
                // CTA 0 writes `flag` again only at the next check, after at least one more
                // cluster barrier, and leaves the kernel only after the next pick's barriers.
                state = *flag0;
                if (state != LKS_INST_RUNNING) break;
            }
        }
        if (rank == 0 && lt == 0) {
            I->cur = cur;
            I->steps = steps;
            I->state = state;
            I->residual = r;
            I->best_r = best;
            I->stall = stall;
            res[slot].state = state;
            res[slot].cur = cur;
            res[slot].steps = steps;
            res[slot].residual = r;
        }
        cl.sync();
    }
}

typedef void (*BatchClusterFn)(InstDev*, const int32_t*, const Ctl*, int32_t*, ResultDev*, int);

template <int COUPLING, bool INPLACE>
BatchClusterFn cluster_kernel_typed(int storage) {
    switch (storage) {
        case 0: return batch_cluster_kernel<double, double, COUPLING, INPLACE>;
        case 1: return batch_cluster_kernel<float, float, COUPLING, INPLACE>;
        case 2: return batch_cluster_kernel<__nv_bfloat16, float, COUPLING, INPLACE>;
        default: return batch_cluster_kernel<__half, float, COUPLING, INPLACE>;
    }
}

BatchClusterFn cluster_kernel_for(const lks_batch_config& c) {
    if (c.coupling == 1) return c.inplace ? cluster_kernel_typed<1, true>(c.storage) : cluster_kernel_typed<1, false>(c.storage);
    return c.inplace ? cluster_kernel_typed<0, true>(c.storage) : cluster_kernel_typed<0, false>(c.storage);
}

typedef void (*BatchKernelFn)(InstDev*, const int32_t*, const Ctl*, int32_t*, ResultDev*, int);

template <int COUPLING, bool INPLACE>
BatchKernelFn kernel_typed(int storage) {
    switch (storage) {
        case 0: return batch_kernel<double, double, COUPLING, INPLACE>;
        case 1: return batch_kernel<float, float, COUPLING, INPLACE>;
        case 2: return batch_kernel<__nv_bfloat16, float, COUPLING, INPLACE>;
        default: return batch_kernel<__half, float, COUPLING, INPLACE>;
    }
}

BatchKernelFn kernel_for(const lks_batch_config& c) {
    if (c.coupling == 1) return c.inplace ? kernel_typed<1, true>(c.storage) : kernel_typed<1, false>(c.storage);
    return c.inplace ? kernel_typed<0, true>(c.storage) : kernel_typed<0, false>(c.storage);
}

const char* validate_desc(const lks_instance_desc* d) {
    if (!d) return "instance description is NULL";
    if (d->nx < 1) return "nx must be >= 1";
    if (d->closure != LKS_LINK && d->closure != LKS_MOMENT) return "closure must be LKS_LINK or LKS_MOMENT";
    if (d->closure == LKS_LINK && d->ny < 2) return "ny must be >= 2 for the link-based closure";
    if (d->closure == LKS_MOMENT && d->ny < 3) return "ny must be >= 3 for the moment-based closure";
    if ((int64_t)d->nx * d->ny > (int64_t)1 << 28) return "instance exceeds 2^28 nodes";
    if (!(d->tau_f > 0.5) || !isfinite(d->tau_f) || !(d->tau_m > 0.5) || !isfinite(d->tau_m))
        return "tau_f and tau_m must be finite and > 1/2";
    if (!isfinite(d->B0) || !isfinite(d->Fx)) return "B0 and Fx must be finite";
    if (!(d->c_bottom >= 0.0) || !(d->c_top >= 0.0)) return "wall conductance ratios must be >= 0";
    if (!(fabs(d->u_bottom) < 0.3) || !(fabs(d->u_top) < 0.3)) return "|wall speed| must be < 0.3";
    if (!isfinite(d->perturb_amp) || fabs(d->perturb_amp) >= 0.3) return "|perturb_amp| must be < 0.3";
    if (!(d->tol > 0.0) || d->check_every < 1 || d->max_steps < 1) return "tol > 0, check_every >= 1, max_steps >= 1";
    if (d->coupling != LKS_MAXWELL && d->coupling != LKS_LORENTZ) return "coupling must be LKS_MAXWELL or LKS_LORENTZ";
    if (d->coupling == LKS_LORENTZ && fabs(d->tau_m - 1.0) < 0.05)
        return "the Lorentz-force coupling needs |tau_m - 1| >= 0.05";
    return nullptr;
}

size_t inst_bytes(int nx, int ny, int storage, int inplace) {
    const size_t N = (size_t)nx * ny;
    const size_t sb = lks::storage_bytes(storage);
    const size_t nbuf = inplace ? 1 : 2;
    return nbuf * (align_up(9 * N * sb) + align_up(10 * N * sb)) + align_up(2 * N * sizeof(double));
}

bool valid_shape(int T, int G, int CS) {
    if (T < 32 || T > 512 || (T & (T - 1)) != 0) return false;
    if (G < 1 || G > kMaxGroups || T * G > 512) return false;
    if (CS != 1 && CS != 2 && CS != 4 && CS != 8) return false;
    if (CS > 1 && G != 1) return false;
    return true;
}

struct Slot {
    bool used = false;
    size_t offset = 0, bytes = 0;
    int nx = 0, ny = 0;
};

}  // namespace

struct lks_batch {
    lks_batch_config cfg;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int device = 0, nsm = 0;
    char* pool = nullptr;
    bool owns = false;
    std::map<size_t, size_t> free_list;  // offset -> bytes
    size_t used_bytes = 0;
    std::vector<Slot> slots;
    InstDev* d_tab = nullptr;
    ResultDev* d_res = nullptr;
    ResultDev* h_res = nullptr;  // pinned mirror of d_res
    int32_t* d_work = nullptr;
    int32_t* h_work = nullptr;   // pinned
    Ctl* d_ctl = nullptr;
    Ctl* h_ctl = nullptr;        // pinned
    int32_t* d_counter = nullptr;
    int T = 256, G = 1, CS = 1;
    cudaGraphExec_t graph = nullptr;
    int graph_T = 0, graph_G = 0, graph_CS = 0;
    std::string err;
};

namespace {

thread_local std::string g_batch_error;

lks_status bfail(lks_batch* b, lks_status s, const std::string& m) {
    if (b)
        b->err = m;
    else
        g_batch_error = m;
    return s;
}

lks_status bcuda(lks_batch* b, cudaError_t e, const char* where) {
    return bfail(b, LKS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool pool_alloc(lks_batch* b, size_t bytes, size_t* off) {
    for (auto it = b->free_list.begin(); it != b->free_list.end(); ++it) {
        if (it->second >= bytes) {
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t roff = it->first + bytes;
            b->free_list.erase(it);
            if (rest) b->free_list[roff] = rest;
            b->used_bytes += bytes;
            return true;
        }
    }
    return false;
}

void pool_free(lks_batch* b, size_t off, size_t bytes) {
    b->used_bytes -= bytes;
    auto it = b->free_list.emplace(off, bytes).first;
    // merge with the next block
    auto nx = std::next(it);
    if (nx != b->free_list.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        b->free_list.erase(nx);
    }
    // merge with the previous block
    if (it != b->free_list.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            b->free_list.erase(it);
        }
    }
}

int blocks_per_sm(lks_batch* b, int T, int G) {
    int nb = 0;
    const size_t smem = (size_t)G * 4 * (T / 32) * sizeof(double);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_for(b->cfg), T * G, smem);
    return nb > 0 ? nb : 1;
}

cudaError_t enqueue_launch(lks_batch* b, cudaStream_t st) {
    const int T = b->T, G = b->G, CS = b->CS;
    const size_t smem = (size_t)G * 4 * (T / 32) * sizeof(double);
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    if (CS == 1) {
        const int grid = blocks_per_sm(b, T, G) * b->nsm;
        kernel_for(b->cfg)<<<grid, T * G, smem, st>>>(b->d_tab, b->d_work, b->d_ctl, b->d_counter, b->d_res,
                                                              T);
    } else {
        cudaLaunchConfig_t lc = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        lc.blockDim = dim3(T);
        lc.dynamicSmemBytes = smem;
        lc.stream = st;
        lc.attrs = attr;
        lc.numAttrs = 1;
        lc.gridDim = dim3(CS * b->nsm);
        int clusters = 0;
        e = cudaOccupancyMaxActiveClusters(&clusters, cluster_kernel_for(b->cfg), &lc);
        if (e != cudaSuccess) return e;
        if (clusters < 1) clusters = 1;
        lc.gridDim = dim3(clusters * CS);
        e = cudaLaunchKernelEx(&lc, cluster_kernel_for(b->cfg), b->d_tab, (const int32_t*)b->d_work,
                               (const Ctl*)b->d_ctl, b->d_counter, b->d_res, T);
        if (e != cudaSuccess) return e;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(b->h_res, b->d_res, b->slots.size() * sizeof(ResultDev), cudaMemcpyDeviceToHost, st);
}

cudaError_t ensure_graph(lks_batch* b) {
    if (b->graph && b->graph_T == b->T && b->graph_G == b->G && b->graph_CS == b->CS) return cudaSuccess;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    const size_t smem = (size_t)b->G * 4 * (b->T / 32) * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel_for(b->cfg), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = enqueue_launch(b, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e == cudaSuccess) {
        b->graph_T = b->T;
        b->graph_G = b->G;
        b->graph_CS = b->CS;
    }
    return e;
}

}  // namespace

extern "C" {

size_t lks_instance_footprint_bytes(const lks_instance_desc* d, int32_t storage, int32_t inplace) {
    if (validate_desc(d) || storage < LKS_F64 || storage > LKS_F16_DEV || (inplace != 0 && inplace != 1)) return 0;
    if (inplace && ((d->check_every & 1) || (d->max_steps & 1))) return 0;
    return inst_bytes(d->nx, d->ny, storage, inplace);
}

lks_status lks_batch_create(const lks_batch_config* cfg, lks_batch** out) {
    if (!out) return bfail(nullptr, LKS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return bfail(nullptr, LKS_EINVAL, "config is NULL");
    if (cfg->storage < LKS_F64 || cfg->storage > LKS_F16_DEV) return bfail(nullptr, LKS_EINVAL, "bad storage");
    if (cfg->coupling != LKS_MAXWELL && cfg->coupling != LKS_LORENTZ) return bfail(nullptr, LKS_EINVAL, "bad coupling");
    if (cfg->inplace != 0 && cfg->inplace != 1) return bfail(nullptr, LKS_EINVAL, "inplace must be 0 or 1");
    if (cfg->max_instances < 1 || cfg->max_instances > (1 << 24)) return bfail(nullptr, LKS_EINVAL, "bad max_instances");
    if (cfg->pool_bytes < kAlign) return bfail(nullptr, LKS_EINVAL, "pool_bytes too small");
    const int T = cfg->threads_per_group ? cfg->threads_per_group : 256;
    const int G = cfg->groups_per_cta ? cfg->groups_per_cta : 1;
    const int CS = cfg->cluster_ctas ? cfg->cluster_ctas : 1;
    if (!valid_shape(T, G, CS))
        return bfail(nullptr, LKS_EINVAL,
                     "threads_per_group must be a power of two in [32,512], groups 1..15, product <= 512, "
                     "cluster_ctas 1/2/4/8 (groups 1 when > 1)");
    lks_batch* b = new (std::nothrow) lks_batch();
    if (!b) return bfail(nullptr, LKS_ENOMEM, "host allocation failed");
    b->cfg = *cfg;
    b->T = T;
    b->G = G;
    b->CS = CS;
    b->stream = (cudaStream_t)cfg->cuda_stream;
    b->slots.resize(cfg->max_instances);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) {
        delete b;
        return bcuda(nullptr, e, "lks_batch_create");
    }
    const size_t pool = cfg->pool_bytes & ~(kAlign - 1);
    if (cfg->dev_buffer) {
        if (cfg->dev_buffer_bytes < pool || ((uintptr_t)cfg->dev_buffer % kAlign) != 0) {
            delete b;
            return bfail(nullptr, LKS_ENOMEM, "dev_buffer smaller than pool_bytes or not 256-byte aligned");
        }
        b->pool = (char*)cfg->dev_buffer;
    } else {
        e = cudaMalloc((void**)&b->pool, pool);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return bfail(nullptr, LKS_ENOMEM, std::string("cudaMalloc of the pool: ") + cudaGetErrorString(e));
        }
        b->owns = true;
    }
    b->free_list[0] = pool;
    const size_t M = cfg->max_instances;
    e = cudaMalloc((void**)&b->d_tab, M * sizeof(InstDev));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_res, M * sizeof(ResultDev));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_work, M * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_ctl, sizeof(Ctl));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_counter, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&b->h_res, M * sizeof(ResultDev), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&b->h_work, M * sizeof(int32_t), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&b->h_ctl, sizeof(Ctl), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        lks_batch_destroy(b);
        return bfail(nullptr, LKS_ENOMEM, std::string("lks_batch_create: ") + cudaGetErrorString(e));
    }
    for (size_t k = 0; k < M; ++k) {
        b->h_res[k].state = LKS_INST_FREE;
        b->h_res[k].cur = 0;
        b->h_res[k].steps = 0;
        b->h_res[k].residual = INFINITY;
    }
    e = cudaMemcpyAsync(b->d_res, b->h_res, M * sizeof(ResultDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        lks_batch_destroy(b);
        return bcuda(nullptr, e, "lks_batch_create");
    }
    *out = b;
    return LKS_OK;
}

lks_status lks_batch_add(lks_batch* b, const lks_instance_desc* d, int32_t* slot_out) {
    if (!b) return bfail(nullptr, LKS_EINVAL, "batch is NULL");
    if (const char* m = validate_desc(d)) return bfail(b, LKS_EINVAL, m);
    if (d->coupling != b->cfg.coupling) return bfail(b, LKS_EINVAL, "instance coupling differs from the batch's");
    if (b->cfg.inplace && ((d->check_every & 1) || (d->max_steps & 1)))
        return bfail(b, LKS_EINVAL, "an in-place batch steps in pairs: check_every and max_steps must be even");
    int slot = -1;
    for (size_t k = 0; k < b->slots.size(); ++k)
        if (!b->slots[k].used) {
            slot = (int)k;
            break;
        }
    if (slot < 0) return bfail(b, LKS_EBUSY, "no free slot");
    const size_t bytes = inst_bytes(d->nx, d->ny, b->cfg.storage, b->cfg.inplace);
    size_t off = 0;
    if (!pool_alloc(b, bytes, &off)) return bfail(b, LKS_EBUSY, "not enough free pool memory");
    Slot& s = b->slots[slot];
    s.used = true;
    s.offset = off;
    s.bytes = bytes;
    s.nx = d->nx;
    s.ny = d->ny;
    const size_t N = (size_t)d->nx * d->ny;
    const size_t sb = lks::storage_bytes(b->cfg.storage);
    InstDev I;
    memset(&I, 0, sizeof(I));
    I.pd = lks::make_step_params(d->nx, d->ny, d->closure, d->tau_f, d->tau_m, d->B0, d->Fx, d->c_bottom, d->c_top,
                                 d->u_bottom, d->u_top, d->coupling);
    char* base = b->pool + off;
    I.f[0] = base;
    I.g[0] = base + align_up(9 * N * sb);
    if (b->cfg.inplace) {  // one population buffer
        I.f[1] = I.f[0];
        I.g[1] = I.g[0];
        I.snap = (double*)(I.g[0] + align_up(10 * N * sb));
    } else {
        I.f[1] = I.g[0] + align_up(10 * N * sb);
        I.g[1] = I.f[1] + align_up(9 * N * sb);
        I.snap = (double*)(I.g[1] + align_up(10 * N * sb));
    }
    I.steps = 0;
    I.check_every = d->check_every;
    I.max_steps = d->max_steps;
    I.tol = d->tol;
    I.stall_below = stall_floor(b->cfg.storage);
    I.tau_m = d->tau_m;
    I.best_r = INFINITY;
    I.residual = INFINITY;
    I.closure = d->closure;
    I.cur = 0;
    I.state = LKS_INST_RUNNING;
    I.stall = 0;
    b->h_res[slot].state = LKS_INST_RUNNING;
    b->h_res[slot].cur = 0;
    b->h_res[slot].steps = 0;
    b->h_res[slot].residual = INFINITY;
    cudaError_t e = cudaMemcpyAsync(b->d_tab + slot, &I, sizeof(InstDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_res + slot, &b->h_res[slot], sizeof(ResultDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = lks::launch_init(b->cfg.storage, I.f[0], I.g[0], d->nx, d->ny, d->B0, d->seed, d->perturb_amp, b->stream);
    if (e == cudaSuccess)
        e = lks::launch_snapshot(b->cfg.storage, I.f[0], I.g[0], d->nx, d->ny, d->B0, d->Fx, I.snap, b->stream,
                                 d->coupling, d->tau_m);
    // the host copy of I is on the stack: make sure the copies have consumed it
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        pool_free(b, off, bytes);
        s.used = false;
        b->h_res[slot].state = LKS_INST_FREE;
        return bcuda(b, e, "lks_batch_add");
    }
    if (slot_out) *slot_out = slot;
    return LKS_OK;
}

lks_status lks_batch_run(lks_batch* b, int64_t quantum, int32_t* n_running) {
    if (!b) return bfail(nullptr, LKS_EINVAL, "batch is NULL");
    nvtxRangePushA("lks_batch_run");
    struct Pop {
        ~Pop() { nvtxRangePop(); }
    } pop;
    if (quantum < 1) return bfail(b, LKS_EINVAL, "quantum_steps must be >= 1");
    if (b->cfg.inplace && (quantum & 1)) return bfail(b, LKS_EINVAL, "an in-place batch steps in pairs: quantum must be even");
    int nwork = 0;
    for (size_t k = 0; k < b->slots.size(); ++k)
        if (b->slots[k].used && b->h_res[k].state == LKS_INST_RUNNING) b->h_work[nwork++] = (int32_t)k;
    if (nwork > 0) {
        b->h_ctl->nwork = nwork;
        b->h_ctl->pad = 0;
        b->h_ctl->quantum = quantum;
        cudaError_t e = ensure_graph(b);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_work, b->h_work, nwork * sizeof(int32_t), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_ctl, b->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "lks_batch_run");
    }
    int running = 0;
    for (size_t k = 0; k < b->slots.size(); ++k)
        if (b->slots[k].used && b->h_res[k].state == LKS_INST_RUNNING) ++running;
    if (n_running) *n_running = running;
    return LKS_OK;
}

lks_status lks_batch_result(const lks_batch* b, int32_t slot, lks_instance_result* out) {
    if (!b || !out) return bfail(nullptr, LKS_EINVAL, "NULL argument");
    if (slot < 0 || slot >= (int32_t)b->slots.size()) return bfail(const_cast<lks_batch*>(b), LKS_EINVAL, "bad slot");
    if (!b->slots[slot].used) {
        out->state = LKS_INST_FREE;
        out->pad = 0;
        out->steps = 0;
        out->residual = INFINITY;
        return LKS_OK;
    }
    const ResultDev& r = b->h_res[slot];
    out->state = r.state;
    out->pad = 0;
    out->steps = r.steps;
    out->residual = r.residual;
    return LKS_OK;
}

lks_status lks_batch_moments(lks_batch* b, int32_t slot, int what, double* host_out) {
    if (!b) return bfail(nullptr, LKS_EINVAL, "batch is NULL");
    if (slot < 0 || slot >= (int32_t)b->slots.size() || !b->slots[slot].used) return bfail(b, LKS_EINVAL, "bad slot");
    if (!host_out || (what != LKS_MOMENTS_NODES && what != LKS_MOMENTS_PROFILES)) return bfail(b, LKS_EINVAL, "bad args");
    InstDev I;
    cudaError_t e = cudaMemcpyAsync(&I, b->d_tab + slot, sizeof(InstDev), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "lks_batch_moments");
    const Slot& s = b->slots[slot];
    const size_t count = (what == LKS_MOMENTS_NODES ? (size_t)s.nx * s.ny : (size_t)s.ny) * 5;
    double* dtmp = nullptr;
    e = cudaMalloc((void**)&dtmp, count * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, LKS_ENOMEM, "cudaMalloc of the moment staging buffer failed");
    }
    e = lks::launch_moments(b->cfg.storage, I.f[I.cur], I.g[I.cur], s.nx, s.ny, I.pd.B0, I.pd.Fx, what, dtmp,
                            b->stream, I.pd.coupling, I.tau_m);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, dtmp, count * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(dtmp);
    if (e != cudaSuccess) return bcuda(b, e, "lks_batch_moments");
    return LKS_OK;
}

lks_status lks_batch_get_state(lks_batch* b, int32_t slot, double* host_f, double* host_g) {
    if (!b) return bfail(nullptr, LKS_EINVAL, "batch is NULL");
    if (slot < 0 || slot >= (int32_t)b->slots.size() || !b->slots[slot].used) return bfail(b, LKS_EINVAL, "bad slot");
    if (!host_f || !host_g) return bfail(b, LKS_EINVAL, "host_f/host_g is NULL");
    InstDev I;
    cudaError_t e = cudaMemcpyAsync(&I, b->d_tab + slot, sizeof(InstDev), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "lks_batch_get_state");
    const Slot& s = b->slots[slot];
    const int64_t N = (int64_t)s.nx * s.ny;
    double* dtmp = nullptr;
    e = cudaMalloc((void**)&dtmp, 19 * (size_t)N * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, LKS_ENOMEM, "cudaMalloc of the state staging buffer failed");
    }
    e = lks::launch_to_abs(b->cfg.storage, I.f[I.cur], I.g[I.cur], N, 0, N, I.pd.B0, dtmp, dtmp + 9 * N, b->stream,
                           I.pd.coupling);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_f, dtmp, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_g, dtmp + 9 * N, 10 * N * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(dtmp);
    if (e != cudaSuccess) return bcuda(b, e, "lks_batch_get_state");
    return LKS_OK;
}

lks_status lks_batch_set_state(lks_batch* b, int32_t slot, const double* host_f, const double* host_g) {
    if (!b) return bfail(nullptr, LKS_EINVAL, "batch is NULL");
    if (slot < 0 || slot >= (int32_t)b->slots.size() || !b->slots[slot].used) return bfail(b, LKS_EINVAL, "bad slot");
    if (!host_f || !host_g) return bfail(b, LKS_EINVAL, "host_f/host_g is NULL");
    InstDev I;
    cudaError_t e = cudaMemcpyAsync(&I, b->d_tab + slot, sizeof(InstDev), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "lks_batch_set_state");
    const Slot& s = b->slots[slot];
    const int64_t N = (int64_t)s.nx * s.ny;
    double* dtmp = nullptr;
    e = cudaMalloc((void**)&dtmp, 19 * (size_t)N * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, LKS_ENOMEM, "cudaMalloc of the state staging buffer failed");
    }
    e = cudaMemcpyAsync(dtmp, host_f, 9 * N * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtmp + 9 * N, host_g, 10 * N * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = lks::launch_from_abs(b->cfg.storage, dtmp, dtmp + 9 * N, N, 0, N, I.pd.B0, I.f[I.cur], I.g[I.cur],
                                 b->stream, I.pd.coupling);
    if (e == cudaSuccess)
        e = lks::launch_snapshot(b->cfg.storage, I.f[I.cur], I.g[I.cur], s.nx, s.ny, I.pd.B0, I.pd.Fx, I.snap,
                                 b->stream, I.pd.coupling, I.tau_m);
    // a fresh start from the new state: step count, residual history and status reset
    I.steps = 0;
    I.state = LKS_INST_RUNNING;
    I.best_r = INFINITY;
    I.residual = INFINITY;
    I.stall = 0;
    b->h_res[slot].state = LKS_INST_RUNNING;
    b->h_res[slot].cur = I.cur;
    b->h_res[slot].steps = 0;
    b->h_res[slot].residual = INFINITY;
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_tab + slot, &I, sizeof(InstDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_res + slot, &b->h_res[slot], sizeof(ResultDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(dtmp);
    if (e != cudaSuccess) return bcuda(b, e, "lks_batch_set_state");
    return LKS_OK;
}

lks_status lks_batch_remove(lks_batch* b, int32_t slot) {
    if (!b) return bfail(nullptr, LKS_EINVAL, "batch is NULL");
    if (slot < 0 || slot >= (int32_t)b->slots.size() || !b->slots[slot].used) return bfail(b, LKS_EINVAL, "bad slot");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "lks_batch_remove");
    Slot& s = b->slots[slot];
    pool_free(b, s.offset, s.bytes);
    s.used = false;
    b->h_res[slot].state = LKS_INST_FREE;
    e = cudaMemcpyAsync(b->d_res + slot, &b->h_res[slot], sizeof(ResultDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "lks_batch_remove");
    return LKS_OK;
}

lks_status lks_batch_set_shape(lks_batch* b, int32_t T, int32_t G, int32_t CS) {
    if (!b) return bfail(nullptr, LKS_EINVAL, "batch is NULL");
    if (!valid_shape(T, G, CS)) return bfail(b, LKS_EINVAL, "invalid thread-group shape");
    b->T = T;
    b->G = G;
    b->CS = CS;
    return LKS_OK;
}

lks_status lks_batch_autotune(lks_batch* b, int64_t probe_steps, const int32_t* Ts, const int32_t* Gs,
                              const int32_t* Cs, int32_t n, double* seconds_out, int32_t* best_index) {
    if (!b) return bfail(nullptr, LKS_EINVAL, "batch is NULL");
    if (!Ts || !Gs || !Cs || n < 1 || probe_steps < 1) return bfail(b, LKS_EINVAL, "bad autotune arguments");
    for (int k = 0; k < n; ++k)
        if (!valid_shape(Ts[k], Gs[k], Cs[k])) return bfail(b, LKS_EINVAL, "invalid candidate shape");
    // save every used instance's state, the table and the results
    const size_t M = b->slots.size();
    size_t total = 0;
    for (size_t k = 0; k < M; ++k)
        if (b->slots[k].used) total += b->slots[k].bytes;
    char* save = nullptr;
    InstDev* save_tab = nullptr;
    ResultDev* save_res = nullptr;
    std::vector<ResultDev> host_res(b->h_res, b->h_res + M);
    cudaError_t e = cudaMalloc((void**)&save, total ? total : kAlign);
    if (e == cudaSuccess) e = cudaMalloc((void**)&save_tab, M * sizeof(InstDev));
    if (e == cudaSuccess) e = cudaMalloc((void**)&save_res, M * sizeof(ResultDev));
    auto copy_states = [&](bool to_save) -> cudaError_t {
        size_t o = 0;
        cudaError_t ce = cudaSuccess;
        for (size_t k = 0; k < M && ce == cudaSuccess; ++k) {
            if (!b->slots[k].used) continue;
            char* pool_p = b->pool + b->slots[k].offset;
            ce = to_save ? cudaMemcpyAsync(save + o, pool_p, b->slots[k].bytes, cudaMemcpyDeviceToDevice, b->stream)
                         : cudaMemcpyAsync(pool_p, save + o, b->slots[k].bytes, cudaMemcpyDeviceToDevice, b->stream);
            o += b->slots[k].bytes;
        }
        if (ce == cudaSuccess)
            ce = to_save ? cudaMemcpyAsync(save_tab, b->d_tab, M * sizeof(InstDev), cudaMemcpyDeviceToDevice, b->stream)
                         : cudaMemcpyAsync(b->d_tab, save_tab, M * sizeof(InstDev), cudaMemcpyDeviceToDevice, b->stream);
        if (ce == cudaSuccess)
            ce = to_save ? cudaMemcpyAsync(save_res, b->d_res, M * sizeof(ResultDev), cudaMemcpyDeviceToDevice, b->stream)
                         : cudaMemcpyAsync(b->d_res, save_res, M * sizeof(ResultDev), cudaMemcpyDeviceToDevice, b->stream);
        return ce;
    };
    if (e == cudaSuccess) e = copy_states(true);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int T0 = b->T, G0 = b->G, C0 = b->CS;
    int best = -1;
    double best_t = INFINITY;
    lks_status st = LKS_OK;
    for (int k = 0; k < n && e == cudaSuccess && st == LKS_OK; ++k) {
        b->T = Ts[k];
        b->G = Gs[k];
        b->CS = Cs[k];
        e = cudaEventRecord(e0, b->stream);
        if (e != cudaSuccess) break;
        st = lks_batch_run(b, probe_steps, nullptr);
        if (st != LKS_OK) break;
        e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (seconds_out) seconds_out[k] = ms / 1e3;
        if (ms / 1e3 < best_t) {
            best_t = ms / 1e3;
            best = k;
        }
        // restore the states and the host view of the results
        if (e == cudaSuccess) e = copy_states(false);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        std::copy(host_res.begin(), host_res.end(), b->h_res);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save);
    cudaFree(save_tab);
    cudaFree(save_res);
    if (st != LKS_OK || e != cudaSuccess || best < 0) {
        b->T = T0;
        b->G = G0;
        b->CS = C0;
        if (st != LKS_OK) return st;
        return bcuda(b, e == cudaSuccess ? cudaErrorUnknown : e, "lks_batch_autotune");
    }
    b->T = Ts[best];
    b->G = Gs[best];
    b->CS = Cs[best];
    if (best_index) *best_index = best;
    return LKS_OK;
}

lks_status lks_batch_memory(const lks_batch* b, size_t* free_bytes, size_t* used_bytes) {
    if (!b) return bfail(nullptr, LKS_EINVAL, "batch is NULL");
    size_t fr = 0;
    for (const auto& kv : b->free_list) fr += kv.second;
    if (free_bytes) *free_bytes = fr;
    if (used_bytes) *used_bytes = b->used_bytes;
    return LKS_OK;
}

lks_status lks_batch_destroy(lks_batch* b) {
    if (!b) return LKS_OK;
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->owns && b->pool) cudaFree(b->pool);
    cudaFree(b->d_tab);
    cudaFree(b->d_res);
    cudaFree(b->d_work);
    cudaFree(b->d_ctl);
    cudaFree(b->d_counter);
    if (b->h_res) cudaFreeHost(b->h_res);
    if (b->h_work) cudaFreeHost(b->h_work);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    return LKS_OK;
}

const char* lks_batch_last_error(const lks_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

}  // extern "C"
