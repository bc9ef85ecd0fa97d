// lks_step_aa.cu -- kernels of the in-place (one-buffer) step; the per-node work and the proof
// that it reproduces the two-buffer step are in lks_aa.cuh.  Same thread layout as the two-buffer
// kernel: consecutive x positions in consecutive threads, a 2D grid (row = blockIdx.y) for wide
// FP32 / 16-bit lattices and a 1D grid otherwise.
#include "lks_aa.cuh"
#include "lks_internal.h"
#include "lks_packed.cuh"

namespace lks {

template <typename S, typename C, int CLOSURE, int COUPLING, int PHASE, bool ROWS2D>
__global__ void __launch_bounds__(256) step_kernel_aa(S* fb, S* gb, const StepParams<C> p) {
    int i, j;
    if (ROWS2D) {
        i = blockIdx.x * blockDim.x + threadIdx.x;
        j = blockIdx.y;
        if (i >= p.nx) return;
    } else {
        const unsigned n32 = blockIdx.x * blockDim.x + threadIdx.x;
        if ((int64_t)n32 >= p.N) return;
        j = (int)(n32 / (unsigned)p.nx);
        i = (int)(n32 - (unsigned)j * (unsigned)p.nx);
    }
    const int64_t n = (int64_t)j * p.nx + i;
    if (PHASE == 0)
        aa_node_pull_push<S, C, CLOSURE, COUPLING>(fb, gb, p, n, i, j);
    else
        aa_node_local<S, C, CLOSURE, COUPLING>(fb, gb, p, n, j);
}

// 16-bit storage, two nodes (x0, x0 + 1) per thread and one 32-bit word per population plane (nx
// even), as the two-buffer pair kernel.  Phase 1 touches only the thread's own words.  Phase 0
// pulls exactly as the pair kernel does and pushes every population into the opposite-direction
// plane of its target node: pushes that stay in the column are whole words; a push to x + 1 fills
// the word (x0, x0 + 1) with (left lane's node x0 - 1, own node x0) through a warp shuffle, a push
// to x - 1 fills it with (own node x0 + 1, right lane's node x0 + 2); at a warp or row edge the lane
// writes only its own half and the edge lane of the neighbouring pair the other one, as 16-bit
// stores.  All shuffles run on all 32 lanes (lanes past the end on a clamped pair, stores masked),
// also where a warp spans two rows.  Each element is written by one thread, after the thread
// that reads it (itself, or through a shuffle fed by its loads) has read it.
template <typename S, int CLOSURE, int COUPLING, int PHASE, bool ROWS2D>
__global__ void __launch_bounds__(256, PHASE == 0 ? 3 : 4) step_kernel_aa_pair(S* fb, S* gb, const StepParams<float> p) {
    typedef Packed<S> P;
    const unsigned FULL = 0xffffffffu;
    const int nx = p.nx, npr = nx >> 1;
    const int64_t N = p.N, NP = N >> 1;
    const int lane = threadIdx.x & 31;
    int j, ip;
    bool active;
    if (ROWS2D) {
        const int ip0 = blockIdx.x * blockDim.x + threadIdx.x;
        active = ip0 < npr;
        ip = active ? ip0 : npr - 1;
        j = blockIdx.y;
    } else {
        const unsigned q0 = blockIdx.x * blockDim.x + threadIdx.x;
        active = (int64_t)q0 < NP;
        const unsigned q1 = active ? q0 : (unsigned)(NP - 1);
        j = (int)(q1 / (unsigned)npr);
        ip = (int)(q1 - (unsigned)j * (unsigned)npr);
    }
    const int64_t q = (int64_t)j * npr + ip;
    const bool bottom = (j == 0), top = (j == p.ny - 1);
    uint32_t* fw = reinterpret_cast<uint32_t*>(fb);
    uint32_t* gxw = reinterpret_cast<uint32_t*>(gb);
    uint32_t* gyw = gxw + 5 * NP;
    float fA[9], fB[9], gxA[5], gxB[5], gyA[5], gyB[5];

    if (PHASE == 1) {
        if (!active) return;  // no shuffles in this phase
        // direction a of both nodes from plane abar of the own word
        auto own = [&](const uint32_t* base, int plane, bool valid, float& A, float& B) {
            const uint32_t w = valid ? base[plane * NP + q] : 0u;
            A = P::lo(w);
            B = P::hi(w);
        };
        const bool skip_up = CLOSURE == 1 && bottom, skip_down = CLOSURE == 1 && top;
        own(fw, 0, true, fA[0], fB[0]);
        own(fw, 3, true, fA[1], fB[1]);
        own(fw, 1, true, fA[3], fB[3]);
        own(fw, 4, !skip_up, fA[2], fB[2]);
        own(fw, 7, !skip_up, fA[5], fB[5]);
        own(fw, 8, !skip_up, fA[6], fB[6]);
        own(fw, 2, !skip_down, fA[4], fB[4]);
        own(fw, 5, !skip_down, fA[7], fB[7]);
        own(fw, 6, !skip_down, fA[8], fB[8]);
        own(gxw, 0, true, gxA[0], gxB[0]);
        own(gxw, 3, true, gxA[1], gxB[1]);
        own(gxw, 1, true, gxA[3], gxB[3]);
        own(gxw, 4, !skip_up, gxA[2], gxB[2]);
        own(gxw, 2, !skip_down, gxA[4], gxB[4]);
        own(gyw, 0, true, gyA[0], gyB[0]);
        own(gyw, 3, true, gyA[1], gyB[1]);
        own(gyw, 1, true, gyA[3], gyB[3]);
        own(gyw, 4, !skip_up, gyA[2], gyB[2]);
        own(gyw, 2, !skip_down, gyA[4], gyB[4]);
        if (CLOSURE == 0) {
            // the wall slots hold the node's own raw outgoing populations
            if (bottom) {
                const WallCoef<float>& w = p.bot;
                fA[5] = fA[5] + w.du; fB[5] = fB[5] + w.du;
                fA[6] = fA[6] - w.du; fB[6] = fB[6] - w.du;
                gxA[2] = ffma(w.r, gxA[2], w.kx); gxB[2] = ffma(w.r, gxB[2], w.kx);
                gyA[2] = -gyA[2]; gyB[2] = -gyB[2];
            }
            if (top) {
                const WallCoef<float>& w = p.top;
                fA[7] = fA[7] - w.du; fB[7] = fB[7] - w.du;
                fA[8] = fA[8] + w.du; fB[8] = fB[8] + w.du;
                gxA[4] = ffma(w.r, gxA[4], w.kx); gxB[4] = ffma(w.r, gxB[4], w.kx);
                gyA[4] = -gyA[4]; gyB[4] = -gyB[4];
            }
        } else {
            if (bottom) {
                moment_closure_bottom<float, COUPLING>(fA, gxA, gyA, p.bot, p);
                moment_closure_bottom<float, COUPLING>(fB, gxB, gyB, p.bot, p);
            }
            if (top) {
                moment_closure_top<float, COUPLING>(fA, gxA, gyA, p.top, p);
                moment_closure_top<float, COUPLING>(fB, gxB, gyB, p.top, p);
            }
        }
        collide<float, COUPLING>(fA, gxA, gyA, p);
        collide<float, COUPLING>(fB, gxB, gyB, p);
#pragma unroll
        for (int a = 0; a < 9; ++a) fw[a * NP + q] = P::pack(fA[a], fB[a]);
#pragma unroll
        for (int a = 0; a < 5; ++a) gxw[a * NP + q] = P::pack(gxA[a], gxB[a]);
#pragma unroll
        for (int a = 0; a < 5; ++a) gyw[a * NP + q] = P::pack(gyA[a], gyB[a]);
        return;
    }
    // ---- phase 0: pull (as the two-buffer pair kernel, coherent loads), close, collide ----
    const int x0 = ip << 1;
    const int64_t rc = (int64_t)j * npr, rs = rc - npr, rn = rc + npr;   // pair-row starts
    const int64_t ec = (int64_t)j * nx, es = ec - nx, en = ec + nx;      // element-row starts
    const bool left_edge = (lane == 0) || (ip == 0);
    const bool right_edge = (lane == 31) || (ip == npr - 1);
    const int xm = (x0 == 0) ? nx - 1 : x0 - 1;   // element left of the pair (periodic)
    const int xp = (x0 + 2 == nx) ? 0 : x0 + 2;   // element right of the pair (periodic)
    S* gxs = gb;
    S* gys = gb + 5 * N;
    auto Wd = [&](const uint32_t* base, int a, int64_t r) -> uint32_t { return base[a * NP + r + ip]; };
    auto Ed = [&](const S* base, int a, int64_t re, int x) -> float {
        return Loader<S, float, false>::ld(base + a * N + re + x);
    };
    auto pull_left = [&](const uint32_t* base, const S* ebase, int a, int64_t r, int64_t re, bool valid, float& A,
                         float& B) {
        const uint32_t w = valid ? Wd(base, a, r) : 0u;
        const uint32_t wl = __shfl_up_sync(FULL, w, 1);
        B = P::lo(w);
        A = P::hi(wl);
        if (valid && left_edge) A = Ed(ebase, a, re, xm);
    };
    auto pull_right = [&](const uint32_t* base, const S* ebase, int a, int64_t r, int64_t re, bool valid, float& A,
                          float& B) {
        const uint32_t w = valid ? Wd(base, a, r) : 0u;
        const uint32_t wr = __shfl_down_sync(FULL, w, 1);
        A = P::hi(w);
        B = P::lo(wr);
        if (valid && right_edge) B = Ed(ebase, a, re, xp);
    };
    auto pull_same = [&](const uint32_t* base, int a, int64_t r, bool valid, float& A, float& B) {
        const uint32_t w = valid ? Wd(base, a, r) : 0u;
        A = P::lo(w);
        B = P::hi(w);
    };
    pull_same(fw, 0, rc, true, fA[0], fB[0]);
    pull_left(fw, fb, 1, rc, ec, true, fA[1], fB[1]);
    pull_right(fw, fb, 3, rc, ec, true, fA[3], fB[3]);
    pull_same(fw, 2, rs, !bottom, fA[2], fB[2]);
    pull_left(fw, fb, 5, rs, es, !bottom, fA[5], fB[5]);
    pull_right(fw, fb, 6, rs, es, !bottom, fA[6], fB[6]);
    pull_same(fw, 4, rn, !top, fA[4], fB[4]);
    pull_right(fw, fb, 7, rn, en, !top, fA[7], fB[7]);
    pull_left(fw, fb, 8, rn, en, !top, fA[8], fB[8]);
    pull_same(gxw, 0, rc, true, gxA[0], gxB[0]);
    pull_left(gxw, gxs, 1, rc, ec, true, gxA[1], gxB[1]);
    pull_right(gxw, gxs, 3, rc, ec, true, gxA[3], gxB[3]);
    pull_same(gxw, 2, rs, !bottom, gxA[2], gxB[2]);
    pull_same(gxw, 4, rn, !top, gxA[4], gxB[4]);
    pull_same(gyw, 0, rc, true, gyA[0], gyB[0]);
    pull_left(gyw, gys, 1, rc, ec, true, gyA[1], gyB[1]);
    pull_right(gyw, gys, 3, rc, ec, true, gyA[3], gyB[3]);
    pull_same(gyw, 2, rs, !bottom, gyA[2], gyB[2]);
    pull_same(gyw, 4, rn, !top, gyA[4], gyB[4]);
    if (CLOSURE == 0) {
        if (bottom) {
            const WallCoef<float>& w = p.bot;
            float a, b;
            pull_same(fw, 4, rc, true, a, b); fA[2] = a; fB[2] = b;
            pull_same(fw, 7, rc, true, a, b); fA[5] = a + w.du; fB[5] = b + w.du;
            pull_same(fw, 8, rc, true, a, b); fA[6] = a - w.du; fB[6] = b - w.du;
            pull_same(gxw, 4, rc, true, a, b); gxA[2] = ffma(w.r, a, w.kx); gxB[2] = ffma(w.r, b, w.kx);
            pull_same(gyw, 4, rc, true, a, b); gyA[2] = -a; gyB[2] = -b;
        }
        if (top) {
            const WallCoef<float>& w = p.top;
            float a, b;
            pull_same(fw, 2, rc, true, a, b); fA[4] = a; fB[4] = b;
            pull_same(fw, 5, rc, true, a, b); fA[7] = a - w.du; fB[7] = b - w.du;
            pull_same(fw, 6, rc, true, a, b); fA[8] = a + w.du; fB[8] = b + w.du;
            pull_same(gxw, 2, rc, true, a, b); gxA[4] = ffma(w.r, a, w.kx); gxB[4] = ffma(w.r, b, w.kx);
            pull_same(gyw, 2, rc, true, a, b); gyA[4] = -a; gyB[4] = -b;
        }
    } else {
        if (bottom) {
            moment_closure_bottom<float, COUPLING>(fA, gxA, gyA, p.bot, p);
            moment_closure_bottom<float, COUPLING>(fB, gxB, gyB, p.bot, p);
        }
        if (top) {
            moment_closure_top<float, COUPLING>(fA, gxA, gyA, p.top, p);
            moment_closure_top<float, COUPLING>(fB, gxB, gyB, p.top, p);
        }
    }
    collide<float, COUPLING>(fA, gxA, gyA, p);
    collide<float, COUPLING>(fB, gxB, gyB, p);

    // ---- push: A_b -> plane bbar at x + e_b; through a wall -> plane b at x ----
    auto st16 = [&](S* ebase, int a, int64_t re, int x, float v) { store_s<S, float>(ebase + a * N + re + x, v); };
    // same column, pair row r
    auto push_same = [&](uint32_t* base, int a, int64_t r, bool valid, float A, float B) {
        if (active && valid) base[a * NP + r + ip] = P::pack(A, B);
    };
    // to x + 1: element x0 <- left lane's B (node x0 - 1), x0 + 1 <- A, x0 + 2 <- B (edge lanes)
    auto push_right = [&](uint32_t* base, S* ebase, int a, int64_t r, int64_t re, bool valid, float A, float B) {
        const float Bl = __shfl_up_sync(FULL, B, 1);
        if (!(active && valid)) return;
        if (!left_edge) base[a * NP + r + ip] = P::pack(Bl, A);
        else st16(ebase, a, re, x0 + 1, A);
        if (right_edge) st16(ebase, a, re, xp, B);
    };
    // to x - 1: element x0 - 1 <- A (edge lanes), x0 <- B, x0 + 1 <- right lane's A (node x0 + 2)
    auto push_left = [&](uint32_t* base, S* ebase, int a, int64_t r, int64_t re, bool valid, float A, float B) {
        const float Ar = __shfl_down_sync(FULL, A, 1);
        if (!(active && valid)) return;
        if (!right_edge) base[a * NP + r + ip] = P::pack(B, Ar);
        else st16(ebase, a, re, x0, B);
        if (left_edge) st16(ebase, a, re, xm, A);
    };
    push_same(fw, 0, rc, true, fA[0], fB[0]);
    push_right(fw, fb, 3, rc, ec, true, fA[1], fB[1]);
    push_left(fw, fb, 1, rc, ec, true, fA[3], fB[3]);
    push_same(fw, 4, rn, !top, fA[2], fB[2]);
    push_same(fw, 2, rc, top, fA[2], fB[2]);
    push_right(fw, fb, 7, rn, en, !top, fA[5], fB[5]);
    push_same(fw, 5, rc, top, fA[5], fB[5]);
    push_left(fw, fb, 8, rn, en, !top, fA[6], fB[6]);
    push_same(fw, 6, rc, top, fA[6], fB[6]);
    push_same(fw, 2, rs, !bottom, fA[4], fB[4]);
    push_same(fw, 4, rc, bottom, fA[4], fB[4]);
    push_left(fw, fb, 5, rs, es, !bottom, fA[7], fB[7]);
    push_same(fw, 7, rc, bottom, fA[7], fB[7]);
    push_right(fw, fb, 6, rs, es, !bottom, fA[8], fB[8]);
    push_same(fw, 8, rc, bottom, fA[8], fB[8]);
    push_same(gxw, 0, rc, true, gxA[0], gxB[0]);
    push_right(gxw, gxs, 3, rc, ec, true, gxA[1], gxB[1]);
    push_left(gxw, gxs, 1, rc, ec, true, gxA[3], gxB[3]);
    push_same(gxw, 4, rn, !top, gxA[2], gxB[2]);
    push_same(gxw, 2, rc, top, gxA[2], gxB[2]);
    push_same(gxw, 2, rs, !bottom, gxA[4], gxB[4]);
    push_same(gxw, 4, rc, bottom, gxA[4], gxB[4]);
    push_same(gyw, 0, rc, true, gyA[0], gyB[0]);
    push_right(gyw, gys, 3, rc, ec, true, gyA[1], gyB[1]);
    push_left(gyw, gys, 1, rc, ec, true, gyA[3], gyB[3]);
    push_same(gyw, 4, rn, !top, gyA[2], gyB[2]);
    push_same(gyw, 2, rc, top, gyA[2], gyB[2]);
    push_same(gyw, 2, rs, !bottom, gyA[4], gyB[4]);
    push_same(gyw, 4, rc, bottom, gyA[4], gyB[4]);
}

template <typename S, typename C, int PHASE, bool R2>
static void launch_aa_grid(S* f, S* g, const StepParams<C>& p, int closure, dim3 grid, cudaStream_t st) {
    if (p.coupling == 0) {
        if (closure == 0) step_kernel_aa<S, C, 0, 0, PHASE, R2><<<grid, 256, 0, st>>>(f, g, p);
        else step_kernel_aa<S, C, 1, 0, PHASE, R2><<<grid, 256, 0, st>>>(f, g, p);
    } else {
        if (closure == 0) step_kernel_aa<S, C, 0, 1, PHASE, R2><<<grid, 256, 0, st>>>(f, g, p);
        else step_kernel_aa<S, C, 1, 1, PHASE, R2><<<grid, 256, 0, st>>>(f, g, p);
    }
}

template <typename S, typename C, int PHASE>
static cudaError_t launch_aa_typed(void* f, void* g, const StepParams<C>& p, int closure, cudaStream_t st) {
    // as in the two-buffer step: FP64 is FP64-pipe-bound and keeps the 1D grid
    if constexpr (sizeof(C) == 4) {
        if (p.nx >= 64 && p.ny <= 65535) {
            launch_aa_grid<S, C, PHASE, true>((S*)f, (S*)g, p, closure, dim3((p.nx + 255) / 256, p.ny), st);
            return cudaGetLastError();
        }
    }
    launch_aa_grid<S, C, PHASE, false>((S*)f, (S*)g, p, closure, dim3((unsigned)((p.N + 255) / 256)), st);
    return cudaGetLastError();
}

template <typename S, int PHASE, bool R2>
static void launch_aa_pair_grid(S* f, S* g, const StepParams<float>& p, int closure, dim3 grid, cudaStream_t st) {
    if (p.coupling == 0) {
        if (closure == 0) step_kernel_aa_pair<S, 0, 0, PHASE, R2><<<grid, 256, 0, st>>>(f, g, p);
        else step_kernel_aa_pair<S, 1, 0, PHASE, R2><<<grid, 256, 0, st>>>(f, g, p);
    } else {
        if (closure == 0) step_kernel_aa_pair<S, 0, 1, PHASE, R2><<<grid, 256, 0, st>>>(f, g, p);
        else step_kernel_aa_pair<S, 1, 1, PHASE, R2><<<grid, 256, 0, st>>>(f, g, p);
    }
}

template <typename S, int PHASE>
static cudaError_t launch_aa_pair(void* f, void* g, const StepParams<float>& p, int closure, cudaStream_t st) {
    const int npr = p.nx / 2;
    if (npr >= 64 && p.ny <= 65535)
        launch_aa_pair_grid<S, PHASE, true>((S*)f, (S*)g, p, closure, dim3((npr + 255) / 256, p.ny), st);
    else
        launch_aa_pair_grid<S, PHASE, false>((S*)f, (S*)g, p, closure, dim3((unsigned)((p.N / 2 + 255) / 256)), st);
    return cudaGetLastError();
}

template <int PHASE>
static cudaError_t launch_aa_phase(int storage, int closure, void* f, void* g, const StepParams<double>& pd,
                                   cudaStream_t st) {
    if (storage == 0) return launch_aa_typed<double, double, PHASE>(f, g, pd, closure, st);
    const StepParams<float> pf = convert_params<float>(pd);
    if (storage == 1) return launch_aa_typed<float, float, PHASE>(f, g, pf, closure, st);
    const bool pairs = (pd.nx % 2) == 0;  // two nodes per thread need whole pairs in every row
    if (storage == 2)
        return pairs ? launch_aa_pair<__nv_bfloat16, PHASE>(f, g, pf, closure, st)
                     : launch_aa_typed<__nv_bfloat16, float, PHASE>(f, g, pf, closure, st);
    return pairs ? launch_aa_pair<__half, PHASE>(f, g, pf, closure, st)
                 : launch_aa_typed<__half, float, PHASE>(f, g, pf, closure, st);
}

cudaError_t launch_step_aa(int storage, int closure, int phase, void* f, void* g, const StepParams<double>& pd,
                           cudaStream_t st) {
    return phase == 0 ? launch_aa_phase<0>(storage, closure, f, g, pd, st)
                      : launch_aa_phase<1>(storage, closure, f, g, pd, st);
}

}  // namespace lks
