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

// 16-bit storage, two nodes per thread and one 32-bit word per population plane (nx even), with
// the rows interleaved as for the two-buffer pair kernel: word w of a row holds nodes x = w and
// x = w + nx/2.  A shift by one node in x is then a shift by one word (halves swapped at the
// periodic row edge), so phase 0 pulls and pushes whole aligned words exactly as the one-node
// in-place kernel does per node: the pulls of word w come from words w - 1 / w / w + 1 of the
// neighbouring rows and the pushes go to the same words.  No two threads touch the same word
// (each word a thread pushes into holds the two elements its own nodes pull in that direction),
// and every thread reads its words before it writes them.  Phase 1 touches only its own words.
template <typename S, int CLOSURE, int COUPLING, int PHASE, bool ROWS2D>
__global__ void __launch_bounds__(256, (CLOSURE == 0 || PHASE == 0) ? 3 : 4) step_kernel_aa_pair(S* fb, S* gb, const StepParams<float> p) {
    typedef Packed<S> P;
    const int H = p.nx >> 1;
    const int64_t NP = p.N >> 1;
    int j, w;
    if (ROWS2D) {
        w = blockIdx.x * blockDim.x + threadIdx.x;
        j = blockIdx.y;
        if (w >= H) return;
    } else {
        const unsigned q0 = blockIdx.x * blockDim.x + threadIdx.x;
        if ((int64_t)q0 >= NP) return;
        j = (int)(q0 / (unsigned)H);
        w = (int)(q0 - (unsigned)j * (unsigned)H);
    }
    const int64_t q = (int64_t)j * H + w;
    const bool bottom = (j == 0), top = (j == p.ny - 1);
    uint32_t* fw = reinterpret_cast<uint32_t*>(fb);
    uint32_t* gxw = reinterpret_cast<uint32_t*>(gb);
    uint32_t* gyw = gxw + 5 * NP;
    float fA[9], fB[9], gxA[5], gxB[5], gyA[5], gyB[5];
    auto take = [](uint32_t v, bool swap, float& A, float& B) {
        if (swap) v = __byte_perm(v, 0, 0x1032);
        A = P::lo(v);
        B = P::hi(v);
    };

    if (PHASE == 1) {
        // direction a of both nodes from plane abar of the own word
        auto own = [&](const uint32_t* base, int plane, bool valid, float& A, float& B) {
            take(valid ? base[plane * NP + q] : 0u, false, A, B);
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
                const WallCoef<float>& wc = p.bot;
                fA[5] = fA[5] + wc.du; fB[5] = fB[5] + wc.du;
                fA[6] = fA[6] - wc.du; fB[6] = fB[6] - wc.du;
                gxA[2] = ffma(wc.r, gxA[2], wc.kx); gxB[2] = ffma(wc.r, gxB[2], wc.kx);
                gyA[2] = -gyA[2]; gyB[2] = -gyB[2];
            }
            if (top) {
                const WallCoef<float>& wc = p.top;
                fA[7] = fA[7] - wc.du; fB[7] = fB[7] - wc.du;
                fA[8] = fA[8] + wc.du; fB[8] = fB[8] + wc.du;
                gxA[4] = ffma(wc.r, gxA[4], wc.kx); gxB[4] = ffma(wc.r, gxB[4], wc.kx);
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
    // ---- phase 0: pull (as the two-buffer pair kernel, coherent loads), close, collide, push ----
    const int64_t rc = (int64_t)j * H, rs = rc - H, rn = rc + H;
    const int wm = (w == 0) ? H - 1 : w - 1, wp = (w == H - 1) ? 0 : w + 1;
    const bool sm = (w == 0), sp = (w == H - 1);
    auto ps = [&](const uint32_t* base, int a, int64_t r, float& A, float& B) { take(base[a * NP + r + w], false, A, B); };
    auto pl = [&](const uint32_t* base, int a, int64_t r, float& A, float& B) { take(base[a * NP + r + wm], sm, A, B); };
    auto pr = [&](const uint32_t* base, int a, int64_t r, float& A, float& B) { take(base[a * NP + r + wp], sp, A, B); };
    ps(fw, 0, rc, fA[0], fB[0]);
    pl(fw, 1, rc, fA[1], fB[1]);
    pr(fw, 3, rc, fA[3], fB[3]);
    ps(gxw, 0, rc, gxA[0], gxB[0]);
    pl(gxw, 1, rc, gxA[1], gxB[1]);
    pr(gxw, 3, rc, gxA[3], gxB[3]);
    ps(gyw, 0, rc, gyA[0], gyB[0]);
    pl(gyw, 1, rc, gyA[1], gyB[1]);
    pr(gyw, 3, rc, gyA[3], gyB[3]);
    if (!bottom) {
        ps(fw, 2, rs, fA[2], fB[2]);
        pl(fw, 5, rs, fA[5], fB[5]);
        pr(fw, 6, rs, fA[6], fB[6]);
        ps(gxw, 2, rs, gxA[2], gxB[2]);
        ps(gyw, 2, rs, gyA[2], gyB[2]);
    }
    if (!top) {
        ps(fw, 4, rn, fA[4], fB[4]);
        pr(fw, 7, rn, fA[7], fB[7]);
        pl(fw, 8, rn, fA[8], fB[8]);
        ps(gxw, 4, rn, gxA[4], gxB[4]);
        ps(gyw, 4, rn, gyA[4], gyB[4]);
    }
    if (CLOSURE == 0) {
        if (bottom) {
            const WallCoef<float>& wc = p.bot;
            float a, b;
            ps(fw, 4, rc, a, b); fA[2] = a; fB[2] = b;
            ps(fw, 7, rc, a, b); fA[5] = a + wc.du; fB[5] = b + wc.du;
            ps(fw, 8, rc, a, b); fA[6] = a - wc.du; fB[6] = b - wc.du;
            ps(gxw, 4, rc, a, b); gxA[2] = ffma(wc.r, a, wc.kx); gxB[2] = ffma(wc.r, b, wc.kx);
            ps(gyw, 4, rc, a, b); gyA[2] = -a; gyB[2] = -b;
        }
        if (top) {
            const WallCoef<float>& wc = p.top;
            float a, b;
            ps(fw, 2, rc, a, b); fA[4] = a; fB[4] = b;
            ps(fw, 5, rc, a, b); fA[7] = a - wc.du; fB[7] = b - wc.du;
            ps(fw, 6, rc, a, b); fA[8] = a + wc.du; fB[8] = b + wc.du;
            ps(gxw, 2, rc, a, b); gxA[4] = ffma(wc.r, a, wc.kx); gxB[4] = ffma(wc.r, b, wc.kx);
            ps(gyw, 2, rc, a, b); gyA[4] = -a; gyB[4] = -b;
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
    // push: A_b -> plane bbar at x + e_b (the word the own nodes pull direction bbar from);
    // through a wall -> plane b of the own word
    auto put = [](uint32_t* at, bool swap, float A, float B) { *at = swap ? P::pack(B, A) : P::pack(A, B); };
    put(fw + 0 * NP + rc + w, false, fA[0], fB[0]);
    put(fw + 3 * NP + rc + wp, sp, fA[1], fB[1]);     // +x -> plane 3 at x + 1
    put(fw + 1 * NP + rc + wm, sm, fA[3], fB[3]);     // -x -> plane 1 at x - 1
    put(gxw + 0 * NP + rc + w, false, gxA[0], gxB[0]);
    put(gxw + 3 * NP + rc + wp, sp, gxA[1], gxB[1]);
    put(gxw + 1 * NP + rc + wm, sm, gxA[3], gxB[3]);
    put(gyw + 0 * NP + rc + w, false, gyA[0], gyB[0]);
    put(gyw + 3 * NP + rc + wp, sp, gyA[1], gyB[1]);
    put(gyw + 1 * NP + rc + wm, sm, gyA[3], gyB[3]);
    if (!top) {
        put(fw + 4 * NP + rn + w, false, fA[2], fB[2]);
        put(fw + 7 * NP + rn + wp, sp, fA[5], fB[5]);
        put(fw + 8 * NP + rn + wm, sm, fA[6], fB[6]);
        put(gxw + 4 * NP + rn + w, false, gxA[2], gxB[2]);
        put(gyw + 4 * NP + rn + w, false, gyA[2], gyB[2]);
    } else {
        put(fw + 2 * NP + rc + w, false, fA[2], fB[2]);
        put(fw + 5 * NP + rc + w, false, fA[5], fB[5]);
        put(fw + 6 * NP + rc + w, false, fA[6], fB[6]);
        put(gxw + 2 * NP + rc + w, false, gxA[2], gxB[2]);
        put(gyw + 2 * NP + rc + w, false, gyA[2], gyB[2]);
    }
    if (!bottom) {
        put(fw + 2 * NP + rs + w, false, fA[4], fB[4]);
        put(fw + 5 * NP + rs + wm, sm, fA[7], fB[7]);
        put(fw + 6 * NP + rs + wp, sp, fA[8], fB[8]);
        put(gxw + 2 * NP + rs + w, false, gxA[4], gxB[4]);
        put(gyw + 2 * NP + rs + w, false, gyA[4], gyB[4]);
    } else {
        put(fw + 4 * NP + rc + w, false, fA[4], fB[4]);
        put(fw + 7 * NP + rc + w, false, fA[7], fB[7]);
        put(fw + 8 * NP + rc + w, false, fA[8], fB[8]);
        put(gxw + 4 * NP + rc + w, false, gxA[4], gxB[4]);
        put(gyw + 4 * NP + rc + w, false, gyA[4], gyB[4]);
    }
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
    const bool pairs = interleave_row(storage, pd.nx, 1) != 0;  // interleaved rows: two nodes per thread
    if (storage == 2)
        return pairs ? launch_aa_pair<__nv_bfloat16, PHASE>(f, g, pf, closure, st)
                     : launch_aa_typed<__nv_bfloat16, float, PHASE>(f, g, pf, closure, st);
    return pairs ? launch_aa_pair<__half, PHASE>(f, g, pf, closure, st)
                 : launch_aa_typed<__half, float, PHASE>(f, g, pf, closure, st);
}

cudaError_t launch_step_aa(int storage, int closure, int phase, void* f, void* g, const StepParams<double>& pd,
                           cudaStream_t st, const StagedStep* ss) {
    if (phase == 0 && ss && staged_step_applies(storage, pd.nx, 1))
        return launch_step_aa_staged(storage, closure, f, g, convert_params<float>(pd), *ss, st);
    return phase == 0 ? launch_aa_phase<0>(storage, closure, f, g, pd, st)
                      : launch_aa_phase<1>(storage, closure, f, g, pd, st);
}

}  // namespace lks
