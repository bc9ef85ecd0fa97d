// lks_step.cu -- the fused collide-stream kernel of one lattice (pull, wall closures, collision, store).
//
// One thread per node (the per-node work is step_node in lks_device.cuh), nodes numbered n = y*nx + x so that a warp reads 32 consecutive
// x positions of each population plane: every one of the 19 loads and 19 stores of a warp
// is a coalesced 128-byte (FP32) / 256-byte (FP64) / 64-byte (16-bit) access; the +-1
// x-shifted pulls straddle one extra sector that the neighbouring warp's load brings into
// L1/L2 anyway.  Each element of the source buffer is read exactly once per step:
//   interior rows pull from rows y-1 / y / y+1 (Eqs. LBMforflowfield, LKSformagneticfield);
//   link-based wall rows take the unknown incoming populations from the same node's
//   outgoing ones (Sec. VI, App. B.1), which nobody else reads;
//   moment-based wall rows reconstruct them from the pulled ones (Sec. VII, App. A, B.2).
#include "lks_device.cuh"
#include "lks_internal.h"
#include "lks_packed.cuh"

namespace lks {

// ROWS2D: grid (ceil(nx/256), ny), the column and row come from the block indices; otherwise a
// 1D grid over n = y*nx + x (narrow lattices), split with one 32-bit division.
template <typename S, typename C, int CLOSURE, int COUPLING, bool ROWS2D>
__global__ void __launch_bounds__(256) step_kernel(const S* __restrict__ fin, const S* __restrict__ gin,
                                                   S* __restrict__ fout, S* __restrict__ gout,
                                                   const StepParams<C> p) {
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
    step_node<S, C, CLOSURE, true, COUPLING>(fin, gin, fout, gout, p, n, i, j);
}

// 16-bit storage moves 2 bytes per population, so the one-node kernel issues twice the load/store
// instructions per byte of the FP32 one and becomes instruction-bound.  This variant gives each
// thread the two nodes (x0, x0+1), x0 even, and moves every population plane as one 32-bit word
// holding both nodes (nx must be even).  A pull from x-1 needs (x0-1, x0): the word of the lane to
// the left supplies x0-1 through a warp shuffle (a direct 16-bit load at a warp or row edge,
// wrapping periodically); a pull from x+1 needs (x0+1, x0+2) likewise from the lane to the right.
// Per node the arithmetic is exactly that of step_node, so results are bit-identical to it.
// Register budget: the moment-based variants fit 64 registers (4 blocks of 256 per SM); the
// link-based ones, which also load the wall node's own outgoing words, spill at 64 and run faster
// with 80 (3 blocks per SM): 69.5 against 61.3 GLUPS for BF16 at 8192^2, while 3 blocks cost the
// moment-based variants 7 % (69.6 against 74.8 GLUPS at 4096^2).
template <typename S, int CLOSURE, int COUPLING, bool ROWS2D>
__global__ void __launch_bounds__(256, CLOSURE == 0 ? 3 : 4) step_kernel_pair(const S* __restrict__ fin, const S* __restrict__ gin,
                                                        S* __restrict__ fout, S* __restrict__ gout,
                                                        const StepParams<float> p) {
    typedef Packed<S> P;
    const unsigned FULL = 0xffffffffu;
    const int nx = p.nx, npr = nx >> 1;
    const int64_t N = p.N, NP = N >> 1;
    const int lane = threadIdx.x & 31;
    // inactive lanes (past the end) still take part in the shuffles, on a clamped pair
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
    const int x0 = ip << 1;
    const int64_t rc = (int64_t)j * npr;         // row starts, in pairs
    const int64_t rs = rc - npr, rn = rc + npr;
    const bool bottom = (j == 0), top = (j == p.ny - 1);
    const bool left_edge = (lane == 0) || (ip == 0);
    const bool right_edge = (lane == 31) || (ip == npr - 1);
    const int xm = (x0 == 0) ? nx - 1 : x0 - 1;  // element pulled by node x0 from the left
    const int xp = (x0 + 2 == nx) ? 0 : x0 + 2;  // element pulled by node x0+1 from the right

    const uint32_t* fw = reinterpret_cast<const uint32_t*>(fin);
    const uint32_t* gw = reinterpret_cast<const uint32_t*>(gin);
    // word of plane `a` (of NP words) at pair row r
    auto W = [&](const uint32_t* base, int a, int64_t r) -> uint32_t { return __ldg(base + a * NP + r + ip); };
    // single element of plane `a` at element row re (= row * nx), column x
    auto E = [&](const S* base, int a, int64_t re, int x) -> float { return load_s<S, float>(base + a * N + re + x); };

    float fA[9], fB[9], gxA[5], gxB[5], gyA[5], gyB[5];
    const S* gxs = gin;
    const S* gys = gin + 5 * N;
    const uint32_t* gxw = gw;
    const uint32_t* gyw = gw + 5 * NP;

    // pull from x-1 in plane a of source pair row r (element row re): node A <- x0-1, node B <- x0
    auto pull_left = [&](const uint32_t* base, const S* ebase, int a, int64_t r, int64_t re, bool valid, float& A,
                         float& B) {
        const uint32_t w = valid ? W(base, a, r) : 0u;
        const uint32_t wl = __shfl_up_sync(FULL, w, 1);
        B = P::lo(w);
        A = P::hi(wl);
        if (valid && left_edge) A = E(ebase, a, re, xm);
    };
    // pull from x+1: node A <- x0+1, node B <- x0+2
    auto pull_right = [&](const uint32_t* base, const S* ebase, int a, int64_t r, int64_t re, bool valid, float& A,
                          float& B) {
        const uint32_t w = valid ? W(base, a, r) : 0u;
        const uint32_t wr = __shfl_down_sync(FULL, w, 1);
        A = P::hi(w);
        B = P::lo(wr);
        if (valid && right_edge) B = E(ebase, a, re, xp);
    };
    auto pull_same = [&](const uint32_t* base, int a, int64_t r, bool valid, float& A, float& B) {
        const uint32_t w = valid ? W(base, a, r) : 0u;
        A = P::lo(w);
        B = P::hi(w);
    };
    const int64_t ec = (int64_t)j * nx, es = ec - nx, en = ec + nx;   // element row starts
    // pull-stream (rows y-1 / y / y+1), periodic in x
    pull_same(fw, 0, rc, true, fA[0], fB[0]);
    pull_left(fw, fin, 1, rc, ec, true, fA[1], fB[1]);
    pull_right(fw, fin, 3, rc, ec, true, fA[3], fB[3]);
    pull_same(fw, 2, rs, !bottom, fA[2], fB[2]);
    pull_left(fw, fin, 5, rs, es, !bottom, fA[5], fB[5]);
    pull_right(fw, fin, 6, rs, es, !bottom, fA[6], fB[6]);
    pull_same(fw, 4, rn, !top, fA[4], fB[4]);
    pull_right(fw, fin, 7, rn, en, !top, fA[7], fB[7]);
    pull_left(fw, fin, 8, rn, en, !top, fA[8], fB[8]);
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
    // wall closures
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
    // moments, equilibria, collision
    collide<float, COUPLING>(fA, gxA, gyA, p);
    collide<float, COUPLING>(fB, gxB, gyB, p);
    // store both nodes of each plane as one word
    if (!active) return;
    uint32_t* fo = reinterpret_cast<uint32_t*>(fout);
    uint32_t* go = reinterpret_cast<uint32_t*>(gout);
#pragma unroll
    for (int a = 0; a < 9; ++a) fo[a * NP + q] = P::pack(fA[a], fB[a]);
#pragma unroll
    for (int a = 0; a < 5; ++a) go[a * NP + q] = P::pack(gxA[a], gxB[a]);
#pragma unroll
    for (int a = 0; a < 5; ++a) go[(5 + a) * NP + q] = P::pack(gyA[a], gyB[a]);
}

// A row-per-grid-row layout when rows are wide enough to fill blocks and ny fits gridDim.y.
static bool rows2d(int row_items, int ny) { return row_items >= 64 && ny <= 65535; }

template <typename S, bool R2>
static void launch_pair_grid(const S* fi, const S* gi, S* fo, S* go, const StepParams<float>& p, int closure,
                             dim3 grid, cudaStream_t st) {
    if (p.coupling == 0) {
        if (closure == 0) step_kernel_pair<S, 0, 0, R2><<<grid, 256, 0, st>>>(fi, gi, fo, go, p);
        else step_kernel_pair<S, 1, 0, R2><<<grid, 256, 0, st>>>(fi, gi, fo, go, p);
    } else {
        if (closure == 0) step_kernel_pair<S, 0, 1, R2><<<grid, 256, 0, st>>>(fi, gi, fo, go, p);
        else step_kernel_pair<S, 1, 1, R2><<<grid, 256, 0, st>>>(fi, gi, fo, go, p);
    }
}

template <typename S>
static cudaError_t launch_pair(const void* fin, const void* gin, void* fout, void* gout, const StepParams<float>& p,
                               int closure, cudaStream_t st) {
    const int npr = p.nx / 2;
    if (rows2d(npr, p.ny))
        launch_pair_grid<S, true>((const S*)fin, (const S*)gin, (S*)fout, (S*)gout, p, closure,
                                  dim3((npr + 255) / 256, p.ny), st);
    else
        launch_pair_grid<S, false>((const S*)fin, (const S*)gin, (S*)fout, (S*)gout, p, closure,
                                   dim3((unsigned)((p.N / 2 + 255) / 256)), st);
    return cudaGetLastError();
}

template <typename S, typename C, bool R2>
static void launch_typed_grid(const S* fi, const S* gi, S* fo, S* go, const StepParams<C>& p, int closure,
                              dim3 grid, cudaStream_t st) {
    if (p.coupling == 0) {
        if (closure == 0) step_kernel<S, C, 0, 0, R2><<<grid, 256, 0, st>>>(fi, gi, fo, go, p);
        else step_kernel<S, C, 1, 0, R2><<<grid, 256, 0, st>>>(fi, gi, fo, go, p);
    } else {
        if (closure == 0) step_kernel<S, C, 0, 1, R2><<<grid, 256, 0, st>>>(fi, gi, fo, go, p);
        else step_kernel<S, C, 1, 1, R2><<<grid, 256, 0, st>>>(fi, gi, fo, go, p);
    }
}

template <typename S, typename C>
static cudaError_t launch_typed(const void* fin, const void* gin, void* fout, void* gout, const StepParams<C>& p,
                                int closure, cudaStream_t st) {
    // FP64 is bound by the FP64 pipe, where the grid shape changes nothing (3.55 GLUPS at 4096^2
    // either way): it keeps the 1D grid, and its 2D kernels are not instantiated
    if constexpr (sizeof(C) == 4) {
        if (rows2d(p.nx, p.ny)) {
            launch_typed_grid<S, C, true>((const S*)fin, (const S*)gin, (S*)fout, (S*)gout, p, closure,
                                          dim3((p.nx + 255) / 256, p.ny), st);
            return cudaGetLastError();
        }
    }
    launch_typed_grid<S, C, false>((const S*)fin, (const S*)gin, (S*)fout, (S*)gout, p, closure,
                                   dim3((unsigned)((p.N + 255) / 256)), st);
    return cudaGetLastError();
}

cudaError_t launch_step(int storage, int closure, const void* fin, const void* gin, void* fout, void* gout,
                        const StepParams<double>& pd, cudaStream_t st, const StagedStep* ss) {
    if (storage == 0) return launch_typed<double, double>(fin, gin, fout, gout, pd, closure, st);
    StepParams<float> pf = convert_params<float>(pd);
    if (storage == 1) return launch_typed<float, float>(fin, gin, fout, gout, pf, closure, st);
    if (ss && staged_step_applies(storage, pd.nx, 0))
        return launch_step_staged(storage, closure, fin, gin, fout, gout, pf, *ss, st);
    const bool pairs = (pd.nx % 2) == 0;  // two nodes per thread need whole pairs in every row
    if (storage == 2)
        return pairs ? launch_pair<__nv_bfloat16>(fin, gin, fout, gout, pf, closure, st)
                     : launch_typed<__nv_bfloat16, float>(fin, gin, fout, gout, pf, closure, st);
    return pairs ? launch_pair<__half>(fin, gin, fout, gout, pf, closure, st)
                 : launch_typed<__half, float>(fin, gin, fout, gout, pf, closure, st);
}

}  // namespace lks
