// lks_step_staged.cu -- the fused step of one lattice with 16-bit deviation storage, rows staged
// through shared memory by the bulk-copy engine (two-buffer handles; nx a multiple of 8 and at least
// kSegX).  The pull, wall closures, collision and store as in step_node_with (lks_device.cuh), with the same per-node
// arithmetic: the results agree bit for bit with the one- and two-node kernels.
//
// A task is a row segment of up to kSegX nodes (x0 .. x0 + T - 1 of row y).  For each of the 19
// population slots (f_0..8, g_x0..4, g_y0..4) a producer warp copies, one slot per lane, the segment
// of the row the slot pulls from (y - e_y; a link-closure wall row takes its own row of the opposite
// plane; a moment-closure wall row fetches nothing for the slots it reconstructs) into one of the
// shared-memory stages, with a 16-byte halo on each side for the x-shifted slots (periodic in x:
// wrapped copies at the row ends), completing on the stage's `full` mbarrier.  Sixteen consumer
// warps take two x-adjacent nodes per thread as one float2 (packed FP32x2 arithmetic): 19 words of
// the staged rows (byte_perm for the x shift), the wall closure, the collision, 19 packed words
// stored.  Each lane first copies its 19 words into its column of the warp's private scratch and
// the warp arrives on the stage's `empty` mbarrier at once, so the producer refills the stage while
// the warp computes from the scratch.  Every wait is bounded (kWaitNs); one that runs out sets *err and
// ends that warp's loop, and the producer waits, within the same limit, for its last copies to each
// stage before it returns.
//
// One block of 16 consumer warps per SM with 1024-node tasks (2 KB copies) beat two blocks of 8
// warps with 512-node tasks at 4096^2: 76-80 against 71-72 GLUPS (the copies per byte halve).  Rows
// without a wall run a compile-time path without the closure code (BF16, moment closure: 79.8
// against 76.1 GLUPS).  Releasing the stage as soon as the words are read, through the per-warp
// scratch (four stages instead of five): BF16 82.8, FP16 80.0 GLUPS against 79.4 and 78.8 with the
// release after the stores.  Holding the words in registers across the release instead spilled at
// the 96 registers a thread of this block has (BF16 78.0, FP16 78.7); a whole producer warpgroup
// that moved registers to the consumers with setmaxnreg (32 / 112) ran at 73.4.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "lks_bulk.cuh"
#include "lks_device.cuh"
#include "lks_internal.h"
#include "lks_packed.cuh"

namespace lks {
namespace {

constexpr int kSegX = 1024;                      // nodes of a task: consumer threads x 2
constexpr int kHaloW = 4;                        // halo words (8 elements = 16 bytes) per side
constexpr int kSlotW = kSegX / 2 + 2 * kHaloW;   // words of a staged slot row
constexpr int kSlots = 19;
constexpr int kStages = 5;
constexpr int kStageW = kSlots * kSlotW;
constexpr int kConsumerWarps = kSegX / 64;
constexpr int kThreads = kSegX / 2 + 32;         // consumers + the producer warp
constexpr uint64_t kWaitNs = 1000000000ull;      // 1 s
constexpr size_t kSmem = 128 + (size_t)kStages * kStageW * 4;
// Both kernels: four stages, and behind them a private scratch area per consumer warp into which each
// lane copies its 19 staged words, so that the warp can hand its stage back at once (the in-place
// phase 0 with it: BF16 81.8, FP16 83.0 GLUPS per pair of steps against 80.9 and 80.5).
constexpr int kStagesTB = 4;
constexpr int kScratchW = kSlots * 32;  // words per consumer warp
constexpr size_t kSmemTB = 128 + (size_t)kStagesTB * kStageW * 4 + (size_t)kConsumerWarps * kScratchW * 4;
static_assert(kSmemTB <= 227 * 1024, "shared memory per block");

// D2Q9 (f) and D2Q5 (g) directions of slot k: k < 9 is f_k, 9..13 is g_x,k-9, 14..18 is g_y,k-14.
__host__ __device__ constexpr int dir_of(int k) { return k < 9 ? k : (k < 14 ? k - 9 : k - 14); }
__host__ __device__ constexpr int ex9(int a) { return (a == 1 || a == 5 || a == 8) ? 1 : (a == 3 || a == 6 || a == 7) ? -1 : 0; }
__host__ __device__ constexpr int ey9(int a) { return (a == 2 || a == 5 || a == 6) ? 1 : (a == 4 || a == 7 || a == 8) ? -1 : 0; }
__host__ __device__ constexpr int opp9(int a) { return a == 0 ? 0 : (a <= 4 ? (a + 1) % 4 + 1 : (a + 1) % 4 + 5); }
// plane of slot k's population table for direction a (f: a; g_x: a; g_y: 5 + a)
__host__ __device__ constexpr int plane_of(int k, int a) { return k < 9 ? a : (k < 14 ? a : 5 + a); }

// Moment closure (wall rows, W) and collision of a node pair.  The Maxwell coupling runs as one
// float2.  The Lorentz coupling runs per node in scalar, as the one- and two-node kernels do: on its
// f update the scalar and the packed forms were measured to round differently in a fraction of the
// nodes, which would end the agreement bit for bit between the kernels.
template <int CLOSURE, int COUPLING, bool W>
__device__ __forceinline__ void close_collide_pair(float2 f[9], float2 gx[5], float2 gy[5], const StepParams<float>& p,
                                                   bool bottom, bool top) {
    if constexpr (COUPLING == 0) {
        if (W && CLOSURE == 1) {
            if (bottom) moment_closure_bottom<float, 0>(f, gx, gy, p.bot, p);
            if (top) moment_closure_top<float, 0>(f, gx, gy, p.top, p);
        }
        collide<float, 0>(f, gx, gy, p);
    } else {
        float fA[9], gxA[5], gyA[5], fB[9], gxB[5], gyB[5];
#pragma unroll
        for (int a = 0; a < 9; ++a) fA[a] = f[a].x, fB[a] = f[a].y;
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            gxA[a] = gx[a].x, gxB[a] = gx[a].y;
            gyA[a] = gy[a].x, gyB[a] = gy[a].y;
        }
        if (W && CLOSURE == 1) {
            if (bottom) {
                moment_closure_bottom<float, 1>(fA, gxA, gyA, p.bot, p);
                moment_closure_bottom<float, 1>(fB, gxB, gyB, p.bot, p);
            }
            if (top) {
                moment_closure_top<float, 1>(fA, gxA, gyA, p.top, p);
                moment_closure_top<float, 1>(fB, gxB, gyB, p.top, p);
            }
        }
        collide<float, 1>(fA, gxA, gyA, p);
        collide<float, 1>(fB, gxB, gyB, p);
#pragma unroll
        for (int a = 0; a < 9; ++a) f[a] = make_float2(fA[a], fB[a]);
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            gx[a] = make_float2(gxA[a], gxB[a]);
            gy[a] = make_float2(gyA[a], gyB[a]);
        }
    }
}

template <typename S, int CLOSURE, int COUPLING>
__global__ void __launch_bounds__(kThreads, 1) step_kernel_staged(const S* __restrict__ fin, const S* __restrict__ gin,
                                                                   S* __restrict__ fout, S* __restrict__ gout,
                                                                   const StepParams<float> p, int* err) {
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t* full = reinterpret_cast<uint64_t*>(sm);
    uint64_t* empty = full + kStagesTB;
    uint32_t* stage0 = reinterpret_cast<uint32_t*>(sm + 128);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nx = p.nx, ny = p.ny;
    const int64_t N = p.N;
    const int nseg = (nx + kSegX - 1) / kSegX;
    const int64_t ntask = (int64_t)ny * nseg;
    const int64_t G = gridDim.x, t0 = blockIdx.x;
    const int64_t nmine = t0 < ntask ? (ntask - 1 - t0) / G + 1 : 0;  // tasks t0, t0 + G, ...
    if (tid == 0) {
        for (int s = 0; s < kStagesTB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        mbar_init_fence();
    }
    __syncthreads();

    if (warp == kConsumerWarps) {  // producer: lane k < 19 fetches slot k
        const int k = lane < kSlots ? lane : 0;
        const int a = dir_of(k), ex = ex9(a), ey = ey9(a);
        const S* base = k < 9 ? fin : gin;
        const S* bn = base + (int64_t)plane_of(k, a) * N;        // the slot's own direction
        const S* bw = base + (int64_t)plane_of(k, opp9(a)) * N;  // the opposite one (link walls)
        int64_t it = 0;
        for (; it < nmine; ++it) {
            const int s = (int)(it % kStagesTB);
            const int64_t u = it / kStagesTB;
            if (u > 0 && !mbar_wait_bounded(&empty[s], (uint32_t)(u - 1) & 1u, kWaitNs)) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            const int64_t t = t0 + it * G;
            const int y = (int)(t / nseg), x0 = (int)(t % nseg) * kSegX;
            const int T = min(kSegX, nx - x0);
            const bool wall = (ey == 1 && y == 0) || (ey == -1 && y == ny - 1);
            uint32_t* dst = stage0 + s * kStageW + k * kSlotW;
            // this lane's copies: (global element offset, shared word offset, elements)
            int64_t g0 = 0, g1 = 0, g2 = 0;
            int w0 = 0, w1 = 0, w2 = 0, n0 = 0, n1 = 0, n2 = 0;
            if (lane < kSlots) {
                if (wall) {
                    if (CLOSURE == 0) {  // link: own row, opposite plane
                        g0 = (int64_t)y * nx + x0;
                        w0 = kHaloW;
                        n0 = T;
                    }
                } else {
                    const int64_t row = (int64_t)(y - ey) * nx;
                    if (ex == 0) {
                        g0 = row + x0, w0 = kHaloW, n0 = T;
                    } else if (x0 >= 8 && x0 + T + 8 <= nx) {  // both halos in one copy
                        g0 = row + x0 - 8, w0 = 0, n0 = T + 16;
                    } else {
                        g0 = row + x0, w0 = kHaloW, n0 = T;
                        if (ex == 1) g1 = row + (x0 == 0 ? nx - 8 : x0 - 8), w1 = 0, n1 = 8;
                        else g2 = row + (x0 + T == nx ? 0 : x0 + T), w2 = kHaloW + T / 2, n2 = 8;
                    }
                }
            }
            const uint32_t mine = 2u * (uint32_t)(n0 + n1 + n2);
            const uint32_t bytes = __reduce_add_sync(0xffffffffu, mine);
            if (lane == 0) mbar_arrive_expect_tx(&full[s], bytes);
            __syncwarp();
            const S* src = (wall && CLOSURE == 0) ? bw : bn;
            if (n0) bulk_g2s(dst + w0, src + g0, 2u * n0, &full[s]);
            if (n1) bulk_g2s(dst + w1, src + g1, 2u * n1, &full[s]);
            if (n2) bulk_g2s(dst + w2, src + g2, 2u * n2, &full[s]);
        }
        // no copy may be left in flight into this block's shared memory: wait for the last phase
        // issued to each stage (already complete unless a consumer gave up)
        for (int s = 0; s < kStagesTB; ++s) {
            if (it <= s) continue;
            const int64_t u_last = (it - 1 - s) / kStagesTB;
            if (!mbar_wait_bounded(&full[s], (uint32_t)u_last & 1u, kWaitNs) && lane == 0) atomicExch(err, 1);
        }
        return;
    }

    // consumers: thread tid holds nodes x0 + 2 tid and x0 + 2 tid + 1 of the task's row
    uint32_t* scr = stage0 + kStagesTB * kStageW + warp * kScratchW;
    typedef Packed<S> P;
    const int xw = kHaloW + tid;
    for (int64_t it = 0; it < nmine; ++it) {
        const int s = (int)(it % kStagesTB);
        if (!mbar_wait_bounded(&full[s], (uint32_t)(it / kStagesTB) & 1u, kWaitNs)) {
            atomicExch(err, 1);
            break;
        }
        const int64_t t = t0 + it * G;
        const int y = (int)(t / nseg), x0 = (int)(t % nseg) * kSegX;
        const int T = min(kSegX, nx - x0);
        const bool active = 2 * tid < T;
        {
            const bool bottom = (y == 0), top = (y == ny - 1);
            const uint32_t* st = stage0 + s * kStageW;
            // rows without a wall (all but two) take a path with no closure code
            auto body = [&](auto walls) {
                constexpr bool W = decltype(walls)::value;
                if (active) {
#pragma unroll
                    for (int k = 0; k < kSlots; ++k) {
                        const int a = dir_of(k), ex = ex9(a), ey = ey9(a);
                        const bool wall = W && ((ey == 1 && bottom) || (ey == -1 && top));
                        const uint32_t* row = st + k * kSlotW;
                        uint32_t w;
                        if (wall || ex == 0)
                            w = row[xw];
                        else if (ex == 1)  // x <- x - 1 (high half of the word before), x + 1 <- x
                            w = __byte_perm(row[xw - 1], row[xw], 0x5432);
                        else  // x <- x + 1, x + 1 <- x + 2 (low half of the word after)
                            w = __byte_perm(row[xw], row[xw + 1], 0x5432);
                        scr[k * 32 + lane] = w;  // this lane's column of the warp's scratch
                    }
                }
                // the warp's words are in its scratch: the stage goes back to the producer before the
                // collision and the stores
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
                if (!active) return;
                float2 v[kSlots];
#pragma unroll
                for (int k = 0; k < kSlots; ++k) {
                    const uint32_t w = scr[k * 32 + lane];
                    v[k] = P::pair(w);
                }
                float2 f[9], gx[5], gy[5];
#pragma unroll
                for (int a = 0; a < 9; ++a) f[a] = v[a];
#pragma unroll
                for (int a = 0; a < 5; ++a) {
                    gx[a] = v[9 + a];
                    gy[a] = v[14 + a];
                }
                // wall closures (the link slots hold the node's own outgoing populations)
                if (W && CLOSURE == 0) {
                    if (bottom) {
                        const WallCoef<float>& w = p.bot;
                        f[5] = f[5] + w.du;
                        f[6] = f[6] - w.du;
                        gx[2] = ffma(w.r, gx[2], w.kx);
                        gy[2] = -gy[2];
                    }
                    if (top) {
                        const WallCoef<float>& w = p.top;
                        f[7] = f[7] - w.du;
                        f[8] = f[8] + w.du;
                        gx[4] = ffma(w.r, gx[4], w.kx);
                        gy[4] = -gy[4];
                    }
                }
                // moment closure, moments, equilibria and collision for both nodes
                close_collide_pair<CLOSURE, COUPLING, W>(f, gx, gy, p, bottom, top);
                const int64_t q = ((int64_t)y * nx + x0) / 2 + tid;  // the pair's word in every plane
                uint32_t* fo = reinterpret_cast<uint32_t*>(fout);
                uint32_t* go = reinterpret_cast<uint32_t*>(gout);
                const int64_t NP = N / 2;
#pragma unroll
                for (int a = 0; a < 9; ++a) fo[a * NP + q] = P::pack(f[a].x, f[a].y);
#pragma unroll
                for (int a = 0; a < 5; ++a) go[a * NP + q] = P::pack(gx[a].x, gx[a].y);
#pragma unroll
                for (int a = 0; a < 5; ++a) go[(5 + a) * NP + q] = P::pack(gy[a].x, gy[a].y);
            };
            if (bottom || top)
                body(std::true_type{});
            else
                body(std::false_type{});
        }
    }
}


// Phase 0 of the in-place pair of steps (lks_aa.cuh) for 16-bit storage, staged the same way.  The
// rows are interleaved (32-bit word w of a row holds nodes x = w and x = w + nx/2), so a shift by one
// node is a shift by one word, with the two halves swapped across the periodic row edge.  A task is
// kSegX/2 words of one row; the producer stages, for each slot, the words the task's nodes pull from
// (row y - e_y; link wall rows their own row of the opposite plane; moment wall rows nothing) with
// 16-byte halos as above.  Each consumer thread takes one word (two nodes), collides them as a
// float2 and pushes every direction b into plane bbar at x + e_b (a direction that would leave
// through a wall into its own plane b of its own word), as the pair kernel does.  Race freedom: the
// location a node pulls from in direction c, plane c at x - e_c, is written in this phase only by
// that node (its push of direction cbar), after its read; halo words a task stages but does not use
// belong to other nodes, and it never writes them.
template <typename S, int CLOSURE, int COUPLING>
__global__ void __launch_bounds__(kThreads, 1) step_kernel_aa_staged(S* __restrict__ fb, S* __restrict__ gb,
                                                                      const StepParams<float> p, int* err) {
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t* full = reinterpret_cast<uint64_t*>(sm);
    uint64_t* empty = full + kStagesTB;
    uint32_t* stage0 = reinterpret_cast<uint32_t*>(sm + 128);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ny = p.ny, H = p.nx / 2;              // words per row
    const int64_t NP = p.N / 2;                     // words per plane
    constexpr int kSegW = kSegX / 2;
    const int nseg = (H + kSegW - 1) / kSegW;
    const int64_t ntask = (int64_t)ny * nseg;
    const int64_t G = gridDim.x, t0 = blockIdx.x;
    const int64_t nmine = t0 < ntask ? (ntask - 1 - t0) / G + 1 : 0;
    uint32_t* fw = reinterpret_cast<uint32_t*>(fb);
    uint32_t* gw = reinterpret_cast<uint32_t*>(gb);
    if (tid == 0) {
        for (int s = 0; s < kStagesTB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        mbar_init_fence();
    }
    __syncthreads();

    if (warp == kConsumerWarps) {  // producer: lane k < 19 fetches slot k
        const int k = lane < kSlots ? lane : 0;
        const int a = dir_of(k), ex = ex9(a), ey = ey9(a);
        const uint32_t* base = k < 9 ? fw : gw;
        const uint32_t* bn = base + (int64_t)plane_of(k, a) * NP;
        const uint32_t* bw = base + (int64_t)plane_of(k, opp9(a)) * NP;
        int64_t it = 0;
        for (; it < nmine; ++it) {
            const int s = (int)(it % kStagesTB);
            const int64_t u = it / kStagesTB;
            if (u > 0 && !mbar_wait_bounded(&empty[s], (uint32_t)(u - 1) & 1u, kWaitNs)) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            const int64_t t = t0 + it * G;
            const int y = (int)(t / nseg), w0 = (int)(t % nseg) * kSegW;
            const int TW = min(kSegW, H - w0);
            const bool wall = (ey == 1 && y == 0) || (ey == -1 && y == ny - 1);
            uint32_t* dst = stage0 + s * kStageW + k * kSlotW;
            // this lane's copies: (global word offset, shared word offset, words)
            int64_t g0 = 0, g1 = 0, g2 = 0;
            int d0 = 0, d1 = 0, d2 = 0, n0 = 0, n1 = 0, n2 = 0;
            if (lane < kSlots) {
                if (wall) {
                    if (CLOSURE == 0) g0 = (int64_t)y * H + w0, d0 = kHaloW, n0 = TW;
                } else {
                    const int64_t row = (int64_t)(y - ey) * H;
                    if (ex == 0) {
                        g0 = row + w0, d0 = kHaloW, n0 = TW;
                    } else if (w0 >= kHaloW && w0 + TW + kHaloW <= H) {  // both halos in one copy
                        g0 = row + w0 - kHaloW, d0 = 0, n0 = TW + 2 * kHaloW;
                    } else {
                        g0 = row + w0, d0 = kHaloW, n0 = TW;
                        if (ex == 1) g1 = row + (w0 == 0 ? H - kHaloW : w0 - kHaloW), d1 = 0, n1 = kHaloW;
                        else g2 = row + (w0 + TW == H ? 0 : w0 + TW), d2 = kHaloW + TW, n2 = kHaloW;
                    }
                }
            }
            const uint32_t mine = 4u * (uint32_t)(n0 + n1 + n2);
            const uint32_t bytes = __reduce_add_sync(0xffffffffu, mine);
            if (lane == 0) mbar_arrive_expect_tx(&full[s], bytes);
            __syncwarp();
            const uint32_t* src = (wall && CLOSURE == 0) ? bw : bn;
            if (n0) bulk_g2s(dst + d0, src + g0, 4u * n0, &full[s]);
            if (n1) bulk_g2s(dst + d1, src + g1, 4u * n1, &full[s]);
            if (n2) bulk_g2s(dst + d2, src + g2, 4u * n2, &full[s]);
        }
        for (int s = 0; s < kStagesTB; ++s) {
            if (it <= s) continue;
            const int64_t u_last = (it - 1 - s) / kStagesTB;
            if (!mbar_wait_bounded(&full[s], (uint32_t)u_last & 1u, kWaitNs) && lane == 0) atomicExch(err, 1);
        }
        return;
    }

    uint32_t* scr = stage0 + kStagesTB * kStageW + warp * kScratchW;
    typedef Packed<S> P;
    const int xw = kHaloW + tid;
    for (int64_t it = 0; it < nmine; ++it) {
        const int s = (int)(it % kStagesTB);
        if (!mbar_wait_bounded(&full[s], (uint32_t)(it / kStagesTB) & 1u, kWaitNs)) {
            atomicExch(err, 1);
            break;
        }
        const int64_t t = t0 + it * G;
        const int y = (int)(t / nseg), w0 = (int)(t % nseg) * kSegW;
        const int TW = min(kSegW, H - w0);
        const bool active = tid < TW;
        {
            const bool bottom = (y == 0), top = (y == ny - 1);
            const uint32_t* st = stage0 + s * kStageW;
            const int w = w0 + tid;                           // the thread's word in its row
            const bool sm = (w == 0), sp = (w == H - 1);      // halves swap across the row edge
            const int wm = sm ? H - 1 : w - 1, wp = sp ? 0 : w + 1;
            auto body = [&](auto walls) {
                constexpr bool W = decltype(walls)::value;
                if (active) {
#pragma unroll
                    for (int k = 0; k < kSlots; ++k) {
                        const int a = dir_of(k), ex = ex9(a), ey = ey9(a);
                        const bool wall = W && ((ey == 1 && bottom) || (ey == -1 && top));
                        const uint32_t* row = st + k * kSlotW;
                        uint32_t u;
                        if (wall || ex == 0)
                            u = row[xw];
                        else if (ex == 1)  // nodes x - 1: the word before (swapped across the left edge)
                            u = sm ? __byte_perm(row[xw - 1], 0, 0x1032) : row[xw - 1];
                        else  // nodes x + 1: the word after (swapped across the right edge)
                            u = sp ? __byte_perm(row[xw + 1], 0, 0x1032) : row[xw + 1];
                        scr[k * 32 + lane] = u;
                    }
                }
                // release the stage at once, as the two-buffer kernel does
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
                if (!active) return;
                float2 v[kSlots];
#pragma unroll
                for (int k = 0; k < kSlots; ++k) {
                    const uint32_t u = scr[k * 32 + lane];
                    v[k] = P::pair(u);
                }
                float2 f[9], gx[5], gy[5];
#pragma unroll
                for (int a = 0; a < 9; ++a) f[a] = v[a];
#pragma unroll
                for (int a = 0; a < 5; ++a) {
                    gx[a] = v[9 + a];
                    gy[a] = v[14 + a];
                }
                if (W && CLOSURE == 0) {
                    if (bottom) {
                        const WallCoef<float>& wc = p.bot;
                        f[5] = f[5] + wc.du;
                        f[6] = f[6] - wc.du;
                        gx[2] = ffma(wc.r, gx[2], wc.kx);
                        gy[2] = -gy[2];
                    }
                    if (top) {
                        const WallCoef<float>& wc = p.top;
                        f[7] = f[7] - wc.du;
                        f[8] = f[8] + wc.du;
                        gx[4] = ffma(wc.r, gx[4], wc.kx);
                        gy[4] = -gy[4];
                    }
                }
                close_collide_pair<CLOSURE, COUPLING, W>(f, gx, gy, p, bottom, top);
                // push: direction b -> plane bbar at x + e_b; through a wall -> plane b, own word
                const int64_t rc = (int64_t)y * H, rs = rc - H, rn = rc + H;
                auto put = [&](uint32_t* at, bool swap, float2 q) { *at = swap ? P::pack(q.y, q.x) : P::pack(q.x, q.y); };
                put(fw + 0 * NP + rc + w, false, f[0]);
                put(fw + 3 * NP + rc + wp, sp, f[1]);
                put(fw + 1 * NP + rc + wm, sm, f[3]);
                put(gw + 0 * NP + rc + w, false, gx[0]);
                put(gw + 3 * NP + rc + wp, sp, gx[1]);
                put(gw + 1 * NP + rc + wm, sm, gx[3]);
                put(gw + 5 * NP + rc + w, false, gy[0]);
                put(gw + 8 * NP + rc + wp, sp, gy[1]);
                put(gw + 6 * NP + rc + wm, sm, gy[3]);
                if (!top) {
                    put(fw + 4 * NP + rn + w, false, f[2]);
                    put(fw + 7 * NP + rn + wp, sp, f[5]);
                    put(fw + 8 * NP + rn + wm, sm, f[6]);
                    put(gw + 4 * NP + rn + w, false, gx[2]);
                    put(gw + 9 * NP + rn + w, false, gy[2]);
                } else {
                    put(fw + 2 * NP + rc + w, false, f[2]);
                    put(fw + 5 * NP + rc + w, false, f[5]);
                    put(fw + 6 * NP + rc + w, false, f[6]);
                    put(gw + 2 * NP + rc + w, false, gx[2]);
                    put(gw + 7 * NP + rc + w, false, gy[2]);
                }
                if (!bottom) {
                    put(fw + 2 * NP + rs + w, false, f[4]);
                    put(fw + 5 * NP + rs + wm, sm, f[7]);
                    put(fw + 6 * NP + rs + wp, sp, f[8]);
                    put(gw + 2 * NP + rs + w, false, gx[4]);
                    put(gw + 7 * NP + rs + w, false, gy[4]);
                } else {
                    put(fw + 4 * NP + rc + w, false, f[4]);
                    put(fw + 7 * NP + rc + w, false, f[7]);
                    put(fw + 8 * NP + rc + w, false, f[8]);
                    put(gw + 4 * NP + rc + w, false, gx[4]);
                    put(gw + 9 * NP + rc + w, false, gy[4]);
                }
            };
            if (bottom || top)
                body(std::true_type{});
            else
                body(std::false_type{});
        }
    }
}

// Failure detection without a GPU fault: one warp waits, with the staged kernels' bounded wait, on
// a freshly initialised mbarrier that nothing arrives on (its first phase never completes), gives
// up after limit_ns and records the timeout in *err as a staged step's wait would.  No copy is in
// flight to that barrier, so returning is safe.
__global__ void wait_timeout_probe_kernel(int* err, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncwarp();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit_ns)) atomicExch(err, 1);
}

template <typename K>
cudaError_t prepare_kernel(K kernel, int* blocks, size_t smem = kSmem) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, smem);
    if (e == cudaSuccess && occ < 1) e = cudaErrorInvalidConfiguration;
    *blocks = occ;
    return e;
}

// Every closure / coupling instance of the two-buffer kernel (inplace = 0) or of the in-place
// phase-0 kernel (inplace = 1); *blocks = the smallest number resident per SM.
template <typename S>
cudaError_t prepare_typed(int inplace, int* blocks) {
    int b[4] = {0, 0, 0, 0};
    cudaError_t e;
    if (inplace) {
        e = prepare_kernel(step_kernel_aa_staged<S, 0, 0>, &b[0], kSmemTB);
        if (e == cudaSuccess) e = prepare_kernel(step_kernel_aa_staged<S, 1, 0>, &b[1], kSmemTB);
        if (e == cudaSuccess) e = prepare_kernel(step_kernel_aa_staged<S, 0, 1>, &b[2], kSmemTB);
        if (e == cudaSuccess) e = prepare_kernel(step_kernel_aa_staged<S, 1, 1>, &b[3], kSmemTB);
    } else {
        e = prepare_kernel(step_kernel_staged<S, 0, 0>, &b[0], kSmemTB);
        if (e == cudaSuccess) e = prepare_kernel(step_kernel_staged<S, 1, 0>, &b[1], kSmemTB);
        if (e == cudaSuccess) e = prepare_kernel(step_kernel_staged<S, 0, 1>, &b[2], kSmemTB);
        if (e == cudaSuccess) e = prepare_kernel(step_kernel_staged<S, 1, 1>, &b[3], kSmemTB);
    }
    *blocks = std::min(std::min(b[0], b[1]), std::min(b[2], b[3]));
    return e;
}

template <typename S>
void launch_typed_aa_staged(void* f, void* g, const StepParams<float>& p, int closure, const StagedStep& ss,
                            cudaStream_t st) {
    const int64_t ntask = (int64_t)p.ny * ((p.nx / 2 + kSegX / 2 - 1) / (kSegX / 2));
    const unsigned grid = (unsigned)std::min<int64_t>(ntask, ss.grid);
    S* fb = (S*)f;
    S* gb = (S*)g;
    if (p.coupling == 0) {
        if (closure == 0) step_kernel_aa_staged<S, 0, 0><<<grid, kThreads, kSmemTB, st>>>(fb, gb, p, ss.err);
        else step_kernel_aa_staged<S, 1, 0><<<grid, kThreads, kSmemTB, st>>>(fb, gb, p, ss.err);
    } else {
        if (closure == 0) step_kernel_aa_staged<S, 0, 1><<<grid, kThreads, kSmemTB, st>>>(fb, gb, p, ss.err);
        else step_kernel_aa_staged<S, 1, 1><<<grid, kThreads, kSmemTB, st>>>(fb, gb, p, ss.err);
    }
}

template <typename S>
void launch_typed_staged(const void* fin, const void* gin, void* fout, void* gout, const StepParams<float>& p,
                         int closure, const StagedStep& ss, cudaStream_t st) {
    const int64_t ntask = (int64_t)p.ny * ((p.nx + kSegX - 1) / kSegX);
    const unsigned grid = (unsigned)std::min<int64_t>(ntask, ss.grid);
    const S* fi = (const S*)fin;
    const S* gi = (const S*)gin;
    S* fo = (S*)fout;
    S* go = (S*)gout;
    if (p.coupling == 0) {
        if (closure == 0) step_kernel_staged<S, 0, 0><<<grid, kThreads, kSmemTB, st>>>(fi, gi, fo, go, p, ss.err);
        else step_kernel_staged<S, 1, 0><<<grid, kThreads, kSmemTB, st>>>(fi, gi, fo, go, p, ss.err);
    } else {
        if (closure == 0) step_kernel_staged<S, 0, 1><<<grid, kThreads, kSmemTB, st>>>(fi, gi, fo, go, p, ss.err);
        else step_kernel_staged<S, 1, 1><<<grid, kThreads, kSmemTB, st>>>(fi, gi, fo, go, p, ss.err);
    }
}

}  // namespace

bool staged_step_applies(int storage, int nx, int inplace) {
    (void)inplace;  // two buffers: the whole step; in place: phase 0 of each pair
    return storage >= 2 && nx % 8 == 0 && nx >= kSegX;
}

cudaError_t prepare_staged_step(int storage, int inplace, unsigned* grid) {
    int dev = 0, sms = 0, blocks = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = storage == 2 ? prepare_typed<__nv_bfloat16>(inplace, &blocks) : prepare_typed<__half>(inplace, &blocks);
    *grid = (unsigned)(sms * blocks);
    return e;
}

cudaError_t launch_wait_timeout_probe(int* err, uint64_t limit_ns, cudaStream_t st) {
    wait_timeout_probe_kernel<<<1, 32, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}

cudaError_t launch_step_aa_staged(int storage, int closure, void* f, void* g, const StepParams<float>& p,
                                  const StagedStep& ss, cudaStream_t st) {
    if (storage == 2)
        launch_typed_aa_staged<__nv_bfloat16>(f, g, p, closure, ss, st);
    else
        launch_typed_aa_staged<__half>(f, g, p, closure, ss, st);
    return cudaGetLastError();
}

cudaError_t launch_step_staged(int storage, int closure, const void* fin, const void* gin, void* fout, void* gout,
                               const StepParams<float>& p, const StagedStep& ss, cudaStream_t st) {
    if (storage == 2)
        launch_typed_staged<__nv_bfloat16>(fin, gin, fout, gout, p, closure, ss, st);
    else
        launch_typed_staged<__half>(fin, gin, fout, gout, p, closure, ss, st);
    return cudaGetLastError();
}

}  // namespace lks
