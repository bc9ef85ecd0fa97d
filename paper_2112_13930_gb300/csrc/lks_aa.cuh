// lks_aa.cuh -- the in-place ("AA pattern") form of the fused step: one population buffer
// instead of two, at the same bytes moved per step.
//
// Steps go in pairs.  With A(x)_a the post-collision population of node x in direction a (what
// the two-buffer step stores in plane a at x) and abar the opposite direction:
//
//   phase 0 (first step of a pair): every node pulls A(x - e_a)_a from plane a at x - e_a
//     exactly as the two-buffer step does (including the wall closures), collides, and writes
//     each new A(x)_b into plane bbar at x + e_b.  A population that would leave through a wall
//     (x + e_b outside) is written, unmodified, into plane b at x itself.
//   phase 1 (second step): every node reads its pulled populations from its own slots --
//     direction a from plane abar at x -- collides, and writes A(x)_a into plane a at x.
//
// After phase 1 the buffer holds the post-collision state in the natural layout, bit for bit the
// state the two-buffer step reaches after the same number of steps, so every readout kernel
// works on it unchanged.  Race freedom: in phase 0 the location (plane c, node y) is read by the
// node y + e_c only (its pull in direction c) and written by that same node (its population in
// direction cbar goes to y = node + e_cbar); the wall slots a node writes are the ones its own
// link closure reads and that nobody else touches.  In phase 1 every node touches only its own
// slots.  So a thread reads all its values before it writes and no two threads share a location.
//
// Wall closures in phase 1: the slots of the incoming populations of a wall node hold the raw
// outgoing ones of the previous phase (as written above), so the link-based closure (Sec. VI,
// App. B.1) applies the same transformation the two-buffer step applies to the node's own
// outgoing populations -- bounce-back with Ladd's moving-wall term for f, the weighted
// (anti-)bounce-back of Eq. (movingwalllinkbasedclosure) for g -- to the value it reads; the
// moment-based closure (Sec. VII, App. A, B.2) reconstructs them from the known populations as
// in the two-buffer step.  Both phases therefore perform the two-buffer step's arithmetic on the
// same inputs.
#pragma once
#include "lks_device.cuh"

namespace lks {

// Phase 0: pull (as step_node_with), close, collide, push to the neighbours' opposite slots.
// L: coherent loads (the buffer is written during the kernel); L2-only loads where the threads
// of one instance span several SMs.
template <typename S, typename C, int CLOSURE, int COUPLING, typename L = Loader<S, C, false>>
__device__ __forceinline__ void aa_node_pull_push(S* fb, S* gb, const StepParams<C>& p, int64_t n, int i, int j) {
    const int nx = p.nx;
    const int64_t N = p.N;
    const int64_t rc = n - i;
    const int64_t rs = rc - nx;
    const int64_t rn = rc + nx;
    const int im = (i == 0) ? nx - 1 : i - 1;
    const int ip = (i == nx - 1) ? 0 : i + 1;
    const bool bottom = (j == 0);
    const bool top = (j == p.ny - 1);

    C f[9], gx[5], gy[5];
    S* gxb = gb;
    S* gyb = gb + 5 * N;
    f[0] = L::ld(fb + 0 * N + rc + i);
    f[1] = L::ld(fb + 1 * N + rc + im);
    f[3] = L::ld(fb + 3 * N + rc + ip);
    gx[0] = L::ld(gxb + 0 * N + rc + i);
    gx[1] = L::ld(gxb + 1 * N + rc + im);
    gx[3] = L::ld(gxb + 3 * N + rc + ip);
    gy[0] = L::ld(gyb + 0 * N + rc + i);
    gy[1] = L::ld(gyb + 1 * N + rc + im);
    gy[3] = L::ld(gyb + 3 * N + rc + ip);
    if (!bottom) {
        f[2] = L::ld(fb + 2 * N + rs + i);
        f[5] = L::ld(fb + 5 * N + rs + im);
        f[6] = L::ld(fb + 6 * N + rs + ip);
        gx[2] = L::ld(gxb + 2 * N + rs + i);
        gy[2] = L::ld(gyb + 2 * N + rs + i);
    }
    if (!top) {
        f[4] = L::ld(fb + 4 * N + rn + i);
        f[7] = L::ld(fb + 7 * N + rn + ip);
        f[8] = L::ld(fb + 8 * N + rn + im);
        gx[4] = L::ld(gxb + 4 * N + rn + i);
        gy[4] = L::ld(gyb + 4 * N + rn + i);
    }
    if (CLOSURE == 0) {
        if (bottom) {
            const WallCoef<C>& w = p.bot;
            f[2] = L::ld(fb + 4 * N + rc + i);
            f[5] = L::ld(fb + 7 * N + rc + i) + w.du;
            f[6] = L::ld(fb + 8 * N + rc + i) - w.du;
            gx[2] = ffma(w.r, L::ld(gxb + 4 * N + rc + i), w.kx);
            gy[2] = -L::ld(gyb + 4 * N + rc + i);
        }
        if (top) {
            const WallCoef<C>& w = p.top;
            f[4] = L::ld(fb + 2 * N + rc + i);
            f[7] = L::ld(fb + 5 * N + rc + i) - w.du;
            f[8] = L::ld(fb + 6 * N + rc + i) + w.du;
            gx[4] = ffma(w.r, L::ld(gxb + 2 * N + rc + i), w.kx);
            gy[4] = -L::ld(gyb + 2 * N + rc + i);
        }
    } else {
        if (bottom) moment_closure_bottom<C, COUPLING>(f, gx, gy, p.bot, p);
        if (top) moment_closure_top<C, COUPLING>(f, gx, gy, p.top, p);
    }
    collide<C, COUPLING>(f, gx, gy, p);
    // push: A_b -> plane bbar at x + e_b; through a wall -> plane b at x
    store_s<S, C>(fb + 0 * N + rc + i, f[0]);
    store_s<S, C>(fb + 3 * N + rc + ip, f[1]);
    store_s<S, C>(fb + 1 * N + rc + im, f[3]);
    store_s<S, C>(gxb + 0 * N + rc + i, gx[0]);
    store_s<S, C>(gxb + 3 * N + rc + ip, gx[1]);
    store_s<S, C>(gxb + 1 * N + rc + im, gx[3]);
    store_s<S, C>(gyb + 0 * N + rc + i, gy[0]);
    store_s<S, C>(gyb + 3 * N + rc + ip, gy[1]);
    store_s<S, C>(gyb + 1 * N + rc + im, gy[3]);
    if (!top) {
        store_s<S, C>(fb + 4 * N + rn + i, f[2]);
        store_s<S, C>(fb + 7 * N + rn + ip, f[5]);
        store_s<S, C>(fb + 8 * N + rn + im, f[6]);
        store_s<S, C>(gxb + 4 * N + rn + i, gx[2]);
        store_s<S, C>(gyb + 4 * N + rn + i, gy[2]);
    } else {
        store_s<S, C>(fb + 2 * N + rc + i, f[2]);
        store_s<S, C>(fb + 5 * N + rc + i, f[5]);
        store_s<S, C>(fb + 6 * N + rc + i, f[6]);
        store_s<S, C>(gxb + 2 * N + rc + i, gx[2]);
        store_s<S, C>(gyb + 2 * N + rc + i, gy[2]);
    }
    if (!bottom) {
        store_s<S, C>(fb + 2 * N + rs + i, f[4]);
        store_s<S, C>(fb + 5 * N + rs + im, f[7]);
        store_s<S, C>(fb + 6 * N + rs + ip, f[8]);
        store_s<S, C>(gxb + 2 * N + rs + i, gx[4]);
        store_s<S, C>(gyb + 2 * N + rs + i, gy[4]);
    } else {
        store_s<S, C>(fb + 4 * N + rc + i, f[4]);
        store_s<S, C>(fb + 7 * N + rc + i, f[7]);
        store_s<S, C>(fb + 8 * N + rc + i, f[8]);
        store_s<S, C>(gxb + 4 * N + rc + i, gx[4]);
        store_s<S, C>(gyb + 4 * N + rc + i, gy[4]);
    }
}

// Phase 1: own slots (direction a from plane abar), close, collide, natural store.
template <typename S, typename C, int CLOSURE, int COUPLING, typename L = Loader<S, C, false>>
__device__ __forceinline__ void aa_node_local(S* fb, S* gb, const StepParams<C>& p, int64_t n, int j) {
    const int64_t N = p.N;
    const bool bottom = (j == 0);
    const bool top = (j == p.ny - 1);
    // moment-based wall rows do not read their unknown incoming slots (they are reconstructed)
    const bool skip_up = CLOSURE == 1 && bottom;   // a = 2, 5, 6 unknown at the bottom wall
    const bool skip_down = CLOSURE == 1 && top;    // a = 4, 7, 8 unknown at the top wall

    C f[9], gx[5], gy[5];
    S* gxb = gb;
    S* gyb = gb + 5 * N;
    f[0] = L::ld(fb + 0 * N + n);
    f[1] = L::ld(fb + 3 * N + n);
    f[3] = L::ld(fb + 1 * N + n);
    gx[0] = L::ld(gxb + 0 * N + n);
    gx[1] = L::ld(gxb + 3 * N + n);
    gx[3] = L::ld(gxb + 1 * N + n);
    gy[0] = L::ld(gyb + 0 * N + n);
    gy[1] = L::ld(gyb + 3 * N + n);
    gy[3] = L::ld(gyb + 1 * N + n);
    if (!skip_up) {
        f[2] = L::ld(fb + 4 * N + n);
        f[5] = L::ld(fb + 7 * N + n);
        f[6] = L::ld(fb + 8 * N + n);
        gx[2] = L::ld(gxb + 4 * N + n);
        gy[2] = L::ld(gyb + 4 * N + n);
    }
    if (!skip_down) {
        f[4] = L::ld(fb + 2 * N + n);
        f[7] = L::ld(fb + 5 * N + n);
        f[8] = L::ld(fb + 6 * N + n);
        gx[4] = L::ld(gxb + 2 * N + n);
        gy[4] = L::ld(gyb + 2 * N + n);
    }
    if (CLOSURE == 0) {
        // the slots hold the node's own raw outgoing populations: same transformation as the
        // two-buffer step's link closure
        if (bottom) {
            const WallCoef<C>& w = p.bot;
            f[5] = f[5] + w.du;
            f[6] = f[6] - w.du;
            gx[2] = ffma(w.r, gx[2], w.kx);
            gy[2] = -gy[2];
        }
        if (top) {
            const WallCoef<C>& w = p.top;
            f[7] = f[7] - w.du;
            f[8] = f[8] + w.du;
            gx[4] = ffma(w.r, gx[4], w.kx);
            gy[4] = -gy[4];
        }
    } else {
        if (bottom) moment_closure_bottom<C, COUPLING>(f, gx, gy, p.bot, p);
        if (top) moment_closure_top<C, COUPLING>(f, gx, gy, p.top, p);
    }
    collide<C, COUPLING>(f, gx, gy, p);
#pragma unroll
    for (int a = 0; a < 9; ++a) store_s<S, C>(fb + a * N + n, f[a]);
#pragma unroll
    for (int a = 0; a < 5; ++a) store_s<S, C>(gxb + a * N + n, gx[a]);
#pragma unroll
    for (int a = 0; a < 5; ++a) store_s<S, C>(gyb + a * N + n, gy[a]);
}

}  // namespace lks
