// lks_step.cu -- the fused collide-stream kernel (hot path steps a1-a6).
//
// One thread per node, nodes numbered n = y*nx + x so that a warp reads 32 consecutive
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

namespace lks {

template <typename S, typename C, int CLOSURE>
__global__ void __launch_bounds__(256) step_kernel(const S* __restrict__ fin, const S* __restrict__ gin,
                                                   S* __restrict__ fout, S* __restrict__ gout,
                                                   const StepParams<C> p) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const int nx = p.nx;
    const int j = (int)(n / nx);
    const int i = (int)(n - (int64_t)j * nx);
    const int64_t N = p.N;
    const int64_t rc = n - i;          // start of row j
    const int64_t rs = rc - nx;        // row j-1
    const int64_t rn = rc + nx;        // row j+1
    const int im = (i == 0) ? nx - 1 : i - 1;
    const int ip = (i == nx - 1) ? 0 : i + 1;
    const bool bottom = (j == 0);
    const bool top = (j == p.ny - 1);

    C f[9], gx[5], gy[5];
    const S* gxin = gin;
    const S* gyin = gin + 5 * N;
    // a1: pull-stream, periodic in x
    f[0] = load_s<S, C>(fin + 0 * N + rc + i);
    f[1] = load_s<S, C>(fin + 1 * N + rc + im);
    f[3] = load_s<S, C>(fin + 3 * N + rc + ip);
    gx[0] = load_s<S, C>(gxin + 0 * N + rc + i);
    gx[1] = load_s<S, C>(gxin + 1 * N + rc + im);
    gx[3] = load_s<S, C>(gxin + 3 * N + rc + ip);
    gy[0] = load_s<S, C>(gyin + 0 * N + rc + i);
    gy[1] = load_s<S, C>(gyin + 1 * N + rc + im);
    gy[3] = load_s<S, C>(gyin + 3 * N + rc + ip);
    if (!bottom) {
        f[2] = load_s<S, C>(fin + 2 * N + rs + i);
        f[5] = load_s<S, C>(fin + 5 * N + rs + im);
        f[6] = load_s<S, C>(fin + 6 * N + rs + ip);
        gx[2] = load_s<S, C>(gxin + 2 * N + rs + i);
        gy[2] = load_s<S, C>(gyin + 2 * N + rs + i);
    }
    if (!top) {
        f[4] = load_s<S, C>(fin + 4 * N + rn + i);
        f[7] = load_s<S, C>(fin + 7 * N + rn + ip);
        f[8] = load_s<S, C>(fin + 8 * N + rn + im);
        gx[4] = load_s<S, C>(gxin + 4 * N + rn + i);
        gy[4] = load_s<S, C>(gyin + 4 * N + rn + i);
    }
    // a2: wall closures
    if (CLOSURE == 0) {
        if (bottom) {
            const WallCoef<C>& w = p.bot;
            f[2] = load_s<S, C>(fin + 4 * N + rc + i);
            f[5] = load_s<S, C>(fin + 7 * N + rc + i) + w.du;
            f[6] = load_s<S, C>(fin + 8 * N + rc + i) - w.du;
            gx[2] = w.r * load_s<S, C>(gxin + 4 * N + rc + i) + w.kx;
            gy[2] = -load_s<S, C>(gyin + 4 * N + rc + i);
        }
        if (top) {
            const WallCoef<C>& w = p.top;
            f[4] = load_s<S, C>(fin + 2 * N + rc + i);
            f[7] = load_s<S, C>(fin + 5 * N + rc + i) - w.du;
            f[8] = load_s<S, C>(fin + 6 * N + rc + i) + w.du;
            gx[4] = w.r * load_s<S, C>(gxin + 2 * N + rc + i) + w.kx;
            gy[4] = -load_s<S, C>(gyin + 2 * N + rc + i);
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

template <typename S, typename C>
static cudaError_t launch_typed(const void* fin, const void* gin, void* fout, void* gout, const StepParams<C>& p,
                                int closure, cudaStream_t st) {
    const int threads = 256;
    const int64_t blocks = (p.N + threads - 1) / threads;
    if (closure == 0)
        step_kernel<S, C, 0><<<(unsigned)blocks, threads, 0, st>>>((const S*)fin, (const S*)gin, (S*)fout,
                                                                    (S*)gout, p);
    else
        step_kernel<S, C, 1><<<(unsigned)blocks, threads, 0, st>>>((const S*)fin, (const S*)gin, (S*)fout,
                                                                    (S*)gout, p);
    return cudaGetLastError();
}

cudaError_t launch_step(int storage, int closure, const void* fin, const void* gin, void* fout, void* gout,
                        const StepParams<double>& pd, cudaStream_t st) {
    if (storage == 0) return launch_typed<double, double>(fin, gin, fout, gout, pd, closure, st);
    StepParams<float> pf = convert_params<float>(pd);
    if (storage == 1) return launch_typed<float, float>(fin, gin, fout, gout, pf, closure, st);
    if (storage == 2) return launch_typed<__nv_bfloat16, float>(fin, gin, fout, gout, pf, closure, st);
    return launch_typed<__half, float>(fin, gin, fout, gout, pf, closure, st);
}

}  // namespace lks
