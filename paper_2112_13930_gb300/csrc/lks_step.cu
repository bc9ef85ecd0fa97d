// lks_step.cu -- the fused collide-stream kernel (hot path steps a1-a6) of one lattice.
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

namespace lks {

template <typename S, typename C, int CLOSURE>
__global__ void __launch_bounds__(256) step_kernel(const S* __restrict__ fin, const S* __restrict__ gin,
                                                   S* __restrict__ fout, S* __restrict__ gout,
                                                   const StepParams<C> p) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    step_node<S, C, CLOSURE, true>(fin, gin, fout, gout, p, n);
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
