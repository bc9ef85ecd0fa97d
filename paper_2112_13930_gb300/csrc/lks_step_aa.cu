// lks_step_aa.cu -- kernels of the in-place (one-buffer) step; the per-node work and the proof
// that it reproduces the two-buffer step are in lks_aa.cuh.  Same thread layout as the two-buffer
// kernel: consecutive x positions in consecutive threads, a 2D grid (row = blockIdx.y) for wide
// FP32 / 16-bit lattices and a 1D grid otherwise.
#include "lks_aa.cuh"
#include "lks_internal.h"

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

template <int PHASE>
static cudaError_t launch_aa_phase(int storage, int closure, void* f, void* g, const StepParams<double>& pd,
                                   cudaStream_t st) {
    if (storage == 0) return launch_aa_typed<double, double, PHASE>(f, g, pd, closure, st);
    const StepParams<float> pf = convert_params<float>(pd);
    if (storage == 1) return launch_aa_typed<float, float, PHASE>(f, g, pf, closure, st);
    if (storage == 2) return launch_aa_typed<__nv_bfloat16, float, PHASE>(f, g, pf, closure, st);
    return launch_aa_typed<__half, float, PHASE>(f, g, pf, closure, st);
}

cudaError_t launch_step_aa(int storage, int closure, int phase, void* f, void* g, const StepParams<double>& pd,
                           cudaStream_t st) {
    return phase == 0 ? launch_aa_phase<0>(storage, closure, f, g, pd, st)
                      : launch_aa_phase<1>(storage, closure, f, g, pd, st);
}

}  // namespace lks
