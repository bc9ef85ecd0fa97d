// lks_internal.h -- host-side declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "lks_device.cuh"

namespace lks {

template <typename C>
inline StepParams<C> convert_params(const StepParams<double>& d) {
    StepParams<C> o;
    o.nx = d.nx;
    o.ny = d.ny;
    o.N = d.N;
    o.omega_f = (C)d.omega_f;
    o.omega_m = (C)d.omega_m;
    o.src_coef = (C)d.src_coef;
    o.Fx = (C)d.Fx;
    o.B0 = (C)d.B0;
    o.om1f = (C)d.om1f;
    o.om1m = (C)d.om1m;
    o.owf0 = (C)d.owf0;
    o.owf1 = (C)d.owf1;
    o.owf5 = (C)d.owf5;
    o.owm0 = (C)d.owm0;
    o.owm1 = (C)d.owm1;
    o.sw0 = (C)d.sw0;
    o.sw1 = (C)d.sw1;
    o.sw5 = (C)d.sw5;
    o.src3 = (C)d.src3;
    o.coupling = d.coupling;
    const WallCoef<double>* src[2] = {&d.bot, &d.top};
    WallCoef<C>* dst[2] = {&o.bot, &o.top};
    for (int k = 0; k < 2; ++k) {
        dst[k]->r = (C)src[k]->r;
        dst[k]->bc = (C)src[k]->bc;
        dst[k]->kx = (C)src[k]->kx;
        dst[k]->du = (C)src[k]->du;
        dst[k]->U = (C)src[k]->U;
    }
    return o;
}

// Step parameters (relaxation rates, force, field and both walls' closure coefficients) of a
// channel; c = INFINITY selects each closure's perfectly conducting limit.
StepParams<double> make_step_params(int nx, int ny, int closure, double tau_f, double tau_m, double B0, double Fx,
                                    double c_bot, double c_top, double u_bot, double u_top, int coupling = 0);

// Bytes per stored population for each lks_storage value.
inline size_t storage_bytes(int storage) { return storage == 0 ? 8 : (storage == 1 ? 4 : 2); }

// Storage order of a single lattice's populations: an in-place handle with 16-bit storage and even
// nx keeps every row interleaved for its two-nodes-per-thread kernels (32-bit word w holds nodes
// x = w and x = w + nx/2, so a shift by one node is a shift by one word); the value is the row
// length the readout kernels need (0: plain node order, all other handles).
inline int interleave_row(int storage, int nx, int inplace) {
    return (inplace && storage >= 2 && (nx % 2) == 0) ? nx : 0;
}

// The staged 16-bit steps (lks_step_staged.cu): rows staged through shared memory by bulk copies.
// They apply to 16-bit storage with nx a multiple of 8 and nx >= 1024: the whole step of a
// two-buffer handle, phase 0 of an in-place handle's pair of steps.  err is a device word set when
// one of their bounded waits runs out, grid the number of resident blocks.
struct StagedStep {
    int* err;
    unsigned grid;
};
bool staged_step_applies(int storage, int nx, int inplace);
// Opt the storage type's staged kernels (two-buffer or in-place) into their shared memory (before any
// graph capture) and return the grid that keeps one wave of blocks resident.
cudaError_t prepare_staged_step(int storage, int inplace, unsigned* grid);
// One warp that waits at most limit_ns on an mbarrier nothing completes, then sets *err (self-test of
// the bounded waits of the staged kernels).
cudaError_t launch_wait_timeout_probe(int* err, uint64_t limit_ns, cudaStream_t st);

cudaError_t launch_step_staged(int storage, int closure, const void* fin, const void* gin, void* fout, void* gout,
                               const StepParams<float>& p, const StagedStep& ss, cudaStream_t st);
cudaError_t launch_step_aa_staged(int storage, int closure, void* f, void* g, const StepParams<float>& p,
                                  const StagedStep& ss, cudaStream_t st);

// One fused step: (fin, gin) -> (fout, gout) on stream st; with ss, 16-bit storage takes the staged
// kernel where it applies.
cudaError_t launch_step(int storage, int closure, const void* fin, const void* gin, void* fout, void* gout,
                        const StepParams<double>& p, cudaStream_t st, const StagedStep* ss = nullptr);
// In-place (one-buffer) step, phase 0 or 1 of a pair (lks_aa.cuh); f, g are the single buffers.
cudaError_t launch_step_aa(int storage, int closure, int phase, void* f, void* g, const StepParams<double>& pd,
                           cudaStream_t st, const StagedStep* ss = nullptr);

// Initial equilibrium state (deviation form) with the counter-based perturbation.
cudaError_t launch_init(int storage, void* f, void* g, int nx, int ny, double B0, uint64_t seed, double amp,
                        cudaStream_t st, int ilv = 0);

// Moments of a stored state: out[m*N + n] (what = 0) or x-averaged profiles out[m*ny + j] (what = 1).
// coupling / tau_m: the moment model of the state (0: Maxwell stress; 1: Lorentz force, which needs tau_m).
cudaError_t launch_moments(int storage, const void* f, const void* g, int nx, int ny, double B0, double Fx,
                           int what, double* out, cudaStream_t st, int coupling = 0, double tau_m = 1.0,
                           int ilv = 0);

// The device address of the host array at p if conversion kernels may access it directly (page-locked
// memory, LKS_HOST_STAGING unset or "0"); nullptr otherwise.
void* host_direct_ptr(const void* p);

// Per-node moments of the M nodes n0 .. n0+M-1 of an N-node state: out[m*M + i] for node n0 + i.
cudaError_t launch_node_moments(int storage, const void* f, const void* g, int64_t N, int64_t n0, int64_t M,
                                double B0, double Fx, double* out, cudaStream_t st, int coupling = 0,
                                double tau_m = 1.0, int ilv = 0);

// Residual partial sums: nblk blocks write partial[4*blk + k] = (sum du^2, sum u^2, sum db^2, sum b^2)
// and refresh the snapshot snap[0..N) = u_x, snap[N..2N) = B_x; then one block reduces in fixed order
// into out[0..4).  residual_blocks(N) never exceeds kResidualMaxBlocks (8 blocks per SM on 152 SMs).
constexpr int kResidualMaxBlocks = 1216;
int residual_blocks(int64_t N);

// Steady-state bookkeeping shared by lks_run_to_steady, lks3_run_to_steady and the batch engine.
// A run is STALLED when its residual has not reached a new minimum for kStallChecks checks in a row
// while already below the rounding floor of the storage type (1e-12 FP64, 1e-4 FP32, 1e-2 16-bit);
// the long window keeps slowly converging runs (residual falling by well under 1 % per check and
// jittering) from being stopped early.
constexpr int kStallChecks = 1000;
inline double stall_floor(int storage) { return storage == 0 ? 1e-12 : (storage == 1 ? 1e-4 : 1e-2); }
// A residual of exactly 0 means that u_x and B_x did not change by one bit over a whole check
// interval.  On a channel driven by a body force or a moving wall, with FP32 or 16-bit storage, that
// is the state stagnating because the per-step increments fell below the resolution of the stored
// deviations -- not convergence: the profile can be far from the steady solution.  It is reported as
// a stall.  (FP64's resolution is far below any tolerance a caller can ask for, and an undriven
// channel has no increment to lose.)
inline bool zero_residual_is_stall(int storage, double Fx, double u_bot, double u_top) {
    return storage != 0 && (Fx != 0.0 || u_bot != 0.0 || u_top != 0.0);
}
cudaError_t launch_residual(int storage, const void* f, const void* g, int nx, int ny, double B0, double Fx,
                            double* snap, double* partial, double* out, cudaStream_t st, int coupling = 0,
                            double tau_m = 1.0, int ilv = 0);
cudaError_t launch_snapshot(int storage, const void* f, const void* g, int nx, int ny, double B0, double Fx,
                            double* snap, cudaStream_t st, int coupling = 0, double tau_m = 1.0, int ilv = 0);

// FP64 absolute populations <-> stored deviations, for the nodes n0 .. n0 + M - 1 of an N-node lattice;
// fabs / gabs hold those nodes in planes of stride M (9 and 10 planes).
cudaError_t launch_to_abs(int storage, const void* f, const void* g, int64_t N, int64_t n0, int64_t M, double B0,
                          double* fabs, double* gabs, cudaStream_t st, int coupling = 0, int ilv = 0);
cudaError_t launch_from_abs(int storage, const double* fabs, const double* gabs, int64_t N, int64_t n0, int64_t M,
                            double B0, void* f, void* g, cudaStream_t st, int coupling = 0, int ilv = 0);

}  // namespace lks
