// lks_api.cu -- the C ABI declared in include/lks.h: parameter validation, device memory
// layout, wall-closure coefficients, CUDA-graph stepping, moments and residual calls.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lks.h"
#include "lks_internal.h"

using lks::StepParams;
using lks::WallCoef;

namespace {

thread_local std::string g_last_error = "";
// Captured graphs of 64, 32, ..., 2 steps (even, so a graph returns the state to the buffer it started
// in), one per size and starting buffer, built on first use: lks_step(n) runs n as a few graph
// launches (n = 100: 64 + 32 + 4) plus at most one direct launch, which matters for small lattices
// whose steps cost less than a launch.
constexpr int kGraphSizes = 6;
constexpr int64_t kGraphSteps[kGraphSizes] = {64, 32, 16, 8, 4, 2};
constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// NVTX range around a C-ABI call (visible in Nsight tools; near-free when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

struct Layout {
    size_t f_bytes, g_bytes, off_fa, off_ga, off_fb, off_gb, off_snap, off_partial, off_out, off_prof, off_flag, total;
};

Layout make_layout(const lks_params* p) {
    Layout L;
    const size_t N = (size_t)p->nx * (size_t)p->ny;
    const size_t sb = lks::storage_bytes(p->storage);
    L.f_bytes = align_up(9 * N * sb);
    L.g_bytes = align_up(10 * N * sb);
    size_t o = 0;
    L.off_fa = o; o += L.f_bytes;
    L.off_ga = o; o += L.g_bytes;
    if (p->inplace) {  // one population buffer (in-place pairs of steps)
        L.off_fb = L.off_fa;
        L.off_gb = L.off_ga;
    } else {
        L.off_fb = o; o += L.f_bytes;
        L.off_gb = o; o += L.g_bytes;
    }
    L.off_snap = o; o += align_up(2 * N * sizeof(double));
    L.off_partial = o; o += align_up(4 * (size_t)lks::residual_blocks((int64_t)N) * sizeof(double));
    L.off_out = o; o += align_up(8 * sizeof(double));
    L.off_prof = o; o += align_up(5 * (size_t)p->ny * sizeof(double));
    L.off_flag = o; o += align_up(sizeof(int));  // set by a staged step whose bounded wait ran out
    L.total = o;
    return L;
}

const char* validate(const lks_params* p) {
    if (!p) return "params is NULL";
    if (p->nx < 1) return "nx must be >= 1";
    if (p->closure != LKS_LINK && p->closure != LKS_MOMENT) return "closure must be LKS_LINK or LKS_MOMENT";
    if (p->closure == LKS_LINK && p->ny < 2) return "ny must be >= 2 for the link-based closure";
    if (p->closure == LKS_MOMENT && p->ny < 3) return "ny must be >= 3 for the moment-based closure";
    if (p->storage < LKS_F64 || p->storage > LKS_F16_DEV) return "storage must be one of lks_storage";
    if ((int64_t)p->nx * (int64_t)p->ny > (int64_t)1 << 30) return "nx*ny exceeds 2^30 nodes";
    if (!(p->tau_f > 0.5) || !isfinite(p->tau_f)) return "tau_f must be finite and > 1/2";
    if (!(p->tau_m > 0.5) || !isfinite(p->tau_m)) return "tau_m must be finite and > 1/2";
    if (!isfinite(p->B0) || !isfinite(p->Fx)) return "B0 and Fx must be finite";
    if (!isfinite(p->perturb_amp) || fabs(p->perturb_amp) >= 0.3) return "|perturb_amp| must be < 0.3";
    if (p->coupling != LKS_MAXWELL && p->coupling != LKS_LORENTZ) return "coupling must be LKS_MAXWELL or LKS_LORENTZ";
    if (p->coupling == LKS_LORENTZ && fabs(p->tau_m - 1.0) < 0.05)
        return "the Lorentz-force coupling needs |tau_m - 1| >= 0.05 (J is read back from the stored g)";
    if (p->inplace != 0 && p->inplace != 1) return "inplace must be 0 or 1";
    return nullptr;
}

}  // namespace

namespace lks {

// Closure coefficients of one wall (see WallCoef).  ey = +1 for the bottom wall's incoming
// direction, -1 for the top wall's.  a is the channel half-width of the closure's wall placement.
static WallCoef<double> wall_coef(int closure, double a, double tau_m, double B0, double c, double U, double ey) {
    WallCoef<double> w;
    w.U = U;
    w.du = 6.0 * (1.0 / 36.0) * U;  // 2 w_a e_ax U / c_s^2 for the diagonal links (|e_ax| = 1)
    if (closure == LKS_LINK) {
        // theta = c a / (tau_m - 1/2) (Eq. weightingfactor); r = (theta-1)/(theta+1),
        // s = 2 theta/(theta+1); kx = -s W e_y B0 U / c_sm^2 with W = 1/6 (Eq. movingwalllinkbasedclosure)
        double r, s;
        if (isinf(c)) {
            r = 1.0;
            s = 2.0;
        } else {
            const double theta = c * a / (tau_m - 0.5);
            r = (theta - 1.0) / (theta + 1.0);
            s = 2.0 * theta / (theta + 1.0);
        }
        w.r = r;
        w.bc = 0.0;
        w.kx = -s * (1.0 / 6.0) * ey * B0 * U * 3.0;
    } else {
        // beta = c a / (tau_m c_sm^2): unknown = [(beta-1) opp - (g0+g1+g3) - e_y beta B0 U]/(beta+1)
        // (Eq. momentconstraintgx and Eq. momentbasedclosureformovingwall multiplied through by c a)
        double r, bc, k;
        if (isinf(c)) {
            r = 1.0;
            bc = 0.0;
            k = 1.0;
        } else {
            const double beta = c * a / (tau_m / 3.0);
            r = (beta - 1.0) / (beta + 1.0);
            bc = 1.0 / (beta + 1.0);
            k = beta / (beta + 1.0);
        }
        w.r = r;
        w.bc = bc;
        w.kx = -ey * k * B0 * U;
    }
    return w;
}

StepParams<double> make_step_params(int nx, int ny, int closure, double tau_f, double tau_m, double B0, double Fx,
                                    double c_bot, double c_top, double u_bot, double u_top, int coupling) {
    StepParams<double> s;
    const double a = closure == LKS_LINK ? 0.5 * ny : 0.5 * (ny - 1);
    s.nx = nx;
    s.ny = ny;
    s.N = (int64_t)nx * ny;
    s.omega_f = 1.0 / tau_f;
    s.omega_m = 1.0 / tau_m;
    s.src_coef = 1.0 - 0.5 / tau_f;
    s.Fx = Fx;
    s.B0 = B0;
    s.om1f = 1.0 - s.omega_f;
    s.om1m = 1.0 - s.omega_m;
    s.owf0 = s.omega_f * (4.0 / 9.0);
    s.owf1 = s.omega_f * (1.0 / 9.0);
    s.owf5 = s.omega_f * (1.0 / 36.0);
    s.owm0 = s.omega_m * (1.0 / 3.0);
    s.owm1 = s.omega_m * (1.0 / 6.0);
    s.sw0 = s.src_coef * 3.0 * Fx * (4.0 / 9.0);
    s.sw1 = s.src_coef * 3.0 * Fx * (1.0 / 9.0);
    s.sw5 = s.src_coef * 3.0 * Fx * (1.0 / 36.0);
    s.src3 = 3.0 * s.src_coef;
    s.coupling = coupling;
    s.bot = wall_coef(closure, a, tau_m, B0, c_bot, u_bot, +1.0);
    s.top = wall_coef(closure, a, tau_m, B0, c_top, u_top, -1.0);
    return s;
}

// The device address through which a kernel may read or write the host array at p directly:
// page-locked memory (cudaHostAlloc, cudaHostRegister) is mapped into the device's address space,
// and kernels stream it at the rate of the host link (NVLink-C2C on a Grace host: 211 GB/s in,
// 194 GB/s out, as fast as the copy engine).  nullptr for pageable memory, whose pages the copy
// engine handles far better (a kernel's first touch of a fresh pageable page faults it in through
// the host page tables one page at a time), and when LKS_HOST_STAGING=1 forces the staged copies.
void* host_direct_ptr(const void* p) {
    const char* env = getenv("LKS_HOST_STAGING");
    if (!p || (env && env[0] && strcmp(env, "0") != 0)) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace lks

struct lks_handle {
    lks_params p;
    Layout L;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    char* base = nullptr;
    bool owns = false;
    void* f[2] = {nullptr, nullptr};
    void* g[2] = {nullptr, nullptr};
    int cur = 0;
    double* snap = nullptr;
    double* partial = nullptr;
    double* dout = nullptr;
    double* prof = nullptr;
    double* state_stage = nullptr;  // 19 * min(N, 2^20) doubles for state and moment transfers, on first use
    double* host_small = nullptr;  // pinned 8 doubles
    int* flag = nullptr;
    bool staged = false;              // 16-bit, nx % 8 == 0, nx >= 1024: the staged kernels
    lks::StagedStep ss = {nullptr, 0};
    double c_bot = 0.0, c_top = 0.0, u_bot = 0.0, u_top = 0.0;
    StepParams<double> sp;
    int64_t steps = 0;
    cudaGraphExec_t graph[kGraphSizes][2] = {};
    bool graphs_disabled = false;
    std::string err;
};

namespace {

lks_status fail(lks_handle* h, lks_status s, const std::string& msg) {
    if (h)
        h->err = msg;
    else
        g_last_error = msg;
    return s;
}

lks_status cuda_fail(lks_handle* h, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, LKS_ECUDA, m);
}

// After a synchronisation: LKS_ETIMEOUT if a staged step gave up waiting for its copies.
lks_status staged_check(lks_handle* h, const char* where) {
    if (!h->staged) return LKS_OK;
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, h->flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, where);
    if (v) return fail(h, LKS_ETIMEOUT, std::string(where) + ": a staged step's shared-memory wait ran out");
    return LKS_OK;
}

void refresh_params(lks_handle* h) {
    const lks_params& p = h->p;
    h->sp = lks::make_step_params(p.nx, p.ny, p.closure, p.tau_f, p.tau_m, p.B0, p.Fx, h->c_bot, h->c_top, h->u_bot,
                                  h->u_top, p.coupling);
}

void drop_graphs(lks_handle* h) {
    for (int g = 0; g < kGraphSizes; ++g)
        for (int k = 0; k < 2; ++k)
            if (h->graph[g][k]) {
                cudaGraphExecDestroy(h->graph[g][k]);
                h->graph[g][k] = nullptr;
            }
}

// One step.  Two-buffer handles step from buffer `src` into the other; in-place handles take
// phase `src` of a pair (0: pull and push to the neighbours, 1: own slots) on their one buffer.
cudaError_t step_once(lks_handle* h, int src, cudaStream_t st) {
    if (h->p.inplace)
        return lks::launch_step_aa(h->p.storage, h->p.closure, src, h->f[0], h->g[0], h->sp, st,
                                   h->staged ? &h->ss : nullptr);
    return lks::launch_step(h->p.storage, h->p.closure, h->f[src], h->g[src], h->f[src ^ 1], h->g[src ^ 1], h->sp, st,
                            h->staged ? &h->ss : nullptr);
}

// Capture kGraphSteps[size] steps starting from buffer `start` into an executable graph.
cudaError_t build_graph(lks_handle* h, int size, int start) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    int src = start;
    cudaError_t le = cudaSuccess;
    for (int64_t k = 0; k < kGraphSteps[size] && le == cudaSuccess; ++k) {
        le = step_once(h, src, h->cap_stream);
        src ^= 1;
    }
    e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return le;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&h->graph[size][start], graph, 0);
    cudaGraphDestroy(graph);
    return e;
}


// Otherwise (pageable host arrays) state transfers and per-node host moments convert kStateChunk nodes
// at a time through a staging buffer the handle keeps, so their device memory stays bounded (152 MB)
// whatever the lattice size.
constexpr int64_t kStateChunk = int64_t(1) << 20;

lks_status state_stage(lks_handle* h, int64_t* chunk) {
    const int64_t N = (int64_t)h->p.nx * h->p.ny;
    *chunk = N < kStateChunk ? N : kStateChunk;
    if (!h->state_stage) {
        cudaError_t e = cudaMalloc((void**)&h->state_stage, 19 * (size_t)*chunk * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->state_stage = nullptr;
            return fail(h, LKS_ENOMEM, "cudaMalloc of the FP64 state staging buffer failed");
        }
    }
    return LKS_OK;
}

int ilv_of(const lks_handle* h) { return lks::interleave_row(h->p.storage, h->p.nx, h->p.inplace); }

// Stored state -> FP64 host arrays, M nodes per chunk: one conversion kernel into the staging buffer,
// then one copy per population plane.
cudaError_t staged_to_host(lks_handle* h, double* host_f, double* host_g, int64_t M) {
    const int64_t N = (int64_t)h->p.nx * h->p.ny;
    double* st = h->state_stage;
    cudaError_t e = cudaSuccess;
    for (int64_t n0 = 0; n0 < N && e == cudaSuccess; n0 += M) {
        const int64_t m = N - n0 < M ? N - n0 : M;
        e = lks::launch_to_abs(h->p.storage, h->f[h->cur], h->g[h->cur], N, n0, m, h->p.B0, st, st + 9 * m,
                               h->stream, h->p.coupling, ilv_of(h));
        for (int a = 0; a < 19 && e == cudaSuccess; ++a) {
            double* dst = a < 9 ? host_f + a * N + n0 : host_g + (a - 9) * N + n0;
            e = cudaMemcpyAsync(dst, st + a * m, m * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        }
    }
    return e;
}

// FP64 host arrays -> stored state, M nodes per chunk.
cudaError_t staged_from_host(lks_handle* h, const double* host_f, const double* host_g, int64_t M) {
    const int64_t N = (int64_t)h->p.nx * h->p.ny;
    double* st = h->state_stage;
    cudaError_t e = cudaSuccess;
    for (int64_t n0 = 0; n0 < N && e == cudaSuccess; n0 += M) {
        const int64_t m = N - n0 < M ? N - n0 : M;
        for (int a = 0; a < 19 && e == cudaSuccess; ++a) {
            const double* src = a < 9 ? host_f + a * N + n0 : host_g + (a - 9) * N + n0;
            e = cudaMemcpyAsync(st + a * m, src, m * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        }
        if (e == cudaSuccess)
            e = lks::launch_from_abs(h->p.storage, st, st + 9 * m, N, n0, m, h->p.B0, h->f[h->cur], h->g[h->cur],
                                     h->stream, h->p.coupling, ilv_of(h));
    }
    return e;
}

// Per-node moments -> host array (5 planes of N), M nodes per chunk.
cudaError_t staged_moments_to_host(lks_handle* h, double* host_out, int64_t M) {
    const int64_t N = (int64_t)h->p.nx * h->p.ny;
    double* st = h->state_stage;
    cudaError_t e = cudaSuccess;
    for (int64_t n0 = 0; n0 < N && e == cudaSuccess; n0 += M) {
        const int64_t m = N - n0 < M ? N - n0 : M;
        e = lks::launch_node_moments(h->p.storage, h->f[h->cur], h->g[h->cur], N, n0, m, h->p.B0, h->p.Fx, st,
                                     h->stream, h->p.coupling, h->p.tau_m, ilv_of(h));
        for (int k = 0; k < 5 && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(host_out + k * N + n0, st + k * m, m * sizeof(double), cudaMemcpyDeviceToHost,
                                h->stream);
    }
    return e;
}

}  // namespace

extern "C" {

size_t lks_footprint_bytes(const lks_params* p) {
    if (validate(p)) return 0;
    return make_layout(p).total;
}

lks_status lks_create(const lks_params* p, lks_handle** out) {
    NvtxRange nvtx_range("lks_create");
    if (!out) return fail(nullptr, LKS_EINVAL, "out is NULL");
    *out = nullptr;
    if (const char* m = validate(p)) return fail(nullptr, LKS_EINVAL, m);
    lks_handle* h = new (std::nothrow) lks_handle();
    if (!h) return fail(nullptr, LKS_ENOMEM, "host allocation of the handle failed");
    h->p = *p;
    h->L = make_layout(p);
    h->stream = (cudaStream_t)p->cuda_stream;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(nullptr, e, "cudaGetDevice");
    }
    if (p->dev_buffer) {
        if (p->dev_buffer_bytes < h->L.total || ((uintptr_t)p->dev_buffer % kAlign) != 0) {
            delete h;
            return fail(nullptr, LKS_ENOMEM, "dev_buffer is smaller than lks_footprint_bytes() or not 256-byte aligned");
        }
        h->base = (char*)p->dev_buffer;
        h->owns = false;
    } else {
        e = cudaMalloc((void**)&h->base, h->L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return fail(nullptr, LKS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        h->owns = true;
    }
    h->f[0] = h->base + h->L.off_fa;
    h->g[0] = h->base + h->L.off_ga;
    h->f[1] = h->base + h->L.off_fb;
    h->g[1] = h->base + h->L.off_gb;
    h->snap = (double*)(h->base + h->L.off_snap);
    h->partial = (double*)(h->base + h->L.off_partial);
    h->dout = (double*)(h->base + h->L.off_out);
    h->prof = (double*)(h->base + h->L.off_prof);
    h->flag = (int*)(h->base + h->L.off_flag);
    e = cudaHostAlloc((void**)&h->host_small, 8 * sizeof(double), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream);
    if (e == cudaSuccess && lks::staged_step_applies(p->storage, p->nx, p->inplace)) {
        e = lks::prepare_staged_step(p->storage, p->inplace, &h->ss.grid);
        h->ss.err = h->flag;
        h->staged = e == cudaSuccess;
    }
    if (e != cudaSuccess) {
        lks_destroy(h);
        return cuda_fail(nullptr, e, "lks_create");
    }
    refresh_params(h);
    const int ilv = lks::interleave_row(p->storage, p->nx, p->inplace);
    e = lks::launch_init(p->storage, h->f[0], h->g[0], p->nx, p->ny, p->B0, p->seed, p->perturb_amp, h->stream, ilv);
    if (e == cudaSuccess)
        e = lks::launch_snapshot(p->storage, h->f[0], h->g[0], p->nx, p->ny, p->B0, p->Fx, h->snap, h->stream,
                                 p->coupling, p->tau_m, ilv);
    if (e != cudaSuccess) {
        lks_destroy(h);
        return cuda_fail(nullptr, e, "lks_create: init kernel");
    }
    *out = h;
    return LKS_OK;
}

lks_status lks_set_walls(lks_handle* h, double c_bottom, double c_top, double u_bottom, double u_top) {
    if (!h) return fail(nullptr, LKS_EINVAL, "handle is NULL");
    if (!(c_bottom >= 0.0) || !(c_top >= 0.0)) return fail(h, LKS_EINVAL, "wall conductance ratios must be >= 0");
    if (!(fabs(u_bottom) < 0.3) || !(fabs(u_top) < 0.3)) return fail(h, LKS_EINVAL, "|wall speed| must be < 0.3");
    h->c_bot = c_bottom;
    h->c_top = c_top;
    h->u_bot = u_bottom;
    h->u_top = u_top;
    refresh_params(h);
    drop_graphs(h);
    return LKS_OK;
}

lks_status lks_step(lks_handle* h, int64_t n) {
    NvtxRange nvtx_range("lks_step");
    if (!h) return fail(nullptr, LKS_EINVAL, "handle is NULL");
    if (n < 0) return fail(h, LKS_EINVAL, "n must be >= 0");
    if (h->p.inplace && (n & 1)) return fail(h, LKS_EINVAL, "an in-place handle steps in pairs: n must be even");
    for (int g = 0; g < kGraphSizes && !h->graphs_disabled; ++g) {
        while (n >= kGraphSteps[g] && !h->graphs_disabled) {
            if (!h->graph[g][h->cur]) {
                cudaError_t e = build_graph(h, g, h->cur);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    h->graphs_disabled = true;  // fall back to direct launches
                    break;
                }
            }
            cudaError_t e = cudaGraphLaunch(h->graph[g][h->cur], h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
            n -= kGraphSteps[g];
            h->steps += kGraphSteps[g];
        }
    }
    for (int64_t k = 0; k < n; ++k) {
        cudaError_t e = step_once(h, h->cur, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step kernel launch");
        h->cur ^= 1;
        h->steps += 1;
    }
    return LKS_OK;
}

int64_t lks_steps_taken(const lks_handle* h) { return h ? h->steps : -1; }

lks_status lks_moments_device(lks_handle* h, int what, double* dev_out) {
    if (!h) return fail(nullptr, LKS_EINVAL, "handle is NULL");
    if (!dev_out) return fail(h, LKS_EINVAL, "dev_out is NULL");
    if (what != LKS_MOMENTS_NODES && what != LKS_MOMENTS_PROFILES) return fail(h, LKS_EINVAL, "bad 'what'");
    cudaError_t e = lks::launch_moments(h->p.storage, h->f[h->cur], h->g[h->cur], h->p.nx, h->p.ny, h->p.B0,
                                        h->p.Fx, what, dev_out, h->stream, h->p.coupling, h->p.tau_m,
                                        lks::interleave_row(h->p.storage, h->p.nx, h->p.inplace));
    if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
    return LKS_OK;
}

lks_status lks_moments(lks_handle* h, int what, double* host_out) {
    NvtxRange nvtx_range("lks_moments");
    if (!h) return fail(nullptr, LKS_EINVAL, "handle is NULL");
    if (!host_out) return fail(h, LKS_EINVAL, "host_out is NULL");
    if (what != LKS_MOMENTS_NODES && what != LKS_MOMENTS_PROFILES) return fail(h, LKS_EINVAL, "bad 'what'");
    cudaError_t e;
    if (what == LKS_MOMENTS_PROFILES) {
        if (lks_status s = lks_moments_device(h, what, h->prof)) return s;
        e = cudaMemcpyAsync(host_out, h->prof, 5 * (size_t)h->p.ny * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream);
    } else if (double* dout = (double*)lks::host_direct_ptr(host_out)) {  // page-locked: written by the kernel
        const int64_t N = (int64_t)h->p.nx * h->p.ny;
        e = lks::launch_node_moments(h->p.storage, h->f[h->cur], h->g[h->cur], N, 0, N, h->p.B0, h->p.Fx, dout,
                                     h->stream, h->p.coupling, h->p.tau_m, ilv_of(h));
    } else {
        int64_t M = 0;
        if (lks_status s = state_stage(h, &M)) return s;
        e = staged_moments_to_host(h, host_out, M);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lks_moments");
    return staged_check(h, "lks_moments");
}

lks_status lks_residual(lks_handle* h, double* r_u, double* r_b) {
    NvtxRange nvtx_range("lks_residual");
    if (!h) return fail(nullptr, LKS_EINVAL, "handle is NULL");
    cudaError_t e = lks::launch_residual(h->p.storage, h->f[h->cur], h->g[h->cur], h->p.nx, h->p.ny, h->p.B0,
                                         h->p.Fx, h->snap, h->partial, h->dout, h->stream, h->p.coupling,
                                         h->p.tau_m, lks::interleave_row(h->p.storage, h->p.nx, h->p.inplace));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->host_small, h->dout, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lks_residual");
    if (lks_status fs = staged_check(h, "lks_residual")) return fs;
    const double* s = h->host_small;
    for (int k = 0; k < 4; ++k)
        if (!isfinite(s[k])) return fail(h, LKS_EUNSTABLE, "the state became non-finite");
    const double ru = s[1] > 1e-60 ? sqrt(s[0] / s[1]) : 0.0;
    const double rb = s[3] > 1e-60 ? sqrt(s[2] / s[3]) : 0.0;
    if (r_u) *r_u = ru;
    if (r_b) *r_b = rb;
    return LKS_OK;
}

lks_status lks_run_to_steady(lks_handle* h, double tol, int64_t check_every, int64_t max_steps, int64_t* steps_out,
                             double* r_out) {
    NvtxRange nvtx_range("lks_run_to_steady");
    if (!h) return fail(nullptr, LKS_EINVAL, "handle is NULL");
    if (check_every < 1 || max_steps < 0 || !(tol > 0.0)) return fail(h, LKS_EINVAL, "bad run_to_steady arguments");
    if (h->p.inplace && ((check_every & 1) || (max_steps & 1)))
        return fail(h, LKS_EINVAL, "an in-place handle steps in pairs: check_every and max_steps must be even");
    int64_t taken = 0;
    double r = INFINITY, best = INFINITY;
    int since_best = 0;
    bool stalled = false;
    const bool zero_stalls = lks::zero_residual_is_stall(h->p.storage, h->p.Fx, h->u_bot, h->u_top);
    lks_status s = LKS_OK;
    while (taken < max_steps) {
        const int64_t n = (max_steps - taken < check_every) ? max_steps - taken : check_every;
        s = lks_step(h, n);
        if (s != LKS_OK) break;
        taken += n;
        double ru, rb;
        s = lks_residual(h, &ru, &rb);
        if (s != LKS_OK) break;
        r = ru > rb ? ru : rb;
        if (r == 0.0 && zero_stalls) {
            stalled = true;
            break;
        }
        if (r < tol) break;
        if (r < best) {
            best = r;
            since_best = 0;
        } else if (++since_best >= lks::kStallChecks && best < lks::stall_floor(h->p.storage)) {
            stalled = true;
            break;
        }
    }
    if (steps_out) *steps_out = taken;
    if (r_out) *r_out = r;
    if (s != LKS_OK) return s;
    if (stalled)
        return fail(h, LKS_ESTALLED,
                    r == 0.0 ? "the state stopped changing (per-step increments below the storage resolution)"
                             : "the residual stopped decreasing at the storage's rounding floor");
    if (!(r < tol)) return fail(h, LKS_ENOTCONVERGED, "max_steps reached before the residual tolerance");
    return LKS_OK;
}

lks_status lks_get_state(lks_handle* h, double* host_f, double* host_g) {
    NvtxRange nvtx_range("lks_get_state");
    if (!h) return fail(nullptr, LKS_EINVAL, "handle is NULL");
    if (!host_f || !host_g) return fail(h, LKS_EINVAL, "host_f/host_g is NULL");
    const int64_t N = (int64_t)h->p.nx * h->p.ny;
    double* df = (double*)lks::host_direct_ptr(host_f);
    double* dg = (double*)lks::host_direct_ptr(host_g);
    cudaError_t e;
    if (df && dg) {  // page-locked: one kernel writes the arrays
        e = lks::launch_to_abs(h->p.storage, h->f[h->cur], h->g[h->cur], N, 0, N, h->p.B0, df, dg, h->stream,
                               h->p.coupling, ilv_of(h));
    } else {
        int64_t M = 0;
        if (lks_status s = state_stage(h, &M)) return s;
        e = staged_to_host(h, host_f, host_g, M);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lks_get_state");
    return staged_check(h, "lks_get_state");
}

lks_status lks_set_state(lks_handle* h, const double* host_f, const double* host_g) {
    NvtxRange nvtx_range("lks_set_state");
    if (!h) return fail(nullptr, LKS_EINVAL, "handle is NULL");
    if (!host_f || !host_g) return fail(h, LKS_EINVAL, "host_f/host_g is NULL");
    const int64_t N = (int64_t)h->p.nx * h->p.ny;
    const double* df = (const double*)lks::host_direct_ptr(host_f);
    const double* dg = (const double*)lks::host_direct_ptr(host_g);
    cudaError_t e;
    if (df && dg) {  // page-locked: one kernel reads the arrays
        e = lks::launch_from_abs(h->p.storage, df, dg, N, 0, N, h->p.B0, h->f[h->cur], h->g[h->cur], h->stream,
                                 h->p.coupling, ilv_of(h));
    } else {
        int64_t M = 0;
        if (lks_status s = state_stage(h, &M)) return s;
        e = staged_from_host(h, host_f, host_g, M);
    }
    if (e == cudaSuccess)
        e = lks::launch_snapshot(h->p.storage, h->f[h->cur], h->g[h->cur], h->p.nx, h->p.ny, h->p.B0, h->p.Fx,
                                 h->snap, h->stream, h->p.coupling, h->p.tau_m, ilv_of(h));
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lks_set_state");
    h->steps = 0;
    return LKS_OK;
}

size_t lks_state_bytes(const lks_handle* h) {
    if (!h) return 0;
    return 19 * (size_t)h->p.nx * (size_t)h->p.ny * lks::storage_bytes(h->p.storage);
}

lks_status lks_get_state_raw(lks_handle* h, void* host, size_t bytes) {
    NvtxRange nvtx_range("lks_get_state_raw");
    if (!h) return fail(nullptr, LKS_EINVAL, "handle is NULL");
    if (!host) return fail(h, LKS_EINVAL, "host is NULL");
    if (bytes != lks_state_bytes(h)) return fail(h, LKS_EINVAL, "bytes differs from lks_state_bytes()");
    const size_t fb = 9 * (size_t)h->p.nx * h->p.ny * lks::storage_bytes(h->p.storage);
    cudaError_t e = cudaMemcpyAsync(host, h->f[h->cur], fb, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((char*)host + fb, h->g[h->cur], bytes - fb, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lks_get_state_raw");
    return staged_check(h, "lks_get_state_raw");
}

lks_status lks_set_state_raw(lks_handle* h, const void* host, size_t bytes) {
    NvtxRange nvtx_range("lks_set_state_raw");
    if (!h) return fail(nullptr, LKS_EINVAL, "handle is NULL");
    if (!host) return fail(h, LKS_EINVAL, "host is NULL");
    if (bytes != lks_state_bytes(h)) return fail(h, LKS_EINVAL, "bytes differs from lks_state_bytes()");
    const size_t fb = 9 * (size_t)h->p.nx * h->p.ny * lks::storage_bytes(h->p.storage);
    cudaError_t e = cudaMemcpyAsync(h->f[h->cur], host, fb, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->g[h->cur], (const char*)host + fb, bytes - fb, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = lks::launch_snapshot(h->p.storage, h->f[h->cur], h->g[h->cur], h->p.nx, h->p.ny, h->p.B0, h->p.Fx,
                                 h->snap, h->stream, h->p.coupling, h->p.tau_m, ilv_of(h));
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lks_set_state_raw");
    h->steps = 0;
    return LKS_OK;
}

lks_status lks_selftest_wait_timeout(lks_handle* h, double limit_s) {
    if (!h) return fail(nullptr, LKS_EINVAL, "handle is NULL");
    if (!h->staged) return fail(h, LKS_EINVAL, "lks_selftest_wait_timeout: the handle runs no staged kernel");
    if (!(limit_s > 0.0 && limit_s <= 1.0)) return fail(h, LKS_EINVAL, "lks_selftest_wait_timeout: limit not in (0, 1] s");
    cudaError_t e = lks::launch_wait_timeout_probe(h->flag, (uint64_t)(limit_s * 1e9), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lks_selftest_wait_timeout");
    return LKS_OK;
}

lks_status lks_sync(lks_handle* h) {
    if (!h) return fail(nullptr, LKS_EINVAL, "handle is NULL");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "lks_sync");
    return staged_check(h, "lks_sync");
}

lks_status lks_destroy(lks_handle* h) {
    if (!h) return LKS_OK;
    if (h->stream || h->base) cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    if (h->state_stage) cudaFree(h->state_stage);
    if (h->owns && h->base) cudaFree(h->base);
    if (h->host_small) cudaFreeHost(h->host_small);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
    return LKS_OK;
}

const char* lks_last_error(const lks_handle* h) { return h ? h->err.c_str() : g_last_error.c_str(); }

const char* lks_status_string(lks_status s) {
    switch (s) {
        case LKS_OK: return "LKS_OK";
        case LKS_EINVAL: return "LKS_EINVAL";
        case LKS_ENOMEM: return "LKS_ENOMEM";
        case LKS_ECUDA: return "LKS_ECUDA";
        case LKS_EUNSTABLE: return "LKS_EUNSTABLE";
        case LKS_ETIMEOUT: return "LKS_ETIMEOUT";
        case LKS_ENOTCONVERGED: return "LKS_ENOTCONVERGED";
        case LKS_EBUSY: return "LKS_EBUSY";
        case LKS_ESTALLED: return "LKS_ESTALLED";
    }
    return "LKS_UNKNOWN";
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// lks_residual_noalloc: the steady-state residual of caller-held state with no allocation at all.
//
// Some callers cannot allocate device memory: applications that reserve the whole device for their
// own pools up front, latency-critical loops in which cudaMalloc/cudaFree (which may synchronise
// the whole device) are not acceptable, and plugin hosts that forbid allocation calls.  This entry
// point runs the same two-pass residual reduction as lks_residual, but its partial sums live in
// the file-scope device array below instead of memory it would have to allocate.  The array holds
// 4 * kNoallocMaxBlocks partial sums plus 4 totals (38.9 KB) and stays allocated on every device
// that loads the library until the process exits.  The reduction never uses more than
// kNoallocMaxBlocks blocks, so any lattice up to the 2^30-node limit fits; larger ones are rejected.
namespace {

constexpr int kNoallocMaxBlocks = lks::kResidualMaxBlocks;  // the largest value residual_blocks() returns
constexpr int kNoallocScratch = 4 * kNoallocMaxBlocks + 8;
static_assert(4 * kNoallocMaxBlocks + 4 <= kNoallocScratch, "partials and totals must fit the static scratch");
constexpr int kNoallocMaxDevices = 64;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratch];
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device: looked up once per device (host code
// only sees a host-side stand-in for the array's name).
cudaError_t noalloc_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" lks_status lks_residual_noalloc(const void* f, const void* g, int32_t storage, int32_t nx, int32_t ny,
                                           double B0, double Fx, int32_t coupling, double tau_m, double* snap,
                                           double* out, void* cuda_stream) {
    if (!f || !g || !snap || !out) return fail(nullptr, LKS_EINVAL, "lks_residual_noalloc: NULL pointer argument");
    if (storage < LKS_F64 || storage > LKS_F16_DEV) return fail(nullptr, LKS_EINVAL, "lks_residual_noalloc: bad storage");
    if (nx < 1 || ny < 1) return fail(nullptr, LKS_EINVAL, "lks_residual_noalloc: nx and ny must be >= 1");
    if (coupling != LKS_MAXWELL && coupling != LKS_LORENTZ)
        return fail(nullptr, LKS_EINVAL, "lks_residual_noalloc: coupling must be LKS_MAXWELL or LKS_LORENTZ");
    if (coupling == LKS_LORENTZ && !(tau_m > 0.5 && isfinite(tau_m) && fabs(tau_m - 1.0) >= 0.05))
        return fail(nullptr, LKS_EINVAL,
                    "lks_residual_noalloc: the Lorentz-force coupling needs tau_m > 1/2 and |tau_m - 1| >= 0.05");
    const int64_t N = (int64_t)nx * (int64_t)ny;
    if (N > ((int64_t)1 << 30))
        return fail(nullptr, LKS_EINVAL, "lks_residual_noalloc: nx*ny exceeds the maximum of 2^30 nodes");
    if (lks::residual_blocks(N) > kNoallocMaxBlocks)
        return fail(nullptr, LKS_EINVAL, "lks_residual_noalloc: reduction exceeds the static scratch");
    double* scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lks_residual_noalloc: cudaGetSymbolAddress");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // The call ends by synchronising the stream, which a stream under capture does not allow.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lks_residual_noalloc: cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(nullptr, LKS_EINVAL, "lks_residual_noalloc: the stream is being captured (the call synchronises it)");
    // Every partial and total slot the reduction reads is written earlier in the same call, so
    // nothing left over from a previous call needs clearing.
    double* partial = scratch;
    double* totals = scratch + 4 * kNoallocMaxBlocks;
    e = lks::launch_residual(storage, f, g, nx, ny, B0, Fx, snap, partial, totals, st, coupling,
                             coupling == LKS_LORENTZ ? tau_m : 1.0);
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(s, totals, sizeof(s), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lks_residual_noalloc");
    for (int k = 0; k < 4; ++k)
        if (!isfinite(s[k])) return fail(nullptr, LKS_EUNSTABLE, "lks_residual_noalloc: the state is non-finite");
    out[0] = s[1] > 1e-60 ? sqrt(s[0] / s[1]) : 0.0;
    out[1] = s[3] > 1e-60 ? sqrt(s[2] / s[3]) : 0.0;
    return LKS_OK;
}
