/*
 * lks.h -- C ABI of the GB300 lattice kinetic scheme for MHD with Shercliff
 * thin-conducting-wall closures (Yahia & Premnath, arXiv 2112.13930).
 *
 * The problem a caller poses (Sec. VI.A, Sec. VII, App. B, App. C): a 2D
 * channel of nx x ny nodes, periodic in x, bounded in y by two plates that
 * carry wall conductance ratios c_bottom, c_top (Eq. wallconductanceratiodefinition)
 * and tangential speeds u_bottom, u_top, with an applied field B0 along y and an
 * optional body force Fx along x.  The library advances the coupled D2Q9
 * hydrodynamic distribution f (Sec. V, Eq. LBMforflowfield, Maxwell stress in
 * f^eq) and D2Q5 vector distribution g for the induced field (Sec. IV,
 * Eq. LKSformagneticfield) with one fused collide-stream kernel per step, the
 * chosen wall closure applied inside the same pass:
 *   LKS_LINK   -- link-based weighted bounce-back / anti-bounce-back for g
 *                 (Eq. linkbasedBCschemefinal, moving wall Eq.
 *                 movingwalllinkbasedclosure) with half-way bounce-back for f
 *                 (Sec. VI; moving wall App. B.1); walls half-way outside rows
 *                 0 and ny-1, half-width a = ny/2;
 *   LKS_MOMENT -- on-node moment-based closure for g (Eqs.
 *                 momentbasedBCslowerboundary, momentbasedBCsupperboundary,
 *                 momentbasedclosureformovingwall) with the moment-based no-slip
 *                 closure for f (App. A, App. B.2); walls on rows 0 and ny-1,
 *                 half-width a = (ny-1)/2.
 *
 * Units: lattice units, dx = dt = 1, c_s^2 = c_sm^2 = 1/3, rho0 = 1, mu_m = 1.
 * Directions: D2Q9 e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1)
 * e6=(-1,1) e7=(-1,-1) e8=(1,-1); D2Q5 uses e0..e4.
 *
 * Memory layout in HBM (structure of arrays, x fastest):
 *   f[a][y][x] for a = 0..8 and g[k][a][y][x] for k = x,y component, a = 0..4,
 *   stored as deviations from the rest equilibrium (rho = 1, u = 0,
 *   B = (0, B0), with the Maxwell stress under LKS_MAXWELL) in the storage type
 *   of lks_params.storage; two such buffers (ping-pong).  The state held between
 *   steps is the post-collision field.
 *
 * Ownership: a handle owns its device buffers, or borrows caller memory
 * (lks_params.dev_buffer), which must outlive the handle.  Host pointers
 * passed to any call are only read or written during that call.  A handle is
 * not thread-safe; separate handles are independent.
 *
 * Streams: all device work of a handle is enqueued on lks_params.cuda_stream
 * (a cudaStream_t, NULL = legacy default stream).  Calls documented as
 * "asynchronous" return before the work finishes; errors of asynchronous work
 * surface at the next synchronising call.
 *
 * Errors: every call returns an lks_status; LKS_OK is 0.  After an error,
 * lks_last_error(h) (or lks_last_error(NULL) for handle-less calls) gives a
 * one-line message.  A state that became non-finite gives LKS_EUNSTABLE.
 *
 * 16-bit storage with nx a multiple of 8 and nx >= 1024 steps through kernels
 * that stage rows in shared memory with the bulk-copy engine (the whole step
 * with two buffers, the first step of each in-place pair).  Their waits are
 * bounded (1 s); a wait that ran out makes the next synchronising call
 * (lks_sync, lks_moments, lks_residual, lks_get_state) return LKS_ETIMEOUT.
 */
#ifndef LKS_H_
#define LKS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LKS_OK = 0,
    LKS_EINVAL = 1,          /* a parameter is out of range */
    LKS_ENOMEM = 2,          /* device or host allocation failed, or dev_buffer too small */
    LKS_ECUDA = 3,           /* a CUDA call failed */
    LKS_EUNSTABLE = 4,       /* the state became non-finite */
    LKS_ETIMEOUT = 5,        /* a bounded device wait gave up */
    LKS_ENOTCONVERGED = 6,   /* max_steps reached before the residual tolerance */
    LKS_EBUSY = 7,           /* no free slot / memory budget (batched and served solves) */
    LKS_ESTALLED = 8         /* lks_run_to_steady: the state stopped changing or the residual
                                stopped decreasing at the storage's rounding floor before reaching
                                the tolerance (see lks_run_to_steady) */
} lks_status;

typedef enum { LKS_LINK = 0, LKS_MOMENT = 1 } lks_closure;

/* How the magnetic field acts on the flow.
 *   LKS_MAXWELL -- Dellar's Maxwell stress (|B|^2 I/2 - BB) in f^eq; the default.
 *   LKS_LORENTZ -- the paper's own form (Sec. IV-V): f^eq without magnetic terms and the Lorentz
 *                  force F_L = J x B in the source term and in rho u = sum f e + F/2, with
 *                  J_z = (Lambda^(1)_yx - Lambda^(1)_xy)/(tau_m c_sm^2) from the non-equilibrium first
 *                  moment of g (Eq. rank2antisymmtensornoneq).  u and J depend on each other linearly
 *                  and are solved together exactly.  At moment-based wall nodes the closure sets the
 *                  node's velocity (sum f e + F/2)/rho to (U, 0), i.e. Pi_10 = rho U - F_x/2 and
 *                  Pi_01 = -F_y/2, and Pi_20 = rho (c_s^2 + U^2).  Requires |tau_m - 1| >= 0.05 (the
 *                  moments of a stored state read J back from the (1 - 1/tau_m)-scaled
 *                  non-equilibrium part of the post-collision g). */
typedef enum { LKS_MAXWELL = 0, LKS_LORENTZ = 1 } lks_coupling;

/* Storage type of the populations; arithmetic is FP64 for LKS_F64 and FP32 otherwise.  Every type
 * stores deviations from the rest equilibrium; LKS_F16_DEV stores each deviation times 2^14 (an exact
 * power-of-two scale that keeps deviations down to 3.7e-9 in FP16's normal range; deviations of
 * magnitude 4 or more overflow, which the residual reports as LKS_EUNSTABLE).  BF16 is unscaled. */
typedef enum { LKS_F64 = 0, LKS_F32 = 1, LKS_BF16_DEV = 2, LKS_F16_DEV = 3 } lks_storage;

typedef struct lks_params {
    int32_t nx;            /* nodes along x (periodic), >= 1 */
    int32_t ny;            /* nodes across the channel: >= 2 (link), >= 3 (moment) */
    int32_t closure;       /* lks_closure */
    int32_t storage;       /* lks_storage */
    double tau_f;          /* relaxation time of f, > 1/2; nu = (tau_f - 1/2)/3 */
    double tau_m;          /* relaxation time of g, > 1/2; eta = (tau_m - 1/2)/3 */
    double B0;             /* applied field along y (Sec. VI.A) */
    double Fx;             /* external body force along x */
    uint64_t seed;         /* seed of the initial velocity perturbation */
    double perturb_amp;    /* 0 => rest start; else u0 ~ U(-amp, amp) per component */
    void* cuda_stream;     /* cudaStream_t; NULL = legacy default stream */
    void* dev_buffer;      /* optional caller-owned device memory (NULL = library allocates) */
    size_t dev_buffer_bytes; /* size of dev_buffer; must be >= lks_footprint_bytes() */
    int32_t coupling;      /* lks_coupling (0 = LKS_MAXWELL) */
    int32_t inplace;       /* 0: two population buffers (each step reads one, writes the
                              other); 1: one buffer updated in place, steps taken in pairs
                              (the "AA" access pattern: the first step of a pair pulls from
                              the neighbours and pushes into their opposite-direction slots,
                              the second reads and writes only the node's own slots), half
                              the population memory at the same bytes per step and the
                              same results bit for bit; lks_step and lks_run_to_steady then
                              take even step counts (LKS_EINVAL otherwise).  With 16-bit
                              storage and even nx the in-place buffer keeps each row
                              interleaved (32-bit word w holds nodes x = w and x = w + nx/2);
                              lks_moments, lks_get_state and lks_set_state present and take
                              node order as always, but raw memory seen through dev_buffer
                              is in that order (and is not a valid input of
                              lks_residual_noalloc, which expects node order) */
} lks_params;

typedef struct lks_handle lks_handle;

/* Device bytes a handle with these parameters needs (the population buffer(s),
 * residual snapshot, reduction and profile buffers); 0 if the parameters are
 * invalid.  Used for admission control. */
size_t lks_footprint_bytes(const lks_params* p);

/* Validate p, allocate (or carve dev_buffer), and enqueue the initial state:
 * equilibria at rho = 1, B = (0, B0), u = u0, where u0 = 0 or, if
 * perturb_amp != 0, each component uniform in [-amp, amp] drawn from
 * SplitMix64(seed XOR counter) with counter 2*node (x) and 2*node+1 (y),
 * node = y*nx + x.  Both walls start insulating and at rest.  Asynchronous.
 * *out is NULL on error. */
lks_status lks_create(const lks_params* p, lks_handle** out);

/* Set the Shercliff wall conductance ratios (>= 0; INFINITY = perfectly
 * conducting) and tangential wall speeds (|u| < 0.3) of the bottom (row 0)
 * and top (row ny-1) walls.  Only the closure coefficients change: theta =
 * c a/(tau_m - 1/2) (Eq. weightingfactor) for LKS_LINK, beta = c a/(tau_m c_sm^2)
 * for LKS_MOMENT (Eq. momentconstraintgx multiplied through by c a).  Takes
 * effect for steps enqueued afterwards. */
lks_status lks_set_walls(lks_handle* h, double c_bottom, double c_top, double u_bottom, double u_top);

/* Enqueue n >= 0 fused collide-stream steps (pull-stream, wall closures, moments, equilibria,
 * collision and store in one kernel per step).  Asynchronous; n runs as captured CUDA graphs of
 * 64, 32, ..., 2 steps (built on first use, rebuilt after lks_set_walls) plus at most one direct
 * launch.  n must be even for an in-place handle (LKS_EINVAL). */
lks_status lks_step(lks_handle* h, int64_t n);

/* Steps taken since lks_create / lks_set_state. */
int64_t lks_steps_taken(const lks_handle* h);

enum {
    LKS_MOMENTS_NODES = 0,   /* out: 5 x ny x nx doubles: rho, u_x, u_y, B_x, B_y */
    LKS_MOMENTS_PROFILES = 1 /* out: 5 x ny doubles: the same fields averaged over x */
};

/* Moments of the current state: rho = sum f, rho u = sum f e - F/2 (the
 * post-collision form of rho u = sum f e + F/2 of Sec. V), B = sum g
 * (Eq. zerothmomentofg), accumulated in FP64.  host_out is caller-allocated
 * host memory; per-node moments are written into it by the moment kernel when
 * it is page-locked, else through the staging buffer, as lks_get_state writes.
 * Synchronises the stream. */
lks_status lks_moments(lks_handle* h, int what, double* host_out);

/* Same as lks_moments but writes into caller-allocated device memory
 * dev_out, asynchronously on the handle's stream. */
lks_status lks_moments_device(lks_handle* h, int what, double* dev_out);

/* Steady-state residual (no criterion in the paper; the reading used here):
 * r_u = |u_x - u_x'|_2 / |u_x|_2 and r_b = |B_x - B_x'|_2 / |B_x|_2 over all
 * nodes, FP64, fixed reduction order, where ' is the snapshot taken by the
 * previous lks_residual call (or at creation); the snapshot is then replaced.
 * A term whose denominator is <= 1e-30 is reported as 0.  Returns
 * LKS_EUNSTABLE if any moment is non-finite.  Synchronises the stream.
 * A value of exactly 0 on a channel driven by a body force or a moving wall
 * with FP32 or 16-bit storage means that u_x and B_x did not change by one bit
 * since the snapshot: the state stagnated (its per-step increments fell below
 * the resolution of the stored deviations), which is not convergence;
 * lks_run_to_steady reports it as LKS_ESTALLED. */
lks_status lks_residual(lks_handle* h, double* r_u, double* r_b);

/* Repeat { lks_step(h, check_every); lks_residual } until max(r_u, r_b) < tol
 * or max_steps steps have been taken.  *steps_out (nullable) gets the steps
 * taken by this call and *r_out (nullable) the last residual.  Returns
 * LKS_ENOTCONVERGED at max_steps, and LKS_ESTALLED (the state is left as it
 * is) when
 *   - the residual is exactly 0 on a driven channel (body force or moving
 *     wall) with FP32 or 16-bit storage: the state stopped changing; or
 *   - the residual has not reached a new minimum for 1000 checks in a row
 *     while its best value is below the storage's rounding floor (1e-12 FP64,
 *     1e-4 FP32, 1e-2 16-bit): it jitters at that floor above tol.
 * For an in-place handle check_every and max_steps must be even (LKS_EINVAL).
 * Synchronises. */
lks_status lks_run_to_steady(lks_handle* h, double tol, int64_t check_every, int64_t max_steps,
                             int64_t* steps_out, double* r_out);

/* Copy the state out as FP64 absolute populations (deviation + rest
 * equilibrium): host_f 9 x ny x nx, host_g 2 x 5 x ny x nx, layouts as above.
 * If host_f and host_g are page-locked (cudaHostAlloc, cudaHostRegister) and
 * LKS_HOST_STAGING is unset or "0", one conversion kernel writes them through
 * their mapped device addresses.  Otherwise the state is converted 2^20 nodes at a
 * time into a staging buffer of 19 x 2^20 doubles (152 MB; fewer for smaller
 * lattices) and copied out plane by plane; the handle allocates that buffer on
 * first use and keeps it until lks_destroy (LKS_ENOMEM if the allocation fails).
 * Either way the arrays must hold the full sizes above.  Synchronises. */
lks_status lks_get_state(lks_handle* h, double* host_f, double* host_g);

/* Replace the state by FP64 absolute populations from host memory (same
 * layout as lks_get_state), rounded to the storage type; resets the step
 * counter and the residual snapshot.  Page-locked arrays are read by the
 * conversion kernel, pageable ones through the staging buffer, as lks_get_state
 * writes them.  Synchronises. */
lks_status lks_set_state(lks_handle* h, const double* host_f, const double* host_g);

/* Bytes of the handle's state in its own storage image: 19 x nx x ny populations of the storage
 * type (lks_storage), the 9 f planes then the 10 g planes, each plane ny x nx -- the deviations as
 * held on the device (FP16 times 2^14; in-place 16-bit handles with even nx keep their rows
 * interleaved, see lks_params.inplace).  0 for a NULL handle. */
size_t lks_state_bytes(const lks_handle* h);

/* Copy the state out in that storage image (a bit-exact checkpoint, at the storage type's size:
 * half the bytes of lks_get_state for FP32, a quarter for 16-bit).  bytes must equal
 * lks_state_bytes(h) (LKS_EINVAL otherwise); host memory is written by the copy engine (page-locked
 * host memory moves at the link's full rate).  Synchronises. */
lks_status lks_get_state_raw(lks_handle* h, void* host, size_t bytes);

/* Replace the state by an image written by lks_get_state_raw of a handle with the same nx, ny,
 * storage, inplace and B0 (the image is taken as is), reset the step counter and take the residual
 * snapshot from it.  bytes must equal lks_state_bytes(h).  Synchronises. */
lks_status lks_set_state_raw(lks_handle* h, const void* host, size_t bytes);

/* Block until all work of the handle has finished; reports asynchronous errors. */
/* Self-test of the bounded device waits (failure detection without a GPU fault): enqueue on the
 * handle's stream one warp that waits, with the staged kernels' bounded wait, on a shared-memory
 * barrier nothing completes, gives up after limit_s seconds (0 < limit_s <= 1) and records the
 * timeout as a staged step's wait would.  The next synchronising call returns LKS_ETIMEOUT and the
 * handle stays in that error state (destroy it; the CUDA context remains usable).  LKS_EINVAL for a
 * handle that runs no staged kernel or a limit out of range. */
lks_status lks_selftest_wait_timeout(lks_handle* h, double limit_s);

lks_status lks_sync(lks_handle* h);

/* Release the handle and the memory it owns.  Safe on NULL. */
lks_status lks_destroy(lks_handle* h);

/* Message of the last error of h (NULL: of the calling thread's last
 * handle-less error).  Never NULL. */
const char* lks_last_error(const lks_handle* h);

/* Steady-state residual of a state held in caller memory, computed with no allocation of any
 * kind.  (The paper has no counterpart: this is a variant of the lks_residual reduction for
 * callers that cannot allocate device memory -- applications that reserve the whole device for
 * their own pools, latency-critical loops where cudaMalloc/cudaFree may synchronise the device,
 * plugin hosts that forbid allocation calls.)
 *   f, g      device pointers to one lattice's populations in the layout above (deviation form,
 *             storage type `storage`, node order), nx x ny nodes; read only.
 *   B0, Fx    the lattice's applied field and body force (needed for B_y and u_x).
 *   coupling  lks_coupling of the state: LKS_MAXWELL, or LKS_LORENTZ, whose u_x includes the half
 *             J x B force recovered from the stored g and so needs the state's tau_m (> 1/2,
 *             |tau_m - 1| >= 0.05, as lks_create requires; tau_m is ignored for LKS_MAXWELL).
 *   snap      device pointer to 2*nx*ny doubles: u_x then B_x per node of the previous call; the
 *             residual compares against it and overwrites it with the current values.
 *   out       host pointer to 2 doubles: r_u, r_b as defined for lks_residual.
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream).  The call synchronises it
 *             before returning, so it must not be a stream under capture (LKS_EINVAL).
 * The partial sums live in a file-scope device array of 4*1216 + 8 doubles (38.9 KB) that every
 * GPU which loads the library keeps until the process exits.  Lattices above 2^30 nodes are
 * rejected with LKS_EINVAL and a message naming the limit.  The first call on each device looks
 * up the array's device address (with that device current).  All calls share the one array: calls
 * that overlap on the GPU (other streams, other threads) race on it and must be serialised by the
 * caller.  Nothing from a previous call needs clearing: each call writes every slot it reads.
 * Errors: LKS_EINVAL, LKS_ECUDA, LKS_EUNSTABLE (non-finite moments); lks_last_error(NULL) gives the
 * message. */
lks_status lks_residual_noalloc(const void* f, const void* g, int32_t storage, int32_t nx, int32_t ny, double B0,
                                double Fx, int32_t coupling, double tau_m, double* snap, double* out,
                                void* cuda_stream);

/* Static name of a status code. */
const char* lks_status_string(lks_status s);

#ifdef __cplusplus
}
#endif

#endif /* LKS_H_ */
