/*
 * lks_batch.h -- C ABI of the batched / served solver: many independent channel instances
 * (each the problem of lks.h: Sec. VI.A, Sec. VII, App. B, App. C of Yahia & Premnath,
 * arXiv 2112.13930) of different sizes and parameters, resident together on one GPU and
 * advanced by one persistent kernel launch per lks_batch_run call.
 *
 * The paper defines the per-instance method only; batching, admission and the work queue are
 * this library's.  Per node the update is the same fused collide-stream step as lks_step (same
 * device code), so an instance's result does not depend on which other instances share the
 * batch: the per-instance residual reduction has a fixed order for a given group size
 * (threads_per_group), and the state of an instance is touched only by the thread group that
 * holds it.
 *
 * Execution: lks_batch_run launches a persistent kernel of (#SMs x resident CTAs) blocks; each
 * CTA is split into groups_per_cta groups of threads_per_group threads; a group takes the next
 * running instance from a work list (one atomic add, no waiting), advances it by up to quantum
 * steps (synchronising only its own threads between steps), checks the steady-state residual
 * every check_every steps, writes its status, and takes the next instance.  With cluster_ctas > 1
 * the worker is instead a thread-block cluster of that many CTAs on as many SMs, synchronised by
 * the hardware cluster barrier between steps, so one large instance advances faster.  The launch
 * (counter reset, kernel, status copy) is a captured CUDA graph.  There are no spin-waits.
 *
 * Memory: instance states live in one device pool (caller memory or allocated at create) that
 * a host-side first-fit allocator carves; lks_batch_add returns LKS_EBUSY when no slot is free
 * or the pool cannot hold the instance (admission by device-memory footprint).
 *
 * Residual (steady-state criterion; the paper gives none): every check_every steps,
 * r = max(|u_x - u_x'|_2 / |u_x|_2, |B_x - B_x'|_2 / |B_x|_2) over the instance's nodes, FP64,
 * against the snapshot of the previous check (a term with a denominator below 1e-30 counts 0).
 * An instance is CONVERGED when r < tol, STALLED when r is below the storage type's rounding floor
 * (1e-12 FP64, 1e-4 FP32, 1e-2 16-bit) and has not reached a new minimum for 1000 checks in a row,
 * or when r is exactly 0 on a channel driven by a body force or a moving wall with FP32 or 16-bit
 * storage (the state stopped changing: its increments fell below the storage's resolution, which
 * is not convergence), UNSTABLE when r is not finite, MAX_STEPS at max_steps.
 *
 * Threading: a batch handle is not thread-safe.
 */
#ifndef LKS_BATCH_H_
#define LKS_BATCH_H_

#include <stddef.h>
#include <stdint.h>

#include "lks.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lks_batch lks_batch;

typedef struct lks_batch_config {
    int32_t storage;            /* lks_storage of every instance's populations */
    int32_t max_instances;      /* slot table size, >= 1 */
    size_t pool_bytes;          /* device bytes for instance states (the admission budget) */
    void* cuda_stream;          /* cudaStream_t; NULL = legacy default stream */
    void* dev_buffer;           /* optional caller-owned pool memory (256-byte aligned) */
    size_t dev_buffer_bytes;    /* must be >= pool_bytes when dev_buffer is given */
    int32_t threads_per_group;  /* power of two in [32, 512]; 0 = 256 */
    int32_t groups_per_cta;     /* 1..15, threads_per_group * groups_per_cta <= 512; 0 = 1 */
    int32_t cluster_ctas;       /* 1, 2, 4 or 8 CTAs (one per SM) per instance; > 1 needs groups_per_cta = 1;
                                   0 = 1 */
    int32_t coupling;           /* lks_coupling of every instance of this batch (0 = LKS_MAXWELL) */
    int32_t inplace;            /* 1: every instance keeps one population buffer, updated in place
                                   in pairs of steps (as lks_params.inplace; same results bit for
                                   bit, half the population memory); quantum_steps, check_every
                                   and max_steps must then be even.  0: two buffers */
    int32_t pad;
} lks_batch_config;

typedef struct lks_instance_desc {
    int32_t nx, ny;             /* as lks_params */
    int32_t closure;            /* lks_closure */
    int32_t coupling;           /* lks_coupling; must equal the batch's; LKS_LORENTZ needs |tau_m - 1| >= 0.05 */
    double tau_f, tau_m, B0, Fx;
    double c_bottom, c_top;     /* wall conductance ratios, >= 0, INFINITY allowed */
    double u_bottom, u_top;     /* tangential wall speeds, |u| < 0.3 */
    uint64_t seed;
    double perturb_amp;         /* initial state as lks_create */
    double tol;                 /* residual tolerance, > 0 */
    int64_t check_every;        /* steps between residual checks, >= 1 */
    int64_t max_steps;          /* >= 1 */
} lks_instance_desc;

enum {
    LKS_INST_FREE = -1,
    LKS_INST_RUNNING = 0,
    LKS_INST_CONVERGED = 1,
    LKS_INST_MAX_STEPS = 2,
    LKS_INST_UNSTABLE = 3,
    LKS_INST_STALLED = 4
};

typedef struct lks_instance_result {
    int32_t state;              /* LKS_INST_* */
    int32_t pad;
    int64_t steps;              /* steps taken */
    double residual;            /* last residual (INFINITY before the first check) */
} lks_instance_result;

/* Pool bytes one instance needs with this storage type in a batch with this inplace setting
 * (two population buffers, or one when inplace = 1, + residual snapshot, 256-byte aligned); 0 if
 * the description is invalid for such a batch. */
size_t lks_instance_footprint_bytes(const lks_instance_desc* d, int32_t storage, int32_t inplace);

/* Create a batch; allocates the pool unless dev_buffer is given.  *out is NULL on error. */
lks_status lks_batch_create(const lks_batch_config* cfg, lks_batch** out);

/* Admit one instance: validate, take a free slot and pool memory (first fit), enqueue its
 * initial state (asynchronous).  *slot gets the slot index.  LKS_EBUSY: no free slot or not
 * enough pool memory right now (nothing changed); LKS_EINVAL: invalid description. */
lks_status lks_batch_add(lks_batch* b, const lks_instance_desc* d, int32_t* slot);

/* One persistent launch: every RUNNING instance advances by up to quantum_steps (>= 1; even for
 * an in-place batch) steps or until it leaves RUNNING.  Synchronises; afterwards lks_batch_result reflects the launch.
 * *n_running (nullable) gets the number of instances still RUNNING. */
lks_status lks_batch_run(lks_batch* b, int64_t quantum_steps, int32_t* n_running);

/* Status of one slot (state LKS_INST_FREE for an empty slot). */
lks_status lks_batch_result(const lks_batch* b, int32_t slot, lks_instance_result* out);

/* Moments of one instance's current state, as lks_moments (what = LKS_MOMENTS_NODES or
 * LKS_MOMENTS_PROFILES).  Synchronises. */
lks_status lks_batch_moments(lks_batch* b, int32_t slot, int what, double* host_out);

/* Copy one instance's current state out as FP64 absolute populations (deviation + rest equilibrium),
 * host_f 9 x ny x nx and host_g 2 x 5 x ny x nx in the layout of lks.h, as lks_get_state does.  With
 * lks_batch_set_state this moves an instance between batches of different storage types -- e.g. an
 * FP32 solve that reached its rounding floor continued in an FP64 batch to a tolerance FP32 cannot
 * certify.  Uses a temporary device buffer of 19 nx ny doubles.  Synchronises. */
lks_status lks_batch_get_state(lks_batch* b, int32_t slot, double* host_f, double* host_g);

/* Replace one instance's state by FP64 absolute populations (layout as lks_batch_get_state), rounded
 * to the batch's storage type, and restart its bookkeeping: step count 0, status RUNNING, residual
 * snapshot taken from the new state, stall history cleared.  Its descriptor (tol, check_every,
 * max_steps, walls, force) is unchanged.  Uses a temporary device buffer of 19 nx ny doubles.
 * Synchronises. */
lks_status lks_batch_set_state(lks_batch* b, int32_t slot, const double* host_f, const double* host_g);

/* Free a slot and its pool memory (the instance may be in any state).  Synchronises. */
lks_status lks_batch_remove(lks_batch* b, int32_t slot);

/* Change the thread-group shape used by later lks_batch_run calls (see lks_batch_config). */
lks_status lks_batch_set_shape(lks_batch* b, int32_t threads_per_group, int32_t groups_per_cta, int32_t cluster_ctas);

/* Time one lks_batch_run of probe_steps on the current instances for each candidate shape
 * (threads_per_group, groups_per_cta, cluster_ctas given as parallel arrays of length n), restoring
 * every instance's state after each candidate, then keep the fastest shape.  seconds_out
 * (nullable, length n) gets each candidate's time.  Synchronises. */
lks_status lks_batch_autotune(lks_batch* b, int64_t probe_steps, const int32_t* threads_per_group,
                              const int32_t* groups_per_cta, const int32_t* cluster_ctas, int32_t n,
                              double* seconds_out, int32_t* best_index);

/* Pool bytes currently free, and in use. */
lks_status lks_batch_memory(const lks_batch* b, size_t* free_bytes, size_t* used_bytes);

lks_status lks_batch_destroy(lks_batch* b);

const char* lks_batch_last_error(const lks_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* LKS_BATCH_H_ */
