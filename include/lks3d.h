/*
 * lks3d.h -- C ABI of the three-dimensional channel: the lattice kinetic scheme for MHD of
 * Yahia & Premnath (arXiv 2112.13930) taken to 3D with the link-based Shercliff closure, which
 * the paper states carries over to three dimensions (Sec. IX) without printing the 3D forms.
 *
 * The problem: a channel of nx x ny x nz nodes, periodic in x and z, between two plane walls at
 * y = -a and y = +a half-way outside rows 0 and ny-1 (a = ny/2), an applied field B0 along y, a
 * body force F_x and tangential wall speeds along x.  Per node and step (one fused kernel):
 *   - D3Q19 f (Sec. V) with the Maxwell stress in f^eq in its 3D (traceful) form
 *       4.5 w_a [ |B|^2 |e_a|^2 / 2 - (e_a.B)^2 - |B|^2 / 6 ],
 *     the body-force source S_a = 3 (e_a - u).F f^eq,hyd_a / rho and rho u = sum f e + F/2;
 *   - one D3Q7 distribution per component of B (Sec. IV): W_0 = 1/4, W_a = 1/8, c_sm^2 = 1/4,
 *     so eta = (tau_m - 1/2)/4, g^eq_ai = W_a (B_i + 4 e_aj (u_j B_i - B_j u_i));
 *   - walls: f by half-way bounce-back with Ladd's moving-wall term (App. B.1); B_x and B_z by the
 *     weighted (anti-)bounce-back of Eq. linkbasedBCschemefinal with theta = c a/(tau_m - 1/2)
 *     (Eq. weightingfactor), plus the moving-wall term of Eq. movingwalllinkbasedclosure on B_x;
 *     the normal component B_y by anti-bounce-back to B0.
 * Populations are stored as deviations from the rest equilibrium (rho = 1, u = 0, B = (0, B0, 0))
 * in FP64, FP32, BF16 or FP16; FP64 storage computes in FP64, the others in FP32.  Moments and
 * residuals accumulate in FP64.
 *
 * Layout: f[19][nz][ny][nx], g[3][7][nz][ny][nx] (component first), node n = (z ny + y) nx + x.
 * D3Q19 order: 0 rest; 1..6 = +x, -x, +y, -y, +z, -z; 7..18 = (1,1,0), (-1,-1,0), (1,-1,0),
 * (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1).
 * D3Q7 order: the first seven of those.
 *
 * Status codes, streams, device-buffer ownership and error reporting follow lks.h.  With 16-bit
 * storage, nx a multiple of 8 and nx <= 512 the step stages rows through shared memory with the
 * bulk-copy engine; its waits are bounded (1 s), and a wait that ran out makes the next
 * synchronising call (lks3_sync, lks3_moments, lks3_residual, lks3_get_state) return LKS_ETIMEOUT.
 */
#ifndef LKS3D_H
#define LKS3D_H

#include <stddef.h>
#include <stdint.h>

#include "lks.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lks3_params {
    int32_t nx, ny, nz;      /* nx, nz >= 1 (periodic); ny >= 2; nx*ny*nz <= 2^30 */
    int32_t storage;         /* lks_storage: FP64, FP32, BF16 or FP16 deviations */
    double tau_f;            /* > 1/2; nu = (tau_f - 1/2)/3 */
    double tau_m;            /* > 1/2; eta = (tau_m - 1/2)/4 on D3Q7 */
    double B0;               /* applied field along y */
    double Fx;               /* body force along x */
    void* cuda_stream;       /* cudaStream_t; NULL = legacy default stream */
    void* dev_buffer;        /* optional caller-owned device memory (NULL = library allocates) */
    size_t dev_buffer_bytes; /* size of dev_buffer; >= lks3_footprint_bytes() */
} lks3_params;

typedef struct lks3_handle lks3_handle;

/* Device bytes a handle needs (two population buffers, residual snapshot, reduction and profile
 * buffers); 0 if the parameters are invalid. */
size_t lks3_footprint_bytes(const lks3_params* p);

/* Validate, allocate (or carve dev_buffer) and enqueue the rest state (rho = 1, u = 0,
 * B = (0, B0, 0)).  Both walls start insulating and at rest.  *out is NULL on error. */
lks_status lks3_create(const lks3_params* p, lks3_handle** out);

/* Wall conductance ratios (>= 0, INFINITY allowed) and tangential (x) wall speeds (|u| < 0.3) of
 * the bottom (below row 0) and top (above row ny-1) walls; for steps enqueued afterwards. */
lks_status lks3_set_walls(lks3_handle* h, double c_bottom, double c_top, double u_bottom, double u_top);

/* Close the channel into a rectangular duct (enable = 1) or reopen it (enable = 0, periodic in z):
 * two more walls, the planes z = -b (below plane 0) and z = +b (above plane nz-1), b = nz/2,
 * parallel to the applied field -- the side walls of a duct whose axis is x, which carry the side
 * (Shercliff) layers the paper names as the next case for its closures (end of Sec. VII, Sec. IX).
 * They are at rest and carry the Shercliff thin-wall condition of Eq. ShercliffBClocalcoordinate for
 * the tangential induced field, with conductance ratios c_back (z = -b) and c_front (z = +b), >= 0,
 * INFINITY allowed, relative to the same half-width a = ny/2 as the Hartmann walls (c a = sigma_w
 * t_w / sigma).  Each cut link is closed by the wall it crosses, with no corner reconstruction: f by
 * half-way bounce-back; B_x and B_y, tangential there, by the weighted (anti-)bounce-back of
 * Eq. linkbasedBCschemefinal with theta = c a/(tau_m - 1/2), B_y around its applied value B0; B_z,
 * normal there, by anti-bounce-back to 0.  A link crossing a y wall and a z wall (D3Q19 only,
 * e_x = 0) is closed by the y wall.  Takes effect for steps enqueued afterwards; a duct handle steps
 * with a one-node-per-thread kernel over the flattened node index for every storage type (fully
 * developed flow: nx = 1).  LKS_EINVAL for nz < 2 when enabling, a negative or NaN ratio. */
lks_status lks3_set_side_walls(lks3_handle* h, int32_t enable, double c_back, double c_front);

/* Enqueue n >= 0 fused steps (asynchronous). */
lks_status lks3_step(lks3_handle* h, int64_t n);

/* Steps taken since lks3_create / lks3_set_state. */
int64_t lks3_steps_taken(const lks3_handle* h);

/* Moments of the stored state, FP64: rho = sum f, rho u = sum f e - F/2, B = sum g.
 * what = LKS_MOMENTS_NODES: host_out is 7 x nz x ny x nx (rho, u_x, u_y, u_z, B_x, B_y, B_z);
 * what = LKS_MOMENTS_PROFILES: 7 x ny, each averaged over x and z.  Synchronises. */
lks_status lks3_moments(lks3_handle* h, int what, double* host_out);

/* Residual as lks_residual: r_u = |u_x - u_x'|_2/|u_x|_2, r_b the same for B_x, against the
 * snapshot of the previous call (or creation), which is then replaced; FP64, fixed order;
 * LKS_EUNSTABLE on a non-finite state.  Synchronises. */
lks_status lks3_residual(lks3_handle* h, double* r_u, double* r_b);

/* Repeat { lks3_step(check_every); lks3_residual } until max(r_u, r_b) < tol or max_steps;
 * LKS_ENOTCONVERGED at max_steps; LKS_ESTALLED under the same two conditions as lks_run_to_steady
 * (an exactly zero residual on a driven channel with FP32 or 16-bit storage, or 1000 checks without
 * a new minimum below the storage's rounding floor).  Synchronises. */
lks_status lks3_run_to_steady(lks3_handle* h, double tol, int64_t check_every, int64_t max_steps,
                              int64_t* steps_out, double* r_out);

/* State as FP64 absolute populations (deviation + rest): host_f 19 x N, host_g 21 x N.
 * Page-locked host arrays are written by the conversion kernel itself (LKS_HOST_STAGING unset or
 * "0"); pageable ones through a staging buffer of 40 x 2^20 doubles (335 MB; fewer for smaller
 * lattices), 2^20 nodes at a time, that the handle allocates on first use and keeps until
 * lks3_destroy (LKS_ENOMEM if that fails).  lks3_moments with LKS_MOMENTS_NODES works the same
 * way.  Synchronises. */
lks_status lks3_get_state(lks3_handle* h, double* host_f, double* host_g);

/* Replace the state by FP64 absolute populations (rounded to the storage type); resets the step
 * counter and the residual snapshot.  Synchronises; same staging buffer. */
lks_status lks3_set_state(lks3_handle* h, const double* host_f, const double* host_g);

/* Self-test of the staged kernel's bounded waits, as lks_selftest_wait_timeout: the next
 * synchronising call returns LKS_ETIMEOUT and the handle stays in that error state; LKS_EINVAL for a
 * handle that runs no staged kernel (FP32/FP64, or nx not a multiple of 8 or above 512) or a limit
 * outside (0, 1] s. */
lks_status lks3_selftest_wait_timeout(lks3_handle* h, double limit_s);

lks_status lks3_sync(lks3_handle* h);
lks_status lks3_destroy(lks3_handle* h);

/* Message of the handle's last error (or of the last failed create on this thread if h is NULL). */
const char* lks3_last_error(const lks3_handle* h);

#ifdef __cplusplus
}
#endif

#endif
