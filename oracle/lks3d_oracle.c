/*
 * lks3d_oracle.c -- FP64 CPU reference of the three-dimensional lattice kinetic scheme for MHD
 * in a plane channel, with the link-based Shercliff closure.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the benchmark's CPU baseline; the
 * product library never calls it and it calls nothing of the product library.
 *
 * The paper states both of its wall schemes carry over to three dimensions (Sec. IX) but prints
 * the 2D forms only.  This oracle takes the 2D scheme to 3D step by step:
 *   - fluid: D3Q19 LBM (Sec. V) with Dellar's Maxwell stress in the equilibrium, the traceful 3D
 *     form  f^eq_a = w_a [rho + 3 rho e.u + 4.5 rho (e.u)^2 - 1.5 rho u^2]
 *                  + 4.5 w_a [ |B|^2 |e_a|^2 / 2 - (e_a.B)^2 - |B|^2 / 6 ]
 *     (T = |B|^2 I / 2 - B B contracted with (e e - c_s^2 I) / (2 c_s^4)), the body-force source
 *     S_a = 3 (e_a - u).F f^eq,hyd_a / rho and rho u = sum f e + F/2;
 *   - induction: one D3Q7 distribution per component of B (Sec. IV), W_0 = 1/4, W_a = 1/8,
 *     c_sm^2 = 1/4, g^eq_ai = W_a (B_i + e_aj Lambda_ji / c_sm^2), Lambda_ji = u_j B_i - B_j u_i;
 *   - walls: planes y = -a (below row 0) and y = +a (above row ny-1), a = ny/2, half-way between
 *     nodes; periodic in x and z.  Tangential field components (B_x, B_z) take the link-based
 *     Shercliff closure of Eq. linkbasedBCschemefinal, g_in = r g~_out + k, r = (theta-1)/(theta+1),
 *     theta = c a/(tau_m - 1/2) (Eq. weightingfactor); its derivation (Sec. VI) does not involve
 *     the lattice weights, so it holds on D3Q7 unchanged.  The moving-wall term of App. B.1
 *     (Eq. movingwalllinkbasedclosure) enters B_x only: at the wall Lambda_yx = -B0 U and
 *     Lambda_yz = 0.  The normal component B_y is fixed to B0 by anti-bounce-back,
 *     g_in = -g~_out + 2 W B0 (Eq. magneticfieldanditsgradientrelation1 with B_y(x_b) = B0).
 *     f takes half-way bounce-back with Ladd's moving-wall term 2 w_a rho0 e_a.U / c_s^2 (App. B.1).
 *
 * Duct (side = 1): two more walls, the planes z = -b (below plane 0) and z = +b (above plane nz-1),
 * b = nz/2, parallel to the applied field -- the side walls of a rectangular duct whose axis is x
 * (flows with side layers, named by the paper as the next case for its closures, end of Sec. VII and
 * Sec. IX).  Each cut link is closed on its own, by the rule of the wall it crosses (no corner
 * reconstruction: D3Q7 has no diagonal links, and a D3Q19 link crossing both a y and a z wall has
 * e_x = 0, so half-way bounce-back applies to it with no moving-wall term whichever wall closes it):
 *   - f: half-way bounce-back (the side walls are at rest);
 *   - B_x and B_y are tangential there: the weighted (anti-)bounce-back of Eq. linkbasedBCschemefinal
 *     with theta_s = c_s a/(tau_m - 1/2), c_s the wall's conductance ratio relative to the same length
 *     a as the Hartmann walls (so c_s a = sigma_w t_w/sigma, the Shercliff condition
 *     b + c_s a db/dn = 0 of Eq. ShercliffBClocalcoordinate for the induced part b); for B_y the
 *     anti-bounce-back half restores the applied value, g_in = r g~_out + (1 - r) W B0;
 *   - B_z is normal to them: anti-bounce-back to B_z = 0, g_in = -g~_out.
 *
 * State: absolute post-collision populations, f[19][nz][ny][nx], g[3][7][nz][ny][nx] (component
 * index first), node n = (z*ny + y)*nx + x.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny, nz, pad;
    double tau_f, tau_m, B0, Fx;
    double c_bot, c_top, u_bot, u_top;
    int32_t side, pad2;     /* 1: walls at the z planes (duct); 0: periodic in z */
    double c_back, c_front; /* conductance ratios of the walls z = -b and z = +b (relative to a) */
} o3_params;

/* D3Q19: rest, 6 faces, 12 edges; opposite of a >= 1 is a + 1 (a odd) or a - 1 (a even). */
static const int E19[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                               {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                               {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                               {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
/* D3Q7: rest and the 6 faces, same order as the first seven of D3Q19. */
static const int E7[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

static double w19(int a) { return a == 0 ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
static double w7(int a) { return a == 0 ? 0.25 : 0.125; }
static int opp(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }

static double dot3(const int e[3], const double v[3]) { return e[0] * v[0] + e[1] * v[1] + e[2] * v[2]; }

/* hydrodynamic part of f^eq (Sec. V) */
static double feq_hyd(int a, double rho, const double u[3]) {
    const double eu = dot3(E19[a], u);
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return w19(a) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
}

/* Maxwell-stress part of f^eq in 3D */
static double feq_mag(int a, const double B[3]) {
    const double e2 = (double)(E19[a][0] * E19[a][0] + E19[a][1] * E19[a][1] + E19[a][2] * E19[a][2]);
    const double eB = dot3(E19[a], B);
    const double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    return 4.5 * w19(a) * (0.5 * B2 * e2 - eB * eB - B2 / 6.0);
}

/* g^eq of component i (Sec. IV on D3Q7): W_a (B_i + e_aj (u_j B_i - B_j u_i) / c_sm^2) */
static double geq(int a, int i, const double u[3], const double B[3]) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s += E7[a][j] * (u[j] * B[i] - B[j] * u[i]);
    return w7(a) * (B[i] + 4.0 * s);
}

/* closure coefficients of one wall for the tangential components: r and theta/(theta+1) */
static void link_coef(const o3_params* p, double c, double* r, double* k) {
    if (isinf(c)) {
        *r = 1.0;
        *k = 1.0;
        return;
    }
    const double a = 0.5 * p->ny;
    const double th = c * a / (p->tau_m - 0.5);
    *r = (th - 1.0) / (th + 1.0);
    *k = th / (th + 1.0);
}

int o3_init(const o3_params* p, double* f, double* g) {
    if (p->nx < 1 || p->ny < 2 || p->nz < 1 || !(p->tau_f > 0.5) || !(p->tau_m > 0.5)) return 1;
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    const double u[3] = {0.0, 0.0, 0.0};
    const double B[3] = {0.0, p->B0, 0.0};
    for (int64_t n = 0; n < N; ++n) {
        for (int a = 0; a < 19; ++a) f[a * N + n] = feq_hyd(a, 1.0, u) + feq_mag(a, B);
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < 7; ++a) g[(i * 7 + a) * N + n] = geq(a, i, u, B);
    }
    return 0;
}

/* One step: pull (periodic in x and z, closures at the y walls), moments, collision.
 * fi/gi -> fo/go, all absolute post-collision populations. */
int o3_step(const o3_params* p, const double* fi, const double* gi, double* fo, double* go) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const int64_t N = (int64_t)nx * ny * nz;
    double rb, kb, rt, kt, rk, kk, rf, kf;
    link_coef(p, p->c_bot, &rb, &kb);
    link_coef(p, p->c_top, &rt, &kt);
    link_coef(p, p->c_back, &rk, &kk);
    link_coef(p, p->c_front, &rf, &kf);
    const double om_f = 1.0 / p->tau_f, om_m = 1.0 / p->tau_m;
#pragma omp parallel for collapse(2) schedule(static) if (N >= 16384)
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                const int64_t n = ((int64_t)z * ny + y) * nx + x;
                double fp[19], gp[3][7];
                for (int a = 0; a < 19; ++a) {
                    const int sy = y - E19[a][1], szr = z - E19[a][2];
                    const int cut_z = p->side && (szr < 0 || szr >= nz);
                    if (sy >= 0 && sy < ny && !cut_z) {
                        const int sx = (x - E19[a][0] + nx) % nx, sz = (szr + nz) % nz;
                        fp[a] = fi[a * N + ((int64_t)sz * ny + sy) * nx + sx];
                    } else if (sy < 0 || sy >= ny) {
                        /* the link crosses a wall: half-way bounce-back of the node's own outgoing
                         * population, with the moving-wall term (App. B.1) */
                        const double U = sy < 0 ? p->u_bot : p->u_top;
                        fp[a] = fi[opp(a) * N + n] + 6.0 * w19(a) * E19[a][0] * U;
                    } else {
                        fp[a] = fi[opp(a) * N + n]; /* side wall at rest: half-way bounce-back */
                    }
                }
                for (int i = 0; i < 3; ++i) {
                    for (int a = 0; a < 7; ++a) {
                        const int sy = y - E7[a][1], szr = z - E7[a][2];
                        const int cut_z = p->side && (szr < 0 || szr >= nz);
                        if (cut_z) {
                            /* side wall (parallel to B0): B_x, B_y tangential, B_z normal */
                            const double go_out = gi[(i * 7 + opp(a)) * N + n];
                            const double r = szr < 0 ? rk : rf;
                            if (i == 2)
                                gp[i][a] = -go_out;
                            else if (i == 0)
                                gp[i][a] = r * go_out;
                            else
                                gp[i][a] = r * go_out + (1.0 - r) * w7(a) * p->B0;
                        } else if (sy >= 0 && sy < ny) {
                            const int sx = (x - E7[a][0] + nx) % nx, sz = (szr + nz) % nz;
                            gp[i][a] = gi[(i * 7 + a) * N + ((int64_t)sz * ny + sy) * nx + sx];
                        } else {
                            const double go_out = gi[(i * 7 + opp(a)) * N + n];
                            const int bottom = sy < 0;
                            const double r = bottom ? rb : rt, k = bottom ? kb : kt;
                            const double U = bottom ? p->u_bot : p->u_top;
                            if (i == 1) {
                                /* normal component: anti-bounce-back to B_y = B0 */
                                gp[i][a] = -go_out + 2.0 * w7(a) * p->B0;
                            } else if (i == 0) {
                                /* B_x: weighted (anti-)bounce-back with the moving-wall term
                                 * -(2 theta/(theta+1)) W e_y B0 U / c_sm^2 */
                                gp[i][a] = r * go_out - 2.0 * k * w7(a) * E7[a][1] * p->B0 * U * 4.0;
                            } else {
                                gp[i][a] = r * go_out; /* B_z: Lambda_yz = 0 at the wall */
                            }
                        }
                    }
                }
                /* moments: rho, rho u = sum f e + F/2, B = sum g */
                double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, B[3] = {0.0, 0.0, 0.0};
                for (int a = 0; a < 19; ++a) {
                    rho += fp[a];
                    for (int d = 0; d < 3; ++d) j[d] += fp[a] * E19[a][d];
                }
                const double F[3] = {p->Fx, 0.0, 0.0};
                double u[3];
                for (int d = 0; d < 3; ++d) u[d] = (j[d] + 0.5 * F[d]) / rho;
                for (int i = 0; i < 3; ++i)
                    for (int a = 0; a < 7; ++a) B[i] += gp[i][a];
                /* BGK collisions with the source term */
                for (int a = 0; a < 19; ++a) {
                    const double fh = feq_hyd(a, rho, u);
                    double ef = 0.0;
                    for (int d = 0; d < 3; ++d) ef += (E19[a][d] - u[d]) * F[d];
                    const double S = 3.0 * ef * fh / rho;
                    fo[a * N + n] = fp[a] - om_f * (fp[a] - (fh + feq_mag(a, B))) + (1.0 - 0.5 * om_f) * S;
                }
                for (int i = 0; i < 3; ++i)
                    for (int a = 0; a < 7; ++a)
                        go[(i * 7 + a) * N + n] = gp[i][a] - om_m * (gp[i][a] - geq(a, i, u, B));
            }
        }
    }
    return 0;
}

/* Moments of the stored post-collision state: rho = sum f, rho u = sum f e - F/2, B = sum g.
 * mom: 7 x N (rho, u_x, u_y, u_z, B_x, B_y, B_z). */
void o3_moments(const o3_params* p, const double* f, const double* g, double* mom) {
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    for (int64_t n = 0; n < N; ++n) {
        double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 19; ++a) {
            rho += f[a * N + n];
            for (int d = 0; d < 3; ++d) j[d] += f[a * N + n] * E19[a][d];
        }
        j[0] -= 0.5 * p->Fx;
        mom[n] = rho;
        for (int d = 0; d < 3; ++d) mom[(1 + d) * N + n] = j[d] / rho;
        for (int i = 0; i < 3; ++i) {
            double b = 0.0;
            for (int a = 0; a < 7; ++a) b += g[(i * 7 + a) * N + n];
            mom[(4 + i) * N + n] = b;
        }
    }
}

/* n steps in place (f, g hold the state before and after). */
int o3_run(const o3_params* p, double* f, double* g, int64_t nsteps) {
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    double* f2 = (double*)malloc(sizeof(double) * 19 * N);
    double* g2 = (double*)malloc(sizeof(double) * 21 * N);
    if (!f2 || !g2) {
        free(f2);
        free(g2);
        return 2;
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        o3_step(p, f, g, f2, g2);
        memcpy(f, f2, sizeof(double) * 19 * N);
        memcpy(g, g2, sizeof(double) * 21 * N);
    }
    free(f2);
    free(g2);
    return 0;
}
