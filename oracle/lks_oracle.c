/*
 * lks_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU reference of one time step of the coupled lattice
 * kinetic scheme (LKS) for magnetohydrodynamics used by Yahia & Premnath,
 * "On Boundary Conditions for Lattice Kinetic Schemes for Magnetohydrodynamics
 * Bounded by Walls with Finite Electrical Conductivities" (arXiv 2112.13930):
 *
 *   - D2Q9 single-relaxation-time LBM for (rho, u) with a body-force source
 *     (Sec. V, Eq. LBMforflowfield), the magnetic field entering the momentum
 *     flux through the Maxwell stress in f^eq (Dellar's LKS, cited in Sec. I/IV);
 *   - D2Q5 vector LKS for the magnetic field B (Sec. IV, Eqs. LKSformagneticfield,
 *     geqmagneticfield, zerothmomentofg);
 *   - the two Shercliff thin-conducting-wall closures: link-based
 *     (Sec. VI, Eq. linkbasedBCschemefinal; moving wall App. B.1,
 *     Eq. movingwalllinkbasedclosure) with half-way bounce-back for f (Sec. VI,
 *     moving wall App. B.1), and on-node moment-based (Sec. VII,
 *     Eqs. momentbasedBCslowerboundary / momentbasedBCsupperboundary; moving
 *     wall App. B.2, Eq. momentbasedclosureformovingwall) with the moment-based
 *     no-slip closure for f (App. A, Eq. hydmomentconstraints; App. B.2).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this file.  The product library never links, calls or includes it, and it
 * shares no code, header or constant table with the CUDA path.
 *
 * Conventions (each a reading of the paper where it is silent):
 *   - lattice units: dx = dt = 1, c_s^2 = c_sm^2 = 1/3, rho0 = 1, mu_m = 1;
 *   - the channel is periodic in x; walls bound it in y;
 *   - D2Q9 directions e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1)
 *     e5=(1,1) e6=(-1,1) e7=(-1,-1) e8=(1,-1) (read off the moment expansions
 *     of App. A); D2Q5 directions are the first five (read off the closures of
 *     Sec. VI.A: the bottom wall's unknown is g_2);
 *   - the stored state is the post-collision population field; one step is
 *     "stream (with wall closures) -> moments -> equilibria -> collide";
 *   - link-based: walls half-way outside rows 0 and ny-1, half-width a = ny/2;
 *     moment-based: walls on rows 0 and ny-1, half-width a = (ny-1)/2;
 *   - moment-based f closure: the Pi_20 target is the full equilibrium value,
 *     which with the Maxwell stress in f^eq is rho (c_s^2 + U^2) + (B_y^2 -
 *     B_x^2)/2 (pi20_literal = 1 selects the printed rho (c_s^2 + U^2));
 *   - the moving-wall constraint of App. B.2 is applied as x-momentum
 *     Pi_10 = rho U_w, y-momentum Pi_01 = 0, which is what the printed closures
 *     satisfy;
 *   - c = +inf is the limit of each closure (no division by c);
 *   - coupling = 1 is the paper's own coupling (Sec. V): no magnetic term in
 *     f^eq, Lorentz force F_L = J x B in the source and in rho u = sum f e + F/2,
 *     with J_z = (Lambda^(1)_yx - Lambda^(1)_xy)/(tau_m c_sm^2) from the
 *     non-equilibrium first moment of g (Sec. IV).  Because Lambda^(0) depends on
 *     u and u on F_L, the two are iterated to a fixed point; the moment-based
 *     Pi_20 target is then rho (c_s^2 + U^2) as printed.
 *
 * Arrays are structure-of-arrays: f[a*N + j*nx + i], g[(k*5 + a)*N + j*nx + i]
 * with N = nx*ny, k = 0 for the x component and 1 for the y component.
 * Moments are mom[m*N + j*nx + i] with m = rho, u_x, u_y, B_x, B_y.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t nx, ny;
    int32_t closure;      /* 0 = link-based (Sec. VI), 1 = moment-based (Sec. VII) */
    int32_t pi20_literal; /* 1 = Pi_20 target rho (c_s^2 + U^2) exactly as printed */
    int32_t freeze_u;     /* 1 = u forced to 0 in g^eq (pure induction-diffusion) */
    int32_t coupling;     /* 0 = Maxwell stress in f^eq; 1 = Lorentz-force source (Sec. IV-V) */
    double tau_f, tau_m;  /* relaxation times of f and g */
    double B0;            /* applied field along y */
    double Fx;            /* external body force along x */
    double c_bot, c_top;  /* wall conductance ratios (>= 0, +inf allowed) */
    double u_bot, u_top;  /* tangential wall speeds */
} orc_params;

#define CS2 (1.0 / 3.0)

/* D2Q9 lattice (Sec. V) */
static const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W9[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* D2Q5 lattice (Sec. IV) */
static const int EX5[5] = {0, 1, 0, -1, 0};
static const int EY5[5] = {0, 0, 1, 0, -1};
static const double W5[5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
static const int OPP5[5] = {0, 3, 4, 1, 2};

static int nthreads_used = 1;

int orc_threads(void) { return nthreads_used; }

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Channel half-width a for each closure's wall placement. */
double orc_half_width(const orc_params* p) {
    return p->closure == 0 ? 0.5 * p->ny : 0.5 * (p->ny - 1);
}

/* f^eq of Sec. V (hydrodynamic part only). */
static double feq_hyd(int a, double rho, double ux, double uy) {
    double eu = EX9[a] * ux + EY9[a] * uy;
    double uu = ux * ux + uy * uy;
    return W9[a] * rho * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Maxwell-stress part of f^eq: w_a (|B|^2 I/2 - BB) : (e e - c_s^2 I) / (2 c_s^4). */
static double feq_mag(int a, double bx, double by) {
    double e2 = (double)(EX9[a] * EX9[a] + EY9[a] * EY9[a]);
    double eb = EX9[a] * bx + EY9[a] * by;
    double b2 = bx * bx + by * by;
    return W9[a] * (0.5 * b2 * e2 - eb * eb) / (2.0 * CS2 * CS2);
}

/* g^eq of Eq. geqmagneticfield: W_a { B_i + e_aj (u_j B_i - B_j u_i) / c_sm^2 }. */
static double geq(int a, int i, double ux, double uy, double bx, double by) {
    double u[2] = {ux, uy}, b[2] = {bx, by}, e[2] = {(double)EX5[a], (double)EY5[a]};
    double s = 0.0;
    for (int j = 0; j < 2; ++j) s += e[j] * (u[j] * b[i] - b[j] * u[i]);
    return W5[a] * (b[i] + s / CS2);
}

/* Source term of Sec. V: S_a = (e_a - u) . F f^eq_a / (rho c_s^2), with the
 * hydrodynamic f^eq (the Maxwell stress already carries the Lorentz force). */
static double source(int a, double rho, double ux, double uy, double fx, double fy) {
    double d = (EX9[a] - ux) * fx + (EY9[a] - uy) * fy;
    return d * feq_hyd(a, rho, ux, uy) / (rho * CS2);
}

/* Counter-based perturbation: SplitMix64 (Steele, Lea & Flood 2014) applied
 * to seed XOR counter, mapped to [0,1) with 53 bits. */
static double splitmix_unit(uint64_t seed, uint64_t counter) {
    uint64_t z = (seed ^ counter) + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* Initial state: equilibria at rho = 1, B = (0, B0), u = u0 where u0 = 0 or
 * uniform in [-amp, amp] per component from the counter-based generator
 * (counter 2*node for u_x, 2*node+1 for u_y). */
int orc_init(const orc_params* p, uint64_t seed, double amp, double* f, double* g) {
    const int nx = p->nx, ny = p->ny;
    const long N = (long)nx * ny;
    if (nx < 1 || ny < 2) return 1;
    for (long n = 0; n < N; ++n) {
        double ux = 0.0, uy = 0.0;
        if (amp != 0.0) {
            ux = amp * (2.0 * splitmix_unit(seed, 2ULL * (uint64_t)n) - 1.0);
            uy = amp * (2.0 * splitmix_unit(seed, 2ULL * (uint64_t)n + 1ULL) - 1.0);
        }
        for (int a = 0; a < 9; ++a)
            f[a * N + n] = feq_hyd(a, 1.0, ux, uy) + (p->coupling == 1 ? 0.0 : feq_mag(a, 0.0, p->B0));
        for (int i = 0; i < 2; ++i)
            for (int a = 0; a < 5; ++a)
                g[(i * 5 + a) * N + n] = geq(a, i, ux, uy, 0.0, p->B0);
    }
    return 0;
}

/* Link-based coefficients of Eq. movingwalllinkbasedclosure with
 * theta = c a / (tau_m - 1/2) (Eq. weightingfactor): r = (theta-1)/(theta+1),
 * s = 2 theta/(theta+1); theta = +inf gives the bounce-back limit r = 1, s = 2. */
static void link_coeffs(double c, double a, double tau_m, double* r, double* s) {
    if (isinf(c)) { *r = 1.0; *s = 2.0; return; }
    double theta = c * a / (tau_m - 0.5);
    *r = (theta - 1.0) / (theta + 1.0);
    *s = 2.0 * theta / (theta + 1.0);
}

/* One full step.  fs, gs: post-collision state at time t.  fo, go: post-
 * collision state at t+1.  fpre, gpre (nullable): post-stream, post-closure,
 * pre-collision populations.  mom (nullable): the moments used in the
 * collision. */
int orc_step(const orc_params* p, const double* fs, const double* gs, double* fo, double* go,
             double* fpre, double* gpre, double* mom) {
    const int nx = p->nx, ny = p->ny;
    const long N = (long)nx * ny;
    if (nx < 1 || ny < (p->closure == 0 ? 2 : 3)) return 1;
    if (!(p->tau_f > 0.5) || !(p->tau_m > 0.5)) return 1;
    if (!(p->c_bot >= 0.0) || !(p->c_top >= 0.0)) return 1;
    /* the Lorentz-force coupling reads J back from the stored (post-collision) g, which carries
     * (1 - 1/tau_m) of the non-equilibrium moment: tau_m must stay away from 1 */
    if (p->coupling == 1 && fabs(p->tau_m - 1.0) < 0.05) return 1;
    const double a_half = orc_half_width(p);
    double rb, sb, rt, st;
    link_coeffs(p->c_bot, a_half, p->tau_m, &rb, &sb);
    link_coeffs(p->c_top, a_half, p->tau_m, &rt, &st);
    const double beta_b = p->c_bot * a_half / (p->tau_m * CS2); /* c a / (tau_m c_sm^2) */
    const double beta_t = p->c_top * a_half / (p->tau_m * CS2);
    const double B0 = p->B0;
    int used = 1;

    /* small lattices run on one thread: a parallel region per step costs more than the work */
#pragma omp parallel if (N >= 16384)
    {
#ifdef _OPENMP
#pragma omp single
        used = omp_get_num_threads();
#endif
#pragma omp for schedule(static)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                const long n = (long)j * nx + i;
                double f[9], g[2][5];
                int known9[9], known5[5];
                /* 1. Streaming (left side of Eqs. LBMforflowfield and
                 *    LKSformagneticfield): pull from x - e_a, periodic in x. */
                for (int a = 0; a < 9; ++a) {
                    int si = ((i - EX9[a]) % nx + nx) % nx, sj = j - EY9[a];
                    known9[a] = (sj >= 0 && sj < ny);
                    f[a] = known9[a] ? fs[a * N + (long)sj * nx + si] : 0.0;
                }
                for (int a = 0; a < 5; ++a) {
                    int si = ((i - EX5[a]) % nx + nx) % nx, sj = j - EY5[a];
                    known5[a] = (sj >= 0 && sj < ny);
                    for (int k = 0; k < 2; ++k)
                        g[k][a] = known5[a] ? gs[(k * 5 + a) * N + (long)sj * nx + si] : 0.0;
                }
                /* 2. Wall closures for the populations that would come from
                 *    outside the channel. */
                if (p->closure == 0) {
                    /* Link-based, wall half-way outside the row. */
                    for (int a = 0; a < 9; ++a) {
                        if (known9[a]) continue;
                        double uw = (EY9[a] > 0) ? p->u_bot : p->u_top;
                        /* half-way bounce-back with Ladd's moving-wall term (App. B.1) */
                        f[a] = fs[OPP9[a] * N + n] + 2.0 * W9[a] * EX9[a] * uw / CS2;
                    }
                    for (int a = 0; a < 5; ++a) {
                        if (known5[a]) continue;
                        int bottom = EY5[a] > 0;
                        double uw = bottom ? p->u_bot : p->u_top;
                        double r = bottom ? rb : rt, s = bottom ? sb : st;
                        /* tangential component: Eq. movingwalllinkbasedclosure,
                         * Lambda^(0)_yx = -B0 U_w at the wall */
                        g[0][a] = r * gs[(0 * 5 + OPP5[a]) * N + n] -
                                  s * W5[a] * EY5[a] * B0 * uw / CS2;
                        /* normal component: Eq. magneticfieldanditsgradientrelation1
                         * with B_y = B0 at the wall */
                        g[1][a] = -gs[(1 * 5 + OPP5[a]) * N + n] + 2.0 * W5[a] * B0;
                    }
                } else if (j == 0 || j == ny - 1) {
                    /* Moment-based, wall on the node.  g first (Sec. VII, App. B.2). */
                    const int bottom = (j == 0);
                    const double uw = bottom ? p->u_bot : p->u_top;
                    const double c = bottom ? p->c_bot : p->c_top;
                    const double beta = bottom ? beta_b : beta_t;
                    if (bottom) {
                        /* Shercliff at y=-a: (1/(tau_m c^2)) (g2x - g4x + B0 U) + B_x/(c a) = 0,
                         * multiplied through by c a; the limit c = inf is g2x = g4x - B0 U. */
                        if (isinf(c))
                            g[0][2] = g[0][4] - B0 * uw;
                        else
                            g[0][2] = ((beta - 1.0) * g[0][4] - (g[0][0] + g[0][1] + g[0][3]) -
                                       beta * B0 * uw) / (beta + 1.0);
                        g[1][2] = B0 - (g[1][0] + g[1][1] + g[1][3] + g[1][4]);
                    } else {
                        /* Shercliff at y=+a (Eq. momentbasedclosureformovingwall). */
                        if (isinf(c))
                            g[0][4] = g[0][2] + B0 * uw;
                        else
                            g[0][4] = ((beta - 1.0) * g[0][2] - (g[0][0] + g[0][1] + g[0][3]) +
                                       beta * B0 * uw) / (beta + 1.0);
                        g[1][4] = B0 - (g[1][0] + g[1][1] + g[1][2] + g[1][3]);
                    }
                    double bx = 0.0, by = 0.0;
                    for (int a = 0; a < 5; ++a) { bx += g[0][a]; by += g[1][a]; }
                    /* Momentum targets.  Maxwell-stress coupling: Pi_10 = rho U, Pi_01 = 0 as printed.
                     * Lorentz-force coupling: the wall node's velocity (Pi + F/2)/rho is set to
                     * (U, 0), i.e. Pi_10 = rho U - F_x/2, Pi_01 = -F_y/2, with F = F_ext + J x B and
                     * J_z from the closed g at u = (U, 0). */
                    double hfx = 0.0, hfy = 0.0;
                    if (p->coupling == 1) {
                        const double lyx = g[0][2] - g[0][4], lxy = g[1][1] - g[1][3];
                        const double l0yx = -by * uw, l0xy = uw * by;
                        const double jz = ((lyx - l0yx) - (lxy - l0xy)) / (p->tau_m * CS2);
                        hfx = 0.5 * (p->Fx - jz * by);
                        hfy = 0.5 * (jz * bx);
                    }
                    if (bottom) {
                        /* App. A: rho_b from Pi_00 and Pi_01 */
                        double rho = f[0] + f[1] + f[3] + 2.0 * (f[4] + f[7] + f[8]) - hfy;
                        double P = rho * (CS2 + uw * uw);
                        if (!p->pi20_literal && p->coupling == 0) P += 0.5 * (by * by - bx * bx);
                        f[2] = -P + f[1] + f[3] + f[4] + 2.0 * (f[7] + f[8]) - hfy;
                        f[5] = 0.5 * (P + rho * uw - hfx) - (f[1] + f[8]);
                        f[6] = 0.5 * (P - rho * uw + hfx) - (f[3] + f[7]);
                    } else {
                        double rho = f[0] + f[1] + f[3] + 2.0 * (f[2] + f[5] + f[6]) + hfy;
                        double P = rho * (CS2 + uw * uw);
                        if (!p->pi20_literal && p->coupling == 0) P += 0.5 * (by * by - bx * bx);
                        f[4] = -P + f[1] + f[2] + f[3] + 2.0 * (f[5] + f[6]) + hfy;
                        f[7] = 0.5 * (P - rho * uw + hfx) - (f[3] + f[6]);
                        f[8] = 0.5 * (P + rho * uw - hfx) - (f[1] + f[5]);
                    }
                }
                if (fpre) for (int a = 0; a < 9; ++a) fpre[a * N + n] = f[a];
                if (gpre)
                    for (int k = 0; k < 2; ++k)
                        for (int a = 0; a < 5; ++a) gpre[(k * 5 + a) * N + n] = g[k][a];
                /* 3. Moments (Sec. V, Eq. zerothmomentofg). */
                double rho = 0.0, mx = 0.0, my = 0.0, bx = 0.0, by = 0.0;
                for (int a = 0; a < 9; ++a) {
                    rho += f[a];
                    mx += f[a] * EX9[a];
                    my += f[a] * EY9[a];
                }
                for (int a = 0; a < 5; ++a) { bx += g[0][a]; by += g[1][a]; }
                double Fx = p->Fx, Fy = 0.0;
                double ux = (mx + 0.5 * Fx) / rho, uy = (my + 0.5 * Fy) / rho;
                if (p->coupling == 1) {
                    /* Lambda_ji = sum_a e_aj g_ai (Sec. IV): Lambda_yx and Lambda_xy */
                    const double lyx = g[0][2] - g[0][4], lxy = g[1][1] - g[1][3];
                    for (int it = 0; it < 100; ++it) {
                        /* Lambda^(0)_ji = u_j B_i - B_j u_i (Eq. rank2antisymmtensoreq) */
                        const double l0yx = uy * bx - by * ux, l0xy = ux * by - bx * uy;
                        /* J_z = -(1/(tau_m c_sm^2)) eps_zjk Lambda^(1)_jk */
                        const double jz = ((lyx - l0yx) - (lxy - l0xy)) / (p->tau_m * CS2);
                        /* F = J x B + F_ext with J = (0, 0, J_z), B = (B_x, B_y, 0) */
                        Fx = p->Fx - jz * by;
                        Fy = jz * bx;
                        const double nux = (mx + 0.5 * Fx) / rho, nuy = (my + 0.5 * Fy) / rho;
                        const double d = fabs(nux - ux) + fabs(nuy - uy);
                        ux = nux;
                        uy = nuy;
                        if (d <= 1e-17 * (fabs(ux) + fabs(uy)) || d == 0.0) break;
                    }
                }
                if (mom) {
                    mom[0 * N + n] = rho; mom[1 * N + n] = ux; mom[2 * N + n] = uy;
                    mom[3 * N + n] = bx; mom[4 * N + n] = by;
                }
                /* 4./5. Equilibria, source and BGK collision (Eqs. LBMforflowfield,
                 *       LKSformagneticfield). */
                for (int a = 0; a < 9; ++a) {
                    double feq = feq_hyd(a, rho, ux, uy) + (p->coupling == 1 ? 0.0 : feq_mag(a, bx, by));
                    double S = source(a, rho, ux, uy, Fx, Fy);
                    fo[a * N + n] = f[a] - (f[a] - feq) / p->tau_f + (1.0 - 0.5 / p->tau_f) * S;
                }
                double gux = p->freeze_u ? 0.0 : ux, guy = p->freeze_u ? 0.0 : uy;
                for (int k = 0; k < 2; ++k)
                    for (int a = 0; a < 5; ++a) {
                        double ge = geq(a, k, gux, guy, bx, by);
                        go[(k * 5 + a) * N + n] = g[k][a] - (g[k][a] - ge) / p->tau_m;
                    }
            }
        }
    }
    nthreads_used = used;
    return 0;
}

/* nsteps steps in place (f, g hold the post-collision state). */
int orc_run(const orc_params* p, double* f, double* g, int64_t nsteps) {
    const long N = (long)p->nx * p->ny;
    double* f2 = (double*)malloc(sizeof(double) * 9 * N);
    double* g2 = (double*)malloc(sizeof(double) * 10 * N);
    if (!f2 || !g2) { free(f2); free(g2); return 2; }
    int rc = 0;
    for (int64_t s = 0; s < nsteps && rc == 0; ++s) {
        rc = orc_step(p, f, g, f2, g2, NULL, NULL, NULL);
        if (rc == 0) {
            memcpy(f, f2, sizeof(double) * 9 * N);
            memcpy(g, g2, sizeof(double) * 10 * N);
        }
    }
    free(f2);
    free(g2);
    return rc;
}

/* Moments of a stored post-collision state.  Collision conserves sum f and
 * sum g and adds F to sum f e, so rho = sum f~, rho u = sum f~ e - F/2,
 * B = sum g~ reproduce the moments that entered that collision. */
void orc_moments(const orc_params* p, const double* f, const double* g, double* mom) {
    const long N = (long)p->nx * p->ny;
    for (long n = 0; n < N; ++n) {
        double rho = 0.0, mx = 0.0, my = 0.0, bx = 0.0, by = 0.0;
        for (int a = 0; a < 9; ++a) {
            rho += f[a * N + n];
            mx += f[a * N + n] * EX9[a];
            my += f[a * N + n] * EY9[a];
        }
        for (int a = 0; a < 5; ++a) { bx += g[a * N + n]; by += g[(5 + a) * N + n]; }
        double ux = (mx - 0.5 * p->Fx) / rho, uy = my / rho;
        if (p->coupling == 1) {
            /* The collision relaxes Lambda - Lambda^(0) by the factor (1 - 1/tau_m), so the
             * stored state carries (1 - 1/tau_m) Lambda^(1) of the last step: J_z (and with it
             * F_L and the F/2 shift of u) is recovered from it, iterated with u as in the step. */
            const double lyx = g[2 * N + n] - g[4 * N + n], lxy = g[(5 + 1) * N + n] - g[(5 + 3) * N + n];
            for (int it = 0; it < 100; ++it) {
                const double l0yx = uy * bx - by * ux, l0xy = ux * by - bx * uy;
                const double jz = ((lyx - l0yx) - (lxy - l0xy)) / ((1.0 - 1.0 / p->tau_m) * p->tau_m * CS2);
                const double fx = p->Fx - jz * by, fy = jz * bx;
                const double nux = (mx - 0.5 * fx) / rho, nuy = (my - 0.5 * fy) / rho;
                const double d = fabs(nux - ux) + fabs(nuy - uy);
                ux = nux;
                uy = nuy;
                if (d <= 1e-17 * (fabs(ux) + fabs(uy)) || d == 0.0) break;
            }
        }
        mom[0 * N + n] = rho;
        mom[1 * N + n] = ux;
        mom[2 * N + n] = uy;
        mom[3 * N + n] = bx;
        mom[4 * N + n] = by;
    }
}
