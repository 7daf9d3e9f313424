/*
 * lbm_oracle.c -- plain FP64 CPU oracle for the lattice Boltzmann permeability
 * method of Li, Ho, Wu & Zhang, "Lattice Boltzmann modelling of intrinsic
 * permeability" (arXiv:1609.09685).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
 * that the CUDA library is checked against.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * header, table or constant generator with the CUDA library: lattice tables,
 * boundary rules, the QSGS generator and the splitmix64 hash are written out
 * here independently.
 *
 * Everything is double precision, single-threaded, with plain loops in the
 * order the method states.  Build with -O2 -ffp-contract=off (no fast-math).
 *
 * Layout: node n = (z*ny + y)*nx + x (x fastest); populations f[n*Q + i]
 * (unshifted, f = physical distribution).  Solid nodes carry f = 0 and are never
 * read.  2D problems use nz = 1 and the D2Q9 lattice.
 *
 * What each function follows:
 *   - Eq. (1): nu = (tau - 1/2)/3 in lattice units (c = dx = dt = 1).
 *   - Sec. 2, D2Q9/D3Q19 BGK with the Qian et al. (1992) lattices and the
 *     quadratic equilibrium; the linear (Stokes) equilibrium is the variant the
 *     paper's 3D discussion uses ("remove the nonlinear velocity terms").
 *   - Sec. 2, Fig. 1: pressure boundary at inlet/outlet (read as the Zou & He
 *     1997 pressure condition; in 3D the Hecht & Harting 2010 form), symmetric
 *     boundary at top/bottom (read as specular reflection), solids by halfway
 *     bounce-back (the paper is silent on the wall rule).
 *   - Sec. 2: permeability from the mass flow rate (the link flux through the
 *     cross-section planes) by Darcy's law.
 *   - Sec. 2: Kn = sqrt(pi/6) (tau - 1/2) / N_x.
 *   - Sec. 2 ("randomly generated quartet structure"): QSGS (Wang et al. 2007)
 *     growth of the solid phase driven by a counter-based splitmix64 hash
 *     (Steele, Lea & Flood 2014), with an exact target solid count.
 *   - Sec. 2 (multi-relaxation models): the TRT collision (Ginzburg 2005).
 *   - Sec. 2, Eq. (2): force-driven flow with every face periodic and the
 *     forcing of Guo, Zheng & Shi (2002); k = nu <u> / g.
 *   - Sec. 2 (local Knudsen number): brute-force distance to the nearest solid
 *     node, pore size 2 D - 1.
 * Every function is pinned by the CPU tests (closed forms, invariants,
 * published values); only the paper-level figure curves are unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Lattices                                                                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    int q;
    int c[19][3];
    double w[19];
    int opp[19];
} lattice;

/* D2Q9 ordering: 0 rest; 1 (1,0); 2 (0,1); 3 (-1,0); 4 (0,-1);
 * 5 (1,1); 6 (-1,1); 7 (-1,-1); 8 (1,-1).  Weights 4/9, 1/9, 1/36. */
static void make_d2q9(lattice* L) {
    static const int c[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                                {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    L->q = 9;
    for (int i = 0; i < 9; ++i) {
        L->c[i][0] = c[i][0];
        L->c[i][1] = c[i][1];
        L->c[i][2] = 0;
        int n2 = c[i][0] * c[i][0] + c[i][1] * c[i][1];
        L->w[i] = (n2 == 0) ? 4.0 / 9.0 : (n2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
}

/* D3Q19 ordering: 0 rest; 1..6 the faces (+x,-x,+y,-y,+z,-z); 7..18 the
 * edges in opposite pairs.  Weights 1/3, 1/18, 1/36. */
static void make_d3q19(lattice* L) {
    static const int c[19][3] = {
        {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
        {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
        {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    L->q = 19;
    for (int i = 0; i < 19; ++i) {
        int n2 = 0;
        for (int a = 0; a < 3; ++a) {
            L->c[i][a] = c[i][a];
            n2 += c[i][a] * c[i][a];
        }
        L->w[i] = (n2 == 0) ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
}

/* The direction whose velocity is c with the listed components negated. */
static int find_dir(const lattice* L, int cx, int cy, int cz) {
    for (int j = 0; j < L->q; ++j)
        if (L->c[j][0] == cx && L->c[j][1] == cy && L->c[j][2] == cz) return j;
    return -1;
}

static void finish_lattice(lattice* L) {
    for (int i = 0; i < L->q; ++i)
        L->opp[i] = find_dir(L, -L->c[i][0], -L->c[i][1], -L->c[i][2]);
}

static int get_lattice(int q, lattice* L) {
    if (q == 9)
        make_d2q9(L);
    else if (q == 19)
        make_d3q19(L);
    else
        return -1;
    finish_lattice(L);
    return 0;
}

/* Exported copies of the tables so tests can check them against the text. */
int oc_lattice(int q, int* c_out /* q*3 */, double* w_out, int* opp_out) {
    lattice L;
    if (get_lattice(q, &L)) return -1;
    for (int i = 0; i < L.q; ++i) {
        for (int a = 0; a < 3; ++a) c_out[i * 3 + a] = L.c[i][a];
        w_out[i] = L.w[i];
        opp_out[i] = L.opp[i];
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Equilibrium and collision                                                  */
/* ------------------------------------------------------------------------- */

enum { EQ_QUADRATIC = 0, EQ_LINEAR = 1 };

/* f_eq_i = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)  (quadratic, c_s^2=1/3)
 * f_eq_i = w_i (rho + 3 c.j)                               (linear / Stokes) */
static double feq(const lattice* L, int i, double rho, const double j[3], int eq) {
    double cj = L->c[i][0] * j[0] + L->c[i][1] * j[1] + L->c[i][2] * j[2];
    if (eq == EQ_LINEAR) return L->w[i] * (rho + 3.0 * cj);
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    double cu = cj / rho;
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return L->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

static void moments(const lattice* L, const double* f, double* rho, double j[3]) {
    *rho = 0.0;
    j[0] = j[1] = j[2] = 0.0;
    for (int i = 0; i < L->q; ++i) {
        *rho += f[i];
        j[0] += L->c[i][0] * f[i];
        j[1] += L->c[i][1] * f[i];
        j[2] += L->c[i][2] * f[i];
    }
}

/* ------------------------------------------------------------------------- */
/* Zou-He pressure boundaries (u_y = u_z = 0)                                 */
/* ------------------------------------------------------------------------- */

/* D2Q9, Zou & He (1997).  Inlet x = 0: unknown f1, f5, f8. */
static void zou_he_d2q9_inlet(double* f, double rho_in) {
    double rux = rho_in - (f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7]));
    f[1] = f[3] + (2.0 / 3.0) * rux;
    f[5] = f[7] - 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * rux;
    f[8] = f[6] + 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * rux;
}

/* D2Q9 outlet x = N_x - 1: unknown f3, f6, f7. */
static void zou_he_d2q9_outlet(double* f, double rho_out) {
    double rux = (f[0] + f[2] + f[4] + 2.0 * (f[1] + f[5] + f[8])) - rho_out;
    f[3] = f[1] - (2.0 / 3.0) * rux;
    f[7] = f[5] + 0.5 * (f[2] - f[4]) - (1.0 / 6.0) * rux;
    f[6] = f[8] - 0.5 * (f[2] - f[4]) - (1.0 / 6.0) * rux;
}

/* D3Q19, Hecht & Harting (2010) form with transverse corrections N_y, N_z.
 * Inlet x = 0: unknown 1 (1,0,0), 7 (1,1,0), 9 (1,-1,0), 11 (1,0,1), 13 (1,0,-1). */
static void zou_he_d3q19_inlet(double* f, double rho_in) {
    double s0 = f[0] + f[3] + f[4] + f[5] + f[6] + f[15] + f[16] + f[17] + f[18];
    double sm = f[2] + f[8] + f[10] + f[12] + f[14];
    double rux = rho_in - (s0 + 2.0 * sm);
    double ny = 0.5 * (f[3] - f[4] + f[15] - f[16] + f[17] - f[18]);
    double nz = 0.5 * (f[5] - f[6] + f[15] - f[16] - f[17] + f[18]);
    f[1] = f[2] + rux / 3.0;
    f[7] = f[8] + rux / 6.0 - ny;
    f[9] = f[10] + rux / 6.0 + ny;
    f[11] = f[12] + rux / 6.0 - nz;
    f[13] = f[14] + rux / 6.0 + nz;
}

/* D3Q19 outlet x = N_x - 1: unknown 2, 8, 10, 12, 14. */
static void zou_he_d3q19_outlet(double* f, double rho_out) {
    double s0 = f[0] + f[3] + f[4] + f[5] + f[6] + f[15] + f[16] + f[17] + f[18];
    double sp = f[1] + f[7] + f[9] + f[11] + f[13];
    double rux = (s0 + 2.0 * sp) - rho_out;
    double ny = 0.5 * (f[3] - f[4] + f[15] - f[16] + f[17] - f[18]);
    double nz = 0.5 * (f[5] - f[6] + f[15] - f[16] - f[17] + f[18]);
    f[2] = f[1] - rux / 3.0;
    f[8] = f[7] - rux / 6.0 + ny;
    f[10] = f[9] - rux / 6.0 - ny;
    f[12] = f[11] - rux / 6.0 + nz;
    f[14] = f[13] - rux / 6.0 - nz;
}

/* ------------------------------------------------------------------------- */
/* One time step                                                              */
/* ------------------------------------------------------------------------- */

static int check_dims(int q, int nx, int ny, int nz) {
    if (nx < 3 || ny < 1 || nz < 1) return -1;
    if (q == 9 && nz != 1) return -1;
    return 0;
}

/*
 * fin: post-collision populations of step t; fout: post-collision populations of
 * step t+1.  Pull streaming, for each fluid node d and direction i with source
 * s = d - c_i:
 *   - s_x outside [0, N_x): unknown, set by the pressure boundary below;
 *   - an out-of-range s_y (s_z) is mirrored back onto d's row (plane) and the
 *     y (z) component of the direction flips (specular symmetry plane half a
 *     link outside the domain);
 *   - s solid: f_i(d) = f*_opp(i)(d)  (halfway bounce-back);
 *   - otherwise f_i(d) = f*_j(s), j the (possibly mirrored) direction.
 * Then Zou-He at fluid nodes of x = 0 and x = N_x - 1, moments, BGK relaxation
 * f* = f - (f - f_eq)/tau.
 */
static int step_impl(int q, int nx, int ny, int nz, const uint8_t* solid, double tau, double tau_minus,
                     int trt, double rho_in, double rho_out, int eq, const double* fin, double* fout) {
    lattice L;
    if (get_lattice(q, &L) || check_dims(q, nx, ny, nz) || !(tau > 0.5) || !(tau_minus > 0.5)) return -1;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long n = ((long)z * ny + y) * nx + x;
                double* out = fout + n * q;
                if (solid[n]) {
                    for (int i = 0; i < q; ++i) out[i] = 0.0;
                    continue;
                }
                double f[19];
                for (int i = 0; i < q; ++i) {
                    int sx = x - L.c[i][0], sy = y - L.c[i][1], sz = z - L.c[i][2];
                    if (sx < 0 || sx >= nx) {
                        f[i] = 0.0; /* unknown: Zou-He sets it */
                        continue;
                    }
                    int jx = L.c[i][0], jy = L.c[i][1], jz = L.c[i][2];
                    int mirrored = 0;
                    if (sy < 0 || sy >= ny) {
                        sy = y;
                        jy = -jy;
                        mirrored = 1;
                    }
                    if (sz < 0 || sz >= nz) {
                        sz = z;
                        jz = -jz;
                        mirrored = 1;
                    }
                    int j = mirrored ? find_dir(&L, jx, jy, jz) : i;
                    long s = ((long)sz * ny + sy) * nx + sx;
                    if (solid[s])
                        f[i] = fin[n * q + L.opp[i]];
                    else
                        f[i] = fin[s * q + j];
                }
                if (x == 0) {
                    if (q == 9) zou_he_d2q9_inlet(f, rho_in);
                    else zou_he_d3q19_inlet(f, rho_in);
                }
                if (x == nx - 1) {
                    if (q == 9) zou_he_d2q9_outlet(f, rho_out);
                    else zou_he_d3q19_outlet(f, rho_out);
                }
                double rho, j[3];
                moments(&L, f, &rho, j);
                if (!trt) {
                    for (int i = 0; i < q; ++i) out[i] = f[i] - (f[i] - feq(&L, i, rho, j, eq)) / tau;
                } else {
                    /* TRT: the parts of f and f_eq even and odd under i -> opp(i)
                     * relax with 1/tau and 1/tau_minus respectively. */
                    for (int i = 0; i < q; ++i) {
                        const int o = L.opp[i];
                        const double ei = feq(&L, i, rho, j, eq), eo = feq(&L, o, rho, j, eq);
                        const double fp = 0.5 * (f[i] + f[o]), fm = 0.5 * (f[i] - f[o]);
                        const double ep = 0.5 * (ei + eo), em = 0.5 * (ei - eo);
                        out[i] = f[i] - (fp - ep) / tau - (fm - em) / tau_minus;
                    }
                }
            }
    return 0;
}

int oc_step(int q, int nx, int ny, int nz, const uint8_t* solid, double tau,
            double rho_in, double rho_out, int eq, const double* fin, double* fout) {
    return step_impl(q, nx, ny, nz, solid, tau, tau, 0, rho_in, rho_out, eq, fin, fout);
}

/*
 * Two-relaxation-time collision (Ginzburg 2005; the paper's Sec. 2 points to
 * multi-relaxation models for a wall location independent of viscosity): the
 * symmetric parts relax with tau (viscosity nu = (tau - 1/2)/3, as in BGK),
 * the antisymmetric parts with tau_minus.  Steady solutions depend on tau and
 * tau_minus only through Lambda = (tau - 1/2)(tau_minus - 1/2).
 */
int oc_step_trt(int q, int nx, int ny, int nz, const uint8_t* solid, double tau, double tau_minus,
                double rho_in, double rho_out, int eq, const double* fin, double* fout) {
    return step_impl(q, nx, ny, nz, solid, tau, tau_minus, 1, rho_in, rho_out, eq, fin, fout);
}

/*
 * Force-driven periodic flow (Sec. 2, the 3D experiment; Eq. 2): every face is
 * periodic, solids bounce back half way, and a body acceleration g along +x
 * drives the flow through the forcing of Guo, Zheng & Shi (2002).  With the
 * force density F = rho_0 g e_x (rho_0 = 1, the reference density of the
 * incompressible Stokes reading) the equilibrium takes the momentum j' = j + F/2,
 * and
 *   f' = f - (f - f_eq(rho, j'))/tau + (1 - 1/(2 tau)) S_i,
 *   S_i = w_i [3 (c_i - u') . F + 9 (c_i . u')(c_i . F)],  u' = j'/rho  (quadratic),
 *   S_i = 3 w_i c_i . F                                                (linear).
 * With the linear (Stokes) equilibrium every term is linear in (f, g).
 */
static int step_forced_impl(int q, int nx, int ny, int nz, const uint8_t* solid, double tau, double tau_minus,
                            int trt, double g, int eq, const double* fin, double* fout) {
    lattice L;
    if (get_lattice(q, &L) || nx < 1 || ny < 1 || nz < 1 || (q == 9 && nz != 1) || !(tau > 0.5) ||
        !(tau_minus > 0.5))
        return -1;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long n = ((long)z * ny + y) * nx + x;
                double* out = fout + n * q;
                if (solid[n]) {
                    for (int i = 0; i < q; ++i) out[i] = 0.0;
                    continue;
                }
                double f[19];
                for (int i = 0; i < q; ++i) {
                    int sx = ((x - L.c[i][0]) % nx + nx) % nx;
                    int sy = ((y - L.c[i][1]) % ny + ny) % ny;
                    int sz = ((z - L.c[i][2]) % nz + nz) % nz;
                    long s = ((long)sz * ny + sy) * nx + sx;
                    f[i] = solid[s] ? fin[n * q + L.opp[i]] : fin[s * q + i];
                }
                double rho, j[3];
                moments(&L, f, &rho, j);
                const double F[3] = {g, 0.0, 0.0}; /* rho_0 g, rho_0 = 1 */
                const double js[3] = {j[0] + 0.5 * F[0], j[1], j[2]};
                const double us[3] = {js[0] / rho, js[1] / rho, js[2] / rho};
                double S[19], E[19];
                for (int i = 0; i < q; ++i) {
                    const double cF = L.c[i][0] * F[0] + L.c[i][1] * F[1] + L.c[i][2] * F[2];
                    if (eq == EQ_LINEAR) {
                        S[i] = 3.0 * L.w[i] * cF;
                    } else {
                        const double cu = L.c[i][0] * us[0] + L.c[i][1] * us[1] + L.c[i][2] * us[2];
                        const double uF = us[0] * F[0] + us[1] * F[1] + us[2] * F[2];
                        S[i] = L.w[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
                    }
                    E[i] = feq(&L, i, rho, js, eq);
                }
                for (int i = 0; i < q; ++i) {
                    if (!trt) {
                        out[i] = f[i] - (f[i] - E[i]) / tau + (1.0 - 0.5 / tau) * S[i];
                    } else {
                        /* TRT: even and odd parts of f - f_eq and of the source
                         * relax with 1/tau and 1/tau_minus */
                        const int o = L.opp[i];
                        const double fp = 0.5 * (f[i] + f[o]), fm = 0.5 * (f[i] - f[o]);
                        const double ep = 0.5 * (E[i] + E[o]), em = 0.5 * (E[i] - E[o]);
                        const double sp = 0.5 * (S[i] + S[o]), sm = 0.5 * (S[i] - S[o]);
                        out[i] = f[i] - (fp - ep) / tau - (fm - em) / tau_minus + (1.0 - 0.5 / tau) * sp +
                                 (1.0 - 0.5 / tau_minus) * sm;
                    }
                }
            }
    return 0;
}

int oc_step_forced(int q, int nx, int ny, int nz, const uint8_t* solid, double tau, double g, int eq,
                   const double* fin, double* fout) {
    return step_forced_impl(q, nx, ny, nz, solid, tau, tau, 0, g, eq, fin, fout);
}

/* The same step with the TRT collision (see oc_step_trt); the even and odd
 * parts of the forcing source take the factors (1 - 1/(2 tau)) and
 * (1 - 1/(2 tau_minus)). */
int oc_step_forced_trt(int q, int nx, int ny, int nz, const uint8_t* solid, double tau, double tau_minus,
                       double g, int eq, const double* fin, double* fout) {
    return step_forced_impl(q, nx, ny, nz, solid, tau, tau_minus, 1, g, eq, fin, fout);
}

/* nsteps steps in place on f; tau_minus <= 0 means BGK. */
int oc_run_forced(int q, int nx, int ny, int nz, const uint8_t* solid, double tau, double tau_minus, double g,
                  int eq, double* f, long nsteps) {
    long nn = (long)nx * ny * nz * q;
    double* tmp = (double*)malloc(sizeof(double) * nn);
    if (!tmp) return -2;
    const int trt = tau_minus > 0.0;
    for (long t = 0; t < nsteps; ++t) {
        int rc = step_forced_impl(q, nx, ny, nz, solid, tau, trt ? tau_minus : tau, trt, g, eq, f, tmp);
        if (rc) {
            free(tmp);
            return rc;
        }
        memcpy(f, tmp, sizeof(double) * nn);
    }
    free(tmp);
    return 0;
}

/* Eq. (2): k = nu <u> / g, <u> the superficial mean of the fluid velocity
 * over all N_grid nodes.  With Guo forcing the fluid momentum is the
 * pre-collision j plus F/2; the stored post-collision state carries j + F,
 * so rho u_x = j*_x - F_x/2 of the stored populations (over rho_0). */
double oc_permeability_forced(int q, int nx, int ny, int nz, const uint8_t* solid, const double* f, double tau,
                              double g, double rho0) {
    lattice L;
    if (get_lattice(q, &L)) return NAN;
    long nn = (long)nx * ny * nz;
    double sum = 0.0;
    for (long n = 0; n < nn; ++n) {
        if (solid[n]) continue;
        double rho, j[3];
        moments(&L, f + n * q, &rho, j);
        sum += j[0] - 0.5 * g * rho0;
    }
    const double nu = (tau - 0.5) / 3.0;
    return nu * (sum / (rho0 * (double)nn)) / g;
}

/* Run nsteps steps in place on f (uses a scratch buffer); tau_minus <= 0
 * means BGK. */
int oc_run_trt(int q, int nx, int ny, int nz, const uint8_t* solid, double tau, double tau_minus,
               double rho_in, double rho_out, int eq, double* f, long nsteps) {
    long nn = (long)nx * ny * nz * q;
    double* tmp = (double*)malloc(sizeof(double) * nn);
    if (!tmp) return -2;
    const int trt = tau_minus > 0.0;
    for (long t = 0; t < nsteps; ++t) {
        int rc = step_impl(q, nx, ny, nz, solid, tau, trt ? tau_minus : tau, trt, rho_in, rho_out, eq, f,
                           tmp);
        if (rc) {
            free(tmp);
            return rc;
        }
        memcpy(f, tmp, sizeof(double) * nn);
    }
    free(tmp);
    return 0;
}

int oc_run(int q, int nx, int ny, int nz, const uint8_t* solid, double tau, double rho_in,
           double rho_out, int eq, double* f, long nsteps) {
    return oc_run_trt(q, nx, ny, nz, solid, tau, 0.0, rho_in, rho_out, eq, f, nsteps);
}

/* ------------------------------------------------------------------------- */
/* Initial state, fields, observables                                         */
/* ------------------------------------------------------------------------- */

/* Equilibrium at rest with rho falling linearly from rho_in at x = 0 to rho_out
 * at x = N_x - 1 on fluid nodes. */
int oc_init(int q, int nx, int ny, int nz, const uint8_t* solid, double rho_in,
            double rho_out, double* f) {
    lattice L;
    if (get_lattice(q, &L) || check_dims(q, nx, ny, nz)) return -1;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long n = ((long)z * ny + y) * nx + x;
                double rho = rho_in + (rho_out - rho_in) * (double)x / (double)(nx - 1);
                for (int i = 0; i < q; ++i) f[n * q + i] = solid[n] ? 0.0 : L.w[i] * rho;
            }
    return 0;
}

/* f = f_eq(rho, u) on fluid nodes (the warm-start initialisation). */
int oc_equilibrium(int q, int nx, int ny, int nz, const uint8_t* solid, int eq,
                   const double* rho, const double* ux, const double* uy,
                   const double* uz, double* f) {
    lattice L;
    if (get_lattice(q, &L) || check_dims(q, nx, ny, nz)) return -1;
    long nn = (long)nx * ny * nz;
    for (long n = 0; n < nn; ++n) {
        if (solid[n]) {
            for (int i = 0; i < q; ++i) f[n * q + i] = 0.0;
            continue;
        }
        double j[3] = {rho[n] * ux[n], rho[n] * uy[n], uz ? rho[n] * uz[n] : 0.0};
        for (int i = 0; i < q; ++i) f[n * q + i] = feq(&L, i, rho[n], j, eq);
    }
    return 0;
}

/* Density and velocity on every node (zero on solids). */
int oc_fields(int q, int nx, int ny, int nz, const uint8_t* solid, const double* f,
              double* rho, double* ux, double* uy, double* uz) {
    lattice L;
    if (get_lattice(q, &L)) return -1;
    long nn = (long)nx * ny * nz;
    for (long n = 0; n < nn; ++n) {
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        if (!solid[n]) moments(&L, f + n * q, &r, j);
        rho[n] = r;
        ux[n] = solid[n] ? 0.0 : j[0] / r;
        uy[n] = solid[n] ? 0.0 : j[1] / r;
        if (uz) uz[n] = solid[n] ? 0.0 : j[2] / r;
    }
    return 0;
}

/* Superficial mean of the x mass flux over all N_grid nodes (Eq. 2's average). */
double oc_mean_jx(int q, int nx, int ny, int nz, const uint8_t* solid, const double* f) {
    lattice L;
    if (get_lattice(q, &L)) return NAN;
    long nn = (long)nx * ny * nz;
    double sum = 0.0;
    for (long n = 0; n < nn; ++n) {
        if (solid[n]) continue;
        double r, j[3];
        moments(&L, f + n * q, &r, j);
        sum += j[0];
    }
    return sum / (double)nn;
}

int oc_link_flux(int q, int nx, int ny, int nz, const uint8_t* solid, const double* f, double* jplane);

/* Sec. 2: the permeability follows from Darcy's law with the simulated mass
 * flow rate.  The mass flow rate is the mass crossing a cross-section per step:
 * the link flux J_{x+1/2} through the plane between columns x and x+1, averaged
 * over the N_x - 1 interior planes (at steady state it is the same on every
 * plane).  With the superficial velocity U = J / (rho A), A = N_y N_z, the
 * dynamic viscosity mu = rho nu (Eq. 1, nu = (tau - 1/2)/3), the pressure drop
 * c_s^2 (rho_in - rho_out) over the length L = N_x - 1 between the imposed
 * pressures, Darcy's U = (k / mu) dP / L gives
 *   k = nu <J> (N_x - 1) / (A c_s^2 (rho_in - rho_out)).
 * Fluid that is not on a through-path (closed pockets, boundary nodes boxed
 * in by solid) carries no link flux across the planes, so it cannot bias k. */
double oc_permeability(int q, int nx, int ny, int nz, const uint8_t* solid, const double* f,
                       double tau, double rho_in, double rho_out) {
    double nu = (tau - 0.5) / 3.0;
    double* J = (double*)malloc(sizeof(double) * (size_t)(nx - 1));
    if (!J || oc_link_flux(q, nx, ny, nz, solid, f, J)) {
        free(J);
        return NAN;
    }
    double sum = 0.0;
    for (int x = 0; x + 1 < nx; ++x) sum += J[x];
    free(J);
    double jmean = sum / (double)(nx - 1);
    return nu * jmean * (double)(nx - 1) / ((double)ny * (double)nz * (1.0 / 3.0) * (rho_in - rho_out));
}

/* Sec. 2: Kn = sqrt(pi/6) (tau - 1/2) / N_x. */
double oc_knudsen(double tau, int nx) { return sqrt(M_PI / 6.0) * (tau - 0.5) / (double)nx; }

/* Link flux through the plane x + 1/2, for x = 0 .. N_x - 2: the post-collision
 * populations that cross the plane in the next streaming, counted + for c_x = +1
 * and - for c_x = -1.  A population whose destination is solid bounces back and
 * does not cross; one whose destination row lies outside [0, N_y) is mirrored
 * back onto its own row (the specular rule of oc_step). */
int oc_link_flux(int q, int nx, int ny, int nz, const uint8_t* solid, const double* f,
                 double* jplane /* nx-1 */) {
    lattice L;
    if (get_lattice(q, &L)) return -1;
    for (int x = 0; x + 1 < nx; ++x) {
        double J = 0.0;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int i = 0; i < q; ++i) {
                    int cx = L.c[i][0];
                    if (cx == 0) continue;
                    int from_x = (cx == 1) ? x : x + 1; /* where the population sits */
                    int to_x = from_x + cx;
                    long n = ((long)z * ny + y) * nx + from_x;
                    if (solid[n]) continue;
                    int ty = y + L.c[i][1], tz = z + L.c[i][2];
                    if (ty < 0 || ty >= ny) ty = y;
                    if (tz < 0 || tz >= nz) tz = z;
                    long t = ((long)tz * ny + ty) * nx + to_x;
                    if (solid[t]) continue;
                    J += cx * f[n * q + i];
                }
        jplane[x] = J;
    }
    return 0;
}

/* Relative velocity change over one check interval:
 * r = sqrt( sum |u^t - u^{t-N}|^2 / sum |u^t|^2 ) over fluid nodes. */
static double residual(const lattice* L, long nn, const uint8_t* solid, const double* f,
                       double* uprev /* 3*nn, updated */) {
    double num = 0.0, den = 0.0;
    for (long n = 0; n < nn; ++n) {
        if (solid[n]) continue;
        double r, j[3];
        moments(L, f + n * L->q, &r, j);
        for (int a = 0; a < 3; ++a) {
            double u = j[a] / r;
            double d = u - uprev[n * 3 + a];
            num += d * d;
            den += u * u;
            uprev[n * 3 + a] = u;
        }
    }
    if (den == 0.0) return num == 0.0 ? 0.0 : INFINITY;
    return sqrt(num / den);
}

/* Iterate until the residual over `interval` steps is below tol, or max_steps.
 * Returns 0 when converged, 1 when max_steps was reached, <0 on error. */
int oc_run_to_steady_trt(int q, int nx, int ny, int nz, const uint8_t* solid, double tau, double tau_minus,
                         double rho_in, double rho_out, int eq, double* f, double tol,
                         long max_steps, int interval, long* steps_out, double* res_out) {
    lattice L;
    if (get_lattice(q, &L) || interval < 1) return -1;
    long nn = (long)nx * ny * nz;
    double* uprev = (double*)calloc((size_t)nn * 3, sizeof(double));
    if (!uprev) return -2;
    double r0 = residual(&L, nn, solid, f, uprev); /* seeds uprev with the start */
    (void)r0;
    long t = 0;
    double r = INFINITY;
    int rc = 1;
    while (t < max_steps) {
        long n = interval;
        if (t + n > max_steps) n = max_steps - t;
        int e = oc_run_trt(q, nx, ny, nz, solid, tau, tau_minus, rho_in, rho_out, eq, f, n);
        if (e) {
            rc = e;
            break;
        }
        t += n;
        r = residual(&L, nn, solid, f, uprev);
        if (!(r == r)) {
            rc = -4;
            break;
        }
        if (r < tol) {
            rc = 0;
            break;
        }
    }
    free(uprev);
    if (steps_out) *steps_out = t;
    if (res_out) *res_out = r;
    return rc;
}

int oc_run_to_steady(int q, int nx, int ny, int nz, const uint8_t* solid, double tau,
                     double rho_in, double rho_out, int eq, double* f, double tol,
                     long max_steps, int interval, long* steps_out, double* res_out) {
    return oc_run_to_steady_trt(q, nx, ny, nz, solid, tau, 0.0, rho_in, rho_out, eq, f, tol, max_steps,
                                interval, steps_out, res_out);
}

/* ------------------------------------------------------------------------- */
/* Local pore size and local Knudsen number                                   */
/* ------------------------------------------------------------------------- */

/*
 * Sec. 2 notes that the local Knudsen number in narrow pores can be much
 * larger than the domain's Kn = sqrt(pi/6)(tau - 1/2)/N_x.  With no pore-size
 * definition in the paper, the local pore size of a fluid node is
 * h = 2 D - 1, D the Euclidean distance (in nodes) to the nearest solid node
 * of the domain: the centre node of a channel of h fluid rows between solid
 * rows gets exactly h.  Faces are not walls (the y/z faces are symmetry
 * planes, the x faces open), so a node that sees no solid node has D = inf.
 * d2_out: squared distance D^2 per node (0 on solids, UINT32_MAX when no
 * solid exists); brute force over all solid nodes, as the definition reads.
 */
int oc_pore_d2(int nx, int ny, int nz, const uint8_t* solid, uint32_t* d2_out) {
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    long nn = (long)nx * ny * nz;
    long ns = 0;
    for (long n = 0; n < nn; ++n) ns += solid[n] ? 1 : 0;
    long* sidx = (long*)malloc(sizeof(long) * (size_t)(ns > 0 ? ns : 1));
    if (!sidx) return -2;
    long k = 0;
    for (long n = 0; n < nn; ++n)
        if (solid[n]) sidx[k++] = n;
    for (long n = 0; n < nn; ++n) {
        if (solid[n]) {
            d2_out[n] = 0;
            continue;
        }
        const long x = n % nx, y = (n / nx) % ny, z = n / ((long)nx * ny);
        uint64_t best = UINT64_MAX;
        for (long m = 0; m < ns; ++m) {
            const long s = sidx[m];
            const long dx = s % nx - x, dy = (s / nx) % ny - y, dz = s / ((long)nx * ny) - z;
            const uint64_t d2 = (uint64_t)(dx * dx + dy * dy + dz * dz);
            if (d2 < best) best = d2;
        }
        d2_out[n] = best == UINT64_MAX ? UINT32_MAX : (uint32_t)best;
    }
    free(sidx);
    return 0;
}

/* Local pore size h = 2 sqrt(D^2) - 1 and local Kn = sqrt(pi/6)(tau - 1/2)/h
 * on fluid nodes (0 on solids; h = inf and Kn = 0 where no solid exists). */
int oc_local_knudsen(int nx, int ny, int nz, const uint8_t* solid, double tau, double* h_out,
                     double* kn_out) {
    long nn = (long)nx * ny * nz;
    uint32_t* d2 = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nn > 0 ? nn : 1));
    if (!d2) return -2;
    int rc = oc_pore_d2(nx, ny, nz, solid, d2);
    if (rc) {
        free(d2);
        return rc;
    }
    for (long n = 0; n < nn; ++n) {
        double h = 0.0, kn = 0.0;
        if (!solid[n]) {
            if (d2[n] == UINT32_MAX) {
                h = INFINITY;
            } else {
                h = 2.0 * sqrt((double)d2[n]) - 1.0;
                kn = sqrt(M_PI / 6.0) * (tau - 0.5) / h;
            }
        }
        if (h_out) h_out[n] = h;
        if (kn_out) kn_out[n] = kn;
    }
    free(d2);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* splitmix64 and the QSGS generator                                          */
/* ------------------------------------------------------------------------- */

/* splitmix64 (Steele, Lea & Flood 2014): state advances by the golden gamma,
 * output is the state passed through the variant-13 finaliser. */
static const uint64_t SM_GAMMA = 0x9e3779b97f4a7c15ULL;

static uint64_t sm_finalise(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* The n-th output (n >= 1) of splitmix64 started from `seed`. */
uint64_t oc_splitmix64(uint64_t seed, uint64_t n) { return sm_finalise(seed + SM_GAMMA * n); }

/* Counter-based draw for growth iteration t, cell `cell`, neighbour slot `dir`:
 * the stream key is output t+1 of splitmix64(seed); the draw is the top 32 bits
 * of output (cell*32 + dir + 1) of splitmix64(key). */
uint32_t oc_qsgs_hash(uint64_t seed, uint32_t t, uint64_t cell, uint32_t dir) {
    uint64_t key = oc_splitmix64(seed, (uint64_t)t + 1);
    return (uint32_t)(oc_splitmix64(key, cell * 32u + dir + 1u) >> 32);
}

typedef struct {
    uint32_t h;
    uint64_t cell;
} cand;

static int cand_cmp(const void* a, const void* b) {
    const cand* x = (const cand*)a;
    const cand* y = (const cand*)b;
    if (x->h != y->h) return x->h < y->h ? -1 : 1;
    if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
    return 0;
}

/* Make candidates solid: all of them if they fit under the target count S,
 * otherwise the S - count smallest by (draw, cell index). */
static long accept(cand* cs, long nc, uint8_t* solid, long count, long S) {
    if (count + nc > S) {
        qsort(cs, (size_t)nc, sizeof(cand), cand_cmp);
        nc = S - count;
    }
    for (long k = 0; k < nc; ++k) solid[cs[k].cell] = 1;
    return count + nc;
}

/* floor(p * 2^32), clamped, as the integer threshold for a probability p. */
static uint32_t prob_threshold(double p) {
    if (p <= 0.0) return 0u;
    double t = floor(p * 4294967296.0);
    if (t >= 4294967295.0) return 4294967295u;
    return (uint32_t)t;
}

/* Neighbour slots in (dz, dy, dx) lexicographic order over {-1,0,1}^3 (only
 * dz = 0 in 2D), skipping the centre, with the growth threshold of each:
 * floor(D 2^32) with D = d_face for axis neighbours, d_face/2 for 3D edge
 * neighbours and d_face/4 for 2D diagonal and 3D corner neighbours. */
static int qsgs_slots(int nz, double d_face, int off[26][3], uint32_t thr[26]) {
    int dz0 = nz > 1 ? -1 : 0, dz1 = nz > 1 ? 1 : 0, nd = 0;
    uint32_t thr_face = prob_threshold(d_face), thr_edge = prob_threshold(d_face / 2.0),
             thr_corner = prob_threshold(d_face / 4.0);
    for (int dz = dz0; dz <= dz1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy && !dz) continue;
                int k = (dx != 0) + (dy != 0) + (dz != 0);
                off[nd][0] = dx;
                off[nd][1] = dy;
                off[nd][2] = dz;
                if (k == 1) thr[nd] = thr_face;
                else if (k == 2) thr[nd] = (nz > 1) ? thr_edge : thr_corner;
                else thr[nd] = thr_corner;
                ++nd;
            }
    return nd;
}

/* Growth iteration t >= 1 on the start-of-iteration mask `start`: a fluid cell
 * is a candidate iff some neighbour that is solid in `start` grows into it,
 * i.e. the draw for that (cell, slot) is below the slot's threshold.  The
 * cell's key is its smallest successful draw.  Writes the candidates to cs and
 * returns their number (ascending cell order). */
static long qsgs_candidates(int nx, int ny, int nz, uint64_t seed, uint32_t t, double d_face,
                            const uint8_t* start, cand* cs) {
    int off[26][3];
    uint32_t thr[26];
    int nd = qsgs_slots(nz, d_face, off, thr);
    long nc = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long c = ((long)z * ny + y) * nx + x;
                if (start[c]) continue;
                uint32_t best = 0xffffffffu;
                int hit = 0;
                for (int d = 0; d < nd; ++d) {
                    int X = x + off[d][0], Y = y + off[d][1], Z = z + off[d][2];
                    if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) continue;
                    if (!start[((long)Z * ny + Y) * nx + X]) continue;
                    uint32_t h = oc_qsgs_hash(seed, t, (uint64_t)c, (uint32_t)d);
                    if (h < thr[d]) {
                        if (!hit || h < best) best = h;
                        hit = 1;
                    }
                }
                if (hit) {
                    cs[nc].h = best;
                    cs[nc].cell = (uint64_t)c;
                    ++nc;
                }
            }
    return nc;
}

/* One growth iteration exposed for tests: cand_out[c] = 1 for candidates. */
int oc_qsgs_grow_once(int nx, int ny, int nz, uint64_t seed, uint32_t t, double d_face,
                      const uint8_t* start, uint8_t* cand_out) {
    long N = (long)nx * ny * nz;
    cand* cs = (cand*)malloc(sizeof(cand) * (size_t)(N > 0 ? N : 1));
    if (!cs) return -2;
    long nc = qsgs_candidates(nx, ny, nz, seed, t, d_face, start, cs);
    memset(cand_out, 0, (size_t)N);
    for (long k = 0; k < nc; ++k) cand_out[cs[k].cell] = 1;
    free(cs);
    return (int)nc;
}

/*
 * Quartet structure generation set (QSGS) growing the solid phase.
 *   t = 0: a cell is a solid core iff its draw is below floor(core_p 2^32).
 *   t >= 1 (synchronous): candidates as in qsgs_candidates.
 *   Growth stops at the target solid count S = round((1 - porosity) N); in the
 *   iteration that would overshoot, candidates are taken in ascending
 *   (key, cell index) order until exactly S.
 * The neighbourhood is clipped at the domain edges.
 * Returns the number of growth iterations, or <0 on error.
 */
int oc_qsgs(int nx, int ny, int nz, uint64_t seed, double core_p, double porosity,
            double d_face, uint8_t* solid) {
    if (nx < 1 || ny < 1 || nz < 1 || porosity < 0.0 || porosity > 1.0) return -1;
    long N = (long)nx * ny * nz;
    long S = (long)floor((1.0 - porosity) * (double)N + 0.5);
    memset(solid, 0, (size_t)N);
    cand* cs = (cand*)malloc(sizeof(cand) * (size_t)(N > 0 ? N : 1));
    uint8_t* start = (uint8_t*)malloc((size_t)(N > 0 ? N : 1));
    if (!cs || !start) {
        free(cs);
        free(start);
        return -2;
    }
    /* t = 0: cores */
    uint32_t thr_core = prob_threshold(core_p);
    long nc = 0;
    for (long c = 0; c < N; ++c) {
        uint32_t h = oc_qsgs_hash(seed, 0u, (uint64_t)c, 0u);
        if (h < thr_core) {
            cs[nc].h = h;
            cs[nc].cell = (uint64_t)c;
            ++nc;
        }
    }
    long count = accept(cs, nc, solid, 0, S);
    int t = 0;
    while (count < S) {
        if (count == 0) {
            t = -3; /* no core: nothing can grow */
            break;
        }
        ++t;
        if (t > 1000000) {
            t = -5;
            break;
        }
        memcpy(start, solid, (size_t)N);
        nc = qsgs_candidates(nx, ny, nz, seed, (uint32_t)t, d_face, start, cs);
        count = accept(cs, nc, solid, count, S);
    }
    free(cs);
    free(start);
    return t;
}

/* Does fluid connect the inlet column to the outlet column?  Connectivity
 * follows the lattice links: 8 neighbours in 2D, the 18 face and edge
 * neighbours in 3D. */
int oc_percolates(int nx, int ny, int nz, const uint8_t* solid) {
    long N = (long)nx * ny * nz;
    uint8_t* seen = (uint8_t*)calloc((size_t)N, 1);
    long* stack = (long*)malloc(sizeof(long) * (size_t)N);
    if (!seen || !stack) {
        free(seen);
        free(stack);
        return -2;
    }
    long top = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y) {
            long n = ((long)z * ny + y) * nx;
            if (!solid[n]) {
                seen[n] = 1;
                stack[top++] = n;
            }
        }
    int found = 0;
    while (top > 0 && !found) {
        long n = stack[--top];
        int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long)nx * ny));
        if (x == nx - 1) {
            found = 1;
            break;
        }
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int k = (dx != 0) + (dy != 0) + (dz != 0);
                    if (k == 0 || k == 3) continue;
                    if (nz == 1 && dz != 0) continue;
                    int X = x + dx, Y = y + dy, Z = z + dz;
                    if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) continue;
                    long m = ((long)Z * ny + Y) * nx + X;
                    if (solid[m] || seen[m]) continue;
                    seen[m] = 1;
                    stack[top++] = m;
                }
    }
    free(seen);
    free(stack);
    return found;
}
