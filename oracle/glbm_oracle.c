/*
 * Plain FP64 CPU oracle of the generalized lattice Boltzmann model (GLBM)
 * used by Wang, Chen, Kang & Rahman, "Permeability prediction of organic
 * shale with generalized lattice Boltzmann model considering surface
 * diffusion effect" (arXiv:1601.00704), Sec. 2.3, Eqs. 27-37.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg load this file.  It shares no
 * source, header, table or helper with the CUDA library: the lattice
 * constants below are typed out here from the D2Q9 definition.
 *
 * Deliberately slow and literal: absolute distributions f_i (not deviations),
 * FP64 throughout, one node at a time in a fixed order (y outer, x inner,
 * i = 0..8), no blocking, fusion or vectorisation.  Each step is the paper's
 * sequence:
 *
 *   stream (left side of Eq. 29)  ->  rho (Eq. 32)  ->  v (Eq. 35)
 *   -> c0, c1 (Eqs. 36, 37)  ->  u (Eq. 34)  ->  F (Eq. 27)
 *   -> f_eq (Eq. 30), F_i (Eq. 31)  ->  BGK collision (right side of Eq. 29).
 *
 * Readings where the paper is silent, garbled or inconsistent:
 *  - Lattice: D2Q9, c = dx/dt = 1, c_s^2 = 1/3 (the paper only says "w_i is
 *    the weighting factor").
 *  - nu = nu_e = (tau - 1/2)/3 (viscosity ratio 1).
 *  - Eq. 28 is typeset as -eps*nu/(K u); read as -(eps*nu/K)*u, consistent
 *    with Eq. 27 and with c0 in Eq. 36.
 *  - Eq. 31's last term lacks the 1/eps that the cited Guo-Zhao forcing
 *    carries.  Default reading: -(3/eps)(u.F), which makes sum_i F_i = 0
 *    (exact mass conservation).  literal_forcing=1 uses the printed -3(u.F).
 *  - F_eps (the Forchheimer geometric function) is never given a value:
 *    0 = the paper's Forchheimer-free model (Eq. 28); >0 = that constant;
 *    <0 = Ergun's form 1.75/sqrt(150 eps^3) evaluated per node.
 *  - Boundaries are not stated: x is periodic; y is periodic or bounded by
 *    halfway bounce-back walls at y = -1/2 and y = ny - 1/2.
 *  - The same u from Eq. 34 enters f_eq, F and F_i; rho0 = 1, u = 0 start.
 *  - Convergence (not in the paper): after every chunk of check_every steps
 *    and at the end of every call, U = mean of u over all nodes is formed;
 *    with tol > 0 the run stops once |Ux - Ux_prev| <= tol*|Ux|, where
 *    Ux_prev is the previous such value (carried between calls).
 *
 * D2Q9 directions: e0=(0,0); e1..e4=(1,0),(0,1),(-1,0),(0,-1);
 * e5..e8=(1,1),(-1,1),(-1,-1),(1,-1).  Weights 4/9, 1/9 (x4), 1/36 (x4).
 * Storage: f[i*ny*nx + y*nx + x] (row-major, x fastest), the post-collision
 * state after the last completed step.
 *
 * Pins (tests/test_oracle_*.py): equilibrium and forcing moments, the
 * Eq. 33 root, Darcy and Forchheimer fixed points, exact Poiseuille at
 * tau = 1/2 + sqrt(3)/4, Brinkman channel convergence, series-layer momentum
 * balance, Taylor-Green viscosity, mass conservation, and the reduction to
 * textbook D2Q9 BGK with Guo forcing.  On two-phase random media the fields
 * have no closed form; there the steady state is pinned by the exact domain
 * momentum balance (sum of rho F = 0, F from Eq. 27).
 *
 * Build: gcc -O2 -shared -fPIC (single thread, parity) or with -fopenmp
 * (rows in parallel, timing only); results are bitwise identical because
 * every node's arithmetic is independent and the velocity sums are formed
 * per row and then added in row order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                            1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

int orc_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Forchheimer geometric function per node (reading above). */
double orc_feps(double feps_mode, double eps) {
    if (feps_mode > 0) return feps_mode;
    if (feps_mode < 0) return 1.75 / sqrt(150.0 * eps * eps * eps);
    return 0.0;
}

/* Eq. 36 and Eq. 37 with dt = 1.  K = +inf gives c0 = 1/2, c1 = 0. */
void orc_c0_c1(double eps, double K, double feps, double nu, double *c0,
               double *c1) {
    *c0 = 0.5 * (1.0 + eps * 0.5 * nu / K);
    *c1 = eps * 0.5 * feps / sqrt(K);
}

/* Eq. 35 then Eq. 34: velocity from the pre-collision moments. */
void orc_velocity(double rho, double mx, double my, double eps, double K,
                  double feps, double nu, double gx, double gy, double *ux,
                  double *uy) {
    double vx = mx / rho + 0.5 * eps * gx;
    double vy = my / rho + 0.5 * eps * gy;
    double c0, c1;
    orc_c0_c1(eps, K, feps, nu, &c0, &c1);
    double vmag = sqrt(vx * vx + vy * vy);
    double den = c0 + sqrt(c0 * c0 + c1 * vmag);
    *ux = vx / den;
    *uy = vy / den;
}

/* Eq. 27: total body force (Darcy drag, Forchheimer drag, external force). */
void orc_body_force(double ux, double uy, double eps, double K, double feps,
                    double nu, double gx, double gy, double *Fx, double *Fy) {
    double umag = sqrt(ux * ux + uy * uy);
    double lin = eps * nu / K;
    double quad = eps * feps / sqrt(K) * umag;
    *Fx = -lin * ux - quad * ux + eps * gx;
    *Fy = -lin * uy - quad * uy + eps * gy;
}

/* Eq. 30 with c = 1. */
void orc_equilibrium(double rho, double ux, double uy, double eps,
                     double feq[9]) {
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        feq[i] = W[i] * rho *
                 (1.0 + 3.0 * eu + 9.0 / (2.0 * eps) * eu * eu -
                  3.0 / (2.0 * eps) * uu);
    }
}

/* Eq. 31 with c = dt = 1; the last term carries 1/eps unless literal. */
void orc_forcing(double rho, double ux, double uy, double Fx, double Fy,
                 double eps, double tau, int literal, double Fi[9]) {
    double uF = ux * Fx + uy * Fy;
    double last = literal ? 3.0 * uF : 3.0 / eps * uF;
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        double eF = EX[i] * Fx + EY[i] * Fy;
        Fi[i] = W[i] * rho * (1.0 - 1.0 / (2.0 * tau)) *
                (3.0 * eF + 9.0 / eps * eu * eF - last);
    }
}

/* Fill f with f_eq(rho, u; eps) node by node (rho/ux/uy NULL -> 1, 0, 0). */
void orc_init_equilibrium(int nx, int ny, const double *eps, const double *rho,
                          const double *ux, const double *uy, double *f) {
    long N = (long)nx * ny;
    for (long n = 0; n < N; ++n) {
        double feq[9];
        orc_equilibrium(rho ? rho[n] : 1.0, ux ? ux[n] : 0.0,
                        uy ? uy[n] : 0.0, eps[n], feq);
        for (int i = 0; i < 9; ++i) f[i * N + n] = feq[i];
    }
}

/* One full step: pull from fsrc (post-collision state at t), write the
 * post-collision state at t+1 into fdst.  Per-row sums of u go to rowsum. */
static void orc_one_step(int nx, int ny, double tau, int periodic_y,
                         int literal, const double *eps, const double *K,
                         double feps_mode, double gx, double gy,
                         const double *fsrc, double *fdst, double *ux_out,
                         double *uy_out, double *rho_out, double *rowsum) {
    const long N = (long)nx * ny;
    const double nu = (tau - 0.5) / 3.0;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        double sx = 0.0, sy = 0.0;
        for (int x = 0; x < nx; ++x) {
            const long n = (long)y * nx + x;
            double f[9];
            /* streaming: f_i(x, t+1) = f*_i(x - e_i, t) */
            for (int i = 0; i < 9; ++i) {
                int xs = ((x - EX[i]) % nx + nx) % nx;
                int ys = y - EY[i];
                if (ys < 0 || ys >= ny) {
                    if (periodic_y) {
                        ys = (ys % ny + ny) % ny;
                    } else {
                        /* halfway bounce-back: the population that left
                         * this node towards the wall comes back reversed */
                        f[i] = fsrc[OPP[i] * N + n];
                        continue;
                    }
                }
                f[i] = fsrc[i * N + (long)ys * nx + xs];
            }
            /* Eq. 32 and the first-moment sum of Eq. 33 / Eq. 35 */
            double rho = 0.0, mx = 0.0, my = 0.0;
            for (int i = 0; i < 9; ++i) {
                rho += f[i];
                mx += f[i] * EX[i];
                my += f[i] * EY[i];
            }
            const double e = eps[n], k = K[n];
            const double fe = orc_feps(feps_mode, e);
            double ux, uy, Fx, Fy;
            orc_velocity(rho, mx, my, e, k, fe, nu, gx, gy, &ux, &uy);
            orc_body_force(ux, uy, e, k, fe, nu, gx, gy, &Fx, &Fy);
            double feq[9], Fi[9];
            orc_equilibrium(rho, ux, uy, e, feq);
            orc_forcing(rho, ux, uy, Fx, Fy, e, tau, literal, Fi);
            /* Eq. 29, right side, dt = 1 */
            for (int i = 0; i < 9; ++i)
                fdst[i * N + n] = f[i] - (f[i] - feq[i]) / tau + Fi[i];
            if (ux_out) ux_out[n] = ux;
            if (uy_out) uy_out[n] = uy;
            if (rho_out) rho_out[n] = rho;
            sx += ux;
            sy += uy;
        }
        rowsum[2 * y] = sx;
        rowsum[2 * y + 1] = sy;
    }
}

/*
 * Advance `nsteps` steps (fewer if converged), starting from the
 * post-collision state in f (in/out).
 *
 *  conv_state[0] (in/out): 1 if conv_state[1] holds a previous mean Ux.
 *  mean_u[2]   (out): mean (Ux, Uy) over all nodes at the last step.
 *  ux, uy, rho (out, may be NULL): the last step's Eq. 34 velocity and
 *              Eq. 32 density per node.
 *  Returns 0, or -1 on bad arguments, -2 on allocation failure,
 *  -4 if a non-finite mean velocity appeared (state kept).
 */
int orc_run(int nx, int ny, double tau, int periodic_y, int literal,
            const double *eps, const double *K, double feps_mode, double gx,
            double gy, double *f, long long nsteps, double tol,
            int check_every, double *ux, double *uy, double *rho,
            double *mean_u, double *conv_state, long long *steps_done,
            int *converged) {
    if (nx < 2 || ny < 2 || !(tau > 0.5) || nsteps < 0 || check_every < 1)
        return -1;
    const long N = (long)nx * ny;
    double *g = (double *)malloc(sizeof(double) * 9 * N);
    double *rows = (double *)malloc(sizeof(double) * 2 * ny);
    if (!g || !rows) {
        free(g);
        free(rows);
        return -2;
    }
    double *cur = f, *nxt = g;
    long long done = 0;
    int conv = 0, status = 0;
    while (done < nsteps && !conv) {
        long long chunk = nsteps - done;
        if (chunk > check_every) chunk = check_every;
        for (long long s = 0; s < chunk; ++s) {
            int last = (s == chunk - 1);
            orc_one_step(nx, ny, tau, periodic_y, literal, eps, K, feps_mode,
                         gx, gy, cur, nxt, last ? ux : NULL,
                         last ? uy : NULL, last ? rho : NULL, rows);
            double *t = cur;
            cur = nxt;
            nxt = t;
        }
        done += chunk;
        double sx = 0.0, sy = 0.0;
        for (int y = 0; y < ny; ++y) {
            sx += rows[2 * y];
            sy += rows[2 * y + 1];
        }
        double Ux = sx / (double)N, Uy = sy / (double)N;
        if (mean_u) {
            mean_u[0] = Ux;
            mean_u[1] = Uy;
        }
        if (!isfinite(Ux) || !isfinite(Uy)) {
            status = -4;
            break;
        }
        if (tol > 0 && conv_state && conv_state[0] != 0.0 &&
            fabs(Ux - conv_state[1]) <= tol * fabs(Ux))
            conv = 1;
        if (conv_state) {
            conv_state[0] = 1.0;
            conv_state[1] = Ux;
        }
    }
    if (cur != f) memcpy(f, cur, sizeof(double) * 9 * N);
    free(g);
    free(rows);
    if (steps_done) *steps_done = done;
    if (converged) *converged = conv;
    return status;
}

/* Darcy upscaling (reading: K_app = nu * <u_x> / G_x, lattice units). */
double orc_permeability(double tau, double mean_ux, double gx) {
    return (tau - 0.5) / 3.0 * mean_ux / gx;
}
