/*
 * FP64 CPU oracle of the per-node apparent permeability of the paper's
 * DGM + GMS model (Wang, Chen, Kang & Rahman, arXiv:1601.00704, Sec. 2.1),
 * single species (methane):
 *
 *   Eq. 3   D_K = (4/3) K_c sqrt(8 R T / (pi M))          Knudsen diffusivity
 *   Eq. 4   K_c = (8/d_p) K0 = (eps/tau)(d_p/4)            -> K0 = eps d_p^2 / (32 tau)
 *   Eq. 18  K_app = (eta M / rho_g) (1/(R T)) (D_K + K0 P / eta)        (IOM)
 *   Eq. 19  K_app = (eta M / rho_g) [(1/(R T))(D_K + K0 P / eta)
 *                                    + (1 - eps) q_sat b D_s / (1 + b P)]   (OM)
 *   Eq. 38  q_sat,k = q_sat,b rho_b / ((1 - eps) TOC) * rho_CH4 / M_CH4
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE (see glbm_oracle.c).  The formulas
 * are evaluated as printed, in the paper's order; readings:
 *  - d_p = 2 r (pore diameter from the pore radius r);
 *  - rho_g is the ideal-gas density P M / (R T) (the paper names no
 *    equation of state);
 *  - eta is a constant (Table "Input parameters of IOM": 18.231e-6 Pa s);
 *  - tau here is the tortuosity (2 in the paper's tables), not the BGK
 *    relaxation time.
 *
 * Pins (tests/test_oracle_dgm.py): Eq. 19 with D_s = 0 equals Eq. 18;
 * K_app is linear in q_sat; K_app -> K0 as P -> infinity; the Knudsen part
 * scales as 1/P and as d_p, K0 as d_p^2, the surface part not with d_p.
 */
#include <math.h>

static const double R_GAS = 8.314462618; /* J / (mol K) */
static const double PI = 3.14159265358979323846;

/* Eq. 4 */
void orc_dgm_kc_k0(double r, double eps, double tort, double *Kc, double *K0) {
    const double dp = 2.0 * r;
    *Kc = eps / tort * dp / 4.0;
    *K0 = *Kc * dp / 8.0;
}

/* Eq. 3 */
double orc_knudsen_diffusivity(double Kc, double T, double M) {
    return 4.0 / 3.0 * Kc * sqrt(8.0 * R_GAS * T / (PI * M));
}

/* Eq. 18 (organic = 0) or Eq. 19 (organic = 1); SI units, result in m^2. */
double orc_kapp(double r, double P, double T, double M, double eta, double eps,
                double tort, int organic, double qsat, double b, double Ds) {
    double Kc, K0;
    orc_dgm_kc_k0(r, eps, tort, &Kc, &K0);
    const double DK = orc_knudsen_diffusivity(Kc, T, M);
    const double rho_g = P * M / (R_GAS * T);
    double bracket = 1.0 / (R_GAS * T) * (DK + K0 / eta * P);
    if (organic) bracket += (1.0 - eps) * qsat * b * Ds / (1.0 + b * P);
    return eta * M / rho_g * bracket;
}

/* Eq. 38 */
double orc_qsat_from_langmuir_volume(double qsat_b, double rho_b, double eps,
                                     double toc, double rho_ch4,
                                     double M_ch4) {
    return qsat_b * rho_b / ((1.0 - eps) * toc) * rho_ch4 / M_ch4;
}

/* Per-node field in lattice units K_app / dx^2 (n nodes). */
void orc_kapp_field(const double *r, const unsigned char *organic,
                    const double *eps, long n, double P, double T, double M,
                    double eta, double tort, double qsat, double b, double Ds,
                    double dx, double *K) {
    for (long i = 0; i < n; ++i)
        K[i] = orc_kapp(r[i], P, T, M, eta, eps[i], tort, organic[i], qsat, b,
                        Ds) /
               (dx * dx);
}
