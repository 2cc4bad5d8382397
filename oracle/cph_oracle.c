/*
 * Plain FP64 CPU oracle for the GB-OBC / C(pH,E)MD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA engine.
 *
 * Every routine is the plain definition written out with double loops, no
 * blocking, no fusion and no reordering.  The paper (Implicit Solvent
 * Calculations section) names the GB model only as Onufriev-Bashford-Case
 * "igb=2"; the formulas below follow the published OBC model with
 * Hawkins-Cramer-Truhlar pairwise descreening:
 *
 *   H(r, rt_i, s_j)  HCT integral of sphere j (radius s_j at distance r)
 *                    outside the ball rt_i;
 *   psi_i = rt_i * 1/2 * sum_{j!=i} H(r_ij, rt_i, s_j);
 *   R_i   = 1 / (1/rt_i - tanh(a psi - b psi^2 + c psi^3) / rho_i);
 *   E_GB  = -1/2 k (1/eps_in - 1/eps_out) sum_i sum_j q_i q_j / f_ij,
 *           f_ij = sqrt(r^2 + R_i R_j exp(-r^2 / (4 R_i R_j))), f_ii = R_i;
 *   E_coul, E_LJ over non-excluded pairs (1-2 and 1-3 excluded),
 *   harmonic bonds and angles.
 *
 * Units: kcal/mol, Angstrom, e, amu, ps, K.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_KCOUL 332.0522173      /* kcal A / (mol e^2) */
#define O_KB 0.0019872041        /* kcal / (mol K) */
#define O_ACC 418.4              /* (kcal/mol/A)/amu -> A/ps^2 */

typedef struct {
    double eps_in, eps_out, offset, alpha, beta, gamma;
    double kappa; /* Debye-Hueckel screening length inverse, 1/A (0: no salt) */
    double sa_gamma, sa_probe; /* nonpolar surface term (ACE), kcal/mol/A^2 and A (0: off) */
    double rgbmax;             /* Born-radius cutoff, A (0: none) */
} ogb;

/* Nonpolar surface term in the ACE approximation (Schaefer & Karplus 1996):
 * E_SA,i = 4 pi gamma (rho_i + r_probe)^2 (rho_i / R_i)^6, which depends on the
 * Born radius R_i: dE_SA,i/dR_i = -6 E_SA,i / R_i. */
static double sa_energy(const ogb *g, double rho, double R) {
    if (g->sa_gamma == 0.0) return 0.0;
    const double a = rho + g->sa_probe, t = rho / R;
    return 4.0 * 3.14159265358979323846 * g->sa_gamma * a * a * t * t * t * t * t * t;
}

typedef struct {
    int n;
    const double *rho, *screen, *sigma, *eps;
    const unsigned char *excl; /* n*n, 1 where Coulomb/LJ is excluded (i != j) */
    int n_bonds;
    const int *bonds;          /* [2*n_bonds] */
    const double *bond_k, *bond_r0;
    int n_angles;
    const int *angles;         /* [3*n_angles] */
    const double *angle_k, *angle_t0;
} osys;

static double dist(const double *x, int i, int j, double d[3]) {
    d[0] = x[3 * i] - x[3 * j];
    d[1] = x[3 * i + 1] - x[3 * j + 1];
    d[2] = x[3 * i + 2] - x[3 * j + 2];
    return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

/* ------------------------------------------------------------------ HCT */

/* H(r, rt, s) is the descreening integral 2 int_L^U f(t) / t^2 dt over the
 * shells t around an atom of offset radius rt, f(t) the fraction of shell t
 * inside a sphere of radius s at distance r: L = max(rt, |r - s|), U = r + s,
 * closed form below, plus 2(1/rt - 1/L) when the ball rt lies wholly inside
 * sphere s (those shells are fully covered); zero when the ball swallows the
 * sphere.  With a Born-radius cutoff rc > 0 (AMBER's rgbmax) only shells
 * t <= rc count: U = min(r + s, rc) and the covered shells end at rc.  The
 * derivatives are total ones: L and U move with r and s (the integrand
 * vanishes on those moving boundaries, but not at a fixed U = rc). */
static double hct_closed(double r, double s, double L, double U) {
    return 1.0 / L - 1.0 / U
         + 0.25 * r * (1.0 / (U * U) - 1.0 / (L * L))
         + 0.5 / r * log(L / U)
         + 0.25 * s * s / r * (1.0 / (L * L) - 1.0 / (U * U));
}

/* Partial derivatives of the closed form with respect to its explicit r, s,
 * L and U arguments. */
static void hct_partials(double r, double s, double L, double U,
                         double *hr, double *hs, double *hL, double *hU) {
    double iL2 = 1.0 / (L * L), iU2 = 1.0 / (U * U);
    *hr = 0.25 * (iU2 - iL2) - 0.5 / (r * r) * log(L / U) - 0.25 * s * s / (r * r) * (iL2 - iU2);
    *hs = 0.5 * s / r * (iL2 - iU2);
    *hL = -iL2 + 0.5 * r / (L * L * L) + 0.5 / (r * L) - 0.5 * s * s / (r * L * L * L);
    *hU = iU2 - 0.5 * r / (U * U * U) - 0.5 / (r * U) + 0.5 * s * s / (r * U * U * U);
}

/* Which branch of L: 1 when L = rt, 0 when L = |r - s|. */
static int hct_L(double r, double rt, double s, double *L) {
    double a = fabs(r - s);
    if (rt > a) { *L = rt; return 1; }
    *L = a;
    return 0;
}

/* U and whether it moves with r and s (1) or sits at the cutoff (0). */
static double hct_U(double r, double s, double rc, int *moving) {
    double U = r + s;
    if (rc > 0.0 && U > rc) { *moving = 0; return rc; }
    *moving = 1;
    return U;
}

/* End of the fully covered shells (ball inside sphere s), capped at rc. */
static double hct_top(double r, double s, double rc, int *capped) {
    double top = s - r;
    *capped = 0;
    if (rc > 0.0 && rc < top) { top = rc; *capped = 1; }
    return top;
}

double o_hct_rc(double r, double rt, double s, double rc) {
    int mv, cap;
    double U = hct_U(r, s, rc, &mv), L;
    hct_L(r, rt, s, &L);
    double h = (L < U) ? hct_closed(r, s, L, U) : 0.0;
    if (rt < s - r) {
        double top = hct_top(r, s, rc, &cap);
        if (rt < top) h += 2.0 * (1.0 / rt - 1.0 / top);
    }
    return h;
}

/* dH/dr, total. */
double o_hct_dr_rc(double r, double rt, double s, double rc) {
    int mv, cap;
    double U = hct_U(r, s, rc, &mv), L;
    int Lrt = hct_L(r, rt, s, &L);
    double d = 0.0;
    if (L < U) {
        double dL = Lrt ? 0.0 : (r > s ? 1.0 : -1.0);
        double hr, hs, hL, hU;
        hct_partials(r, s, L, U, &hr, &hs, &hL, &hU);
        d = hr + hL * dL + hU * (mv ? 1.0 : 0.0);
    }
    if (rt < s - r) {
        double top = hct_top(r, s, rc, &cap);
        if (rt < top && !cap) d += -2.0 / (top * top); /* d(-2/top)/dr, top = s - r */
    }
    return d;
}

/* dH/d(rt), total. */
double o_hct_drt_rc(double r, double rt, double s, double rc) {
    int mv, cap;
    double U = hct_U(r, s, rc, &mv), L;
    int Lrt = hct_L(r, rt, s, &L);
    double d = 0.0;
    if (L < U && Lrt) {
        double hr, hs, hL, hU;
        hct_partials(r, s, L, U, &hr, &hs, &hL, &hU);
        d = hL;
    }
    if (rt < s - r) {
        double top = hct_top(r, s, rc, &cap);
        if (rt < top) d += -2.0 / (rt * rt);
    }
    return d;
}

/* dH/ds, total. */
double o_hct_ds_rc(double r, double rt, double s, double rc) {
    int mv, cap;
    double U = hct_U(r, s, rc, &mv), L;
    int Lrt = hct_L(r, rt, s, &L);
    double d = 0.0;
    if (L < U) {
        double dL = Lrt ? 0.0 : (s > r ? 1.0 : -1.0);
        double hr, hs, hL, hU;
        hct_partials(r, s, L, U, &hr, &hs, &hL, &hU);
        d = hs + hL * dL + hU * (mv ? 1.0 : 0.0);
    }
    if (rt < s - r) {
        double top = hct_top(r, s, rc, &cap);
        if (rt < top && !cap) d += 2.0 / (top * top); /* d(-2/top)/ds, top = s - r */
    }
    return d;
}

double o_hct(double r, double rt, double s) { return o_hct_rc(r, rt, s, 0.0); }
double o_hct_dr(double r, double rt, double s) { return o_hct_dr_rc(r, rt, s, 0.0); }
double o_hct_drt(double r, double rt, double s) { return o_hct_drt_rc(r, rt, s, 0.0); }
double o_hct_ds(double r, double rt, double s) { return o_hct_ds_rc(r, rt, s, 0.0); }

/* ----------------------------------------------------------- Born radii */

/* psi_i and R_i for every atom of one configuration. */
void o_born(int n, const double *x, const double *rho, const double *screen,
            const ogb *g, double *psi, double *R) {
    for (int i = 0; i < n; i++) {
        double rti = rho[i] - g->offset;
        double sum = 0.0;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3];
            double r = dist(x, i, j, d);
            double sj = screen[j] * (rho[j] - g->offset);
            sum += o_hct_rc(r, rti, sj, g->rgbmax);
        }
        double p = 0.5 * rti * sum;
        double th = tanh(g->alpha * p - g->beta * p * p + g->gamma * p * p * p);
        psi[i] = p;
        R[i] = 1.0 / (1.0 / rti - th / rho[i]);
    }
}

/* A GB pair at effective distance f (a self term: f = R) contributes
 * -k q_i q_j tau(f) / f, with tau(f) = 1/eps_in - exp(-kappa f)/eps_out: the
 * solvent's reaction field screened by salt in the Debye-Hueckel form
 * (kappa = 0: the salt-free constant 1/eps_in - 1/eps_out).  Its derivative is
 * d(tau(f)/f)/df = -taud(f)/f^2 with taud(f) = tau(f) - kappa f exp(-kappa f)/eps_out. */
static double gb_tauf(const ogb *g, double f) { return 1.0 / g->eps_in - exp(-g->kappa * f) / g->eps_out; }
static double gb_taud(const ogb *g, double f) {
    return gb_tauf(g, f) - g->kappa * f * exp(-g->kappa * f) / g->eps_out;
}

/* ------------------------------------------------- electrostatics only */

/* U_el = E_coul + E_GB for charges q at positions x with Born radii R. */
double o_uel(const osys *S, const ogb *g, const double *x, const double *q, const double *R) {
    int n = S->n;
    double e = 0.0;
    for (int i = 0; i < n; i++) e += -0.5 * O_KCOUL * gb_tauf(g, R[i]) * q[i] * q[i] / R[i];
    for (int i = 0; i < n; i++) {
        for (int j = i + 1; j < n; j++) {
            double d[3];
            double r = dist(x, i, j, d);
            double RR = R[i] * R[j];
            double f = sqrt(r * r + RR * exp(-r * r / (4.0 * RR)));
            e += -O_KCOUL * gb_tauf(g, f) * q[i] * q[j] / f;
            if (!S->excl[(size_t)i * n + j]) e += O_KCOUL * q[i] * q[j] / (g->eps_in * r);
        }
    }
    return e;
}

/* ------------------------------------------------ energies and forces */

/* terms[0..5] = E_GB, E_coul, E_LJ, E_bond, E_angle, total.  F (may be NULL)
 * receives -grad E including the Born-radius chain rule.  R and psi (may be
 * NULL) receive the Born radii and psi. */
void o_energy(const osys *S, const ogb *g, const double *x, const double *q,
              double *terms, double *F, double *Rout, double *psiout) {
    int n = S->n;
    double *psi = (double *)malloc(sizeof(double) * n);
    double *R = (double *)malloc(sizeof(double) * n);
    double *dEdR = (double *)calloc(n, sizeof(double));
    double *Fl = (double *)calloc(3 * (size_t)n, sizeof(double));
    o_born(n, x, S->rho, S->screen, g, psi, R);

    double egb = 0.0, ecoul = 0.0, elj = 0.0, ebond = 0.0, eang = 0.0;
    for (int i = 0; i < n; i++) {
        egb += -0.5 * O_KCOUL * gb_tauf(g, R[i]) * q[i] * q[i] / R[i];
        dEdR[i] += 0.5 * O_KCOUL * gb_taud(g, R[i]) * q[i] * q[i] / (R[i] * R[i]);
        const double esa = sa_energy(g, S->rho[i], R[i]); /* reported with E_GB */
        egb += esa;
        dEdR[i] += -6.0 * esa / R[i];
    }
    for (int i = 0; i < n; i++) {
        for (int j = i + 1; j < n; j++) {
            double d[3];
            double r = dist(x, i, j, d);
            double RR = R[i] * R[j];
            double D = r * r / (4.0 * RR);
            double ex = exp(-D);
            double f = sqrt(r * r + RR * ex);
            double qq = q[i] * q[j];
            egb += -O_KCOUL * gb_tauf(g, f) * qq / f;
            double dEdf = O_KCOUL * gb_taud(g, f) * qq / (f * f);
            double dfdr = r / f * (1.0 - 0.25 * ex);
            dEdR[i] += dEdf * R[j] * ex * (1.0 + D) / (2.0 * f);
            dEdR[j] += dEdf * R[i] * ex * (1.0 + D) / (2.0 * f);
            double dEdr = dEdf * dfdr;
            if (!S->excl[(size_t)i * n + j]) {
                ecoul += O_KCOUL * qq / (g->eps_in * r);
                dEdr += -O_KCOUL * qq / (g->eps_in * r * r);
                double sig = 0.5 * (S->sigma[i] + S->sigma[j]);
                double ep = sqrt(S->eps[i] * S->eps[j]);
                double sr6 = pow(sig / r, 6.0);
                elj += 4.0 * ep * (sr6 * sr6 - sr6);
                dEdr += 4.0 * ep * (-12.0 * sr6 * sr6 / r + 6.0 * sr6 / r);
            }
            for (int c = 0; c < 3; c++) {
                Fl[3 * i + c] -= dEdr * d[c] / r;
                Fl[3 * j + c] += dEdr * d[c] / r;
            }
        }
    }
    /* chain rule through the Born radii: dE/dR_k dR_k/dpsi_k dpsi_k/dr_kj */
    for (int k = 0; k < n; k++) {
        double p = psi[k];
        double rtk = S->rho[k] - g->offset;
        double th = tanh(g->alpha * p - g->beta * p * p + g->gamma * p * p * p);
        double dRdpsi = R[k] * R[k] * (1.0 - th * th)
                      * (g->alpha - 2.0 * g->beta * p + 3.0 * g->gamma * p * p) / S->rho[k];
        double ck = dEdR[k] * dRdpsi * 0.5 * rtk;
        for (int j = 0; j < n; j++) {
            if (j == k) continue;
            double d[3];
            double r = dist(x, k, j, d);
            double sj = S->screen[j] * (S->rho[j] - g->offset);
            double gr = ck * o_hct_dr_rc(r, rtk, sj, g->rgbmax);
            for (int c = 0; c < 3; c++) {
                Fl[3 * k + c] -= gr * d[c] / r;
                Fl[3 * j + c] += gr * d[c] / r;
            }
        }
    }
    for (int b = 0; b < S->n_bonds; b++) {
        int i = S->bonds[2 * b], j = S->bonds[2 * b + 1];
        double d[3];
        double r = dist(x, i, j, d);
        double dr = r - S->bond_r0[b];
        ebond += S->bond_k[b] * dr * dr;
        double dEdr = 2.0 * S->bond_k[b] * dr;
        for (int c = 0; c < 3; c++) {
            Fl[3 * i + c] -= dEdr * d[c] / r;
            Fl[3 * j + c] += dEdr * d[c] / r;
        }
    }
    for (int a = 0; a < S->n_angles; a++) {
        int i = S->angles[3 * a], j = S->angles[3 * a + 1], k = S->angles[3 * a + 2];
        double u[3], v[3];
        double ru = dist(x, i, j, u);
        double rv = dist(x, k, j, v);
        double c = (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) / (ru * rv);
        if (c > 1.0) c = 1.0;
        if (c < -1.0) c = -1.0;
        double th = acos(c);
        double dth = th - S->angle_t0[a];
        eang += S->angle_k[a] * dth * dth;
        double dEdth = 2.0 * S->angle_k[a] * dth;
        double dthdc = -1.0 / sqrt(1.0 - c * c);
        for (int m = 0; m < 3; m++) {
            double dcdu = v[m] / (ru * rv) - c * u[m] / (ru * ru);
            double dcdv = u[m] / (ru * rv) - c * v[m] / (rv * rv);
            double gi = dEdth * dthdc * dcdu;
            double gk = dEdth * dthdc * dcdv;
            Fl[3 * i + m] -= gi;
            Fl[3 * k + m] -= gk;
            Fl[3 * j + m] += gi + gk;
        }
    }
    terms[0] = egb;
    terms[1] = ecoul;
    terms[2] = elj;
    terms[3] = ebond;
    terms[4] = eang;
    terms[5] = egb + ecoul + elj + ebond + eang;
    if (F) memcpy(F, Fl, sizeof(double) * 3 * (size_t)n);
    if (Rout) memcpy(Rout, R, sizeof(double) * n);
    if (psiout) memcpy(psiout, psi, sizeof(double) * n);
    free(psi);
    free(R);
    free(dEdR);
    free(Fl);
}

/* ------------------------------------------- GB energy and its gradient */

/* E_GB of one configuration and its gradient with respect to the positions,
 * the charges and the intrinsic radii (screening factors held fixed).  Any
 * gradient pointer may be NULL. */
void o_gb_grad(int n, const double *x, const double *q, const double *rho,
               const double *screen, const ogb *g, double *E,
               double *dx, double *dq, double *drho) {
    double *psi = (double *)malloc(sizeof(double) * n);
    double *R = (double *)malloc(sizeof(double) * n);
    double *dEdR = (double *)calloc(n, sizeof(double));
    double *gx = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *gq = (double *)calloc(n, sizeof(double));
    double *gr = (double *)calloc(n, sizeof(double));
    o_born(n, x, rho, screen, g, psi, R);
    double e = 0.0;
    for (int i = 0; i < n; i++) {
        const double ts = gb_tauf(g, R[i]);
        e += -0.5 * O_KCOUL * ts * q[i] * q[i] / R[i];
        gq[i] += -O_KCOUL * ts * q[i] / R[i];
        dEdR[i] += 0.5 * O_KCOUL * gb_taud(g, R[i]) * q[i] * q[i] / (R[i] * R[i]);
        const double esa = sa_energy(g, rho[i], R[i]);
        e += esa;
        dEdR[i] += -6.0 * esa / R[i];
        /* explicit rho dependence of E_SA at fixed R */
        if (esa != 0.0) gr[i] += esa * (2.0 / (rho[i] + g->sa_probe) + 6.0 / rho[i]);
    }
    for (int i = 0; i < n; i++) {
        for (int j = i + 1; j < n; j++) {
            double d[3];
            double r = dist(x, i, j, d);
            double RR = R[i] * R[j];
            double D = r * r / (4.0 * RR);
            double ex = exp(-D);
            double f = sqrt(r * r + RR * ex);
            double qq = q[i] * q[j];
            const double tf = gb_tauf(g, f);
            e += -O_KCOUL * tf * qq / f;
            gq[i] += -O_KCOUL * tf * q[j] / f;
            gq[j] += -O_KCOUL * tf * q[i] / f;
            double dEdf = O_KCOUL * gb_taud(g, f) * qq / (f * f);
            dEdR[i] += dEdf * R[j] * ex * (1.0 + D) / (2.0 * f);
            dEdR[j] += dEdf * R[i] * ex * (1.0 + D) / (2.0 * f);
            double dEdr = dEdf * r / f * (1.0 - 0.25 * ex);
            for (int c = 0; c < 3; c++) {
                gx[3 * i + c] += dEdr * d[c] / r;
                gx[3 * j + c] -= dEdr * d[c] / r;
            }
        }
    }
    for (int k = 0; k < n; k++) {
        double p = psi[k];
        double rtk = rho[k] - g->offset;
        double th = tanh(g->alpha * p - g->beta * p * p + g->gamma * p * p * p);
        double dRdpsi = R[k] * R[k] * (1.0 - th * th)
                      * (g->alpha - 2.0 * g->beta * p + 3.0 * g->gamma * p * p) / rho[k];
        double gpsi = dEdR[k] * dRdpsi;
        /* R_k through 1/rt_k and tanh/rho_k with psi held fixed */
        gr[k] += dEdR[k] * (R[k] * R[k] / (rtk * rtk) - R[k] * R[k] * th / (rho[k] * rho[k]));
        /* psi_k = rt_k * I_k, I_k = 1/2 sum_j H(r_kj, rt_k, s_j) */
        double Ik = (rtk != 0.0) ? p / rtk : 0.0;
        gr[k] += gpsi * Ik;
        for (int j = 0; j < n; j++) {
            if (j == k) continue;
            double d[3];
            double r = dist(x, k, j, d);
            double sj = screen[j] * (rho[j] - g->offset);
            double hdr = o_hct_dr_rc(r, rtk, sj, g->rgbmax);
            for (int c = 0; c < 3; c++) {
                gx[3 * k + c] += gpsi * 0.5 * rtk * hdr * d[c] / r;
                gx[3 * j + c] -= gpsi * 0.5 * rtk * hdr * d[c] / r;
            }
            gr[k] += gpsi * 0.5 * rtk * o_hct_drt_rc(r, rtk, sj, g->rgbmax);
            gr[j] += gpsi * 0.5 * rtk * o_hct_ds_rc(r, rtk, sj, g->rgbmax) * screen[j];
        }
    }
    *E = e;
    if (dx) memcpy(dx, gx, sizeof(double) * 3 * (size_t)n);
    if (dq) memcpy(dq, gq, sizeof(double) * n);
    if (drho) memcpy(drho, gr, sizeof(double) * n);
    free(psi);
    free(R);
    free(dEdR);
    free(gx);
    free(gq);
    free(gr);
}

/* ------------------------------------------------------- Philox4x32-10 */

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
 * multiplies words 0 and 2 by the two round constants, XORs the high halves
 * with words 1 and 3 and the key, and permutes; the key advances by the two
 * Weyl constants between rounds. */
void o_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Counter layout: (index, stream, step low word, purpose | step high bits << 8);
 * key = (seed low word, seed high word). */
static void o_draw(uint64_t seed, uint32_t index, uint32_t stream, uint64_t step,
                   uint32_t purpose, uint32_t out[4]) {
    uint32_t ctr[4] = {index, stream, (uint32_t)step,
                       (purpose & 0xffu) | ((uint32_t)(step >> 32) << 8)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    o_philox(ctr, key, out);
}

/* u in (0, 1): u32 * 2^-32 + 2^-33 */
static double o_unit(uint32_t u) { return (double)u * 2.3283064365386963e-10 + 1.1641532182693481e-10; }

void o_uniforms(uint64_t seed, uint32_t index, uint32_t stream, uint64_t step,
                uint32_t purpose, double out[4]) {
    uint32_t w[4];
    o_draw(seed, index, stream, step, purpose, w);
    for (int i = 0; i < 4; i++) out[i] = o_unit(w[i]);
}

/* Three standard normals from one Philox call: Box-Muller on (u0,u1) gives
 * two, Box-Muller on (u2,u3) gives the third (its cosine branch). */
void o_normals3(uint64_t seed, uint32_t index, uint32_t stream, uint64_t step,
                uint32_t purpose, double z[3]) {
    double u[4];
    o_uniforms(seed, index, stream, step, purpose, u);
    const double two_pi = 6.283185307179586;
    double r0 = sqrt(-2.0 * log(u[0]));
    double r1 = sqrt(-2.0 * log(u[2]));
    z[0] = r0 * cos(two_pi * u[1]);
    z[1] = r0 * sin(two_pi * u[1]);
    z[2] = r1 * cos(two_pi * u[3]);
}

/* --------------------------------------------------------- Langevin step */

/* Leapfrog Langevin (the form of AMBER's ntt=3):
 *   v' = [(1 - g dt/2) v + dt (A F / m) + sqrt(2 g kB T A dt / m) z] / (1 + g dt/2)
 *   x' = x + dt v'
 * with A = 418.4 and z standard normals drawn for (atom, walker, step). */
void o_langevin(int n, double *x, double *v, const double *F, const double *mass,
                double dt, double gamma, double T, uint64_t seed, uint32_t walker,
                uint64_t step) {
    double a = 1.0 - 0.5 * gamma * dt;
    double b = 1.0 / (1.0 + 0.5 * gamma * dt);
    for (int i = 0; i < n; i++) {
        double z[3];
        o_normals3(seed, (uint32_t)i, walker, step, 1u, z);
        double sd = sqrt(2.0 * gamma * O_KB * T * O_ACC * dt / mass[i]);
        for (int c = 0; c < 3; c++) {
            double vn = (a * v[3 * i + c] + dt * O_ACC * F[3 * i + c] / mass[i] + sd * z[c]) * b;
            v[3 * i + c] = vn;
            x[3 * i + c] += dt * vn;
        }
    }
}
