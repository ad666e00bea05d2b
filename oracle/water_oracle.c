/*
 * Oracle for the Langevin NPT step of rigid 3-site water -- TEST INFRASTRUCTURE ONLY (conventions
 * and who may load it: rbe_oracle.c).
 *
 * The paper's bulk-water runs (Sec. 5.1) keep the molecules rigid with SHAKE, while its equations
 * of motion (Sec. 3.2) are written for point particles.  Reading used here:
 *   - each molecule's centre of mass R_I (mass M_I, momentum P_I = sum_i p_i, force F_I = sum_i
 *     F_i) follows the isotropic Langevin NPT equations of Sec. 3.2 with the splitting of Sec. 3.3
 *     (V^p/2, R^p/2, V/2, R/2, O^p, O, R/2, V/2, forces, R^p/2, V^p/2); the cell scales the centres
 *     only, so every molecule keeps its shape;
 *   - the internal motion (d_i = r_i - R_I, internal momenta p_i - m_i P_I / M_I) is constrained
 *     motion under the internal forces F_i - m_i F_I / M_I: R^p/2 kicks it by (dt/2) 100 F_i, R/2
 *     moves it freely by (dt/2) p/m and SHAKE restores the three distances (O-H, O-H, H-H), the
 *     displacement SHAKE adds entering the momenta as m_i dd_i / (dt/2) (RATTLE's position stage);
 *   - O acts on every site, p_i <- g p_i + sqrt(100 kT m_i (1 - g^2)) z_i (the centre's part is the
 *     exact OU update with M_I);
 *   - after every stage that changes momenta (R^p/2, R/2, O) the momenta are projected onto the
 *     velocity constraints (v_a - v_b) . (r_a - r_b) = 0 (RATTLE's velocity stage, a 3x3 linear
 *     solve per molecule), which changes no centre-of-mass momentum;
 *   - pressure: P_ins = (sum_I |P_I|^2 / M_I / 100 + W_mol) / (3V) with the molecular virial
 *     W_mol = W - sum_i F_i . d_i (W the atomic virial trace), -3V dU/dV at fixed scaled centres
 *     and fixed molecular shapes; the constraint forces add nothing to it.
 * Forces: the RBE k-space over all sites (batch of the step, exact sampler, weights S/P) times
 * qqr2e, minus the intramolecular part of the Ewald sum, -qqr2e q_i q_j erf(sqrt(a) r)/r for the
 * three site pairs of each molecule, plus the real space between sites of different molecules
 * (qqr2e q_i q_j erfc(sqrt(a) r)/r within rc, nearest image) and LJ 12-6 between oxygens.
 * Sites are ordered O, H, H per molecule.  After each step every molecule is moved by the lattice
 * vector that brings its oxygen into [0, L), so molecules stay whole in storage (sites may sit up
 * to a bond length outside the box): wrapping the sites one by one would let a box change between
 * the wrap and the next use of the nearest image distort a molecule that straddles the boundary
 * by the change of L.  A molecule is rebuilt whole from its oxygen by the nearest image (a no-op
 * on stored molecules), and its centre is taken from that whole molecule.
 * Extended energy (orc_water_run): sum p^2/(2 m)/100 + U + P V + p_V^2/(2 M_V).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { WAT_OK = 0, WAT_EINVAL = 1, WAT_ENOMEM = 2, WAT_ESHAKE = 3 };
#define FCONV 100.0

#include "npt_params.h"

typedef struct {
    double d_OH, d_HH; /* constraint lengths, A */
    double tol;        /* SHAKE stops after a sweep in which every |r^2 - d^2| <= tol d^2 */
    int32_t max_iter;  /* SHAKE sweeps at most (more: WAT_ESHAKE) */
    int32_t pad;
} orc_water_params;

int orc_sample_k(const double box[3], double alpha, int32_t P, uint64_t seed, uint64_t step, int32_t* m_out,
                 double* S_out);
int orc_rbe_kspace(int64_t N, const double* pos, const double* q, const double box[3], double alpha, int32_t P,
                   const int32_t* m, const double* wl, double* F, double W[9], double E[2], double* rho);
void orc_npt_normals(uint64_t seed, uint32_t stream, uint64_t step, uint32_t index, double z[4]);

static double nearest(double x, double L) { return x - L * nearbyint(x / L); }

/* the molecule I made whole around its oxygen: x[s] = r_O + nearest(r_s - r_O) */
static void whole(const double* r, const double L[3], int64_t I, double x[3][3])
{
    for (int t = 0; t < 3; ++t) x[0][t] = r[9 * I + t];
    for (int s = 1; s < 3; ++s)
        for (int t = 0; t < 3; ++t) x[s][t] = x[0][t] + nearest(r[9 * I + 3 * s + t] - x[0][t], L[t]);
}

static void centre(const double x[3][3], const double* m3, double R[3])
{
    const double M = m3[0] + m3[1] + m3[2];
    for (int t = 0; t < 3; ++t) R[t] = (m3[0] * x[0][t] + m3[1] * x[1][t] + m3[2] * x[2][t]) / M;
}

/* Real space between sites of different molecules within rc (nearest image): erfc Coulomb for
 * every such pair, LJ 12-6 for oxygen pairs.  F accumulates (+=); W[0] the virial trace sum f r^2;
 * E[0] Coulomb, E[1] LJ (accumulated). */
static void water_pairs(int64_t Nmol, const double* r, const double* q, const double L[3], double alpha, double rc,
                        double qqr2e, double sig, double eps, double* F, double* W, double E[2])
{
    const int64_t N = 3 * Nmol;
    const double sa = sqrt(alpha);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = i + 1; j < N; ++j) {
            if (i / 3 == j / 3) continue;
            double d[3];
            for (int t = 0; t < 3; ++t) d[t] = nearest(r[3 * j + t] - r[3 * i + t], L[t]);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rc * rc)) continue;
            const double rr = sqrt(r2), qq = qqr2e * q[i] * q[j], ec = erfc(sa * rr);
            double f = qq * (ec / r2 + 2.0 * sa * exp(-alpha * r2) / (sqrt(M_PI) * rr)) / rr;
            E[0] += qq * ec / rr;
            if (eps != 0.0 && i % 3 == 0 && j % 3 == 0) {
                const double sr2 = sig * sig / r2, sr6 = sr2 * sr2 * sr2;
                E[1] += 4.0 * eps * (sr6 * sr6 - sr6);
                f += 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2;
            }
            for (int t = 0; t < 3; ++t) {
                F[3 * j + t] += f * d[t];
                F[3 * i + t] -= f * d[t];
            }
            *W += f * r2;
        }
}

/* The intramolecular part removed from the Ewald sum: U = -qqr2e q_i q_j erf(sqrt(a) r)/r for the
 * site pairs (0,1), (0,2), (1,2) of every molecule (nearest image).  F, W, E accumulate. */
static void water_exclusions(int64_t Nmol, const double* r, const double* q, const double L[3], double alpha,
                             double qqr2e, double* F, double* W, double* E)
{
    static const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    const double sa = sqrt(alpha);
    for (int64_t I = 0; I < Nmol; ++I)
        for (int c = 0; c < 3; ++c) {
            const int64_t i = 3 * I + pa[c], j = 3 * I + pb[c];
            double d[3];
            for (int t = 0; t < 3; ++t) d[t] = nearest(r[3 * j + t] - r[3 * i + t], L[t]);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], rr = sqrt(r2);
            const double qq = qqr2e * q[i] * q[j], ef = erf(sa * rr);
            /* U = -qq erf(s r)/r; f = -(dU/dr)/r = qq (2 s e^{-a r^2}/(sqrt(pi) r) - erf/r^2) / r */
            const double f = qq * (2.0 * sa * exp(-alpha * r2) / (sqrt(M_PI) * rr) - ef / r2) / rr;
            *E -= qq * ef / rr;
            for (int t = 0; t < 3; ++t) {
                F[3 * j + t] += f * d[t];
                F[3 * i + t] -= f * d[t];
            }
            *W += f * r2;
        }
}

/* Real space and exclusions: F (overwritten), W[0] the atomic virial trace, E = {Coulomb between
 * molecules, LJ, exclusion}. */
int orc_water_real(int64_t Nmol, const double* r, const double* q, const double L[3], double alpha, double rc,
                   double qqr2e, double lj_sigma, double lj_eps, double* F, double* W, double E[3])
{
    if (Nmol < 0 || !(rc > 0.0)) return WAT_EINVAL;
    for (int t = 0; t < 3; ++t)
        if (!(L[t] > 0.0) || rc > 0.5 * L[t]) return WAT_EINVAL;
    for (int64_t i = 0; i < 9 * Nmol; ++i) F[i] = 0.0;
    *W = 0.0;
    E[0] = E[1] = E[2] = 0.0;
    water_pairs(Nmol, r, q, L, alpha, rc, qqr2e, lj_sigma, lj_eps, F, W, E);
    water_exclusions(Nmol, r, q, L, alpha, qqr2e, F, W, &E[2]);
    return WAT_OK;
}

/* -sum_i F_i . d_i, d_i the site's offset from its molecule's centre (whole molecule): added to
 * the atomic virial trace it gives the molecular virial. */
double orc_water_virial_corr(int64_t Nmol, const double* r, const double* m, const double L[3], const double* F)
{
    double s = 0.0;
    for (int64_t I = 0; I < Nmol; ++I) {
        double x[3][3], R[3];
        whole(r, L, I, x);
        centre(x, m + 3 * I, R);
        for (int k = 0; k < 3; ++k)
            for (int t = 0; t < 3; ++t) s -= F[9 * I + 3 * k + t] * (x[k][t] - R[t]);
    }
    return s;
}

/* ------------------------------------------------------------------------------ */
static const int kPa[3] = {0, 0, 1}, kPb[3] = {1, 2, 2};

/* SHAKE for one molecule: x (whole) after an unconstrained move from the constrained xo.  Sweeps
 * over the constraints (0,1), (0,2), (1,2) in that order; each moves its two sites along their
 * old separation so that the distance becomes d (to first order), g = (d^2 - |s|^2) /
 * (2 (1/m_a + 1/m_b) s . s_old); the sweeps stop after one in which every constraint was within
 * tol d^2 before its correction. */
static int shake(double x[3][3], const double xo[3][3], const double m3[3], const orc_water_params* wp)
{
    const double dd[3] = {wp->d_OH * wp->d_OH, wp->d_OH * wp->d_OH, wp->d_HH * wp->d_HH};
    for (int it = 0; it < wp->max_iter; ++it) {
        int done = 1;
        for (int c = 0; c < 3; ++c) {
            const int a = kPa[c], b = kPb[c];
            double s[3], so[3];
            for (int t = 0; t < 3; ++t) {
                s[t] = x[a][t] - x[b][t];
                so[t] = xo[a][t] - xo[b][t];
            }
            const double diff = dd[c] - (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
            if (fabs(diff) > wp->tol * dd[c]) done = 0;
            const double g = diff / (2.0 * (1.0 / m3[a] + 1.0 / m3[b]) * (s[0] * so[0] + s[1] * so[1] + s[2] * so[2]));
            for (int t = 0; t < 3; ++t) {
                x[a][t] += g * so[t] / m3[a];
                x[b][t] -= g * so[t] / m3[b];
            }
        }
        if (done) return WAT_OK;
    }
    return WAT_ESHAKE;
}

/* RATTLE's velocity stage for one molecule: p_i += sum_c mu_c s_c (e_{i,a_c} - e_{i,b_c}) with
 * s_c = x_{a_c} - x_{b_c}, mu from the 3x3 system that makes every (v_a - v_b) . s_c vanish
 * (Cramer's rule).  The sum of the momenta does not change. */
static void rattle_project(double p[3][3], const double x[3][3], const double m3[3])
{
    double s[3][3];
    for (int c = 0; c < 3; ++c)
        for (int t = 0; t < 3; ++t) s[c][t] = x[kPa[c]][t] - x[kPb[c]][t];
    double A[3][3], b[3];
    for (int c = 0; c < 3; ++c) {
        const int a = kPa[c], bb = kPb[c];
        double dv = 0.0;
        for (int t = 0; t < 3; ++t) dv += (p[a][t] / m3[a] - p[bb][t] / m3[bb]) * s[c][t];
        b[c] = -dv;
        for (int d = 0; d < 3; ++d) {
            /* the change of v_a - v_b per unit mu_d, dotted with s_c */
            const double k = ((a == kPa[d]) - (a == kPb[d])) / m3[a] - ((bb == kPa[d]) - (bb == kPb[d])) / m3[bb];
            A[c][d] = k * (s[c][0] * s[d][0] + s[c][1] * s[d][1] + s[c][2] * s[d][2]);
        }
    }
    const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                       A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                       A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    double mu[3];
    for (int k = 0; k < 3; ++k) {
        double B[3][3];
        memcpy(B, A, sizeof(B));
        for (int c = 0; c < 3; ++c) B[c][k] = b[c];
        mu[k] = (B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) - B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
                 B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0])) / det;
    }
    for (int c = 0; c < 3; ++c)
        for (int t = 0; t < 3; ++t) {
            p[kPa[c]][t] += mu[c] * s[c][t];
            p[kPb[c]][t] -= mu[c] * s[c][t];
        }
}

/* Forces at the current state: RBE k-space (batch of `step`) x qqr2e, exclusions, real space.
 * F (3 Nmol x 3); *Wmol the molecular virial; E = {k-space incl. self, Coulomb between
 * molecules, LJ, exclusion}. */
int orc_water_forces(int64_t Nmol, const double* r, const double* q, const double* m, const double L[3],
                     uint64_t step, const orc_npt_params* prm, double* F, double* Wmol, double E[4])
{
    const int64_t N = 3 * Nmol;
    double* tmp = (double*)calloc((size_t)(3 * N + 3), sizeof(double));
    if (!tmp) return WAT_ENOMEM;
    for (int64_t i = 0; i < 3 * N; ++i) F[i] = 0.0;
    E[0] = E[1] = E[2] = E[3] = 0.0;
    double W = 0.0;
    int st = WAT_OK;
    if (prm->kspace) {
        int32_t* mk = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(prm->P > 0 ? prm->P : 1));
        double* wl = (double*)malloc(sizeof(double) * (size_t)(prm->P > 0 ? prm->P : 1));
        double S = 0.0, Wk[9], Ek[2];
        if (!mk || !wl) st = WAT_ENOMEM;
        if (st == WAT_OK) st = orc_sample_k(L, prm->alpha, prm->P, prm->seed, step, mk, &S) ? WAT_EINVAL : WAT_OK;
        if (st == WAT_OK) {
            for (int32_t l = 0; l < prm->P; ++l) wl[l] = S / (double)prm->P;
            st = orc_rbe_kspace(N, r, q, L, prm->alpha, prm->P, mk, wl, tmp, Wk, Ek, NULL) ? WAT_EINVAL : WAT_OK;
        }
        if (st == WAT_OK) {
            for (int64_t i = 0; i < 3 * N; ++i) F[i] += prm->qqr2e * tmp[i];
            W += prm->qqr2e * (Wk[0] + Wk[4] + Wk[8]);
            E[0] = prm->qqr2e * (Ek[0] + Ek[1]);
        }
        free(mk);
        free(wl);
    }
    if (st == WAT_OK && prm->real) {
        double Wr, Er[3];
        st = orc_water_real(Nmol, r, q, L, prm->alpha, prm->rc, prm->qqr2e, prm->lj_sigma, prm->lj_eps, tmp, &Wr, Er);
        if (st == WAT_OK) {
            for (int64_t i = 0; i < 3 * N; ++i) F[i] += tmp[i];
            W += Wr;
            E[1] = Er[0];
            E[2] = Er[1];
            E[3] = Er[2];
        }
    }
    free(tmp);
    if (st == WAT_OK) *Wmol = W + orc_water_virial_corr(Nmol, r, m, L, F);
    return st;
}

static double expm1_over_w(double x, double t)
{
    if (fabs(x) < 1e-8) return t * (1.0 + x * (0.5 + x * (1.0 / 6.0 + x / 24.0)));
    return t * expm1(x) / x;
}

/* sum_I |P_I|^2 / M_I / 100 = 2 K of the centres */
static double kinetic2_mol(int64_t Nmol, const double* p, const double* m)
{
    double s = 0.0;
    for (int64_t I = 0; I < Nmol; ++I) {
        double P[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 3; ++k)
            for (int t = 0; t < 3; ++t) P[t] += p[9 * I + 3 * k + t];
        s += (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / (m[3 * I] + m[3 * I + 1] + m[3 * I + 2]);
    }
    return s / FCONV;
}

/* R^p/2 with eps frozen: P_I <- P_I e^{-eps h} + 100 F_I (1 - e^{-eps h})/eps, the internal
 * momenta kicked by 100 h (F_i - m_i F_I / M_I); then the velocity projection. */
static void kick_mol(int64_t Nmol, double* p, const double* F, const double* r, const double* m, const double L[3],
                     double eps, double h)
{
    const double a = exp(-eps * h), b = expm1_over_w(-eps * h, h);
    for (int64_t I = 0; I < Nmol; ++I) {
        const double* m3 = m + 3 * I;
        const double M = m3[0] + m3[1] + m3[2];
        double P[3] = {0, 0, 0}, Ft[3] = {0, 0, 0}, pp[3][3], x[3][3];
        for (int k = 0; k < 3; ++k)
            for (int t = 0; t < 3; ++t) {
                pp[k][t] = p[9 * I + 3 * k + t];
                P[t] += pp[k][t];
                Ft[t] += F[9 * I + 3 * k + t];
            }
        double dP[3];
        for (int t = 0; t < 3; ++t) dP[t] = P[t] * a + FCONV * Ft[t] * b - P[t];
        for (int k = 0; k < 3; ++k)
            for (int t = 0; t < 3; ++t)
                pp[k][t] += FCONV * h * (F[9 * I + 3 * k + t] - m3[k] * Ft[t] / M) + (m3[k] / M) * dP[t];
        whole(r, L, I, x);
        rattle_project(pp, x, m3);
        for (int k = 0; k < 3; ++k)
            for (int t = 0; t < 3; ++t) p[9 * I + 3 * k + t] = pp[k][t];
    }
}

/* R/2 with eps frozen: R_I <- R_I e^{eps h} + (P_I/M_I)(e^{eps h} - 1)/eps (the peculiar part
 * capped), the internal offsets moved by h p/m then SHAKEn, the SHAKE displacement added to the
 * momenta as m dd / h, then the velocity projection at the new positions. */
static int drift_mol(int64_t Nmol, double* r, double* p, const double* m, const double L[3], double eps, double h,
                     double cap, const orc_water_params* wp)
{
    const double a = exp(eps * h), b = expm1_over_w(eps * h, h);
    for (int64_t I = 0; I < Nmol; ++I) {
        const double* m3 = m + 3 * I;
        const double M = m3[0] + m3[1] + m3[2];
        double x[3][3], R[3], d[3][3], dn[3][3], pp[3][3], P[3] = {0, 0, 0};
        whole(r, L, I, x);
        centre(x, m3, R);
        for (int k = 0; k < 3; ++k)
            for (int t = 0; t < 3; ++t) {
                pp[k][t] = p[9 * I + 3 * k + t];
                P[t] += pp[k][t];
                d[k][t] = x[k][t] - R[t];
            }
        double D[3];
        for (int t = 0; t < 3; ++t) D[t] = (P[t] / M) * b;
        if (cap > 0.0) {
            const double len = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
            if (len > cap)
                for (int t = 0; t < 3; ++t) D[t] *= cap / len;
        }
        double Rn[3];
        for (int t = 0; t < 3; ++t) Rn[t] = R[t] + R[t] * (a - 1.0) + D[t];
        for (int k = 0; k < 3; ++k)
            for (int t = 0; t < 3; ++t) dn[k][t] = d[k][t] + h * (pp[k][t] / m3[k] - P[t] / M);
        double ds[3][3];
        memcpy(ds, dn, sizeof(ds));
        if (shake(ds, d, m3, wp) != WAT_OK) return WAT_ESHAKE;
        for (int k = 0; k < 3; ++k)
            for (int t = 0; t < 3; ++t) {
                pp[k][t] += m3[k] * (ds[k][t] - dn[k][t]) / h;
                x[k][t] = Rn[t] + ds[k][t];
            }
        rattle_project(pp, x, m3);
        for (int k = 0; k < 3; ++k)
            for (int t = 0; t < 3; ++t) {
                p[9 * I + 3 * k + t] = pp[k][t];
                r[9 * I + 3 * k + t] = x[k][t];
            }
    }
    return WAT_OK;
}

/* the Langevin update of every site, then the velocity projection */
static void langevin_mol(int64_t Nmol, double* p, const double* r, const double* m, const double L[3], uint64_t step,
                         const orc_npt_params* prm)
{
    const double g = exp(-prm->gamma * prm->dt);
    for (int64_t i = 0; i < 3 * Nmol; ++i) {
        double z[4] = {0.0, 0.0, 0.0, 0.0};
        if (prm->noise) orc_npt_normals(prm->seed, 1u, step, (uint32_t)i, z);
        const double s = sqrt(prm->kT * FCONV * m[i] * (1.0 - g * g));
        for (int t = 0; t < 3; ++t) p[3 * i + t] = p[3 * i + t] * g + s * z[t];
    }
    for (int64_t I = 0; I < Nmol; ++I) {
        double pp[3][3], x[3][3];
        whole(r, L, I, x);
        for (int k = 0; k < 3; ++k)
            for (int t = 0; t < 3; ++t) pp[k][t] = p[9 * I + 3 * k + t];
        rattle_project(pp, x, m + 3 * I);
        for (int k = 0; k < 3; ++k)
            for (int t = 0; t < 3; ++t) p[9 * I + 3 * k + t] = pp[k][t];
    }
}

static void scale_box_w(double L[3], double Vnew)
{
    const double f = cbrt(Vnew / (L[0] * L[1] * L[2]));
    for (int t = 0; t < 3; ++t) L[t] *= f;
}

/* One step.  State in/out: r, p, F (forces at r), L, pV, Wmol (molecular virial at r); E the
 * energies at the new state. */
int orc_water_step(int64_t Nmol, double* r, double* p, double* F, const double* q, const double* m, double L[3],
                   double* pV, double* Wmol, uint64_t step, const orc_npt_params* prm, const orc_water_params* wp,
                   double E[4])
{
    if (prm->barostat < 0 || prm->barostat > 1 || !(prm->dt > 0.0)) return WAT_EINVAL;
    const double h = 0.5 * prm->dt, cap = 0.5 * prm->max_disp;
    double V = L[0] * L[1] * L[2];
    if (prm->barostat) *pV += h * ((kinetic2_mol(Nmol, p, m) + *Wmol) / (3.0 * V) - prm->P_ext); /* V^p/2 */
    double eps = prm->barostat ? *pV / (3.0 * prm->M_V * V) : 0.0;
    kick_mol(Nmol, p, F, r, m, L, eps, h); /* R^p/2 */
    if (prm->barostat) {                   /* V/2 */
        scale_box_w(L, V + h * (*pV) / prm->M_V);
        V = L[0] * L[1] * L[2];
    }
    eps = prm->barostat ? *pV / (3.0 * prm->M_V * V) : 0.0;
    int st = drift_mol(Nmol, r, p, m, L, eps, h, cap, wp); /* R/2 */
    if (st != WAT_OK) return st;
    if (prm->barostat) { /* O^p */
        const double g = exp(-prm->gamma_V * prm->dt);
        *pV *= g;
        if (prm->noise) {
            double z[4];
            orc_npt_normals(prm->seed, 2u, step, 0u, z);
            *pV += sqrt(prm->kT * prm->M_V * (1.0 - g * g)) * z[0];
        }
    }
    langevin_mol(Nmol, p, r, m, L, step, prm); /* O */
    eps = prm->barostat ? *pV / (3.0 * prm->M_V * V) : 0.0;
    st = drift_mol(Nmol, r, p, m, L, eps, h, cap, wp); /* R/2 */
    if (st != WAT_OK) return st;
    if (prm->barostat) { /* V/2 */
        scale_box_w(L, V + h * (*pV) / prm->M_V);
        V = L[0] * L[1] * L[2];
    }
    /* wrap by molecule: the lattice vector that brings the oxygen into [0, L) moves all its sites */
    for (int64_t I = 0; I < Nmol; ++I)
        for (int t = 0; t < 3; ++t) {
            const double sh = L[t] * floor(r[9 * I + t] / L[t]);
            for (int k = 0; k < 3; ++k) r[9 * I + 3 * k + t] -= sh;
        }
    st = orc_water_forces(Nmol, r, q, m, L, step, prm, F, Wmol, E);
    if (st != WAT_OK) return st;
    eps = prm->barostat ? *pV / (3.0 * prm->M_V * V) : 0.0;
    kick_mol(Nmol, p, F, r, m, L, eps, h); /* R^p/2 */
    if (prm->barostat) *pV += h * ((kinetic2_mol(Nmol, p, m) + *Wmol) / (3.0 * V) - prm->P_ext); /* V^p/2 */
    return WAT_OK;
}

/* Largest relative violation of the distance constraints |r - d| / d and of the velocity
 * constraints |(v_a - v_b) . s| / (|v_a - v_b| |s|) over every molecule. */
void orc_water_violation(int64_t Nmol, const double* r, const double* p, const double* m, const double L[3],
                         const orc_water_params* wp, double out[2])
{
    out[0] = out[1] = 0.0;
    const double d[3] = {wp->d_OH, wp->d_OH, wp->d_HH};
    for (int64_t I = 0; I < Nmol; ++I) {
        double x[3][3];
        whole(r, L, I, x);
        const double* m3 = m + 3 * I;
        for (int c = 0; c < 3; ++c) {
            const int a = kPa[c], b = kPb[c];
            double s[3], v[3];
            for (int t = 0; t < 3; ++t) {
                s[t] = x[a][t] - x[b][t];
                v[t] = p[9 * I + 3 * a + t] / m3[a] - p[9 * I + 3 * b + t] / m3[b];
            }
            const double ls = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
            const double lv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            const double e0 = fabs(ls - d[c]) / d[c];
            const double e1 = lv > 0.0 ? fabs(v[0] * s[0] + v[1] * s[1] + v[2] * s[2]) / (lv * ls) : 0.0;
            if (e0 > out[0]) out[0] = e0;
            if (e1 > out[1]) out[1] = e1;
        }
    }
}

/* n steps from step0; per step V, P_ins (molecular) and the extended energy
 * sum p^2/(2m)/100 + U + P V + p_V^2/(2 M_V) (optional arrays). */
int orc_water_run(int64_t Nmol, double* r, double* p, double* F, const double* q, const double* m, double L[3],
                  double* pV, double* Wmol, uint64_t step0, int32_t n, const orc_npt_params* prm,
                  const orc_water_params* wp, double* V_out, double* P_out, double* H_out)
{
    for (int32_t s = 0; s < n; ++s) {
        double E[4];
        const int st = orc_water_step(Nmol, r, p, F, q, m, L, pV, Wmol, step0 + (uint64_t)s, prm, wp, E);
        if (st != WAT_OK) return st;
        const double V = L[0] * L[1] * L[2];
        if (V_out) V_out[s] = V;
        if (P_out) P_out[s] = (kinetic2_mol(Nmol, p, m) + *Wmol) / (3.0 * V);
        if (H_out) {
            double K = 0.0;
            for (int64_t i = 0; i < 3 * Nmol; ++i)
                K += (p[3 * i] * p[3 * i] + p[3 * i + 1] * p[3 * i + 1] + p[3 * i + 2] * p[3 * i + 2]) / (2.0 * m[i]);
            H_out[s] = K / FCONV + E[0] + E[1] + E[2] + E[3] + prm->P_ext * V +
                       (prm->barostat ? (*pV) * (*pV) / (2.0 * prm->M_V) : 0.0);
        }
    }
    return WAT_OK;
}
