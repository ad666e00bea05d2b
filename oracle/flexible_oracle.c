/*
 * Oracle for the Langevin NPT step of the fully flexible cell (App. A, the fully flexible cells)
 * -- TEST INFRASTRUCTURE ONLY (conventions and who may load it: rbe_oracle.c).
 *
 * Cell h (3x3, row-major, the cell vectors as columns), momenta p^h (3x3), masses M_te (3x3).
 * Equations of motion (the paper's, with the Hamiltonian of Gao et al.):
 *   dr/dt = p/m + A r,          dp/dt = F - A^T p - gamma p + sqrt(2 kT m gamma) xi,   A = (dh/dt) h^{-1}
 *   dh/dt = p^h / M (entrywise), dp^h/dt = (Kt + W - (P V + chi kT) I) h^{-T} - gamma_h p^h + noise,
 * with Kt = sum_i p_i p_i^T / m_i (the kinetic tensor, /100 to kJ/mol), W the full virial tensor
 * (k-space x qqr2e plus real space), V = det h, and chi = d - 1 = 2 from the det(h)^{1-d} factor
 * of the flexible cell's distribution.  Extended energy
 *   H = K + U + P V + chi kT ln V + sum_te (p^h_te)^2 / (2 M_te).
 * Splitting (Sec. 3.3 with the cell matrix): V^p/2, R^p/2, V/2, R/2, O^p, O, R/2, V/2, [forces],
 * R^p/2, V^p/2.  R: r <- e^{At} r + phi(At) t p/m; R^p: p <- e^{-A^T t} p + phi(-A^T t) t 100 F,
 * with A frozen over the sub-step and phi(X) = sum_k X^k/(k+1)!; both series summed until the
 * term is below 1e-20 of the running sum (|At| is small).  The displacement cap holds the peculiar
 * part phi(At) t p/m.  V/2: h <- h + (dt/2) p^h / M.  O^p: p^h_te <- g p^h_te + sqrt(kT M_te
 * (1 - g^2)) z_te with the cell normals of stream 2: index 0 gives z for the diagonal (z[0], z[1],
 * z[2], the rectangular step's), indices 1 and 2 the off-diagonal entries in row-major order.
 * Forces: RBE k-space in the general cell with the MH frequencies of general_oracle.c (batch of
 * the step, weights S/P) times qqr2e, plus the real space (erfc Coulomb x qqr2e + LJ 12-6) over
 * every image within rc.  Positions are wrapped into the cell after each step (s -= floor(s)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { FLX_OK = 0, FLX_EINVAL = 1, FLX_ENOMEM = 2 };
#define FCONV 100.0

double orc_gen_inverse(const double h[9], double hinv[9]);
int orc_gen_kspace(int64_t N, const double* pos, const double* q, const double h[9], double alpha, int32_t K,
                   const int32_t* m, const double* wl, double* F, double W[9], double E[2]);
int orc_gen_sample_k_mh(const double h[9], double alpha, int32_t P, uint64_t seed, uint64_t step, int32_t* state,
                        double* S_out);
void orc_npt_normals(uint64_t seed, uint32_t stream, uint64_t step, uint32_t index, double z[4]);

typedef struct {
    double dt, kT, P_ext, gamma, gamma_h;
    double M[9];      /* cell masses, kJ/mol ps^2 / A^2 */
    double alpha, rc, qqr2e, lj_sigma, lj_eps, max_disp, chi;
    int32_t P, kspace, real, noise;
    uint64_t seed;
    int32_t* chain;   /* P x 3 MH state (kspace) */
} orc_flex_params;

static void matmul(const double a[9], const double b[9], double c[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

static double maxabs(const double a[9])
{
    double m = 0.0;
    for (int i = 0; i < 9; ++i) m = fabs(a[i]) > m ? fabs(a[i]) : m;
    return m;
}

/* E = e^X and Phi = sum_k X^k/(k+1)! by their Taylor series */
static void exp_phi(const double X[9], double E[9], double Phi[9])
{
    double term[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, t2[9];
    for (int i = 0; i < 9; ++i) {
        E[i] = term[i];
        Phi[i] = term[i];
    }
    for (int k = 1; k <= 40; ++k) {
        matmul(term, X, t2);
        for (int i = 0; i < 9; ++i) term[i] = t2[i] / (double)k; /* X^k / k! */
        for (int i = 0; i < 9; ++i) {
            E[i] += term[i];
            Phi[i] += term[i] / (double)(k + 1);
        }
        if (maxabs(term) < 1e-20 * maxabs(E)) break;
    }
}

/* Real space in the general cell: every image within rc, qqr2e q_i q_j erfc(sqrt(a) r)/r +
 * 4 eps ((s/r)^12 - (s/r)^6), forces on both ends, the full virial sum f d d^T; E[0] Coulomb,
 * E[1] LJ.  The self images (i = j, n != 0) count half. */
int orc_flex_pair_real(int64_t N, const double* pos, const double* q, const double h[9], double alpha, double rc,
                       double qqr2e, double lj_sigma, double lj_eps, double* F, double W[9], double E[2])
{
    double hinv[9];
    if (!(orc_gen_inverse(h, hinv) > 0.0) || !(rc > 0.0)) return FLX_EINVAL;
    int32_t R[3];
    for (int t = 0; t < 3; ++t) {
        double rn = sqrt(hinv[3 * t] * hinv[3 * t] + hinv[3 * t + 1] * hinv[3 * t + 1] + hinv[3 * t + 2] * hinv[3 * t + 2]);
        R[t] = (int32_t)ceil(rc * rn) + 1;
    }
    for (int64_t i = 0; i < 3 * N; ++i) F[i] = 0.0;
    for (int j = 0; j < 9; ++j) W[j] = 0.0;
    E[0] = E[1] = 0.0;
    double sa = sqrt(alpha);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = i; j < N; ++j)
            for (int32_t a = -R[0]; a <= R[0]; ++a)
                for (int32_t b = -R[1]; b <= R[1]; ++b)
                    for (int32_t c = -R[2]; c <= R[2]; ++c) {
                        if (i == j && a == 0 && b == 0 && c == 0) continue;
                        double d[3];
                        for (int t = 0; t < 3; ++t)
                            d[t] = pos[3 * j + t] - pos[3 * i + t] + h[3 * t] * a + h[3 * t + 1] * b + h[3 * t + 2] * c;
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (!(r2 < rc * rc)) continue;
                        double r = sqrt(r2), wgt = (i == j) ? 0.5 : 1.0;
                        double qq = qqr2e * q[i] * q[j], ec = erfc(sa * r);
                        double f = qq * (ec / r2 + 2.0 * sa * exp(-alpha * r2) / (sqrt(M_PI) * r)) / r;
                        E[0] += wgt * qq * ec / r;
                        if (lj_eps != 0.0) {
                            double sr2 = lj_sigma * lj_sigma / r2, sr6 = sr2 * sr2 * sr2;
                            E[1] += wgt * 4.0 * lj_eps * (sr6 * sr6 - sr6);
                            f += 24.0 * lj_eps * (2.0 * sr6 * sr6 - sr6) / r2;
                        }
                        f *= wgt;
                        for (int t = 0; t < 3; ++t) {
                            F[3 * j + t] += f * d[t];
                            F[3 * i + t] -= f * d[t];
                        }
                        for (int x = 0; x < 3; ++x)
                            for (int y = 0; y < 3; ++y) W[3 * x + y] += f * d[x] * d[y];
                    }
    return FLX_OK;
}

/* Forces (kJ/mol/A), the full virial tensor W (kJ/mol) and the energies E[0] k-space (incl.
 * self), E[1] real Coulomb, E[2] LJ at the current state; the RBE batch of `step`. */
int orc_flex_forces(int64_t N, const double* r, const double* q, const double h[9], uint64_t step,
                    const orc_flex_params* prm, double* F, double W[9], double E[3])
{
    double* tmp = (double*)calloc((size_t)(3 * N + 3), sizeof(double));
    if (!tmp) return FLX_ENOMEM;
    for (int64_t i = 0; i < 3 * N; ++i) F[i] = 0.0;
    for (int j = 0; j < 9; ++j) W[j] = 0.0;
    E[0] = E[1] = E[2] = 0.0;
    int st = FLX_OK;
    if (prm->kspace) {
        double* wl = (double*)malloc(sizeof(double) * (size_t)(prm->P > 0 ? prm->P : 1));
        double S = 0.0, Wk[9], Ek[2];
        if (!wl || !prm->chain) st = wl ? FLX_EINVAL : FLX_ENOMEM;
        if (st == FLX_OK) st = orc_gen_sample_k_mh(h, prm->alpha, prm->P, prm->seed, step, prm->chain, &S);
        if (st == FLX_OK) {
            for (int32_t l = 0; l < prm->P; ++l) wl[l] = S / (double)prm->P;
            st = orc_gen_kspace(N, r, q, h, prm->alpha, prm->P, prm->chain, wl, tmp, Wk, Ek);
        }
        if (st == FLX_OK) {
            for (int64_t i = 0; i < 3 * N; ++i) F[i] += prm->qqr2e * tmp[i];
            for (int j = 0; j < 9; ++j) W[j] += prm->qqr2e * Wk[j];
            E[0] = prm->qqr2e * (Ek[0] + Ek[1]);
        }
        free(wl);
    }
    if (st == FLX_OK && prm->real) {
        double Wr[9], Er[2];
        st = orc_flex_pair_real(N, r, q, h, prm->alpha, prm->rc, prm->qqr2e, prm->lj_sigma, prm->lj_eps, tmp, Wr, Er);
        if (st == FLX_OK) {
            for (int64_t i = 0; i < 3 * N; ++i) F[i] += tmp[i];
            for (int j = 0; j < 9; ++j) W[j] += Wr[j];
            E[1] = Er[0];
            E[2] = Er[1];
        }
    }
    free(tmp);
    return st;
}

/* the cell's rate matrix A = (p^h / M) h^{-1} */
static void rate_matrix(const double h[9], const double ph[9], const orc_flex_params* prm, double A[9])
{
    double hinv[9], hd[9];
    orc_gen_inverse(h, hinv);
    for (int i = 0; i < 9; ++i) hd[i] = ph[i] / prm->M[i];
    matmul(hd, hinv, A);
}

static void kinetic_tensor(int64_t N, const double* p, const double* m, double Kt[9])
{
    for (int a = 0; a < 9; ++a) Kt[a] = 0.0;
    for (int64_t i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Kt[3 * a + b] += p[3 * i + a] * p[3 * i + b] / m[i];
    for (int a = 0; a < 9; ++a) Kt[a] /= FCONV;
}

/* V^p/2: p^h += (dt/2) (Kt + W - (P V + chi kT) I) h^{-T} */
static void kick_cell(double ph[9], const double h[9], const double Kt[9], const double W[9], const orc_flex_params* prm)
{
    double hinv[9];
    double V = orc_gen_inverse(h, hinv);
    double X[9];
    for (int a = 0; a < 9; ++a) X[a] = Kt[a] + W[a];
    for (int a = 0; a < 3; ++a) X[4 * a] -= prm->P_ext * V + prm->chi * prm->kT;
    for (int t = 0; t < 3; ++t)
        for (int e = 0; e < 3; ++e)
            ph[3 * t + e] += 0.5 * prm->dt * (X[3 * t] * hinv[3 * e] + X[3 * t + 1] * hinv[3 * e + 1] + X[3 * t + 2] * hinv[3 * e + 2]);
}

/* R^p/2: p <- e^{-A^T t} p + phi(-A^T t) t 100 F */
static void kick_particles(int64_t N, double* p, const double* F, const double A[9], double t)
{
    double X[9], E[9], Phi[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) X[3 * a + b] = -A[3 * b + a] * t;
    exp_phi(X, E, Phi);
    for (int64_t i = 0; i < N; ++i) {
        double pn[3];
        for (int a = 0; a < 3; ++a)
            pn[a] = E[3 * a] * p[3 * i] + E[3 * a + 1] * p[3 * i + 1] + E[3 * a + 2] * p[3 * i + 2] +
                    t * FCONV * (Phi[3 * a] * F[3 * i] + Phi[3 * a + 1] * F[3 * i + 1] + Phi[3 * a + 2] * F[3 * i + 2]);
        for (int a = 0; a < 3; ++a) p[3 * i + a] = pn[a];
    }
}

/* R/2: r <- e^{A t} r + cap(phi(A t) t p/m) */
static void drift(int64_t N, double* r, const double* p, const double* m, const double A[9], double t, double cap)
{
    double X[9], E[9], Phi[9];
    for (int a = 0; a < 9; ++a) X[a] = A[a] * t;
    exp_phi(X, E, Phi);
    for (int64_t i = 0; i < N; ++i) {
        double d[3], rn[3];
        for (int a = 0; a < 3; ++a)
            d[a] = t * (Phi[3 * a] * p[3 * i] + Phi[3 * a + 1] * p[3 * i + 1] + Phi[3 * a + 2] * p[3 * i + 2]) / m[i];
        if (cap > 0.0) {
            double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (len > cap)
                for (int a = 0; a < 3; ++a) d[a] *= cap / len;
        }
        for (int a = 0; a < 3; ++a)
            rn[a] = E[3 * a] * r[3 * i] + E[3 * a + 1] * r[3 * i + 1] + E[3 * a + 2] * r[3 * i + 2] + d[a];
        for (int a = 0; a < 3; ++a) r[3 * i + a] = rn[a];
    }
}

/* V/2 */
static void move_cell(double h[9], const double ph[9], const orc_flex_params* prm)
{
    for (int a = 0; a < 9; ++a) h[a] += 0.5 * prm->dt * ph[a] / prm->M[a];
}

/* One step; F and W hold the forces and virial at the input state and are updated. */
int orc_flex_step(int64_t N, double* r, double* p, double* F, const double* q, const double* m, double h[9],
                  double ph[9], double W[9], uint64_t step, const orc_flex_params* prm, double E[3])
{
    double hinv[9];
    if (!(orc_gen_inverse(h, hinv) > 0.0) || !(prm->dt > 0.0)) return FLX_EINVAL;
    for (int a = 0; a < 9; ++a)
        if (!(prm->M[a] > 0.0)) return FLX_EINVAL;
    const double t = 0.5 * prm->dt;
    double Kt[9], A[9];
    kinetic_tensor(N, p, m, Kt);
    kick_cell(ph, h, Kt, W, prm);
    rate_matrix(h, ph, prm, A);
    kick_particles(N, p, F, A, t);
    move_cell(h, ph, prm);
    rate_matrix(h, ph, prm, A);
    drift(N, r, p, m, A, t, 0.5 * prm->max_disp);
    {   /* O^p */
        double g = exp(-prm->gamma_h * prm->dt);
        double z0[4] = {0, 0, 0, 0}, z1[4] = {0, 0, 0, 0}, z2[4] = {0, 0, 0, 0};
        if (prm->noise) {
            orc_npt_normals(prm->seed, 2u, step, 0u, z0);
            orc_npt_normals(prm->seed, 2u, step, 1u, z1);
            orc_npt_normals(prm->seed, 2u, step, 2u, z2);
        }
        /* diagonal te = 0, 4, 8 take z0[0..2]; off-diagonal 1, 2, 3, 5, 6, 7 take z1[0..3], z2[0..1] */
        const double zz[9] = {z0[0], z1[0], z1[1], z1[2], z0[1], z1[3], z2[0], z2[1], z0[2]};
        for (int a = 0; a < 9; ++a) {
            ph[a] *= g;
            if (prm->noise) ph[a] += sqrt(prm->kT * prm->M[a] * (1.0 - g * g)) * zz[a];
        }
    }
    {   /* O */
        double g = exp(-prm->gamma * prm->dt);
        for (int64_t i = 0; i < N; ++i) {
            double z[4] = {0.0, 0.0, 0.0, 0.0};
            if (prm->noise) orc_npt_normals(prm->seed, 1u, step, (uint32_t)i, z);
            double sg = sqrt(prm->kT * FCONV * m[i] * (1.0 - g * g));
            for (int a = 0; a < 3; ++a) p[3 * i + a] = p[3 * i + a] * g + sg * z[a];
        }
    }
    rate_matrix(h, ph, prm, A);
    drift(N, r, p, m, A, t, 0.5 * prm->max_disp);
    move_cell(h, ph, prm);
    /* wrap: s = h^{-1} r into [0, 1) */
    if (!(orc_gen_inverse(h, hinv) > 0.0)) return FLX_EINVAL;
    for (int64_t i = 0; i < N; ++i) {
        double s[3];
        for (int a = 0; a < 3; ++a) {
            s[a] = hinv[3 * a] * r[3 * i] + hinv[3 * a + 1] * r[3 * i + 1] + hinv[3 * a + 2] * r[3 * i + 2];
            s[a] -= floor(s[a]);
        }
        for (int a = 0; a < 3; ++a) r[3 * i + a] = h[3 * a] * s[0] + h[3 * a + 1] * s[1] + h[3 * a + 2] * s[2];
    }
    int st = orc_flex_forces(N, r, q, h, step, prm, F, W, E);
    if (st != FLX_OK) return st;
    rate_matrix(h, ph, prm, A);
    kick_particles(N, p, F, A, t);
    kinetic_tensor(N, p, m, Kt);
    kick_cell(ph, h, Kt, W, prm);
    return FLX_OK;
}

/* n steps; per step the cell (h_out, 9 each), the pressure tensor (P_out, 9 each) and the extended
 * energy K + U + P V + chi kT ln V + sum (p^h)^2 / 2M (H_out), each optional. */
int orc_flex_run(int64_t N, double* r, double* p, double* F, const double* q, const double* m, double h[9],
                 double ph[9], double W[9], uint64_t step0, int32_t n, const orc_flex_params* prm, double* h_out,
                 double* P_out, double* H_out)
{
    for (int32_t s = 0; s < n; ++s) {
        double E[3], Kt[9], hinv[9];
        int st = orc_flex_step(N, r, p, F, q, m, h, ph, W, step0 + (uint64_t)s, prm, E);
        if (st != FLX_OK) return st;
        double V = orc_gen_inverse(h, hinv);
        kinetic_tensor(N, p, m, Kt);
        if (h_out) memcpy(h_out + 9 * s, h, 9 * sizeof(double));
        if (P_out)
            for (int a = 0; a < 9; ++a) P_out[9 * s + a] = (Kt[a] + W[a]) / V;
        if (H_out) {
            double H = 0.5 * (Kt[0] + Kt[4] + Kt[8]) + E[0] + E[1] + E[2] + prm->P_ext * V + prm->chi * prm->kT * log(V);
            for (int a = 0; a < 9; ++a) H += ph[a] * ph[a] / (2.0 * prm->M[a]);
            H_out[s] = H;
        }
    }
    return FLX_OK;
}
