/*
 * Oracle for the k-space part of the Ewald sum and of RBE in a general (triclinic) cell
 * (App. C: the fully flexible cell) -- TEST INFRASTRUCTURE ONLY (conventions and who may load
 * it: rbe_oracle.c).
 *
 * Cell: h = (a | b | c), a 3x3 matrix whose COLUMNS are the cell vectors, row-major in memory
 * (h[3*i + j] = component i of vector j); r = h s with s the scaled coordinates, V = det h > 0.
 * Wave vectors k = 2 pi h^{-T} m for integer m, so k.r = 2 pi m.s and
 * |k|^2 = 4 pi^2 m^T G m with G = h^{-1} h^{-T}.
 *   E_k = (2 pi / V) sum_{m != 0} exp(-|k|^2/4a)/|k|^2 |rho(k)|^2             (App. C; Sec. 4.1)
 *   F_i = -sum (4 pi q_i k / (V |k|^2)) exp(-|k|^2/4a) Im(e^{-ik.r_i} rho(k))
 *   W   = (2 pi / V) sum |rho|^2/|k|^2 exp(-|k|^2/4a) [I - 2 (1/|k|^2 + 1/4a) k k^T]
 *                                                          (App. C Eq. (pressuretensorflexible))
 * RBE on a batch: the same sums over the sampled m with weights w_l in place of exp(-|k|^2/4a).
 *
 * Sampling (App. C: the law P(m) ~ exp(-pi^2 m^T G m / alpha) does not factorise in a general
 * cell; the paper suggests discrete Metropolis--Hastings): an independence MH chain per slot whose
 * proposal is an exact product law prod_j exp(-c_j m_j^2) on Z^3 \ {0}, drawn by the per-axis
 * inverse CDF of rbe_oracle.c with effective lengths l_j, c_j = pi^2/(alpha l_j^2).  The lengths
 * make the proposal's precision diag(c) no larger than the target's A = pi^2 G / alpha:
 * l_j^2 = lambda |a_j|^2 with |a_j| the length of cell vector j ((G^{-1})_jj = (h^T h)_jj) and
 * lambda = max_j (1 + sum_{k != j} |cos theta_jk|), a Gershgorin bound on the largest eigenvalue
 * of the matrix of the cell vectors' angle cosines.  Then target / proposal is bounded (the chain
 * mixes uniformly), and a rectangular cell (lambda = 1) proposes the target itself.  With
 * O(m) = (pi^2/alpha) m^T G m - sum_j c_j m_j^2 >= 0, m' is accepted when O(m') <= O(m), else
 * when u < exp(O(m) - O(m')) (the tables' exponential).  A slot at m = 0 starts from the proposal
 * of its first step.  Proposals use the exact sampler's counters
 * (stream 0) at the step, the acceptance uniform stream 5: (l, 0, step_lo, (5 << 24) | step_hi24).
 *
 * S = sum_{m != 0} exp(-pi^2 m^T G m / alpha), the importance normalisation (Eq. (S)), from the
 * Poisson summation of the Gaussian over the lattice:
 *   S = (alpha/pi)^{3/2} V sum_{n in Z^3} exp(-alpha |h n|^2) - 1,
 * the dual sum over the n with alpha |h n|^2 <= 60 ln 2 + 50 (terms below 2^-60 e^-50 dropped).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { GEN_OK = 0, GEN_EINVAL = 1, GEN_ENOMEM = 2, GEN_ESAMPLE = 6 };

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_exp(double x);
int orc_sample_k(const double box[3], double alpha, int32_t P, uint64_t seed, uint64_t step, int32_t* m_out,
                 double* S_out);

/* h^{-1} by cofactors; returns det h (0 when singular). */
double orc_gen_inverse(const double h[9], double hinv[9])
{
    double c00 = h[4] * h[8] - h[5] * h[7], c01 = h[5] * h[6] - h[3] * h[8], c02 = h[3] * h[7] - h[4] * h[6];
    double det = h[0] * c00 + h[1] * c01 + h[2] * c02;
    if (det == 0.0) return 0.0;
    hinv[0] = c00 / det;
    hinv[1] = (h[2] * h[7] - h[1] * h[8]) / det;
    hinv[2] = (h[1] * h[5] - h[2] * h[4]) / det;
    hinv[3] = c01 / det;
    hinv[4] = (h[0] * h[8] - h[2] * h[6]) / det;
    hinv[5] = (h[2] * h[3] - h[0] * h[5]) / det;
    hinv[6] = c02 / det;
    hinv[7] = (h[1] * h[6] - h[0] * h[7]) / det;
    hinv[8] = (h[0] * h[4] - h[1] * h[3]) / det;
    return det;
}

/* k = 2 pi h^{-T} m: k_i = 2 pi sum_j hinv[j][i] m_j */
static void wave_vector(const double hinv[9], const int32_t m[3], double k[3])
{
    for (int i = 0; i < 3; ++i)
        k[i] = 2.0 * M_PI * (hinv[0 * 3 + i] * m[0] + hinv[1 * 3 + i] * m[1] + hinv[2 * 3 + i] * m[2]);
}

/* G = h^{-1} h^{-T}: G_ij = sum_k hinv[i][k] hinv[j][k] */
void orc_gen_metric(const double h[9], double G[9])
{
    double hinv[9];
    orc_gen_inverse(h, hinv);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            G[3 * i + j] = hinv[3 * i] * hinv[3 * j] + hinv[3 * i + 1] * hinv[3 * j + 1] +
                           hinv[3 * i + 2] * hinv[3 * j + 2];
}

/* The k-space sums over the listed m (K of them) with weights w_l (Ewald: exp(-|k|^2/4a); RBE:
 * S/P): forces F[N][3], virial W[9] (energy units), E[0] = E_k, E[1] = E_self = -sqrt(a/pi) sum q^2.
 * rho(k) = sum_i q_i e^{i k.r_i} with the phase formed as 2 pi m.s, s = h^{-1} r. */
int orc_gen_kspace(int64_t N, const double* pos, const double* q, const double h[9], double alpha, int32_t K,
                   const int32_t* m, const double* wl, double* F, double W[9], double E[2])
{
    double hinv[9];
    double V = orc_gen_inverse(h, hinv);
    if (!(V > 0.0) || N < 0 || K < 0 || !(alpha > 0.0)) return GEN_EINVAL;
    double* s = (double*)malloc(sizeof(double) * (size_t)(3 * N + 3));
    double* cs = (double*)malloc(sizeof(double) * (size_t)(2 * N + 2));
    if (!s || !cs) {
        free(s);
        free(cs);
        return GEN_ENOMEM;
    }
    for (int64_t i = 0; i < N; ++i)
        for (int t = 0; t < 3; ++t)
            s[3 * i + t] = hinv[3 * t] * pos[3 * i] + hinv[3 * t + 1] * pos[3 * i + 1] + hinv[3 * t + 2] * pos[3 * i + 2];
    for (int64_t i = 0; i < 3 * N; ++i) F[i] = 0.0;
    for (int j = 0; j < 9; ++j) W[j] = 0.0;
    double Ek = 0.0;
    for (int32_t l = 0; l < K; ++l) {
        const int32_t* ml = m + 3 * l;
        double k[3];
        wave_vector(hinv, ml, k);
        double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        if (kk == 0.0) continue;
        double re = 0.0, im = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double th = 2.0 * M_PI * (ml[0] * s[3 * i] + ml[1] * s[3 * i + 1] + ml[2] * s[3 * i + 2]);
            cs[2 * i] = cos(th);
            cs[2 * i + 1] = sin(th);
            re += q[i] * cs[2 * i];
            im += q[i] * cs[2 * i + 1];
        }
        double g = wl[l] / kk, rho2 = re * re + im * im;
        Ek += (2.0 * M_PI / V) * g * rho2;
        double b = 2.0 * (1.0 / kk + 1.0 / (4.0 * alpha));
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c)
                W[3 * a + c] += (2.0 * M_PI / V) * g * rho2 * ((a == c ? 1.0 : 0.0) - b * k[a] * k[c]);
        for (int64_t i = 0; i < N; ++i) {
            /* Im(e^{-ik.r_i} rho) = cos(th_i) im - sin(th_i) re */
            double imv = cs[2 * i] * im - cs[2 * i + 1] * re;
            double f = -(4.0 * M_PI * q[i] / V) * g * imv;
            for (int t = 0; t < 3; ++t) F[3 * i + t] += f * k[t];
        }
    }
    double q2 = 0.0;
    for (int64_t i = 0; i < N; ++i) q2 += q[i] * q[i];
    E[0] = Ek;
    E[1] = -sqrt(alpha / M_PI) * q2;
    free(s);
    free(cs);
    return GEN_OK;
}

/* The full Ewald k-space sum over the cube |m_j| <= kmax, m != 0. */
int orc_gen_ewald_kspace(int64_t N, const double* pos, const double* q, const double h[9], double alpha,
                         int32_t kmax, double* F, double W[9], double E[2])
{
    double hinv[9];
    if (!(orc_gen_inverse(h, hinv) > 0.0) || kmax < 0) return GEN_EINVAL;
    int64_t side = 2 * (int64_t)kmax + 1, K = side * side * side - 1;
    int32_t* m = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(K > 0 ? K : 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
    if (!m || !w) {
        free(m);
        free(w);
        return GEN_ENOMEM;
    }
    int64_t l = 0;
    for (int32_t a = -kmax; a <= kmax; ++a)
        for (int32_t b = -kmax; b <= kmax; ++b)
            for (int32_t c = -kmax; c <= kmax; ++c) {
                if (a == 0 && b == 0 && c == 0) continue;
                int32_t mm[3] = {a, b, c};
                double k[3];
                wave_vector(hinv, mm, k);
                m[3 * l] = a;
                m[3 * l + 1] = b;
                m[3 * l + 2] = c;
                w[l] = exp(-(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]) / (4.0 * alpha));
                ++l;
            }
    int st = orc_gen_kspace(N, pos, q, h, alpha, (int32_t)K, m, w, F, W, E);
    free(m);
    free(w);
    return st;
}

/* Real space with every image within rc (not only the nearest): sum over pairs i < j and over
 * n in Z^3 of q_i q_j erfc(sqrt(a) |d|)/|d|, d = r_j - r_i + h n, plus the self-image terms
 * (i = j, n != 0) with weight 1/2; forces on both ends, virial sum f d d^T (f = -(dU/dr)/r). */
int orc_gen_ewald_real(int64_t N, const double* pos, const double* q, const double h[9], double alpha, double rc,
                       double* F, double W[9], double* E)
{
    double hinv[9];
    double V = orc_gen_inverse(h, hinv);
    if (!(V > 0.0) || !(rc > 0.0)) return GEN_EINVAL;
    /* image range: |n_j| <= ceil(rc / width_j) + 1 with width_j = V / |a_k x a_l| = 1 / |row j of h^{-1}| */
    int32_t R[3];
    for (int t = 0; t < 3; ++t) {
        double rn = sqrt(hinv[3 * t] * hinv[3 * t] + hinv[3 * t + 1] * hinv[3 * t + 1] + hinv[3 * t + 2] * hinv[3 * t + 2]);
        R[t] = (int32_t)ceil(rc * rn) + 1;
    }
    for (int64_t i = 0; i < 3 * N; ++i) F[i] = 0.0;
    for (int j = 0; j < 9; ++j) W[j] = 0.0;
    double U = 0.0, sa = sqrt(alpha);
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
                        double ec = erfc(sa * r);
                        U += wgt * q[i] * q[j] * ec / r;
                        double f = wgt * q[i] * q[j] * (ec / r2 + 2.0 * sa * exp(-alpha * r2) / (sqrt(M_PI) * r)) / r;
                        for (int t = 0; t < 3; ++t) {
                            F[3 * j + t] += f * d[t];
                            F[3 * i + t] -= f * d[t];
                        }
                        for (int x = 0; x < 3; ++x)
                            for (int y = 0; y < 3; ++y) W[3 * x + y] += f * d[x] * d[y];
                    }
    *E = U;
    return GEN_OK;
}

/* S by the dual (Poisson) sum: (alpha/pi)^{3/2} V sum_n exp(-alpha |h n|^2) - 1. */
double orc_gen_S(const double h[9], double alpha)
{
    double hinv[9];
    double V = orc_gen_inverse(h, hinv);
    if (!(V > 0.0) || !(alpha > 0.0)) return NAN;
    double cut = (60.0 * 0.69314718055994530942 + 50.0) / alpha; /* |h n|^2 beyond this drops out */
    int32_t R[3];
    for (int t = 0; t < 3; ++t) {
        double rn = sqrt(hinv[3 * t] * hinv[3 * t] + hinv[3 * t + 1] * hinv[3 * t + 1] + hinv[3 * t + 2] * hinv[3 * t + 2]);
        R[t] = (int32_t)ceil(sqrt(cut) * rn) + 1;
    }
    double sum = 0.0;
    for (int32_t a = -R[0]; a <= R[0]; ++a)
        for (int32_t b = -R[1]; b <= R[1]; ++b)
            for (int32_t c = -R[2]; c <= R[2]; ++c) {
                double x[3];
                for (int t = 0; t < 3; ++t) x[t] = h[3 * t] * a + h[3 * t + 1] * b + h[3 * t + 2] * c;
                double d2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
                if (d2 <= cut) sum += exp(-alpha * d2);
            }
    return pow(alpha / M_PI, 1.5) * V * sum - 1.0;
}

/* S by the direct sum over m (for the pins): all m with pi^2 m^T G m / alpha <= 60 ln 2 + 50. */
double orc_gen_S_direct(const double h[9], double alpha)
{
    double G[9], hinv[9];
    if (!(orc_gen_inverse(h, hinv) > 0.0)) return NAN;
    orc_gen_metric(h, G);
    double cut = (60.0 * 0.69314718055994530942 + 50.0) * alpha / (M_PI * M_PI);
    /* bounding box of the ellipsoid m^T G m <= cut: |m_j| <= sqrt(cut (G^{-1})_jj), G^{-1} = h^T h */
    int32_t R[3];
    for (int t = 0; t < 3; ++t) {
        double hh = h[t] * h[t] + h[3 + t] * h[3 + t] + h[6 + t] * h[6 + t];
        R[t] = (int32_t)ceil(sqrt(cut * hh)) + 1;
    }
    double sum = 0.0;
    for (int32_t a = -R[0]; a <= R[0]; ++a)
        for (int32_t b = -R[1]; b <= R[1]; ++b)
            for (int32_t c = -R[2]; c <= R[2]; ++c) {
                if (a == 0 && b == 0 && c == 0) continue;
                double mm[3] = {a, b, c}, Q = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) Q += G[3 * i + j] * mm[i] * mm[j];
                Q *= M_PI * M_PI / alpha;
                if (Q <= cut * M_PI * M_PI / alpha) sum += exp(-Q);
            }
    return sum;
}

/* Effective lengths of the proposal: l_j = sqrt(lambda |a_j|^2), |a_j|^2 = sum_i h_ij^2,
 * cos theta_jk = (a_j . a_k) / sqrt(|a_j|^2 |a_k|^2), lambda = max_j (1 + sum_{k != j} |cos|). */
void orc_gen_proposal_lengths(const double h[9], double leff[3])
{
    double g[9];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) g[3 * j + k] = h[j] * h[k] + h[3 + j] * h[3 + k] + h[6 + j] * h[6 + k];
    double lam = 1.0;
    for (int j = 0; j < 3; ++j) {
        double row = 1.0;
        for (int k = 0; k < 3; ++k)
            if (k != j) row = row + fabs(g[3 * j + k] / sqrt(g[3 * j + j] * g[3 * k + k]));
        if (row > lam) lam = row;
    }
    for (int j = 0; j < 3; ++j) leff[j] = sqrt(lam * g[3 * j + j]);
}

/* O(m) = (pi^2/alpha) m^T G m - sum_j c_j m_j^2, summed in a fixed order. */
static double off_part(const double G[9], const double c[3], double co, const int32_t* m)
{
    double q = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) q = q + (G[3 * i + j] * (double)m[i]) * (double)m[j];
    double d = 0.0;
    for (int j = 0; j < 3; ++j) d = d + (c[j] * (double)m[j]) * (double)m[j];
    return co * q - d;
}

/* The general-cell MH sampler: state[P][3] in/out (rows of zeros start from the proposal of this
 * step); S_out = S (dual sum).  Effective lengths 1/sqrt(G_jj) give the diagonal proposal. */
int orc_gen_sample_k_mh(const double h[9], double alpha, int32_t P, uint64_t seed, uint64_t step, int32_t* state,
                        double* S_out)
{
    double G[9], hinv[9];
    if (!(orc_gen_inverse(h, hinv) > 0.0) || P < 0 || !(alpha > 0.0) || (step >> 56) != 0) return GEN_EINVAL;
    orc_gen_metric(h, G);
    double leff[3], c[3];
    orc_gen_proposal_lengths(h, leff);
    for (int t = 0; t < 3; ++t) c[t] = (M_PI * M_PI) / (alpha * (leff[t] * leff[t]));
    int32_t* prop = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(P > 0 ? P : 1));
    if (!prop) return GEN_ENOMEM;
    int st = orc_sample_k(leff, alpha, P, seed, step, prop, NULL);
    double co = (M_PI * M_PI) / alpha;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int32_t l = 0; l < P && st == GEN_OK; ++l) {
        int32_t* m = state + 3 * l;
        const int32_t* mp = prop + 3 * l;
        if (m[0] == 0 && m[1] == 0 && m[2] == 0) {
            for (int t = 0; t < 3; ++t) m[t] = mp[t];
            continue;
        }
        double Om = off_part(G, c, co, m), Op = off_part(G, c, co, mp);
        double d = Om - Op;
        int accept;
        if (d >= 0.0) {
            accept = 1;
        } else if (d < -700.0) {
            accept = 0;
        } else {
            uint32_t ctr[4] = {(uint32_t)l, 0u, (uint32_t)step, (5u << 24) | (uint32_t)((step >> 32) & 0xFFFFFFu)};
            uint32_t w[4];
            orc_philox4x32_10(ctr, key, w);
            double u = (double)((((uint64_t)w[0]) << 21) | (uint64_t)(w[1] >> 11)) * 0x1.0p-53;
            accept = u < orc_exp(d);
        }
        if (accept)
            for (int t = 0; t < 3; ++t) m[t] = mp[t];
    }
    free(prop);
    if (st == GEN_OK && S_out) *S_out = orc_gen_S(h, alpha);
    return st;
}
