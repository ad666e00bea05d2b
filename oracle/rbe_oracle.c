/*
 * Oracle for the random batch Ewald (RBE) k-space path -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of what the GPU library computes, written from
 * "A random batch Ewald method for charged particles in the isothermal-isobaric
 * ensemble" (Liang, Tan, Hong, Jin, Xu, Li).  Loops run in index order; there is no
 * blocking, fusion or reordering beyond what the formulas state.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load this
 * code.  It shares no source with the CUDA library.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (see oracle/__init__.py).
 * -ffp-contract=off keeps every multiply and add separately rounded, which the
 * sampler's table (bit-exact against the device) relies on.
 *
 * Conventions (Sec. 4.1): Gaussian units, U = 1/2 sum' q_i q_j / |r_ij + h n|.
 * Box h = diag(l_x, l_y, l_z), V = l_x l_y l_z, k = 2 pi m / l componentwise.
 * Virials are returned in energy units (W = V * pressure tensor), row-major 3x3.
 *
 * Pins (tests/test_oracle_*.py): Philox words against an independent library
 * implementation; the exponential against libm; per-axis marginals of the sampler
 * against the exact probability mass (chi-square); H against the Poisson-summation
 * identity of Eq. (psf); the NaCl and CsCl Madelung constants; alpha-independence;
 * a brute-force image sum; finite-difference volume/length derivatives of the Ewald
 * energy; zero net force per sampled k; the weighted full-k mode against the plain
 * Ewald sum; Monte-Carlo unbiasedness with the variances of Proposition 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ESAMPLE = 6 };

/* ------------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11).  Ten rounds of the 4x32 S-box: two 32x32->64 multiplications by
 * the constants 0xD2511F53 and 0xCD9E8D57, whose high halves are xored with the
 * other two words and the round key; the key advances by the Weyl increments
 * 0x9E3779B9 and 0xBB67AE85 between rounds. The paper of the method specifies no
 * generator; this one is a design choice shared (by specification, not by code)
 * with the device sampler. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* A uniform double in [0, 1) from 53 bits: the 32 bits of a and the top 21 of b. */
double orc_uniform53(uint32_t a, uint32_t b)
{
    uint64_t bits = ((uint64_t)a << 21) | (uint64_t)(b >> 11);
    return (double)bits * 0x1.0p-53;
}

/* Counter layout for the k-sampling stream (stream id 0):
 * (sample index l, 2*attempt + half, step bits 0..31, (stream << 24) | step bits 32..55).
 * Two Philox calls (half = 0, 1) give 8 words; words (0,1), (2,3), (4,5) make the
 * x, y and z uniforms. */
static void sample_uniforms(uint64_t seed, uint64_t step, uint32_t l, uint32_t attempt, uint64_t U[3])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[8];
    for (uint32_t half = 0; half < 2; ++half) {
        uint32_t ctr[4] = {l, 2u * attempt + half, (uint32_t)step,
                           (0u << 24) | (uint32_t)((step >> 32) & 0xFFFFFFu)};
        orc_philox4x32_10(ctr, key, w + 4 * half);
    }
    U[0] = ((uint64_t)w[0] << 21) | (uint64_t)(w[1] >> 11);
    U[1] = ((uint64_t)w[2] << 21) | (uint64_t)(w[3] >> 11);
    U[2] = ((uint64_t)w[4] << 21) | (uint64_t)(w[5] >> 11);
}

/* ------------------------------------------------------------------------------ */
/* exp(x) for x <= 0 by Cody--Waite reduction and a Taylor polynomial.
 * x = n ln2 + r with n = rint(x / ln2) and |r| <= ln2/2; ln2 is split into a head of
 * 32 significant bits (so n * head is exact for |n| < 2^21) and a tail.  e^r is the
 * Taylor series to degree 13 in Horner form (truncation below 2^-56 relative), and
 * the result is scaled by 2^n.  Every operation is a separately rounded IEEE double
 * operation, so a device implementation that performs the same operations in the
 * same order gets the same bits.  Used only for the sampler's weight table. */
static const double ORC_INV_LN2 = 0x1.71547652b82fep+0;
static const double ORC_LN2_HI = 0x1.62e42fee00000p-1;
static const double ORC_LN2_LO = 0x1.a39ef35793c76p-33;
static const double ORC_INV_FACT[14] = {
    0x1.0000000000000p+0, 0x1.0000000000000p+0, 0x1.0000000000000p-1, 0x1.5555555555555p-3,
    0x1.5555555555555p-5, 0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13,
    0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
    0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};

double orc_exp(double x)
{
    if (x > 0.0 || x < -700.0 || x != x) return NAN; /* the table needs only [-700, 0] */
    double n = nearbyint(x * ORC_INV_LN2);
    double r = (x - n * ORC_LN2_HI) - n * ORC_LN2_LO;
    double p = ORC_INV_FACT[13];
    for (int j = 12; j >= 0; --j) p = p * r + ORC_INV_FACT[j];
    return ldexp(p, (int)n);
}

/* ------------------------------------------------------------------------------ */
/* Per-axis discrete Gaussian (Sec. 4.2 Eqs. (S), (psf), (probexpression); App. C item 1:
 * for a rectangular box the three components of m are independent).
 * P(m) is proportional to exp(-|k|^2/(4 alpha)) = prod_theta exp(-c_theta m_theta^2)
 * with c_theta = pi^2 / (alpha l_theta^2).
 * The table keeps |m| <= M with M = ceil(sqrt(60 ln2 / c)), i.e. it drops terms below
 * 2^-60 of the peak.  w_j = exp(-c (j - M)^2), j = 0..2M, computed once per |m| so the
 * table is exactly symmetric.  The weights are held as integers W_j = rint(w_j 2^sh) with
 * sh = 62 - bitlength(2M + 1), so that their sum fits 63 bits; the cumulative sums
 * C_j = W_0 + ... + W_j are exact, and H = C_2M 2^-sh (Eq. (psf)). */
int32_t orc_axis_M(double alpha, double ell)
{
    double c = (M_PI * M_PI) / (alpha * (ell * ell));
    double M = ceil(sqrt((60.0 * 0.69314718055994530942) / c));
    return (int32_t)M;
}

int orc_axis_shift(int32_t M)
{
    uint64_t n = (uint64_t)(2 * M + 1);
    int bits = 0;
    while (n) { ++bits; n >>= 1; }
    return 62 - bits;
}

/* Writes w[2M+1] (the weights), cum[2M+1] (the integer cumulative sums) and returns H. */
double orc_axis_table(double alpha, double ell, double* w, uint64_t* cum)
{
    double c = (M_PI * M_PI) / (alpha * (ell * ell));
    int32_t M = orc_axis_M(alpha, ell);
    int sh = orc_axis_shift(M);
    for (int32_t a = 0; a <= M; ++a) {
        double v = orc_exp(-(c * ((double)a * (double)a)));
        w[M + a] = v;
        w[M - a] = v;
    }
    uint64_t acc = 0;
    for (int32_t j = 0; j <= 2 * M; ++j) {
        acc += (uint64_t)llrint(ldexp(w[j], sh));
        cum[j] = acc;
    }
    return ldexp((double)cum[2 * M], -sh);
}

/* Inverse CDF on the integer table: with U the 53-bit uniform integer,
 * T = floor(U * C_2M / 2^53), m = (smallest j with T < C_j) - M. */
static int32_t axis_draw(const uint64_t* cum, int32_t M, uint64_t U)
{
    unsigned __int128 prod = (unsigned __int128)U * (unsigned __int128)cum[2 * M];
    uint64_t T = (uint64_t)(prod >> 53);
    for (int32_t j = 0; j <= 2 * M; ++j)
        if (T < cum[j]) return j - M;
    return M; /* unreachable: T < C_2M */
}

#define ORC_MAX_ATTEMPTS (1u << 20)

/* Draws P i.i.d. frequencies m_l in Z^3 \ {0} from the discrete Gaussian of
 * Eq. (probexpression), per axis by inverse CDF, redrawing (attempt + 1) whenever all
 * three components are zero.  Writes m_out[P][3] and S = H_x H_y H_z - 1 (Eq. (S)). */
int orc_sample_k(const double box[3], double alpha, int32_t P, uint64_t seed, uint64_t step,
                 int32_t* m_out, double* S_out)
{
    if (P < 0 || !(alpha > 0.0) || (step >> 56) != 0) return ORC_EINVAL;
    double H[3];
    uint64_t* cum[3] = {NULL, NULL, NULL};
    int32_t M[3];
    for (int t = 0; t < 3; ++t) {
        if (!(box[t] > 0.0)) return ORC_EINVAL;
        M[t] = orc_axis_M(alpha, box[t]);
    }
    int status = ORC_OK;
    for (int t = 0; t < 3; ++t) {
        double* w = (double*)malloc(sizeof(double) * (size_t)(2 * M[t] + 1));
        cum[t] = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(2 * M[t] + 1));
        if (!w || !cum[t]) {
            free(w);
            for (int u = 0; u <= t; ++u) free(cum[u]);
            return ORC_ENOMEM;
        }
        H[t] = orc_axis_table(alpha, box[t], w, cum[t]);
        free(w);
    }
    for (int32_t l = 0; l < P && status == ORC_OK; ++l) {
        uint32_t attempt = 0;
        for (;;) {
            if (attempt >= ORC_MAX_ATTEMPTS) { status = ORC_ESAMPLE; break; }
            uint64_t U[3];
            sample_uniforms(seed, step, (uint32_t)l, attempt, U);
            int32_t m[3];
            for (int t = 0; t < 3; ++t) m[t] = axis_draw(cum[t], M[t], U[t]);
            if (m[0] != 0 || m[1] != 0 || m[2] != 0) {
                m_out[3 * l + 0] = m[0];
                m_out[3 * l + 1] = m[1];
                m_out[3 * l + 2] = m[2];
                break;
            }
            ++attempt;
        }
    }
    if (S_out) *S_out = H[0] * H[1] * H[2] - 1.0;
    for (int t = 0; t < 3; ++t) free(cum[t]);
    return status;
}

/* ------------------------------------------------------------------------------ */
/* Exact target: the Ewald k-space sum over the cube |m_theta| <= kmax, m != 0.
 *   E_k  = (2 pi / V) sum_k exp(-|k|^2/4a)/|k|^2 |rho(k)|^2                    Eq. (U1fourier)
 *   E_self = -sqrt(a/pi) sum_i q_i^2                                           Eq. (U1fourier)
 *   F_i = -sum_k (4 pi q_i k / (V |k|^2)) exp(-|k|^2/4a) Im(e^{-ik.r_i} rho(k)) Eq. (force)
 *   W   = (2 pi / V) sum_k |rho|^2/|k|^2 exp(-|k|^2/4a) [I - 2(1/|k|^2 + 1/4a) k k]
 *                                                    App. C Eq. (pressuretensorflexible)
 * rho(k) = sum_i q_i e^{i k.r_i} (Sec. 4.1). The phase k.r_i is formed directly. */
int orc_ewald_kspace(int64_t N, const double* pos, const double* q, const double box[3],
                     double alpha, int32_t kmax, double* F, double W[9], double E[2])
{
    if (N < 0 || kmax < 0 || !(alpha > 0.0)) return ORC_EINVAL;
    for (int t = 0; t < 3; ++t) if (!(box[t] > 0.0)) return ORC_EINVAL;
    double V = box[0] * box[1] * box[2];
    double* cs = (double*)malloc(sizeof(double) * (size_t)(2 * N + 2));
    if (!cs) return ORC_ENOMEM;
    for (int64_t i = 0; i < 3 * N; ++i) F[i] = 0.0;
    for (int j = 0; j < 9; ++j) W[j] = 0.0;
    double Ek = 0.0;
    for (int32_t mx = -kmax; mx <= kmax; ++mx)
    for (int32_t my = -kmax; my <= kmax; ++my)
    for (int32_t mz = -kmax; mz <= kmax; ++mz) {
        if (mx == 0 && my == 0 && mz == 0) continue;
        double k[3] = {2.0 * M_PI * mx / box[0], 2.0 * M_PI * my / box[1], 2.0 * M_PI * mz / box[2]};
        double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double g = exp(-kk / (4.0 * alpha)) / kk;
        double re = 0.0, im = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double th = k[0] * pos[3 * i] + k[1] * pos[3 * i + 1] + k[2] * pos[3 * i + 2];
            cs[2 * i] = cos(th);
            cs[2 * i + 1] = sin(th);
            re += q[i] * cs[2 * i];
            im += q[i] * cs[2 * i + 1];
        }
        double rho2 = re * re + im * im;
        Ek += (2.0 * M_PI / V) * g * rho2;
        for (int64_t i = 0; i < N; ++i) {
            /* Im(e^{-i th} rho) = cos(th) Im rho - sin(th) Re rho */
            double imt = cs[2 * i] * im - cs[2 * i + 1] * re;
            double f = -(4.0 * M_PI * q[i] / V) * g * imt;
            F[3 * i] += f * k[0];
            F[3 * i + 1] += f * k[1];
            F[3 * i + 2] += f * k[2];
        }
        double b = 2.0 * (1.0 / kk + 1.0 / (4.0 * alpha));
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c)
                W[3 * a + c] += (2.0 * M_PI / V) * g * rho2 * ((a == c ? 1.0 : 0.0) - b * k[a] * k[c]);
    }
    double q2 = 0.0;
    for (int64_t i = 0; i < N; ++i) q2 += q[i] * q[i];
    E[0] = Ek;
    E[1] = -sqrt(alpha / M_PI) * q2;
    free(cs);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------ */
/* The RBE estimators on a given batch m[P][3] (Sec. 4.2 Eqs. (appforce), (apppress);
 * App. C for the tensor), with a per-frequency weight w_l in place of
 * exp(-|k|^2/4a).  The method uses w_l = S/P for every l; passing every m of the cube
 * with w = exp(-|k|^2/4a) recovers the Ewald sum above.
 *   rho_l = sum_i q_i e^{i k_l.r_i}
 *   F_i   = -sum_l w_l (4 pi q_i k_l / (V |k_l|^2)) Im(e^{-i k_l.r_i} rho_l)
 *   W     = (2 pi / V) sum_l w_l |rho_l|^2/|k_l|^2 [I - 2(1/|k_l|^2 + 1/4a) k_l k_l]
 *   E_k   = (2 pi / V) sum_l w_l |rho_l|^2/|k_l|^2 ;  E_self as above.
 * rho (2P doubles, interleaved re/im) may be NULL.
 * Built with -fopenmp (the all-cores timing build), the rho loop runs its frequencies and
 * the force loop its particles on several threads; each iteration's sums keep the index
 * order above, so both builds return the same bits. */
static int rbe_check(int64_t N, const double box[3], double alpha, int32_t P, const int32_t* m)
{
    if (N < 0 || P < 0 || !(alpha > 0.0)) return ORC_EINVAL;
    for (int t = 0; t < 3; ++t) if (!(box[t] > 0.0)) return ORC_EINVAL;
    for (int32_t l = 0; l < P; ++l)
        if (m[3 * l] == 0 && m[3 * l + 1] == 0 && m[3 * l + 2] == 0) return ORC_EINVAL;
    return ORC_OK;
}

/* rho_l = sum_i q_i e^{i k_l.r_i}, rr[2l] = Re, rr[2l+1] = Im (Sec. 4.1). */
static void rbe_rho(int64_t N, const double* pos, const double* q, const double box[3], int32_t P,
                    const int32_t* m, double* rr)
{
#pragma omp parallel for schedule(static)
    for (int32_t l = 0; l < P; ++l) {
        double k[3] = {2.0 * M_PI * m[3 * l] / box[0], 2.0 * M_PI * m[3 * l + 1] / box[1],
                       2.0 * M_PI * m[3 * l + 2] / box[2]};
        double re = 0.0, im = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double th = k[0] * pos[3 * i] + k[1] * pos[3 * i + 1] + k[2] * pos[3 * i + 2];
            re += q[i] * cos(th);
            im += q[i] * sin(th);
        }
        rr[2 * l] = re;
        rr[2 * l + 1] = im;
    }
}

/* F_i = -sum_l w_l (4 pi q_i k_l / (V |k_l|^2)) Im(e^{-i k_l.r_i} rho_l) for one particle
 * (Eq. (appforce)). */
static void rbe_force_one(const double* r, double qi, const double box[3], double V, int32_t P,
                          const int32_t* m, const double* wl, const double* rr, double f[3])
{
    f[0] = f[1] = f[2] = 0.0;
    for (int32_t l = 0; l < P; ++l) {
        double k[3] = {2.0 * M_PI * m[3 * l] / box[0], 2.0 * M_PI * m[3 * l + 1] / box[1],
                       2.0 * M_PI * m[3 * l + 2] / box[2]};
        double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double th = k[0] * r[0] + k[1] * r[1] + k[2] * r[2];
        double imt = cos(th) * rr[2 * l + 1] - sin(th) * rr[2 * l];
        double s = -wl[l] * (4.0 * M_PI * qi / (V * kk)) * imt;
        f[0] += s * k[0];
        f[1] += s * k[1];
        f[2] += s * k[2];
    }
}

/* W (App. C) and E_k, E_self from rho (Eqs. (apppress), (U1fourier)). */
static void rbe_virial_energy(int64_t N, const double* q, const double box[3], double alpha, int32_t P,
                              const int32_t* m, const double* wl, const double* rr, double W[9], double E[2])
{
    double V = box[0] * box[1] * box[2];
    for (int j = 0; j < 9; ++j) W[j] = 0.0;
    double Ek = 0.0;
    for (int32_t l = 0; l < P; ++l) {
        double k[3] = {2.0 * M_PI * m[3 * l] / box[0], 2.0 * M_PI * m[3 * l + 1] / box[1],
                       2.0 * M_PI * m[3 * l + 2] / box[2]};
        double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double rho2 = rr[2 * l] * rr[2 * l] + rr[2 * l + 1] * rr[2 * l + 1];
        double e = (2.0 * M_PI / V) * wl[l] * rho2 / kk;
        Ek += e;
        double b = 2.0 * (1.0 / kk + 1.0 / (4.0 * alpha));
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c)
                W[3 * a + c] += e * ((a == c ? 1.0 : 0.0) - b * k[a] * k[c]);
    }
    double q2 = 0.0;
    for (int64_t i = 0; i < N; ++i) q2 += q[i] * q[i];
    E[0] = Ek;
    E[1] = -sqrt(alpha / M_PI) * q2;
}

int orc_rbe_kspace(int64_t N, const double* pos, const double* q, const double box[3],
                   double alpha, int32_t P, const int32_t* m, const double* wl,
                   double* F, double W[9], double E[2], double* rho)
{
    int st = rbe_check(N, box, alpha, P, m);
    if (st != ORC_OK) return st;
    double V = box[0] * box[1] * box[2];
    double* rr = (double*)malloc(sizeof(double) * (size_t)(2 * P + 2));
    if (!rr) return ORC_ENOMEM;
    rbe_rho(N, pos, q, box, P, m, rr);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) rbe_force_one(pos + 3 * i, q[i], box, V, P, m, wl, rr, F + 3 * i);
    rbe_virial_energy(N, q, box, alpha, P, m, wl, rr, W, E);
    if (rho) for (int32_t l = 0; l < 2 * P; ++l) rho[l] = rr[l];
    free(rr);
    return ORC_OK;
}

/* The same estimators with the forces of listed particles only: rho over all N particles,
 * F_sub[j] = F_{idx[j]} (each row the bits orc_rbe_kspace gives for that particle), W and E
 * as above.  For the largest workloads, where the forces of every particle would double a
 * long oracle run, the forces are compared on a seeded subset. */
int orc_rbe_kspace_subset(int64_t N, const double* pos, const double* q, const double box[3],
                          double alpha, int32_t P, const int32_t* m, const double* wl,
                          int64_t n_sub, const int64_t* idx, double* F_sub, double W[9], double E[2],
                          double* rho)
{
    int st = rbe_check(N, box, alpha, P, m);
    if (st != ORC_OK) return st;
    if (n_sub < 0) return ORC_EINVAL;
    for (int64_t j = 0; j < n_sub; ++j) if (idx[j] < 0 || idx[j] >= N) return ORC_EINVAL;
    double V = box[0] * box[1] * box[2];
    double* rr = (double*)malloc(sizeof(double) * (size_t)(2 * P + 2));
    if (!rr) return ORC_ENOMEM;
    rbe_rho(N, pos, q, box, P, m, rr);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n_sub; ++j)
        rbe_force_one(pos + 3 * idx[j], q[idx[j]], box, V, P, m, wl, rr, F_sub + 3 * j);
    rbe_virial_energy(N, q, box, alpha, P, m, wl, rr, W, E);
    if (rho) for (int32_t l = 0; l < 2 * P; ++l) rho[l] = rr[l];
    free(rr);
    return ORC_OK;
}

/* RBE on one snapshot: sample (orc_sample_k) and evaluate with w_l = S/P (Eq. (appforce)). */
int orc_rbe_snapshot(int64_t N, const double* pos, const double* q, const double box[3],
                     double alpha, int32_t P, uint64_t seed, uint64_t step,
                     double* F, double W[9], double E[2], int32_t* m_out, double* S_out)
{
    if (P < 1) return ORC_EINVAL;
    double S = 0.0;
    int st = orc_sample_k(box, alpha, P, seed, step, m_out, &S);
    if (st != ORC_OK) return st;
    double* wl = (double*)malloc(sizeof(double) * (size_t)P);
    if (!wl) return ORC_ENOMEM;
    for (int32_t l = 0; l < P; ++l) wl[l] = S / (double)P;
    st = orc_rbe_kspace(N, pos, q, box, alpha, P, m_out, wl, F, W, E, NULL);
    free(wl);
    if (S_out) *S_out = S;
    return st;
}

/* ------------------------------------------------------------------------------ */
/* Real-space part with the nearest image only (Sec. 4.1 Eqs. (U2), (force); Sec. 4.2
 * uses the nearest image within the cutoff rc <= min(l)/2).
 *   E_r = sum_{i<j, r<rc} q_i q_j erfc(sqrt(a) r)/r
 *   G(r) = erfc(sqrt(a) r)/r^2 + 2 sqrt(a) exp(-a r^2)/(sqrt(pi) r)
 *   with d = r_j - r_i (nearest image): force on j is q_i q_j G(r) d/r, on i the negative.
 *   W_r = sum_{i<j} q_i q_j G(r)/r d (x) d, which is -l_theta dE_r/dl_theta at fixed s
 *   on the diagonal (the derivative -dU_2/dV at fixed s, Sec. 4.1, taken directly). */
int orc_ewald_real(int64_t N, const double* pos, const double* q, const double box[3],
                   double alpha, double rc, double* F, double W[9], double* E)
{
    if (N < 0 || !(alpha > 0.0) || !(rc > 0.0)) return ORC_EINVAL;
    for (int t = 0; t < 3; ++t)
        if (!(box[t] > 0.0) || rc > 0.5 * box[t]) return ORC_EINVAL;
    for (int64_t i = 0; i < 3 * N; ++i) F[i] = 0.0;
    for (int j = 0; j < 9; ++j) W[j] = 0.0;
    double sa = sqrt(alpha);
    double Er = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        for (int64_t j = i + 1; j < N; ++j) {
            double d[3];
            for (int t = 0; t < 3; ++t) {
                double x = pos[3 * j + t] - pos[3 * i + t];
                d[t] = x - box[t] * nearbyint(x / box[t]);
            }
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double r = sqrt(r2);
            if (!(r < rc)) continue;
            double qq = q[i] * q[j];
            double ec = erfc(sa * r);
            Er += qq * ec / r;
            double G = ec / r2 + 2.0 * sa * exp(-alpha * r2) / (sqrt(M_PI) * r);
            double f = qq * G / r;
            for (int t = 0; t < 3; ++t) {
                F[3 * j + t] += f * d[t];
                F[3 * i + t] -= f * d[t];
            }
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) W[3 * a + c] += f * d[a] * d[c];
        }
    }
    *E = Er;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------ */
/* Brute-force Coulomb energy of the periodic system: 1/2 sum over image cells
 * n with |n| <= R (a sphere of whole cells), sum' q_i q_j / |r_j - r_i + h n| (Eq. (energy)).
 * For a neutral cell with zero dipole the R -> infinity limit equals the Ewald energy. */
double orc_direct_sum(int64_t N, const double* pos, const double* q, const double box[3], int32_t R)
{
    double E = 0.0;
    for (int32_t nx = -R; nx <= R; ++nx)
    for (int32_t ny = -R; ny <= R; ++ny)
    for (int32_t nz = -R; nz <= R; ++nz) {
        if (nx * nx + ny * ny + nz * nz > R * R) continue;
        double sh[3] = {nx * box[0], ny * box[1], nz * box[2]};
        for (int64_t i = 0; i < N; ++i)
            for (int64_t j = 0; j < N; ++j) {
                if (i == j && nx == 0 && ny == 0 && nz == 0) continue;
                double dx = pos[3 * j] - pos[3 * i] + sh[0];
                double dy = pos[3 * j + 1] - pos[3 * i + 1] + sh[1];
                double dz = pos[3 * j + 2] - pos[3 * i + 2] + sh[2];
                E += 0.5 * q[i] * q[j] / sqrt(dx * dx + dy * dy + dz * dz);
            }
    }
    return E;
}
