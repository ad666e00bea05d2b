/*
 * Oracle for the paper's own frequency-sampling strategies (Sec. 4.3) as variants of the
 * exact sampler of rbe_oracle.c -- TEST INFRASTRUCTURE ONLY (conventions and who may load
 * it: rbe_oracle.c).
 *
 * Offline approach: Gaussian variables z drawn independently of the box, scaled by
 * sqrt(alpha l^2 / (2 pi^2)) and rounded to the nearest integer, per axis; a vector that
 * rounds to m = 0 is drawn again.  The rounding is not corrected, so the sample law is the
 * rounded continuous Gaussian, not the discrete Gaussian of Eq. (probexpression): a bias the
 * paper points out.
 *
 * Online approach: a Metropolis--Hastings chain per frequency slot, started from the previous
 * step's m, whose proposal is the rounded continuous Gaussian (the offline draw of this step)
 * and whose target is the discrete Gaussian exp(-pi^2 m_j^2/(alpha l_j^2)) on Z^3 \ {0}.  The
 * proposal mass of an integer is the Gaussian mass of [m - 1/2, m + 1/2), written with erfc.
 * A slot whose state is m = 0 (no previous step) starts from the exact draw of this step.
 *
 * Every floating-point step that decides an integer here (the logarithm of the polar method,
 * the erfc of the proposal masses, the exponentials of the target) is written out below with
 * separately rounded IEEE operations only (square root and division included), so that a
 * device implementation of the same operations in the same order draws the same m.  These
 * functions are not libm's: the logarithm is the atanh series after a binary reduction, erf
 * its Taylor series on [0, 2] and erfc the Laplace continued fraction beyond, all pinned
 * against libm / SciPy in tests/test_oracle_samplers.py.
 *
 * Random numbers (Philox-4x32-10, key = seed): the offline normals use stream 3, counter
 * (l, d, step_lo, (3 << 24) | step_hi24) for the d-th polar trial of slot l; the MH acceptance
 * uniform uses stream 4, counter (l, 0, step_lo, (4 << 24) | step_hi24).  Uniforms are 53-bit:
 * (w0 << 21 | w1 >> 11) 2^-53.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { SMP_OK = 0, SMP_EINVAL = 1, SMP_ENOMEM = 2, SMP_ESAMPLE = 6 };

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_exp(double x);
int32_t orc_axis_M(double alpha, double ell);
double orc_axis_table(double alpha, double ell, double* w, uint64_t* cum);
int orc_sample_k(const double box[3], double alpha, int32_t P, uint64_t seed, uint64_t step, int32_t* m_out,
                 double* S_out);

#define SMP_MAX_TRIALS (1u << 20) /* polar trials per slot and step */

/* ------------------------------------------------------------------------------ */
/* ln x for positive finite x: x = 2^e f with f in [sqrt(1/2), sqrt(2)) (exact), and
 * ln f = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), s = (f - 1)/(f + 1), |s| <= 0.1716, summed
 * to s^29 in Horner form (the next term is below 2^-70 of the sum); ln x = e ln2_hi +
 * (e ln2_lo + ln f) with ln 2 split into a 32-bit head (e ln2_hi is exact) and a tail. */
static const double SMP_LN2_HI = 0x1.62e42fee00000p-1;
static const double SMP_LN2_LO = 0x1.a39ef35793c76p-33;
static const double SMP_SQRT_HALF = 0x1.6a09e667f3bcdp-1;

double orc_own_log(double x)
{
    int e;
    double f = frexp(x, &e);
    if (f < SMP_SQRT_HALF) {
        f = f * 2.0;
        e = e - 1;
    }
    double s = (f - 1.0) / (f + 1.0);
    double z = s * s;
    double p = 1.0 / 29.0;
    for (int n = 13; n >= 0; --n) p = p * z + 1.0 / (double)(2 * n + 1);
    double lnf = 2.0 * s * p;
    return (double)e * SMP_LN2_HI + ((double)e * SMP_LN2_LO + lnf);
}

/* erf(x) on [0, 2]: the Taylor series sum_n (-1)^n x^(2n+1) / (n! (2n+1)) times 2/sqrt(pi).
 * Term n is t_n = t_{n-1} (-x^2) (1/n), added as t_n (1/(2n+1)), with the reciprocals rounded
 * once (1.0 / n, an IEEE division); the sum stops after the first term whose contribution is
 * below 2^-60 of the running sum (at most 60 terms; 31 at x = 2). */
static const double SMP_TWO_OVER_SQRTPI = 0x1.20dd750429b6dp+0;
static const double SMP_SQRTPI = 0x1.c5bf891b4ef6bp+0;

static double own_erf_series(double x)
{
    double x2 = x * x, t = x, sum = x;
    for (int n = 1; n <= 60; ++n) {
        t = (t * (-x2)) * (1.0 / (double)n);
        double term = t * (1.0 / (double)(2 * n + 1));
        sum = sum + term;
        if (fabs(term) < 0x1.0p-60 * fabs(sum)) break;
    }
    return sum * SMP_TWO_OVER_SQRTPI;
}

/* exp(x) for x <= 0, 0 below -700 (the exponential of rbe_oracle.c). */
static double exp_or_zero(double x)
{
    return x < -700.0 ? 0.0 : orc_exp(x);
}

/* erfc(x) for x >= 0: 1 - erf on [0, 2]; beyond, exp(-x^2)/(sqrt(pi) K) with the continued
 * fraction K = x + (1/2)/(x + 1/(x + (3/2)/(x + ...))) evaluated backwards from depth
 * ceil(10 + 200/x^2) (58 at x = 2, 15 at x = 6: above the depth that reaches 1e-16 relative,
 * 56 and 13); 0 from x = 26 on (erfc(26) < 1e-295). */
double orc_own_erfc(double x)
{
    if (x <= 2.0) return 1.0 - own_erf_series(x);
    if (x >= 26.0) return 0.0;
    double f = x;
    int depth = (int)ceil(10.0 + 200.0 / (x * x));
    for (int n = depth; n >= 1; --n) f = x + (0.5 * (double)n) / f;
    return exp_or_zero(-(x * x)) / (SMP_SQRTPI * f);
}

static double own_erf(double x)
{
    return x <= 2.0 ? own_erf_series(x) : 1.0 - orc_own_erfc(x);
}

/* Gaussian mass of [m - 1/2, m + 1/2) for the standard deviation sigma, with
 * g = 1/(sigma sqrt 2): erf(g/2) at m = 0, (erfc((|m| - 1/2) g) - erfc((|m| + 1/2) g)) / 2
 * otherwise. */
double orc_rounded_gauss_mass(int32_t m, double g)
{
    int32_t a = m < 0 ? -m : m;
    if (a == 0) return own_erf(0.5 * g);
    double lo = ((double)a - 0.5) * g, hi = ((double)a + 0.5) * g;
    return 0.5 * (orc_own_erfc(lo) - orc_own_erfc(hi));
}

/* ------------------------------------------------------------------------------ */
/* One trial of Marsaglia's polar method from Philox call d of slot l: v = 2u - 1 (exact) for
 * two 53-bit uniforms, s = v1^2 + v2^2; on 0 < s < 1 the normals v sqrt(-2 ln s / s). */
static uint64_t u53_bits(uint32_t a, uint32_t b)
{
    return ((uint64_t)a << 21) | (uint64_t)(b >> 11);
}

int orc_polar_pair(uint64_t seed, uint64_t step, uint32_t l, uint32_t d, double z[2])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {l, d, (uint32_t)step, (3u << 24) | (uint32_t)((step >> 32) & 0xFFFFFFu)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    double v1 = 2.0 * ((double)u53_bits(w[0], w[1]) * 0x1.0p-53) - 1.0;
    double v2 = 2.0 * ((double)u53_bits(w[2], w[3]) * 0x1.0p-53) - 1.0;
    double s = v1 * v1 + v2 * v2;
    if (!(s > 0.0 && s < 1.0)) return 0;
    double f = sqrt((-2.0 * orc_own_log(s)) / s);
    z[0] = v1 * f;
    z[1] = v2 * f;
    return 1;
}

/* The offline draw of slot l at this step: three normals (two polar trials that succeed; the
 * second trial's second normal is unused), m_j = rint(sigma_j z_j); m = 0 is drawn again
 * with the following trials. */
static int offline_vector(const double sig[3], uint64_t seed, uint64_t step, uint32_t l, int32_t m[3])
{
    uint32_t d = 0;
    for (;;) {
        double z[3];
        int have = 0;
        while (have < 3) {
            if (d >= SMP_MAX_TRIALS) return SMP_ESAMPLE;
            double pr[2];
            if (orc_polar_pair(seed, step, l, d++, pr)) {
                z[have++] = pr[0];
                if (have < 3) z[have++] = pr[1];
            }
        }
        for (int t = 0; t < 3; ++t) {
            double v = nearbyint(sig[t] * z[t]);
            if (!(fabs(v) <= 1073741824.0)) return SMP_ESAMPLE;
            m[t] = (int32_t)v;
        }
        if (m[0] != 0 || m[1] != 0 || m[2] != 0) return SMP_OK;
    }
}

/* sigma_j = sqrt(alpha/2) l_j / pi: the standard deviation of m_j under exp(-pi^2 m^2/(alpha l^2)) */
static void axis_sigmas(const double box[3], double alpha, double sig[3])
{
    double r = sqrt(alpha * 0.5);
    for (int t = 0; t < 3; ++t) sig[t] = (r * box[t]) / M_PI;
}

/* S = H_x H_y H_z - 1 of the exact sampler's tables (Eq. (S)), for the weights S/P. */
static int tables_S(const double box[3], double alpha, double* S)
{
    double H[3];
    for (int t = 0; t < 3; ++t) {
        int32_t M = orc_axis_M(alpha, box[t]);
        double* w = (double*)malloc(sizeof(double) * (size_t)(2 * M + 1));
        uint64_t* cum = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(2 * M + 1));
        if (!w || !cum) {
            free(w);
            free(cum);
            return SMP_ENOMEM;
        }
        H[t] = orc_axis_table(alpha, box[t], w, cum);
        free(w);
        free(cum);
    }
    *S = H[0] * H[1] * H[2] - 1.0;
    return SMP_OK;
}

static int check_args(const double box[3], double alpha, int32_t P, uint64_t step)
{
    if (P < 0 || !(alpha > 0.0) || (step >> 56) != 0) return SMP_EINVAL;
    for (int t = 0; t < 3; ++t)
        if (!(box[t] > 0.0) || !(box[t] < 1e300)) return SMP_EINVAL;
    return SMP_OK;
}

/* Offline approach (Sec. 4.3): m_out[P][3] and S (the weights stay S/P). */
int orc_sample_k_offline(const double box[3], double alpha, int32_t P, uint64_t seed, uint64_t step,
                         int32_t* m_out, double* S_out)
{
    int st = check_args(box, alpha, P, step);
    if (st != SMP_OK) return st;
    double sig[3];
    axis_sigmas(box, alpha, sig);
    for (int32_t l = 0; l < P; ++l) {
        st = offline_vector(sig, seed, step, (uint32_t)l, m_out + 3 * l);
        if (st != SMP_OK) return st;
    }
    return S_out ? tables_S(box, alpha, S_out) : SMP_OK;
}

/* Online approach (Sec. 4.3): one Metropolis--Hastings step per slot.  state[P][3] holds each
 * slot's m from the previous step (in) and this step's (out); a slot at m = 0 starts from the
 * exact draw of this step.  With c_j = pi^2/(alpha l_j^2), g_j = pi/(sqrt(alpha) l_j), target
 * pi(m) = prod_j exp(-c_j m_j^2) and proposal q(m) = prod_j mass(m_j) (the offline draw, whose
 * redraw of m = 0 conditions both q's alike), the proposal m' is accepted when
 * u prod_j exp(-c_j m_j^2) mass(m'_j) < prod_j exp(-c_j m'_j^2) mass(m_j). */
int orc_sample_k_mh(const double box[3], double alpha, int32_t P, uint64_t seed, uint64_t step, int32_t* state,
                    double* S_out)
{
    int st = check_args(box, alpha, P, step);
    if (st != SMP_OK) return st;
    double sig[3], c[3], g[3];
    axis_sigmas(box, alpha, sig);
    double ra = sqrt(alpha);
    for (int t = 0; t < 3; ++t) {
        c[t] = (M_PI * M_PI) / (alpha * (box[t] * box[t]));
        g[t] = M_PI / (ra * box[t]);
    }
    int32_t* exact = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(P > 0 ? P : 1));
    if (!exact) return SMP_ENOMEM;
    double S = 0.0;
    st = orc_sample_k(box, alpha, P, seed, step, exact, &S);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int32_t l = 0; l < P && st == SMP_OK; ++l) {
        int32_t* m = state + 3 * l;
        if (m[0] == 0 && m[1] == 0 && m[2] == 0) {
            for (int t = 0; t < 3; ++t) m[t] = exact[3 * l + t];
            continue;
        }
        int32_t mp[3];
        st = offline_vector(sig, seed, step, (uint32_t)l, mp);
        if (st != SMP_OK) break;
        uint32_t ctr[4] = {(uint32_t)l, 0u, (uint32_t)step, (4u << 24) | (uint32_t)((step >> 32) & 0xFFFFFFu)};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        double u = (double)u53_bits(w[0], w[1]) * 0x1.0p-53;
        double num = 1.0, den = 1.0;
        for (int t = 0; t < 3; ++t) {
            double a = (double)mp[t], b = (double)m[t];
            num = num * (exp_or_zero(-(c[t] * (a * a))) * orc_rounded_gauss_mass(m[t], g[t]));
            den = den * (exp_or_zero(-(c[t] * (b * b))) * orc_rounded_gauss_mass(mp[t], g[t]));
        }
        if (u * den < num)
            for (int t = 0; t < 3; ++t) m[t] = mp[t];
    }
    free(exact);
    if (st == SMP_OK && S_out) *S_out = S;
    return st;
}
