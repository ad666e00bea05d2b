// The paper's own frequency-sampling strategies (Sec. 4.3) as variants of the exact sampler:
//   offline  Gaussian z independent of the box, m_j = rint(z_j sqrt(alpha l_j^2 / (2 pi^2))),
//            a vector that rounds to m = 0 drawn again; the weights stay S/P, so the rounding
//            is a systematic bias (the paper says so)
//   online   one Metropolis--Hastings step per frequency slot from the previous step's m, with
//            the rounded continuous Gaussian (the offline draw) as an independence proposal and
//            the discrete Gaussian exp(-pi^2 m_j^2/(alpha l_j^2)) on Z^3 \ {0} as the target; the
//            proposal mass of an integer is the Gaussian mass of [m - 1/2, m + 1/2)
// Every floating-point step that decides an integer (the logarithm of the polar method, the
// erfc of the proposal masses, the exponentials of the target) is a separately rounded IEEE
// operation written out here, so the draws are the same bits on any conforming machine: the
// logarithm is the atanh series after a binary reduction, erf its Taylor series on [0, 2] and
// erfc the Laplace continued fraction beyond, the exponential the tables' own (table_exp).
// Random numbers: Philox-4x32-10 with the context's key; the offline normals on stream 3,
// counter (l, d, step_lo, (3 << 24) | step_hi24) for the d-th polar trial of slot l; the MH
// acceptance uniform on stream 4, counter (l, 0, step_lo, (4 << 24) | step_hi24).
#pragma once

#include "rbe_device.cuh"

namespace rbe {

enum SamplerMode { kSamplerExact = 0, kSamplerOffline = 1, kSamplerMH = 2 };
constexpr uint32_t kMaxPolarTrials = 1u << 20;  // polar trials per slot and step

// ln x for positive finite x: x = 2^e f, f in [sqrt(1/2), sqrt(2)) (exact); ln f = 2 atanh(s),
// s = (f - 1)/(f + 1), summed to s^29 in Horner form; ln x = e ln2_hi + (e ln2_lo + ln f).
__device__ __forceinline__ double smp_log(double x)
{
    const double ln2_hi = 0x1.62e42fee00000p-1;
    const double ln2_lo = 0x1.a39ef35793c76p-33;
    int e;
    double f = frexp(x, &e);
    if (f < 0x1.6a09e667f3bcdp-1) {
        f = __dmul_rn(f, 2.0);
        e = e - 1;
    }
    const double s = __ddiv_rn(__dsub_rn(f, 1.0), __dadd_rn(f, 1.0));
    const double z = __dmul_rn(s, s);
    double p = __ddiv_rn(1.0, 29.0);
    for (int n = 13; n >= 0; --n) p = __dadd_rn(__dmul_rn(p, z), __ddiv_rn(1.0, (double)(2 * n + 1)));
    const double lnf = __dmul_rn(__dmul_rn(2.0, s), p);
    const double ed = (double)e;
    return __dadd_rn(__dmul_rn(ed, ln2_hi), __dadd_rn(__dmul_rn(ed, ln2_lo), lnf));
}

// exp(x) for x <= 0, 0 below -700.
__device__ __forceinline__ double smp_exp0(double x)
{
    return x < -700.0 ? 0.0 : table_exp(x);
}

// erf on [0, 2]: sum_n (-1)^n x^(2n+1) / (n! (2n+1)) times 2/sqrt(pi), 60 terms.
__device__ __forceinline__ double smp_erf_series(double x)
{
    const double x2 = __dmul_rn(x, x);
    double t = x, sum = x;
    for (int n = 1; n <= 60; ++n) {
        t = __ddiv_rn(__dmul_rn(t, -x2), (double)n);
        sum = __dadd_rn(sum, __ddiv_rn(t, (double)(2 * n + 1)));
    }
    return __dmul_rn(sum, 0x1.20dd750429b6dp+0);
}

// erfc for x >= 0: 1 - erf on [0, 2], exp(-x^2)/(sqrt(pi) K) beyond with the continued
// fraction K = x + (1/2)/(x + 1/(x + (3/2)/(x + ...))) from depth 80, 0 from 26 on.
__device__ __forceinline__ double smp_erfc(double x)
{
    if (x <= 2.0) return __dsub_rn(1.0, smp_erf_series(x));
    if (x >= 26.0) return 0.0;
    double f = x;
    for (int n = 80; n >= 1; --n) f = __dadd_rn(x, __ddiv_rn(__dmul_rn(0.5, (double)n), f));
    return __ddiv_rn(smp_exp0(-__dmul_rn(x, x)), __dmul_rn(0x1.c5bf891b4ef6bp+0, f));
}

// Gaussian mass of [m - 1/2, m + 1/2) with g = 1/(sigma sqrt 2).
__device__ __forceinline__ double smp_mass(int m, double g)
{
    const int a = m < 0 ? -m : m;
    if (a == 0) {
        const double x = __dmul_rn(0.5, g);
        return x <= 2.0 ? smp_erf_series(x) : __dsub_rn(1.0, smp_erfc(x));
    }
    const double lo = __dmul_rn(__dsub_rn((double)a, 0.5), g), hi = __dmul_rn(__dadd_rn((double)a, 0.5), g);
    return __dmul_rn(0.5, __dsub_rn(smp_erfc(lo), smp_erfc(hi)));
}

__device__ __forceinline__ double smp_u53(uint32_t a, uint32_t b)
{
    return (double)(((unsigned long long)a << 21) | (unsigned long long)(b >> 11)) * 0x1.0p-53;
}

// One polar trial (Philox call d of slot l): v = 2u - 1, s = v1^2 + v2^2; on 0 < s < 1 the
// normals v sqrt(-2 ln s / s).
__device__ __forceinline__ bool smp_polar(uint32_t k0, uint32_t k1, uint32_t c2, uint32_t c3s, int l, uint32_t d,
                                          double& z0, double& z1)
{
    const uint4 w = philox4x32_10(make_uint4((uint32_t)l, d, c2, c3s), k0, k1);
    const double v1 = __dsub_rn(__dmul_rn(2.0, smp_u53(w.x, w.y)), 1.0);
    const double v2 = __dsub_rn(__dmul_rn(2.0, smp_u53(w.z, w.w)), 1.0);
    const double s = __dadd_rn(__dmul_rn(v1, v1), __dmul_rn(v2, v2));
    if (!(s > 0.0 && s < 1.0)) return false;
    const double f = __dsqrt_rn(__ddiv_rn(__dmul_rn(-2.0, smp_log(s)), s));
    z0 = __dmul_rn(v1, f);
    z1 = __dmul_rn(v2, f);
    return true;
}

// The offline draw of slot l: three normals from polar trials (the second trial's second
// normal unused), m_j = rint(sigma_j z_j), drawn again while m = 0.  False when the trials
// run out or a component leaves +-2^30.
__device__ __forceinline__ bool smp_offline(const double sig[3], uint32_t k0, uint32_t k1, uint32_t c2, uint32_t c3,
                                            int l, int4& m)
{
    const uint32_t c3s = (3u << 24) | c3;
    uint32_t d = 0;
    for (;;) {
        double z[3];
        int have = 0;
        while (have < 3) {
            if (d >= kMaxPolarTrials) return false;
            double a, b;
            if (smp_polar(k0, k1, c2, c3s, l, d++, a, b)) {
                z[have++] = a;
                if (have < 3) z[have++] = b;
            }
        }
        int v[3];
        for (int t = 0; t < 3; ++t) {
            const double r = rint(__dmul_rn(sig[t], z[t]));
            if (!(fabs(r) <= 1073741824.0)) return false;
            v[t] = (int)r;
        }
        if (v[0] != 0 || v[1] != 0 || v[2] != 0) {
            m = make_int4(v[0], v[1], v[2], 0);
            return true;
        }
    }
}

// The exact draw of slot l (the inverse CDF of sample_body, on the tables in global memory).
__device__ __forceinline__ bool smp_exact(const unsigned long long* __restrict__ cum, int cap,
                                          const KState* __restrict__ ks, uint32_t k0, uint32_t k1, uint32_t c2,
                                          uint32_t c3, int l, int4& m)
{
    const unsigned long long* tx = cum;
    const unsigned long long* ty = cum + cap;
    const unsigned long long* tz = cum + 2 * (size_t)cap;
    const int Mx = ks->M[0], My = ks->M[1], Mz = ks->M[2];
    const unsigned long long Cx = tx[2 * Mx], Cy = ty[2 * My], Cz = tz[2 * Mz];
    for (uint32_t attempt = 0; attempt < kMaxAttempts; ++attempt) {
        const uint4 w0 = philox4x32_10(make_uint4((uint32_t)l, 2u * attempt, c2, c3), k0, k1);
        const uint4 w1 = philox4x32_10(make_uint4((uint32_t)l, 2u * attempt + 1u, c2, c3), k0, k1);
        m.x = inverse_cdf_int(tx, Mx, scaled_target(((unsigned long long)w0.x << 21) | (w0.y >> 11), Cx));
        m.y = inverse_cdf_int(ty, My, scaled_target(((unsigned long long)w0.z << 21) | (w0.w >> 11), Cy));
        m.z = inverse_cdf_int(tz, Mz, scaled_target(((unsigned long long)w1.x << 21) | (w1.y >> 11), Cz));
        m.w = 0;
        if (m.x != 0 || m.y != 0 || m.z != 0) return true;
    }
    return false;
}

// Slots lbase + threadIdx.x of the offline or MH sampler; chain[P] holds the MH state (m = 0:
// start from the exact draw).  Weights as the exact sampler's (force slots [0, Pf), pressure
// slots [Pf, P)).
__device__ __forceinline__ void sample_variant_body(int lbase, uint64_t seed, uint64_t step_arg,
                                                    const unsigned long long* __restrict__ step_dev, int P, int Pf,
                                                    const unsigned long long* __restrict__ cum, int cap,
                                                    const KState* __restrict__ ks, int mode, int4* __restrict__ chain,
                                                    int4* __restrict__ m_out, double* __restrict__ w_out,
                                                    unsigned* __restrict__ status)
{
    pdl_trigger();
    const int l = lbase + (int)threadIdx.x;
    if (l >= P) return;
    const uint64_t step = step_dev ? *step_dev : step_arg;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t c2 = (uint32_t)step, c3 = (uint32_t)((step >> 32) & 0xFFFFFFu);
    const double alpha = ks->alpha;
    double sig[3];
    const double ra2 = __dsqrt_rn(__dmul_rn(alpha, 0.5));
    for (int t = 0; t < 3; ++t) sig[t] = __ddiv_rn(__dmul_rn(ra2, ks->L[t]), kPi);
    int4 m = make_int4(1, 0, 0, 0);
    bool ok;
    if (mode == kSamplerOffline) {
        ok = smp_offline(sig, k0, k1, c2, c3, l, m);
    } else {
        int4 cur = chain[l];
        if (cur.x == 0 && cur.y == 0 && cur.z == 0) {
            ok = smp_exact(cum, cap, ks, k0, k1, c2, c3, l, cur);
        } else {
            int4 mp;
            ok = smp_offline(sig, k0, k1, c2, c3, l, mp);
            if (ok) {
                const uint4 w = philox4x32_10(make_uint4((uint32_t)l, 0u, c2, (4u << 24) | c3), k0, k1);
                const double u = smp_u53(w.x, w.y);
                const double ra = __dsqrt_rn(alpha);
                const int a_[3] = {mp.x, mp.y, mp.z}, b_[3] = {cur.x, cur.y, cur.z};
                double num = 1.0, den = 1.0;
                for (int t = 0; t < 3; ++t) {
                    const double c = axis_c(alpha, ks->L[t]);
                    const double g = __ddiv_rn(kPi, __dmul_rn(ra, ks->L[t]));
                    const double a = (double)a_[t], b = (double)b_[t];
                    num = __dmul_rn(num, __dmul_rn(smp_exp0(-__dmul_rn(c, __dmul_rn(a, a))), smp_mass(b_[t], g)));
                    den = __dmul_rn(den, __dmul_rn(smp_exp0(-__dmul_rn(c, __dmul_rn(b, b))), smp_mass(a_[t], g)));
                }
                if (__dmul_rn(u, den) < num) cur = mp;
            }
        }
        if (ok) chain[l] = cur;
        m = cur;
    }
    if (!ok) {
        atomicOr(status, kStatusSample);
        m = make_int4(1, 0, 0, 0);  // keeps the evaluation finite; the call reports RBE_ESAMPLE
    }
    m_out[l] = m;
    if (w_out) w_out[l] = l < Pf ? ks->wP : ks->S / (double)(P - Pf);
}

}  // namespace rbe
