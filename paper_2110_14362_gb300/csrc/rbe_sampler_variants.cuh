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

// 1/n and 1/(2n + 1), n = 0..60, each the correctly rounded quotient (constant-folded IEEE
// division), so that multiplying by them gives the same bits as a host that divides 1.0 by n.
static __constant__ double kSmpInvN[61] = {0.0, 1.0 / 1.0, 1.0 / 2.0, 1.0 / 3.0, 1.0 / 4.0, 1.0 / 5.0, 1.0 / 6.0, 1.0 / 7.0, 1.0 / 8.0, 1.0 / 9.0, 1.0 / 10.0, 1.0 / 11.0, 1.0 / 12.0, 1.0 / 13.0, 1.0 / 14.0, 1.0 / 15.0, 1.0 / 16.0, 1.0 / 17.0, 1.0 / 18.0, 1.0 / 19.0, 1.0 / 20.0, 1.0 / 21.0, 1.0 / 22.0, 1.0 / 23.0, 1.0 / 24.0, 1.0 / 25.0, 1.0 / 26.0, 1.0 / 27.0, 1.0 / 28.0, 1.0 / 29.0, 1.0 / 30.0, 1.0 / 31.0, 1.0 / 32.0, 1.0 / 33.0, 1.0 / 34.0, 1.0 / 35.0, 1.0 / 36.0, 1.0 / 37.0, 1.0 / 38.0, 1.0 / 39.0, 1.0 / 40.0, 1.0 / 41.0, 1.0 / 42.0, 1.0 / 43.0, 1.0 / 44.0, 1.0 / 45.0, 1.0 / 46.0, 1.0 / 47.0, 1.0 / 48.0, 1.0 / 49.0, 1.0 / 50.0, 1.0 / 51.0, 1.0 / 52.0, 1.0 / 53.0, 1.0 / 54.0, 1.0 / 55.0, 1.0 / 56.0, 1.0 / 57.0, 1.0 / 58.0, 1.0 / 59.0, 1.0 / 60.0};
static __constant__ double kSmpInvOdd[61] = {1.0 / 1.0, 1.0 / 3.0, 1.0 / 5.0, 1.0 / 7.0, 1.0 / 9.0, 1.0 / 11.0, 1.0 / 13.0, 1.0 / 15.0, 1.0 / 17.0, 1.0 / 19.0, 1.0 / 21.0, 1.0 / 23.0, 1.0 / 25.0, 1.0 / 27.0, 1.0 / 29.0, 1.0 / 31.0, 1.0 / 33.0, 1.0 / 35.0, 1.0 / 37.0, 1.0 / 39.0, 1.0 / 41.0, 1.0 / 43.0, 1.0 / 45.0, 1.0 / 47.0, 1.0 / 49.0, 1.0 / 51.0, 1.0 / 53.0, 1.0 / 55.0, 1.0 / 57.0, 1.0 / 59.0, 1.0 / 61.0, 1.0 / 63.0, 1.0 / 65.0, 1.0 / 67.0, 1.0 / 69.0, 1.0 / 71.0, 1.0 / 73.0, 1.0 / 75.0, 1.0 / 77.0, 1.0 / 79.0, 1.0 / 81.0, 1.0 / 83.0, 1.0 / 85.0, 1.0 / 87.0, 1.0 / 89.0, 1.0 / 91.0, 1.0 / 93.0, 1.0 / 95.0, 1.0 / 97.0, 1.0 / 99.0, 1.0 / 101.0, 1.0 / 103.0, 1.0 / 105.0, 1.0 / 107.0, 1.0 / 109.0, 1.0 / 111.0, 1.0 / 113.0, 1.0 / 115.0, 1.0 / 117.0, 1.0 / 119.0, 1.0 / 121.0};

// erf on [0, 2]: sum_n (-1)^n x^(2n+1) / (n! (2n+1)) times 2/sqrt(pi); term n is
// t_n = t_(n-1) (-x^2) (1/n), added as t_n (1/(2n+1)); the sum stops after the first term below
// 2^-60 of the running sum (at most 60 terms).
__device__ __forceinline__ double smp_erf_series(double x)
{
    const double x2 = __dmul_rn(x, x);
    double t = x, sum = x;
    for (int n = 1; n <= 60; ++n) {
        t = __dmul_rn(__dmul_rn(t, -x2), kSmpInvN[n]);
        const double term = __dmul_rn(t, kSmpInvOdd[n]);
        sum = __dadd_rn(sum, term);
        if (fabs(term) < __dmul_rn(0x1.0p-60, fabs(sum))) break;
    }
    return __dmul_rn(sum, 0x1.20dd750429b6dp+0);
}

// erfc for x >= 0: 1 - erf on [0, 2], exp(-x^2)/(sqrt(pi) K) beyond with the continued
// fraction K = x + (1/2)/(x + 1/(x + (3/2)/(x + ...))) from depth ceil(10 + 200/x^2), 0 from 26 on.
__device__ __forceinline__ double smp_erfc(double x)
{
    if (x <= 2.0) return __dsub_rn(1.0, smp_erf_series(x));
    if (x >= 26.0) return 0.0;
    double f = x;
    const int depth = (int)ceil(__dadd_rn(10.0, __ddiv_rn(200.0, __dmul_rn(x, x))));
    for (int n = depth; n >= 1; --n) f = __dadd_rn(x, __ddiv_rn(__dmul_rn(0.5, (double)n), f));
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

namespace rbe {

// The MH step of 32 slots per block (6 warps): warp 0 forms the proposals (and the exact draw of
// a slot whose chain is at m = 0); warps 0..5 each form one factor of the acceptance for all 32
// slots, F = exp(-c_a m'_a^2) mass(m_a) (warps 0..2, axis a, numerator) or exp(-c_a m_a^2)
// mass(m'_a) (warps 3..5, denominator), so that no warp runs more than one mass's FP64 chain
// (each FP64 warp instruction occupies GB300's narrow pipe for the whole warp, however few lanes
// are active: the six chains must sit on different warps); warp 0 multiplies the factors in
// axis order, exactly as one thread would, and accepts.  Same draws as sample_variant_body.
constexpr int kMhSlots = 32, kMhWarps = 6;

static __global__ void __launch_bounds__(kMhWarps * 32)
k_sample_mh(uint64_t seed, uint64_t step_arg, const unsigned long long* __restrict__ step_dev, int P, int Pf,
            const unsigned long long* __restrict__ cum, int cap, const KState* __restrict__ ks,
            int4* __restrict__ chain, int4* __restrict__ m_out, double* __restrict__ w_out,
            unsigned* __restrict__ status)
{
    __shared__ int4 s_cur[kMhSlots], s_mp[kMhSlots];
    __shared__ int s_state[kMhSlots];  // 0 propose, 1 exact start, 2 failed
    __shared__ double s_f[kMhWarps][kMhSlots];
    pdl_wait();
    pdl_trigger();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int l = blockIdx.x * kMhSlots + lane;
    const bool live = l < P;
    const uint64_t step = step_dev ? *step_dev : step_arg;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t c2 = (uint32_t)step, c3 = (uint32_t)((step >> 32) & 0xFFFFFFu);
    const double alpha = ks->alpha;
    if (warp == 0 && live) {
        double sig[3];
        const double ra2 = __dsqrt_rn(__dmul_rn(alpha, 0.5));
        for (int t = 0; t < 3; ++t) sig[t] = __ddiv_rn(__dmul_rn(ra2, ks->L[t]), kPi);
        int4 cur = chain[l], mp = make_int4(0, 0, 0, 0);
        int state = 0;
        if (cur.x == 0 && cur.y == 0 && cur.z == 0) {
            state = smp_exact(cum, cap, ks, k0, k1, c2, c3, l, cur) ? 1 : 2;
        } else if (!smp_offline(sig, k0, k1, c2, c3, l, mp)) {
            state = 2;
        }
        s_cur[lane] = cur;
        s_mp[lane] = mp;
        s_state[lane] = state;
    }
    __syncthreads();
    if (live && s_state[lane] == 0) {
        const int a = warp % 3;
        const bool numerator = warp < 3;
        const int4 cur = s_cur[lane], mp = s_mp[lane];
        const int ca[3] = {cur.x, cur.y, cur.z}, pa[3] = {mp.x, mp.y, mp.z};
        const double c = axis_c(alpha, ks->L[a]);
        const double g = __ddiv_rn(kPi, __dmul_rn(__dsqrt_rn(alpha), ks->L[a]));
        const double e = (double)(numerator ? pa[a] : ca[a]);
        s_f[warp][lane] = __dmul_rn(smp_exp0(-__dmul_rn(c, __dmul_rn(e, e))), smp_mass(numerator ? ca[a] : pa[a], g));
    }
    __syncthreads();
    if (warp != 0 || !live) return;
    int4 cur = s_cur[lane];
    const int state = s_state[lane];
    if (state == 0) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)l, 0u, c2, (4u << 24) | c3), k0, k1);
        const double u = smp_u53(w.x, w.y);
        double num = 1.0, den = 1.0;
        for (int t = 0; t < 3; ++t) {
            num = __dmul_rn(num, s_f[t][lane]);
            den = __dmul_rn(den, s_f[3 + t][lane]);
        }
        if (__dmul_rn(u, den) < num) cur = s_mp[lane];
    }
    int4 m = cur;
    if (state == 2) {
        atomicOr(status, kStatusSample);
        m = make_int4(1, 0, 0, 0);  // keeps the evaluation finite; the call reports RBE_ESAMPLE
    } else {
        chain[l] = cur;
    }
    m_out[l] = m;
    if (w_out) w_out[l] = l < Pf ? ks->wP : ks->S / (double)(P - Pf);
}

}  // namespace rbe
