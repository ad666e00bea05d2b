// Device-side building blocks of the RBE k-space path (sm_103a).
//
//  * Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) for the counter-based sampler.
//  * A Cody--Waite + Taylor exponential for the sampler's weight table, written with
//    explicitly rounded double operations so that no multiply-add is contracted.
//  * Fixed-point scaled coordinates: s = r / l mod 1 as a 32-bit fraction, so that the
//    phase m.s mod 1 is exact in wrapping 32-bit integer arithmetic.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rbe {

constexpr double kPi = 3.14159265358979323846;
constexpr double kLn2 = 0.69314718055994530942;
constexpr uint32_t kMaxAttempts = 1u << 20;

// Status bits latched on the device.
constexpr unsigned kStatusSample = 1u;     // a sample stayed at m = 0 for kMaxAttempts redraws
constexpr unsigned kStatusNonFinite = 2u;  // rho or an output is NaN/Inf
constexpr unsigned kStatusTable = 4u;      // the sampling table did not fit its capacity
constexpr unsigned kStatusTimeout = 8u;    // a bounded wait gave up
constexpr unsigned kStatusBox = 16u;       // NPT: the box outgrew the cell list or broke rc <= l/2
constexpr unsigned kStatusList = 32u;      // NPT: a particle had more neighbours than the list holds
constexpr unsigned kStatusShake = 64u;     // rigid water: SHAKE did not converge within its sweep limit

// ---------------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor in the stream is still running;
// pdl_wait() blocks until the predecessor grid has completed and its writes are visible
// (it returns at once for a normal launch).  pdl_trigger() lets the successor launch.
// Every kernel here reads its predecessor's outputs, and writes global memory, only
// after pdl_wait().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------------
// Philox-4x32-10: ten rounds; each multiplies words 0 and 2 by 0xD2511F53 and
// 0xCD9E8D57 (32x32 -> 64 bits), xors the high halves with words 1 and 3 and the round
// key, and permutes; the key advances by 0x9E3779B9 and 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// ---------------------------------------------------------------------------------
// exp(x) for x in [-700, 0]: n = rint(x / ln2), r = (x - n ln2_hi) - n ln2_lo with a
// 32-significant-bit head of ln2 (n * head exact), e^r by its Taylor series to degree 13
// in Horner form, times 2^n.  Every step is a separately rounded IEEE operation.
__device__ __forceinline__ double table_exp(double x)
{
    const double inv_ln2 = 0x1.71547652b82fep+0;
    const double ln2_hi = 0x1.62e42fee00000p-1;
    const double ln2_lo = 0x1.a39ef35793c76p-33;
    const double c[14] = {0x1.0000000000000p+0, 0x1.0000000000000p+0, 0x1.0000000000000p-1,
                          0x1.5555555555555p-3, 0x1.5555555555555p-5, 0x1.1111111111111p-7,
                          0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16,
                          0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
                          0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};
    const double n = rint(__dmul_rn(x, inv_ln2));
    const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(n, ln2_hi)), __dmul_rn(n, ln2_lo));
    double p = c[13];
#pragma unroll
    for (int j = 12; j >= 0; --j) p = __dadd_rn(__dmul_rn(p, r), c[j]);
    return ldexp(p, (int)n);
}

// c = pi^2 / (alpha l^2), the per-axis exponent of exp(-|k|^2 / 4 alpha) in m.
__device__ __forceinline__ double axis_c(double alpha, double ell)
{
    return __ddiv_rn(__dmul_rn(kPi, kPi), __dmul_rn(alpha, __dmul_rn(ell, ell)));
}

// Truncation |m| <= M = ceil(sqrt(60 ln2 / c)): drops weights below 2^-60 of the peak.
// M is formed in FP64 and compared with the table's room before any integer conversion,
// so that no box length (huge, infinite, NaN) can overflow the index arithmetic: beyond
// the room, or for a box that is not finite and positive, *bad is set and M is clamped.
__device__ __forceinline__ int axis_M_capped(double ell, double c, int cap, bool* bad)
{
    const double Md = ceil(__dsqrt_rn(__ddiv_rn(__dmul_rn(60.0, kLn2), c)));
    const int Mmax = (cap - 1) / 2;
    if (!(ell > 0.0) || !isfinite(ell) || !(Md <= (double)Mmax)) {
        *bad = true;
        return Mmax;
    }
    *bad = false;
    return (int)Md;
}

// ---------------------------------------------------------------------------------
// 32-bit fixed-point fraction of r / l (wrapping: any real r maps into [0, 2^32)).
__device__ __forceinline__ uint32_t fixed_frac(double r, double inv_l)
{
    return (uint32_t)(unsigned long long)__double2ll_rn(__dmul_rn(r, inv_l) * 4294967296.0);
}

// Phase of m.s for 32-bit fixed-point s, as an angle in [-pi, pi) (FP32).
// t = m.s + 2^31 + 2^8 (mod 2^32) is exact; its top 23 bits under the exponent bits of
// 1.0f give a float f in [1, 2) with f - 1 = (m.s + 1/2) mod 1 rounded to 2^-23
// revolutions, and one FFMA maps it to 2 pi (f - 1.5).  The FP32 constants 2 pi and
// 3 pi shift every angle by the same ~2.4e-7 rad (plus a relative 3e-8 scale error); a
// common shift of all phases multiplies rho(k) by a unit phase factor that cancels in
// |rho|^2 and in Im(e^{-ik.r} rho(k)), so it leaves forces, energy and virial unchanged.
// (t >> 9) | 0x3f800000 in one funnel shift: the 64-bit word (0x7f : t) shifted right by 9.
__device__ __forceinline__ uint32_t phase_bits(uint32_t t) { return __funnelshift_r(t, 0x7fu, 9); }

// Sine and cosine by the MUFU approximations with subnormal inputs flushed (sin.approx.ftz,
// cos.approx.ftz).  The phases of fixed_phase are (b - 3/2) 2 pi for b in [1, 2) with a 23-bit
// mantissa: zero or at least 2 pi 2^-23 in magnitude, never subnormal, so the flush changes no
// result, and the instruction needs no subnormal handling around the MUFU operation.
__device__ __forceinline__ float mufu_sin(float x)
{
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float mufu_cos(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float fixed_phase(int mx, int my, int mz, uint32_t sx, uint32_t sy, uint32_t sz)
{
    uint32_t t = (uint32_t)mx * sx + 0x80000100u;
    t += (uint32_t)my * sy;
    t += (uint32_t)mz * sz;
    return fmaf(__uint_as_float(phase_bits(t)), 6.28318530717958647692f, -9.42477796076937971538f);
}

// The same mapping of m.s - phi, for a phase offset given in the same fixed point: off =
// 2^31 + 2^8 - phi (mod 2^32), phi in revolutions x 2^32.  The force pass uses it to take
// one sine per pair (sin(theta - arg rho) instead of the pair sin theta, cos theta).
__device__ __forceinline__ float fixed_phase_off(int mx, int my, int mz, uint32_t sx, uint32_t sy, uint32_t sz,
                                                 uint32_t off)
{
    uint32_t t = (uint32_t)mx * sx + off;
    t += (uint32_t)my * sy;
    t += (uint32_t)mz * sz;
    return fmaf(__uint_as_float(phase_bits(t)), 6.28318530717958647692f, -9.42477796076937971538f);
}

// ---------------------------------------------------------------------------------
// Integer-only conversions.  GB300 executes FP64 instructions on a narrow pipe (about
// 1.7 FP64 FMA per clock per SM), so the FP32-phase path converts its FP64 inputs with
// 32/64-bit integer operations on the IEEE bit patterns instead.

// 1/l as a 64-bit mantissa and a power of two: 1/l = q * 2^e, q in [2^63, 2^64).
struct FixScale {
    unsigned long long q;
    int e;
};

// round(r / l * 2^32) mod 2^32 for a finite double r (zero/subnormal r -> 0): the
// 117-bit product of r's 53-bit mantissa and q, shifted and rounded to nearest.
__host__ __device__ inline uint32_t fixed_frac_int(unsigned long long rb, FixScale sc)
{
    const unsigned er = (unsigned)(rb >> 52) & 0x7ffu;
    if (er == 0u || er == 0x7ffu) return 0u;
    const unsigned long long mr = (rb & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = (int)er - 1075 + sc.e + 32;  // r / l * 2^32 = mr * q * 2^sh
#ifdef __CUDA_ARCH__
    const unsigned long long hi = __umul64hi(mr, sc.q);
#else
    const unsigned long long hi = (unsigned long long)(((unsigned __int128)mr * sc.q) >> 64);
#endif
    const unsigned long long lo = mr * sc.q;
    uint32_t res;
    if (sh >= 0) {
        res = sh >= 32 ? 0u : (uint32_t)(lo << sh);
    } else {
        const int d = -sh;
        unsigned long long lo2 = lo, hi2 = hi;
        if (d <= 64) {
            lo2 = lo + (1ull << (d - 1));
            hi2 = hi + (lo2 < lo ? 1ull : 0ull);
        } else if (d < 128) {
            hi2 = hi + (1ull << (d - 65));
        }
        if (d < 64) res = (uint32_t)((lo2 >> d) | (hi2 << (64 - d)));
        else if (d < 128) res = (uint32_t)(hi2 >> (d - 64));
        else res = 0u;
    }
    return (rb >> 63) ? 0u - res : res;
}

// Nearest float to a double (round half to even); zero/subnormal -> signed zero,
// overflow -> infinity, NaN stays NaN.  Integer operations only.
__host__ __device__ inline float double_to_float_int(unsigned long long b)
{
    const uint32_t sign = (uint32_t)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    uint32_t out;
    if (e == 0x7ff) {
        out = sign | 0x7f800000u | (m ? 0x400000u : 0u);
    } else {
        int fe = e - 1023 + 127;
        if (e == 0 || fe <= 0) {
            out = sign;
        } else {
            uint32_t mant = (uint32_t)(m >> 29);
            const uint32_t rem = (uint32_t)(m & 0x1FFFFFFFu);
            if (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) {
                if (++mant == 0x800000u) {
                    mant = 0u;
                    ++fe;
                }
            }
            out = fe >= 255 ? (sign | 0x7f800000u) : (sign | ((uint32_t)fe << 23) | mant);
        }
    }
#ifdef __CUDA_ARCH__
    return __uint_as_float(out);
#else
    float f;
    __builtin_memcpy(&f, &out, 4);
    return f;
#endif
}

// The double equal to a float (exact), with integer operations only.
__host__ __device__ inline unsigned long long float_to_double_bits(uint32_t b)
{
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    int e = (int)((b >> 23) & 0xff);
    uint32_t m = b & 0x7fffffu;
    if (e == 0xff) return sign | (0x7ffull << 52) | ((unsigned long long)m << 29);
    if (e == 0) {
        if (m == 0u) return sign;
        int lz = 0;  // subnormal float: normalise
        while (!(m & 0x800000u)) {
            m <<= 1;
            ++lz;
        }
        m &= 0x7fffffu;
        e = 1 - lz;
    }
    return sign | ((unsigned long long)(e - 127 + 1023) << 52) | ((unsigned long long)m << 29);
}

// Exponent field == 0x7ff: infinity or NaN.
__host__ __device__ inline bool nonfinite_bits(unsigned long long b)
{
    return ((b >> 52) & 0x7ffull) == 0x7ffull;
}

// Float-float accumulation (Knuth's TwoSum): (hi, lo) += x with the rounding error of
// the FP32 addition carried in lo; about 48 significant bits from FP32 operations.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo += err;
}

// (hi, lo) += (xh, xl)
__device__ __forceinline__ void ff_add2(float& hi, float& lo, float xh, float xl)
{
    ff_add(hi, lo, xh);
    lo += xl;
}

}  // namespace rbe
