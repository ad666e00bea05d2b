// Tile bodies of the RBE k-space FP32-phase path and the table/sampler kernels, as device
// functions with explicit tile indices.  The single-system kernels (rbe_kspace.cu) call them
// with their block indices; the batched kernels (rbe_batch.cu) with the tiles of a work list
// over many systems.  See rbe_kspace.cu for the pass structure (Sec. 4.2 of the paper).
#pragma once

#include <cuda_runtime.h>

#include "rbe_context.h"
#include "rbe_device.cuh"

namespace rbe {

constexpr int kTableThreads = 1024;   // k_tables block (tables_body runs with any block of >= 160 threads)
constexpr int kMaxRhoThreads = 256;   // threads of a rho block with one frequency per thread
constexpr int kRhoThreadsF = 128;     // threads of a rho block with 2 or 4 frequencies per thread
constexpr int kReduceThreads = 256;
constexpr int kForceWarps = 8;
constexpr int kForceThreads = 32 * kForceWarps;
// Force-pass tile parameters (compile-time; the defaults are the measured best on GB300):
// particles per lane, unroll of the frequency loop, resident blocks per SM the registers are
// sized for.
#ifndef RBE_FORCE_PPT
#define RBE_FORCE_PPT 2
#endif
#ifndef RBE_FORCE_LUNROLL
#define RBE_FORCE_LUNROLL 16
#endif
#ifndef RBE_FORCE_MINB
#define RBE_FORCE_MINB 4
#endif
constexpr int kForcePPT = RBE_FORCE_PPT;
constexpr int kForceLUnroll = RBE_FORCE_LUNROLL;
constexpr int kForceRound = 32 * kForcePPT;  // particles per round of the FP32 force pass
// frequencies staged at once (dynamic shared memory, 32 B each): 16 KB leaves room for five
// resident blocks per SM; more frequencies are restaged in tiles for every round of particles
#ifndef RBE_FORCE_STAGEK
#define RBE_FORCE_STAGEK 512
#endif
constexpr int kForceStageK = RBE_FORCE_STAGEK;
// shared memory per staged frequency: (mx, my, mz, phase offset) and (R, R mx, R my, R mz)
constexpr int kForceSmemPerK = 32;

__device__ __forceinline__ FixScale fs(const FixScaleH& h) { return FixScale{h.q, h.e}; }

// =================================================================================
// Tables and box constants (Sec. 4.2 Eqs. (S), (psf); App. C item 1).  One block.
// Per axis: c = pi^2/(alpha l^2), M = ceil(sqrt(60 ln2 / c)), w_a = exp(-c a^2) by the
// library's own exponential, W_j = rint(w_{|j-M|} 2^sh) with sh = 62 - bitlength(2M+1),
// C_j = W_0 + ... + W_j (exact integers: any summation order gives the same bits, so the
// prefix sum runs in parallel), H = C_2M 2^-sh, S = H_x H_y H_z - 1.
__device__ __forceinline__ int bitlength(unsigned x) { return 32 - __clz(x); }

__device__ __forceinline__ void tables_body(double bx, double by, double bz, const double* __restrict__ box_dev,
                                            double alpha, int P,
         unsigned long long* __restrict__ cum, int cap, KState* __restrict__ ks, unsigned* __restrict__ status)
{
    __shared__ int sM[3], sSh[3];
    __shared__ double sc[3], sL[3];
    __shared__ unsigned long long wsum[32];
    const int nthr = blockDim.x;  // a multiple of 32, at least 160 (the box-constant threads)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 3) {
        const double ell = box_dev ? box_dev[tid] : (tid == 0 ? bx : (tid == 1 ? by : bz));
        const double c = axis_c(alpha, ell);
        bool bad;
        const int M = axis_M_capped(ell, c, cap, &bad);
        if (bad) atomicOr(status, kStatusTable);
        sL[tid] = ell;
        sc[tid] = c;
        sM[tid] = M;
        sSh[tid] = 62 - bitlength((unsigned)(2 * M + 1));
    }
    __syncthreads();
    // integer weights, written once per |m| into both halves of the row; the (axis, a)
    // entries of the three rows are spread over all threads
    {
        const int n0 = sM[0] + 1, n1 = sM[1] + 1, n2 = sM[2] + 1;
        for (int e = tid; e < n0 + n1 + n2; e += nthr) {
            const int t = e < n0 ? 0 : (e < n0 + n1 ? 1 : 2);
            const int a = e - (t == 0 ? 0 : (t == 1 ? n0 : n0 + n1));
            const int M = sM[t];
            unsigned long long* row = cum + (size_t)t * cap;
            const double v = table_exp(-__dmul_rn(sc[t], (double)a * (double)a));
            const unsigned long long W = (unsigned long long)__double2ll_rn(ldexp(v, sSh[t]));
            row[M + a] = W;
            row[M - a] = W;
        }
    }
    __syncthreads();
    // inclusive prefix sums, one row at a time: each thread owns a contiguous segment
    for (int t = 0; t < 3; ++t) {
        const int n = 2 * sM[t] + 1;
        unsigned long long* row = cum + (size_t)t * cap;
        const int per = (n + nthr - 1) / nthr;
        const int j0 = min(n, tid * per), j1 = min(n, j0 + per);
        unsigned long long local = 0;
        for (int j = j0; j < j1; ++j) local += row[j];
        unsigned long long incl = local;  // inclusive scan of the segment sums over the block
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long v = lane < (nthr >> 5) ? wsum[lane] : 0ull;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long o = __shfl_up_sync(0xffffffffu, v, off);
                if (lane >= off) v += o;
            }
            wsum[lane] = v;
        }
        __syncthreads();
        unsigned long long run = incl - local + (warp > 0 ? wsum[warp - 1] : 0ull);
        for (int j = j0; j < j1; ++j) {
            run += row[j];
            row[j] = run;
        }
        __syncthreads();
    }
    // box constants: independent FP64 chains on separate threads (GB300 runs FP64 at a low
    // rate, so a single thread computing all of them would serialise their latency)
    __shared__ double sH[3];
    if (tid < 3) {
        const unsigned long long C = cum[(size_t)tid * cap + 2 * sM[tid]];
        sH[tid] = ldexp((double)C, -sSh[tid]);
        ks->H[tid] = sH[tid];
        ks->M[tid] = sM[tid];
        ks->sh[tid] = sSh[tid];
        ks->L[tid] = sL[tid];
    } else if (tid >= 32 && tid < 35) {
        const int t = tid - 32;
        const double inv = 1.0 / sL[t];
        ks->inv[t] = inv;
        const unsigned long long b = (unsigned long long)__double_as_longlong(inv);
        const int e = (int)((b >> 52) & 0x7ff) - 1075;
        ks->sc[t].q = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 11;
        ks->sc[t].e = e - 11;
    } else if (tid >= 64 && tid < 67) {
        const int t = tid - 64;
        const float c = (float)(2.0 * kPi / sL[t]);
        if (t == 0) ks->cx = c;
        else if (t == 1) ks->cy = c;
        else ks->cz = c;
    } else if (tid == 96) {
        const double V = sL[0] * sL[1] * sL[2];
        ks->V = V;
        ks->ce = 2.0 * kPi / V;
    } else if (tid == 97) {
        ks->cb = 4.0 * kPi / (sL[0] * sL[1] * sL[2]);
    } else if (tid == 128) {
        ks->alpha = alpha;
        ks->P = P;
        ks->inv4a = 0.25 / alpha;
    } else if (tid == 129) {
        ks->cself = -sqrt(alpha / kPi);
    }
    __syncthreads();
    if (tid == 0) {
        const double S = __dsub_rn(__dmul_rn(__dmul_rn(sH[0], sH[1]), sH[2]), 1.0);
        ks->S = S;
        ks->wP = S / (double)P;
    }
}

// Smallest j in [0, 2M] with T < C_j, minus M (C non-decreasing).
__device__ __forceinline__ int inverse_cdf_int(const unsigned long long* __restrict__ row, int M,
                                               unsigned long long T)
{
    int lo = 0, hi = 2 * M;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (T < row[mid]) hi = mid;
        else lo = mid + 1;
    }
    return lo - M;
}

// T = floor(U * C_2M / 2^53) for a 53-bit uniform integer U (exact, 128-bit product).
__device__ __forceinline__ unsigned long long scaled_target(unsigned long long U, unsigned long long Ctot)
{
    const unsigned long long hi = __umul64hi(U, Ctot), lo = U * Ctot;
    return (hi << 11) | (lo >> 53);
}

// =================================================================================
// Frequency sampling (Sec. 4.2-4.3): sample l uses Philox key (seed_lo, seed_hi) and
// counters (l, 2 attempt + half, step_lo, step_hi24); redraw while m = 0.  Integer
// operations only: U from 53 bits of Philox output, T = floor(U C_2M / 2^53), and the
// search over the integer cumulative weights.  The block copies the three rows to shared
// memory when they fit (smem_cap > 0).
// Slots [0, Pf) are the force batch (weight S/P_f, the tables' wP); slots [Pf, P), when P > Pf,
// a separate pressure batch (weight S/(P - Pf), Eq. (apppress) with its own p~).
__device__ __forceinline__ void sample_body(int lbase, uint64_t seed, uint64_t step_arg,
                                            const unsigned long long* __restrict__ step_dev, int P, int Pf,
                         const unsigned long long* __restrict__ cum, int cap, int smem_cap,
                         const KState* __restrict__ ks, int4* __restrict__ m_out, double* __restrict__ w_out,
                         unsigned* __restrict__ status)
{
    extern __shared__ unsigned long long s_cum[];
    pdl_trigger();  // the rho pass may start staging its particles meanwhile
    const uint64_t step = step_dev ? *step_dev : step_arg;  // a device-resident step index when given
    const double wP = ks->wP;
    const unsigned long long* tx = cum;
    const unsigned long long* ty = cum + cap;
    const unsigned long long* tz = cum + 2 * (size_t)cap;
    if (smem_cap > 0) {  // smem_cap == cap: copy the three rows whole, without waiting for M
        // eight loads per thread issued before their stores, so that the copy takes one round
        // trip to L2 per eight entries instead of one per entry
        const int n = 3 * smem_cap;
        for (int j0 = threadIdx.x; j0 < n; j0 += 8 * (int)blockDim.x) {
            unsigned long long v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u * (int)blockDim.x;
                v[u] = j < n ? cum[j] : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u * (int)blockDim.x;
                if (j < n) s_cum[j] = v[u];
            }
        }
    }
    const int Mx = ks->M[0], My = ks->M[1], Mz = ks->M[2];
    if (smem_cap > 0) {
        __syncthreads();
        tx = s_cum;
        ty = s_cum + smem_cap;
        tz = s_cum + 2 * smem_cap;
    }
    const int l = lbase + (int)threadIdx.x;
    if (l >= P) return;
    const unsigned long long Cx = tx[2 * Mx], Cy = ty[2 * My], Cz = tz[2 * Mz];
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t c2 = (uint32_t)step, c3 = (uint32_t)((step >> 32) & 0xFFFFFFu);
    int4 m = make_int4(0, 0, 0, 0);
    bool found = false;
    for (uint32_t attempt = 0; attempt < kMaxAttempts; ++attempt) {
        const uint4 w0 = philox4x32_10(make_uint4((uint32_t)l, 2u * attempt, c2, c3), k0, k1);
        const uint4 w1 = philox4x32_10(make_uint4((uint32_t)l, 2u * attempt + 1u, c2, c3), k0, k1);
        m.x = inverse_cdf_int(tx, Mx, scaled_target(((unsigned long long)w0.x << 21) | (w0.y >> 11), Cx));
        m.y = inverse_cdf_int(ty, My, scaled_target(((unsigned long long)w0.z << 21) | (w0.w >> 11), Cy));
        m.z = inverse_cdf_int(tz, Mz, scaled_target(((unsigned long long)w1.x << 21) | (w1.y >> 11), Cz));
        if (m.x != 0 || m.y != 0 || m.z != 0) {
            found = true;
            break;
        }
    }
    if (!found) {
        atomicOr(status, kStatusSample);
        m = make_int4(1, 0, 0, 0);  // keeps the evaluation finite; the call reports RBE_ESAMPLE
    }
    m_out[l] = m;
    if (w_out) w_out[l] = l < Pf ? wP : ks->S / (double)(P - Pf);
}

// Fixed-order block sum of a float-float value per thread; valid in thread 0.
__device__ __forceinline__ void block_sum_ff(float& hi, float& lo, float (*scratch)[32])
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, off);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, off);
        ff_add2(hi, lo, oh, ol);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        scratch[0][warp] = hi;
        scratch[1][warp] = lo;
    }
    __syncthreads();
    if (warp == 0) {
        const bool on = lane < (int)(blockDim.x >> 5);
        hi = on ? scratch[0][lane] : 0.f;
        lo = on ? scratch[1][lane] : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, off);
            const float ol = __shfl_xor_sync(0xffffffffu, lo, off);
            ff_add2(hi, lo, oh, ol);
        }
    }
}

// Fixed-order block sums of two float-float values per thread (one shared-memory round for
// both); valid in thread 0.
__device__ __forceinline__ void block_sum_ff2(float& ah, float& al, float& bh, float& bl, float (*scratch)[32])
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float oah = __shfl_xor_sync(0xffffffffu, ah, off), oal = __shfl_xor_sync(0xffffffffu, al, off);
        const float obh = __shfl_xor_sync(0xffffffffu, bh, off), obl = __shfl_xor_sync(0xffffffffu, bl, off);
        ff_add2(ah, al, oah, oal);
        ff_add2(bh, bl, obh, obl);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        scratch[0][warp] = ah;
        scratch[1][warp] = al;
        scratch[2][warp] = bh;
        scratch[3][warp] = bl;
    }
    __syncthreads();
    if (warp == 0) {
        const bool on = lane < (int)(blockDim.x >> 5);
        ah = on ? scratch[0][lane] : 0.f;
        al = on ? scratch[1][lane] : 0.f;
        bh = on ? scratch[2][lane] : 0.f;
        bl = on ? scratch[3][lane] : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float oah = __shfl_xor_sync(0xffffffffu, ah, off), oal = __shfl_xor_sync(0xffffffffu, al, off);
            const float obh = __shfl_xor_sync(0xffffffffu, bh, off), obl = __shfl_xor_sync(0xffffffffu, bl, off);
            ff_add2(ah, al, oah, oal);
            ff_add2(bh, bl, obh, obl);
        }
    }
}

// Loads particle i as (s_x, s_y, s_z) 32-bit fixed point and q as float, with integer
// operations only; flags non-finite inputs.
__device__ __forceinline__ uint4 load_fixed(const double* __restrict__ pos, const double* __restrict__ q,
                                            int64_t i, FixScale scx, FixScale scy, FixScale scz,
                                            unsigned* __restrict__ status)
{
    const unsigned long long bx = (unsigned long long)__double_as_longlong(pos[3 * i]);
    const unsigned long long by = (unsigned long long)__double_as_longlong(pos[3 * i + 1]);
    const unsigned long long bz = (unsigned long long)__double_as_longlong(pos[3 * i + 2]);
    const unsigned long long bq = (unsigned long long)__double_as_longlong(q[i]);
    if (nonfinite_bits(bx) || nonfinite_bits(by) || nonfinite_bits(bz) || nonfinite_bits(bq))
        atomicOr(status, kStatusNonFinite);  // status may be a shared-memory flag (before pdl_wait)
    return make_uint4(fixed_frac_int(bx, scx), fixed_frac_int(by, scy), fixed_frac_int(bz, scz),
                      __float_as_uint(double_to_float_int(bq)));
}

// The same record from a float4 (x, y, z, q) input: each coordinate is widened to the double
// it equals (exact) and converted as above, so a float position gives the fixed point of that
// double; q is taken as it is.
__device__ __forceinline__ uint4 load_fixed_f4(const float4* __restrict__ xyzq, int64_t i, FixScale scx,
                                               FixScale scy, FixScale scz, unsigned* __restrict__ status)
{
    const float4 v = xyzq[i];
    const uint32_t bx = __float_as_uint(v.x), by = __float_as_uint(v.y), bz = __float_as_uint(v.z);
    const uint32_t bq = __float_as_uint(v.w);
    if (((bx >> 23) & 0xffu) == 0xffu || ((by >> 23) & 0xffu) == 0xffu || ((bz >> 23) & 0xffu) == 0xffu ||
        ((bq >> 23) & 0xffu) == 0xffu)
        atomicOr(status, kStatusNonFinite);  // infinity or NaN
    return make_uint4(fixed_frac_int(float_to_double_bits(bx), scx), fixed_frac_int(float_to_double_bits(by), scy),
                      fixed_frac_int(float_to_double_bits(bz), scz), bq);
}

// A particle's record from either input form: XYZQ selects the float4 (x, y, z, q) array in
// pos (q unused), else pos is N x 3 double and q N double.
template <bool XYZQ>
__device__ __forceinline__ uint4 load_record(const void* __restrict__ pos, const double* __restrict__ q, int64_t i,
                                             FixScale scx, FixScale scy, FixScale scz, unsigned* __restrict__ status)
{
    if (XYZQ) return load_fixed_f4(static_cast<const float4*>(pos), i, scx, scy, scz, status);
    return load_fixed(static_cast<const double*>(pos), q, i, scx, scy, scz, status);
}

// =================================================================================
// rho pass, FP32-phase path.  Block (kt, c) has blockDim.x = T S threads (whole warps): S
// particle sub-streams of T frequency lanes.  It covers the frequency tile of T F frequencies:
// thread j of sub-stream s owns frequencies kt T F + f T + j (f < F), and runs over its
// contiguous share (kRhoStage / S particles) of every tile of the chunk's particles
// [c * chunk_len, (c + 1) * chunk_len), staged in shared memory kRhoStage at a time as 32-bit
// fixed-point (s_x, s_y, s_z) plus q as float and read as broadcasts: one shared-memory load
// feeds F pairs.  The sub-streams let a small frequency tile fill a block of several warps;
// their sums are added in sub-stream order at the end.  No FP64 instruction runs per particle
// or per pair: sums across staged tiles are float-float.
// ACC: RBE_RHO_COMP32 (compensated FP32: 16-term partial sums added with Kahan's
//      compensation, an error bound that does not grow with the particle count),
//      RBE_RHO_FP32 (plain FP32 within a tile), RBE_RHO_FP64 (FP64 per pair; slow on GB300).
// Partials: float4 (Re hi, Re lo, Im hi, Im lo) at [l * nchunks + c]; row K holds the
// chunk's sum of q^2 (hi, lo).  The box constants are read from ks before pdl_wait: the
// kernel that wrote them (k_tables) runs before the sampler, which is this launch's
// predecessor, and the sampler starts only after k_tables has completed.
#ifndef RBE_RHO_STAGE
#define RBE_RHO_STAGE 512
#endif
constexpr int kRhoStage = RBE_RHO_STAGE;  // particles staged per tile
// Particles per FP32 partial sum of the compensated path: 16 (one compensated addition per 16
// pairs; groups of 4 and 8 measured 7 % and 3 % slower at N = 4e6, P = 2000).
#ifndef RBE_RHO_GROUP
#define RBE_RHO_GROUP 16
#endif
constexpr int kRhoGroup = RBE_RHO_GROUP;
static_assert(kRhoGroup == 4 || kRhoGroup == 8 || kRhoGroup == 16, "groups of 4, 8 or 16 particles");

// NT: the most threads a block of this tile has (the size of its shared float-float sums).
template <int ACC, int F, bool XYZQ = false, int NT = (F == 1 ? kMaxRhoThreads : kRhoThreadsF)>
__device__ __forceinline__ void rho_f32_tile(int kt, int c, const void* __restrict__ pos,
                                             const double* __restrict__ q, int64_t N, const KState* __restrict__ ks,
          const int4* __restrict__ m, int K, int64_t chunk_len, int nchunks, float4* __restrict__ partials,
          unsigned* __restrict__ status, int S = 1, int T_lanes = 0)
{
    __shared__ uint4 sp[kRhoStage];
    __shared__ float red[2][32];
    __shared__ unsigned bad;
    const int tid = threadIdx.x, nt = blockDim.x;
    // T frequency lanes per sub-stream (by default the block divided evenly; any T with S T <= the
    // block's threads otherwise, the threads beyond S T idle), S particle sub-streams
    const int T = T_lanes > 0 ? T_lanes : nt / S, j = tid % T, ss = tid / T;
    const bool act = ss < S;
    const int lbase = kt * T * F + j;
    // each sub-stream's share of a staged tile is a multiple of kRhoGroup particles (the
    // compensated sums take them a group at a time), so that no group reaches into the next share
    const int share = kRhoGroup * (kRhoStage / (kRhoGroup * S)), p0 = ss * share;
    const int stage = S * share;  // particles staged per tile (kRhoStage for S = 1, 2, 4, 8, 16)
    const FixScale scx = fs(ks->sc[0]), scy = fs(ks->sc[1]), scz = fs(ks->sc[2]);
    // the float-float sums across staged tiles, (Re hi, Re lo, Im hi, Im lo) per frequency, live
    // in shared memory: they change once per tile, and registers go to the pair loop
    __shared__ float4 acc_s[NT * F];
    if (act) {
#pragma unroll
        for (int f = 0; f < F; ++f) acc_s[(ss * F + f) * T + j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float q2h = 0.f, q2l = 0.f;
    const int64_t start = (int64_t)c * chunk_len;
    const int64_t end = min(N, start + chunk_len);
    if (tid == 0) bad = 0u;
    __syncthreads();
    // the first tile is staged before waiting for the sampler (inputs only)
    for (int u = tid; u < stage; u += nt) {
        const int64_t i = start + u;
        uint4 rec = make_uint4(0u, 0u, 0u, 0u);
        if (i < end) {
            rec = load_record<XYZQ>(pos, q, i, scx, scy, scz, &bad);
            const float qf = __uint_as_float(rec.w);
            ff_add(q2h, q2l, qf * qf);
        }
        sp[u] = rec;
    }
    pdl_wait();
    pdl_trigger();
    int4 mv[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const int l = lbase + f * T;
        mv[f] = l < K ? m[l] : make_int4(0, 0, 0, 0);
    }
    for (int64_t base = start; base < end; base += stage) {
        if (base != start) {
            __syncthreads();  // every thread is done with the previous tile
            for (int u = tid; u < stage; u += nt) {
                const int64_t i = base + u;
                uint4 rec = make_uint4(0u, 0u, 0u, 0u);
                if (i < end) {
                    rec = load_record<XYZQ>(pos, q, i, scx, scy, scz, status);
                    const float qf = __uint_as_float(rec.w);
                    ff_add(q2h, q2l, qf * qf);
                }
                sp[u] = rec;
            }
        }
        __syncthreads();
        if (!act) continue;  // idle threads only stage
        // this sub-stream's particles of the tile: [p0, p0 + n_here)
        const int n_here = (int)max((int64_t)0, min((int64_t)share, end - base - p0));
        float re[F], im[F], cre[F], cim[F];
        double are[F], aim[F];
#pragma unroll
        for (int f = 0; f < F; ++f) {
            re[f] = im[f] = cre[f] = cim[f] = 0.f;
            are[f] = aim[f] = 0.0;
        }
        if (ACC == RBE_RHO_COMP32) {
            // Compensated summation: the terms of kRhoGroup consecutive particles form an FP32
            // partial sum (four at a time from the staged records), and the partial sums are
            // added with Kahan's compensation (the rounding error of each addition carried into
            // the next), so the error does not grow with the number of particles: to first
            // order at most (kRhoGroup + 1) eps sum_i |q_i| (kRhoGroup - 1 eps from the
            // partials, 2 eps from the compensated additions; 17 eps for groups of 16).
            // Records past the end of the chunk are staged as zeros (q = 0), so the last group
            // is padded.
            const int ng = (n_here + kRhoGroup - 1) & ~(kRhoGroup - 1);
            for (int p = p0; p < p0 + ng; p += kRhoGroup) {
                float2 x[F];
#pragma unroll
                for (int h = 0; h < kRhoGroup; h += 4) {
                    const uint4 r0 = sp[p + h], r1 = sp[p + h + 1], r2 = sp[p + h + 2], r3 = sp[p + h + 3];
                    const float2 q0 = make_float2(__uint_as_float(r0.w), __uint_as_float(r0.w));
                    const float2 q1 = make_float2(__uint_as_float(r1.w), __uint_as_float(r1.w));
                    const float2 q2 = make_float2(__uint_as_float(r2.w), __uint_as_float(r2.w));
                    const float2 q3 = make_float2(__uint_as_float(r3.w), __uint_as_float(r3.w));
#pragma unroll
                    for (int f = 0; f < F; ++f) {
                        float2 e0, e1, e2, e3;  // (cos, sin) of the four phases
                        const float th0 = fixed_phase(mv[f].x, mv[f].y, mv[f].z, r0.x, r0.y, r0.z);
                        e0 = make_float2(mufu_cos(th0), mufu_sin(th0));
                        const float th1 = fixed_phase(mv[f].x, mv[f].y, mv[f].z, r1.x, r1.y, r1.z);
                        e1 = make_float2(mufu_cos(th1), mufu_sin(th1));
                        const float th2 = fixed_phase(mv[f].x, mv[f].y, mv[f].z, r2.x, r2.y, r2.z);
                        e2 = make_float2(mufu_cos(th2), mufu_sin(th2));
                        const float th3 = fixed_phase(mv[f].x, mv[f].y, mv[f].z, r3.x, r3.y, r3.z);
                        e3 = make_float2(mufu_cos(th3), mufu_sin(th3));
                        // (Re, Im) as packed pairs: each FP32x2 operation is the scalar one per lane
                        x[f] = h == 0 ? __fmul2_rn(q0, e0) : __ffma2_rn(q0, e0, x[f]);
                        x[f] = __ffma2_rn(q1, e1, x[f]);
                        x[f] = __ffma2_rn(q2, e2, x[f]);
                        x[f] = __ffma2_rn(q3, e3, x[f]);
                    }
                }
                const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    // the group's partial sum added with compensation (x - c is fma(c, -1, x),
                    // rounded once like the subtraction)
                    const float2 acc = make_float2(re[f], im[f]), cmp = make_float2(cre[f], cim[f]);
                    const float2 y = __ffma2_rn(cmp, m1, x[f]);
                    const float2 t = __fadd2_rn(acc, y);
                    const float2 c = __ffma2_rn(y, m1, __ffma2_rn(acc, m1, t));
                    re[f] = t.x;
                    im[f] = t.y;
                    cre[f] = c.x;
                    cim[f] = c.y;
                }
            }
        } else {
#pragma unroll 2
            for (int p = p0; p < p0 + n_here; ++p) {
                const uint4 r = sp[p];
                const float qp = __uint_as_float(r.w);
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    const float th = fixed_phase(mv[f].x, mv[f].y, mv[f].z, r.x, r.y, r.z);
                    const float sn = mufu_sin(th), cs = mufu_cos(th);
                    if (ACC == RBE_RHO_FP32) {
                        re[f] = fmaf(qp, cs, re[f]);
                        im[f] = fmaf(qp, sn, im[f]);
                    } else {
                        are[f] = fma((double)qp, (double)cs, are[f]);
                        aim[f] = fma((double)qp, (double)sn, aim[f]);
                    }
                }
            }
        }
#pragma unroll
        for (int f = 0; f < F; ++f) {
            float4 a = acc_s[(ss * F + f) * T + j];
            if (ACC == RBE_RHO_FP64) {
                const float ah = (float)are[f], bh = (float)aim[f];
                ff_add2(a.x, a.y, ah, (float)(are[f] - (double)ah));
                ff_add2(a.z, a.w, bh, (float)(aim[f] - (double)bh));
            } else {
                ff_add(a.x, a.y, re[f]);
                a.y -= cre[f];
                ff_add(a.z, a.w, im[f]);
                a.w -= cim[f];
            }
            acc_s[(ss * F + f) * T + j] = a;
        }
    }
    if (tid == 0 && bad) atomicOr(status, kStatusNonFinite);  // flagged while staging the first tile
    if (S > 1) __syncthreads();  // every sub-stream's sums are in shared memory
    if (ss == 0) {
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const int l = lbase + f * T;
            float4 a = acc_s[f * T + j];
            for (int u = 1; u < S; ++u) {  // sub-streams in order
                const float4 b = acc_s[(u * F + f) * T + j];
                ff_add2(a.x, a.y, b.x, b.y);
                ff_add2(a.z, a.w, b.z, b.w);
            }
            if (l < K) partials[(size_t)l * nchunks + c] = a;
        }
    }
    if (kt == 0) {
        block_sum_ff(q2h, q2l, red);  // sum of q^2 over the chunk, for E_self
        if (tid == 0) partials[(size_t)K * nchunks + c] = make_float4(q2h, q2l, 0.f, 0.f);
    }
}

// =================================================================================
// Reduction for the FP32-phase path.  Block l (of K + 1; whole warps, at most kReduceThreads)
// sums row l of the partials over the chunks as float-float in a fixed order; thread 0 then widens rho_l to FP64 and forms
// the per-frequency energy and virial terms in FP64 (App. C Eq. (pressuretensorflexible):
// |rho|^2 of a float-float rho, the importance weight, 1/|k|^2 and the k k products), and the
// force pass's FP32 coefficients.  Row K carries the sum of q^2.  The sums over l run in the
// force launch (k_force_f32's extra block, final_sums), concurrently with the force pass.
//
// GB300 runs FP64 at a low rate and long latency, so the FP64 work of a frequency is split:
// everything that does not depend on rho_l (1/|k|^2 and the tensor factors, freq_pre) is
// formed before the reduction, while the partial sums are still being written, and only a few
// multiplications follow it (freq_post).
__device__ __forceinline__ double ff_to_double(float hi, float lo)
{
    return __longlong_as_double((long long)float_to_double_bits(__float_as_uint(hi))) +
           __longlong_as_double((long long)float_to_double_bits(__float_as_uint(lo)));
}

// The rho-independent factors of frequency m with weight w:
//   c[0] = (2 pi / V) w / |k|^2                 (e = c[0] |rho|^2)
//   c[1..3] = 1 - b k_a^2, c[4..6] = -b k_x k_y, -b k_x k_z, -b k_y k_z,  b = 2 (1/|k|^2 + 1/4a)
//   c[7] = (4 pi / V) w / |k|^2                 (the force amplitude R = c[7] |rho|)
__device__ __forceinline__ void freq_pre(int4 mi, double wd, const KState* __restrict__ ks, double* __restrict__ c)
{
    const double kx = 2.0 * kPi * (double)mi.x * ks->inv[0];
    const double ky = 2.0 * kPi * (double)mi.y * ks->inv[1];
    const double kz = 2.0 * kPi * (double)mi.z * ks->inv[2];
    const double kk = kx * kx + ky * ky + kz * kz;
    const double ikk = 1.0 / kk;
    const double wk = wd * ikk;
    const double b = 2.0 * (ikk + ks->inv4a);
    c[0] = ks->ce * wk;
    c[1] = 1.0 - b * kx * kx;
    c[2] = 1.0 - b * ky * ky;
    c[3] = 1.0 - b * kz * kz;
    c[4] = -b * kx * ky;
    c[5] = -b * kx * kz;
    c[6] = -b * ky * kz;
    c[7] = ks->cb * wk;
}

// Energy and virial terms of one frequency in FP64 into t[0..6] (e = c[0] |rho|^2 and
// e [delta - 2 (1/|k|^2 + 1/4a) k k] as xx, yy, zz, xy, xz, yz), and the force pass's data:
// Im(e^{-ik.r} rho) = |rho| sin(arg rho - theta), so the pass takes one sine per pair of the
// phase shifted by arg rho (harmonic addition), its amplitude R = c[7] |rho| folded into the
// FP32 coefficients, and arg rho as a 32-bit fixed-point offset of the phase.
__device__ __forceinline__ void freq_post(int4 mi, const double* __restrict__ c, double re, double im,
                                          double* __restrict__ t, int4* __restrict__ cm, float4* __restrict__ cf)
{
    const double rho2 = re * re + im * im;
    const double e = c[0] * rho2;
    t[0] = e;
#pragma unroll
    for (int a = 1; a < 7; ++a) t[a] = e * c[a];
    t[7] = 0.0;
    const float Rf = (float)c[7] * sqrtf((float)rho2);
    const double phi = (double)atan2f((float)im, (float)re) * 683565275.57643158978;  // revolutions x 2^32
    const uint32_t off = 0x80000100u - (uint32_t)(unsigned long long)__double2ll_rn(phi);
    *cm = make_int4(mi.x, mi.y, mi.z, (int)off);
    *cf = make_float4(Rf, Rf * (float)mi.x, Rf * (float)mi.y, Rf * (float)mi.z);
}

// Row sums by one warp (lane-strided float-float sums over the chunks, then a fixed shuffle
// tree; every lane ends with the total), and the outputs of row l from its sum: the batched
// kernel sums four rows per warp and finishes 32 rows at once on the lanes of one warp, so
// that a row's FP64 work is one lane of a warp instruction, not a warp instruction of its own.
__device__ __forceinline__ double2 warp_row_sum(const float4* __restrict__ row, int nchunks)
{
    const int lane = threadIdx.x & 31;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int j = lane; j < nchunks; j += 32) {
        const float4 v = row[j];
        ff_add2(rh, rl, v.x, v.y);
        ff_add2(ih, il, v.z, v.w);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float a = __shfl_xor_sync(0xffffffffu, rh, off), b = __shfl_xor_sync(0xffffffffu, rl, off);
        const float c = __shfl_xor_sync(0xffffffffu, ih, off), d = __shfl_xor_sync(0xffffffffu, il, off);
        ff_add2(rh, rl, a, b);
        ff_add2(ih, il, c, d);
    }
    return make_double2(ff_to_double(rh, rl), ff_to_double(ih, il));
}

// Row l's outputs from its sum (re, im) and its factors c (freq_pre; unused for l == K, the
// row of the sum of q^2).
__device__ __forceinline__ void row_finish(int l, int K, double re, double im, int4 mi, const double* __restrict__ c,
                                           double2* __restrict__ rho, double* __restrict__ terms,
                                           int4* __restrict__ coef_m, float4* __restrict__ coef_f,
                                           unsigned* __restrict__ status)
{
    double* t = terms + (size_t)l * 8;
    if (l == K) {
        t[0] = re;  // sum of q^2
        return;
    }
    freq_post(mi, c, re, im, t, coef_m + l, coef_f + l);
    rho[l] = make_double2(re, im);
    if (!isfinite(re) || !isfinite(im)) atomicOr(status, kStatusNonFinite);
}

__device__ __forceinline__ void reduce_f32_row(int l, const float4* __restrict__ partials, int nchunks, int K,
                                               const int4* __restrict__ m,
             const double* __restrict__ w, const KState* __restrict__ ks, double2* __restrict__ rho,
             double* __restrict__ terms, int4* __restrict__ coef_m, float4* __restrict__ coef_f,
             unsigned* __restrict__ status)
{
    __shared__ float red[4][32];
    // the sampler completed before the rho pass passed its wait, and the rho pass lets this
    // launch start only after that wait: m, w and ks are final here
    int4 mi = make_int4(0, 0, 0, 0);
    double c[8];
    if (threadIdx.x == 0 && l < K) {
        mi = m[l];
        freq_pre(mi, w[l], ks, c);
    }
    pdl_wait();
    pdl_trigger();
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    const float4* row = partials + (size_t)l * nchunks;
    for (int j = threadIdx.x; j < nchunks; j += blockDim.x) {
        const float4 v = row[j];
        ff_add2(rh, rl, v.x, v.y);
        ff_add2(ih, il, v.z, v.w);
    }
    block_sum_ff2(rh, rl, ih, il, red);
    if (threadIdx.x != 0) return;
    row_finish(l, K, ff_to_double(rh, rl), ff_to_double(ih, il), mi, c, rho, terms, coef_m, coef_f, status);
}

// Energy and virial: fixed-order FP64 sums of the per-frequency terms over l by one block of
// kForceWarps warps; E_self = cself sum q^2 in FP64.  Lane (part p = lane / 8, term a = lane
// % 8) of warp v sums term a of rows l = 4 (v + kForceWarps i) + p, i = 0, 1, ... in order
// (one FP64 add per row and lane: a warp instruction covers four rows of all seven terms);
// the four parts are then combined by a fixed shuffle pair and the warps in order.
__device__ __forceinline__ void final_sums(const double* __restrict__ terms, int K, const KState* __restrict__ ks,
                                           double* __restrict__ W_out, double* __restrict__ E_out,
                                           unsigned* __restrict__ status)
{
    __shared__ double fin[kForceWarps][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = lane >> 3, a = lane & 7;
    double acc = 0.0;
    for (int l = 4 * warp + p; l < K; l += 4 * kForceWarps) acc += terms[(size_t)l * 8 + a];
    acc += __shfl_xor_sync(0xffffffffu, acc, 8);
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    if (lane < 8) fin[warp][lane] = acc;
    __syncthreads();
    // thread a (< 7) finishes term a; thread 7 the self energy
    if (threadIdx.x < 8) {
        double v = 0.0;
        if (a < 7) {
            for (int wv = 0; wv < kForceWarps; ++wv) v += fin[wv][a];
        } else {
            v = ks->cself * terms[(size_t)K * 8];
        }
        if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
        if (a == 0 && E_out) E_out[0] = v;
        if (a == 7 && E_out) E_out[1] = v;
        if (W_out) {
            if (a == 1) W_out[0] = v;
            if (a == 2) W_out[4] = v;
            if (a == 3) W_out[8] = v;
            if (a == 4) { W_out[1] = v; W_out[3] = v; }
            if (a == 5) { W_out[2] = v; W_out[6] = v; }
            if (a == 6) { W_out[5] = v; W_out[7] = v; }
        }
    }
}

// =================================================================================
// Force pass, FP32-phase path (Eq. (appforce)).  Block b owns particles [b * per_block,
// (b+1) * per_block); its warps take whole rounds of kForceRound particles (kForcePPT per lane,
// read from global memory straight into registers as fixed-point records) over all K
// frequencies, warp w the rounds w, w + warps, ... of the block, so that no partial force
// crosses warps (no shared-memory sums, no block barrier per round).  The frequencies are
// staged in shared memory as (mx, my, mz, off_l) and (R_l, R_l mx, R_l my, R_l mz), R_l =
// beta_l |rho_l| and off_l the fixed-point phase offset of arg rho_l: once per block when K <=
// kForceStageK, else kForceStageK at a time for every round (the warps then run the same number
// of rounds, idle ones included, around the staging barriers).  No FP64 instruction runs:
//   F_i,theta = q_i (2 pi / l_theta) sum_l R_l m_l,theta sin(theta_il - arg rho_l)
// (one sine per pair) is one FP32 sum over l = 0 .. K - 1 in order, widened to double exactly.
// The launch carries one extra block that computes the energy and virial sums (final_sums)
// meanwhile.
template <bool XYZQ = false, int LU = kForceLUnroll>
__device__ __forceinline__ void force_f32_block(int64_t blk, const void* __restrict__ pos,
                                                const double* __restrict__ q, int64_t N, int64_t per_block,
                                                const KState* __restrict__ ks, const int4* __restrict__ coef_m,
                                                const float4* __restrict__ coef_f, int K, double* __restrict__ F,
                                                unsigned* __restrict__ status)
{
    extern __shared__ int4 s_dyn[];
    __shared__ unsigned bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = (int)(blockDim.x >> 5);
    const int kstage = min(K, kForceStageK);
    int4* sm = s_dyn;
    float4* sf = reinterpret_cast<float4*>(s_dyn + kstage);
    unsigned long long* Fb = reinterpret_cast<unsigned long long*>(F);
    const FixScale scx = fs(ks->sc[0]), scy = fs(ks->sc[1]), scz = fs(ks->sc[2]);
    const float cx = ks->cx, cy = ks->cy, cz = ks->cz;
    const int64_t b0 = blk * per_block;
    const int64_t b1 = min(N, b0 + per_block);
    const bool multi = K > kstage;
    const int64_t nround = b1 > b0 ? (b1 - b0 + kForceRound - 1) / kForceRound : 0;
    const int64_t rlim = multi ? (nround + nwarps - 1) / nwarps * nwarps : nround;
    if (tid == 0) bad = 0u;
    __syncthreads();
    uint4 pr[kForcePPT];
    // the first round's records are read before waiting for the reduction (inputs only)
#pragma unroll
    for (int p = 0; p < kForcePPT; ++p) {
        const int64_t i = b0 + (int64_t)warp * kForceRound + 32 * p + lane;
        pr[p] = i < b1 ? load_record<XYZQ>(pos, q, i, scx, scy, scz, &bad) : make_uint4(0u, 0u, 0u, 0u);
    }
    pdl_wait();
    if (!multi) {
        for (int j = tid; j < K; j += blockDim.x) {
            sm[j] = coef_m[j];
            sf[j] = coef_f[j];
        }
    }
    __syncthreads();  // the frequencies staged; every first-round flag raised
    if (tid == 0 && bad) atomicOr(status, kStatusNonFinite);
    for (int64_t r = warp; r < rlim; r += nwarps) {
        const int64_t base = b0 + r * kForceRound;
        if (r != warp) {
#pragma unroll
            for (int p = 0; p < kForcePPT; ++p) {
                const int64_t i = base + 32 * p + lane;
                pr[p] = i < b1 ? load_record<XYZQ>(pos, q, i, scx, scy, scz, status) : make_uint4(0u, 0u, 0u, 0u);
            }
        }
        float gx[kForcePPT], gy[kForcePPT], gz[kForcePPT];
#pragma unroll
        for (int p = 0; p < kForcePPT; ++p) gx[p] = gy[p] = gz[p] = 0.f;
        for (int k0 = 0; k0 < K; k0 += kstage) {
            const int nk = min(kstage, K - k0);
            if (multi) {
                __syncthreads();
                for (int j = tid; j < nk; j += blockDim.x) {
                    sm[j] = coef_m[k0 + j];
                    sf[j] = coef_f[k0 + j];
                }
                __syncthreads();
            }
            if (r < nround) {
#pragma unroll LU
                for (int l = 0; l < nk; ++l) {
                    const int4 a = sm[l];
                    const float4 b = sf[l];
#pragma unroll
                    for (int p = 0; p < kForcePPT; ++p) {
                        const float g = mufu_sin(fixed_phase_off(a.x, a.y, a.z, pr[p].x, pr[p].y, pr[p].z,
                                                               (uint32_t)a.w));
                        gx[p] = fmaf(g, b.y, gx[p]);
                        gy[p] = fmaf(g, b.z, gy[p]);
                        gz[p] = fmaf(g, b.w, gz[p]);
                    }
                }
            }
        }
        if (r < nround) {
#pragma unroll
            for (int p = 0; p < kForcePPT; ++p) {
                const int64_t i = base + 32 * p + lane;
                if (i < b1) {
                    const float qf = __uint_as_float(pr[p].w);
                    Fb[3 * i] = float_to_double_bits(__float_as_uint(qf * cx * gx[p]));
                    Fb[3 * i + 1] = float_to_double_bits(__float_as_uint(qf * cy * gy[p]));
                    Fb[3 * i + 2] = float_to_double_bits(__float_as_uint(qf * cz * gz[p]));
                }
            }
        }
    }
}

}  // namespace rbe
