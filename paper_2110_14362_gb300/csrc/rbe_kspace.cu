// RBE k-space kernels for sm_103a and their launchers (the FP32-phase bodies live in
// rbe_kspace_tiles.cuh, shared with the batched kernels of rbe_batch.cu).
//
// One evaluation (Sec. 4.2 of the paper) is up to five launches on the context's stream:
//   k_tables   per-axis weights exp(-c m^2) as exact integers, their cumulative sums, H,
//              S and the box constants (KState)                            Eqs. (S), (psf)
//              (only when the box changed; the box may come from the host or the device)
//   k_sample   one thread per frequency: Philox -> 3 uniforms -> inverse CDF  Eq. (probexpression)
//   k_rho_*    particle-chunk x frequency-tile blocks: partial rho(k_l) per chunk
//   k_reduce*  fixed-order sum of the partials -> rho(k_l), the per-frequency terms and
//              force coefficients (and, on the FP64 path, the energy and virial)
//                                              Eq. (apppress); App. C Eq. (pressuretensorflexible)
//   k_force_*  particle tiles x all frequencies: F_i                             Eq. (appforce)
// No floating-point atomics: every sum runs in an order fixed by (N, K, plan), so
// results are bitwise reproducible run to run.  The host-buffer call can run the passes in
// two particle groups with its copies pipelined (launch_evaluate_staged).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "rbe_context.h"
#include "rbe_device.cuh"
#include "rbe_kspace_tiles.cuh"
#include "rbe_sampler_variants.cuh"

namespace rbe {

// Rho-pass planning constants (compile-time): particle sub-streams per block at most, the
// fewest particles per chunk, and the most pairs N K of the latency-bound regime (one short
// wave: one frequency per thread and no sub-streams run it fastest).  RBE_RHO_FORCE_F, when
// defined, fixes the frequencies per thread (1, 2 or 4) for tuning.
#ifndef RBE_RHO_MAXSUB
#define RBE_RHO_MAXSUB 4
#endif
#ifndef RBE_RHO_MINCHUNK
#define RBE_RHO_MINCHUNK 64
#endif
#ifndef RBE_RHO_LATENCY_PAIRS
#define RBE_RHO_LATENCY_PAIRS 2.0e7
#endif
// Fewest particle rounds per block of the FP32 force pass: below four, a block's warps mostly
// idle at small N and hold resident slots that concurrent replicas' kernels could use (the
// serving loop, 256 replicas of 1e3-1e5 charges: 21.3k replica-steps/s at one round per block,
// 22.0k at four, 22.2k at eight, which slows a lone replica at N = 1e3 by 2 %).
#ifndef RBE_FORCE_MIN_ROUNDS
#define RBE_FORCE_MIN_ROUNDS 4
#endif
constexpr int kRhoMaxSub = RBE_RHO_MAXSUB;
constexpr int kRhoWideMaxSub = 8;  // particle sub-streams of a wide two-frequency tile at most
#ifndef RBE_RHO_WIDE_MAXKT
#define RBE_RHO_WIDE_MAXKT 1  // frequency tiles of a wide plan at most (slab: one tile 39.1 us, two 40.2 us)
#endif
constexpr int kRhoMinChunk = RBE_RHO_MINCHUNK;
constexpr double kRhoLatencyPairs = RBE_RHO_LATENCY_PAIRS;

constexpr int kT = 128;               // threads per block of the FP64 force pass
constexpr int kForceKT = 256;         // frequencies staged per tile in the FP64 force pass

__global__ void __launch_bounds__(kTableThreads)
k_tables(double bx, double by, double bz, const double* __restrict__ box_dev, double alpha, int P,
         unsigned long long* __restrict__ cum, int cap, KState* __restrict__ ks, unsigned* __restrict__ status)
{
    tables_body(bx, by, bz, box_dev, alpha, P, cum, cap, ks, status);
}

// Tables of the device box and the sampler in one block (the NPT step, where the box changes
// every step): one launch instead of two, the tables read back from this block's own writes.
// reuse > 1 (samples kept for `reuse` steps, Sec. 4.3): at a step s with s mod reuse = 0 the
// block draws reuse * P slots (counter step s, slot i P + l for batch i) from this step's tables
// into m_all; step s + i takes batch i, with the weights of its own (current) tables.
__global__ void __launch_bounds__(kTableThreads)
k_tables_sample(const double* __restrict__ box_dev, double alpha, int Pf, int P, unsigned long long* __restrict__ cum,
                int cap, int smem_cap, KState* __restrict__ ks, uint64_t seed,
                const unsigned long long* __restrict__ step_dev, int4* __restrict__ m_out,
                double* __restrict__ w_out, unsigned* __restrict__ status, int mode, int4* __restrict__ chain,
                int reuse, int4* __restrict__ m_all)
{
    tables_body(0.0, 0.0, 0.0, box_dev, alpha, Pf, cum, cap, ks, status);
    __syncthreads();
    if (reuse <= 1) {
        for (int lb = 0; lb < P; lb += kTableThreads) {
            if (mode == kSamplerExact)
                sample_body(lb, seed, 0, step_dev, P, Pf, cum, cap, smem_cap, ks, m_out, w_out, status);
            else
                sample_variant_body(lb, seed, 0, step_dev, P, Pf, cum, cap, ks, mode, chain, m_out, w_out, status);
        }
        return;
    }
    const uint64_t step = *step_dev;
    const int i = (int)(step % (uint64_t)reuse);  // the same for every thread
    if (i == 0) {
        const int Pall = reuse * P;
        for (int lb = 0; lb < Pall; lb += kTableThreads) {
            if (mode == kSamplerExact)
                sample_body(lb, seed, 0, step_dev, Pall, Pall, cum, cap, smem_cap, ks, m_all, nullptr, status);
            else
                sample_variant_body(lb, seed, 0, step_dev, Pall, Pall, cum, cap, ks, mode, chain, m_all, nullptr,
                                    status);
        }
        __syncthreads();
    }
    pdl_trigger();
    const double wP = ks->wP, wT = P > Pf ? ks->S / (double)(P - Pf) : 0.0;
    for (int l = threadIdx.x; l < P; l += kTableThreads) {
        m_out[l] = m_all[(size_t)i * P + l];
        w_out[l] = l < Pf ? wP : wT;
    }
}

// Frequency sampling, one thread per frequency (body in rbe_kspace_tiles.cuh).
__global__ void k_sample(uint64_t seed, uint64_t step_arg, const unsigned long long* __restrict__ step_dev, int P, int Pf,
                         const unsigned long long* __restrict__ cum, int cap, int smem_cap,
                         const KState* __restrict__ ks, int4* __restrict__ m_out, double* __restrict__ w_out,
                         unsigned* __restrict__ status, int mode, int4* __restrict__ chain)
{
    // the mode is the same for every thread: the exact sampler's code path is unchanged
    if (mode == kSamplerExact)
        sample_body((int)(blockIdx.x * blockDim.x), seed, step_arg, step_dev, P, Pf, cum, cap, smem_cap, ks, m_out,
                    w_out, status);
    else
        sample_variant_body((int)(blockIdx.x * blockDim.x), seed, step_arg, step_dev, P, Pf, cum, cap, ks, mode,
                            chain, m_out, w_out, status);
}

// Caller-given frequencies and weights (weighted mode).
__global__ void k_weights_from_list(int K, const int32_t* __restrict__ m3, const double* __restrict__ w,
                                    int4* __restrict__ m_out, double* __restrict__ w_out)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= K) return;
    m_out[l] = make_int4(m3[3 * l], m3[3 * l + 1], m3[3 * l + 2], 0);
    w_out[l] = w[l];
}

// Fixed-order block sum of one double per thread (warp shuffles, then warp 0); the
// result is valid in thread 0.  blockDim.x is a multiple of 32, at most 1024.
__device__ __forceinline__ double block_sum(double v, double* scratch32)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch32[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? scratch32[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    }
    return v;
}

// Block (kt, c) handles frequency tile kt and particle chunk c_off + c (c_off: the first chunk
// of a piece when the staged host call feeds the pass piece by piece).
// F frequencies per thread: blocks of at most kMaxRhoThreads threads for F = 1, kRhoThreadsF
// threads for F = 2 and 4.
// XYZQ: positions and charges as one float4 (x, y, z, q) per particle in pos (q unused).
template <int ACC, int F, bool XYZQ>
#ifndef RBE_RHO_MINB_F
#define RBE_RHO_MINB_F 8
#endif
__global__ void __launch_bounds__(F == 1 ? kMaxRhoThreads : kRhoThreadsF, F == 1 ? 6 : RBE_RHO_MINB_F)
k_rho_f32(const void* __restrict__ pos, const double* __restrict__ q, int64_t N, const KState* __restrict__ ks,
          const int4* __restrict__ m, int K, int64_t chunk_len, int nchunks, float4* __restrict__ partials,
          unsigned* __restrict__ status, int c_off, int S)
{
    rho_f32_tile<ACC, F, XYZQ>((int)blockIdx.x, c_off + (int)blockIdx.y, pos, q, N, ks, m, K, chunk_len, nchunks,
                               partials, status, S);
}

// Two frequencies per thread in blocks of up to kMaxRhoThreads threads with any lane count T
// (a tile of 2 T frequencies, S = threads / T particle sub-streams, the threads beyond S T idle):
// small K, where the kRhoThreadsF-thread tiles of k_rho_f32<ACC, 2> would leave lanes without a
// frequency (K = 200: one tile of 100 lanes in two sub-streams).
#ifndef RBE_RHO_WIDE_MINB
#define RBE_RHO_WIDE_MINB 4
#endif
template <int ACC, bool XYZQ>
__global__ void __launch_bounds__(kMaxRhoThreads, RBE_RHO_WIDE_MINB)
k_rho_f32_wide(const void* __restrict__ pos, const double* __restrict__ q, int64_t N, const KState* __restrict__ ks,
               const int4* __restrict__ m, int K, int64_t chunk_len, int nchunks, float4* __restrict__ partials,
               unsigned* __restrict__ status, int c_off, int S, int T)
{
    rho_f32_tile<ACC, 2, XYZQ, kMaxRhoThreads>((int)blockIdx.x, c_off + (int)blockIdx.y, pos, q, N, ks, m, K,
                                               chunk_len, nchunks, partials, status, S, T);
}

using RhoKernel = void (*)(const void*, const double*, int64_t, const KState*, const int4*, int, int64_t, int,
                           float4*, unsigned*, int, int);
using RhoWideKernel = void (*)(const void*, const double*, int64_t, const KState*, const int4*, int, int64_t, int,
                               float4*, unsigned*, int, int, int);

template <int ACC, bool XYZQ>
static RhoKernel rho_kernel_f(int F)
{
    return F == 4 ? k_rho_f32<ACC, 4, XYZQ> : (F == 2 ? k_rho_f32<ACC, 2, XYZQ> : k_rho_f32<ACC, 1, XYZQ>);
}

template <bool XYZQ>
static RhoKernel rho_kernel_x(int accum, int F)
{
    return accum == RBE_RHO_FP64     ? rho_kernel_f<RBE_RHO_FP64, XYZQ>(F)
           : accum == RBE_RHO_COMP32 ? rho_kernel_f<RBE_RHO_COMP32, XYZQ>(F)
                                     : rho_kernel_f<RBE_RHO_FP32, XYZQ>(F);
}

static RhoKernel rho_kernel(int accum, int F, bool xyzq = false)
{
    return xyzq ? rho_kernel_x<true>(accum, F) : rho_kernel_x<false>(accum, F);
}

template <bool XYZQ>
static RhoWideKernel rho_wide_kernel_x(int accum)
{
    return accum == RBE_RHO_FP64     ? k_rho_f32_wide<RBE_RHO_FP64, XYZQ>
           : accum == RBE_RHO_COMP32 ? k_rho_f32_wide<RBE_RHO_COMP32, XYZQ>
                                     : k_rho_f32_wide<RBE_RHO_FP32, XYZQ>;
}

static RhoWideKernel rho_wide_kernel(int accum, bool xyzq = false)
{
    return xyzq ? rho_wide_kernel_x<true>(accum) : rho_wide_kernel_x<false>(accum);
}


// rho pass, FP64 path: s = r / l wrapped to [0, 1); t = m.s - rint(m.s); sincospi(2t).
__global__ void __launch_bounds__(kMaxRhoThreads)
k_rho_f64(const double* __restrict__ pos, const double* __restrict__ q, int64_t N, const KState* __restrict__ ks,
          const int4* __restrict__ m, int K, int64_t chunk_len, int nchunks, double2* __restrict__ partials,
          unsigned* __restrict__ status)
{
    __shared__ double4_32a sp[kMaxRhoThreads];
    __shared__ double red[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int l = blockIdx.x * nt + tid;
    const int c = blockIdx.y;
    const double ilx = ks->inv[0], ily = ks->inv[1], ilz = ks->inv[2];
    const int4 mv = l < K ? m[l] : make_int4(0, 0, 0, 0);
    const double mx = mv.x, my = mv.y, mz = mv.z;
    double re = 0.0, im = 0.0, q2 = 0.0;
    const int64_t start = (int64_t)c * chunk_len;
    const int64_t end = min(N, start + chunk_len);
    for (int64_t base = start; base < end; base += nt) {
        const int64_t i = base + tid;
        double4_32a rec = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        if (i < end) {
            double sx = pos[3 * i] * ilx, sy = pos[3 * i + 1] * ily, sz = pos[3 * i + 2] * ilz;
            sx -= floor(sx); sy -= floor(sy); sz -= floor(sz);
            const double qi = q[i];
            if (!isfinite(sx + sy + sz + qi)) atomicOr(status, kStatusNonFinite);
            q2 += qi * qi;
            rec = make_double4_32a(sx, sy, sz, qi);
        }
        sp[tid] = rec;
        __syncthreads();
        const int n_here = (int)min((int64_t)nt, end - base);
#pragma unroll 2
        for (int p = 0; p < n_here; ++p) {
            const double4_32a r = sp[p];
            double t = fma(mx, r.x, fma(my, r.y, mz * r.z));
            t -= rint(t);
            double sn, cs;
            sincospi(2.0 * t, &sn, &cs);
            re = fma(r.w, cs, re);
            im = fma(r.w, sn, im);
        }
        __syncthreads();
    }
    if (l < K) partials[(size_t)l * nchunks + c] = make_double2(re, im);
    if (blockIdx.x == 0) {
        const double s = block_sum(q2, red);
        if (tid == 0) partials[(size_t)K * nchunks + c] = make_double2(s, 0.0);
    }
}

// =================================================================================
// FP64 reduction: block l (of K + 1) sums its row over the chunks in a fixed order and
// forms the per-frequency terms; the last block to finish sums those over l.
//   e_l = (2 pi / V) w_l |rho_l|^2 / |k_l|^2
//   W  += e_l [I - 2 (1/|k_l|^2 + 1/4a) k_l k_l]
//   beta_l = w_l 4 pi / (V |k_l|^2), A_l = beta_l Im rho_l, B_l = beta_l Re rho_l, so that
//   F_i = q_i sum_l k_l (sin(k_l.r_i) B_l - cos(k_l.r_i) A_l).
__global__ void __launch_bounds__(kReduceThreads)
k_reduce(const double2* __restrict__ partials, int nchunks, int K, const int4* __restrict__ m,
         const double* __restrict__ w, const KState* __restrict__ ks, double2* __restrict__ rho,
         double* __restrict__ terms, double2* __restrict__ coef_d, unsigned* __restrict__ counter,
         unsigned* __restrict__ status, double* __restrict__ W_out, double* __restrict__ E_out)
{
    __shared__ double red[32];
    __shared__ double fin[kReduceThreads / 32][7];
    __shared__ bool is_last;
    const int l = blockIdx.x;
    double re = 0.0, im = 0.0;
    const double2* row = partials + (size_t)l * nchunks;
    for (int j = threadIdx.x; j < nchunks; j += kReduceThreads) {
        const double2 v = row[j];
        re += v.x;
        im += v.y;
    }
    re = block_sum(re, red);
    im = block_sum(im, red);
    const double alpha = ks->alpha;
    if (threadIdx.x == 0) {
        double* t = terms + (size_t)l * 8;
        if (l < K) {
            const int4 mi = m[l];
            const double bx = ks->L[0], by = ks->L[1], bz = ks->L[2];
            const double V = bx * by * bz;
            const double kx = 2.0 * kPi * mi.x / bx, ky = 2.0 * kPi * mi.y / by, kz = 2.0 * kPi * mi.z / bz;
            const double kk = kx * kx + ky * ky + kz * kz;
            const double rho2 = re * re + im * im;
            const double e = (2.0 * kPi / V) * w[l] * rho2 / kk;
            const double b = 2.0 * (1.0 / kk + 1.0 / (4.0 * alpha));
            t[0] = e;
            t[1] = e * (1.0 - b * kx * kx);
            t[2] = e * (1.0 - b * ky * ky);
            t[3] = e * (1.0 - b * kz * kz);
            t[4] = -e * b * kx * ky;
            t[5] = -e * b * kx * kz;
            t[6] = -e * b * ky * kz;
            t[7] = 0.0;
            const double beta = w[l] * (4.0 * kPi / (V * kk));
            rho[l] = make_double2(re, im);
            coef_d[l] = make_double2(beta * im, beta * re);
            if (!isfinite(re) || !isfinite(im)) atomicOr(status, kStatusNonFinite);
        } else {
            t[0] = re;  // sum of q^2
        }
        __threadfence();
        is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < K; j += kReduceThreads) {
        const double* t = terms + (size_t)j * 8;
#pragma unroll
        for (int a = 0; a < 7; ++a) acc[a] += __ldcg(t + a);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < 7; ++a) {
        double v = acc[a];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) fin[warp][a] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[7];
        for (int a = 0; a < 7; ++a) {
            tot[a] = 0.0;
            for (int wv = 0; wv < kReduceThreads / 32; ++wv) tot[a] += fin[wv][a];
        }
        const double q2 = __ldcg(terms + (size_t)K * 8);
        const double Ek = tot[0];
        const double Es = -sqrt(alpha / kPi) * q2;
        if (W_out) {
            W_out[0] = tot[1]; W_out[4] = tot[2]; W_out[8] = tot[3];
            W_out[1] = W_out[3] = tot[4];
            W_out[2] = W_out[6] = tot[5];
            W_out[5] = W_out[7] = tot[6];
        }
        if (E_out) { E_out[0] = Ek; E_out[1] = Es; }
        bool ok = isfinite(Ek) && isfinite(Es);
        for (int a = 1; a < 7; ++a) ok = ok && isfinite(tot[a]);
        if (!ok) atomicOr(status, kStatusNonFinite);
        *counter = 0u;  // ready for the next launch
    }
}

__global__ void __launch_bounds__(kReduceThreads)
k_reduce_f32(const float4* __restrict__ partials, int nchunks, int K, const int4* __restrict__ m,
             const double* __restrict__ w, const KState* __restrict__ ks, double2* __restrict__ rho,
             double* __restrict__ terms, int4* __restrict__ coef_m, float4* __restrict__ coef_f,
             unsigned* __restrict__ status)
{
    reduce_f32_row((int)blockIdx.x, partials, nchunks, K, m, w, ks, rho, terms, coef_m, coef_f, status);
}

// Force pass, FP32-phase path (body in rbe_kspace_tiles.cuh); the launch carries one extra
// block that computes the energy and virial sums (final_sums_f32) meanwhile.
// Blocks [0, gridDim.x - final) take particle blocks b_off + blockIdx.x; with final = 1 the
// last block computes the energy and virial sums.
template <bool XYZQ>
__global__ void __launch_bounds__(kForceThreads, RBE_FORCE_MINB)
k_force_f32(const void* __restrict__ pos, const double* __restrict__ q, int64_t N, int64_t per_block,
            const KState* __restrict__ ks, const int4* __restrict__ coef_m, const float4* __restrict__ coef_f,
            int K, double* __restrict__ F, unsigned* __restrict__ status, const double* __restrict__ terms,
            double* __restrict__ W_out, double* __restrict__ E_out, int64_t b_off, int final)
{
    if (final && blockIdx.x == gridDim.x - 1) {
        pdl_wait();
        final_sums(terms, K, ks, W_out, E_out, status);
        return;
    }
    force_f32_block<XYZQ>(b_off + (int64_t)blockIdx.x, pos, q, N, per_block, ks, coef_m, coef_f, K, F, status);
}

// Force pass, FP64 path: particle tiles of kT * PPT, frequencies staged kForceKT at a time.
template <int PPT>
__global__ void __launch_bounds__(kT) k_force_f64(const double* __restrict__ pos, const double* __restrict__ q,
                                                  int64_t N, int64_t per_block, const KState* __restrict__ ks,
                                                  const int4* __restrict__ mk, const double2* __restrict__ coef_d,
                                                  int K, double* __restrict__ F)
{
    __shared__ double4_32a sk[kForceKT];  // (mx, my, mz, A)
    __shared__ double sb[kForceKT];       // B
    const int tid = threadIdx.x;
    const double ilx = ks->inv[0], ily = ks->inv[1], ilz = ks->inv[2];
    const bool one_tile = K <= kForceKT;
    if (one_tile) {
        for (int j = tid; j < K; j += kT) {
            const int4 mm = mk[j];
            const double2 ab = coef_d[j];
            sk[j] = make_double4_32a((double)mm.x, (double)mm.y, (double)mm.z, ab.x);
            sb[j] = ab.y;
        }
        __syncthreads();
    }
    const int64_t b0 = (int64_t)blockIdx.x * per_block;
    const int64_t b1 = min(N, b0 + per_block);
    const double cx = 2.0 * kPi * ilx, cy = 2.0 * kPi * ily, cz = 2.0 * kPi * ilz;
    for (int64_t base = b0; base < b1; base += (int64_t)kT * PPT) {
        double sx[PPT], sy[PPT], sz[PPT], fx[PPT], fy[PPT], fz[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int64_t i = base + (int64_t)p * kT + tid;
            if (i < b1) {
                sx[p] = pos[3 * i] * ilx; sy[p] = pos[3 * i + 1] * ily; sz[p] = pos[3 * i + 2] * ilz;
                sx[p] -= floor(sx[p]); sy[p] -= floor(sy[p]); sz[p] -= floor(sz[p]);
            } else {
                sx[p] = sy[p] = sz[p] = 0.0;
            }
            fx[p] = fy[p] = fz[p] = 0.0;
        }
        for (int k0 = 0; k0 < K; k0 += kForceKT) {
            const int nk = min(kForceKT, K - k0);
            if (!one_tile) {
                __syncthreads();
                for (int j = tid; j < nk; j += kT) {
                    const int4 mm = mk[k0 + j];
                    const double2 ab = coef_d[k0 + j];
                    sk[j] = make_double4_32a((double)mm.x, (double)mm.y, (double)mm.z, ab.x);
                    sb[j] = ab.y;
                }
                __syncthreads();
            }
            for (int l = 0; l < nk; ++l) {
                const double4_32a a = sk[l];
                const double B = sb[l];
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    double t = fma(a.x, sx[p], fma(a.y, sy[p], a.z * sz[p]));
                    t -= rint(t);
                    double sn, cs;
                    sincospi(2.0 * t, &sn, &cs);
                    const double g = sn * B - cs * a.w;
                    fx[p] = fma(g, a.x, fx[p]);
                    fy[p] = fma(g, a.y, fy[p]);
                    fz[p] = fma(g, a.z, fz[p]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int64_t i = base + (int64_t)p * kT + tid;
            if (i < b1) {
                const double qi = q[i];
                F[3 * i] = qi * cx * fx[p];
                F[3 * i + 1] = qi * cy * fy[p];
                F[3 * i + 2] = qi * cz * fz[p];
            }
        }
    }
}

// =================================================================================
// Host launchers.

void record_event(rbe_ctx ctx, int idx)
{
    if (ctx->timing && ctx->ev[idx]) cudaEventRecord(ctx->ev[idx], ctx->stream);
}

static rbe_status check_launch(rbe_ctx ctx, const char* what)
{
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(ctx, err, what);
    return RBE_OK;
}

// Capacity of the table rows: the host estimate of 2M+1 with headroom for boxes that grow
// on the device.
rbe_status ensure_table_capacity(rbe_ctx ctx, int need)
{
    if (need <= ctx->d.tab_cap) return RBE_OK;
    if (ctx->d.cum) ctx_free(ctx, ctx->d.cum);
    ctx->d.cum = nullptr;
    ctx->d.tab_cap = 0;
    const int cap = need + need / 4 + 16;
    cudaError_t err = ctx_alloc(ctx, &ctx->d.cum, sizeof(unsigned long long) * 3 * (size_t)cap);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaMalloc(tables)");
    ctx->d.tab_cap = cap;
    return RBE_OK;
}

rbe_status launch_tables(rbe_ctx ctx, const double* box_dev)
{
    k_tables<<<1, kTableThreads, 0, ctx->stream>>>(ctx->box[0], ctx->box[1], ctx->box[2], box_dev, ctx->alpha,
                                                   ctx->P, ctx->d.cum, ctx->d.tab_cap, ctx->d.ks, ctx->d.status);
    return check_launch(ctx, "k_tables");
}

// Tables and box state of an explicit box (the general cell's proposal lengths and its unit cube);
// the context's own box tables are rebuilt at the next rectangular evaluation.
rbe_status launch_tables_box(rbe_ctx ctx, const double box[3])
{
    k_tables<<<1, kTableThreads, 0, ctx->stream>>>(box[0], box[1], box[2], nullptr, ctx->alpha, ctx->P, ctx->d.cum,
                                                   ctx->d.tab_cap, ctx->d.ks, ctx->d.status);
    ctx->tables_dirty = true;
    return check_launch(ctx, "k_tables");
}

rbe_status ensure_tables(rbe_ctx ctx)
{
    if (!ctx->tables_dirty) return RBE_OK;
    int need = 0;
    for (int t = 0; t < 3; ++t) need = std::max(need, 2 * host_axis_M(ctx->alpha, ctx->box[t]) + 1);
    rbe_status st = ensure_table_capacity(ctx, need);
    if (st != RBE_OK) return st;
    st = launch_tables(ctx, nullptr);
    if (st == RBE_OK) ctx->tables_dirty = false;
    return st;
}

rbe_status ensure_k_capacity(rbe_ctx ctx, int K)
{
    if (K <= ctx->d.kcap) return RBE_OK;
    DeviceBuffers& d = ctx->d;
    ctx_free(ctx, d.m); ctx_free(ctx, d.w); ctx_free(ctx, d.rho); ctx_free(ctx, d.terms);
    ctx_free(ctx, d.coef_m); ctx_free(ctx, d.coef_f); ctx_free(ctx, d.coef_d);
    d.m = nullptr; d.w = nullptr; d.rho = nullptr; d.terms = nullptr;
    d.coef_m = nullptr; d.coef_f = nullptr; d.coef_d = nullptr;
    d.kcap = 0;
    cudaError_t err = cudaSuccess;
    if ((err = ctx_alloc(ctx, &d.m, sizeof(int4) * K)) != cudaSuccess ||
        (err = ctx_alloc(ctx, &d.w, sizeof(double) * K)) != cudaSuccess ||
        (err = ctx_alloc(ctx, &d.rho, sizeof(double2) * K)) != cudaSuccess ||
        (err = ctx_alloc(ctx, &d.terms, sizeof(double) * 8 * (size_t)(K + 1))) != cudaSuccess ||
        (err = ctx_alloc(ctx, &d.coef_m, sizeof(int4) * K)) != cudaSuccess ||
        (err = ctx_alloc(ctx, &d.coef_f, sizeof(float4) * K)) != cudaSuccess ||
        (err = ctx_alloc(ctx, &d.coef_d, sizeof(double2) * K)) != cudaSuccess)
        return cuda_fail(ctx, err, "cudaMalloc(frequency buffers)");
    d.kcap = K;
    return RBE_OK;
}

constexpr int kSampleSmemMax = 48 * 1024;

rbe_status launch_sample(rbe_ctx ctx, uint64_t step, int P)
{
    rbe_status st = ensure_tables(ctx);
    if (st != RBE_OK) return st;
    return launch_sample_device_box(ctx, step, P, nullptr);
}

// The sampler on the tables already on the device (built by launch_tables from any box);
// step_dev, when not NULL, points at a device-resident step index used instead of step.
// The MH chain holds one state per frequency slot; a sampling call for more slots than it holds
// is refused (rbe_set_sampler sizes it for the context's P).
static rbe_status check_chain(rbe_ctx ctx, int P)
{
    if (ctx->sampler == kSamplerMH && (!ctx->chain || ctx->chain_cap < P))
        return fail(ctx, RBE_ESTATE, "the Metropolis-Hastings chain holds fewer slots than this call samples");
    return RBE_OK;
}

// P is the force batch; with a pressure batch (ctx->Ptilde > 0) the sampler draws P + Ptilde
// slots, the pressure batch in slots [P, P + Ptilde) (Philox slot counters continue past P).
rbe_status launch_sample_device_box(rbe_ctx ctx, uint64_t step, int P, const unsigned long long* step_dev)
{
    const int Ptot = P + ctx->Ptilde;
    rbe_status st = ensure_k_capacity(ctx, Ptot);
    if (st != RBE_OK) return st;
    if ((st = check_chain(ctx, Ptot)) != RBE_OK) return st;
    record_event(ctx, 0);
    if (ctx->sampler == kSamplerMH) {
        k_sample_mh<<<(Ptot + kMhSlots - 1) / kMhSlots, kMhWarps * 32, 0, ctx->stream>>>(
            ctx->seed, step, step_dev, Ptot, P, ctx->d.cum, ctx->d.tab_cap, ctx->d.ks, ctx->chain, ctx->d.m,
            ctx->d.w, ctx->d.status);
        record_event(ctx, 1);
        return check_launch(ctx, "k_sample_mh");
    }
    const int threads = 128;
    const size_t smem = sizeof(unsigned long long) * 3 * (size_t)ctx->d.tab_cap;
    const int smem_cap = smem <= (size_t)kSampleSmemMax ? ctx->d.tab_cap : 0;
    k_sample<<<(Ptot + threads - 1) / threads, threads, smem_cap ? smem : 0, ctx->stream>>>(
        ctx->seed, step, step_dev, Ptot, P, ctx->d.cum, ctx->d.tab_cap, smem_cap, ctx->d.ks, ctx->d.m, ctx->d.w,
        ctx->d.status, ctx->sampler, ctx->chain);
    record_event(ctx, 1);
    return check_launch(ctx, "k_sample");
}

// The NPT step's tables (from the device box) and sampler (at the device step index) in one
// launch.
rbe_status launch_tables_sample_device(rbe_ctx ctx, int P, const double* box_dev, const unsigned long long* step_dev)
{
    const int Ptot = P + ctx->Ptilde;
    rbe_status st = ensure_k_capacity(ctx, Ptot);
    if (st != RBE_OK) return st;
    if ((st = check_chain(ctx, Ptot)) != RBE_OK) return st;
    const int reuse = ctx->reuse > 1 ? ctx->reuse : 1;
    if (reuse > 1) {
        if (ctx->sampler == kSamplerMH)
            return fail(ctx, RBE_ESTATE, "sample reuse and the Metropolis-Hastings chain exclude each other");
        const int64_t need = (int64_t)reuse * Ptot;
        if (need > ctx->m_all_cap) {
            ctx_free(ctx, ctx->m_all);
            ctx->m_all = nullptr;
            ctx->m_all_cap = 0;
            cudaError_t e = ctx_alloc(ctx, &ctx->m_all, sizeof(int4) * (size_t)need);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMallocAsync(reused samples)");
            ctx->m_all_cap = need;
        }
    }
    record_event(ctx, 0);
    const size_t smem = sizeof(unsigned long long) * 3 * (size_t)ctx->d.tab_cap;
    const int smem_cap = smem <= (size_t)kSampleSmemMax ? ctx->d.tab_cap : 0;
    // the MH chain runs in its own multi-warp launch after the tables (k_sample_mh)
    const bool mh = ctx->sampler == kSamplerMH;
    k_tables_sample<<<1, kTableThreads, smem_cap ? smem : 0, ctx->stream>>>(
        box_dev, ctx->alpha, P, mh ? 0 : Ptot, ctx->d.cum, ctx->d.tab_cap, smem_cap, ctx->d.ks, ctx->seed, step_dev,
        ctx->d.m, ctx->d.w, ctx->d.status, ctx->sampler, ctx->chain, reuse, ctx->m_all);
    if (mh) {
        if ((st = check_launch(ctx, "k_tables_sample")) != RBE_OK) return st;
        k_sample_mh<<<(Ptot + kMhSlots - 1) / kMhSlots, kMhWarps * 32, 0, ctx->stream>>>(
            ctx->seed, 0, step_dev, Ptot, P, ctx->d.cum, ctx->d.tab_cap, ctx->d.ks, ctx->chain, ctx->d.m, ctx->d.w,
            ctx->d.status);
    }
    record_event(ctx, 1);
    return check_launch(ctx, mh ? "k_sample_mh" : "k_tables_sample");
}

rbe_status launch_weights_from_list(rbe_ctx ctx, int K, const int32_t* m, const double* w)
{
    rbe_status st = ensure_tables(ctx);  // the box constants live in the same state
    if (st != RBE_OK) return st;
    st = ensure_k_capacity(ctx, K);
    if (st != RBE_OK) return st;
    const int threads = 128;
    k_weights_from_list<<<(K + threads - 1) / threads, threads, 0, ctx->stream>>>(K, m, w, ctx->d.m, ctx->d.w);
    return check_launch(ctx, "k_weights_from_list");
}

// Resident blocks per SM of a kernel at a block size: the occupancy API's answer, capped
// by a count from the kernel's own register and shared-memory use (registers are
// allocated per warp in units of 256).
template <typename Kern>
static int blocks_per_sm(Kern kern, int threads, size_t dyn_smem = 0)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, dyn_smem) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess) {
        int dev = 0, regs_sm = 65536, smem_sm = 228 * 1024, thr_sm = 2048;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
        const int warps = (threads + 31) / 32;
        const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
        int lim = regs_warp > 0 ? regs_sm / (regs_warp * warps) : n;
        const size_t smem_blk = fa.sharedSizeBytes + dyn_smem + 1024;  // 1 KB reserved per block
        lim = std::min<int>(lim, (int)(smem_sm / std::max<size_t>(smem_blk, 1)));
        lim = std::min(lim, thr_sm / (warps * 32));
        n = std::min(n, lim);
    } else {
        cudaGetLastError();
    }
    return std::max(1, n);
}

// Launch plan.  rho pass: frequency tiles of kthreads x kf frequencies (kf frequencies per
// thread), particle chunks so that the grid is one full wave of resident blocks with equal
// particle counts.  Force pass: whole rounds of force_unit particles per block, at most one
// resident wave.
static Plan make_plan(rbe_ctx ctx, int64_t N, int K, const RhoShape& rs, int rho_bps, int force_bps, int force_unit,
                      int min_rounds)
{
    Plan p{};
    p.kf = rs.kf;
    p.ktiles = rs.ktiles;
    p.kthreads = rs.kthreads;
    p.ksub = rs.ksub;
    p.klanes = rs.klanes;
    const int64_t want = std::max<int64_t>(1, (int64_t)ctx->num_sms * rho_bps / p.ktiles);
    // at least one staged tile of particles per chunk (fewer leave the block's fixed costs unpaid)
    const int64_t max_chunks = std::max<int64_t>(1, (N + kRhoMinChunk - 1) / kRhoMinChunk);
    p.nchunks = (int)std::min<int64_t>(want, max_chunks);
    p.chunk_len = std::max<int64_t>(1, (N + p.nchunks - 1) / p.nchunks);
    p.nchunks = (int)std::max<int64_t>(1, (N + p.chunk_len - 1) / p.chunk_len);
    p.ppt = kForcePPT;
    const int64_t resident = std::max<int64_t>(1, (int64_t)ctx->num_sms * force_bps);
    const int64_t rounds = (N + force_unit - 1) / force_unit;
    int64_t per = rounds > 0 ? (rounds + resident - 1) / resident : 0;  // rounds per block
    if (per > 0) per = std::max<int64_t>(per, min_rounds);
    p.per_block = per * force_unit;
    p.fblocks = per > 0 ? (int)((rounds + per - 1) / per) : 0;
    return p;
}

// Launch with programmatic stream serialization (the kernel calls pdl_wait()).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// The FP32-phase rho pass of plan p on stream s (the wide two-frequency kernel when p.klanes > 0).
static cudaError_t launch_rho_f32(int accum, bool xyzq, const Plan& p, dim3 grid, cudaStream_t s, const void* pos,
                                  const double* q, int64_t N, const KState* ks, const int4* m, int K, int nchunks,
                                  float4* part, unsigned* status)
{
    if (p.klanes > 0)
        return launch_pdl(rho_wide_kernel(accum, xyzq), grid, dim3(p.kthreads), 0, s, pos, q, N, ks, m, K, p.chunk_len,
                          nchunks, part, status, 0, p.ksub, p.klanes);
    return launch_pdl(rho_kernel(accum, p.kf, xyzq), grid, dim3(p.kthreads), 0, s, pos, q, N, ks, m, K, p.chunk_len,
                      nchunks, part, status, 0, p.ksub);
}

// The reduction's block: the fewest whole warps (up to kReduceThreads) that leave each thread at
// most four partials of its row, so that short rows take small blocks (more of them resident
// per SM, and the rows' FP64 work spread over the SMs).
static cudaError_t launch_reduce_f32(cudaStream_t s, const float4* part32, int nchunks, int K, const int4* m,
                                     const double* w, const KState* ks, const DeviceBuffers& d)
{
    int threads = 32;
    while (threads < kReduceThreads && threads * 4 < nchunks) threads *= 2;
    return launch_pdl(k_reduce_f32, dim3(K + 1), dim3(threads), 0, s, part32, nchunks, K, m, w, ks, d.rho,
                      d.terms, d.coef_m, d.coef_f, d.status);
}

// Launch plan and partials capacity of one evaluation of N particles and K frequencies.
struct EvalShape {
    Plan p;
    size_t force_smem;
    bool fp64;
};

// Frequency tiling of the FP32-phase rho pass: kf frequencies per thread (1, 2 or 4) and
// kthreads threads per block (whole warps).  Up to kRhoLatencyPairs pairs the pass is one short
// wave bound by latency, not by issue: one frequency per thread, tiles of up to kMaxRhoThreads.
// Above it, one or two frequencies per thread (two: one broadcast particle record feeds two
// pairs, tiles of up to kRhoThreadsF threads), whichever minimises a per-pair instruction
// estimate: the pair's own work (base), one broadcast load per kf pairs, the particle
// conversion spread over the tile's frequencies, divided by the fraction of lanes that hold a
// frequency.  Measured on GB300 from N K = 1e5 to 8e9, four frequencies per thread never ran
// faster than two (equal where the tile is full, slower where a narrow tile needs particle
// sub-streams), so they are left to tuning (RBE_RHO_FORCE_F).  A tile narrower than
// kRhoThreadsF threads is given particle sub-streams (S = block threads / T, a power of two, at
// most kRhoMaxSub).
static RhoShape rho_shape(int64_t N, int K, int accum)
{
    const double base = accum == RBE_RHO_COMP32 ? 12.0 : (accum == RBE_RHO_FP64 ? 14.0 : 10.0);
    const bool latency = (double)N * (double)K <= kRhoLatencyPairs;
    RhoShape best{1, 1, 32, 1, 0};
    double best_cost = 1e30, best_eff = 0.0;
#ifdef RBE_RHO_FORCE_F
    (void)latency;
    for (int F : {RBE_RHO_FORCE_F}) {
#else
    for (int F : {2, 1}) {
        if (latency && F != 1) continue;
#endif
        const int tmax = F == 1 ? kMaxRhoThreads : kRhoThreadsF;
        const int ktiles = (K + tmax * F - 1) / (tmax * F);
        const int per = (K + ktiles - 1) / ktiles;  // frequencies per tile
        const int T = std::min(tmax, 32 * ((per + F * 32 - 1) / (F * 32)));
        const double eff = (double)K / ((double)ktiles * T * F);
        const double cost = (base + 1.0 / F + 55.0 / (T * F)) / eff;
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best_eff = eff;
            int S = 1;
            while (T * S * 2 <= kRhoThreadsF && S * 2 <= kRhoMaxSub) S *= 2;
            best = RhoShape{F, ktiles, T * S, S, 0};
        }
    }
#ifndef RBE_RHO_FORCE_F
    // the wide two-frequency tiles, where the tiles above leave more than 5 % of the lanes without
    // a frequency: the frequencies split evenly into kt tiles of 2 T, T lanes of any count, as
    // many whole sub-streams as fit kMaxRhoThreads (at most kRhoWideMaxSub)
    for (int kt = 1; !latency && best_eff < 0.95 && kt <= RBE_RHO_WIDE_MAXKT; ++kt) {
        const int per = (K + kt - 1) / kt;
        const int T = (per + 1) / 2;
        if (T < 16 || T > kMaxRhoThreads || (kt > 1 && (K + 2 * T - 1) / (2 * T) != kt)) continue;
        const int S = std::min(kRhoWideMaxSub, kMaxRhoThreads / T);
        const int threads = 32 * ((S * T + 31) / 32);
        const double eff = (double)K / ((double)kt * 2 * T) * (double)(S * T) / threads;
        const double cost = (base + 0.5 + 55.0 / (2 * T)) / eff;
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = RhoShape{2, kt, threads, S, T};
        }
    }
#endif
    return best;
}

static rbe_status evaluate_shape(rbe_ctx ctx, int64_t N, int K, EvalShape* out)
{
    DeviceBuffers& d = ctx->d;
    const bool fp64 = ctx->precision == RBE_FP64;
    static int rho64_threads = 0, bps_f64 = 0;
    static int rho32_bps[3][4] = {{0}};  // [accum][F index, 3: wide] resident threads per SM
    if (!rho64_threads) {
        rho64_threads = blocks_per_sm(k_rho_f64, kMaxRhoThreads) * kMaxRhoThreads;
        bps_f64 = blocks_per_sm(k_force_f64<2>, kT);
        cudaFuncSetAttribute(k_force_f32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kForceSmemPerK * kForceStageK));
        cudaFuncSetAttribute(k_force_f32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kForceSmemPerK * kForceStageK));
    }
    const int kstage = std::min(K, kForceStageK);
    const size_t force_smem = fp64 ? 0 : (size_t)kForceSmemPerK * kstage;
    static int cached_kstage = -1, cached_bps_force = 1;
    if (!fp64 && kstage != cached_kstage) {
        cached_bps_force = blocks_per_sm(k_force_f32<false>, kForceThreads, force_smem);
        cached_kstage = kstage;
    }
    const int bps_force = fp64 ? bps_f64 : cached_bps_force;
    RhoShape rs;
    int rho_bps;
    if (fp64) {
        rs.kf = 1;
        rs.ktiles = (K + kMaxRhoThreads - 1) / kMaxRhoThreads;
        rs.kthreads = std::min(kMaxRhoThreads, 32 * (((K + rs.ktiles - 1) / rs.ktiles + 31) / 32));
        rs.ksub = 1;
        rs.klanes = 0;
        rho_bps = std::max(1, std::min(32, rho64_threads / rs.kthreads));
    } else {
        rs = rho_shape(N, K, ctx->rho_accum);
        const int a = ctx->rho_accum < 0 || ctx->rho_accum > 2 ? 1 : ctx->rho_accum;
        const bool wide = rs.klanes > 0;
        const int fi = wide ? 3 : (rs.kf == 4 ? 2 : (rs.kf == 2 ? 1 : 0));
        int& bps = rho32_bps[a][fi];
        if (!bps) {
            const int tmax = rs.kf == 1 || wide ? kMaxRhoThreads : kRhoThreadsF;
            bps = std::max(1, (wide ? blocks_per_sm(rho_wide_kernel(a), tmax) : blocks_per_sm(rho_kernel(a, rs.kf), tmax)) *
                                  tmax);  // resident threads per SM
        }
        rho_bps = std::max(1, std::min(32, bps / rs.kthreads));
    }
    const Plan p = make_plan(ctx, N, K, rs, rho_bps, bps_force,
                             fp64 ? kT * 2 : kForceRound, fp64 ? 1 : RBE_FORCE_MIN_ROUNDS);
    const size_t need = (size_t)(K + 1) * p.nchunks;
    if (need > d.part_cap) {
        ctx_free(ctx, d.partials);
        d.partials = nullptr;
        d.part_cap = 0;
        cudaError_t err = ctx_alloc(ctx, &d.partials, 16 * need);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaMalloc(partials)");
        d.part_cap = need;
    }
    *out = EvalShape{p, force_smem, fp64};
    return RBE_OK;
}

// One evaluation over the frequencies [koff, koff + K) of the sampled batch: rho, reduction and,
// with forces, the force pass; W and E (either may be NULL) from the same frequencies.  Without
// forces only the energy and virial are formed (the pressure batch of Eq. (apppress)).
static rbe_status launch_evaluate_range(rbe_ctx ctx, int64_t N, const void* pos, const double* q, int koff, int K,
                                        bool forces, double* F, double* W, double* E, bool xyzq)
{
    DeviceBuffers& d = ctx->d;
    const int4* m_in = d.m + koff;
    const double* w_in = d.w + koff;
    EvalShape sh;
    rbe_status st0 = evaluate_shape(ctx, N, K, &sh);
    if (st0 != RBE_OK) return st0;
    const Plan& p = sh.p;
    const bool fp64 = sh.fp64;
    const size_t force_smem = sh.force_smem;
    const dim3 grid(p.ktiles, p.nchunks);
    cudaStream_t s = ctx->stream;
    double2* part64 = static_cast<double2*>(d.partials);
    float4* part32 = static_cast<float4*>(d.partials);
    const KState* ks = d.ks;
    if (fp64) {
        k_rho_f64<<<grid, p.kthreads, 0, s>>>(static_cast<const double*>(pos), q, N, ks, m_in, K, p.chunk_len,
                                              p.nchunks, part64, d.status);
    } else {
        cudaError_t err = launch_rho_f32(ctx->rho_accum, xyzq, p, grid, s, pos, q, N, ks, m_in, K, p.nchunks, part32,
                                         d.status);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "launch k_rho_f32");
    }
    rbe_status st = check_launch(ctx, "k_rho");
    if (st != RBE_OK) return st;
    record_event(ctx, 2);
    if (fp64) {
        k_reduce<<<K + 1, kReduceThreads, 0, s>>>(part64, p.nchunks, K, m_in, w_in, ks, d.rho, d.terms, d.coef_d,
                                                   d.counter, d.status, W, E);
    } else {
        cudaError_t err = launch_reduce_f32(s, (const float4*)part32, p.nchunks, K, m_in, w_in, ks, d);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "launch k_reduce_f32");
    }
    st = check_launch(ctx, "k_reduce");
    if (st != RBE_OK) return st;
    record_event(ctx, 3);
    if (fp64) {
        if (forces && p.fblocks > 0) {
            k_force_f64<2><<<p.fblocks, kT, 0, s>>>(static_cast<const double*>(pos), q, N, p.per_block, ks, d.m,
                                                    d.coef_d, K, F);
            st = check_launch(ctx, "k_force");
        }
    } else {
        // one extra block computes the energy and virial sums
        cudaError_t err = launch_pdl(xyzq ? k_force_f32<true> : k_force_f32<false>, dim3((forces ? p.fblocks : 0) + 1),
                                     dim3(kForceThreads), force_smem, s, pos, q,
                                     N, p.per_block, ks, (const int4*)d.coef_m, (const float4*)d.coef_f, K, F,
                                     d.status, (const double*)d.terms, W, E, (int64_t)0, 1);
        st = err == cudaSuccess ? RBE_OK : cuda_fail(ctx, err, "launch k_force_f32");
    }
    if (st != RBE_OK) return st;
    record_event(ctx, 4);
    ctx->last_K = K;
    return RBE_OK;
}

rbe_status launch_evaluate(rbe_ctx ctx, int64_t N, const double* pos, const double* q, int K,
                           bool /*uniform_weight*/, double* F, double* W, double* E)
{
    return launch_evaluate_range(ctx, N, pos, q, 0, K, true, F, W, E, false);
}

// The RBE evaluation of a sampled step: forces from the force batch (slots [0, P)) and, with a
// pressure batch (ctx->Ptilde > 0), energy and virial from slots [P, P + Ptilde) with weights
// S/Ptilde (Eqs. (appforce), (apppress) with p and p~); otherwise all from the one batch.
rbe_status launch_rbe(rbe_ctx ctx, int64_t N, const void* pos, const double* q, int P, double* F, double* W,
                      double* E, bool xyzq)
{
    if (ctx->Ptilde <= 0) return launch_evaluate_range(ctx, N, pos, q, 0, P, true, F, W, E, xyzq);
    rbe_status st = launch_evaluate_range(ctx, N, pos, q, 0, P, true, F, nullptr, nullptr, xyzq);
    if (st != RBE_OK) return st;
    return launch_evaluate_range(ctx, N, pos, q, P, ctx->Ptilde, false, nullptr, W, E, xyzq);
}

// The host-buffer evaluation on the FP32-phase path, pipelined in quarters: the particles
// are split into `pieces` contiguous groups, each evaluated by full-GPU passes of its own
// plan.  Group g's positions and charges go to the device on the context's copy stream while
// the rho pass of group g - 1 runs; after the reduction (over the chunks of all groups), group
// g's forces come back on the copy stream while group g + 1's force pass runs.  The chunk
// partition differs from a single evaluation's, so the results agree with
// rbe_kspace_forces_virial to FP32 rounding (not bit for bit) and are reproducible run to run.
// d_pos, d_q, d_F: device staging of at least N particles; W, E: device outputs.
rbe_status launch_evaluate_staged(rbe_ctx ctx, int64_t N, const double* h_pos, const double* h_q, double* h_F,
                                  double* d_pos, double* d_q, double* d_F, int K, double* W, double* E,
                                  int pieces)
{
    DeviceBuffers& d = ctx->d;
    pieces = std::max(1, std::min(pieces, kMaxPieces));
    if (N < pieces) pieces = 1;
    EvalShape whole;
    rbe_status st = evaluate_shape(ctx, N, K, &whole);  // occupancy caches, frequency tile shape
    if (st != RBE_OK) return st;
    Plan pl[kMaxPieces];
    int64_t i0[kMaxPieces + 1];
    int coff[kMaxPieces + 1];
    coff[0] = 0;
    // four groups: a small first and last one (an eighth each), so that the copy in before the
    // first pass and the copy out after the last are short; else equal groups
    static const int kEighths4[5] = {0, 1, 4, 7, 8};
    for (int g = 0; g <= pieces; ++g) i0[g] = pieces == 4 ? N * kEighths4[g] / 8 : N * g / pieces;
    for (int g = 0; g < pieces; ++g) {
        EvalShape sg;
        if ((st = evaluate_shape(ctx, i0[g + 1] - i0[g], K, &sg)) != RBE_OK) return st;
        pl[g] = sg.p;
        coff[g + 1] = coff[g] + pl[g].nchunks;
    }
    const int nchunks = coff[pieces];
    const size_t need = (size_t)(K + 1) * nchunks;
    if (need > d.part_cap) {
        ctx_free(ctx, d.partials);
        d.partials = nullptr;
        d.part_cap = 0;
        cudaError_t e = ctx_alloc(ctx, &d.partials, 16 * need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(partials)");
        d.part_cap = need;
    }
    cudaStream_t s = ctx->stream, cs = ctx->copy_stream;
    const KState* ks = d.ks;
    float4* part32 = static_cast<float4*>(d.partials);
    cudaError_t err;
    // (the caller has ordered the copy stream after the main stream's earlier work)
    for (int g = 0; g < pieces; ++g) {
        const int64_t a = i0[g], n = i0[g + 1] - i0[g];
        if ((err = cudaMemcpyAsync(d_pos + 3 * a, h_pos + 3 * a, sizeof(double) * 3 * n, cudaMemcpyHostToDevice,
                                   cs)) != cudaSuccess ||
            (err = cudaMemcpyAsync(d_q + a, h_q + a, sizeof(double) * n, cudaMemcpyHostToDevice, cs)) != cudaSuccess)
            return cuda_fail(ctx, err, "staged: H2D");
        if ((err = cudaEventRecord(ctx->pev[1 + g], cs)) != cudaSuccess ||
            (err = cudaStreamWaitEvent(s, ctx->pev[1 + g], 0)) != cudaSuccess)
            return cuda_fail(ctx, err, "staged: input event");
        // group g: rows of stride nchunks, its columns from coff[g]
        err = launch_rho_f32(ctx->rho_accum, false, pl[g], dim3(pl[g].ktiles, pl[g].nchunks), s,
                             (const double*)(d_pos + 3 * a), (const double*)(d_q + a), n, ks, (const int4*)d.m, K,
                             nchunks, part32 + coff[g], d.status);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "staged: k_rho_f32");
    }
    err = launch_reduce_f32(s, (const float4*)part32, nchunks, K, (const int4*)d.m, (const double*)d.w, ks, d);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "staged: k_reduce_f32");
    for (int g = 0; g < pieces; ++g) {
        const int64_t a = i0[g], n = i0[g + 1] - i0[g];
        const int final_block = g == pieces - 1 ? 1 : 0;
        err = launch_pdl(k_force_f32<false>, dim3(pl[g].fblocks + final_block), dim3(kForceThreads), whole.force_smem, s,
                         (const double*)(d_pos + 3 * a), (const double*)(d_q + a), n, pl[g].per_block, ks,
                         (const int4*)d.coef_m, (const float4*)d.coef_f, K, d_F + 3 * a, d.status,
                         (const double*)d.terms, W, E, (int64_t)0, final_block);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "staged: k_force_f32");
        if ((err = cudaEventRecord(ctx->pev[1 + kMaxPieces + g], s)) != cudaSuccess ||
            (err = cudaStreamWaitEvent(cs, ctx->pev[1 + kMaxPieces + g], 0)) != cudaSuccess)
            return cuda_fail(ctx, err, "staged: force event");
        if (h_F && (err = cudaMemcpyAsync(h_F + 3 * a, d_F + 3 * a, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost,
                                          cs)) != cudaSuccess)
            return cuda_fail(ctx, err, "staged: D2H forces");
    }
    ctx->last_K = K;
    return RBE_OK;
}

}  // namespace rbe
