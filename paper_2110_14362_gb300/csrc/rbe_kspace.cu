// RBE k-space kernels for sm_103a and their launchers.
//
// One evaluation (Sec. 4.2 of the paper) is five launches on the context's stream:
//   k_tables   per-axis weights exp(-c m^2), cumulative sums, H and S        Eqs. (S), (psf)
//                (only when the box changed)
//   k_sample   one thread per frequency: Philox -> 3 uniforms -> inverse CDF  Eq. (probexpression)
//   k_rho_*    particle-chunk x frequency-tile blocks: partial rho(k_l) per chunk
//   k_reduce   fixed-order FP64 sum of the partials -> rho(k_l), the per-frequency
//              force coefficients, and (last block) the energy and the 3x3 virial
//                                              Eq. (apppress); App. C Eq. (pressuretensorflexible)
//   k_force_*  particle tiles x all frequencies: F_i                             Eq. (appforce)
// No floating-point atomics: every sum runs in an order fixed by (N, K, plan), so
// results are bitwise reproducible run to run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>

#include "rbe_context.h"
#include "rbe_device.cuh"

namespace rbe {

constexpr int kT = 128;        // threads per block of the force pass
constexpr int kForceKT = 256;  // frequencies staged per tile in the force pass

// =================================================================================
// Sampling tables (Sec. 4.2 Eqs. (S), (psf); App. C item 1).
__global__ void k_tables(double bx, double by, double bz, const double* __restrict__ box_dev, double alpha,
                         double* __restrict__ cdf, int cap, TableHeader* __restrict__ hdr,
                         unsigned* __restrict__ status)
{
    __shared__ int sM[3];
    __shared__ double sc[3];
    const int tid = threadIdx.x;
    if (tid < 3) {
        double ell = box_dev ? box_dev[tid] : (tid == 0 ? bx : (tid == 1 ? by : bz));
        double c = axis_c(alpha, ell);
        int M = axis_M(c);
        if (2 * M + 1 > cap) {
            atomicOr(status, kStatusTable);
            M = (cap - 1) / 2;
        }
        sM[tid] = M;
        sc[tid] = c;
    }
    __syncthreads();
    for (int t = 0; t < 3; ++t) {
        const int M = sM[t];
        const double c = sc[t];
        double* row = cdf + (size_t)t * cap;
        for (int a = tid; a <= M; a += blockDim.x) {
            const double v = table_exp(-__dmul_rn(c, (double)a * (double)a));
            row[M + a] = v;
            row[M - a] = v;
        }
    }
    __syncthreads();
    if (tid < 3) {
        const int M = sM[tid];
        double* row = cdf + (size_t)tid * cap;
        double acc = 0.0;
        for (int j = 0; j <= 2 * M; ++j) {
            acc = __dadd_rn(acc, row[j]);
            row[j] = acc;
        }
        hdr->M[tid] = M;
        hdr->H[tid] = acc;
    }
    __syncthreads();
    if (tid == 0) hdr->S = __dsub_rn(__dmul_rn(__dmul_rn(hdr->H[0], hdr->H[1]), hdr->H[2]), 1.0);
}

// Smallest j in [0, 2M] with target < cdf[j] (cdf is non-decreasing), minus M.
__device__ __forceinline__ int inverse_cdf(const double* __restrict__ row, int M, double u)
{
    const double target = __dmul_rn(u, row[2 * M]);
    int lo = 0, hi = 2 * M;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (target < row[mid]) hi = mid;
        else lo = mid + 1;
    }
    return lo - M;
}

// =================================================================================
// Frequency sampling (Sec. 4.2-4.3): sample l uses Philox key (seed_lo, seed_hi) and
// counters (l, 2 attempt + half, step_lo, step_hi24); redraw while m = 0.  When the three
// cumulative tables fit (smem_entries > 0) the block first copies them to shared memory,
// so that the binary searches do not wait on global memory.
__global__ void k_sample(uint64_t seed, uint64_t step, int P, const double* __restrict__ cdf, int cap,
                         int smem_cap, const TableHeader* __restrict__ hdr, int4* __restrict__ m_out,
                         double* __restrict__ w_out, unsigned* __restrict__ status)
{
    extern __shared__ double s_cdf[];
    const int Mx = hdr->M[0], My = hdr->M[1], Mz = hdr->M[2];
    const double* tx = cdf;
    const double* ty = cdf + cap;
    const double* tz = cdf + 2 * (size_t)cap;
    if (smem_cap > 0) {
        for (int j = threadIdx.x; j <= 2 * Mx; j += blockDim.x) s_cdf[j] = tx[j];
        for (int j = threadIdx.x; j <= 2 * My; j += blockDim.x) s_cdf[smem_cap + j] = ty[j];
        for (int j = threadIdx.x; j <= 2 * Mz; j += blockDim.x) s_cdf[2 * smem_cap + j] = tz[j];
        __syncthreads();
        tx = s_cdf;
        ty = s_cdf + smem_cap;
        tz = s_cdf + 2 * smem_cap;
    }
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= P) return;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t c2 = (uint32_t)step, c3 = (uint32_t)((step >> 32) & 0xFFFFFFu);
    int4 m = make_int4(0, 0, 0, 0);
    bool found = false;
    for (uint32_t attempt = 0; attempt < kMaxAttempts; ++attempt) {
        const uint4 w0 = philox4x32_10(make_uint4((uint32_t)l, 2u * attempt, c2, c3), k0, k1);
        const uint4 w1 = philox4x32_10(make_uint4((uint32_t)l, 2u * attempt + 1u, c2, c3), k0, k1);
        m.x = inverse_cdf(tx, Mx, uniform53(w0.x, w0.y));
        m.y = inverse_cdf(ty, My, uniform53(w0.z, w0.w));
        m.z = inverse_cdf(tz, Mz, uniform53(w1.x, w1.y));
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
    w_out[l] = hdr->S / (double)P;
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

// =================================================================================
// rho pass, FP32-phase path.  Block (kt, c) has blockDim.x (a multiple of 32, <= 256)
// threads; thread j owns frequency kt * blockDim.x + j and runs over the particles
// [c * chunk_len, (c + 1) * chunk_len), staged in shared memory blockDim.x at a time as
// 32-bit fixed-point (s_x, s_y, s_z) plus q as float and read as broadcasts.
// ACC: RBE_RHO_FP32 (plain FP32 within a staged tile, FP64 across tiles),
//      RBE_RHO_COMP32 (Kahan-compensated FP32 within a tile), RBE_RHO_FP64 (per pair).
constexpr int kMaxRhoThreads = 256;

template <int ACC>
__global__ void __launch_bounds__(kMaxRhoThreads)
k_rho_f32(const double* __restrict__ pos, const double* __restrict__ q, int64_t N, double ilx, double ily,
          double ilz, const int4* __restrict__ m, int K, int64_t chunk_len, int nchunks,
          double2* __restrict__ partials, unsigned* __restrict__ status, uint32_t mul23)
{
    __shared__ uint4 sp[kMaxRhoThreads];
    __shared__ double red[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int l = blockIdx.x * nt + tid;
    const int c = blockIdx.y;
    const int4 mv = l < K ? m[l] : make_int4(0, 0, 0, 0);
    double are = 0.0, aim = 0.0, q2 = 0.0;
    const int64_t start = (int64_t)c * chunk_len;
    const int64_t end = min(N, start + chunk_len);
    for (int64_t base = start; base < end; base += nt) {
        const int64_t i = base + tid;
        uint4 rec = make_uint4(0u, 0u, 0u, 0u);
        if (i < end) {
            const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
            const double qi = q[i];
            if (!isfinite(x + y + z + qi)) atomicOr(status, kStatusNonFinite);
            q2 += qi * qi;
            rec = make_uint4(fixed_frac(x, ilx), fixed_frac(y, ily), fixed_frac(z, ilz), __float_as_uint((float)qi));
        }
        sp[tid] = rec;
        __syncthreads();
        const int n_here = (int)min((int64_t)nt, end - base);
        float re = 0.f, im = 0.f, cre = 0.f, cim = 0.f;
#pragma unroll 4
        for (int p = 0; p < n_here; ++p) {
            const uint4 r = sp[p];
            const float qp = __uint_as_float(r.w);
            const float th = fixed_phase(mv.x, mv.y, mv.z, r.x, r.y, r.z, mul23);
            float sn, cs;
            __sincosf(th, &sn, &cs);
            if (ACC == RBE_RHO_FP32) {
                re = fmaf(qp, cs, re);
                im = fmaf(qp, sn, im);
            } else if (ACC == RBE_RHO_COMP32) {
                const float yr = qp * cs - cre;
                const float tr = re + yr;
                cre = (tr - re) - yr;
                re = tr;
                const float yi = qp * sn - cim;
                const float ti = im + yi;
                cim = (ti - im) - yi;
                im = ti;
            } else {
                are = fma((double)qp, (double)cs, are);
                aim = fma((double)qp, (double)sn, aim);
            }
        }
        if (ACC != RBE_RHO_FP64) {
            are += (double)re - (double)cre;
            aim += (double)im - (double)cim;
        }
        __syncthreads();
    }
    if (l < K) partials[(size_t)l * nchunks + c] = make_double2(are, aim);
    if (blockIdx.x == 0) {
        const double s = block_sum(q2, red);  // sum of q^2 over the chunk, for E_self
        if (tid == 0) partials[(size_t)K * nchunks + c] = make_double2(s, 0.0);
    }
}

// rho pass, FP64 path: s = r / l wrapped to [0, 1); t = m.s - rint(m.s); sincospi(2t).
__global__ void __launch_bounds__(kMaxRhoThreads)
k_rho_f64(const double* __restrict__ pos, const double* __restrict__ q, int64_t N, double ilx, double ily,
          double ilz, const int4* __restrict__ m, int K, int64_t chunk_len, int nchunks,
          double2* __restrict__ partials, unsigned* __restrict__ status)
{
    __shared__ double4_32a sp[kMaxRhoThreads];
    __shared__ double red[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int l = blockIdx.x * nt + tid;
    const int c = blockIdx.y;
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
// Reduction of the partials: block l (of K + 1) sums its row over the chunks in a fixed
// order (strided per thread, then a fixed tree), forms the per-frequency terms, and the
// last block to finish sums those over l in a fixed order.
//   e_l = (2 pi / V) w_l |rho_l|^2 / |k_l|^2
//   W  += e_l [I - 2 (1/|k_l|^2 + 1/4a) k_l k_l]
//   beta_l = w_l 4 pi / (V |k_l|^2), A_l = beta_l Im rho_l, B_l = beta_l Re rho_l, so that
//   F_i = q_i sum_l k_l (sin(k_l.r_i) B_l - cos(k_l.r_i) A_l).
constexpr int kReduceThreads = 256;

__global__ void __launch_bounds__(kReduceThreads)
k_reduce(const double2* __restrict__ partials, int nchunks, int K, const int4* __restrict__ m,
         const double* __restrict__ w, double bx, double by, double bz, double alpha,
         double2* __restrict__ rho, double* __restrict__ terms, int4* __restrict__ coef_m,
         float4* __restrict__ coef_f, double2* __restrict__ coef_d, unsigned* __restrict__ counter,
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
    if (threadIdx.x == 0) {
        double* t = terms + (size_t)l * 8;
        if (l < K) {
            const int4 mi = m[l];
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
            const double A = beta * im, B = beta * re;
            rho[l] = make_double2(re, im);
            coef_d[l] = make_double2(A, B);
            coef_m[l] = make_int4(mi.x, mi.y, mi.z, __float_as_int((float)A));
            coef_f[l] = make_float4((float)B, (float)mi.x, (float)mi.y, (float)mi.z);
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

// =================================================================================
// Force pass, FP32-phase path.  Block b owns particles [b * per_block, (b+1) * per_block),
// processed kT * PPT at a time (PPT per thread).  Frequencies are staged in shared memory
// kForceKT at a time as (mx, my, mz, A) and (B, mx, my, mz) and read as broadcasts; when
// K <= kForceKT they are staged once per block.
// F_i,theta = q_i (2 pi / l_theta) sum_l m_l,theta (sin B_l - cos A_l): FP32 within a
// staged frequency tile, FP64 across tiles.
template <int PPT>
__global__ void __launch_bounds__(kT) k_force_f32(const double* __restrict__ pos, const double* __restrict__ q,
                                                  int64_t N, int64_t per_block, double ilx, double ily,
                                                  double ilz, const int4* __restrict__ coef_m,
                                                  const float4* __restrict__ coef_f, int K,
                                                  double* __restrict__ F, uint32_t mul23)
{
    __shared__ int4 sm[kForceKT];
    __shared__ float4 sf[kForceKT];
    const int tid = threadIdx.x;
    const bool one_tile = K <= kForceKT;
    if (one_tile) {
        for (int j = tid; j < K; j += kT) {
            sm[j] = coef_m[j];
            sf[j] = coef_f[j];
        }
        __syncthreads();
    }
    const int64_t b0 = (int64_t)blockIdx.x * per_block;
    const int64_t b1 = min(N, b0 + per_block);
    const double cx = 2.0 * kPi * ilx, cy = 2.0 * kPi * ily, cz = 2.0 * kPi * ilz;
    for (int64_t base = b0; base < b1; base += (int64_t)kT * PPT) {
        uint32_t sx[PPT], sy[PPT], sz[PPT];
        double fx[PPT], fy[PPT], fz[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int64_t i = base + (int64_t)p * kT + tid;
            if (i < b1) {
                sx[p] = fixed_frac(pos[3 * i], ilx);
                sy[p] = fixed_frac(pos[3 * i + 1], ily);
                sz[p] = fixed_frac(pos[3 * i + 2], ilz);
            } else {
                sx[p] = sy[p] = sz[p] = 0u;
            }
            fx[p] = fy[p] = fz[p] = 0.0;
        }
        for (int k0 = 0; k0 < K; k0 += kForceKT) {
            const int nk = min(kForceKT, K - k0);
            if (!one_tile) {
                __syncthreads();
                for (int j = tid; j < nk; j += kT) {
                    sm[j] = coef_m[k0 + j];
                    sf[j] = coef_f[k0 + j];
                }
                __syncthreads();
            }
            float gx[PPT], gy[PPT], gz[PPT];
#pragma unroll
            for (int p = 0; p < PPT; ++p) gx[p] = gy[p] = gz[p] = 0.f;
#pragma unroll 2
            for (int l = 0; l < nk; ++l) {
                const int4 a = sm[l];
                const float4 b = sf[l];
                const float A = __int_as_float(a.w);
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    const float th = fixed_phase(a.x, a.y, a.z, sx[p], sy[p], sz[p], mul23);
                    float sn, cs;
                    __sincosf(th, &sn, &cs);
                    const float g = fmaf(sn, b.x, -cs * A);
                    gx[p] = fmaf(g, b.y, gx[p]);
                    gy[p] = fmaf(g, b.z, gy[p]);
                    gz[p] = fmaf(g, b.w, gz[p]);
                }
            }
#pragma unroll
            for (int p = 0; p < PPT; ++p) { fx[p] += gx[p]; fy[p] += gy[p]; fz[p] += gz[p]; }
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

// Force pass, FP64 path (same blocking, FP64 throughout).
template <int PPT>
__global__ void __launch_bounds__(kT) k_force_f64(const double* __restrict__ pos, const double* __restrict__ q,
                                                  int64_t N, int64_t per_block, double ilx, double ily,
                                                  double ilz, const int4* __restrict__ mk,
                                                  const double2* __restrict__ coef_d, int K,
                                                  double* __restrict__ F)
{
    __shared__ double4_32a sk[kForceKT];  // (mx, my, mz, A)
    __shared__ double sb[kForceKT];       // B
    const int tid = threadIdx.x;
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

rbe_status ensure_tables(rbe_ctx ctx)
{
    if (!ctx->tables_dirty) return RBE_OK;
    int need = 0;
    for (int t = 0; t < 3; ++t) need = std::max(need, 2 * host_axis_M(ctx->alpha, ctx->box[t]) + 1);
    if (need > ctx->d.tab_cap) {
        if (ctx->d.cdf) cudaFree(ctx->d.cdf);
        ctx->d.cdf = nullptr;
        ctx->d.tab_cap = 0;
        const int cap = need + need / 4 + 16;  // headroom for boxes that grow on the device
        cudaError_t err = cudaMalloc(&ctx->d.cdf, sizeof(double) * 3 * (size_t)cap);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaMalloc(tables)");
        ctx->d.tab_cap = cap;
    }
    k_tables<<<1, 256, 0, ctx->stream>>>(ctx->box[0], ctx->box[1], ctx->box[2], nullptr, ctx->alpha,
                                         ctx->d.cdf, ctx->d.tab_cap, ctx->d.hdr, ctx->d.status);
    rbe_status st = check_launch(ctx, "k_tables");
    if (st == RBE_OK) ctx->tables_dirty = false;
    return st;
}

rbe_status ensure_k_capacity(rbe_ctx ctx, int K)
{
    if (K <= ctx->d.kcap) return RBE_OK;
    DeviceBuffers& d = ctx->d;
    cudaFree(d.m); cudaFree(d.w); cudaFree(d.rho); cudaFree(d.terms);
    cudaFree(d.coef_m); cudaFree(d.coef_f); cudaFree(d.coef_d);
    d.m = nullptr; d.w = nullptr; d.rho = nullptr; d.terms = nullptr;
    d.coef_m = nullptr; d.coef_f = nullptr; d.coef_d = nullptr;
    d.kcap = 0;
    cudaError_t err = cudaSuccess;
    if ((err = cudaMalloc(&d.m, sizeof(int4) * K)) != cudaSuccess ||
        (err = cudaMalloc(&d.w, sizeof(double) * K)) != cudaSuccess ||
        (err = cudaMalloc(&d.rho, sizeof(double2) * K)) != cudaSuccess ||
        (err = cudaMalloc(&d.terms, sizeof(double) * 8 * (size_t)(K + 1))) != cudaSuccess ||
        (err = cudaMalloc(&d.coef_m, sizeof(int4) * K)) != cudaSuccess ||
        (err = cudaMalloc(&d.coef_f, sizeof(float4) * K)) != cudaSuccess ||
        (err = cudaMalloc(&d.coef_d, sizeof(double2) * K)) != cudaSuccess)
        return cuda_fail(ctx, err, "cudaMalloc(frequency buffers)");
    d.kcap = K;
    return RBE_OK;
}

constexpr int kSampleSmemMax = 48 * 1024;

rbe_status launch_sample(rbe_ctx ctx, uint64_t step, int P)
{
    rbe_status st = ensure_tables(ctx);
    if (st != RBE_OK) return st;
    st = ensure_k_capacity(ctx, P);
    if (st != RBE_OK) return st;
    record_event(ctx, 0);
    const int threads = 128;
    const size_t smem = sizeof(double) * 3 * (size_t)ctx->d.tab_cap;
    const int smem_cap = smem <= (size_t)kSampleSmemMax ? ctx->d.tab_cap : 0;
    k_sample<<<(P + threads - 1) / threads, threads, smem_cap ? smem : 0, ctx->stream>>>(
        ctx->seed, step, P, ctx->d.cdf, ctx->d.tab_cap, smem_cap, ctx->d.hdr, ctx->d.m, ctx->d.w, ctx->d.status);
    record_event(ctx, 1);
    return check_launch(ctx, "k_sample");
}

rbe_status launch_weights_from_list(rbe_ctx ctx, int K, const int32_t* m, const double* w)
{
    rbe_status st = ensure_k_capacity(ctx, K);
    if (st != RBE_OK) return st;
    const int threads = 128;
    k_weights_from_list<<<(K + threads - 1) / threads, threads, 0, ctx->stream>>>(K, m, w, ctx->d.m, ctx->d.w);
    return check_launch(ctx, "k_weights_from_list");
}

// Resident blocks per SM of a kernel at a block size (cached per process).
template <typename Kern>
static int blocks_per_sm(Kern kern, int threads)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return std::max(1, n);
}

// Launch plan.  rho pass: frequency tiles of at most 256 threads, sized in whole warps
// so that few lanes idle; particle chunks so that the grid is one full wave of resident
// blocks with equal particle counts.  Force pass: a grid that is a multiple of the SM
// count, equal particle ranges per block.
static Plan make_plan(rbe_ctx ctx, int64_t N, int K, int rho_bps, int force_bps)
{
    Plan p{};
    p.ktiles = (K + kMaxRhoThreads - 1) / kMaxRhoThreads;
    const int per_tile = (K + p.ktiles - 1) / p.ktiles;
    p.kthreads = std::min(kMaxRhoThreads, 32 * ((per_tile + 31) / 32));
    const int64_t want = std::max<int64_t>(1, (int64_t)ctx->num_sms * rho_bps / p.ktiles);
    const int64_t max_chunks = std::max<int64_t>(1, (N + 63) / 64);  // at least 64 particles per chunk
    p.nchunks = (int)std::min<int64_t>(want, max_chunks);
    p.chunk_len = std::max<int64_t>(1, (N + p.nchunks - 1) / p.nchunks);
    p.nchunks = (int)std::max<int64_t>(1, (N + p.chunk_len - 1) / p.chunk_len);
    p.ppt = 2;
    const int64_t fwant = (int64_t)ctx->num_sms * force_bps;
    const int64_t fmax = (N + kT * p.ppt - 1) / (kT * p.ppt);
    p.fblocks = (int)std::min<int64_t>(fwant, fmax);
    p.per_block = p.fblocks > 0 ? (N + p.fblocks - 1) / p.fblocks : 0;
    if (p.per_block > 0) p.fblocks = (int)((N + p.per_block - 1) / p.per_block);
    return p;
}

rbe_status launch_evaluate(rbe_ctx ctx, int64_t N, const double* pos, const double* q, int K,
                           bool /*uniform_weight*/, double* F, double* W, double* E)
{
    DeviceBuffers& d = ctx->d;
    static int bps_rho32 = 0, bps_rho64 = 0, bps_f32 = 0, bps_f64 = 0;
    if (!bps_rho32) {
        bps_rho32 = blocks_per_sm(k_rho_f32<RBE_RHO_FP32>, kMaxRhoThreads) * kMaxRhoThreads;
        bps_rho64 = blocks_per_sm(k_rho_f64, kMaxRhoThreads) * kMaxRhoThreads;
        bps_f32 = blocks_per_sm(k_force_f32<2>, kT);
        bps_f64 = blocks_per_sm(k_force_f64<2>, kT);
    }
    const bool fp64 = ctx->precision == RBE_FP64;
    // resident rho blocks per SM at the tile's block size (threads per SM / block size)
    const int ktiles = (K + kMaxRhoThreads - 1) / kMaxRhoThreads;
    const int kthreads = std::min(kMaxRhoThreads, 32 * (((K + ktiles - 1) / ktiles + 31) / 32));
    const int rho_bps = std::max(1, std::min(32, (fp64 ? bps_rho64 : bps_rho32) / kthreads));
    const Plan p = make_plan(ctx, N, K, rho_bps, fp64 ? bps_f64 : bps_f32);
    const size_t need = (size_t)(K + 1) * p.nchunks;
    if (need > d.part_cap) {
        cudaFree(d.partials);
        d.partials = nullptr;
        d.part_cap = 0;
        cudaError_t err = cudaMalloc(&d.partials, sizeof(double2) * need);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaMalloc(partials)");
        d.part_cap = need;
    }
    const double ilx = 1.0 / ctx->box[0], ily = 1.0 / ctx->box[1], ilz = 1.0 / ctx->box[2];
    const dim3 grid(p.ktiles, p.nchunks);
    const uint32_t mul23 = 1u << 23;
    cudaStream_t s = ctx->stream;
    if (fp64) {
        k_rho_f64<<<grid, p.kthreads, 0, s>>>(pos, q, N, ilx, ily, ilz, d.m, K, p.chunk_len, p.nchunks, d.partials,
                                              d.status);
    } else {
        switch (ctx->rho_accum) {
        case RBE_RHO_FP64:
            k_rho_f32<RBE_RHO_FP64><<<grid, p.kthreads, 0, s>>>(pos, q, N, ilx, ily, ilz, d.m, K, p.chunk_len,
                                                                 p.nchunks, d.partials, d.status, mul23);
            break;
        case RBE_RHO_COMP32:
            k_rho_f32<RBE_RHO_COMP32><<<grid, p.kthreads, 0, s>>>(pos, q, N, ilx, ily, ilz, d.m, K, p.chunk_len,
                                                                   p.nchunks, d.partials, d.status, mul23);
            break;
        default:
            k_rho_f32<RBE_RHO_FP32><<<grid, p.kthreads, 0, s>>>(pos, q, N, ilx, ily, ilz, d.m, K, p.chunk_len,
                                                                 p.nchunks, d.partials, d.status, mul23);
            break;
        }
    }
    rbe_status st = check_launch(ctx, "k_rho");
    if (st != RBE_OK) return st;
    record_event(ctx, 2);
    k_reduce<<<K + 1, kReduceThreads, 0, s>>>(d.partials, p.nchunks, K, d.m, d.w, ctx->box[0], ctx->box[1],
                                               ctx->box[2], ctx->alpha, d.rho, d.terms, d.coef_m, d.coef_f,
                                               d.coef_d, d.counter, d.status, W, E);
    st = check_launch(ctx, "k_reduce");
    if (st != RBE_OK) return st;
    record_event(ctx, 3);
    if (p.fblocks > 0) {
        if (fp64)
            k_force_f64<2><<<p.fblocks, kT, 0, s>>>(pos, q, N, p.per_block, ilx, ily, ilz, d.m, d.coef_d, K, F);
        else
            k_force_f32<2><<<p.fblocks, kT, 0, s>>>(pos, q, N, p.per_block, ilx, ily, ilz, d.coef_m, d.coef_f, K, F,
                                                    mul23);
        st = check_launch(ctx, "k_force");
        if (st != RBE_OK) return st;
    }
    record_event(ctx, 4);
    ctx->last_K = K;
    return RBE_OK;
}

}  // namespace rbe
