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

constexpr int kT = 128;        // threads per block of the pair kernels
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
// counters (l, 2 attempt + half, step_lo, step_hi24); redraw while m = 0.
__global__ void k_sample(uint64_t seed, uint64_t step, int P, const double* __restrict__ cdf, int cap,
                         const TableHeader* __restrict__ hdr, int4* __restrict__ m_out,
                         double* __restrict__ w_out, unsigned* __restrict__ status)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= P) return;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int Mx = hdr->M[0], My = hdr->M[1], Mz = hdr->M[2];
    int4 m = make_int4(0, 0, 0, 0);
    bool found = false;
    for (uint32_t attempt = 0; attempt < kMaxAttempts; ++attempt) {
        const uint4 w0 = philox4x32_10(make_uint4((uint32_t)l, 2u * attempt, (uint32_t)step,
                                                  (uint32_t)((step >> 32) & 0xFFFFFFu)), k0, k1);
        const uint4 w1 = philox4x32_10(make_uint4((uint32_t)l, 2u * attempt + 1u, (uint32_t)step,
                                                  (uint32_t)((step >> 32) & 0xFFFFFFu)), k0, k1);
        m.x = inverse_cdf(cdf, Mx, uniform53(w0.x, w0.y));
        m.y = inverse_cdf(cdf + cap, My, uniform53(w0.z, w0.w));
        m.z = inverse_cdf(cdf + 2 * (size_t)cap, Mz, uniform53(w1.x, w1.y));
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

// =================================================================================
// rho pass, FP32-phase path.  Block (kt, c): frequencies kt*kT*KPT + j*kT + tid
// (j < KPT) against particles [c*chunk_len, (c+1)*chunk_len).  Particles are staged in
// shared memory kT at a time as (s_x, s_y, s_z) 32-bit fixed point plus q as float;
// each thread keeps its frequencies in registers and reads the particles as broadcasts.
// ACC: RBE_RHO_FP32 (plain FP32 within a staged tile, FP64 across tiles),
//      RBE_RHO_COMP32 (Kahan-compensated FP32 within a tile), RBE_RHO_FP64 (per pair).
template <int KPT, int ACC>
__global__ void __launch_bounds__(kT) k_rho_f32(const double* __restrict__ pos, const double* __restrict__ q,
                                                int64_t N, double ilx, double ily, double ilz,
                                                const int4* __restrict__ m, int K, int chunk_len,
                                                int nchunks, double2* __restrict__ partials,
                                                unsigned* __restrict__ status)
{
    __shared__ uint4 sp[kT];
    const int tid = threadIdx.x;
    const int kt = blockIdx.x;
    const int c = blockIdx.y;
    int mx[KPT], my[KPT], mz[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        const int l = kt * kT * KPT + j * kT + tid;
        int4 v = l < K ? m[l] : make_int4(0, 0, 0, 0);
        mx[j] = v.x; my[j] = v.y; mz[j] = v.z;
    }
    double are[KPT], aim[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) { are[j] = 0.0; aim[j] = 0.0; }
    double q2 = 0.0;
    const int64_t start = (int64_t)c * chunk_len;
    const int64_t end = min(N, start + (int64_t)chunk_len);
    for (int64_t base = start; base < end; base += kT) {
        const int64_t i = base + tid;
        uint4 rec = make_uint4(0u, 0u, 0u, 0u);
        if (i < end) {
            const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
            const double qi = q[i];
            if (!isfinite(x + y + z + qi)) atomicOr(status, kStatusNonFinite);
            q2 += qi * qi;
            rec = make_uint4(fixed_frac(x, ilx), fixed_frac(y, ily), fixed_frac(z, ilz),
                             __float_as_uint((float)qi));
        }
        sp[tid] = rec;
        __syncthreads();
        const int n_here = (int)min((int64_t)kT, end - base);
        float re[KPT], im[KPT], cre[KPT], cim[KPT];
#pragma unroll
        for (int j = 0; j < KPT; ++j) { re[j] = 0.f; im[j] = 0.f; cre[j] = 0.f; cim[j] = 0.f; }
#pragma unroll 4
        for (int p = 0; p < n_here; ++p) {
            const uint4 r = sp[p];
            const float qp = __uint_as_float(r.w);
#pragma unroll
            for (int j = 0; j < KPT; ++j) {
                const float th = fixed_phase(mx[j], my[j], mz[j], r.x, r.y, r.z);
                float sn, cs;
                __sincosf(th, &sn, &cs);
                if (ACC == RBE_RHO_FP32) {
                    re[j] = fmaf(qp, cs, re[j]);
                    im[j] = fmaf(qp, sn, im[j]);
                } else if (ACC == RBE_RHO_COMP32) {
                    const float yr = qp * cs - cre[j];
                    const float tr = re[j] + yr;
                    cre[j] = (tr - re[j]) - yr;
                    re[j] = tr;
                    const float yi = qp * sn - cim[j];
                    const float ti = im[j] + yi;
                    cim[j] = (ti - im[j]) - yi;
                    im[j] = ti;
                } else {
                    are[j] = fma((double)qp, (double)cs, are[j]);
                    aim[j] = fma((double)qp, (double)sn, aim[j]);
                }
            }
        }
        if (ACC != RBE_RHO_FP64) {
#pragma unroll
            for (int j = 0; j < KPT; ++j) {
                are[j] += (double)re[j] - (double)cre[j];
                aim[j] += (double)im[j] - (double)cim[j];
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        const int l = kt * kT * KPT + j * kT + tid;
        if (l < K) partials[(size_t)l * nchunks + c] = make_double2(are[j], aim[j]);
    }
    if (kt == 0) {
        // sum of q^2 over the chunk for E_self: fixed-order tree over the block
        __shared__ double sq[kT];
        sq[tid] = q2;
        __syncthreads();
        for (int s = kT / 2; s > 0; s >>= 1) {
            if (tid < s) sq[tid] += sq[tid + s];
            __syncthreads();
        }
        if (tid == 0) partials[(size_t)K * nchunks + c] = make_double2(sq[0], 0.0);
    }
}

// rho pass, FP64 path: s = r / l wrapped to [0, 1); t = m.s - rint(m.s); sincospi(2t).
template <int KPT>
__global__ void __launch_bounds__(kT) k_rho_f64(const double* __restrict__ pos, const double* __restrict__ q,
                                                int64_t N, double ilx, double ily, double ilz,
                                                const int4* __restrict__ m, int K, int chunk_len,
                                                int nchunks, double2* __restrict__ partials,
                                                unsigned* __restrict__ status)
{
    __shared__ double4_32a sp[kT];
    const int tid = threadIdx.x;
    const int kt = blockIdx.x;
    const int c = blockIdx.y;
    double mx[KPT], my[KPT], mz[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        const int l = kt * kT * KPT + j * kT + tid;
        int4 v = l < K ? m[l] : make_int4(0, 0, 0, 0);
        mx[j] = v.x; my[j] = v.y; mz[j] = v.z;
    }
    double re[KPT], im[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) { re[j] = 0.0; im[j] = 0.0; }
    double q2 = 0.0;
    const int64_t start = (int64_t)c * chunk_len;
    const int64_t end = min(N, start + (int64_t)chunk_len);
    for (int64_t base = start; base < end; base += kT) {
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
        const int n_here = (int)min((int64_t)kT, end - base);
#pragma unroll 2
        for (int p = 0; p < n_here; ++p) {
            const double4_32a r = sp[p];
#pragma unroll
            for (int j = 0; j < KPT; ++j) {
                double t = fma(mx[j], r.x, fma(my[j], r.y, mz[j] * r.z));
                t -= rint(t);
                double sn, cs;
                sincospi(2.0 * t, &sn, &cs);
                re[j] = fma(r.w, cs, re[j]);
                im[j] = fma(r.w, sn, im[j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        const int l = kt * kT * KPT + j * kT + tid;
        if (l < K) partials[(size_t)l * nchunks + c] = make_double2(re[j], im[j]);
    }
    if (kt == 0) {
        __shared__ double sq[kT];
        sq[tid] = q2;
        __syncthreads();
        for (int s = kT / 2; s > 0; s >>= 1) {
            if (tid < s) sq[tid] += sq[tid + s];
            __syncthreads();
        }
        if (tid == 0) partials[(size_t)K * nchunks + c] = make_double2(sq[0], 0.0);
    }
}

// =================================================================================
// Reduction of the partials (one warp per frequency, fixed order), the per-frequency
// terms, and -- in the last block to finish -- the energy and virial sums over l.
//   e_l = (2 pi / V) w_l |rho_l|^2 / |k_l|^2
//   W  += e_l [I - 2 (1/|k_l|^2 + 1/4a) k_l k_l]
//   force coefficients beta_l = w_l 4 pi / (V |k_l|^2), A_l = beta_l Im rho_l, B_l = beta_l Re rho_l,
//   so that F_i = q_i sum_l k_l (sin(k_l.r_i) B_l - cos(k_l.r_i) A_l).
constexpr int kReduceWarps = 8;

__global__ void __launch_bounds__(32 * kReduceWarps)
k_reduce(const double2* __restrict__ partials, int nchunks, int K, const int4* __restrict__ m,
         const double* __restrict__ w, double bx, double by, double bz, double alpha,
         double2* __restrict__ rho, double* __restrict__ terms, int4* __restrict__ coef_m,
         float4* __restrict__ coef_f, double2* __restrict__ coef_d, unsigned* __restrict__ counter,
         unsigned* __restrict__ status, double* __restrict__ W_out, double* __restrict__ E_out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int l = blockIdx.x * kReduceWarps + warp;
    if (l <= K) {
        double re = 0.0, im = 0.0;
        const double2* row = partials + (size_t)l * nchunks;
        for (int j = lane; j < nchunks; j += 32) {
            const double2 v = row[j];
            re += v.x;
            im += v.y;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, off);
            im += __shfl_xor_sync(0xffffffffu, im, off);
        }
        if (lane == 0) {
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
        }
    }
    // Last block to finish sums the per-frequency terms in a fixed order.
    __shared__ bool is_last;
    __shared__ double red[32 * kReduceWarps][7];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        const double* t = terms + (size_t)j * 8;
#pragma unroll
        for (int a = 0; a < 7; ++a) acc[a] += __ldcg(t + a);
    }
#pragma unroll
    for (int a = 0; a < 7; ++a) red[threadIdx.x][a] = acc[a];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int a = 0; a < 7; ++a) red[threadIdx.x][a] += red[threadIdx.x + s][a];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double q2 = __ldcg(terms + (size_t)K * 8);
        const double Ek = red[0][0];
        const double Es = -sqrt(alpha / kPi) * q2;
        if (W_out) {
            W_out[0] = red[0][1]; W_out[4] = red[0][2]; W_out[8] = red[0][3];
            W_out[1] = W_out[3] = red[0][4];
            W_out[2] = W_out[6] = red[0][5];
            W_out[5] = W_out[7] = red[0][6];
        }
        if (E_out) { E_out[0] = Ek; E_out[1] = Es; }
        bool ok = isfinite(Ek) && isfinite(Es);
        for (int a = 1; a < 7; ++a) ok = ok && isfinite(red[0][a]);
        if (!ok) atomicOr(status, kStatusNonFinite);
        *counter = 0u;  // ready for the next launch
    }
}

// =================================================================================
// Force pass, FP32-phase path.  Each thread owns PPT particles; frequencies are staged
// in shared memory kForceKT at a time as (mx, my, mz, A) and (B, mx, my, mz).
// F_i,theta = q_i (2 pi / l_theta) sum_l m_l,theta (sin B_l - cos A_l): FP32 within a
// staged tile, FP64 across tiles.
template <int PPT>
__global__ void __launch_bounds__(kT) k_force_f32(const double* __restrict__ pos, const double* __restrict__ q,
                                                  int64_t N, double ilx, double ily, double ilz,
                                                  const int4* __restrict__ coef_m,
                                                  const float4* __restrict__ coef_f, int K,
                                                  double* __restrict__ F)
{
    __shared__ int4 sm[kForceKT];
    __shared__ float4 sf[kForceKT];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * kT * PPT + tid;
    uint32_t sx[PPT], sy[PPT], sz[PPT];
    double fx[PPT], fy[PPT], fz[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int64_t i = i0 + (int64_t)p * kT;
        if (i < N) {
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
        for (int j = tid; j < nk; j += kT) {
            sm[j] = coef_m[k0 + j];
            sf[j] = coef_f[k0 + j];
        }
        __syncthreads();
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
                const float th = fixed_phase(a.x, a.y, a.z, sx[p], sy[p], sz[p]);
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
        __syncthreads();
    }
    const double cx = 2.0 * kPi * ilx, cy = 2.0 * kPi * ily, cz = 2.0 * kPi * ilz;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int64_t i = i0 + (int64_t)p * kT;
        if (i < N) {
            const double qi = q[i];
            F[3 * i] = qi * cx * fx[p];
            F[3 * i + 1] = qi * cy * fy[p];
            F[3 * i + 2] = qi * cz * fz[p];
        }
    }
}

// Force pass, FP64 path.
template <int PPT>
__global__ void __launch_bounds__(kT) k_force_f64(const double* __restrict__ pos, const double* __restrict__ q,
                                                  int64_t N, double ilx, double ily, double ilz,
                                                  const int4* __restrict__ mk, const double2* __restrict__ coef_d,
                                                  int K, double* __restrict__ F)
{
    __shared__ double4_32a sk[kForceKT];  // (mx, my, mz, A)
    __shared__ double sb[kForceKT];   // B
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * kT * PPT + tid;
    double sx[PPT], sy[PPT], sz[PPT], fx[PPT], fy[PPT], fz[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int64_t i = i0 + (int64_t)p * kT;
        if (i < N) {
            sx[p] = pos[3 * i] * ilx; sy[p] = pos[3 * i + 1] * ily; sz[p] = pos[3 * i + 2] * ilz;
            sx[p] -= floor(sx[p]); sy[p] -= floor(sy[p]); sz[p] -= floor(sz[p]);
        } else {
            sx[p] = sy[p] = sz[p] = 0.0;
        }
        fx[p] = fy[p] = fz[p] = 0.0;
    }
    for (int k0 = 0; k0 < K; k0 += kForceKT) {
        const int nk = min(kForceKT, K - k0);
        for (int j = tid; j < nk; j += kT) {
            const int4 mm = mk[k0 + j];
            const double2 ab = coef_d[k0 + j];
            sk[j] = make_double4_32a((double)mm.x, (double)mm.y, (double)mm.z, ab.x);
            sb[j] = ab.y;
        }
        __syncthreads();
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
        __syncthreads();
    }
    const double cx = 2.0 * kPi * ilx, cy = 2.0 * kPi * ily, cz = 2.0 * kPi * ilz;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int64_t i = i0 + (int64_t)p * kT;
        if (i < N) {
            const double qi = q[i];
            F[3 * i] = qi * cx * fx[p];
            F[3 * i + 1] = qi * cy * fy[p];
            F[3 * i + 2] = qi * cz * fz[p];
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

rbe_status launch_sample(rbe_ctx ctx, uint64_t step, int P)
{
    rbe_status st = ensure_tables(ctx);
    if (st != RBE_OK) return st;
    st = ensure_k_capacity(ctx, P);
    if (st != RBE_OK) return st;
    record_event(ctx, 0);
    const int threads = 128;
    k_sample<<<(P + threads - 1) / threads, threads, 0, ctx->stream>>>(
        ctx->seed, step, P, ctx->d.cdf, ctx->d.tab_cap, ctx->d.hdr, ctx->d.m, ctx->d.w, ctx->d.status);
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

// Launch plan: frequencies per thread from K; particle chunks so that the rho grid
// holds about one resident wave; chunk lengths in whole staging tiles.
static Plan make_plan(rbe_ctx ctx, int64_t N, int K)
{
    Plan p{};
    p.kpt = K <= kT ? 1 : (K <= 2 * kT ? 2 : 4);
    p.ktiles = (K + kT * p.kpt - 1) / (kT * p.kpt);
    const int resident = ctx->num_sms * 8;  // 8 blocks of 128 threads per SM
    int64_t want = std::max<int64_t>(1, resident / p.ktiles);
    int64_t tiles = std::max<int64_t>(1, (N + kT - 1) / kT);
    int64_t nch = std::min<int64_t>(want, tiles);
    int64_t tiles_per_chunk = (tiles + nch - 1) / nch;
    p.chunk_len = (int)(tiles_per_chunk * kT);
    p.nchunks = (int)std::max<int64_t>(1, (N + p.chunk_len - 1) / p.chunk_len);
    p.ppt = 2;
    p.fblocks = (int)((N + (int64_t)kT * p.ppt - 1) / ((int64_t)kT * p.ppt));
    return p;
}

rbe_status launch_evaluate(rbe_ctx ctx, int64_t N, const double* pos, const double* q, int K,
                           bool /*uniform_weight*/, double* F, double* W, double* E)
{
    DeviceBuffers& d = ctx->d;
    const Plan p = make_plan(ctx, N, K);
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
    cudaStream_t s = ctx->stream;
    if (ctx->precision == RBE_FP64) {
        switch (p.kpt) {
        case 1: k_rho_f64<1><<<grid, kT, 0, s>>>(pos, q, N, ilx, ily, ilz, d.m, K, p.chunk_len, p.nchunks, d.partials, d.status); break;
        case 2: k_rho_f64<2><<<grid, kT, 0, s>>>(pos, q, N, ilx, ily, ilz, d.m, K, p.chunk_len, p.nchunks, d.partials, d.status); break;
        default: k_rho_f64<4><<<grid, kT, 0, s>>>(pos, q, N, ilx, ily, ilz, d.m, K, p.chunk_len, p.nchunks, d.partials, d.status); break;
        }
    } else {
#define RBE_RHO32(KPT, ACC) \
    k_rho_f32<KPT, ACC><<<grid, kT, 0, s>>>(pos, q, N, ilx, ily, ilz, d.m, K, p.chunk_len, p.nchunks, d.partials, d.status)
#define RBE_RHO32_ACC(KPT)                                      \
    switch (ctx->rho_accum) {                                   \
    case RBE_RHO_FP64: RBE_RHO32(KPT, RBE_RHO_FP64); break;     \
    case RBE_RHO_COMP32: RBE_RHO32(KPT, RBE_RHO_COMP32); break; \
    default: RBE_RHO32(KPT, RBE_RHO_FP32); break;               \
    }
        switch (p.kpt) {
        case 1: RBE_RHO32_ACC(1); break;
        case 2: RBE_RHO32_ACC(2); break;
        default: RBE_RHO32_ACC(4); break;
        }
#undef RBE_RHO32_ACC
#undef RBE_RHO32
    }
    rbe_status st = check_launch(ctx, "k_rho");
    if (st != RBE_OK) return st;
    record_event(ctx, 2);
    const int rblocks = (K + 1 + kReduceWarps - 1) / kReduceWarps;
    k_reduce<<<rblocks, 32 * kReduceWarps, 0, s>>>(d.partials, p.nchunks, K, d.m, d.w, ctx->box[0], ctx->box[1],
                                                   ctx->box[2], ctx->alpha, d.rho, d.terms, d.coef_m, d.coef_f,
                                                   d.coef_d, d.counter, d.status, W, E);
    st = check_launch(ctx, "k_reduce");
    if (st != RBE_OK) return st;
    record_event(ctx, 3);
    if (p.fblocks > 0) {
        if (ctx->precision == RBE_FP64)
            k_force_f64<2><<<p.fblocks, kT, 0, s>>>(pos, q, N, ilx, ily, ilz, d.m, d.coef_d, K, F);
        else
            k_force_f32<2><<<p.fblocks, kT, 0, s>>>(pos, q, N, ilx, ily, ilz, d.coef_m, d.coef_f, K, F);
        st = check_launch(ctx, "k_force");
        if (st != RBE_OK) return st;
    }
    record_event(ctx, 4);
    ctx->last_K = K;
    return RBE_OK;
}

}  // namespace rbe
