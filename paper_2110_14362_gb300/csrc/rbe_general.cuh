// General-cell (triclinic) pieces shared by the k-space evaluation of rbe_general.cu and the
// device-resident flexible-cell step of rbe_flex.cu: the cell quantities, the MH step of one
// frequency slot (App. C) and the virial from rho (App. C Eq. (pressuretensorflexible)).
#pragma once

#include <cuda_runtime.h>

#include "rbe_device.cuh"
#include "rbe_kspace_tiles.cuh"
#include "rbe_sampler_variants.cuh"

namespace rbe {

struct GenCell {
    double hinv[9];  // h^{-1}, row-major
    double G[9];     // h^{-1} h^{-T}
    double leff[3];  // proposal lengths
    double c[3];     // proposal precisions pi^2 / (alpha l_j^2)
    double co;       // pi^2 / alpha
    double V, S, wP; // det h, the dual-sum S, S / P
};

// O(m) = co m^T G m - sum_j c_j m_j^2, in the oracle's order, separately rounded.
__device__ __forceinline__ double gen_off(const GenCell& g, const int m[3])
{
    double q = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) q = __dadd_rn(q, __dmul_rn(__dmul_rn(g.G[3 * i + j], (double)m[i]), (double)m[j]));
    double d = 0.0;
    for (int j = 0; j < 3; ++j) d = __dadd_rn(d, __dmul_rn(__dmul_rn(g.c[j], (double)m[j]), (double)m[j]));
    return __dsub_rn(__dmul_rn(g.co, q), d);
}

// One MH step of frequency slot l (the kernels k_gen_mh and, for the device-resident flexible
// cell, k_flex_mh): the proposal from the product tables, acceptance, the chain state, m and w'.
__device__ __forceinline__ void gen_mh_slot(int l, uint64_t seed, uint64_t step, const unsigned long long* __restrict__ cum,
                                            int cap, const KState* __restrict__ ks, int4* __restrict__ chain,
                                            const GenCell& g, int4* __restrict__ m_out, double* __restrict__ w_out,
                                            unsigned* __restrict__ status)
{
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t c2 = (uint32_t)step, c3 = (uint32_t)((step >> 32) & 0xFFFFFFu);
    int4 mp;
    if (!smp_exact(cum, cap, ks, k0, k1, c2, c3, l, mp)) {
        atomicOr(status, kStatusSample);
        m_out[l] = make_int4(1, 0, 0, 0);  // keeps the evaluation finite; the call reports RBE_ESAMPLE
        w_out[l] = 0.0;
        return;
    }
    int4 cur = chain[l];
    if (cur.x == 0 && cur.y == 0 && cur.z == 0) {
        cur = mp;
    } else {
        const int a[3] = {cur.x, cur.y, cur.z}, b[3] = {mp.x, mp.y, mp.z};
        const double d = __dsub_rn(gen_off(g, a), gen_off(g, b));
        bool accept;
        if (d >= 0.0) {
            accept = true;
        } else if (d < -700.0) {
            accept = false;
        } else {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)l, 0u, c2, (5u << 24) | c3), k0, k1);
            accept = smp_u53(w.x, w.y) < table_exp(d);
        }
        if (accept) cur = mp;
    }
    chain[l] = cur;
    m_out[l] = cur;
    const double mx = cur.x, my = cur.y, mz = cur.z;
    const double mm = mx * mx + my * my + mz * mz;
    double mgm = 0.0;
    const double v[3] = {mx, my, mz};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) mgm += g.G[3 * i + j] * v[i] * v[j];
    w_out[l] = g.wP * mm / (g.V * mgm);
}


constexpr int kGenVirThreads = 256;

// The general virial from rho (one block of kGenVirThreads threads, fixed-order sums).
__device__ __forceinline__ void gen_virial_block(int P, const int4* __restrict__ m, const double2* __restrict__ rho,
                                                 const GenCell& g, double alpha, double* __restrict__ W_out,
                                                 unsigned* __restrict__ status)
{
    __shared__ double red[6][kGenVirThreads];
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const double twopi = 2.0 * kPi;
    for (int l = threadIdx.x; l < P; l += kGenVirThreads) {
        const int4 mi = m[l];
        double k[3];
        for (int t = 0; t < 3; ++t)
            k[t] = twopi * (g.hinv[t] * mi.x + g.hinv[3 + t] * mi.y + g.hinv[6 + t] * mi.z);
        const double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        const double2 r = rho[l];
        const double e = (twopi / g.V) * (g.wP / kk) * (r.x * r.x + r.y * r.y);
        const double b = 2.0 * (1.0 / kk + 1.0 / (4.0 * alpha));
        acc[0] += e * (1.0 - b * k[0] * k[0]);
        acc[1] += e * (1.0 - b * k[1] * k[1]);
        acc[2] += e * (1.0 - b * k[2] * k[2]);
        acc[3] -= e * b * k[0] * k[1];
        acc[4] -= e * b * k[0] * k[2];
        acc[5] -= e * b * k[1] * k[2];
    }
    for (int a = 0; a < 6; ++a) red[a][threadIdx.x] = acc[a];
    __syncthreads();
    for (int half = kGenVirThreads / 2; half > 0; half >>= 1) {
        if ((int)threadIdx.x < half)
            for (int a = 0; a < 6; ++a) red[a][threadIdx.x] += red[a][threadIdx.x + half];
        __syncthreads();
    }
    if (threadIdx.x == 0 && W_out) {
        W_out[0] = red[0][0];
        W_out[4] = red[1][0];
        W_out[8] = red[2][0];
        W_out[1] = W_out[3] = red[3][0];
        W_out[2] = W_out[6] = red[4][0];
        W_out[5] = W_out[7] = red[5][0];
        for (int a = 0; a < 6; ++a)
            if (!isfinite(red[a][0])) atomicOr(status, kStatusNonFinite);
    }
}

}  // namespace rbe
