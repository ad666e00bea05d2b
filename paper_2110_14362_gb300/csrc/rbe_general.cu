// RBE k-space forces, virial and energy in a general (triclinic) cell (App. C: the fully
// flexible cell), on the tuned rectangular passes.
//
// Cell h = (a | b | c) with the cell vectors as columns, r = h s, V = det h, k = 2 pi h^{-T} m, so
// the phase k.r = 2 pi m.s is the unit cube's phase of the scaled coordinates s.  One evaluation:
//   k_tables        per-axis tables of the MH proposal (effective lengths l_j, see below)
//   k_gen_mh        one MH step per frequency slot (App. C suggests discrete MH: the law
//                   exp(-pi^2 m^T G m / alpha), G = h^{-1} h^{-T}, does not factorise) and the
//                   unit-cube weight w'_l = (S/P) |m|^2 / (V m^T G m) of each frequency
//   k_tables        the unit cube's box state
//   k_gen_scale     s = h^{-1} r
//   rho, reduction, force pass of the rectangular path on s in the unit cube: with the weights
//                   w' its energy is (2 pi / V) sum (S/P) |rho|^2 / |k|^2 and its forces the
//                   gradient in s, dE/ds = h^T dE/dr
//   k_gen_finish    F = h^{-T} F_s
//   k_gen_virial    W = (2 pi / V) sum (S/P) |rho|^2/|k|^2 [I - 2 (1/|k|^2 + 1/4 alpha) k k^T]
//                   (App. C Eq. (pressuretensorflexible)) from rho and the true k
// MH proposal: the exact product of per-axis discrete Gaussians with effective lengths
// l_j = sqrt(lambda |a_j|^2), lambda = max_j (1 + sum_{k != j} |cos theta_jk|), whose precision
// stays below the target's (bounded ratio: uniform mixing; a rectangular cell proposes the target
// itself).  Acceptance with O(m) = (pi^2/alpha) m^T G m - sum_j c_j m_j^2: m' when O(m') <= O(m),
// else when u < exp(O(m) - O(m')), u from Philox stream 5 (l, 0, step_lo, (5 << 24) | step_hi24).
// S, the importance normalisation, from the dual lattice sum (alpha/pi)^{3/2} V sum_n
// exp(-alpha |h n|^2) - 1 (Poisson summation).  The cell quantities that decide integers (G, c_j,
// pi^2/alpha) are formed on the host with separately rounded operations (no contraction).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "rbe_context.h"
#include "rbe_device.cuh"
#include "rbe_kspace_tiles.cuh"
#include "rbe_sampler_variants.cuh"
#include "rbe_general.cuh"

namespace rbe {

__global__ void k_gen_mh(uint64_t seed, uint64_t step, int P, const unsigned long long* __restrict__ cum, int cap,
                         const KState* __restrict__ ks, int4* __restrict__ chain, const GenCell g,
                         int4* __restrict__ m_out, double* __restrict__ w_out, unsigned* __restrict__ status)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= P) return;
    gen_mh_slot(l, seed, step, cum, cap, ks, chain, g, m_out, w_out, status);
}

__global__ void k_gen_scale(int64_t N, const double* __restrict__ pos, const GenCell g, double* __restrict__ s)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    for (int t = 0; t < 3; ++t) s[3 * i + t] = g.hinv[3 * t] * x + g.hinv[3 * t + 1] * y + g.hinv[3 * t + 2] * z;
}

// F = h^{-T} F_s in place
__global__ void k_gen_finish(int64_t N, double* __restrict__ F, const GenCell g)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double a = F[3 * i], b = F[3 * i + 1], c = F[3 * i + 2];
    for (int t = 0; t < 3; ++t) F[3 * i + t] = g.hinv[t] * a + g.hinv[3 + t] * b + g.hinv[6 + t] * c;
}

// The general virial from rho (one block, fixed-order sums).
__global__ void __launch_bounds__(kGenVirThreads)
k_gen_virial(int P, const int4* __restrict__ m, const double2* __restrict__ rho, const GenCell g, double alpha,
             double* __restrict__ W_out, unsigned* __restrict__ status)
{
    gen_virial_block(P, m, rho, g, alpha, W_out, status);
}

}  // namespace rbe

// ---------------------------------------------------------------------------------
// Host side.
namespace rbe {

constexpr double kPiHost = 3.14159265358979323846;

// The cell quantities, each with separately rounded operations (the host build disables
// contraction) in the same order as the oracle's: h^{-1} by cofactors, G, the proposal lengths.
static bool gen_cell(const double h[9], double alpha, int P, GenCell& g)
{
    const double c00 = h[4] * h[8] - h[5] * h[7], c01 = h[5] * h[6] - h[3] * h[8], c02 = h[3] * h[7] - h[4] * h[6];
    const double det = h[0] * c00 + h[1] * c01 + h[2] * c02;
    if (!(det > 0.0) || !std::isfinite(det)) return false;
    double* hi = g.hinv;
    hi[0] = c00 / det;
    hi[1] = (h[2] * h[7] - h[1] * h[8]) / det;
    hi[2] = (h[1] * h[5] - h[2] * h[4]) / det;
    hi[3] = c01 / det;
    hi[4] = (h[0] * h[8] - h[2] * h[6]) / det;
    hi[5] = (h[2] * h[3] - h[0] * h[5]) / det;
    hi[6] = c02 / det;
    hi[7] = (h[1] * h[6] - h[0] * h[7]) / det;
    hi[8] = (h[0] * h[4] - h[1] * h[3]) / det;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            g.G[3 * i + j] = hi[3 * i] * hi[3 * j] + hi[3 * i + 1] * hi[3 * j + 1] + hi[3 * i + 2] * hi[3 * j + 2];
    double gg[9];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) gg[3 * j + k] = h[j] * h[k] + h[3 + j] * h[3 + k] + h[6 + j] * h[6 + k];
    double lam = 1.0;
    for (int j = 0; j < 3; ++j) {
        double row = 1.0;
        for (int k = 0; k < 3; ++k)
            if (k != j) row = row + std::fabs(gg[3 * j + k] / std::sqrt(gg[3 * j + j] * gg[3 * k + k]));
        if (row > lam) lam = row;
    }
    for (int j = 0; j < 3; ++j) {
        g.leff[j] = std::sqrt(lam * gg[3 * j + j]);
        g.c[j] = (kPiHost * kPiHost) / (alpha * (g.leff[j] * g.leff[j]));
    }
    g.co = (kPiHost * kPiHost) / alpha;
    g.V = det;
    // S by the dual sum over the n with alpha |h n|^2 <= 60 ln 2 + 50
    const double cut = (60.0 * 0.69314718055994530942 + 50.0) / alpha;
    int R[3];
    for (int t = 0; t < 3; ++t) {
        const double rn = std::sqrt(hi[3 * t] * hi[3 * t] + hi[3 * t + 1] * hi[3 * t + 1] + hi[3 * t + 2] * hi[3 * t + 2]);
        const double Rd = std::ceil(std::sqrt(cut) * rn) + 1.0;
        if (!(Rd <= 4096.0)) return false;
        R[t] = (int)Rd;
    }
    double sum = 0.0;
    for (int a = -R[0]; a <= R[0]; ++a)
        for (int b = -R[1]; b <= R[1]; ++b)
            for (int c = -R[2]; c <= R[2]; ++c) {
                double x[3];
                for (int t = 0; t < 3; ++t) x[t] = h[3 * t] * a + h[3 * t + 1] * b + h[3 * t + 2] * c;
                const double d2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
                if (d2 <= cut) sum += std::exp(-alpha * d2);
            }
    g.S = std::pow(alpha / kPiHost, 1.5) * det * sum - 1.0;
    g.wP = g.S / (double)P;
    return std::isfinite(g.S) && g.S > 0.0;
}

}  // namespace rbe

using namespace rbe;

rbe_status rbe_kspace_forces_virial_general(rbe_ctx ctx, int64_t N, const double* positions, const double* charges,
                                            const double h[9], uint64_t step, double* forces_out,
                                            double* virial_out, double* energy_out)
{
    if (!ctx) return RBE_EINVAL;
    if (!h) return fail(ctx, RBE_EINVAL, "h is NULL");
    if (N < 0 || N > ((int64_t)1 << 31) - 256) return fail(ctx, RBE_EINVAL, "N out of range [0, 2^31 - 256]");
    if ((step >> 56) != 0) return fail(ctx, RBE_EINVAL, "step must be < 2^56");
    rbe_status st;
    if ((st = check_dev(ctx, positions, "positions", N > 0)) != RBE_OK ||
        (st = check_dev(ctx, charges, "charges", N > 0)) != RBE_OK ||
        (st = check_dev(ctx, forces_out, "forces_out", N > 0)) != RBE_OK ||
        (st = check_dev(ctx, virial_out, "virial_out", false)) != RBE_OK ||
        (st = check_dev(ctx, energy_out, "energy_out", false)) != RBE_OK)
        return st;
    for (int t = 0; t < 9; ++t)
        if (!std::isfinite(h[t])) return fail(ctx, RBE_EINVAL, "h must be finite");
    const int P = ctx->P;
    GenCell g;
    if (!gen_cell(h, ctx->alpha, P, g)) return fail(ctx, RBE_EINVAL, "h must have a positive determinant and a sane size");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != ctx->device) cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    cudaError_t e;
    // tables for the proposal lengths
    int need = 0;
    for (int t = 0; t < 3; ++t) {
        const int M = host_axis_M(ctx->alpha, g.leff[t]);
        if (M > (1 << 20)) return fail(ctx, RBE_EINVAL, "alpha |a_j|^2 too large for the per-axis tables");
        need = std::max(need, 2 * M + 1);
    }
    if ((st = ensure_table_capacity(ctx, need)) != RBE_OK) return st;
    if ((st = ensure_k_capacity(ctx, P)) != RBE_OK) return st;
    if (ctx->gchain_cap < P) {
        ctx_free(ctx, ctx->gchain);
        ctx->gchain = nullptr;
        ctx->gchain_cap = 0;
        if ((e = ctx_alloc(ctx, &ctx->gchain, sizeof(int4) * (size_t)std::max(P, 1))) != cudaSuccess ||
            (e = cudaMemsetAsync(ctx->gchain, 0, sizeof(int4) * (size_t)std::max(P, 1), s)) != cudaSuccess)
            return cuda_fail(ctx, e, "general-cell MH chain");
        ctx->gchain_cap = P;
    }
    if (N > ctx->gpos_cap) {
        ctx_free(ctx, ctx->gpos);
        ctx->gpos = nullptr;
        ctx->gpos_cap = 0;
        if ((e = ctx_alloc(ctx, &ctx->gpos, sizeof(double) * 3 * (size_t)N)) != cudaSuccess)
            return cuda_fail(ctx, e, "scaled coordinates");
        ctx->gpos_cap = N;
    }
    if ((st = launch_tables_box(ctx, g.leff)) != RBE_OK) return st;
    if (P > 0)
        k_gen_mh<<<(P + 127) / 128, 128, 0, s>>>(ctx->seed, step, P, ctx->d.cum, ctx->d.tab_cap, ctx->d.ks, ctx->gchain,
                                                 g, ctx->d.m, ctx->d.w, ctx->d.status);
    const double unit[3] = {1.0, 1.0, 1.0};
    if ((st = launch_tables_box(ctx, unit)) != RBE_OK) return st;
    const int nb = (int)((N + 255) / 256);
    if (N > 0) k_gen_scale<<<nb, 256, 0, s>>>(N, positions, g, ctx->gpos);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "k_gen_mh/k_gen_scale");
    if ((st = launch_evaluate(ctx, N, ctx->gpos, charges, P, false, forces_out, nullptr, energy_out)) != RBE_OK)
        return st;
    if (N > 0) k_gen_finish<<<nb, 256, 0, s>>>(N, forces_out, g);
    k_gen_virial<<<1, kGenVirThreads, 0, s>>>(P, ctx->d.m, ctx->d.rho, g, ctx->alpha, virial_out, ctx->d.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "k_gen_finish/k_gen_virial");
    return RBE_OK;
}
