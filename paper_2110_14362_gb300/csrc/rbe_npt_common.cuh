// Definitions shared by the NPT steps of the rectangular cells (rbe_npt.cu) and of the fully
// flexible cell (rbe_flex.cu): launch shapes, the Langevin normals, the cell-list constants and
// the real-space pair constants.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "rbe_device.cuh"

namespace rbe {

constexpr double kFConv = 100.0;  // kJ/mol/A per g/mol -> A/ps^2
constexpr int kNptThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kSortWarps = 8;        // k_cl_sort: warps (cells) per block
constexpr int kPairWarps = 8;        // k_pair: warps (particles in flight) per block
constexpr int kPairBlocksPerSM = 4;  // k_pair (FP32): resident blocks per SM the grid is sized for
constexpr int kPairBlocksPerSM64 = 2;  // k_pair (FP64): more registers per thread
constexpr int kListBatch = 4;        // k_pair (list): list entries per lane loaded together
constexpr int kHitCap = 32 * (kListBatch + 1);  // k_pair: buffered candidates per warp (< 32 + 32 kListBatch)
// Per-block partial sums of the pair and finishing kernels: 8 doubles per block.  Isotropic:
// finishing blocks {2K} at slot 0, pair blocks {W, E_coul, E_lj} at 1..3.  Rectangular cells:
// finishing blocks {2K_x, 2K_y, 2K_z} at 0..2, pair blocks {W_xx, W_yy, W_zz, E_coul, E_lj} at 3..7.
// Flexible cell: finishing blocks {K_xx, K_yy, K_zz, K_xy, K_xz, K_yz} at 0..5, pair blocks
// {W_xx, W_yy, W_zz, W_xy, W_xz, W_yz, E_coul, E_lj} at 0..7.
constexpr int kPartStride = 8;

// Four standard normals from one Philox call: u = (w + 1/2) 2^-32, Box--Muller.
__device__ __forceinline__ void npt_normals(uint64_t seed, uint32_t stream, uint64_t step, uint32_t index,
                                            double z[4])
{
    const uint4 w = philox4x32_10(make_uint4(index, 0u, (uint32_t)step,
                                             (stream << 24) | (uint32_t)((step >> 32) & 0xFFFFFFu)),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u0 = ((double)w.x + 0.5) * 0x1.0p-32, u1 = ((double)w.y + 0.5) * 0x1.0p-32;
    const double u2 = ((double)w.z + 0.5) * 0x1.0p-32, u3 = ((double)w.w + 0.5) * 0x1.0p-32;
    double s, c;
    const double r0 = sqrt(-2.0 * log(u0));
    sincospi(2.0 * u1, &s, &c);
    z[0] = r0 * c;
    z[1] = r0 * s;
    const double r1 = sqrt(-2.0 * log(u2));
    sincospi(2.0 * u3, &s, &c);
    z[2] = r1 * c;
    z[3] = r1 * s;
}

// The same four normals in FP32 (FP32-phase path): Box--Muller with the fast logarithm and
// sine/cosine; the angle 2 pi u is taken as 2 pi (u - 1/2) + pi, so that the argument of the
// fast sine/cosine stays in [-pi, pi).
__device__ __forceinline__ void npt_normals_f32(uint64_t seed, uint32_t stream, uint64_t step, uint32_t index,
                                                double z[4])
{
    const uint4 w = philox4x32_10(make_uint4(index, 0u, (uint32_t)step,
                                             (stream << 24) | (uint32_t)((step >> 32) & 0xFFFFFFu)),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    const float k = 0x1.0p-32f, two_pi = 6.28318530717958647692f;
    const float u0 = ((float)w.x + 0.5f) * k, u1 = ((float)w.y + 0.5f) * k;
    const float u2 = ((float)w.z + 0.5f) * k, u3 = ((float)w.w + 0.5f) * k;
    float s, c;
    const float r0 = sqrtf(-2.0f * __logf(u0));
    __sincosf(two_pi * (u1 - 0.5f), &s, &c);
    z[0] = -(double)(r0 * c);
    z[1] = -(double)(r0 * s);
    const float r1 = sqrtf(-2.0f * __logf(u2));
    __sincosf(two_pi * (u3 - 0.5f), &s, &c);
    z[2] = -(double)(r1 * c);
    z[3] = -(double)(r1 * s);
}

// Constants of the cell list for the current box, written once per step (by the cell
// update, or k_cell_consts before the first forces), so that no kernel of the step divides
// by the box or by rc itself (FP64 divisions are slow on this GPU).
struct CellConsts {
    double L[3], invL[3];
    float Lf[3], invLf[3];
    float pass64;  // FP64 path: squared FP32 search radius (rc plus 2^-16 l_max)
    int nc[3];     // cells per axis, floor(l / rc) clamped to 1..2^20
    int ncell;     // nc0 nc1 nc2, or -1 when that exceeds the cell arrays
    int ok;        // ncell >= 0 and rc <= l/2 on every axis
};

// erfc(x) for x >= 0 in FP32 by the Chebyshev fit of Press, Teukolsky, Vetterling and Flannery
// (Numerical Recipes, 2nd ed., Sec. 6.2): erfc(x) = t exp(-x^2 + c(t)), t = 1 / (1 + x / 2),
// with c a degree-9 polynomial in t; fractional error below 1.2e-7 for every x >= 0 (plus the
// FP32 rounding of its steps).  The FP32-phase real space uses it in place of erfcf: one
// reciprocal, one exponential and ten FMAs per pair, the same accuracy class, 4 % less time per
// NPT step at N = 1e5.  (Hastings' form t P(t) exp(-x^2), which would reuse the force term's
// exponential, has an absolute error of 1.5e-7: a large relative error near the cutoff, where
// erfc is about 1e-5, which moved the box of a three-step run by 2e-9 relative.)
__device__ __forceinline__ float erfc_nr(float x)
{
    const float t = __fdividef(1.0f, fmaf(0.5f, x, 1.0f));
    float c = fmaf(t, 0.17087277f, -0.82215223f);
    c = fmaf(t, c, 1.48851587f);
    c = fmaf(t, c, -1.13520398f);
    c = fmaf(t, c, 0.27886807f);
    c = fmaf(t, c, -0.18628806f);
    c = fmaf(t, c, 0.09678418f);
    c = fmaf(t, c, 0.37409196f);
    c = fmaf(t, c, 1.00002368f);
    c = fmaf(t, c, -1.26551223f);
    return t * __expf(fmaf(-x, x, c));
}

__device__ __forceinline__ int cell_dim(double l, double rc)
{
    // clamped in FP64 before the conversion: any box (huge, infinite, NaN) gives 1..2^20
    // cells per axis, whose product cannot overflow and is checked against the capacity
    const double f = floor(l / rc);
    return f >= 1.0 ? (f <= 1048576.0 ? (int)f : 1048576) : 1;
}

// Pair constants, formed on the host in FP64 and rounded once: the kernel never derives
// them itself (the FP32 kernel would otherwise recompute FP64 products in its loops).
struct PairConst {
    double rc, rc2, sa, a, two_sa_pi, qk, s2, e4, e24;
    float rcf, rc2f, saf, af, two_sa_pif, qkf, s2f, e4f, e24f;
    int lj;
};

static inline PairConst make_pair_const(double rc, double alpha, double qqr2e, double lj_sigma, double lj_eps)
{
    PairConst c;
    c.rc = rc;
    c.rc2 = rc * rc;
    c.sa = std::sqrt(alpha);
    c.a = alpha;
    c.two_sa_pi = 2.0 * std::sqrt(alpha / 3.14159265358979323846);
    c.qk = qqr2e;
    c.s2 = lj_sigma * lj_sigma;
    c.e4 = 4.0 * lj_eps;
    c.e24 = 24.0 * lj_eps;
    c.rcf = (float)c.rc;
    c.rc2f = (float)c.rc2;
    c.saf = (float)c.sa;
    c.af = (float)c.a;
    c.two_sa_pif = (float)c.two_sa_pi;
    c.qkf = (float)c.qk;
    c.s2f = (float)c.s2;
    c.e4f = (float)c.e4;
    c.e24f = (float)c.e24;
    c.lj = lj_eps != 0.0;
    return c;
}

// Neighbour-list state of a replica.  The list holds, for every slot of the cell order of its
// build, the slots within rl = rc + skin (by the nearest image) at the build.  With D the
// largest displacement since then (in units of the build's box) and f the smallest ratio of
// the box edges to the build's, every unlisted pair is now at least f (rl - 2 D) apart: the
// list stands while that is at least rc.
struct NListState {
    double Lref[3];    // box at the last build
    float rl, rc;
    unsigned maxd2;    // bits of the largest squared displacement of this step (non-negative float)
    unsigned counter;  // last-block counter of the check
    int rebuild;       // 1: this step rebuilds the list
    int force;         // 1: build at the next step (set by rbe_npt_init)
};

// Sub-step coefficients of one step, per axis (the isotropic cell writes the same value on
// every axis).
struct NptCoef {
    double a1[3], b1[3];    // R^p/2 before the forces: p_j <- a1_j p_j + 100 F_j b1_j
    double a2m1[3], b2[3];  // first R/2: r_j <- r_j + r_j (a2_j - 1) + (p_j/m) b2_j
    double g, og;           // O: p <- g p + sqrt(og m) z, og = 100 kT (1 - g^2)
    double sog;             // sqrt(og): the O noise amplitude is sog sqrt(m)
    double a3m1[3], b3[3];  // second R/2
    double a4[3], b4[3];    // R^p/2 after the forces
    double L[3];        // box after the second V/2
    double invL[3];     // 1 / L
    double half_cap;    // displacement cap per R/2
    double V;
    int noise;
    int pad;
};

// The step index lives in the cell block (cell[kCellStep], 64-bit integer bits).
constexpr int kCellStep = 11;

__device__ __forceinline__ uint64_t cell_step(const double* cell)
{
    return (uint64_t)__double_as_longlong(cell[kCellStep]);
}

}  // namespace rbe
