// Langevin NPT step on the device (Sec. 3.2-3.3 of the paper; the rectangular cell of the
// appendix, anisotropic or semi-isotropic, by the same splitting per axis) with RBE k-space
// forces (rbe_kspace.cu) and a nearest-image real space on a deterministic cell list, with or
// without a neighbour list.
//
// One step is a fixed sequence of launches on the context's stream:
//   k_npt_cell_a   one block: V^p/2, the sub-step coefficients, V/2, O^p, V/2 (new box),
//                  and the cell-list constants of the new box (k_npt_cell_rect for the
//                  rectangular cell: the same per axis)
//   k_npt_drift    particles: R^p/2, R/2, O, R/2, wrap into the new box
//   k-space        tables for the new box, sampler, rho, reduction, force pass
//   k_nl_check     (neighbour list) packed positions in the list's order, largest
//                  displacement since the build, rebuild decision on the device
//   cell list      count, scan, fill, per-cell sort (deterministic order), packed positions
//                  (with a list: only on rebuild steps; the launches exit at once otherwise)
//   k_pair         real-space forces, virial trace and energies (one warp per particle):
//                  from a cell search, or the list build (rebuild steps) and the list
//   k_npt_finish   F = qqr2e F_k + F_r, R^p/2, kinetic sum; last block: P_ins and V^p/2
// Nothing leaves the device between steps; the step index drives the RBE batch and noise.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <type_traits>
#include <cmath>
#include <string>

#include "rbe_context.h"
#include "rbe_device.cuh"
#include "rbe_npt_common.cuh"

namespace rbe {

// rbe_npt_init sizes the per-axis tables and the cell list for box edges up to this many
// times the initial ones; a box beyond it is flagged (RBE_ESTATE) by the step.
constexpr double kBoxHeadroom = 2.0;


// (e^x - 1)/x * t with x = eps t; the series for tiny x.
__device__ __forceinline__ double expm1_over(double x, double t)
{
    if (fabs(x) < 1e-8) return t * (1.0 + x * (0.5 + x * (1.0 / 6.0 + x / 24.0)));
    return t * expm1(x) / x;
}


// ---------------------------------------------------------------------------------
// Cell-variable part of the step (Sec. 3.3): V^p/2, R^p/2 coefficient, V/2, R/2
// coefficient, O^p, R/2 coefficient, V/2, R^p/2 coefficient.  cell = {l, p_V, W, 2K, ...}.
// The step index lives on the device (cell[kCellStep] as 64-bit integer bits), so that a
// captured sequence of steps can be replayed: every kernel reads it, k_npt_finish advances it.


// Lanes 0..2 of one warp: axis `lane` of the box L; then lane 0 the totals.  Cells of at
// least rcell (rc, or rc + skin when a neighbour list is built from them).
__device__ __forceinline__ void write_cell_consts(int lane, const double* L, double rc, double rcell, int cellcap,
                                                  CellConsts* __restrict__ cc)
{
    if (lane < 3) {
        const double l = L[lane];
        cc->L[lane] = l;
        cc->invL[lane] = 1.0 / l;
        cc->Lf[lane] = (float)l;
        cc->invLf[lane] = (float)(1.0 / l);
        cc->nc[lane] = cell_dim(l, rcell);
    }
    __syncwarp();
    if (lane == 0) {
        const int64_t n = (int64_t)cc->nc[0] * cc->nc[1] * cc->nc[2];
        cc->ncell = n <= (int64_t)cellcap ? (int)n : -1;
        cc->ok = cc->ncell >= 0 && 2.0 * rc <= L[0] && 2.0 * rc <= L[1] && 2.0 * rc <= L[2];
        const double lmax = fmax(L[0], fmax(L[1], L[2]));
        const double rp = rc + lmax * 0x1.0p-16;
        cc->pass64 = (float)(rp * rp);
    }
}

__global__ void k_cell_consts(const double* __restrict__ cell, double rc, double rcell, int cellcap,
                              CellConsts* __restrict__ cc)
{
    write_cell_consts(threadIdx.x, cell, rc, rcell, cellcap, cc);
}


// Per step, before the cell list: refresh the packed positions in the list's slot order and
// decide whether the list must be rebuilt.  Until the first build there is no slot order:
// the kernel then only asks for a build.
template <bool kF64>
__global__ void __launch_bounds__(kNptThreads)
k_nl_check(int64_t N, const double* __restrict__ pos, const double* __restrict__ q, const int* __restrict__ sorted,
           float4* __restrict__ spos32, double4_32a* __restrict__ spos64, const float4* __restrict__ sref,
           const CellConsts* __restrict__ cc, NListState* __restrict__ nls)
{
    __shared__ float smax[kNptThreads / 32];
    __shared__ bool last;
    const bool force = nls->force != 0;
    float d2max = 0.f;
    if (!force) {
        const float Lr[3] = {(float)nls->Lref[0], (float)nls->Lref[1], (float)nls->Lref[2]};
        const double inv[3] = {cc->invL[0], cc->invL[1], cc->invL[2]};
        for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < N; u += (int64_t)gridDim.x * blockDim.x) {
            const int64_t i = sorted[u];
            const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2], qq = q[i];
            spos32[u] = make_float4((float)x, (float)y, (float)z, (float)qq);
            if (kF64) {
                double4_32a v;
                v.x = x;
                v.y = y;
                v.z = z;
                v.w = qq;
                spos64[u] = v;
            }
            const float4 r0 = sref[u];
            float dx = (float)(x * inv[0]) - r0.x, dy = (float)(y * inv[1]) - r0.y, dz = (float)(z * inv[2]) - r0.z;
            dx = (dx - rintf(dx)) * Lr[0];
            dy = (dy - rintf(dy)) * Lr[1];
            dz = (dz - rintf(dz)) * Lr[2];
            const float d2 = dx * dx + dy * dy + dz * dz;
            d2max = d2 > d2max ? d2 : d2max;  // NaN compares false: caught by the box checks
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d2max = fmaxf(d2max, __shfl_xor_sync(0xffffffffu, d2max, off));
    if (lane == 0) smax[warp] = d2max;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < kNptThreads / 32; ++w) m = fmaxf(m, smax[w]);
        atomicMax(&nls->maxd2, __float_as_uint(m));
        __threadfence();
        last = atomicAdd(&nls->counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    const float D = sqrtf(__uint_as_float(atomicAdd(&nls->maxd2, 0u)));
    double f = 1e300;
    for (int t = 0; t < 3; ++t) f = fmin(f, cc->L[t] / nls->Lref[t]);
    // a margin of 1e-3 A covers the FP32 rounding of the displacements
    const bool stands = !force && f * ((double)nls->rl - 2.0 * (double)D - 1e-3) >= (double)nls->rc;
    nls->rebuild = stands ? 0 : 1;
    nls->maxd2 = 0u;
    nls->counter = 0u;
}

__global__ void k_nl_init(NListState* __restrict__ nls, float rl, float rc)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    nls->Lref[0] = nls->Lref[1] = nls->Lref[2] = 1.0;
    nls->rl = rl;
    nls->rc = rc;
    nls->maxd2 = 0u;
    nls->counter = 0u;
    nls->rebuild = 1;
    nls->force = 1;
}

// 1/m and sqrt(m) per particle, once per rbe_npt_init.
__global__ void k_mass_props(int64_t N, const double* __restrict__ mass, double2* __restrict__ mprop)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) mprop[i] = make_double2(1.0 / mass[i], sqrt(mass[i]));
}

__global__ void k_npt_set_step(double* __restrict__ cell, uint64_t step)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) cell[kCellStep] = __longlong_as_double((long long)step);
}

constexpr int kCellWarps = 4;  // k_npt_cell_a: warps

__global__ void __launch_bounds__(kCellWarps * 32)
k_npt_cell_a(double* __restrict__ cell, NptCoef* __restrict__ cf, rbe_npt_params prm, uint64_t seed, int cellcap,
             CellConsts* __restrict__ cc)
{
    // The chain p_V -> box -> p_V -> box runs on warp 0; the exponentials of the sub-step
    // coefficients and the cell noise, independent of one another, run on warps 1..3 (lane 0
    // of each), i.e. on other SM sub-partitions: a single FP64 chain is slow on this GPU,
    // parallel ones are not.  The arithmetic is the same as one thread doing it all.
    __shared__ double sh[24];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t step = cell_step(cell);
    const double h = 0.5 * prm.dt;
    const double MV = prm.M_V;
    if (lane == 0) {
        if (warp == 0) {
            double L[3] = {cell[0], cell[1], cell[2]};
            double V = L[0] * L[1] * L[2];
            double pV = prm.barostat ? cell[3] : 0.0;
            const double W = cell[4], K2 = cell[5];
            if (prm.barostat) pV += h * ((K2 + W) / (3.0 * V) - prm.P_ext);
            sh[0] = prm.barostat ? pV / (3.0 * MV * V) : 0.0;  // eps for the first R^p/2
            if (prm.barostat) {
                const double Vn = V + h * pV / MV;
                const double f = cbrt(Vn / V);
                for (int t = 0; t < 3; ++t) L[t] *= f;
                V = L[0] * L[1] * L[2];
            }
            sh[1] = prm.barostat ? pV / (3.0 * MV * V) : 0.0;  // eps for the first R/2
            sh[2] = pV;
            sh[3] = L[0];
            sh[4] = L[1];
            sh[5] = L[2];
            sh[6] = V;
        } else if (warp == 1) {
            // O^p: friction factor and the noise term of the cell
            double gV = 1.0, nz = 0.0;
            if (prm.barostat) {
                gV = exp(-prm.gamma_V * prm.dt);
                if (prm.noise) {
                    double z[4];
                    npt_normals(seed, 2u, step, 0u, z);
                    nz = sqrt(prm.kT * MV * (1.0 - gV * gV)) * z[0];
                }
            }
            sh[7] = gV;
            sh[8] = nz;
        } else if (warp == 2) {
            const double g = exp(-prm.gamma * prm.dt);
            const double og = prm.kT * kFConv * (1.0 - g * g);
            sh[9] = g;
            sh[10] = og;
            sh[11] = sqrt(og);
        }
    }
    __syncthreads();
    if (lane == 0) {
        if (warp == 0) {
            double L[3] = {sh[3], sh[4], sh[5]};
            double V = sh[6], pV = sh[2];
            if (prm.barostat) {
                pV *= sh[7];
                if (prm.noise) pV += sh[8];
            }
            sh[12] = prm.barostat ? pV / (3.0 * MV * V) : 0.0;  // eps for the second R/2
            if (prm.barostat) {
                const double Vn = V + h * pV / MV;
                const double f = cbrt(Vn / V);
                for (int t = 0; t < 3; ++t) L[t] *= f;
                V = L[0] * L[1] * L[2];
            }
            sh[13] = prm.barostat ? pV / (3.0 * MV * V) : 0.0;  // eps for the second R^p/2
            sh[2] = pV;
            sh[3] = L[0];
            sh[4] = L[1];
            sh[5] = L[2];
            sh[6] = V;
        } else if (warp == 1) {
            sh[14] = exp(-sh[0] * h);
            sh[15] = expm1_over(-sh[0] * h, h);
        } else if (warp == 2) {
            sh[16] = exp(sh[1] * h) - 1.0;
        } else {
            sh[17] = expm1_over(sh[1] * h, h);
        }
    }
    __syncthreads();
    if (warp == 0) {
        write_cell_consts(lane, sh + 3, prm.rc, prm.rc + (prm.skin > 0.0 ? prm.skin : 0.0), cellcap, cc);
    } else if (lane == 0) {
        if (warp == 1) {
            sh[18] = exp(sh[12] * h) - 1.0;
            sh[19] = expm1_over(sh[12] * h, h);
        } else if (warp == 2) {
            sh[20] = exp(-sh[13] * h);
        } else {
            sh[21] = expm1_over(-sh[13] * h, h);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        NptCoef c;
        c.g = sh[9];
        c.og = sh[10];
        c.sog = sh[11];
        for (int t = 0; t < 3; ++t) {
            c.a1[t] = sh[14];
            c.b1[t] = sh[15];
            c.a2m1[t] = sh[16];
            c.b2[t] = sh[17];
            c.a3m1[t] = sh[18];
            c.b3[t] = sh[19];
            c.a4[t] = sh[20];
            c.b4[t] = sh[21];
            c.L[t] = sh[3 + t];
            c.invL[t] = cc->invL[t];
        }
        c.half_cap = 0.5 * prm.max_disp;
        c.V = sh[6];
        c.noise = prm.noise;
        c.pad = 0;
        *cf = c;
        cell[0] = sh[3];
        cell[1] = sh[4];
        cell[2] = sh[5];
        cell[3] = sh[2];
        cell[10] = sh[6];
    }
}

// ---------------------------------------------------------------------------------
// Cell-variable part of the step for the rectangular cell (appendix: barostat 2, the edges
// l_j with momenta pc_j; barostat 3, the area A = l_x l_y and the height L), the splitting of
// k_npt_cell_a with one strain rate per axis.  The chain of cell slot j (V^p/2, V/2, O^p,
// V/2 with the strain rates between) runs on warp j (slots 0 and 2 when semi-isotropic); the
// twelve exponentials of each stage (four per axis) run on warps 4..15, one each, since a
// single FP64 chain is slow on this GPU and parallel ones are not.
constexpr int kRectWarps = 16;
constexpr int kCellPc = 12;   // cell momenta of the rectangular cell
constexpr int kCellWd = 16;   // virial diagonal
constexpr int kCellK2d = 19;  // sum p_j^2/m /100 per axis
constexpr int kCellPd = 22;   // diagonal pressure

// strain rate of slot j for cell momentum pc and edge l (semi-isotropic slot 0: A = l l)
__device__ __forceinline__ double rect_eps(bool aniso, int j, double pc, double M, double l)
{
    return (aniso || j == 2) ? pc / (M * l) : pc / (2.0 * M * (l * l));
}

// V/2 of slot j: the edge (or the area, whose square root is the new edge) moves by h pc / M
__device__ __forceinline__ double rect_move(bool aniso, int j, double pc, double M, double l, double h)
{
    return (aniso || j == 2) ? l + h * pc / M : sqrt(l * l + h * pc / M);
}

__global__ void __launch_bounds__(kRectWarps * 32)
k_npt_cell_rect(double* __restrict__ cell, NptCoef* __restrict__ cf, rbe_npt_params prm, uint64_t seed, int cellcap,
                CellConsts* __restrict__ cc)
{
    // shared: slot j at 8 j + {0 pc, 1 eps1, 2 eps2, 3 l', 4 eps3, 5 eps4, 6 l''}; 24..27 cell
    // normals; 28 friction factor of O^p; 29..31 O coefficients; 32..55 the per-axis
    // coefficients a1, b1, a2m1, b2, a3m1, b3, a4, b4 (3 each); 56..58 the new box
    __shared__ double sh[64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t step = cell_step(cell);
    const double h = 0.5 * prm.dt;
    const bool aniso = prm.barostat == 2;
    if (lane == 0) {
        if (warp < 3) {
            const int j = warp;
            if (aniso || j != 1) {
                // V^p/2 with the pressure of the current state, eps for R^p/2, V/2, eps for R/2
                const double L0 = cell[0], L1 = cell[1], L2 = cell[2];
                const double l = cell[j], M = prm.M_cell[j];
                double pc = cell[kCellPc + j];
                if (aniso) {
                    const double V = L0 * L1 * L2;
                    pc += h * ((cell[kCellK2d + j] + cell[kCellWd + j] - prm.P_ext * V) / l);
                } else if (j == 0) {
                    const double A = L0 * L1;
                    pc += h * ((cell[kCellK2d] + cell[kCellWd] + cell[kCellK2d + 1] + cell[kCellWd + 1]) / (2.0 * A) -
                               prm.P_ext * L2 + prm.gamma0);
                } else {
                    const double A = L0 * L1;
                    pc += h * ((cell[kCellK2d + 2] + cell[kCellWd + 2]) / L2 - prm.P_ext * A);
                }
                const double ln = rect_move(aniso, j, pc, M, l, h);
                sh[8 * j] = pc;
                sh[8 * j + 1] = rect_eps(aniso, j, pc, M, l);
                sh[8 * j + 2] = rect_eps(aniso, j, pc, M, ln);
                sh[8 * j + 3] = ln;
            }
        } else if (warp == 3) {
            const double g = exp(-prm.gamma * prm.dt);
            const double og = prm.kT * kFConv * (1.0 - g * g);
            sh[29] = g;
            sh[30] = og;
            sh[31] = sqrt(og);
        } else if (warp == 4) {
            double z[4] = {0.0, 0.0, 0.0, 0.0};
            if (prm.noise) npt_normals(seed, 2u, step, 0u, z);
            for (int t = 0; t < 4; ++t) sh[24 + t] = z[t];
        } else if (warp == 5) {
            sh[28] = exp(-prm.gamma_V * prm.dt);
        }
    }
    __syncthreads();
    if (lane == 0) {
        if (warp < 3) {
            const int j = warp;
            if (aniso || j != 1) {
                // O^p (slot j takes the cell normal z[j]), eps for R/2, V/2, eps for R^p/2
                const double M = prm.M_cell[j], gV = sh[28];
                double pc = sh[8 * j] * gV;
                if (prm.noise) pc += sqrt(prm.kT * M * (1.0 - gV * gV)) * sh[24 + j];
                const double l = sh[8 * j + 3];
                const double ln = rect_move(aniso, j, pc, M, l, h);
                sh[8 * j] = pc;
                sh[8 * j + 4] = rect_eps(aniso, j, pc, M, l);
                sh[8 * j + 5] = rect_eps(aniso, j, pc, M, ln);
                sh[8 * j + 6] = ln;
            }
        } else if (warp >= 4) {
            const int a = (warp - 4) >> 2, k = (warp - 4) & 3;
            const int sl = (aniso || a != 1) ? a : 0;  // semi-isotropic: y moves with x
            const double e1 = sh[8 * sl + 1], e2 = sh[8 * sl + 2];
            if (k == 0) sh[32 + a] = exp(-e1 * h);
            else if (k == 1) sh[35 + a] = expm1_over(-e1 * h, h);
            else if (k == 2) sh[38 + a] = exp(e2 * h) - 1.0;
            else sh[41 + a] = expm1_over(e2 * h, h);
        }
    }
    __syncthreads();
    if (warp == 0) {
        if (lane == 0) {
            sh[56] = sh[6];
            sh[57] = aniso ? sh[14] : sh[6];
            sh[58] = sh[22];
        }
        __syncwarp();
        write_cell_consts(lane, sh + 56, prm.rc, prm.rc + (prm.skin > 0.0 ? prm.skin : 0.0), cellcap, cc);
    } else if (lane == 0 && warp >= 4) {
        const int a = (warp - 4) >> 2, k = (warp - 4) & 3;
        const int sl = (aniso || a != 1) ? a : 0;
        const double e3 = sh[8 * sl + 4], e4 = sh[8 * sl + 5];
        if (k == 0) sh[44 + a] = exp(e3 * h) - 1.0;
        else if (k == 1) sh[47 + a] = expm1_over(e3 * h, h);
        else if (k == 2) sh[50 + a] = exp(-e4 * h);
        else sh[53 + a] = expm1_over(-e4 * h, h);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        NptCoef c;
        c.g = sh[29];
        c.og = sh[30];
        c.sog = sh[31];
        for (int t = 0; t < 3; ++t) {
            c.a1[t] = sh[32 + t];
            c.b1[t] = sh[35 + t];
            c.a2m1[t] = sh[38 + t];
            c.b2[t] = sh[41 + t];
            c.a3m1[t] = sh[44 + t];
            c.b3[t] = sh[47 + t];
            c.a4[t] = sh[50 + t];
            c.b4[t] = sh[53 + t];
            c.L[t] = sh[56 + t];
            c.invL[t] = cc->invL[t];
        }
        c.half_cap = 0.5 * prm.max_disp;
        c.V = sh[56] * sh[57] * sh[58];
        c.noise = prm.noise;
        c.pad = 0;
        *cf = c;
        for (int t = 0; t < 3; ++t) cell[t] = sh[56 + t];
        cell[3] = 0.0;
        cell[kCellPc] = sh[0];
        cell[kCellPc + 1] = aniso ? sh[8] : 0.0;
        cell[kCellPc + 2] = sh[16];
        cell[10] = c.V;
    }
}

// r += r (a - 1) + d with |d| capped at cap (cap > 0): the cap holds the peculiar part d =
// (p/m) b of an R/2 sub-step, not the affine part r (a - 1), which is the cell's dilation
// and scales with |r|.  The square root only for a step that is capped.
__device__ __forceinline__ void drift_add(double r[3], const double am1[3], double d[3], double cap)
{
    if (cap > 0.0) {
        const double l2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (l2 > cap * cap) {
            const double s = cap / sqrt(l2);
            d[0] *= s; d[1] *= s; d[2] *= s;
        }
    }
    r[0] += r[0] * am1[0] + d[0];
    r[1] += r[1] * am1[1] + d[1];
    r[2] += r[2] * am1[2] + d[2];
}


// Particle part before the forces: R^p/2, R/2, O, R/2, wrap into the new box.  kF32Noise:
// the Langevin normals in FP32 (FP32-phase path); the state stays FP64 either way.  kRect:
// per-axis coefficients (rectangular cell); otherwise those of axis 0 serve every axis, which
// keeps the isotropic kernel's registers (and occupancy) as low as a scalar strain rate needs.
template <bool kF32Noise, bool kRect>
__global__ void __launch_bounds__(kNptThreads)
k_npt_drift(int64_t N, double* __restrict__ pos, double* __restrict__ mom, const double* __restrict__ force,
            const double2* __restrict__ mprop, const NptCoef* __restrict__ cfp, uint64_t seed,
            const double* __restrict__ cell)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint64_t step = cell_step(cell);
    const NptCoef& c = *cfp;
    const double2 mp = mprop[i];  // (1/m, sqrt(m))
    const double inv_m = mp.x;
    double r[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    double p[3] = {mom[3 * i], mom[3 * i + 1], mom[3 * i + 2]};
    for (int t = 0; t < 3; ++t) {
        const int x = kRect ? t : 0;
        p[t] = p[t] * c.a1[x] + kFConv * force[3 * i + t] * c.b1[x];
    }
    double d[3], am1[3];
    for (int t = 0; t < 3; ++t) {
        const int x = kRect ? t : 0;
        am1[t] = c.a2m1[x];
        d[t] = (p[t] * inv_m) * c.b2[x];
    }
    drift_add(r, am1, d, c.half_cap);
    double z[4] = {0.0, 0.0, 0.0, 0.0};
    if (c.noise) {
        if (kF32Noise) npt_normals_f32(seed, 1u, step, (uint32_t)i, z);
        else npt_normals(seed, 1u, step, (uint32_t)i, z);
    }
    const double s = c.sog * mp.y;
    for (int t = 0; t < 3; ++t) p[t] = p[t] * c.g + s * z[t];
    for (int t = 0; t < 3; ++t) {
        const int x = kRect ? t : 0;
        am1[t] = c.a3m1[x];
        d[t] = (p[t] * inv_m) * c.b3[x];
    }
    drift_add(r, am1, d, c.half_cap);
    for (int t = 0; t < 3; ++t) {
        r[t] -= c.L[t] * floor(r[t] * c.invL[t]);
        pos[3 * i + t] = r[t];
        mom[3 * i + t] = p[t];
    }
}

// ---------------------------------------------------------------------------------
// Cell list.  Cells per axis nc = floor(l / rc) (>= 3, checked by the host with headroom and
// here), cell of a wrapped position s = r / l: floor(s nc).
// Cell of a position: s = r / l (as r times 1/l), wrapped into [0, 1), times nc, clamped.
__device__ __forceinline__ int cell_of(const double r[3], const double* inv_l, const int nc[3])
{
    int c[3];
    for (int t = 0; t < 3; ++t) {
        const double s = r[t] * inv_l[t];
        c[t] = min(nc[t] - 1, max(0, (int)floor((s - floor(s)) * nc[t])));
    }
    return (c[2] * nc[1] + c[1]) * nc[0] + c[0];
}

__global__ void __launch_bounds__(kNptThreads)
k_cl_count(int64_t N, const double* __restrict__ pos, const CellConsts* __restrict__ cc, int* __restrict__ cid,
           int* __restrict__ cnt, unsigned* __restrict__ status, const NListState* __restrict__ nls)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (i == 0 && !cc->ok) atomicOr(status, kStatusBox);
    if (nls && !nls->rebuild) return;  // the neighbour list stands: no cell list this step
    // (a box that outgrew the cell arrays, or broke rc <= l/2, was reported above)
    if (cc->ncell < 0) {
        cid[i] = 0;
        return;
    }
    const int nc[3] = {cc->nc[0], cc->nc[1], cc->nc[2]};
    const double inv[3] = {cc->invL[0], cc->invL[1], cc->invL[2]};
    const double r[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    const int c = cell_of(r, inv, nc);
    cid[i] = c;
    atomicAdd(&cnt[c], 1);
}

// Exclusive scan of the counts (one block); cursor = start.
__global__ void __launch_bounds__(kScanThreads)
k_cl_scan(const CellConsts* __restrict__ cc, const int* __restrict__ cnt, int* __restrict__ start,
          int* __restrict__ cursor, const NListState* __restrict__ nls)
{
    __shared__ int wsum[kScanThreads / 32];
    if (nls && !nls->rebuild) return;
    // a box beyond the cell arrays put every particle in cell 0 with a count of 0: start and
    // cursor of cell 0 are still written (0), so the fill stays in bounds
    const int n = cc->ncell < 0 ? 1 : cc->ncell;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int j0 = min(n, tid * per), j1 = min(n, j0 + per);
    int local = 0;
    for (int j = j0; j < j1; ++j) local += cnt[j];
    int incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = wsum[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += o;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int run = incl - local + (warp > 0 ? wsum[warp - 1] : 0);
    for (int j = j0; j < j1; ++j) {
        start[j] = run;
        cursor[j] = run;
        run += cnt[j];
    }
}

__global__ void k_cl_fill(int64_t N, const int* __restrict__ cid, int* __restrict__ cursor, int* __restrict__ fill,
                          const NListState* __restrict__ nls)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (nls && !nls->rebuild) return;
    const int slot = atomicAdd(&cursor[cid[i]], 1);
    fill[slot] = (int)i;
}

// Per cell, one warp: order the members by particle index (a fixed order for every run,
// whatever order the fill's atomics gave): the member with index i goes to rank = number of
// members with a smaller index.  Then pack positions and charges in that order: FP32 xyzq
// always (the pair search runs on it), FP64 as well when spos64 is given.
__global__ void __launch_bounds__(kSortWarps * 32)
k_cl_sort(const CellConsts* __restrict__ cc, const int* __restrict__ cnt, const int* __restrict__ start,
          const int* __restrict__ fill, int* __restrict__ sorted, const double* __restrict__ pos,
          const double* __restrict__ q, float4* __restrict__ spos32, double4_32a* __restrict__ spos64,
          const NListState* __restrict__ nls)
{
    if (nls && !nls->rebuild) return;
    const int64_t ncell = cc->ncell;  // -1: nothing to sort
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= ncell) return;  // c is the same for the whole warp
    const int s0 = start[c], k = cnt[c];
    for (int a0 = 0; a0 < k; a0 += 32) {
        const int a = a0 + lane;
        const int ia = a < k ? fill[s0 + a] : INT_MAX;
        int rank = 0;
        for (int b0 = 0; b0 < k; b0 += 32) {
            const int b = b0 + lane;
            const int ib = b < k ? fill[s0 + b] : INT_MAX;
#pragma unroll 8
            for (int t = 0; t < 32; ++t) rank += __shfl_sync(0xffffffffu, ib, t) < ia ? 1 : 0;
        }
        if (a < k) {
            const double x = pos[3 * (int64_t)ia], y = pos[3 * (int64_t)ia + 1], z = pos[3 * (int64_t)ia + 2];
            const double qq = q[ia];
            sorted[s0 + rank] = ia;
            spos32[s0 + rank] = make_float4((float)x, (float)y, (float)z, (float)qq);
            if (spos64) {
                double4_32a v;
                v.x = x;
                v.y = y;
                v.z = z;
                v.w = qq;
                spos64[s0 + rank] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// Real-space forces (Sec. 4.1 Eqs. (U2), (force)) on the cell list: one warp per particle
// i, taken in cell order (slot u of the sorted array), so that neighbouring warps search
// the same cells.  For each of the 3 x 3 rows (dy, dz) of neighbour cells the cells
// cx-1..cx+1 are contiguous slots (split in two where the row wraps); the lanes stride over
// them.  With 3 or more cells on an axis the periodic image of a neighbour cell is fixed
// (shift -l, 0 or +l where the row or column wraps); with fewer, each pair takes the nearest
// image.  Every distinct cell is visited once, and rc <= l/2 makes the image within rc the
// nearest one.
//   Search: FP32 positions; a candidate within the cutoff (FP64 path: within rc plus a
//   margin above the FP32 rounding of the distance) is appended to the warp's buffer in
//   shared memory (ballot order, so the order is fixed).
//   Evaluation: every 32 buffered candidates, one per lane; the FP64 path recomputes the
//   distance from the FP64 positions and applies the exact cutoff.
//   f = -(dU/dr)/r for U = qqr2e q_i q_j erfc(sqrt(a) r)/r + 4 eps ((s/r)^12 - (s/r)^6); the
//   lane sums go through a fixed shuffle tree, so the result does not depend on timing.  The
//   FP32 path evaluates erfc by a published Chebyshev fit (erfc_nr).
// Each pair is visited from both ends: energies and the virial take half.  The warps stride
// over the slots (grid-stride); per-block partials {W_r, E_coul, E_lj} at slots 1..3, or with
// kDiag (rectangular cells) {W_xx, W_yy, W_zz, E_coul, E_lj} at slots 3..7 (W_jj = sum f d_j^2).  A box that
// outgrew the cell arrays (flagged by k_cl_count) leaves F_r = 0.

// Modes of the pair kernel: search the cells and evaluate (no list), search the cells within
// the list radius and write the list (only on a rebuild step), evaluate the listed pairs.
enum PairMode { kPairCells = 0, kPairBuild = 1, kPairList = 2 };

// Neighbour-list arguments of the pair kernel (unused without a list).
struct ListArgs {
    NListState* nls;
    int* nbr;          // [slot * cap + k]
    int* nnb;          // per slot
    float4* sref;      // per slot: scaled position at the build
    unsigned* status;  // kStatusList on overflow
    int cap;
};

template <bool kF64, int kMode, bool kDiag = false>
__global__ void __launch_bounds__(kPairWarps * 32, kF64 ? kPairBlocksPerSM64 : kPairBlocksPerSM)
k_pair(int64_t N, const CellConsts* __restrict__ cc, const PairConst pc, const int* __restrict__ cid,
       const int* __restrict__ cnt,
       const int* __restrict__ start, const int* __restrict__ sorted, const float4* __restrict__ spos32,
       const double4_32a* __restrict__ spos64, double* __restrict__ Fr, double* __restrict__ partials,
       const ListArgs la)
{
    using R = typename std::conditional<kF64, double, float>::type;
    using Hit = typename std::conditional<kF64, int2, float4>::type;  // FP64: (slot, image code)
    constexpr bool kBuild = kMode == kPairBuild, kList = kMode == kPairList;
    if (kBuild && !la.nls->rebuild) return;  // the list stands (the same for every thread)
    __shared__ Hit hits[kPairWarps][kHitCap];
    __shared__ double red[kDiag ? 5 : 3][kPairWarps];
    __shared__ double sL[3], sInvL[3];
    __shared__ float sLf[3], sInvLf[3], sPass;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // box constants once per block (shared memory)
    if (threadIdx.x < 3) {
        sL[threadIdx.x] = cc->L[threadIdx.x];
        sInvL[threadIdx.x] = cc->invL[threadIdx.x];
        sLf[threadIdx.x] = cc->Lf[threadIdx.x];
        sInvLf[threadIdx.x] = cc->invLf[threadIdx.x];
    } else if (threadIdx.x == 32) {
        // FP64 path: the FP32 search keeps candidates within rc plus 2^-16 l_max, far above
        // the FP32 rounding of a distance, and the exact cutoff is applied in FP64.  A build
        // keeps every candidate within rl plus the same margin (a superset is harmless).
        if (kBuild) {
            const double lmax = fmax(cc->L[0], fmax(cc->L[1], cc->L[2]));
            const double rp = (double)la.nls->rl + lmax * 0x1.0p-16;
            sPass = (float)(rp * rp);
        } else {
            sPass = kF64 ? cc->pass64 : pc.rc2f;
        }
    }
    __syncthreads();
    const int nc[3] = {cc->nc[0], cc->nc[1], cc->nc[2]};
    // this warp's particles (lane 0): FP64 sums on the FP64 path; float-float sums on the FP32
    // path, where no per-particle FP64 instruction runs (each costs a whole warp issue slot on
    // GB300's narrow FP64 pipe)
    double wsum = 0.0, ecsum = 0.0, elsum = 0.0;
    float wh = 0.f, wl = 0.f, ech = 0.f, ecl = 0.f, elh = 0.f, ell = 0.f;
    // kDiag: w, wsum, (wh, wl) hold the x part of the virial; y and z here
    double wysum = 0.0, wzsum = 0.0;
    float wyh = 0.f, wyl = 0.f, wzh = 0.f, wzl = 0.f;
    // no cell list this step (box beyond the cell arrays, flagged), or no list built yet
    const bool cells_ok = kList ? la.nls->force == 0 : cc->ncell >= 0;
    if (!cells_ok) {
        if (!kBuild)
            for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < 3 * N;
                 j += (int64_t)gridDim.x * blockDim.x)
                Fr[j] = 0.0;
    } else {
        const double* L = sL;
        const double* invL = sInvL;
        const float* Lf = sLf;
        const float* invLf = sInvLf;
        // nearest image per pair on the axes with fewer than 3 cells, and on all axes for the
        // listed pairs (the list keeps slots, not images)
        const bool mi[3] = {kList || nc[0] < 3, kList || nc[1] < 3, kList || nc[2] < 3};
        const float rc2_pass = sPass;
        R rc2, sa, aR, two_sa_pi, qk, s2, e4, e24;
        if constexpr (kF64) {
            rc2 = pc.rc2, sa = pc.sa, aR = pc.a, two_sa_pi = pc.two_sa_pi;
            qk = pc.qk, s2 = pc.s2, e4 = pc.e4, e24 = pc.e24;
        } else {
            rc2 = pc.rc2f, sa = pc.saf, aR = pc.af, two_sa_pi = pc.two_sa_pif;
            qk = pc.qkf, s2 = pc.s2f, e4 = pc.e4f, e24 = pc.e24f;
        }
        const bool lj = pc.lj != 0;
        const int nwarps = gridDim.x * kPairWarps;
        for (int u = blockIdx.x * kPairWarps + wib; u < (int)N; u += nwarps) {
            const int i = sorted[u];
            const float4 me = spos32[u];
            R xi, yi, zi, qi;
            if constexpr (kF64) {
                const double4_32a m64 = spos64[u];
                xi = m64.x;
                yi = m64.y;
                zi = m64.z;
                qi = m64.w;
            } else {
                xi = me.x;
                yi = me.y;
                zi = me.z;
                qi = me.w;
            }
            // Segments, one per lane (lanes 0..17): row r = lane / 2 of the 3 x 3 rows (dy, dz),
            // part lane % 2 (a row that wraps in x has two parts).  Each lane finds its slot
            // range [lo, hi), its image (sx, sy, sz) and the search centre me - shift.
            int lo = 0, hi = 0, code = 0;
            float ctx = 0.f, cty = 0.f, ctz = 0.f;
            if (!kList) {
                const int c = cid[i];
                const int cxy = nc[0] * nc[1];
                const int cz = c / cxy, cy = (c - cz * cxy) / nc[0], cx = c - cz * cxy - cy * nc[0];
                const int r = lane >> 1, part = lane & 1;
                const int dy = r % 3 - 1, dz = r / 3 - 1;
                const bool row_ok = r < 9 && (dy >= (nc[1] >= 3 ? -1 : 0)) && (dy <= (nc[1] >= 2 ? 1 : 0)) &&
                                    (dz >= (nc[2] >= 3 ? -1 : 0)) && (dz <= (nc[2] >= 2 ? 1 : 0));
                if (row_ok) {
                    const int uy = cy + dy, uz = cz + dz;
                    const int yy = uy < 0 ? uy + nc[1] : (uy >= nc[1] ? uy - nc[1] : uy);
                    const int zz = uz < 0 ? uz + nc[2] : (uz >= nc[2] ? uz - nc[2] : uz);
                    const int sy = mi[1] ? 0 : (uy < 0 ? -1 : (uy >= nc[1] ? 1 : 0));
                    const int sz = mi[2] ? 0 : (uz < 0 ? -1 : (uz >= nc[2] ? 1 : 0));
                    const int row = (zz * nc[1] + yy) * nc[0], nx = nc[0];
                    int a = -1, e = -1, sx = 0;  // cells a..e of the row, image sx
                    if (mi[0]) {
                        if (part == 0) a = 0, e = nx - 1;
                    } else if (cx == 0) {
                        if (part == 0) a = 0, e = 1;
                        else a = e = nx - 1, sx = -1;
                    } else if (cx == nx - 1) {
                        if (part == 0) a = nx - 2, e = nx - 1;
                        else a = e = 0, sx = 1;
                    } else if (part == 0) {
                        a = cx - 1, e = cx + 1;
                    }
                    if (a >= 0) {
                        lo = start[row + a];
                        hi = start[row + e] + cnt[row + e];
                        code = (sx + 1) | ((sy + 1) << 2) | ((sz + 1) << 4);
                        ctx = me.x - (float)sx * Lf[0];
                        cty = me.y - (float)sy * Lf[1];
                        ctz = me.z - (float)sz * Lf[2];
                    }
                }
            }
            R fx = 0, fy = 0, fz = 0, w = 0, ec = 0, el = 0;
            R wy = 0, wz = 0;
            int nh = 0;
            // one buffered candidate per lane (lanes >= count idle)
            auto evaluate = [&](int count, int base = 0) {
                if (lane >= count) return;
                const Hit h = hits[wib][base + lane];
                R dx, dy, dz, qj;
                if constexpr (kF64) {
                    const double4_32a o = spos64[h.x];
                    const int cd = h.y;
                    dx = (o.x - xi) + (double)((cd & 3) - 1) * L[0];
                    dy = (o.y - yi) + (double)(((cd >> 2) & 3) - 1) * L[1];
                    dz = (o.z - zi) + (double)(((cd >> 4) & 3) - 1) * L[2];
                    if (mi[0]) dx -= L[0] * rint(dx * invL[0]);
                    if (mi[1]) dy -= L[1] * rint(dy * invL[1]);
                    if (mi[2]) dz -= L[2] * rint(dz * invL[2]);
                    qj = o.w;
                } else {
                    dx = h.x;
                    dy = h.y;
                    dz = h.z;
                    qj = h.w;
                }
                const R r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < rc2)) return;
                R inv_r, r, ex;
                if constexpr (kF64) {
                    r = sqrt(r2);
                    inv_r = 1.0 / r;
                    ex = exp(-aR * r2);
                } else {
                    inv_r = rsqrtf(r2);
                    r = r2 * inv_r;
                    ex = __expf(-aR * r2);
                }
                const R inv_r2 = inv_r * inv_r;
                const R coul = qk * qi * qj * inv_r;  // qqr2e q_i q_j / r
                R er;
                if constexpr (kF64) er = erfc(sa * r);
                else er = erfc_nr(sa * r);
                ec += coul * er;
                R f = coul * (er + two_sa_pi * r * ex) * inv_r2;
                if (lj) {
                    const R sr2 = s2 * inv_r2;
                    const R sr6 = sr2 * sr2 * sr2;
                    el += e4 * (sr6 * sr6 - sr6);
                    f += e24 * (2 * sr6 * sr6 - sr6) * inv_r2;
                }
                // force on i is -f d (d points from i to the neighbour)
                fx -= f * dx;
                fy -= f * dy;
                fz -= f * dz;
                if constexpr (kDiag) {
                    w += f * dx * dx;
                    wy += f * dy * dy;
                    wz += f * dz * dz;
                } else {
                    w += f * r2;
                }
            };
            // the search over one segment; MI: some axis has fewer than 3 cells (nearest image
            // per candidate there).  The loop body has no divergent branch: out-of-range lanes
            // load an in-range slot and are masked out of the hit.
            auto search = [&](auto mi_tag, int glo, int ghi, int gcode, float gx, float gy, float gz) {
                constexpr bool MI = decltype(mi_tag)::value;
                for (int s0 = glo; s0 < ghi; s0 += 32) {
                    const int s = s0 + lane;
                    const bool valid = s < ghi && s != u;
                    const float4 o = spos32[s < ghi ? s : glo];
                    float dx = o.x - gx, dy = o.y - gy, dz = o.z - gz;
                    if constexpr (MI) {
                        if (mi[0]) dx -= Lf[0] * rintf(dx * invLf[0]);
                        if (mi[1]) dy -= Lf[1] * rintf(dy * invLf[1]);
                        if (mi[2]) dz -= Lf[2] * rintf(dz * invLf[2]);
                    }
                    const bool hit = valid && dx * dx + dy * dy + dz * dz < rc2_pass;
                    const unsigned m = __ballot_sync(0xffffffffu, hit);
                    if constexpr (kBuild) {
                        if (hit) {
                            const int p = nh + __popc(m & ((1u << lane) - 1u));
                            if (p < la.cap) la.nbr[(int64_t)u * la.cap + p] = s;
                        }
                        nh += __popc(m);
                        continue;
                    }
                    if (hit) {
                        const int p = nh + __popc(m & ((1u << lane) - 1u));
                        if constexpr (kF64) hits[wib][p] = make_int2(s, gcode);
                        else hits[wib][p] = make_float4(dx, dy, dz, o.w);
                    }
                    nh += __popc(m);
                    if (nh >= 32) {
                        __syncwarp();
                        evaluate(32);
                        __syncwarp();
                        if (lane < nh - 32) hits[wib][lane] = hits[wib][32 + lane];
                        __syncwarp();
                        nh -= 32;
                    }
                }
            };
            if constexpr (kList) {
                // the listed slots, kListBatch x 32 at a time: all their list entries are loaded,
                // then all their positions, so that the loads overlap; nearest image by compare
                // and select (positions lie in [0, l)); then the same compaction and evaluation
                const int nn = la.nnb[u];
                const int* row = la.nbr + (int64_t)u * la.cap;
                const float hx = 0.5f * Lf[0], hy = 0.5f * Lf[1], hz = 0.5f * Lf[2];
                for (int k0 = 0; k0 < nn; k0 += 32 * kListBatch) {
                    int sj[kListBatch];
                    float4 o[kListBatch];
#pragma unroll
                    for (int a = 0; a < kListBatch; ++a) {
                        const int k = k0 + 32 * a + lane;
                        sj[a] = row[k < nn ? k : nn - 1];
                    }
#pragma unroll
                    for (int a = 0; a < kListBatch; ++a) o[a] = spos32[sj[a]];
#pragma unroll
                    for (int a = 0; a < kListBatch; ++a) {
                        const int k = k0 + 32 * a + lane;
                        float dx = o[a].x - me.x, dy = o[a].y - me.y, dz = o[a].z - me.z;
                        dx = dx > hx ? dx - Lf[0] : (dx < -hx ? dx + Lf[0] : dx);
                        dy = dy > hy ? dy - Lf[1] : (dy < -hy ? dy + Lf[1] : dy);
                        dz = dz > hz ? dz - Lf[2] : (dz < -hz ? dz + Lf[2] : dz);
                        const bool hit = k < nn && dx * dx + dy * dy + dz * dz < rc2_pass;
                        const unsigned m = __ballot_sync(0xffffffffu, hit);
                        if (hit) {
                            const int p = nh + __popc(m & ((1u << lane) - 1u));
                            if constexpr (kF64) hits[wib][p] = make_int2(sj[a], 1 | (1 << 2) | (1 << 4));  // no shift
                            else hits[wib][p] = make_float4(dx, dy, dz, o[a].w);
                        }
                        nh += __popc(m);
                    }
                    // evaluate whole groups of 32 and keep the rest at the front
                    __syncwarp();
                    int b0 = 0;
                    for (; b0 + 32 <= nh; b0 += 32) evaluate(32, b0);
                    __syncwarp();
                    if (b0 > 0 && lane < nh - b0) hits[wib][lane] = hits[wib][b0 + lane];
                    __syncwarp();
                    nh -= b0;
                }
            } else {
                const bool any_mi = mi[0] || mi[1] || mi[2];
                for (int g = 0; g < 18; ++g) {
                    const int glo = __shfl_sync(0xffffffffu, lo, g), ghi = __shfl_sync(0xffffffffu, hi, g);
                    if (glo >= ghi) continue;  // the same for every lane
                    const int gcode = __shfl_sync(0xffffffffu, code, g);
                    const float gx = __shfl_sync(0xffffffffu, ctx, g), gy = __shfl_sync(0xffffffffu, cty, g),
                                gz = __shfl_sync(0xffffffffu, ctz, g);
                    if (any_mi) search(std::true_type{}, glo, ghi, gcode, gx, gy, gz);
                    else search(std::false_type{}, glo, ghi, gcode, gx, gy, gz);
                }
            }
            if constexpr (kBuild) {
                if (lane == 0) {
                    la.nnb[u] = nh < la.cap ? nh : la.cap;
                    la.sref[u] = make_float4(me.x * invLf[0], me.y * invLf[1], me.z * invLf[2], 0.f);
                    if (nh > la.cap) atomicOr(la.status, kStatusList);
                }
                continue;
            }
            __syncwarp();
            evaluate(nh);
            __syncwarp();
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                fx += __shfl_xor_sync(0xffffffffu, fx, off);
                fy += __shfl_xor_sync(0xffffffffu, fy, off);
                fz += __shfl_xor_sync(0xffffffffu, fz, off);
                w += __shfl_xor_sync(0xffffffffu, w, off);
                if constexpr (kDiag) {
                    wy += __shfl_xor_sync(0xffffffffu, wy, off);
                    wz += __shfl_xor_sync(0xffffffffu, wz, off);
                }
                ec += __shfl_xor_sync(0xffffffffu, ec, off);
                el += __shfl_xor_sync(0xffffffffu, el, off);
            }
            if (lane == 0) {
                if constexpr (kF64) {
                    Fr[3 * (int64_t)i] = fx;
                    Fr[3 * (int64_t)i + 1] = fy;
                    Fr[3 * (int64_t)i + 2] = fz;
                    wsum += 0.5 * w;
                    if constexpr (kDiag) {
                        wysum += 0.5 * wy;
                        wzsum += 0.5 * wz;
                    }
                    ecsum += 0.5 * ec;
                    elsum += 0.5 * el;
                } else {
                    // exact widening by integer operations
                    unsigned long long* Fb = reinterpret_cast<unsigned long long*>(Fr);
                    Fb[3 * (int64_t)i] = float_to_double_bits(__float_as_uint(fx));
                    Fb[3 * (int64_t)i + 1] = float_to_double_bits(__float_as_uint(fy));
                    Fb[3 * (int64_t)i + 2] = float_to_double_bits(__float_as_uint(fz));
                    ff_add(wh, wl, 0.5f * w);
                    if constexpr (kDiag) {
                        ff_add(wyh, wyl, 0.5f * wy);
                        ff_add(wzh, wzl, 0.5f * wz);
                    }
                    ff_add(ech, ecl, 0.5f * ec);
                    ff_add(elh, ell, 0.5f * el);
                }
            }
        }
    }
    if constexpr (kBuild) {
        // the build's box; the list now stands until the next check says otherwise (a build
        // without a cell list leaves the list pending)
        if (cells_ok && blockIdx.x == 0 && threadIdx.x == 0) {
            for (int t = 0; t < 3; ++t) la.nls->Lref[t] = cc->L[t];
            la.nls->force = 0;
        }
        return;
    }
    // fixed-order block sums
    if (lane == 0) {
        if (!kF64) {
            wsum = (double)wh + (double)wl;
            ecsum = (double)ech + (double)ecl;
            elsum = (double)elh + (double)ell;
            if (kDiag) {
                wysum = (double)wyh + (double)wyl;
                wzsum = (double)wzh + (double)wzl;
            }
        }
        constexpr int o = kDiag ? 2 : 0;
        red[0][wib] = wsum;
        if (kDiag) {
            red[1][wib] = wysum;
            red[2][wib] = wzsum;
        }
        red[o + 1][wib] = ecsum;
        red[o + 2][wib] = elsum;
    }
    __syncthreads();
    constexpr int nsum = kDiag ? 5 : 3;
    if (threadIdx.x < nsum) {
        double t = 0.0;
        for (int wv = 0; wv < kPairWarps; ++wv) t += red[threadIdx.x][wv];
        partials[kPartStride * (size_t)blockIdx.x + (kDiag ? 3 : 1) + threadIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------------
// Forces F = qqr2e F_k + F_r; with do_kick, R^p/2 with (a4, b4); the kinetic sum per block
// (2K, or per axis for the rectangular cell); the last block sums the partials in a fixed
// order and finishes the pressure.  Isotropic: W = qqr2e tr(W_k) + W_r, P_ins = (2K + W)/(3V),
// with do_kick V^p/2.  Rectangular cell: W_jj = qqr2e (W_k)_jj + (W_r)_jj, (P_ins)_jj =
// (2K_j + W_jj)/V, with do_kick V^p/2 of the cell momenta (the forces of k_npt_cell_rect).
template <bool kDiag>
__global__ void __launch_bounds__(kNptThreads)
k_npt_finish(int64_t N, double* __restrict__ mom, double* __restrict__ force, const double2* __restrict__ mprop,
             const double* __restrict__ Fk, const double* __restrict__ Fr, const double* __restrict__ WEk,
             const NptCoef* __restrict__ cfp, double* __restrict__ partials, int nblocks_pair,
             unsigned* __restrict__ counter, double* __restrict__ cell, rbe_npt_params prm, int do_kick,
             unsigned* __restrict__ status)
{
    __shared__ double red[3][kNptThreads / 32];
    __shared__ bool is_last;
    constexpr bool diag = kDiag;  // rectangular cell
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double k2 = 0.0, k2d[3] = {0.0, 0.0, 0.0};
    if (i < N) {
        const double inv_m = mprop[i].x;
        for (int t = 0; t < 3; ++t) {
            const double F = (prm.kspace ? prm.qqr2e * Fk[3 * i + t] : 0.0) + (prm.real ? Fr[3 * i + t] : 0.0);
            force[3 * i + t] = F;
            double p = mom[3 * i + t];
            if (do_kick) {
                p = p * cfp->a4[diag ? t : 0] + kFConv * F * cfp->b4[diag ? t : 0];
                mom[3 * i + t] = p;
            }
            if constexpr (diag) k2d[t] = p * p * inv_m * (1.0 / kFConv);
            else k2 += p * p * inv_m;
        }
        k2 *= 1.0 / kFConv;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nf = diag ? 3 : 1;  // kinetic partials per block
    if constexpr (diag) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            for (int t = 0; t < 3; ++t) k2d[t] += __shfl_xor_sync(0xffffffffu, k2d[t], off);
        if (lane == 0)
            for (int t = 0; t < 3; ++t) red[t][warp] = k2d[t];
    } else {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) k2 += __shfl_xor_sync(0xffffffffu, k2, off);
        if (lane == 0) red[0][warp] = k2;
    }
    __syncthreads();
    if (threadIdx.x < nf) {
        double sum = 0.0;
        for (int wv = 0; wv < kNptThreads / 32; ++wv) sum += red[threadIdx.x][wv];
        partials[kPartStride * (size_t)(nblocks_pair + blockIdx.x) + threadIdx.x] = sum;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // the last block: thread t sums the partials t, t + 256, ... and a fixed shared-memory
    // tree combines the threads, so the sums do not depend on which block came last
    __shared__ double fin[diag ? 8 : 4][kNptThreads];
    constexpr int na = diag ? 8 : 4;  // slots [0, nf) kinetic, [nf, na) pair
    {
        double v[na];
#pragma unroll
        for (int a = 0; a < na; ++a) v[a] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += kNptThreads)
#pragma unroll
            for (int a = 0; a < nf; ++a) v[a] += __ldcg(partials + kPartStride * (size_t)(nblocks_pair + b) + a);
        if (prm.real)
            for (int b = threadIdx.x; b < nblocks_pair; b += kNptThreads)
#pragma unroll
                for (int a = nf; a < na; ++a) v[a] += __ldcg(partials + kPartStride * (size_t)b + a);
#pragma unroll
        for (int a = 0; a < na; ++a) fin[a][threadIdx.x] = v[a];
    }
    __syncthreads();
    for (int half = kNptThreads / 2; half > 0; half >>= 1) {
        if (threadIdx.x < half)
#pragma unroll
            for (int a = 0; a < na; ++a) fin[a][threadIdx.x] += fin[a][threadIdx.x + half];
        __syncthreads();
    }
    if constexpr (!diag) {
        if (threadIdx.x != 0) return;
        const double K2 = fin[0][0], Wr = fin[1][0], Ec = fin[2][0], El = fin[3][0];
        double Wk = 0.0, Ek = 0.0;
        if (prm.kspace) {
            Wk = prm.qqr2e * (__ldcg(WEk + 0) + __ldcg(WEk + 4) + __ldcg(WEk + 8));
            Ek = prm.qqr2e * (__ldcg(WEk + 9) + __ldcg(WEk + 10));
        }
        const double W = Wk + Wr;
        const double V = cell[0] * cell[1] * cell[2];
        const double Pins = (K2 + W) / (3.0 * V);
        double pV = prm.barostat ? cell[3] : 0.0;
        if (do_kick && prm.barostat) pV += 0.5 * prm.dt * (Pins - prm.P_ext);
        cell[3] = pV;
        cell[4] = W;
        cell[5] = K2;
        cell[6] = Pins;
        cell[7] = Ek;
        cell[8] = Ec;
        cell[9] = El;
        cell[10] = V;
        if (do_kick) cell[kCellStep] = __longlong_as_double((long long)(cell_step(cell) + 1));
        if (!isfinite(Pins) || !isfinite(pV)) atomicOr(status, kStatusNonFinite);
        *counter = 0u;
        return;
    }
    // rectangular cell: lane j of warp 0 takes axis j
    if (!diag || threadIdx.x >= 32) return;
    __shared__ double sK[3], sW[3];
    const int j = threadIdx.x;
    if (j < 3) {
        const double Wk = prm.kspace ? prm.qqr2e * __ldcg(WEk + 4 * j) : 0.0;
        sK[j] = fin[j][0];
        sW[j] = Wk + fin[3 + j][0];
    }
    __syncwarp();
    const double L0 = cell[0], L1 = cell[1], L2 = cell[2];
    const double V = L0 * L1 * L2;
    if (j < 3) {
        const double h = 0.5 * prm.dt;
        double pc = cell[kCellPc + j];
        if (do_kick) {
            if (prm.barostat == 2) {
                pc += h * ((sK[j] + sW[j] - prm.P_ext * V) / cell[j]);
            } else if (j == 0) {
                const double A = L0 * L1;
                pc += h * ((sK[0] + sW[0] + sK[1] + sW[1]) / (2.0 * A) - prm.P_ext * L2 + prm.gamma0);
            } else if (j == 2) {
                const double A = L0 * L1;
                pc += h * ((sK[2] + sW[2]) / L2 - prm.P_ext * A);
            }
        }
        const double Pd = (sK[j] + sW[j]) / V;
        cell[kCellPc + j] = pc;
        cell[kCellWd + j] = sW[j];
        cell[kCellK2d + j] = sK[j];
        cell[kCellPd + j] = Pd;
        if (!isfinite(pc) || !isfinite(Pd)) atomicOr(status, kStatusNonFinite);
    }
    if (j == 0) {
        const double K2 = sK[0] + sK[1] + sK[2], W = sW[0] + sW[1] + sW[2];
        const double Ek = prm.kspace ? prm.qqr2e * (__ldcg(WEk + 9) + __ldcg(WEk + 10)) : 0.0;
        cell[3] = 0.0;
        cell[4] = W;
        cell[5] = K2;
        cell[6] = (K2 + W) / (3.0 * V);
        cell[7] = Ek;
        cell[8] = fin[6][0];
        cell[9] = fin[7][0];
        cell[10] = V;
        if (do_kick) cell[kCellStep] = __longlong_as_double((long long)(cell_step(cell) + 1));
        *counter = 0u;
    }
}

// ---------------------------------------------------------------------------------
// Host side.

static rbe_status npt_fail(rbe_ctx ctx, cudaError_t e, const char* what) { return cuda_fail(ctx, e, what); }

static rbe_status npt_check(rbe_ctx ctx, const char* what)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RBE_OK : npt_fail(ctx, e, what);
}

// Blocks of the pair kernel: one warp per particle, at most one resident wave (the warps
// stride over the rest).  The FP32 count is the larger one and sizes the partials.
int pair_blocks(rbe_ctx ctx, int64_t N, bool fp64)
{
    const int64_t want = (N + kPairWarps - 1) / kPairWarps;
    const int per_sm = fp64 ? kPairBlocksPerSM64 : kPairBlocksPerSM;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ctx->num_sms * per_sm));
}

// Grow the NPT scratch for N particles and a box whose edges may double; with skin > 0 also
// the neighbour list (twice the expected neighbours at the initial density, plus 64).
rbe_status npt_ensure(rbe_ctx ctx, int64_t N, const double box[3], double rc, double skin)
{
    NptBuffers& b = ctx->npt;
    cudaError_t e;
    if (!b.WEk) {
        if ((e = ctx_alloc(ctx, &b.WEk, 16 * sizeof(double))) != cudaSuccess ||
            (e = ctx_alloc(ctx, &b.cellc, sizeof(CellConsts))) != cudaSuccess ||
            (e = ctx_alloc(ctx, &b.coef, sizeof(NptCoef))) != cudaSuccess ||
            (e = ctx_alloc(ctx, &b.counter, sizeof(unsigned))) != cudaSuccess ||
            (e = cudaMemsetAsync(b.counter, 0, sizeof(unsigned), ctx->stream)) != cudaSuccess)
            return npt_fail(ctx, e, "cudaMalloc(npt)");
    }
    if (N > b.ncap) {
        ctx_free(ctx, b.Fk); ctx_free(ctx, b.Fr); ctx_free(ctx, b.cid); ctx_free(ctx, b.fill); ctx_free(ctx, b.sorted);
        ctx_free(ctx, b.spos32); ctx_free(ctx, b.spos64); ctx_free(ctx, b.mprop);
        b.Fk = b.Fr = nullptr; b.cid = b.fill = b.sorted = nullptr; b.spos32 = nullptr; b.spos64 = nullptr; b.ncap = 0;
        b.mprop = nullptr;
        b.n64 = 0;
        if ((e = ctx_alloc(ctx, &b.Fk, 3 * sizeof(double) * N)) != cudaSuccess ||
            (e = ctx_alloc(ctx, &b.Fr, 3 * sizeof(double) * N)) != cudaSuccess ||
            (e = ctx_alloc(ctx, &b.cid, sizeof(int) * N)) != cudaSuccess ||
            (e = ctx_alloc(ctx, &b.fill, sizeof(int) * N)) != cudaSuccess ||
            (e = ctx_alloc(ctx, &b.sorted, sizeof(int) * N)) != cudaSuccess ||
            (e = ctx_alloc(ctx, &b.spos32, sizeof(float4) * N)) != cudaSuccess ||
            (e = ctx_alloc(ctx, &b.mprop, sizeof(double2) * N)) != cudaSuccess)
            return npt_fail(ctx, e, "cudaMalloc(npt particles)");
        b.ncap = N;
    }
    // FP64 packed positions only for the FP64 path
    if (ctx->precision == RBE_FP64 && N > b.n64) {
        ctx_free(ctx, b.spos64);
        b.spos64 = nullptr;
        b.n64 = 0;
        if ((e = ctx_alloc(ctx, &b.spos64, sizeof(double4_32a) * N)) != cudaSuccess)
            return npt_fail(ctx, e, "cudaMalloc(npt FP64 positions)");
        b.n64 = N;
    }
    int64_t cells = 1;
    for (int t = 0; t < 3; ++t) {
        const double f = std::floor(kBoxHeadroom * box[t] / rc);
        if (!(f <= 4096.0)) return fail(ctx, RBE_EINVAL, "box / rc too large for the cell list (> 2048 cells per axis)");
        cells *= std::max<int64_t>(1, (int64_t)f);
    }
    if (cells > b.cellcap) {
        ctx_free(ctx, b.cnt); ctx_free(ctx, b.start); ctx_free(ctx, b.cursor);
        b.cnt = b.start = b.cursor = nullptr;
        b.cellcap = 0;
        if ((e = ctx_alloc(ctx, &b.cnt, sizeof(int) * cells)) != cudaSuccess ||
            (e = ctx_alloc(ctx, &b.start, sizeof(int) * cells)) != cudaSuccess ||
            (e = ctx_alloc(ctx, &b.cursor, sizeof(int) * cells)) != cudaSuccess)
            return npt_fail(ctx, e, "cudaMalloc(cells)");
        b.cellcap = (int)cells;
    }
    if (skin > 0.0) {
        if (!b.nls && (e = ctx_alloc(ctx, reinterpret_cast<NListState**>(&b.nls), sizeof(NListState))) != cudaSuccess)
            return npt_fail(ctx, e, "cudaMalloc(list state)");
        const double rl = rc + skin, V = box[0] * box[1] * box[2];
        const double expect = 4.0 / 3.0 * 3.14159265358979323846 * rl * rl * rl * (double)N / V;
        const double capd = std::ceil((2.0 * expect + 64.0) / 32.0) * 32.0;
        if (!(capd <= 65536.0)) return fail(ctx, RBE_EINVAL, "neighbour list too long: reduce rc + skin");
        const int cap = (int)capd;
        const int64_t entries = (int64_t)cap * N;
        if (entries > b.nl_entries || N > b.ncap_list) {
            ctx_free(ctx, b.nbr); ctx_free(ctx, b.nnb); ctx_free(ctx, b.sref);
            b.nbr = nullptr; b.nnb = nullptr; b.sref = nullptr; b.nl_entries = 0; b.ncap_list = 0;
            if ((e = ctx_alloc(ctx, &b.nbr, sizeof(int) * entries)) != cudaSuccess ||
                (e = ctx_alloc(ctx, &b.nnb, sizeof(int) * N)) != cudaSuccess ||
                (e = ctx_alloc(ctx, &b.sref, sizeof(float4) * N)) != cudaSuccess)
                return npt_fail(ctx, e, "cudaMalloc(neighbour list)");
            b.nl_entries = entries;
            b.ncap_list = N;
        }
        b.nbr_cap = cap;
    }
    const int need = pair_blocks(ctx, N, false) + (int)((N + kNptThreads - 1) / kNptThreads);
    if (need > b.partcap) {
        ctx_free(ctx, b.partials);
        b.partials = nullptr;
        b.partcap = 0;
        if ((e = ctx_alloc(ctx, &b.partials, sizeof(double) * kPartStride * (size_t)need)) != cudaSuccess)
            return npt_fail(ctx, e, "cudaMalloc(npt partials)");
        b.partcap = need;
    }
    return RBE_OK;
}

// The cell list of the constants in ctx->npt.cellc: count, scan, fill, per-cell sort and the
// packed positions (FP64 as well with fp64).  With a neighbour list (nls) the launches exit at
// once on steps that do not rebuild it.
rbe_status launch_cell_list(rbe_ctx ctx, int64_t N, const double* pos, const double* q, void* nls_v, bool fp64)
{
    NptBuffers& b = ctx->npt;
    cudaStream_t s = ctx->stream;
    NListState* nls = static_cast<NListState*>(nls_v);
    const CellConsts* cc = static_cast<const CellConsts*>(b.cellc);
    const int nb = (int)((N + kNptThreads - 1) / kNptThreads);
    cudaError_t e = cudaMemsetAsync(b.cnt, 0, sizeof(int) * b.cellcap, s);
    if (e != cudaSuccess) return npt_fail(ctx, e, "cudaMemsetAsync(cells)");
    k_cl_count<<<nb, kNptThreads, 0, s>>>(N, pos, cc, b.cid, b.cnt, ctx->d.status, nls);
    k_cl_scan<<<1, kScanThreads, 0, s>>>(cc, b.cnt, b.start, b.cursor, nls);
    k_cl_fill<<<nb, kNptThreads, 0, s>>>(N, b.cid, b.cursor, b.fill, nls);
    const int64_t sort_blocks = ((int64_t)b.cellcap + kSortWarps - 1) / kSortWarps;
    k_cl_sort<<<(unsigned)sort_blocks, kSortWarps * 32, 0, s>>>(cc, b.cnt, b.start, b.fill, b.sorted, pos, q, b.spos32,
                                                              fp64 ? b.spos64 : nullptr, nls);
    return npt_check(ctx, "cell list");
}

// Forces, virial and energies at the current state (k-space batch `batch`), then the
// finishing kernel (with or without the R^p/2 and V^p/2 of the step's end).  `parts` selects
// the k-space (1), the real space (2) and the finishing kernel (4): a caller that evaluates
// the k-space itself (into npt.Fk and npt.WEk) runs 2 and 4 only.
static rbe_status npt_forces(rbe_ctx ctx, rbe_system* sys, uint64_t batch, int do_kick, int parts = 7)
{
    NptBuffers& b = ctx->npt;
    const rbe_npt_params& prm = sys->params;
    cudaStream_t s = ctx->stream;
    const int64_t N = sys->N;
    const int nb = (int)((N + kNptThreads - 1) / kNptThreads);
    const int nbp = pair_blocks(ctx, N, ctx->precision == RBE_FP64);
    rbe_status st;
    if (prm.kspace && (parts & 1)) {
        // tables from the device box and the sampler (one launch), then the evaluation
        (void)batch;  // the batch index is the device-resident step index (set by the caller)
        if ((st = launch_tables_sample_device(ctx, ctx->P, sys->cell,
                                              reinterpret_cast<const unsigned long long*>(sys->cell + kCellStep))) !=
            RBE_OK)
            return st;
        ctx->tables_dirty = true;  // the snapshot API must rebuild from its own box
        if ((st = launch_rbe(ctx, N, sys->pos, sys->charge, ctx->P, b.Fk, b.WEk, b.WEk + 9)) != RBE_OK)
            return st;
    }
    if (prm.real && N > 0 && (parts & 2)) {
        const bool fp64 = ctx->precision == RBE_FP64;
        if (fp64 && b.n64 < N) return fail(ctx, RBE_ESTATE, "precision changed to FP64 after rbe_npt_init: call it again");
        const bool list = prm.skin > 0.0;
        if (list && (!b.nls || b.ncap_list < N)) return fail(ctx, RBE_ESTATE, "skin changed after rbe_npt_init: call it again");
        NListState* nls = list ? static_cast<NListState*>(b.nls) : nullptr;
        const CellConsts* cc = static_cast<const CellConsts*>(b.cellc);
        if (list) {
            const int grid = (int)std::min<int64_t>(nb, (int64_t)ctx->num_sms * 4);
            if (fp64)
                k_nl_check<true><<<grid, kNptThreads, 0, s>>>(N, sys->pos, sys->charge, b.sorted, b.spos32, b.spos64,
                                                            b.sref, cc, nls);
            else
                k_nl_check<false><<<grid, kNptThreads, 0, s>>>(N, sys->pos, sys->charge, b.sorted, b.spos32, nullptr,
                                                             b.sref, cc, nls);
        }
        if ((st = launch_cell_list(ctx, N, sys->pos, sys->charge, nls, fp64)) != RBE_OK) return st;
        const PairConst pc = make_pair_const(prm.rc, ctx->alpha, prm.qqr2e, prm.lj_sigma, prm.lj_eps);
        const ListArgs la{nls, b.nbr, b.nnb, b.sref, ctx->d.status, b.nbr_cap};
        const double4_32a* s64 = fp64 ? b.spos64 : nullptr;
        const bool diag = prm.barostat >= 2;  // rectangular cell: the virial diagonal
        auto pair = [&](auto f64_tag, auto mode_tag) {
            constexpr bool F64 = decltype(f64_tag)::value;
            constexpr int MODE = decltype(mode_tag)::value;
            if constexpr (MODE == kPairBuild)
                k_pair<F64, MODE><<<nbp, kPairWarps * 32, 0, s>>>(N, cc, pc, b.cid, b.cnt, b.start, b.sorted,
                                                                  b.spos32, s64, b.Fr, b.partials, la);
            else if (diag)
                k_pair<F64, MODE, true><<<nbp, kPairWarps * 32, 0, s>>>(N, cc, pc, b.cid, b.cnt, b.start, b.sorted,
                                                                        b.spos32, s64, b.Fr, b.partials, la);
            else
                k_pair<F64, MODE><<<nbp, kPairWarps * 32, 0, s>>>(N, cc, pc, b.cid, b.cnt, b.start, b.sorted,
                                                                  b.spos32, s64, b.Fr, b.partials, la);
        };
        using T = std::true_type;
        using F = std::false_type;
        using Cells = std::integral_constant<int, kPairCells>;
        using Build = std::integral_constant<int, kPairBuild>;
        using List = std::integral_constant<int, kPairList>;
        if (!list) {
            if (fp64) pair(T{}, Cells{});
            else pair(F{}, Cells{});
        } else if (fp64) {
            pair(T{}, Build{});
            pair(T{}, List{});
        } else {
            pair(F{}, Build{});
            pair(F{}, List{});
        }
        if ((st = npt_check(ctx, "real-space kernels")) != RBE_OK) return st;
    }
    if (!(parts & 4)) return RBE_OK;
    if (prm.barostat >= 2)
        k_npt_finish<true><<<std::max(1, nb), kNptThreads, 0, s>>>(
            N, sys->mom, sys->force, b.mprop, b.Fk, b.Fr, b.WEk, reinterpret_cast<const NptCoef*>(b.coef), b.partials,
            nbp, b.counter, sys->cell, prm, do_kick, ctx->d.status);
    else
        k_npt_finish<false><<<std::max(1, nb), kNptThreads, 0, s>>>(
            N, sys->mom, sys->force, b.mprop, b.Fk, b.Fr, b.WEk, reinterpret_cast<const NptCoef*>(b.coef), b.partials,
            nbp, b.counter, sys->cell, prm, do_kick, ctx->d.status);
    return npt_check(ctx, "k_npt_finish");
}

rbe_status npt_validate(rbe_ctx ctx, const rbe_system* sys)
{
    if (!sys) return fail(ctx, RBE_EINVAL, "system is NULL");
    const rbe_npt_params& p = sys->params;
    if (sys->N < 1 || sys->N > ((int64_t)1 << 31) - 256) return fail(ctx, RBE_EINVAL, "N out of range");
    if (!sys->pos || !sys->mom || !sys->force || !sys->charge || !sys->mass || !sys->cell)
        return fail(ctx, RBE_EINVAL, "system buffers must not be NULL");
    if (!(p.dt > 0.0) || !(p.kT >= 0.0) || !(p.gamma >= 0.0) || !(p.gamma_V >= 0.0) || !(p.rc > 0.0) ||
        !(p.max_disp >= 0.0) || !(p.skin >= 0.0) || !std::isfinite(p.skin))
        return fail(ctx, RBE_EINVAL, "invalid NPT parameters");
    if (p.barostat < 0 || p.barostat > 3) return fail(ctx, RBE_EINVAL, "barostat must be 0, 1, 2 or 3");
    if (p.barostat == 1 && !(p.M_V > 0.0 && std::isfinite(p.M_V)))
        return fail(ctx, RBE_EINVAL, "isotropic barostat needs M_V > 0");
    for (int j = 0; j < 3; ++j)
        if (((p.barostat == 2) || (p.barostat == 3 && j != 1)) && !(p.M_cell[j] > 0.0 && std::isfinite(p.M_cell[j])))
            return fail(ctx, RBE_EINVAL, "rectangular barostat needs positive finite cell masses");
    if (p.barostat == 3 && !std::isfinite(p.gamma0)) return fail(ctx, RBE_EINVAL, "gamma0 must be finite");
    if ((sys->step >> 56) != 0) return fail(ctx, RBE_EINVAL, "step must be < 2^56");
    return RBE_OK;
}

// The nearest-image real space needs rc <= l/2.  The host checks the box it is given (the
// caller's initial box, read back once by rbe_npt_init).
static rbe_status npt_box_check(rbe_ctx ctx, const rbe_system* sys, double box[3])
{
    cudaError_t e = cudaMemcpyAsync(box, sys->cell, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return npt_fail(ctx, e, "read box");
    for (int t = 0; t < 3; ++t) {
        if (!(box[t] > 0.0) || !std::isfinite(box[t])) return fail(ctx, RBE_EINVAL, "cell box must be > 0");
        if (sys->params.real && box[t] < 2.0 * sys->params.rc)
            return fail(ctx, RBE_EINVAL, "real space needs rc <= l/2 on every axis");
    }
    if (sys->params.barostat == 3 && box[0] != box[1])
        return fail(ctx, RBE_EINVAL, "the semi-isotropic cell needs l_x = l_y");
    return RBE_OK;
}

// Everything of rbe_npt_init before the first forces: the box check, scratch, tables, 1/m and
// sqrt(m), the cell-list constants of the initial box, the list state, the step index set to
// `batch` (shared with the rigid-water step).
rbe_status npt_prepare(rbe_ctx ctx, rbe_system* sys, uint64_t batch)
{
    rbe_status st;
    double box[3];
    if ((st = npt_box_check(ctx, sys, box)) != RBE_OK) return st;
    if ((st = npt_ensure(ctx, sys->N, box, sys->params.rc, sys->params.skin)) != RBE_OK) return st;
    // tables for boxes up to twice as long as the initial one
    int need = 0;
    for (int t = 0; t < 3; ++t) {
        const int M = host_axis_M(ctx->alpha, kBoxHeadroom * box[t]);
        if (M > (1 << 20)) return fail(ctx, RBE_EINVAL, "alpha l^2 too large for the per-axis tables");
        need = std::max(need, 2 * M + 1);
    }
    if ((st = ensure_table_capacity(ctx, need)) != RBE_OK) return st;
    ctx->npt_ready_N = sys->N;
    ctx->flex_ready_N = -1;  // the shared scratch now holds this system's masses and cell list
    ctx->water_ready_N = -1;
    // per-particle 1/m and sqrt(m), and the cell-list constants of the initial box
    NptBuffers& b = ctx->npt;
    k_mass_props<<<(unsigned)((sys->N + kNptThreads - 1) / kNptThreads), kNptThreads, 0, ctx->stream>>>(
        sys->N, sys->mass, b.mprop);
    const double skin = sys->params.skin > 0.0 ? sys->params.skin : 0.0;
    k_cell_consts<<<1, 32, 0, ctx->stream>>>(sys->cell, sys->params.rc, sys->params.rc + skin, b.cellcap,
                                             static_cast<CellConsts*>(b.cellc));
    if (skin > 0.0)
        k_nl_init<<<1, 32, 0, ctx->stream>>>(static_cast<NListState*>(b.nls), (float)(sys->params.rc + skin),
                                             (float)sys->params.rc);
    k_npt_set_step<<<1, 32, 0, ctx->stream>>>(sys->cell, batch);
    return npt_check(ctx, "k_npt_set_step");
}

rbe_status launch_npt_set_step(rbe_ctx ctx, double* cell, uint64_t step)
{
    k_npt_set_step<<<1, 32, 0, ctx->stream>>>(cell, step);
    return npt_check(ctx, "k_npt_set_step");
}

// The isotropic cell part of a step (k_npt_cell_a) into ctx->npt.coef and the cell constants.
rbe_status launch_npt_cell_iso(rbe_ctx ctx, rbe_system* sys)
{
    k_npt_cell_a<<<1, kCellWarps * 32, 0, ctx->stream>>>(sys->cell, reinterpret_cast<NptCoef*>(ctx->npt.coef),
                                                       sys->params, ctx->seed, ctx->npt.cellcap,
                                                       static_cast<CellConsts*>(ctx->npt.cellc));
    return npt_check(ctx, "k_npt_cell_a");
}

rbe_status npt_init(rbe_ctx ctx, rbe_system* sys, uint64_t batch)
{
    rbe_status st = npt_validate(ctx, sys);
    if (st != RBE_OK) return st;
    if ((st = npt_prepare(ctx, sys, batch)) != RBE_OK) return st;
    st = npt_forces(ctx, sys, batch, 0);
    if (st != RBE_OK) return st;
    k_npt_set_step<<<1, 32, 0, ctx->stream>>>(sys->cell, sys->step);
    return npt_check(ctx, "k_npt_set_step");
}

// The first part of a step: the cell update (V^p/2, V/2, O^p, V/2) and the particles' drift
// (R^p/2, R/2, O, R/2).
static rbe_status npt_move(rbe_ctx ctx, rbe_system* sys)
{
    cudaStream_t s = ctx->stream;
    const int64_t N = sys->N;
    const int nb = (int)((N + kNptThreads - 1) / kNptThreads);
    NptCoef* cf = reinterpret_cast<NptCoef*>(ctx->npt.coef);
    const NptBuffers& b = ctx->npt;
    if (sys->params.barostat >= 2)
        k_npt_cell_rect<<<1, kRectWarps * 32, 0, s>>>(sys->cell, cf, sys->params, ctx->seed, b.cellcap,
                                                      static_cast<CellConsts*>(b.cellc));
    else
        k_npt_cell_a<<<1, kCellWarps * 32, 0, s>>>(sys->cell, cf, sys->params, ctx->seed, b.cellcap,
                                                   static_cast<CellConsts*>(b.cellc));
    const bool rect = sys->params.barostat >= 2;
    auto drift = [&](auto f32_tag, auto rect_tag) {
        k_npt_drift<decltype(f32_tag)::value, decltype(rect_tag)::value><<<nb, kNptThreads, 0, s>>>(
            N, sys->pos, sys->mom, sys->force, b.mprop, cf, ctx->seed, sys->cell);
    };
    using T = std::true_type;
    using F = std::false_type;
    if (ctx->precision == RBE_FP64) rect ? drift(F{}, T{}) : drift(F{}, F{});
    else rect ? drift(T{}, T{}) : drift(T{}, F{});
    return npt_check(ctx, "k_npt_cell_a/k_npt_drift");
}

rbe_status npt_run(rbe_ctx ctx, rbe_system* sys, int32_t nsteps)
{
    if (nsteps < 1) return fail(ctx, RBE_EINVAL, "nsteps must be >= 1");
    rbe_status st = npt_validate(ctx, sys);
    if (st != RBE_OK) return st;
    if (ctx->npt_ready_N != sys->N) return fail(ctx, RBE_ESTATE, "call rbe_npt_init for this system first");
    for (int32_t k = 0; k < nsteps; ++k) {
        const uint64_t step = sys->step;
        if ((st = npt_move(ctx, sys)) != RBE_OK) return st;
        if ((st = npt_forces(ctx, sys, step, 1)) != RBE_OK) return st;
        sys->step = step + 1;
    }
    return RBE_OK;
}

rbe_status npt_step_phase(rbe_ctx ctx, rbe_system* sys, int phase)
{
    if (ctx->npt_ready_N != sys->N) return fail(ctx, RBE_ESTATE, "call rbe_npt_init for this system first");
    if (phase == kNptPhaseMove) return npt_move(ctx, sys);
    if (phase == kNptPhaseReal) return npt_forces(ctx, sys, sys->step, 1, 2);
    rbe_status st = npt_forces(ctx, sys, sys->step, 1, 4);
    if (st == RBE_OK) sys->step += 1;
    return st;
}

}  // namespace rbe
