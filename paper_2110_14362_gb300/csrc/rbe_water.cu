// Langevin NPT step of rigid 3-site water on the device (the paper's water runs keep molecules
// rigid, Sec. 5.1; the equations of Sec. 3.2 act on the molecular centres, SHAKE and RATTLE hold
// the internal geometry).  Sites are stored O, H, H per molecule; molecules stay whole in storage
// (after each step a molecule moves by the lattice vector that brings its oxygen into the box).
//
// One step is a fixed sequence of launches on the context's stream:
//   k_npt_cell_a    the isotropic cell part (rbe_npt.cu): V^p/2 with the molecular pressure, the
//                   sub-step coefficients, V/2, O^p, V/2, the cell-list constants
//   k_water_drift   one thread per molecule: R^p/2, R/2, O, R/2 of the centre (exact flows) and of
//                   the internal motion (kick, free move, SHAKE, momentum correction, projection)
//   k-space         tables of the device box, sampler, rho, force pass over all sites
//   cell list       count, scan, fill, sort (rbe_npt.cu)
//   k_water_pair    one warp per site: erfc Coulomb with sites of other molecules, LJ between
//                   oxygens, nearest image per pair
//   k_water_finish  one thread per molecule: total forces with the intramolecular exclusion,
//                   R^p/2, the centres' 2K and the molecular virial; last block: P_ins, V^p/2
// Everything runs in FP64 except the k-space, which follows the context's precision.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "rbe_context.h"
#include "rbe_device.cuh"
#include "rbe_npt_common.cuh"

namespace rbe {

// Molecules per block of the per-molecule kernels (k_water_whole, k_water_drift, k_water_finish):
// one warp, so that their FP64 constraint and virial arithmetic spreads over as many SMs'
// FP64 pipes as there are warps of molecules (3000 molecules: 94 SMs, against 24 with blocks of
// 128, where the drift took 97 us bound by the FP64 pipe of those 24 SMs).
constexpr int kWaterThreads = 32;
constexpr int kCellExcl = 25;       // cell block: the exclusion energy
constexpr int kWaterHitCap = 64;    // buffered candidates per warp (< 32 buffered + 32 new)

// the sites of constraint c: (0,1), (0,2), (1,2)
__host__ __device__ constexpr int wpa(int c) { return c == 2 ? 1 : 0; }
__host__ __device__ constexpr int wpb(int c) { return c == 0 ? 1 : 2; }

// The molecule starting at site 3I made whole from its oxygen by the nearest image.
__device__ __forceinline__ void w_whole(const double* __restrict__ pos, int64_t I, const double L[3],
                                        const double inv[3], double x[3][3])
{
    #pragma unroll
    for (int t = 0; t < 3; ++t) x[0][t] = pos[9 * I + t];
    for (int s = 1; s < 3; ++s)
        #pragma unroll
        for (int t = 0; t < 3; ++t) {
            const double d = pos[9 * I + 3 * s + t] - x[0][t];
            x[s][t] = x[0][t] + (d - L[t] * rint(d * inv[t]));
        }
}

__device__ __forceinline__ double det3(const double A[3][3])
{
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
           A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// x = A^{-1} b by Cramer's rule with one reciprocal of det A.
__device__ __forceinline__ void solve3(const double A[3][3], const double b[3], double x[3])
{
    const double id = 1.0 / det3(A);
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        double B[3][3];
        #pragma unroll
        for (int c = 0; c < 3; ++c)
            #pragma unroll
            for (int d = 0; d < 3; ++d) B[c][d] = d == k ? b[c] : A[c][d];
        x[k] = det3(B) * id;
    }
}

// The change of (x_a - x_b) of constraint c per unit multiplier of constraint d, in units of
// s_d: ((a_c == a_d) - (a_c == b_d))/m_{a_c} - ((b_c == a_d) - (b_c == b_d))/m_{b_c}.
__device__ __forceinline__ double coupling(int c, int d, const double im[3])
{
    const int a = wpa(c), b = wpb(c);
    return ((a == wpa(d)) - (a == wpb(d))) * im[a] - ((b == wpa(d)) - (b == wpb(d))) * im[b];
}

// The position constraints of one molecule after an unconstrained move from the constrained xo:
// x_i <- x_i + sum_d lambda_d s_old,d (e_{i,a_d} - e_{i,b_d}) / m_i with lambda making every
// |x_a - x_b|^2 = d^2, the equations SHAKE solves (corrections along the old separations).  Here by
// Newton's method on lambda (each step an exact 3x3 solve, quadratic convergence from lambda = 0):
// it stops once every |r^2 - d^2| <= tol d^2, at the root SHAKE's sweeps converge to.  Returns
// false when max_iter iterations did not get there.
__device__ bool w_shake(double x[3][3], const double xo[3][3], const double im[3], const rbe_water_params& wp)
{
    const double dd[3] = {wp.d_OH * wp.d_OH, wp.d_OH * wp.d_OH, wp.d_HH * wp.d_HH};
    double so[3][3], K[3][3];
    #pragma unroll
    for (int c = 0; c < 3; ++c) {
        #pragma unroll
        for (int t = 0; t < 3; ++t) so[c][t] = xo[wpa(c)][t] - xo[wpb(c)][t];
        #pragma unroll
        for (int d = 0; d < 3; ++d) K[c][d] = coupling(c, d, im);
    }
    for (int it = 0; it < wp.shake_max_iter; ++it) {
        double s[3][3], g[3];
        bool done = true;
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
            #pragma unroll
            for (int t = 0; t < 3; ++t) s[c][t] = x[wpa(c)][t] - x[wpb(c)][t];
            g[c] = s[c][0] * s[c][0] + s[c][1] * s[c][1] + s[c][2] * s[c][2] - dd[c];
            if (fabs(g[c]) > wp.shake_tol * dd[c]) done = false;
        }
        if (done) return true;
        double J[3][3], dl[3], rhs[3] = {-g[0], -g[1], -g[2]};
        #pragma unroll
        for (int c = 0; c < 3; ++c)
            #pragma unroll
            for (int d = 0; d < 3; ++d)
                J[c][d] = 2.0 * K[c][d] * (s[c][0] * so[d][0] + s[c][1] * so[d][1] + s[c][2] * so[d][2]);
        solve3(J, rhs, dl);
        #pragma unroll
        for (int d = 0; d < 3; ++d)
            #pragma unroll
            for (int t = 0; t < 3; ++t) {
                x[wpa(d)][t] += dl[d] * so[d][t] * im[wpa(d)];
                x[wpb(d)][t] -= dl[d] * so[d][t] * im[wpb(d)];
            }
    }
    return false;
}

// RATTLE's velocity stage: p_i += sum_c mu_c s_c (e_{i,a_c} - e_{i,b_c}), s_c = x_{a_c} - x_{b_c},
// mu solving the 3x3 system that makes every (v_a - v_b) . s_c vanish (Cramer's rule).
__device__ void w_project(double p[3][3], const double x[3][3], const double im[3])
{
    double s[3][3];
    #pragma unroll
    for (int c = 0; c < 3; ++c)
        #pragma unroll
        for (int t = 0; t < 3; ++t) s[c][t] = x[wpa(c)][t] - x[wpb(c)][t];
    double A[3][3], b[3], mu[3];
    #pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int a = wpa(c), bb = wpb(c);
        double dv = 0.0;
        #pragma unroll
        for (int t = 0; t < 3; ++t) dv += (p[a][t] * im[a] - p[bb][t] * im[bb]) * s[c][t];
        b[c] = -dv;
        #pragma unroll
        for (int d = 0; d < 3; ++d)
            A[c][d] = coupling(c, d, im) * (s[c][0] * s[d][0] + s[c][1] * s[d][1] + s[c][2] * s[d][2]);
    }
    solve3(A, b, mu);
    #pragma unroll
    for (int c = 0; c < 3; ++c)
        #pragma unroll
        for (int t = 0; t < 3; ++t) {
            p[wpa(c)][t] += mu[c] * s[c][t];
            p[wpb(c)][t] -= mu[c] * s[c][t];
        }
}

// R^p/2 of one molecule: the centre's exact flow P <- P a + 100 F b, the internal momenta kicked by
// 100 h (F_i - m_i F / M), then the projection.
__device__ void w_kick(double p[3][3], const double F[3][3], const double x[3][3], const double m3[3],
                       const double im[3], double a, double b, double h)
{
    const double M = m3[0] + m3[1] + m3[2];
    double P[3] = {0.0, 0.0, 0.0}, Ft[3] = {0.0, 0.0, 0.0};
    #pragma unroll
    for (int k = 0; k < 3; ++k)
        #pragma unroll
        for (int t = 0; t < 3; ++t) {
            P[t] += p[k][t];
            Ft[t] += F[k][t];
        }
    double dP[3];
    #pragma unroll
    for (int t = 0; t < 3; ++t) dP[t] = P[t] * a + kFConv * Ft[t] * b - P[t];
    #pragma unroll
    for (int k = 0; k < 3; ++k)
        #pragma unroll
        for (int t = 0; t < 3; ++t) p[k][t] += kFConv * h * (F[k][t] - m3[k] * Ft[t] / M) + (m3[k] / M) * dP[t];
    w_project(p, x, im);
}

// R/2 of one molecule: the centre R <- R + R (a - 1) + cap((P/M) b), the offsets moved by h (p/m
// - P/M) and SHAKEn, the SHAKE displacement added to the momenta as m dd / h, then the projection
// at the new positions.  Returns false when SHAKE did not converge.
__device__ bool w_drift(double x[3][3], double p[3][3], const double m3[3], const double im[3], double am1, double b,
                        double h, double cap, const rbe_water_params& wp)
{
    const double M = m3[0] + m3[1] + m3[2];
    double R[3], P[3] = {0.0, 0.0, 0.0}, d[3][3], dn[3][3], ds[3][3];
    #pragma unroll
    for (int t = 0; t < 3; ++t) R[t] = (m3[0] * x[0][t] + m3[1] * x[1][t] + m3[2] * x[2][t]) / M;
    #pragma unroll
    for (int k = 0; k < 3; ++k)
        #pragma unroll
        for (int t = 0; t < 3; ++t) {
            P[t] += p[k][t];
            d[k][t] = x[k][t] - R[t];
        }
    double D[3];
    #pragma unroll
    for (int t = 0; t < 3; ++t) D[t] = (P[t] / M) * b;
    if (cap > 0.0) {
        const double len = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
        if (len > cap)
            #pragma unroll
            for (int t = 0; t < 3; ++t) D[t] *= cap / len;
    }
    double Rn[3];
    #pragma unroll
    for (int t = 0; t < 3; ++t) Rn[t] = R[t] + R[t] * am1 + D[t];
    #pragma unroll
    for (int k = 0; k < 3; ++k)
        #pragma unroll
        for (int t = 0; t < 3; ++t) {
            dn[k][t] = d[k][t] + h * (p[k][t] * im[k] - P[t] / M);
            ds[k][t] = dn[k][t];
        }
    const bool ok = w_shake(ds, d, im, wp);
    #pragma unroll
    for (int k = 0; k < 3; ++k)
        #pragma unroll
        for (int t = 0; t < 3; ++t) {
            p[k][t] += m3[k] * (ds[k][t] - dn[k][t]) / h;
            x[k][t] = Rn[t] + ds[k][t];
        }
    w_project(p, x, im);
    return ok;
}

// The molecules made whole from their oxygen and moved by the lattice vector that brings the
// oxygen into [0, L) (rbe_water_init: the caller's sites may be wrapped one by one).
__global__ void __launch_bounds__(kWaterThreads)
k_water_whole(int64_t Nmol, double* __restrict__ pos, const double* __restrict__ cell)
{
    const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= Nmol) return;
    const double L[3] = {cell[0], cell[1], cell[2]};
    const double inv[3] = {1.0 / L[0], 1.0 / L[1], 1.0 / L[2]};
    double x[3][3];
    w_whole(pos, I, L, inv, x);
    #pragma unroll
    for (int t = 0; t < 3; ++t) {
        const double sh = L[t] * floor(x[0][t] * inv[t]);
        #pragma unroll
        for (int k = 0; k < 3; ++k) pos[9 * I + 3 * k + t] = x[k][t] - sh;
    }
}

// Particles before the forces, one thread per molecule: R^p/2, R/2, O, R/2, the wrap by molecule.
__global__ void __launch_bounds__(kWaterThreads)
k_water_drift(int64_t Nmol, double* __restrict__ pos, double* __restrict__ mom, const double* __restrict__ force,
              const double* __restrict__ mass, const NptCoef* __restrict__ cfp, uint64_t seed,
              const double* __restrict__ cell, const rbe_water_params wp, double dt, unsigned* __restrict__ status)
{
    const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= Nmol) return;
    const uint64_t step = cell_step(cell);
    const NptCoef& c = *cfp;
    const double h = 0.5 * dt;
    const double m3[3] = {mass[3 * I], mass[3 * I + 1], mass[3 * I + 2]};
    double x[3][3], p[3][3], F[3][3];
    w_whole(pos, I, c.L, c.invL, x);
    #pragma unroll
    for (int k = 0; k < 3; ++k)
        #pragma unroll
        for (int t = 0; t < 3; ++t) {
            p[k][t] = mom[9 * I + 3 * k + t];
            F[k][t] = force[9 * I + 3 * k + t];
        }
    const double im[3] = {1.0 / m3[0], 1.0 / m3[1], 1.0 / m3[2]};
    w_kick(p, F, x, m3, im, c.a1[0], c.b1[0], h);
    bool ok = w_drift(x, p, m3, im, c.a2m1[0], c.b2[0], h, c.half_cap, wp);
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        double z[4] = {0.0, 0.0, 0.0, 0.0};
        if (c.noise) npt_normals(seed, 1u, step, (uint32_t)(3 * I + k), z);
        const double s = c.sog * sqrt(m3[k]);
        #pragma unroll
        for (int t = 0; t < 3; ++t) p[k][t] = p[k][t] * c.g + s * z[t];
    }
    w_project(p, x, im);
    ok = w_drift(x, p, m3, im, c.a3m1[0], c.b3[0], h, c.half_cap, wp) && ok;
    if (!ok) atomicOr(status, kStatusShake);
    #pragma unroll
    for (int t = 0; t < 3; ++t) {
        const double sh = c.L[t] * floor(x[0][t] * c.invL[t]);
        #pragma unroll
        for (int k = 0; k < 3; ++k) {
            pos[9 * I + 3 * k + t] = x[k][t] - sh;
            mom[9 * I + 3 * k + t] = p[k][t];
        }
    }
}

// ---------------------------------------------------------------------------------
// Real space between sites of different molecules (Sec. 4.1 Eqs. (U2), (force)) on the cell list
// of the current box: one warp per site in cell order; the lanes set up the 18 row segments of
// the neighbouring cells (an axis with fewer than 3 cells visits each of its cells once) and
// stride over their slots; the separation is the nearest image per pair (sites may sit up to a
// bond outside the box).  The search runs on the FP32 packed positions with rc plus a margin above
// their rounding; the hits (slots) go to a per-warp buffer in ballot order and are evaluated 32 at a
// time, one per lane, in FP64 from the FP64 packed positions with the exact cutoff.  A hit of the
// same molecule (site index / 3) is skipped; LJ acts between oxygens (site index divisible by 3).
// Lane sums through a fixed shuffle tree.  Each pair is
// visited from both ends: energies and the virial take half.  Per-block partials {W_r, E_coul,
// E_lj} at slots 1..3 (the isotropic layout).  A box beyond the cell arrays leaves F_r = 0.
__global__ void __launch_bounds__(kPairWarps * 32, kPairBlocksPerSM64)
k_water_pair(int64_t N, const CellConsts* __restrict__ cc, const PairConst pc, const int* __restrict__ cid,
             const int* __restrict__ cnt, const int* __restrict__ start, const int* __restrict__ sorted,
             const float4* __restrict__ spos32, const double4_32a* __restrict__ spos64, double* __restrict__ Fr,
             double* __restrict__ partials)
{
    __shared__ int hits[kPairWarps][kWaterHitCap];  // slots of candidates within the FP32 search radius
    __shared__ double red[3][kPairWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nc[3] = {cc->nc[0], cc->nc[1], cc->nc[2]};
    const double L[3] = {cc->L[0], cc->L[1], cc->L[2]}, inv[3] = {cc->invL[0], cc->invL[1], cc->invL[2]};
    const float Lf[3] = {cc->Lf[0], cc->Lf[1], cc->Lf[2]}, invf[3] = {cc->invLf[0], cc->invLf[1], cc->invLf[2]};
    // FP32 search radius: rc plus 2^-16 l_max, far above the FP32 rounding of a separation; the
    // exact cutoff is applied in FP64
    const float pass = cc->pass64;
    double wsum = 0.0, ecsum = 0.0, elsum = 0.0;
    if (cc->ncell < 0) {
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < 3 * N; j += (int64_t)gridDim.x * blockDim.x)
            Fr[j] = 0.0;
    } else {
        const int nwarps = gridDim.x * kPairWarps;
        for (int u = blockIdx.x * kPairWarps + wib; u < (int)N; u += nwarps) {
            const int i = sorted[u];
            const double4_32a me = spos64[u];
            const float4 me32 = spos32[u];
            const int mol_i = i / 3;
            const bool oxy_i = i % 3 == 0;
            int lo = 0, hi = 0;
            {
                const int c = cid[i];
                const int cxy = nc[0] * nc[1];
                const int cz = c / cxy, cy = (c - cz * cxy) / nc[0], cx = c - cz * cxy - cy * nc[0];
                const int r = lane >> 1, part = lane & 1;
                const int dy = r % 3 - 1, dz = r / 3 - 1;
                const bool row_ok = r < 9 && dy >= (nc[1] >= 3 ? -1 : 0) && dy <= (nc[1] >= 2 ? 1 : 0) &&
                                    dz >= (nc[2] >= 3 ? -1 : 0) && dz <= (nc[2] >= 2 ? 1 : 0);
                if (row_ok) {
                    const int uy = cy + dy, uz = cz + dz;
                    const int yy = uy < 0 ? uy + nc[1] : (uy >= nc[1] ? uy - nc[1] : uy);
                    const int zz = uz < 0 ? uz + nc[2] : (uz >= nc[2] ? uz - nc[2] : uz);
                    const int row = (zz * nc[1] + yy) * nc[0], nx = nc[0];
                    int a = -1, b = -1;
                    if (nx < 3) {
                        if (part == 0) a = 0, b = nx - 1;
                    } else if (cx == 0) {
                        if (part == 0) a = 0, b = 1;
                        else a = b = nx - 1;
                    } else if (cx == nx - 1) {
                        if (part == 0) a = nx - 2, b = nx - 1;
                        else a = b = 0;
                    } else if (part == 0) {
                        a = cx - 1, b = cx + 1;
                    }
                    if (a >= 0) {
                        lo = start[row + a];
                        hi = start[row + b] + cnt[row + b];
                    }
                }
            }
            double fx = 0.0, fy = 0.0, fz = 0.0, w = 0.0, ec = 0.0, el = 0.0;
            int nh = 0;
            auto evaluate = [&](int count) {
                if (lane >= count) return;
                const int sj = hits[wib][lane];
                const int j = sorted[sj];
                if (j / 3 == mol_i) return;  // the same molecule (the site itself included)
                const double4_32a o = spos64[sj];
                double d[3] = {o.x - me.x, o.y - me.y, o.z - me.z};
                #pragma unroll
                for (int t = 0; t < 3; ++t) d[t] -= L[t] * rint(d[t] * inv[t]);
                const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!(r2 < pc.rc2)) return;
                const double r = sqrt(r2), inv_r = 1.0 / r, inv_r2 = inv_r * inv_r;
                const double coul = pc.qk * me.w * o.w * inv_r;
                const double er = erfc(pc.sa * r);
                ec += coul * er;
                double f = coul * (er + pc.two_sa_pi * r * exp(-pc.a * r2)) * inv_r2;
                if (oxy_i && j % 3 == 0 && pc.lj) {
                    const double sr2 = pc.s2 * inv_r2, sr6 = sr2 * sr2 * sr2;
                    el += pc.e4 * (sr6 * sr6 - sr6);
                    f += pc.e24 * (2.0 * sr6 * sr6 - sr6) * inv_r2;
                }
                fx -= f * d[0];
                fy -= f * d[1];
                fz -= f * d[2];
                w += f * r2;
            };
            for (int g = 0; g < 18; ++g) {
                const int glo = __shfl_sync(0xffffffffu, lo, g), ghi = __shfl_sync(0xffffffffu, hi, g);
                for (int s0 = glo; s0 < ghi; s0 += 32) {  // the same trip count on every lane
                    const int sl = s0 + lane;
                    const float4 o = spos32[sl < ghi ? sl : glo];
                    float dx = o.x - me32.x, dy = o.y - me32.y, dz = o.z - me32.z;
                    dx -= Lf[0] * rintf(dx * invf[0]);
                    dy -= Lf[1] * rintf(dy * invf[1]);
                    dz -= Lf[2] * rintf(dz * invf[2]);
                    const bool hit = sl < ghi && sl != u && dx * dx + dy * dy + dz * dz < pass;
                    const unsigned m = __ballot_sync(0xffffffffu, hit);
                    if (hit) hits[wib][nh + __popc(m & ((1u << lane) - 1u))] = sl;
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
                ec += __shfl_xor_sync(0xffffffffu, ec, off);
                el += __shfl_xor_sync(0xffffffffu, el, off);
            }
            if (lane == 0) {
                Fr[3 * (int64_t)i] = fx;
                Fr[3 * (int64_t)i + 1] = fy;
                Fr[3 * (int64_t)i + 2] = fz;
                wsum += 0.5 * w;
                ecsum += 0.5 * ec;
                elsum += 0.5 * el;
            }
        }
    }
    if (lane == 0) {
        red[0][wib] = wsum;
        red[1][wib] = ecsum;
        red[2][wib] = elsum;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int wv = 0; wv < kPairWarps; ++wv) t += red[threadIdx.x][wv];
        partials[kPartStride * (size_t)blockIdx.x + 1 + threadIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------------
// One thread per molecule: F_i = qqr2e F_k,i + F_r,i plus the intramolecular exclusion
// -qqr2e q_a q_b erf(sqrt(alpha) r)/r of its three site pairs (with real space on); with do_kick,
// R^p/2; the centres' 2K, the exclusion's virial plus the molecular correction -sum_i F_i . d_i,
// and the exclusion energy as block partials {0: 2K, 4: W, 5: E_excl}.  The last block sums the
// partials in a fixed order, forms W_mol = qqr2e tr(W_k) + W_r + W, P_ins = (2K + W_mol)/(3V) and,
// with do_kick, V^p/2 and the step index.
__global__ void __launch_bounds__(kWaterThreads)
k_water_finish(int64_t Nmol, double* __restrict__ mom, double* __restrict__ force, const double* __restrict__ pos,
               const double* __restrict__ q, const double* __restrict__ mass, const double* __restrict__ Fk,
               const double* __restrict__ Fr, const double* __restrict__ WEk, const NptCoef* __restrict__ cfp,
               double* __restrict__ partials, int nblocks_pair, unsigned* __restrict__ counter,
               double* __restrict__ cell, rbe_npt_params prm, double alpha, int do_kick, unsigned* __restrict__ status)
{
    __shared__ double red[3][kWaterThreads / 32];
    __shared__ bool is_last;
    const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double k2 = 0.0, wc = 0.0, ex = 0.0;
    if (I < Nmol) {
        const NptCoef& c = *cfp;
        const double L[3] = {cell[0], cell[1], cell[2]};
        const double inv[3] = {1.0 / L[0], 1.0 / L[1], 1.0 / L[2]};
        const double m3[3] = {mass[3 * I], mass[3 * I + 1], mass[3 * I + 2]};
        double x[3][3], F[3][3], p[3][3];
        w_whole(pos, I, L, inv, x);
        #pragma unroll
        for (int k = 0; k < 3; ++k)
            #pragma unroll
            for (int t = 0; t < 3; ++t) {
                const int64_t j = 9 * I + 3 * k + t;
                F[k][t] = (prm.kspace ? prm.qqr2e * Fk[j] : 0.0) + (prm.real ? Fr[j] : 0.0);
                p[k][t] = mom[j];
            }
        if (prm.real) {
            const double sa = sqrt(alpha), tsp = 2.0 * sqrt(alpha / kPi);
            #pragma unroll
            for (int cp = 0; cp < 3; ++cp) {
                const int a = wpa(cp), b = wpb(cp);
                double d[3];
                #pragma unroll
                for (int t = 0; t < 3; ++t) d[t] = x[b][t] - x[a][t];
                const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r = sqrt(r2);
                const double qq = prm.qqr2e * q[3 * I + a] * q[3 * I + b], ef = erf(sa * r);
                const double f = qq * (tsp * exp(-alpha * r2) / r - ef / r2) / r;
                ex -= qq * ef / r;
                #pragma unroll
                for (int t = 0; t < 3; ++t) {
                    F[b][t] += f * d[t];
                    F[a][t] -= f * d[t];
                }
                wc += f * r2;
            }
        }
        const double M = m3[0] + m3[1] + m3[2];
        double R[3];
        #pragma unroll
        for (int t = 0; t < 3; ++t) R[t] = (m3[0] * x[0][t] + m3[1] * x[1][t] + m3[2] * x[2][t]) / M;
        #pragma unroll
        for (int k = 0; k < 3; ++k)
            #pragma unroll
            for (int t = 0; t < 3; ++t) {
                wc -= F[k][t] * (x[k][t] - R[t]);
                force[9 * I + 3 * k + t] = F[k][t];
            }
        if (do_kick) {
            const double im[3] = {1.0 / m3[0], 1.0 / m3[1], 1.0 / m3[2]};
            w_kick(p, F, x, m3, im, c.a4[0], c.b4[0], 0.5 * prm.dt);
            #pragma unroll
            for (int k = 0; k < 3; ++k)
                #pragma unroll
                for (int t = 0; t < 3; ++t) mom[9 * I + 3 * k + t] = p[k][t];
        }
        double P[3] = {0.0, 0.0, 0.0};
        #pragma unroll
        for (int k = 0; k < 3; ++k)
            #pragma unroll
            for (int t = 0; t < 3; ++t) P[t] += p[k][t];
        k2 = (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / M * (1.0 / kFConv);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        k2 += __shfl_xor_sync(0xffffffffu, k2, off);
        wc += __shfl_xor_sync(0xffffffffu, wc, off);
        ex += __shfl_xor_sync(0xffffffffu, ex, off);
    }
    if (lane == 0) {
        red[0][warp] = k2;
        red[1][warp] = wc;
        red[2][warp] = ex;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double sum = 0.0;
        for (int wv = 0; wv < kWaterThreads / 32; ++wv) sum += red[threadIdx.x][wv];
        const int slot = threadIdx.x == 0 ? 0 : 3 + threadIdx.x;  // 0, 4, 5
        partials[kPartStride * (size_t)(nblocks_pair + blockIdx.x) + slot] = sum;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // fin: 0 2K, 1 W_r, 2 E_coul, 3 E_lj, 4 W (exclusion + correction), 5 E_excl
    __shared__ double fin[6][kWaterThreads];
    {
        double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int b = threadIdx.x; b < (int)gridDim.x; b += kWaterThreads) {
            const double* pb = partials + kPartStride * (size_t)(nblocks_pair + b);
            v[0] += __ldcg(pb);
            v[4] += __ldcg(pb + 4);
            v[5] += __ldcg(pb + 5);
        }
        if (prm.real)
            for (int b = threadIdx.x; b < nblocks_pair; b += kWaterThreads)
                for (int a = 1; a <= 3; ++a) v[a] += __ldcg(partials + kPartStride * (size_t)b + a);
        for (int a = 0; a < 6; ++a) fin[a][threadIdx.x] = v[a];
    }
    __syncthreads();
    for (int half = kWaterThreads / 2; half > 0; half >>= 1) {
        if (threadIdx.x < half)
            for (int a = 0; a < 6; ++a) fin[a][threadIdx.x] += fin[a][threadIdx.x + half];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double Wk = 0.0, Ek = 0.0;
    if (prm.kspace) {
        Wk = prm.qqr2e * (__ldcg(WEk + 0) + __ldcg(WEk + 4) + __ldcg(WEk + 8));
        Ek = prm.qqr2e * (__ldcg(WEk + 9) + __ldcg(WEk + 10));
    }
    const double K2 = fin[0][0], W = Wk + fin[1][0] + fin[4][0];
    const double V = cell[0] * cell[1] * cell[2];
    const double Pins = (K2 + W) / (3.0 * V);
    double pV = prm.barostat ? cell[3] : 0.0;
    if (do_kick && prm.barostat) pV += 0.5 * prm.dt * (Pins - prm.P_ext);
    cell[3] = pV;
    cell[4] = W;
    cell[5] = K2;
    cell[6] = Pins;
    cell[7] = Ek;
    cell[8] = fin[2][0];
    cell[9] = fin[3][0];
    cell[10] = V;
    cell[kCellExcl] = fin[5][0];
    if (do_kick) cell[kCellStep] = __longlong_as_double((long long)(cell_step(cell) + 1));
    if (!isfinite(Pins) || !isfinite(pV)) atomicOr(status, kStatusNonFinite);
    *counter = 0u;
}

// ---------------------------------------------------------------------------------
// Host side.

static rbe_status water_check(rbe_ctx ctx, const char* what)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RBE_OK : cuda_fail(ctx, e, what);
}

static rbe_status water_validate(rbe_ctx ctx, const rbe_system* sys, const rbe_water_params* wp)
{
    rbe_status st = npt_validate(ctx, sys);
    if (st != RBE_OK) return st;
    if (!wp) return fail(ctx, RBE_EINVAL, "water parameters are NULL");
    if (sys->N % 3 != 0) return fail(ctx, RBE_EINVAL, "N must count whole molecules (3 sites each)");
    if (sys->params.barostat > 1) return fail(ctx, RBE_EINVAL, "rigid water runs with barostat 0 or 1");
    if (sys->params.skin > 0.0) return fail(ctx, RBE_EINVAL, "rigid water runs without a neighbour list (skin 0)");
    if (!(wp->d_OH > 0.0) || !(wp->d_HH > 0.0) || !std::isfinite(wp->d_OH) || !std::isfinite(wp->d_HH) ||
        !(wp->d_HH < 2.0 * wp->d_OH) || !(wp->shake_tol > 0.0) || !(wp->shake_tol < 1e-3) || wp->shake_max_iter < 1)
        return fail(ctx, RBE_EINVAL, "invalid water parameters");
    return RBE_OK;
}

// Forces, molecular virial and energies at the current state (batch = the device step index),
// then the finishing kernel.
static rbe_status water_forces(rbe_ctx ctx, rbe_system* sys, int do_kick)
{
    NptBuffers& b = ctx->npt;
    const rbe_npt_params& prm = sys->params;
    cudaStream_t s = ctx->stream;
    const int64_t N = sys->N, Nmol = N / 3;
    const int nbp = pair_blocks(ctx, N, true);
    rbe_status st;
    if (prm.kspace) {
        if ((st = launch_tables_sample_device(ctx, ctx->P, sys->cell,
                                              reinterpret_cast<const unsigned long long*>(sys->cell + kCellStep))) !=
            RBE_OK)
            return st;
        ctx->tables_dirty = true;
        if ((st = launch_rbe(ctx, N, sys->pos, sys->charge, ctx->P, b.Fk, b.WEk, b.WEk + 9)) != RBE_OK) return st;
    }
    if (prm.real) {
        if (b.n64 < N) return fail(ctx, RBE_ESTATE, "the FP64 packed positions are missing: call rbe_water_init again");
        if ((st = launch_cell_list(ctx, N, sys->pos, sys->charge, nullptr, true)) != RBE_OK) return st;
        const PairConst pc = make_pair_const(prm.rc, ctx->alpha, prm.qqr2e, prm.lj_sigma, prm.lj_eps);
        k_water_pair<<<nbp, kPairWarps * 32, 0, s>>>(N, static_cast<const CellConsts*>(b.cellc), pc, b.cid, b.cnt,
                                                     b.start, b.sorted, b.spos32, b.spos64, b.Fr, b.partials);
        if ((st = water_check(ctx, "k_water_pair")) != RBE_OK) return st;
    }
    const int nbm = (int)std::max<int64_t>(1, (Nmol + kWaterThreads - 1) / kWaterThreads);
    k_water_finish<<<nbm, kWaterThreads, 0, s>>>(Nmol, sys->mom, sys->force, sys->pos, sys->charge, sys->mass, b.Fk,
                                                 b.Fr, b.WEk, reinterpret_cast<const NptCoef*>(b.coef), b.partials, nbp,
                                                 b.counter, sys->cell, prm, ctx->alpha, do_kick, ctx->d.status);
    return water_check(ctx, "k_water_finish");
}

rbe_status water_init(rbe_ctx ctx, rbe_system* sys, const rbe_water_params* wp, uint64_t batch)
{
    rbe_status st = water_validate(ctx, sys, wp);
    if (st != RBE_OK) return st;
    // the pair kernel reads FP64 packed positions whatever the context's precision
    const int prec = ctx->precision;
    ctx->precision = RBE_FP64;
    st = npt_prepare(ctx, sys, batch);
    ctx->precision = prec;
    if (st != RBE_OK) return st;
    ctx->npt_ready_N = -1;  // the shared scratch now holds a water system
    ctx->flex_ready_N = -1;
    const int64_t Nmol = sys->N / 3;
    // block partials: the pair pass's blocks, then one slot row per finishing block
    NptBuffers& b = ctx->npt;
    const int need = pair_blocks(ctx, sys->N, true) + (int)std::max<int64_t>(1, (Nmol + kWaterThreads - 1) / kWaterThreads);
    if (need > b.partcap) {
        ctx_free(ctx, b.partials);
        b.partials = nullptr;
        b.partcap = 0;
        cudaError_t e = ctx_alloc(ctx, &b.partials, sizeof(double) * kPartStride * (size_t)need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(water partials)");
        b.partcap = need;
    }
    k_water_whole<<<(unsigned)((Nmol + kWaterThreads - 1) / kWaterThreads), kWaterThreads, 0, ctx->stream>>>(
        Nmol, sys->pos, sys->cell);
    if ((st = water_check(ctx, "k_water_whole")) != RBE_OK) return st;
    if ((st = water_forces(ctx, sys, 0)) != RBE_OK) return st;
    ctx->water_ready_N = sys->N;
    return launch_npt_set_step(ctx, sys->cell, sys->step);
}

rbe_status water_run(rbe_ctx ctx, rbe_system* sys, const rbe_water_params* wp, int32_t nsteps)
{
    if (nsteps < 1) return fail(ctx, RBE_EINVAL, "nsteps must be >= 1");
    rbe_status st = water_validate(ctx, sys, wp);
    if (st != RBE_OK) return st;
    if (ctx->water_ready_N != sys->N) return fail(ctx, RBE_ESTATE, "call rbe_water_init for this system first");
    const int64_t Nmol = sys->N / 3;
    const unsigned nbm = (unsigned)((Nmol + kWaterThreads - 1) / kWaterThreads);
    for (int32_t k = 0; k < nsteps; ++k) {
        if ((st = launch_npt_cell_iso(ctx, sys)) != RBE_OK) return st;
        k_water_drift<<<nbm, kWaterThreads, 0, ctx->stream>>>(Nmol, sys->pos, sys->mom, sys->force, sys->mass,
                                                              reinterpret_cast<const NptCoef*>(ctx->npt.coef),
                                                              ctx->seed, sys->cell, *wp, sys->params.dt, ctx->d.status);
        if ((st = water_check(ctx, "k_water_drift")) != RBE_OK) return st;
        if ((st = water_forces(ctx, sys, 1)) != RBE_OK) return st;
        sys->step += 1;
    }
    return RBE_OK;
}

}  // namespace rbe
