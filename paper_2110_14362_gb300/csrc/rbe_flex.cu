// Langevin NPT step of the fully flexible cell on the device (App. A, the fully flexible cells;
// the k-space of App. C in a general cell).  The cell h (cell vectors as columns) moves with nine
// momenta p^h; the particles follow dr/dt = p/m + A r, dp/dt = 100 F - A^T p with A = (dh/dt) h^{-1}.
//
// One step is a fixed sequence of launches on the context's stream:
//   k_flex_cell    one block: V^p/2, V/2, O^p, V/2 of the cell (one lane per entry of the 3x3
//                  matrices), the four sub-step flows e^X and phi(X) (one warp each), the
//                  general-cell quantities of the new cell (h^{-1}, G, the MH proposal lengths
//                  and precisions, S by the dual lattice sum) and the cell-list constants
//   k_flex_drift   particles: R^p/2, R/2, O, R/2, wrap to s in [0, 1), scaled coordinates
//   k-space        proposal tables (device lengths), k_flex_mh, unit-cube tables, rho and force
//                  passes on s, k_flex_kvirial (the full virial from rho)
//   cell list      on s (rbe_npt.cu's count, scan, fill and sort)
//   k_flex_pair    real-space forces, full virial and energies by the minimum image in s
//   k_flex_finish  F = qqr2e h^{-T} F_s + F_r, R^p/2, kinetic tensor; last block: W, V^p/2, H
// The step index lives on the device (cell[50]); nothing leaves the device between steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <type_traits>

#include "rbe_context.h"
#include "rbe_device.cuh"
#include "rbe_general.cuh"
#include "rbe_npt_common.cuh"

namespace rbe {

// slots of the cell block (include/rbe.h)
constexpr int kFxH = 0, kFxPh = 9, kFxW = 18, kFxKt = 27, kFxPt = 36;
constexpr int kFxEk = 45, kFxEc = 46, kFxEl = 47, kFxV = 48, kFxHam = 49, kFxStep = 50;
// rbe_flex_init sizes the tables and the cell list for cell vectors and widths up to this many
// times the initial ones; a cell beyond it is flagged (RBE_ESTATE) by the step.
constexpr double kFlexHeadroom = 2.0;
// The S dual sum runs over n in [-R, R]^3 with R <= kDualMax per axis; a larger R (a cell far
// beyond the prepared range) is flagged instead of summed.
constexpr int kDualMax = 24;

// Sub-step coefficients of one step (written by k_flex_cell).  The flows with A frozen:
// R^p: p <- E p + 100 P F,  R: r <- E r + cap(P p / m), with E = e^X, P = t phi(X), t = dt/2,
// X = -A^T t (R^p) or A t (R).
struct FlexCoef {
    double E[4][9], P[4][9];  // 0: R^p/2 before the forces, 1: first R/2, 2: second R/2, 3: R^p/2 after
    double h[9], hinv[9];     // the cell after the second V/2 and its inverse
    double V;                 // det h
    double g, sog;            // O: p <- g p + sog sqrt(m) z
    double half_cap;          // cap of the peculiar displacement per R/2
    int noise, pad;
};

constexpr int kFxBuilds = 51;  // neighbour-list builds so far (cell block)

// Neighbour-list state of the flexible cell.  The list holds, for every slot of the cell order of
// its build, the slots within rl = rc + skin by the minimum image at the build (rl <= w_j / 2, so
// every other image of a pair is at least rl away too).  Since then the cell has deformed by
// F = h h_ref^{-1} and every particle has moved by at most D (measured with the current h): an
// unlisted pair is now at least sigma_min(F) rl - 2 D >= (1 - |F - I|_F) rl - 2 D apart, and the
// list stands while that is at least rc.
struct FlexNList {
    NListState base;             // rl, rc, the displacement maximum and the rebuild flags (the
                                 // cell-list kernels read base.rebuild)
    double href[9], hrefinv[9];  // the cell at the last build and its inverse
};

// The listed pairs are evaluated in Cartesian coordinates: each particle's unwrapped position
// r_u = h (s + n_wrap) (n_wrap: the lattice vector its s has wrapped by since the build) and, per
// list entry, the image n of the pair at the build (a byte, (n_x + 1) + 3 (n_y + 1) + 9 (n_z + 1)),
// so that the separation is r_u,j - r_u,i + h n with the current h.  Every other image of a listed
// pair was at least rl away at the build, so the bound above keeps it beyond rc as well.
struct FlexListArgs {
    FlexNList* nl;
    int* nbr;              // [slot * cap + k]
    unsigned char* code;   // [slot * cap + k]: image of the entry at the build
    int* nnb;              // per slot
    float4* sref;          // per slot: s at the build
    float4* cpos32;        // per slot: unwrapped Cartesian position and charge (FP32)
    double4_32a* cpos64;   // per slot: the same in FP64 (FP64 path)
    const double* sbuf;    // per particle: s in [0, 1)
    unsigned* status;      // kStatusList on overflow
    double* cell;          // the build count
    int cap;
};

__device__ __forceinline__ int image_code(int nx, int ny, int nz) { return (nx + 1) + 3 * (ny + 1) + 9 * (nz + 1); }

__device__ __forceinline__ uint64_t flex_step(const double* cell)
{
    return (uint64_t)__double_as_longlong(cell[kFxStep]);
}

// 3x3 matrices across the lanes of one warp: lane e < 9 holds entry e = 3a + b (row-major);
// lanes 9..31 mirror lane 8 so that every shuffle stays in range.  All 32 lanes call these.
__device__ __forceinline__ double m_get(double v, int idx) { return __shfl_sync(0xffffffffu, v, idx); }

// (X Y)[a][b]
__device__ __forceinline__ double m_mul(double x, double y, int a, int b)
{
    const double x0 = m_get(x, 3 * a), x1 = m_get(x, 3 * a + 1), x2 = m_get(x, 3 * a + 2);
    const double y0 = m_get(y, b), y1 = m_get(y, 3 + b), y2 = m_get(y, 6 + b);
    return x0 * y0 + x1 * y1 + x2 * y2;
}

__device__ __forceinline__ double m_transpose(double x, int a, int b) { return m_get(x, 3 * b + a); }

// (h^{-1})[a][b] = cof(b, a) / det h, the cofactors with cyclic indices; det on every lane.
__device__ __forceinline__ double m_inv(double h, int a, int b, double& det)
{
    const int a1 = (a + 1) % 3, a2 = (a + 2) % 3, b1 = (b + 1) % 3, b2 = (b + 2) % 3;
    const double num = m_get(h, 3 * b1 + a1) * m_get(h, 3 * b2 + a2) - m_get(h, 3 * b1 + a2) * m_get(h, 3 * b2 + a1);
    det = m_get(h, 0) * m_get(num, 0) + m_get(h, 1) * m_get(num, 3) + m_get(h, 2) * m_get(num, 6);
    return num / det;
}

// 1/k for k = 0..41 (entry 0 unused), rounded once by the compiler: the series below multiply by
// them instead of dividing (an FP64 division is a long instruction sequence on this GPU).
__constant__ double kInvK[42] = {
    0.0,        1.0,        1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,  1.0 / 7,  1.0 / 8,  1.0 / 9,
    1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18, 1.0 / 19,
    1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29,
    1.0 / 30, 1.0 / 31, 1.0 / 32, 1.0 / 33, 1.0 / 34, 1.0 / 35, 1.0 / 36, 1.0 / 37, 1.0 / 38, 1.0 / 39,
    1.0 / 40, 1.0 / 41};

// The biased exponent and leading mantissa bits of |v| (the high word without its sign): ordered
// like |v| to within a factor of 2^(2^-20).
__device__ __forceinline__ int m_mag(double v) { return __double2hiint(v) & 0x7fffffff; }

// e^X and phi(X) = sum_k X^k / (k+1)! by their Taylor series, summed until the largest entry of
// the term is 2^-67 (7e-21) or less of the largest entry of the sum (at most 40 terms).  The
// comparison runs on the exponent bits (integer instructions).
__device__ __forceinline__ void m_exp_phi(double x, int e, int a, int b, double& E, double& Phi)
{
    double term = (e == 0 || e == 4 || e == 8) ? 1.0 : 0.0;
    E = term;
    Phi = term;
    const double x0 = m_get(x, b), x1 = m_get(x, 3 + b), x2 = m_get(x, 6 + b);
    for (int k = 1; k <= 40; ++k) {
        const double t0 = m_get(term, 3 * a), t1 = m_get(term, 3 * a + 1), t2 = m_get(term, 3 * a + 2);
        term = (t0 * x0 + t1 * x1 + t2 * x2) * kInvK[k];
        E += term;
        Phi += term * kInvK[k + 1];
        const int mt = __reduce_max_sync(0xffffffffu, m_mag(term)), me = __reduce_max_sync(0xffffffffu, m_mag(E));
        if (mt < me - (67 << 20)) break;  // the same on every lane
    }
}

// The general-cell quantities of h across the lanes of one warp, each entry with separately
// rounded operations in the order of the host's construction for rbe_kspace_forces_virial_general
// (h^{-1} by cofactors, G = h^{-1} h^{-T}, the Gram matrix of the cell vectors, lambda, the
// proposal lengths and precisions), so that the MH decisions of both paths agree.  Lane e < 9
// writes entry e; lane 0 the scalars.  Returns det h on every lane.
__device__ __forceinline__ double gen_cell_lanes(const double* h, double alpha, int lane, GenCell& g)
{
    // the cofactor numerator of each entry of h^{-1}: h[p] h[q] - h[r] h[s]
    constexpr int kIdx[9][4] = {{4, 8, 5, 7}, {2, 7, 1, 8}, {1, 5, 2, 4}, {5, 6, 3, 8}, {0, 8, 2, 6},
                                {2, 3, 0, 5}, {3, 7, 4, 6}, {1, 6, 0, 7}, {0, 4, 1, 3}};
    const int e = lane < 9 ? lane : 8, i = e / 3, j = e % 3;
    const double num = __dsub_rn(__dmul_rn(h[kIdx[e][0]], h[kIdx[e][1]]), __dmul_rn(h[kIdx[e][2]], h[kIdx[e][3]]));
    const double c00 = m_get(num, 0), c01 = m_get(num, 3), c02 = m_get(num, 6);
    const double det = __dadd_rn(__dadd_rn(__dmul_rn(h[0], c00), __dmul_rn(h[1], c01)), __dmul_rn(h[2], c02));
    const double hi = __ddiv_rn(num, det);
    const double Gij = __dadd_rn(__dadd_rn(__dmul_rn(m_get(hi, 3 * i), m_get(hi, 3 * j)),
                                           __dmul_rn(m_get(hi, 3 * i + 1), m_get(hi, 3 * j + 1))),
                                 __dmul_rn(m_get(hi, 3 * i + 2), m_get(hi, 3 * j + 2)));
    const double gg = __dadd_rn(__dadd_rn(__dmul_rn(h[i], h[j]), __dmul_rn(h[3 + i], h[3 + j])),
                                __dmul_rn(h[6 + i], h[6 + j]));
    // row sums 1 + sum_{k != j} |cos theta_jk| on lanes 0..2 (row j = lane)
    const int r = lane < 3 ? lane : 0;
    const double gjj = m_get(gg, 4 * r);
    double row = 1.0;
    for (int k = 0; k < 3; ++k) {
        const double gjk = m_get(gg, 3 * r + k), gkk = m_get(gg, 4 * k);
        if (k != r) row = __dadd_rn(row, fabs(__ddiv_rn(gjk, __dsqrt_rn(__dmul_rn(gjj, gkk)))));
    }
    double lam = 1.0;
    for (int k = 0; k < 3; ++k) {
        const double rk = m_get(row, k);
        if (rk > lam) lam = rk;
    }
    if (lane < 9) {
        g.hinv[e] = hi;
        g.G[e] = Gij;
    }
    if (lane < 3) {
        const double le = __dsqrt_rn(__dmul_rn(lam, gjj));
        g.leff[lane] = le;
        g.c[lane] = __ddiv_rn(__dmul_rn(kPi, kPi), __dmul_rn(alpha, __dmul_rn(le, le)));
    }
    if (lane == 0) {
        g.co = __ddiv_rn(__dmul_rn(kPi, kPi), alpha);
        g.V = det;
    }
    return det;
}

// ---------------------------------------------------------------------------------
// The cell part of the step.  Stage 0: the cell normals and friction factors.  Stage 1 (warp 0,
// one lane per entry): V^p/2, the rate A, V/2, A, O^p, A, V/2, A, giving the exponents of the
// four flows.  Stage 2: the four e^X, phi(X) (warps 0..3), the general-cell quantities (warp 4),
// the dual lattice sum of S (warps 5..7).  Stage 3: the coefficients, the general cell, the
// cell-list constants in the unit cube of s (n_j = floor(w_j / rc) cells along s_j, w_j =
// 1/|row j of h^{-1}| the distance between the lattice planes, so that a pair within rc lies in
// neighbouring cells; rcell = rc + skin with a neighbour list, whose build searches the cells
// within rc + skin).  With advance = 0 only the quantities of the current cell (the first forces).  A cell that is not invertible, or whose dual sum would leave the prepared range, is
// flagged (kStatusBox) and its step's results are not to be used.
constexpr int kFlexCellWarps = 8;
constexpr int kDualThreads = 3 * 32;  // warps 5..7

__global__ void __launch_bounds__(kFlexCellWarps * 32)
k_flex_cell(double* __restrict__ cell, FlexCoef* __restrict__ cf, GenCell* __restrict__ gc, CellConsts* __restrict__ cc,
            const rbe_flex_params prm, double alpha, int P, uint64_t seed, int cellcap, double rcell, int advance,
            unsigned* __restrict__ status)
{
    __shared__ double sX[4][9], sE[4][9], sP[4][9];
    __shared__ double sh[9], shi[9], sph[9], sz[9];
    __shared__ double sg[4];  // g_h, g, sog, det h
    __shared__ double sS[kDualThreads];
    __shared__ int sR[4];     // dual-sum ranges, [3] = 1 when out of range
    __shared__ GenCell sgc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = lane < 9 ? lane : 8, ea = e / 3, eb = e % 3;
    const uint64_t step = flex_step(cell);
    const double t = 0.5 * prm.dt;
    if (warp == 1 && lane < 3) {
        // the cell normals of counter indices 0, 1, 2 on three lanes: the diagonal entries 0, 4, 8
        // take index 0's z[0..2] (the rectangular cell's slots); the off-diagonal entries
        // 1, 2, 3, 5, 6, 7 take index 1's z[0..3] and index 2's z[0..1]
        double z[4] = {0.0, 0.0, 0.0, 0.0};
        if (advance && prm.noise) npt_normals(seed, 2u, step, (uint32_t)lane, z);
        if (lane == 0) {
            sz[0] = z[0]; sz[4] = z[1]; sz[8] = z[2];
        } else if (lane == 1) {
            sz[1] = z[0]; sz[2] = z[1]; sz[3] = z[2]; sz[5] = z[3];
        } else {
            sz[6] = z[0]; sz[7] = z[1];
        }
    } else if (warp == 2 && lane == 0) {
        sg[0] = exp(-prm.gamma_h * prm.dt);
    } else if (warp == 3 && lane == 0) {
        const double g = exp(-prm.gamma * prm.dt);
        sg[1] = g;
        sg[2] = sqrt(prm.kT * kFConv * (1.0 - g * g));
    }
    __syncthreads();
    if (warp == 0) {
        double h = cell[kFxH + e], ph = cell[kFxPh + e];
        const double M = prm.M[e];
        double det;
        double hi = m_inv(h, ea, eb, det);
        if (advance) {
            const double W = cell[kFxW + e], Kt = cell[kFxKt + e];
            double X = Kt + W;
            if (ea == eb) X -= prm.P_ext * det + prm.chi * prm.kT;
            ph += t * m_mul(X, m_transpose(hi, ea, eb), ea, eb);       // V^p/2
            double A = m_mul(ph / M, hi, ea, eb);
            const double X0 = -m_transpose(A, ea, eb) * t;             // R^p/2
            h += t * ph / M;                                           // V/2
            hi = m_inv(h, ea, eb, det);
            A = m_mul(ph / M, hi, ea, eb);
            const double X1 = A * t;                                   // R/2
            const double gh = sg[0];
            ph *= gh;                                                  // O^p
            if (prm.noise) ph += sqrt(prm.kT * M * (1.0 - gh * gh)) * sz[e];
            A = m_mul(ph / M, hi, ea, eb);
            const double X2 = A * t;                                   // R/2
            h += t * ph / M;                                           // V/2
            hi = m_inv(h, ea, eb, det);
            A = m_mul(ph / M, hi, ea, eb);
            const double X3 = -m_transpose(A, ea, eb) * t;             // R^p/2
            if (lane < 9) {
                sX[0][e] = X0;
                sX[1][e] = X1;
                sX[2][e] = X2;
                sX[3][e] = X3;
            }
        }
        if (lane < 9) {
            sh[e] = h;
            shi[e] = hi;
            sph[e] = ph;
        }
        __syncwarp();
        if (lane == 0) {
            sg[3] = det;
            // dual-sum ranges: alpha |h n|^2 <= 60 ln 2 + 50 needs |n_t| <= sqrt(cut) |row t of h^{-1}|
            const double cut = (60.0 * 0.69314718055994530942 + 50.0) / alpha;
            bool bad = !(det > 0.0) || !isfinite(det);
            for (int r = 0; r < 3; ++r) {
                const double rn = sqrt(shi[3 * r] * shi[3 * r] + shi[3 * r + 1] * shi[3 * r + 1] + shi[3 * r + 2] * shi[3 * r + 2]);
                const double Rd = ceil(sqrt(cut) * rn) + 1.0;
                bad = bad || !(Rd <= (double)kDualMax);
                sR[r] = Rd <= (double)kDualMax ? (int)Rd : 0;
            }
            sR[3] = bad ? 1 : 0;
            if (bad) atomicOr(status, kStatusBox);
        }
    }
    __syncthreads();
    if (warp < 4) {
        if (advance) {
            double E, Phi;
            m_exp_phi(sX[warp][e], e, ea, eb, E, Phi);
            if (lane < 9) {
                sE[warp][e] = E;
                sP[warp][e] = t * Phi;
            }
        }
    } else if (warp == 4) {
        gen_cell_lanes(sh, alpha, lane, sgc);
    } else {
        // S = (alpha/pi)^{3/2} V sum_n exp(-alpha |h n|^2) - 1 (Poisson summation), the n with
        // alpha |h n|^2 <= 60 ln 2 + 50 (the host's rule), fixed-order partial sums
        const int tid = threadIdx.x - 5 * 32;
        double part = 0.0;
        if (!sR[3]) {
            const double cut = (60.0 * 0.69314718055994530942 + 50.0) / alpha;
            const int n0 = 2 * sR[0] + 1, n1 = 2 * sR[1] + 1, n2 = 2 * sR[2] + 1;
            const int total = n0 * n1 * n2;
            for (int idx = tid; idx < total; idx += kDualThreads) {
                const int a = idx % n0 - sR[0], b = (idx / n0) % n1 - sR[1], c = idx / (n0 * n1) - sR[2];
                double x[3];
                for (int r = 0; r < 3; ++r) x[r] = sh[3 * r] * a + sh[3 * r + 1] * b + sh[3 * r + 2] * c;
                const double d2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
                if (d2 <= cut) part += exp(-alpha * d2);
            }
        }
        sS[tid] = part;
    }
    __syncthreads();
    if (warp == 5) {
        // the dual sum: three partials per lane, then a fixed shuffle tree
        double v = sS[lane] + sS[32 + lane] + sS[64 + lane];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) {
            const double ap = alpha / kPi;
            const double S = ap * sqrt(ap) * sgc.V * v - 1.0;
            sgc.S = S;
            sgc.wP = S / (double)(P > 0 ? P : 1);
            if (!(S > 0.0) || !isfinite(S)) atomicOr(status, kStatusBox);
        }
    } else if (warp == 6 && lane < 3) {
        // cell-list constants of the unit cube of s
        const double w = 1.0 / sqrt(shi[3 * lane] * shi[3 * lane] + shi[3 * lane + 1] * shi[3 * lane + 1] +
                                    shi[3 * lane + 2] * shi[3 * lane + 2]);
        cc->L[lane] = 1.0;
        cc->invL[lane] = 1.0;
        cc->Lf[lane] = 1.0f;
        cc->invLf[lane] = 1.0f;
        const int n = cell_dim(w, rcell);
        cc->nc[lane] = n;
        const bool okw = 2.0 * rcell <= w;
        const unsigned m = __ballot_sync(0x7u, okw);
        const int n0 = __shfl_sync(0x7u, n, 0), n1 = __shfl_sync(0x7u, n, 1), n2 = __shfl_sync(0x7u, n, 2);
        if (lane == 0) {
            const int64_t nn = (int64_t)n0 * n1 * n2;
            cc->ncell = nn <= (int64_t)cellcap ? (int)nn : -1;
            cc->ok = cc->ncell >= 0 && m == 0x7u;
            cc->pass64 = 0.f;
        }
    } else if (warp == 7 && lane < 9) {
        cell[kFxH + lane] = sh[lane];
        cell[kFxPh + lane] = sph[lane];
    }
    __syncthreads();
    // stage 3: write the coefficients and the general cell
    const int tid = threadIdx.x;
    if (tid < 36) {
        const int w = tid / 9, x = tid % 9;
        cf->E[w][x] = advance ? sE[w][x] : ((x == 0 || x == 4 || x == 8) ? 1.0 : 0.0);
        cf->P[w][x] = advance ? sP[w][x] : 0.0;
    } else if (tid < 45) {
        cf->h[tid - 36] = sh[tid - 36];
        cf->hinv[tid - 36] = shi[tid - 36];
    } else if (tid == 45) {
        cf->V = sg[3];
        cf->g = sg[1];
        cf->sog = sg[2];
        cf->half_cap = 0.5 * prm.max_disp;
        cf->noise = prm.noise;
        cf->pad = 0;
    } else if (tid == 64) {
        *gc = sgc;
    }
}

__global__ void k_flex_set_step(double* __restrict__ cell, uint64_t step)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) cell[kFxStep] = __longlong_as_double((long long)step);
}

// 1/m and sqrt(m) per particle, once per rbe_flex_init.
__global__ void k_flex_mass(int64_t N, const double* __restrict__ mass, double2* __restrict__ mprop)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) mprop[i] = make_double2(1.0 / mass[i], sqrt(mass[i]));
}

// Scaled coordinates s = h^{-1} r wrapped into [0, 1) (the first forces; positions unchanged).
__global__ void __launch_bounds__(kNptThreads)
k_flex_scale(int64_t N, const double* __restrict__ pos, const FlexCoef* __restrict__ cf, double* __restrict__ sbuf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double* hi = cf->hinv;
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    for (int a = 0; a < 3; ++a) {
        const double sa = hi[3 * a] * x + hi[3 * a + 1] * y + hi[3 * a + 2] * z;
        sbuf[3 * i + a] = sa - floor(sa);
    }
}

// y = M v for a row-major 3x3 M
__device__ __forceinline__ void mat3_vec(const double* __restrict__ M, const double v[3], double y[3])
{
    for (int a = 0; a < 3; ++a) y[a] = M[3 * a] * v[0] + M[3 * a + 1] * v[1] + M[3 * a + 2] * v[2];
}

// r <- E r + d, with |d| capped at cap (cap > 0): the cap holds the peculiar part d = t phi(A t)
// p/m, not the cell's deformation of r.
__device__ __forceinline__ void flex_drift_add(double r[3], const double* __restrict__ E, double d[3], double cap)
{
    if (cap > 0.0) {
        const double l2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (l2 > cap * cap) {
            const double f = cap / sqrt(l2);
            d[0] *= f; d[1] *= f; d[2] *= f;
        }
    }
    double er[3];
    mat3_vec(E, r, er);
    for (int a = 0; a < 3; ++a) r[a] = er[a] + d[a];
}

// Particles before the forces: R^p/2, R/2, O, R/2, wrap to s in [0, 1); writes r, p and s.
// kF32Noise: the Langevin normals in FP32 arithmetic (FP32-phase path).
template <bool kF32Noise>
__global__ void __launch_bounds__(kNptThreads)
k_flex_drift(int64_t N, double* __restrict__ pos, double* __restrict__ mom, const double* __restrict__ force,
             const double2* __restrict__ mprop, const FlexCoef* __restrict__ cf, uint64_t seed,
             const double* __restrict__ cell, double* __restrict__ sbuf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint64_t step = flex_step(cell);
    const double2 mp = mprop[i];  // (1/m, sqrt(m))
    double r[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    double p[3] = {mom[3 * i], mom[3 * i + 1], mom[3 * i + 2]};
    const double F[3] = {force[3 * i], force[3 * i + 1], force[3 * i + 2]};
    double u[3], v[3], d[3];
    mat3_vec(cf->E[0], p, u);  // R^p/2
    mat3_vec(cf->P[0], F, v);
    for (int a = 0; a < 3; ++a) p[a] = u[a] + kFConv * v[a];
    mat3_vec(cf->P[1], p, d);  // R/2
    for (int a = 0; a < 3; ++a) d[a] *= mp.x;
    flex_drift_add(r, cf->E[1], d, cf->half_cap);
    double z[4] = {0.0, 0.0, 0.0, 0.0};  // O
    if (cf->noise) {
        if (kF32Noise) npt_normals_f32(seed, 1u, step, (uint32_t)i, z);
        else npt_normals(seed, 1u, step, (uint32_t)i, z);
    }
    const double sg = cf->sog * mp.y, g = cf->g;
    for (int a = 0; a < 3; ++a) p[a] = p[a] * g + sg * z[a];
    mat3_vec(cf->P[2], p, d);  // R/2
    for (int a = 0; a < 3; ++a) d[a] *= mp.x;
    flex_drift_add(r, cf->E[2], d, cf->half_cap);
    double sc[3];
    mat3_vec(cf->hinv, r, sc);
    for (int a = 0; a < 3; ++a) sc[a] -= floor(sc[a]);
    mat3_vec(cf->h, sc, r);
    for (int a = 0; a < 3; ++a) {
        pos[3 * i + a] = r[a];
        mom[3 * i + a] = p[a];
        sbuf[3 * i + a] = sc[a];
    }
}

// One MH step per frequency slot with the device's general cell and step index.
__global__ void k_flex_mh(uint64_t seed, const double* __restrict__ cell, int P,
                          const unsigned long long* __restrict__ cum, int cap, const KState* __restrict__ ks,
                          int4* __restrict__ chain, const GenCell* __restrict__ gc, int4* __restrict__ m_out,
                          double* __restrict__ w_out, unsigned* __restrict__ status)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= P) return;
    const GenCell g = *gc;
    gen_mh_slot(l, seed, flex_step(cell), cum, cap, ks, chain, g, m_out, w_out, status);
}

// The k-space virial tensor from rho with the device's general cell.
__global__ void __launch_bounds__(kGenVirThreads)
k_flex_kvirial(int P, const int4* __restrict__ m, const double2* __restrict__ rho, const GenCell* __restrict__ gc,
               double alpha, double* __restrict__ W_out, unsigned* __restrict__ status)
{
    __shared__ GenCell g;
    if (threadIdx.x == 0) g = *gc;
    __syncthreads();
    gen_virial_block(P, m, rho, g, alpha, W_out, status);
}

// Per step with a neighbour list, before the cell list: the unwrapped Cartesian positions and
// charges packed in the list's slot order, the largest displacement since the build (length with
// the current h, FP32), and on the last block the rebuild decision.  Until the first build
// there is no slot order: the kernel then only asks for a build.
template <bool kF64>
__global__ void __launch_bounds__(kNptThreads)
k_flex_nl_check(int64_t N, const double* __restrict__ sbuf, const double* __restrict__ q,
                const int* __restrict__ sorted, float4* __restrict__ cpos32, double4_32a* __restrict__ cpos64,
                const float4* __restrict__ sref, const FlexCoef* __restrict__ cf, FlexNList* __restrict__ nl)
{
    __shared__ float smax[kNptThreads / 32];
    __shared__ bool last;
    const bool force = nl->base.force != 0;
    float d2max = 0.f;
    if (!force) {
        double h[9];
        float hf[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            h[a] = cf->h[a];
            hf[a] = (float)h[a];
        }
        for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < N; u += (int64_t)gridDim.x * blockDim.x) {
            const int64_t i = sorted[u];
            const float4 r0 = sref[u];
            // s unwrapped since the build: s + n_wrap, n_wrap = -rint(s - s_ref)
            double su[3] = {sbuf[3 * i], sbuf[3 * i + 1], sbuf[3 * i + 2]};
            su[0] -= rint(su[0] - (double)r0.x);
            su[1] -= rint(su[1] - (double)r0.y);
            su[2] -= rint(su[2] - (double)r0.z);
            const double qq = q[i];
            double r[3];
            for (int a = 0; a < 3; ++a) r[a] = h[3 * a] * su[0] + h[3 * a + 1] * su[1] + h[3 * a + 2] * su[2];
            cpos32[u] = make_float4((float)r[0], (float)r[1], (float)r[2], (float)qq);
            if (kF64) {
                double4_32a v;
                v.x = r[0];
                v.y = r[1];
                v.z = r[2];
                v.w = qq;
                cpos64[u] = v;
            }
            const float a = (float)su[0] - r0.x, b = (float)su[1] - r0.y, c = (float)su[2] - r0.z;
            const float dx = hf[0] * a + hf[1] * b + hf[2] * c, dy = hf[3] * a + hf[4] * b + hf[5] * c,
                        dz = hf[6] * a + hf[7] * b + hf[8] * c;
            const float d2 = dx * dx + dy * dy + dz * dz;
            d2max = d2 > d2max ? d2 : d2max;  // NaN compares false: caught by the cell checks
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
        atomicMax(&nl->base.maxd2, __float_as_uint(m));
        __threadfence();
        last = atomicAdd(&nl->base.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || warp != 0) return;
    __threadfence();
    // warp 0 of the last block: F = h h_ref^{-1} one entry per lane, |F - I|_F by a shuffle sum
    const int e = lane < 9 ? lane : 8, ea = e / 3, eb = e % 3;
    const double F = m_mul(cf->h[e], nl->hrefinv[e], ea, eb);
    double d = lane < 9 ? F - (ea == eb ? 1.0 : 0.0) : 0.0;
    d *= d;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    if (lane == 0) {
        const double D = sqrt((double)__uint_as_float(atomicAdd(&nl->base.maxd2, 0u)));
        const double f = 1.0 - sqrt(d);
        // a margin of 1e-3 A covers the FP32 rounding of the displacements
        const bool stands = !force && f * ((double)nl->base.rl) - 2.0 * D - 1e-3 >= (double)nl->base.rc;
        nl->base.rebuild = stands ? 0 : 1;
        nl->base.maxd2 = 0u;
        nl->base.counter = 0u;
    }
}

__global__ void k_flex_nl_init(FlexNList* __restrict__ nl, float rl, float rc, double* __restrict__ cell)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int a = 0; a < 3; ++a) nl->base.Lref[a] = 1.0;
    nl->base.rl = rl;
    nl->base.rc = rc;
    nl->base.maxd2 = 0u;
    nl->base.counter = 0u;
    nl->base.rebuild = 1;
    nl->base.force = 1;
    for (int a = 0; a < 9; ++a) {
        nl->href[a] = (a % 4 == 0) ? 1.0 : 0.0;
        nl->hrefinv[a] = (a % 4 == 0) ? 1.0 : 0.0;
    }
    cell[kFxBuilds] = 0.0;
}

// ---------------------------------------------------------------------------------
// Real space in the general cell (Sec. 4.1 Eqs. (U2), (force)): one warp per particle in cell
// order, the 3 x 3 rows of neighbouring cells of the cell list in s (the cells cx-1..cx+1 of a
// row are contiguous slots, split in two where the row wraps; an axis with fewer than 3 cells
// visits each of its cells once).  A pair's separation is the minimum image in s, d = h (s_j -
// s_i - rint(s_j - s_i)): with rc <= w_j / 2 on every axis the image within rc, if any, is
// that one (|b_j . d| <= rc / w_j <= 1/2 for the reciprocal rows b_j of h^{-1}).  Hits within rc
// are buffered per warp (ballot order) and evaluated 32 at a time, one per lane; the lane sums
// go through a fixed shuffle tree.  FP64 path: everything in FP64; FP32 path: FP32 search and
// evaluation, float-float sums per warp.  Each pair is visited from both ends: energies and
// the virial take half.  Per-block partials {W_xx, W_yy, W_zz, W_xy, W_xz, W_yz, E_coul, E_lj}
// at slots 0..7.  A cell beyond the cell arrays (flagged by k_cl_count) leaves F_r = 0.
constexpr int kFlexHitCap = 32 * (kListBatch + 1);  // < 32 buffered + 32 kListBatch new (the list pass)

// Modes as the rectangular kernel's: search the cells and evaluate, search the cells within
// rc + skin and write the list (rebuild steps only), evaluate the listed pairs.
template <bool kF64, int kMode>
__global__ void __launch_bounds__(kPairWarps * 32, kF64 ? kPairBlocksPerSM64 : (kMode == 2 ? kPairBlocksPerSM : 3))
k_flex_pair(int64_t N, const CellConsts* __restrict__ cc, const PairConst pc, const FlexCoef* __restrict__ cf,
            const int* __restrict__ cid, const int* __restrict__ cnt, const int* __restrict__ start,
            const int* __restrict__ sorted, const float4* __restrict__ spos32, const double4_32a* __restrict__ spos64,
            double* __restrict__ Fr, double* __restrict__ partials, const FlexListArgs la)
{
    constexpr bool kBuild = kMode == 1, kList = kMode == 2;
    if (kBuild && !la.nl->base.rebuild) return;  // the list stands (the same for every thread)
    using R = typename std::conditional<kF64, double, float>::type;
    struct Hit {
        R x, y, z, q;
    };
    __shared__ Hit hits[kPairWarps][kFlexHitCap];
    __shared__ double red[8][kPairWarps];
    __shared__ R shm[9];
    __shared__ R sshift[27][3];  // list: the images h n, n in {-1, 0, 1}^3, by code
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (threadIdx.x < 9) shm[threadIdx.x] = (R)cf->h[threadIdx.x];
    if (kList && threadIdx.x >= 32 && threadIdx.x < 32 + 27) {
        const int c = threadIdx.x - 32;
        const double n[3] = {(double)(c % 3 - 1), (double)((c / 3) % 3 - 1), (double)(c / 9 - 1)};
        for (int a = 0; a < 3; ++a) sshift[c][a] = (R)(cf->h[3 * a] * n[0] + cf->h[3 * a + 1] * n[1] + cf->h[3 * a + 2] * n[2]);
    }
    __syncthreads();
    const int nc[3] = {cc->nc[0], cc->nc[1], cc->nc[2]};
    double ws[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, ecsum = 0.0, elsum = 0.0;  // FP64 path
    float wh[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, wl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // FP32 path
    float ech = 0.f, ecl = 0.f, elh = 0.f, ell = 0.f;
    // no cell list this step (a cell beyond the cell arrays, flagged), or no list built yet
    const bool cells_ok = kList ? la.nl->base.force == 0 : cc->ncell >= 0;
    if (!cells_ok) {
        if (!kBuild)
            for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < 3 * N;
                 j += (int64_t)gridDim.x * blockDim.x)
                Fr[j] = 0.0;
    } else {
        R h[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) h[a] = shm[a];
        R rc2, sa, aR, two_sa_pi, qk, s2, e4, e24;
        if constexpr (kF64) {
            rc2 = pc.rc2, sa = pc.sa, aR = pc.a, two_sa_pi = pc.two_sa_pi;
            qk = pc.qk, s2 = pc.s2, e4 = pc.e4, e24 = pc.e24;
        } else {
            rc2 = pc.rc2f, sa = pc.saf, aR = pc.af, two_sa_pi = pc.two_sa_pif;
            qk = pc.qkf, s2 = pc.s2f, e4 = pc.e4f, e24 = pc.e24f;
        }
        const bool lj = pc.lj != 0;
        // the build keeps every candidate within rl plus a margin above the rounding of a
        // distance (a superset is harmless)
        const R search2 = kBuild ? (R)((double)la.nl->base.rl * (double)la.nl->base.rl * (1.0 + 1e-5)) : rc2;
        const int nwarps = gridDim.x * kPairWarps;
        for (int u = blockIdx.x * kPairWarps + wib; u < (int)N; u += nwarps) {
            const int i = sorted[u];
            R si[3], qi;  // cells and build: s; list: the unwrapped Cartesian position
            if constexpr (kF64) {
                const double4_32a m64 = kList ? la.cpos64[u] : spos64[u];
                si[0] = m64.x, si[1] = m64.y, si[2] = m64.z, qi = m64.w;
            } else {
                const float4 m32 = kList ? la.cpos32[u] : spos32[u];
                si[0] = m32.x, si[1] = m32.y, si[2] = m32.z, qi = m32.w;
            }
            // segment of this lane: row r = lane / 2 of the 3 x 3 rows, part lane % 2
            int lo = 0, hi = 0;
            if (!kList) {
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
                    int a = -1, b = -1;  // cells a..b of the row
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
            R fx = 0, fy = 0, fz = 0, ec = 0, el = 0;
            R w[6] = {0, 0, 0, 0, 0, 0};  // xx, yy, zz, xy, xz, yz
            int nh = 0;
            auto evaluate = [&](int count, int base) {
                if (lane >= count) return;
                const Hit ht = hits[wib][base + lane];
                const R dx = ht.x, dy = ht.y, dz = ht.z, qj = ht.q;
                const R r2 = dx * dx + dy * dy + dz * dz;
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
                const R coul = qk * qi * qj * inv_r;
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
                fx -= f * dx;
                fy -= f * dy;
                fz -= f * dz;
                w[0] += f * dx * dx;
                w[1] += f * dy * dy;
                w[2] += f * dz * dz;
                w[3] += f * dx * dy;
                w[4] += f * dx * dz;
                w[5] += f * dy * dz;
            };
            // one candidate slot sj per lane (valid: a candidate at all): its separation by the
            // minimum image in s; hits go to the buffer (build: to the list)
            auto consider = [&](bool valid, int sj) {
                R ds[3], qj;
                if constexpr (kF64) {
                    const double4_32a o = spos64[sj];
                    ds[0] = o.x - si[0], ds[1] = o.y - si[1], ds[2] = o.z - si[2], qj = o.w;
                } else {
                    const float4 o = spos32[sj];
                    ds[0] = o.x - si[0], ds[1] = o.y - si[1], ds[2] = o.z - si[2], qj = o.w;
                }
                R n[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    n[a] = rint(ds[a]);
                    ds[a] -= n[a];
                }
                const R dx = h[0] * ds[0] + h[1] * ds[1] + h[2] * ds[2];
                const R dy = h[3] * ds[0] + h[4] * ds[1] + h[5] * ds[2];
                const R dz = h[6] * ds[0] + h[7] * ds[1] + h[8] * ds[2];
                const bool hit = valid && dx * dx + dy * dy + dz * dz < search2;
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if constexpr (kBuild) {
                    if (hit) {
                        const int p = nh + __popc(m & ((1u << lane) - 1u));
                        if (p < la.cap) {
                            la.nbr[(int64_t)u * la.cap + p] = sj;
                            // the image added to s_j - s_i is -n
                            la.code[(int64_t)u * la.cap + p] = (unsigned char)image_code(-(int)n[0], -(int)n[1], -(int)n[2]);
                        }
                    }
                    nh += __popc(m);
                    return;
                }
                if (hit) {
                    const int slot = nh + __popc(m & ((1u << lane) - 1u));
                    hits[wib][slot] = Hit{dx, dy, dz, qj};
                }
                nh += __popc(m);
                if (nh >= 32) {
                    __syncwarp();
                    evaluate(32, 0);
                    __syncwarp();
                    if (lane < nh - 32) hits[wib][lane] = hits[wib][32 + lane];
                    __syncwarp();
                    nh -= 32;
                }
            };
            if constexpr (kList) {
                // the listed entries: r_u,j - r_u,i + h n (the build's image)
                const int nn = la.nnb[u];
                const int* row = la.nbr + (int64_t)u * la.cap;
                const unsigned char* crow = la.code + (int64_t)u * la.cap;
                // kListBatch x 32 entries at a time: all their list entries and images are loaded,
                // then all their positions, so that the loads overlap; then the compaction
                for (int k0 = 0; k0 < nn; k0 += 32 * kListBatch) {  // the same trip count on every lane
                    int sj[kListBatch], cd[kListBatch];
#pragma unroll
                    for (int a = 0; a < kListBatch; ++a) {
                        const int k = k0 + 32 * a + lane;
                        const int kk = k < nn ? k : nn - 1;
                        sj[a] = row[kk];
                        cd[a] = crow[kk];
                    }
                    R ox[kListBatch], oy[kListBatch], oz[kListBatch], oq[kListBatch];
#pragma unroll
                    for (int a = 0; a < kListBatch; ++a) {
                        if constexpr (kF64) {
                            const double4_32a o = la.cpos64[sj[a]];
                            ox[a] = o.x, oy[a] = o.y, oz[a] = o.z, oq[a] = o.w;
                        } else {
                            const float4 o = la.cpos32[sj[a]];
                            ox[a] = o.x, oy[a] = o.y, oz[a] = o.z, oq[a] = o.w;
                        }
                    }
#pragma unroll
                    for (int a = 0; a < kListBatch; ++a) {
                        const int k = k0 + 32 * a + lane;
                        const R dx = (ox[a] - si[0]) + sshift[cd[a]][0], dy = (oy[a] - si[1]) + sshift[cd[a]][1],
                                dz = (oz[a] - si[2]) + sshift[cd[a]][2];
                        const bool hit = k < nn && dx * dx + dy * dy + dz * dz < rc2;
                        const unsigned m = __ballot_sync(0xffffffffu, hit);
                        if (hit) {
                            const int slot = nh + __popc(m & ((1u << lane) - 1u));
                            hits[wib][slot] = Hit{dx, dy, dz, oq[a]};
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
                for (int g = 0; g < 18; ++g) {
                    const int glo = __shfl_sync(0xffffffffu, lo, g), ghi = __shfl_sync(0xffffffffu, hi, g);
                    for (int s0 = glo; s0 < ghi; s0 += 32) {  // the same trip count on every lane
                        const int sl = s0 + lane;
                        consider(sl < ghi && sl != u, sl < ghi ? sl : glo);
                    }
                }
            }
            if constexpr (kBuild) {
                if (lane == 0) {
                    la.nnb[u] = nh < la.cap ? nh : la.cap;
                    la.sref[u] = make_float4((float)si[0], (float)si[1], (float)si[2], 0.f);
                    if (nh > la.cap) atomicOr(la.status, kStatusList);
                } else if (lane == 1) {
                    // the slot's Cartesian position at the build (no wraps yet) for the list pass
                    const double s0 = la.sbuf[3 * (int64_t)i], s1 = la.sbuf[3 * (int64_t)i + 1], s2 = la.sbuf[3 * (int64_t)i + 2];
                    double r[3];
                    for (int a = 0; a < 3; ++a) r[a] = cf->h[3 * a] * s0 + cf->h[3 * a + 1] * s1 + cf->h[3 * a + 2] * s2;
                    la.cpos32[u] = make_float4((float)r[0], (float)r[1], (float)r[2], (float)qi);
                    if (kF64) {
                        double4_32a v;
                        v.x = r[0];
                        v.y = r[1];
                        v.z = r[2];
                        v.w = qi;
                        la.cpos64[u] = v;
                    }
                }
                continue;
            }
            __syncwarp();
            evaluate(nh, 0);
            __syncwarp();
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                fx += __shfl_xor_sync(0xffffffffu, fx, off);
                fy += __shfl_xor_sync(0xffffffffu, fy, off);
                fz += __shfl_xor_sync(0xffffffffu, fz, off);
#pragma unroll
                for (int a = 0; a < 6; ++a) w[a] += __shfl_xor_sync(0xffffffffu, w[a], off);
                ec += __shfl_xor_sync(0xffffffffu, ec, off);
                el += __shfl_xor_sync(0xffffffffu, el, off);
            }
            if (lane == 0) {
                if constexpr (kF64) {
                    Fr[3 * (int64_t)i] = fx;
                    Fr[3 * (int64_t)i + 1] = fy;
                    Fr[3 * (int64_t)i + 2] = fz;
#pragma unroll
                    for (int a = 0; a < 6; ++a) ws[a] += 0.5 * w[a];
                    ecsum += 0.5 * ec;
                    elsum += 0.5 * el;
                } else {
                    unsigned long long* Fb = reinterpret_cast<unsigned long long*>(Fr);
                    Fb[3 * (int64_t)i] = float_to_double_bits(__float_as_uint(fx));
                    Fb[3 * (int64_t)i + 1] = float_to_double_bits(__float_as_uint(fy));
                    Fb[3 * (int64_t)i + 2] = float_to_double_bits(__float_as_uint(fz));
#pragma unroll
                    for (int a = 0; a < 6; ++a) ff_add(wh[a], wl[a], 0.5f * w[a]);
                    ff_add(ech, ecl, 0.5f * ec);
                    ff_add(elh, ell, 0.5f * el);
                }
            }
        }
    }
    if constexpr (kBuild) {
        // the build's cell; the list now stands until a check says otherwise (a build without a
        // cell list leaves the list pending)
        if (cells_ok && blockIdx.x == 0) {
            if (threadIdx.x < 9) {
                la.nl->href[threadIdx.x] = cf->h[threadIdx.x];
                la.nl->hrefinv[threadIdx.x] = cf->hinv[threadIdx.x];
            } else if (threadIdx.x == 32) {
                la.nl->base.force = 0;
                la.cell[kFxBuilds] += 1.0;
            }
        }
        return;
    }
    if (lane == 0) {
        if (!kF64) {
#pragma unroll
            for (int a = 0; a < 6; ++a) ws[a] = (double)wh[a] + (double)wl[a];
            ecsum = (double)ech + (double)ecl;
            elsum = (double)elh + (double)ell;
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) red[a][wib] = ws[a];
        red[6][wib] = ecsum;
        red[7][wib] = elsum;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double t = 0.0;
        for (int wv = 0; wv < kPairWarps; ++wv) t += red[threadIdx.x][wv];
        partials[kPartStride * (size_t)blockIdx.x + threadIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------------
// Forces F = qqr2e h^{-T} F_s + F_r (F_s the k-space force in s); with do_kick, R^p/2 with the
// fourth flow; the kinetic tensor per block.  The last block sums the partials in a fixed order
// and, on warp 0 (one lane per entry), forms W = qqr2e W_k + W_r, with do_kick V^p/2 of p^h, the
// pressure tensor and H; with do_kick it advances the step index.
__global__ void __launch_bounds__(kNptThreads)
k_flex_finish(int64_t N, double* __restrict__ mom, double* __restrict__ force, const double2* __restrict__ mprop,
              const double* __restrict__ Fk, const double* __restrict__ Fr, const double* __restrict__ WEk,
              const FlexCoef* __restrict__ cf, double* __restrict__ partials, int nblocks_pair,
              unsigned* __restrict__ counter, double* __restrict__ cell, const rbe_flex_params prm, int do_kick,
              unsigned* __restrict__ status)
{
    __shared__ double red[6][kNptThreads / 32];
    __shared__ bool is_last;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double kt[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (i < N) {
        const double inv_m = mprop[i].x;
        double F[3] = {0.0, 0.0, 0.0};
        if (prm.kspace) {
            const double* hi = cf->hinv;
            const double a = Fk[3 * i], b = Fk[3 * i + 1], c = Fk[3 * i + 2];
            for (int t = 0; t < 3; ++t) F[t] = prm.qqr2e * (hi[t] * a + hi[3 + t] * b + hi[6 + t] * c);
        }
        if (prm.real)
            for (int t = 0; t < 3; ++t) F[t] += Fr[3 * i + t];
        double p[3] = {mom[3 * i], mom[3 * i + 1], mom[3 * i + 2]};
        if (do_kick) {
            double u[3], v[3];
            mat3_vec(cf->E[3], p, u);
            mat3_vec(cf->P[3], F, v);
            for (int t = 0; t < 3; ++t) p[t] = u[t] + kFConv * v[t];
            for (int t = 0; t < 3; ++t) mom[3 * i + t] = p[t];
        }
        for (int t = 0; t < 3; ++t) force[3 * i + t] = F[t];
        const double s = inv_m * (1.0 / kFConv);
        kt[0] = p[0] * p[0] * s;
        kt[1] = p[1] * p[1] * s;
        kt[2] = p[2] * p[2] * s;
        kt[3] = p[0] * p[1] * s;
        kt[4] = p[0] * p[2] * s;
        kt[5] = p[1] * p[2] * s;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int a = 0; a < 6; ++a) kt[a] += __shfl_xor_sync(0xffffffffu, kt[a], off);
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < 6; ++a) red[a][warp] = kt[a];
    __syncthreads();
    if (threadIdx.x < 6) {
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
    // thread t sums the partials t, t + 256, ...; a fixed shared-memory tree combines them:
    // fin[0..5] the kinetic tensor, fin[6..13] the pair sums
    __shared__ double fin[14][kNptThreads];
    {
        double v[14];
#pragma unroll
        for (int a = 0; a < 14; ++a) v[a] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += kNptThreads)
#pragma unroll
            for (int a = 0; a < 6; ++a) v[a] += __ldcg(partials + kPartStride * (size_t)(nblocks_pair + b) + a);
        if (prm.real)
            for (int b = threadIdx.x; b < nblocks_pair; b += kNptThreads)
#pragma unroll
                for (int a = 0; a < 8; ++a) v[6 + a] += __ldcg(partials + kPartStride * (size_t)b + a);
#pragma unroll
        for (int a = 0; a < 14; ++a) fin[a][threadIdx.x] = v[a];
    }
    __syncthreads();
    for (int half = kNptThreads / 2; half > 0; half >>= 1) {
        if (threadIdx.x < half)
#pragma unroll
            for (int a = 0; a < 14; ++a) fin[a][threadIdx.x] += fin[a][threadIdx.x + half];
        __syncthreads();
    }
    if (warp != 0) return;
    constexpr int kSym[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};  // entry (a, b) -> {xx, yy, zz, xy, xz, yz}
    const int e = lane < 9 ? lane : 8, ea = e / 3, eb = e % 3;
    const double Kt = fin[kSym[e]][0];
    const double Wr = prm.real ? fin[6 + kSym[e]][0] : 0.0;
    const double W = (prm.kspace ? prm.qqr2e * __ldcg(WEk + e) : 0.0) + Wr;
    const double V = cf->V;
    double ph = cell[kFxPh + e];
    if (do_kick) {
        double X = Kt + W;
        if (ea == eb) X -= prm.P_ext * V + prm.chi * prm.kT;
        ph += 0.5 * prm.dt * m_mul(X, m_transpose(cf->hinv[e], ea, eb), ea, eb);
    }
    // sum over the nine entries of (p^h)^2 / 2M (lanes 9..31 add nothing)
    double pe = lane < 9 ? ph * ph / (2.0 * prm.M[e]) : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) pe += __shfl_xor_sync(0xffffffffu, pe, off);
    const double Pt = (Kt + W) / V;
    if (lane < 9) {
        cell[kFxPh + e] = ph;
        cell[kFxW + e] = W;
        cell[kFxKt + e] = Kt;
        cell[kFxPt + e] = Pt;
    }
    const bool bad = lane < 9 && (!isfinite(ph) || !isfinite(Pt));
    const unsigned anybad = __ballot_sync(0xffffffffu, bad);
    if (lane == 0) {
        const double Ek = prm.kspace ? prm.qqr2e * (__ldcg(WEk + 9) + __ldcg(WEk + 10)) : 0.0;
        const double Ec = prm.real ? fin[12][0] : 0.0, El = prm.real ? fin[13][0] : 0.0;
        const double K = 0.5 * (fin[0][0] + fin[1][0] + fin[2][0]);
        const double H = K + Ek + Ec + El + prm.P_ext * V + prm.chi * prm.kT * log(V) + pe;
        cell[kFxEk] = Ek;
        cell[kFxEc] = Ec;
        cell[kFxEl] = El;
        cell[kFxV] = V;
        cell[kFxHam] = H;
        if (do_kick) cell[kFxStep] = __longlong_as_double((long long)(flex_step(cell) + 1));
        if (anybad || !isfinite(H)) atomicOr(status, kStatusNonFinite);
        *counter = 0u;
    }
}

// ---------------------------------------------------------------------------------
// Host side.

static rbe_status flex_check(rbe_ctx ctx, const char* what)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RBE_OK : cuda_fail(ctx, e, what);
}

static rbe_status flex_validate(rbe_ctx ctx, const rbe_flex_system* sys)
{
    if (!sys) return fail(ctx, RBE_EINVAL, "system is NULL");
    const rbe_flex_params& p = sys->params;
    if (sys->N < 1 || sys->N > ((int64_t)1 << 31) - 256) return fail(ctx, RBE_EINVAL, "N out of range");
    if (!sys->pos || !sys->mom || !sys->force || !sys->charge || !sys->mass || !sys->cell)
        return fail(ctx, RBE_EINVAL, "system buffers must not be NULL");
    if (!(p.dt > 0.0) || !std::isfinite(p.dt) || !(p.kT >= 0.0) || !std::isfinite(p.kT) || !(p.gamma >= 0.0) ||
        !std::isfinite(p.gamma) || !(p.gamma_h >= 0.0) || !std::isfinite(p.gamma_h) || !std::isfinite(p.P_ext) ||
        !(p.rc > 0.0) || !std::isfinite(p.rc) || !(p.max_disp >= 0.0) || !std::isfinite(p.chi) ||
        !std::isfinite(p.qqr2e) || !std::isfinite(p.lj_sigma) || !std::isfinite(p.lj_eps) || !(p.skin >= 0.0) ||
        !std::isfinite(p.skin))
        return fail(ctx, RBE_EINVAL, "invalid flexible-cell parameters");
    for (int a = 0; a < 9; ++a)
        if (!(p.M[a] > 0.0) || !std::isfinite(p.M[a])) return fail(ctx, RBE_EINVAL, "cell masses must be positive and finite");
    if ((sys->step >> 56) != 0) return fail(ctx, RBE_EINVAL, "step must be < 2^56");
    return RBE_OK;
}

// The host's view of a cell: det h > 0, the lengths |a_j| and the widths w_j = 1/|row j of h^{-1}|.
static bool flex_cell_geometry(const double h[9], double len[3], double width[3])
{
    for (int a = 0; a < 9; ++a)
        if (!std::isfinite(h[a])) return false;
    const double c00 = h[4] * h[8] - h[5] * h[7], c01 = h[5] * h[6] - h[3] * h[8], c02 = h[3] * h[7] - h[4] * h[6];
    const double det = h[0] * c00 + h[1] * c01 + h[2] * c02;
    if (!(det > 0.0) || !std::isfinite(det)) return false;
    // |row j of h^{-1}| = |a_k x a_l| / det with (j, k, l) cyclic
    for (int j = 0; j < 3; ++j) {
        const int k = (j + 1) % 3, l = (j + 2) % 3;
        const double ak[3] = {h[k], h[3 + k], h[6 + k]}, al[3] = {h[l], h[3 + l], h[6 + l]};
        const double cx = ak[1] * al[2] - ak[2] * al[1], cy = ak[2] * al[0] - ak[0] * al[2],
                     cz = ak[0] * al[1] - ak[1] * al[0];
        width[j] = det / std::sqrt(cx * cx + cy * cy + cz * cz);
        len[j] = std::sqrt(h[j] * h[j] + h[3 + j] * h[3 + j] + h[6 + j] * h[6 + j]);
        if (!(width[j] > 0.0) || !std::isfinite(width[j])) return false;
    }
    return true;
}

// Forces, virial tensor and energies at the current state (the batch is the device step
// index), then the finishing kernel.
static rbe_status flex_forces(rbe_ctx ctx, rbe_flex_system* sys, int do_kick)
{
    NptBuffers& b = ctx->npt;
    const rbe_flex_params& prm = sys->params;
    cudaStream_t s = ctx->stream;
    const int64_t N = sys->N;
    const int nb = (int)((N + kNptThreads - 1) / kNptThreads);
    const bool fp64 = ctx->precision == RBE_FP64;
    const int nbp = pair_blocks(ctx, N, fp64);
    const FlexCoef* cf = static_cast<const FlexCoef*>(ctx->flex_coef);
    const GenCell* gc = static_cast<const GenCell*>(ctx->gcell_dev);
    int nbp_eval = nbp;  // blocks of the evaluating pair launch (their partials)
    rbe_status st;
    if (prm.kspace) {
        const int P = ctx->P;
        // proposal tables of the device's lengths, one MH step per slot, the unit cube's tables
        const double* leff = reinterpret_cast<const double*>(reinterpret_cast<const char*>(gc) + offsetof(GenCell, leff));
        if ((st = launch_tables(ctx, leff)) != RBE_OK) return st;
        ctx->tables_dirty = true;
        if (P > 0)
            k_flex_mh<<<(P + 127) / 128, 128, 0, s>>>(ctx->seed, sys->cell, P, ctx->d.cum, ctx->d.tab_cap, ctx->d.ks,
                                                      ctx->gchain, gc, ctx->d.m, ctx->d.w, ctx->d.status);
        if ((st = flex_check(ctx, "k_flex_mh")) != RBE_OK) return st;
        const double unit[3] = {1.0, 1.0, 1.0};
        if ((st = launch_tables_box(ctx, unit)) != RBE_OK) return st;
        if ((st = launch_evaluate(ctx, N, ctx->gpos, sys->charge, P, false, b.Fk, nullptr, b.WEk + 9)) != RBE_OK)
            return st;
        k_flex_kvirial<<<1, kGenVirThreads, 0, s>>>(P, ctx->d.m, ctx->d.rho, gc, ctx->alpha, b.WEk, ctx->d.status);
        if ((st = flex_check(ctx, "k_flex_kvirial")) != RBE_OK) return st;
    }
    if (prm.real) {
        if (fp64 && b.n64 < N) return fail(ctx, RBE_ESTATE, "precision changed to FP64 after rbe_flex_init: call it again");
        const bool list = prm.skin > 0.0;
        FlexNList* nl = static_cast<FlexNList*>(ctx->flex_nls);
        if (list && (!nl || b.ncap_list < N || ctx->flex_cpos_cap < N || ctx->flex_code_cap < b.nl_entries ||
                     (fp64 && ctx->flex_cpos64_cap < N)))
            return fail(ctx, RBE_ESTATE, "skin or precision changed after rbe_flex_init: call it again");
        double4_32a* s64 = fp64 ? b.spos64 : nullptr;
        double4_32a* c64 = fp64 ? ctx->flex_cpos64 : nullptr;
        if (list) {
            const int grid = (int)std::min<int64_t>(nb, (int64_t)ctx->num_sms * 4);
            if (fp64)
                k_flex_nl_check<true><<<grid, kNptThreads, 0, s>>>(N, ctx->gpos, sys->charge, b.sorted,
                                                                 ctx->flex_cpos32, c64, b.sref, cf, nl);
            else
                k_flex_nl_check<false><<<grid, kNptThreads, 0, s>>>(N, ctx->gpos, sys->charge, b.sorted,
                                                                  ctx->flex_cpos32, nullptr, b.sref, cf, nl);
        }
        if ((st = launch_cell_list(ctx, N, ctx->gpos, sys->charge, list ? &nl->base : nullptr, fp64)) != RBE_OK)
            return st;
        const PairConst pc = make_pair_const(prm.rc, ctx->alpha, prm.qqr2e, prm.lj_sigma, prm.lj_eps);
        const CellConsts* cc = static_cast<const CellConsts*>(b.cellc);
        const FlexListArgs la{nl,       b.nbr,     ctx->flex_code, b.nnb,     b.sref, ctx->flex_cpos32,
                              c64,      ctx->gpos, ctx->d.status,  sys->cell, b.nbr_cap};
        // one resident wave of the variant launched: the warps stride over the slots, and a second
        // partial wave would run at a fraction of the occupancy
        auto pair = [&](auto f64_tag, auto mode_tag) {
            constexpr bool F64 = decltype(f64_tag)::value;
            constexpr int MODE = decltype(mode_tag)::value;
            static int bps = 0;
            if (!bps) {
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_flex_pair<F64, MODE>, kPairWarps * 32, 0) !=
                        cudaSuccess ||
                    bps < 1)
                    bps = 1;
                cudaGetLastError();
            }
            const int grid = std::max(1, std::min(nbp, ctx->num_sms * bps));
            if (MODE != 1) nbp_eval = grid;
            k_flex_pair<F64, MODE><<<grid, kPairWarps * 32, 0, s>>>(N, cc, pc, cf, b.cid, b.cnt, b.start, b.sorted,
                                                                    b.spos32, s64, b.Fr, b.partials, la);
        };
        using T = std::true_type;
        using F = std::false_type;
        using Cells = std::integral_constant<int, 0>;
        using Build = std::integral_constant<int, 1>;
        using List = std::integral_constant<int, 2>;
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
        if ((st = flex_check(ctx, "k_flex_pair")) != RBE_OK) return st;
    }
    k_flex_finish<<<std::max(1, nb), kNptThreads, 0, s>>>(N, sys->mom, sys->force, b.mprop, b.Fk, b.Fr, b.WEk, cf,
                                                          b.partials, nbp_eval, b.counter, sys->cell, prm, do_kick,
                                                          ctx->d.status);
    return flex_check(ctx, "k_flex_finish");
}

static rbe_status flex_cell_launch(rbe_ctx ctx, rbe_flex_system* sys, int advance)
{
    k_flex_cell<<<1, kFlexCellWarps * 32, 0, ctx->stream>>>(
        sys->cell, static_cast<FlexCoef*>(ctx->flex_coef), static_cast<GenCell*>(ctx->gcell_dev),
        static_cast<CellConsts*>(ctx->npt.cellc), sys->params, ctx->alpha, ctx->P, ctx->seed, ctx->npt.cellcap,
        sys->params.rc + sys->params.skin, advance, ctx->d.status);
    return flex_check(ctx, "k_flex_cell");
}

rbe_status flex_init(rbe_ctx ctx, rbe_flex_system* sys, uint64_t batch)
{
    rbe_status st = flex_validate(ctx, sys);
    if (st != RBE_OK) return st;
    const rbe_flex_params& prm = sys->params;
    double h[9];
    cudaError_t e = cudaMemcpyAsync(h, sys->cell + kFxH, 9 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read the cell");
    double len[3], width[3];
    if (!flex_cell_geometry(h, len, width)) return fail(ctx, RBE_EINVAL, "the cell must be finite with det h > 0");
    if (prm.real)
        for (int j = 0; j < 3; ++j)
            if (width[j] < 2.0 * (prm.rc + prm.skin))
                return fail(ctx, RBE_EINVAL, "real space needs rc + skin <= w/2 for every width of the cell");
    // scratch of the rectangular step, its cell list sized for widths up to twice the initial (and
    // with skin > 0 the neighbour list, sized by the density N / (w_0 w_1 w_2) >= N / V)
    if ((st = npt_ensure(ctx, sys->N, width, prm.rc, prm.skin)) != RBE_OK) return st;
    if (prm.skin > 0.0) {
        if (!ctx->flex_nls) {
            FlexNList* nl = nullptr;
            if ((e = ctx_alloc(ctx, &nl, sizeof(FlexNList))) != cudaSuccess)
                return cuda_fail(ctx, e, "flexible-cell list state");
            ctx->flex_nls = nl;
        }
        NptBuffers& nb_ = ctx->npt;
        if (ctx->flex_code_cap < nb_.nl_entries) {
            ctx_free(ctx, ctx->flex_code);
            ctx->flex_code = nullptr;
            ctx->flex_code_cap = 0;
            if ((e = ctx_alloc(ctx, &ctx->flex_code, (size_t)nb_.nl_entries)) != cudaSuccess)
                return cuda_fail(ctx, e, "flexible-cell list images");
            ctx->flex_code_cap = nb_.nl_entries;
        }
        if (ctx->flex_cpos_cap < sys->N) {
            ctx_free(ctx, ctx->flex_cpos32);
            ctx->flex_cpos32 = nullptr;
            ctx->flex_cpos_cap = 0;
            if ((e = ctx_alloc(ctx, &ctx->flex_cpos32, sizeof(float4) * (size_t)sys->N)) != cudaSuccess)
                return cuda_fail(ctx, e, "flexible-cell list positions");
            ctx->flex_cpos_cap = sys->N;
        }
        if (ctx->precision == RBE_FP64 && ctx->flex_cpos64_cap < sys->N) {
            ctx_free(ctx, ctx->flex_cpos64);
            ctx->flex_cpos64 = nullptr;
            ctx->flex_cpos64_cap = 0;
            if ((e = ctx_alloc(ctx, &ctx->flex_cpos64, sizeof(double4_32a) * (size_t)sys->N)) != cudaSuccess)
                return cuda_fail(ctx, e, "flexible-cell list positions (FP64)");
            ctx->flex_cpos64_cap = sys->N;
        }
    }
    // proposal tables for lengths up to sqrt(3) x twice the initial cell vectors, and the unit cube
    int need = 2 * host_axis_M(ctx->alpha, 1.0) + 1;
    for (int j = 0; j < 3; ++j) {
        const int M = host_axis_M(ctx->alpha, std::sqrt(3.0) * kFlexHeadroom * len[j]);
        if (M > (1 << 20)) return fail(ctx, RBE_EINVAL, "alpha |a_j|^2 too large for the per-axis tables");
        need = std::max(need, 2 * M + 1);
    }
    if ((st = ensure_table_capacity(ctx, need)) != RBE_OK) return st;
    const int P = ctx->P;
    if ((st = ensure_k_capacity(ctx, std::max(P, 1))) != RBE_OK) return st;
    if (ctx->gchain_cap < P) {
        ctx_free(ctx, ctx->gchain);
        ctx->gchain = nullptr;
        ctx->gchain_cap = 0;
        if ((e = ctx_alloc(ctx, &ctx->gchain, sizeof(int4) * (size_t)std::max(P, 1))) != cudaSuccess ||
            (e = cudaMemsetAsync(ctx->gchain, 0, sizeof(int4) * (size_t)std::max(P, 1), ctx->stream)) != cudaSuccess)
            return cuda_fail(ctx, e, "general-cell MH chain");
        ctx->gchain_cap = P;
    }
    if (sys->N > ctx->gpos_cap) {
        ctx_free(ctx, ctx->gpos);
        ctx->gpos = nullptr;
        ctx->gpos_cap = 0;
        if ((e = ctx_alloc(ctx, &ctx->gpos, sizeof(double) * 3 * (size_t)sys->N)) != cudaSuccess)
            return cuda_fail(ctx, e, "scaled coordinates");
        ctx->gpos_cap = sys->N;
    }
    if (!ctx->flex_coef) {
        FlexCoef* c = nullptr;
        GenCell* g = nullptr;
        if ((e = ctx_alloc(ctx, &c, sizeof(FlexCoef))) != cudaSuccess || (e = ctx_alloc(ctx, &g, sizeof(GenCell))) != cudaSuccess) {
            ctx_free(ctx, c);
            return cuda_fail(ctx, e, "flexible-cell coefficients");
        }
        ctx->flex_coef = c;
        ctx->gcell_dev = g;
    }
    ctx->flex_ready_N = sys->N;
    ctx->npt_ready_N = -1;  // the shared scratch now holds this system's masses and cell list
    ctx->water_ready_N = -1;
    NptBuffers& b = ctx->npt;
    const int nb = (int)((sys->N + kNptThreads - 1) / kNptThreads);
    k_flex_mass<<<nb, kNptThreads, 0, ctx->stream>>>(sys->N, sys->mass, b.mprop);
    k_flex_set_step<<<1, 32, 0, ctx->stream>>>(sys->cell, batch);
    if (prm.skin > 0.0)
        k_flex_nl_init<<<1, 32, 0, ctx->stream>>>(static_cast<FlexNList*>(ctx->flex_nls), (float)(prm.rc + prm.skin),
                                                  (float)prm.rc, sys->cell);
    if ((st = flex_check(ctx, "k_flex_set_step")) != RBE_OK) return st;
    if ((st = flex_cell_launch(ctx, sys, 0)) != RBE_OK) return st;
    k_flex_scale<<<nb, kNptThreads, 0, ctx->stream>>>(sys->N, sys->pos, static_cast<const FlexCoef*>(ctx->flex_coef),
                                                      ctx->gpos);
    if ((st = flex_check(ctx, "k_flex_scale")) != RBE_OK) return st;
    if ((st = flex_forces(ctx, sys, 0)) != RBE_OK) return st;
    k_flex_set_step<<<1, 32, 0, ctx->stream>>>(sys->cell, sys->step);
    return flex_check(ctx, "k_flex_set_step");
}

rbe_status flex_run(rbe_ctx ctx, rbe_flex_system* sys, int32_t nsteps)
{
    if (nsteps < 1) return fail(ctx, RBE_EINVAL, "nsteps must be >= 1");
    rbe_status st = flex_validate(ctx, sys);
    if (st != RBE_OK) return st;
    if (ctx->flex_ready_N != sys->N || !ctx->flex_coef) return fail(ctx, RBE_ESTATE, "call rbe_flex_init for this system first");
    if (sys->params.real && ctx->precision == RBE_FP64 && ctx->npt.n64 < sys->N)
        return fail(ctx, RBE_ESTATE, "precision changed to FP64 after rbe_flex_init: call it again");
    const int64_t N = sys->N;
    const int nb = (int)((N + kNptThreads - 1) / kNptThreads);
    const FlexCoef* cf = static_cast<const FlexCoef*>(ctx->flex_coef);
    for (int32_t k = 0; k < nsteps; ++k) {
        if ((st = flex_cell_launch(ctx, sys, 1)) != RBE_OK) return st;
        if (ctx->precision == RBE_FP64)
            k_flex_drift<false><<<nb, kNptThreads, 0, ctx->stream>>>(N, sys->pos, sys->mom, sys->force, ctx->npt.mprop, cf,
                                                                   ctx->seed, sys->cell, ctx->gpos);
        else
            k_flex_drift<true><<<nb, kNptThreads, 0, ctx->stream>>>(N, sys->pos, sys->mom, sys->force, ctx->npt.mprop, cf,
                                                                  ctx->seed, sys->cell, ctx->gpos);
        if ((st = flex_check(ctx, "k_flex_drift")) != RBE_OK) return st;
        if ((st = flex_forces(ctx, sys, 1)) != RBE_OK) return st;
        sys->step += 1;
    }
    return RBE_OK;
}

}  // namespace rbe
