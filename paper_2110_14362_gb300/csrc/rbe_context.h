// Host-side state of an RBE context and the launchers shared by the library's
// translation units.  Not part of the public ABI (include/rbe.h is).
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/rbe.h"

namespace rbe {

// Box-dependent state of an evaluation, written on the device by k_tables whenever the
// box changes (from host values or from a device-resident box) and read by every other
// kernel: the sampling tables' sizes and sums, S, and the constants of both precisions.
struct FixScaleH {  // host mirror of rbe::FixScale (1/l = q 2^e)
    unsigned long long q;
    int e;
    int pad;
};

struct KState {
    double L[3];        // box lengths
    double inv[3];      // 1 / l
    double V;           // l_x l_y l_z
    double alpha;
    int M[3];           // table truncation per axis
    int sh[3];          // fixed-point shift of the integer weights per axis
    double H[3];        // per-axis sums (Eq. (psf))
    double S;           // H_x H_y H_z - 1 (Eq. (S))
    double wP;          // S / P
    FixScaleH sc[3];    // 1/l as a 64-bit mantissa and a power of two (FP32-phase path)
    float cx, cy, cz;   // 2 pi / l
    int P;
    double ce;          // 2 pi / V
    double cb;          // 4 pi / V
    double inv4a;       // 1 / (4 alpha)
    double cself;       // -sqrt(alpha / pi)
};

// Frequency tiling of the rho pass (rho_shape in rbe_kspace.cu).
struct RhoShape {
    int kf;             // frequencies per thread (1, 2 or 4)
    int ktiles;         // frequency tiles
    int kthreads;       // threads per block: whole warps (ksub sub-streams of kthreads / ksub lanes)
    int ksub;           // particle sub-streams per block
    int klanes;         // frequency lanes per sub-stream of a two-frequency wide tile (0: kthreads / ksub)
};

// Launch plan of the N x K pair kernels (chosen by make_plan in rbe_kspace.cu).
struct Plan {
    int kf;             // frequencies per thread in the rho pass
    int ktiles;         // frequency tiles in the rho pass (kthreads x kf frequencies each)
    int kthreads;       // threads per rho block: whole warps, <= 256
    int ksub;           // particle sub-streams per rho block
    int klanes;         // lanes per sub-stream of a wide two-frequency tile (0: kthreads / ksub)
    int nchunks;        // particle chunks in the rho pass
    int64_t chunk_len;  // particles per chunk
    int ppt;            // particles per thread in the force pass
    int fblocks;        // blocks of the force pass
    int64_t per_block;  // particles per force block
};

// Scratch of the NPT step (grown on demand).
struct NptBuffers {
    double* Fk = nullptr;          // N*3 k-space forces (Gaussian units)
    double* Fr = nullptr;          // N*3 real-space forces (kJ/mol/A)
    double* WEk = nullptr;         // 11: k-space virial (9) + energy (2)
    double* coef = nullptr;        // per-step coefficients (NptCoef)
    int* cid = nullptr;            // N cell index per particle
    int* fill = nullptr;           // N particle indices grouped by cell (atomic fill order)
    int* sorted = nullptr;         // N particle indices grouped by cell, by index within a cell
    float4* spos32 = nullptr;      // N packed FP32 positions+charge in sorted order
    double4_32a* spos64 = nullptr; // N packed FP64 positions+charge (FP64 path)
    double2* mprop = nullptr;      // N (1/m, sqrt(m)), set by rbe_npt_init
    void* cellc = nullptr;         // cell-list constants of the current box (rbe_npt.cu)
    int* nbr = nullptr;            // neighbour list: slots of the neighbours of slot u at [u * nbr_cap, ...)
    int* nnb = nullptr;            // neighbours per slot
    float4* sref = nullptr;        // per slot: scaled position s = r / l at the last build
    void* nls = nullptr;           // neighbour-list state (rbe_npt.cu)
    int64_t nl_entries = 0;        // allocated list entries
    int64_t ncap_list = 0;         // slots of nnb and sref
    int nbr_cap = 0;               // list entries per slot
    int* cnt = nullptr;            // cells: counts
    int* start = nullptr;          // cells: exclusive prefix sums
    int* cursor = nullptr;         // cells: fill cursors
    double* partials = nullptr;    // per-block partial sums (K2, W_r, E_coul, E_lj)
    unsigned* counter = nullptr;   // last-block counter of the finishing kernel
    int64_t ncap = 0;
    int64_t n64 = 0;
    int cellcap = 0;
    int partcap = 0;
};

struct DeviceBuffers {
    unsigned long long* cum = nullptr;  // [3][tab_cap] integer cumulative weights
    int tab_cap = 0;                  // entries per axis (>= 2M+1)
    KState* ks = nullptr;             // box-dependent state
    int4* m = nullptr;                // [kcap] (mx, my, mz, 0)
    double* w = nullptr;              // [kcap] per-frequency weight (S/P for RBE)
    double2* rho = nullptr;           // [kcap]
    double* terms = nullptr;          // [kcap + 1][8] per-frequency energy/virial terms
    int4* coef_m = nullptr;           // [kcap] FP32 force data (mx, my, mz, bits of A)
    float4* coef_f = nullptr;         // [kcap] FP32 force data (B, mx, my, mz)
    double2* coef_d = nullptr;        // [kcap] FP64 force data (A, B)
    int kcap = 0;
    void* partials = nullptr;         // [(K + 1) * nchunks] double2 (FP64) or float4 (FP32-phase)
    size_t part_cap = 0;              // in 16-byte entries
    unsigned* counter = nullptr;      // last-block counter of the reduction
    unsigned* status = nullptr;       // latched device status bits
    double* pos = nullptr;            // host-API staging
    double* q = nullptr;
    double* F = nullptr;
    double* WE = nullptr;             // 11 doubles: virial (9) + energy (2)
    int64_t ncap = 0;
};

}  // namespace rbe

struct rbe_ctx_s {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    double box[3] = {0, 0, 0};
    double alpha = 0;
    int32_t P = 0;
    uint64_t seed = 0;
    int32_t precision = RBE_FP64;
    int32_t rho_accum = RBE_RHO_COMP32;
    int32_t sampler = 0;             // rbe_sampler: exact, offline or Metropolis--Hastings (Sec. 4.3)
    int4* chain = nullptr;           // MH state per frequency slot (m = 0: start from the exact draw)
    int32_t chain_cap = 0;
    int32_t Ptilde = 0;              // frequencies of a separate pressure batch (0: the force batch)
    int32_t reuse = 1;               // NPT: samples drawn every `reuse` steps, kept on the device
    int4* m_all = nullptr;           // reuse > 1: the kept batches, reuse x (P + Ptilde)
    int64_t m_all_cap = 0;
    int4* gchain = nullptr;          // general cell: the MH state per slot (m = 0: start from the proposal)
    int32_t gchain_cap = 0;
    double* gpos = nullptr;          // general cell: scaled coordinates s = h^{-1} r, N x 3
    int64_t gpos_cap = 0;
    bool tables_dirty = true;
    int32_t last_K = 0;
    rbe::NptBuffers npt;
    int64_t npt_ready_N = -1;        // N of the system rbe_npt_init prepared the scratch for
    int64_t flex_ready_N = -1;       // N of the system rbe_flex_init prepared the scratch for
    int64_t water_ready_N = -1;      // N of the system rbe_water_init prepared the scratch for
    void* flex_coef = nullptr;       // per-step coefficients of the flexible-cell step (rbe_flex.cu)
    void* gcell_dev = nullptr;       // general-cell quantities of the current cell (rbe_flex.cu)
    void* flex_nls = nullptr;        // neighbour-list state of the flexible-cell step (rbe_flex.cu)
    float4* flex_cpos32 = nullptr;   // flexible cell with a list: unwrapped Cartesian positions per slot
    double4_32a* flex_cpos64 = nullptr;  // the same in FP64 (FP64 path)
    unsigned char* flex_code = nullptr;  // image of each list entry at the build
    int64_t flex_cpos_cap = 0, flex_cpos64_cap = 0, flex_code_cap = 0;
    bool timing = false;             // record CUDA events around each evaluation kernel
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // pipelined host-buffer calls: a copy stream, its events, pinned outputs (virial, energy,
    // status word)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t pev[17] = {};  // 1 + 2 kMaxPieces
    double* h_out = nullptr;
    rbe::DeviceBuffers d;
    std::string last_error;
};

namespace rbe {

// Stream-ordered (re)allocation of context scratch: it never synchronises the device, so
// contexts on other streams keep running while one grows its buffers.
template <typename T>
inline cudaError_t ctx_alloc(rbe_ctx ctx, T** p, size_t bytes)
{
    return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, ctx->stream);
}

inline void ctx_free(rbe_ctx ctx, void* p)
{
    if (p) cudaFreeAsync(p, ctx->stream);
}

// Device validation helpers (rbe_api.cu).
rbe_status fail(rbe_ctx ctx, rbe_status st, const std::string& msg);
rbe_status cuda_fail(rbe_ctx ctx, cudaError_t err, const char* what);
// A device pointer argument: NULL allowed unless required, 8-byte aligned, device memory (rbe_api.cu).
rbe_status check_dev(rbe_ctx ctx, const void* p, const char* name, bool required);

// The status of latched device bits (the message set on ctx), RBE_OK for none (rbe_api.cu).
rbe_status status_from_bits(rbe_ctx ctx, unsigned bits);

// Host-side rule shared by create/set_box: the per-axis table size for (alpha, l).
int host_axis_M(double alpha, double ell);

// Launchers (rbe_kspace.cu).  All asynchronous on ctx->stream.
rbe_status ensure_tables(rbe_ctx ctx);
rbe_status ensure_table_capacity(rbe_ctx ctx, int need);
rbe_status launch_tables(rbe_ctx ctx, const double* box_dev);
rbe_status ensure_k_capacity(rbe_ctx ctx, int K);
rbe_status launch_sample(rbe_ctx ctx, uint64_t step, int P);
rbe_status launch_sample_device_box(rbe_ctx ctx, uint64_t step, int P, const unsigned long long* step_dev);
rbe_status launch_tables_sample_device(rbe_ctx ctx, int P, const double* box_dev, const unsigned long long* step_dev);
rbe_status npt_init(rbe_ctx ctx, rbe_system* sys, uint64_t batch);
rbe_status npt_run(rbe_ctx ctx, rbe_system* sys, int32_t nsteps);
// One NPT step in phases, for a caller that evaluates the step's k-space itself into npt.Fk
// and npt.WEk (between kNptPhaseMove and kNptPhaseFinish; the real space may run beside it):
// the cell update and drift; the real space; the finishing kernel, which advances the step.
constexpr int kNptPhaseMove = 0, kNptPhaseReal = 1, kNptPhaseFinish = 2;
rbe_status npt_step_phase(rbe_ctx ctx, rbe_system* sys, int phase);
// Shared with the flexible-cell step (rbe_npt.cu): scratch for N particles and cells of edges up
// to twice `box` (plus a list with skin > 0), the pair kernel's grid, the cell list of the
// constants in npt.cellc (nls: the neighbour-list state or NULL).
rbe_status npt_ensure(rbe_ctx ctx, int64_t N, const double box[3], double rc, double skin);
int pair_blocks(rbe_ctx ctx, int64_t N, bool fp64);
rbe_status launch_cell_list(rbe_ctx ctx, int64_t N, const double* pos, const double* q, void* nls, bool fp64);
// Shared with the rigid-water step (rbe_npt.cu): parameter checks, the setup of rbe_npt_init
// before its first forces, the device step index, the isotropic cell part of a step.
rbe_status npt_validate(rbe_ctx ctx, const rbe_system* sys);
rbe_status npt_prepare(rbe_ctx ctx, rbe_system* sys, uint64_t batch);
rbe_status launch_npt_set_step(rbe_ctx ctx, double* cell, uint64_t step);
rbe_status launch_npt_cell_iso(rbe_ctx ctx, rbe_system* sys);
// The rigid-water step (rbe_water.cu).
rbe_status water_init(rbe_ctx ctx, rbe_system* sys, const rbe_water_params* wp, uint64_t batch);
rbe_status water_run(rbe_ctx ctx, rbe_system* sys, const rbe_water_params* wp, int32_t nsteps);
// The flexible-cell step (rbe_flex.cu).
rbe_status flex_init(rbe_ctx ctx, rbe_flex_system* sys, uint64_t batch);
rbe_status flex_run(rbe_ctx ctx, rbe_flex_system* sys, int32_t nsteps);
rbe_status launch_evaluate(rbe_ctx ctx, int64_t N, const double* pos, const double* q, int K,
                           bool uniform_weight, double* F, double* W, double* E);
// pos: N x 3 double with charges q, or with xyzq one float4 (x, y, z, q) per particle (q unused,
// FP32-phase path only).
rbe_status launch_rbe(rbe_ctx ctx, int64_t N, const void* pos, const double* q, int P, double* F, double* W,
                      double* E, bool xyzq = false);
rbe_status launch_tables_box(rbe_ctx ctx, const double box[3]);
// Pieces of the pipelined host-buffer evaluation (copy stream events: 1 + 2 kMaxPieces).
constexpr int kMaxPieces = 8;
rbe_status launch_evaluate_staged(rbe_ctx ctx, int64_t N, const double* h_pos, const double* h_q, double* h_F,
                                  double* d_pos, double* d_q, double* d_F, int K, double* W, double* E,
                                  int pieces);
void record_event(rbe_ctx ctx, int idx);
rbe_status launch_weights_from_list(rbe_ctx ctx, int K, const int32_t* m, const double* w);

}  // namespace rbe
