// Batched RBE k-space evaluation: many systems of uneven N in five launches in total.
//
// Each item is one system (its own positions, charges, box, Philox key and batch index) with
// the batch's alpha and P, on the FP32-phase path with compensated FP32 accumulation inside
// a staged tile (RBE_RHO_COMP32) and FP64 energy and virial terms.  Per evaluation:
//   k_btables   one block per item whose box changed: tables and box constants  (H1)
//   k_bsample   blocks of 128 frequencies per item                             (H2)
//   k_brho      persistent grid over the work list of (item, frequency tile, particle
//               chunk) tiles: partial rho(k) per chunk                         (H4)
//   k_breduce   one block per (item, frequency): rho(k), terms, force coefficients (H3, H6)
//   k_bforce    persistent grid over (item, particle block) tiles, then one final-sum tile
//               per item: forces, virial, energies                             (H5, H6)
// The tiles run the single-system kernels' bodies (rbe_kspace_tiles.cuh).  Tile shapes
// (frequencies per rho tile, particles per rho chunk, particles per force block) are the
// batch's, set by hand or by rbe_batch_autotune, which times the candidate shapes on the
// caller's items.  An item's result depends only on its own inputs and the tile shapes, never
// on the other items (fixed-order sums inside the item's tiles).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "rbe_context.h"
#include "rbe_device.cuh"
#include "rbe_kspace_tiles.cuh"

namespace rbe {

// Per item, on the device.
struct BItem {
    const double* pos;
    const double* q;
    double* F;
    double* W;
    double* E;
    int64_t N;
    uint64_t seed, step;
    int64_t chunk_len, per_block;
    int64_t part_off;  // float4 offset of the item's (P + 1) x nchunks partials
    int nchunks, fblocks;
};

constexpr int kSampleBlock = 128;

__global__ void __launch_bounds__(kTableThreads)
k_btables(const double* __restrict__ boxes, const int* __restrict__ which, double alpha, int P,
          unsigned long long* __restrict__ cum, int cap, KState* __restrict__ ks, unsigned* __restrict__ status)
{
    const int r = which[blockIdx.x];
    const double* b = boxes + 3 * (size_t)r;
    tables_body(b[0], b[1], b[2], nullptr, alpha, P, cum + (size_t)r * 3 * cap, cap, ks + r, status);
}

__global__ void k_bsample(const BItem* __restrict__ items, int P, int blocks_per_item,
                          const unsigned long long* __restrict__ cum, int cap, int smem_cap,
                          const KState* __restrict__ ks, int4* __restrict__ m, double* __restrict__ w,
                          unsigned* __restrict__ status)
{
    const int r = blockIdx.x / blocks_per_item;
    const int lb = (blockIdx.x % blocks_per_item) * kSampleBlock;
    const BItem it = items[r];
    sample_body(lb, it.seed, it.step, nullptr, P, P, cum + (size_t)r * 3 * cap, cap, smem_cap, ks + r,
                m + (size_t)r * P, w + (size_t)r * P, status);
}

// Persistent: block b takes tiles b, b + gridDim.x, ...; tile = (item, frequency tile,
// particle chunk).  blockDim.x = frequencies per tile.
__global__ void __launch_bounds__(kMaxRhoThreads, 8)
k_brho(const BItem* __restrict__ items, const int4* __restrict__ tiles, int ntiles, const KState* __restrict__ ks,
       const int4* __restrict__ m, int P, float4* __restrict__ partials, unsigned* __restrict__ status)
{
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const BItem it = items[tl.x];
        rho_f32_tile<RBE_RHO_COMP32, 1>(tl.y, tl.z, it.pos, it.q, it.N, ks + tl.x, m + (size_t)tl.x * P, P, it.chunk_len,
                                   it.nchunks, partials + it.part_off, status);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kReduceThreads)
k_breduce(const BItem* __restrict__ items, int P, const float4* __restrict__ partials, const int4* __restrict__ m,
          const double* __restrict__ w, const KState* __restrict__ ks, double2* __restrict__ rho,
          double* __restrict__ terms, int4* __restrict__ coef_m, float4* __restrict__ coef_f,
          unsigned* __restrict__ status)
{
    const int r = blockIdx.x / (P + 1), l = blockIdx.x % (P + 1);
    const BItem it = items[r];
    const size_t o = (size_t)r * P;
    reduce_f32_row(l, partials + it.part_off, it.nchunks, P, m + o, w + o, ks + r, rho + o,
                   terms + (size_t)r * (P + 1) * 8, coef_m + o, coef_f + o, status);
}

// Persistent: tiles [0, nforce) are (item, particle block); tiles [nforce, nforce + R) the
// per-item energy and virial sums.
__global__ void __launch_bounds__(kForceThreads, RBE_FORCE_MINB)
k_bforce(const BItem* __restrict__ items, const int2* __restrict__ tiles, int nforce, int R,
         const KState* __restrict__ ks, const int4* __restrict__ coef_m, const float4* __restrict__ coef_f, int P,
         const double* __restrict__ terms, unsigned* __restrict__ status)
{
    for (int t = blockIdx.x; t < nforce + R; t += gridDim.x) {
        if (t < nforce) {
            const int2 tl = tiles[t];
            const BItem it = items[tl.x];
            const size_t o = (size_t)tl.x * P;
            force_f32_block<false>((int64_t)tl.y, it.pos, it.q, it.N, it.per_block, ks + tl.x, coef_m + o, coef_f + o, P,
                            it.F, status);
        } else {
            const int r = t - nforce;
            const BItem it = items[r];
            final_sums(terms + (size_t)r * (P + 1) * 8, P, ks + r, it.W, it.E, status);
        }
        __syncthreads();
    }
}

template <typename Kern>
static int resident_blocks(Kern kern, int threads, size_t dyn_smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, dyn_smem) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return std::max(1, n);
}

}  // namespace rbe

using namespace rbe;

struct rbe_batch_s {
    int device = 0;
    int num_sms = 1;
    cudaStream_t stream = nullptr;
    double alpha = 0.0;
    int P = 0;
    int max_items = 0;
    int cap = 0;  // table entries per axis
    // tile shapes
    int rho_k = 0, rho_chunk = 0, force_block = 0;
    // device buffers
    BItem* d_items = nullptr;
    double* d_boxes = nullptr;
    int* d_which = nullptr;
    KState* d_ks = nullptr;
    unsigned long long* d_cum = nullptr;
    int4* d_m = nullptr;
    double* d_w = nullptr;
    double2* d_rho = nullptr;
    double* d_terms = nullptr;
    int4* d_coef_m = nullptr;
    float4* d_coef_f = nullptr;
    unsigned* d_status = nullptr;
    float4* d_part = nullptr;
    size_t part_cap = 0;
    int4* d_rtiles = nullptr;
    size_t rtile_cap = 0;
    int2* d_ftiles = nullptr;
    size_t ftile_cap = 0;
    // host staging (pinned) and the shapes the device work lists were built for
    BItem* h_items = nullptr;
    double* h_boxes = nullptr;
    int* h_which = nullptr;
    std::vector<double> last_boxes;
    std::vector<int64_t> plan_N;
    int plan_k = -1, plan_chunk = -1, plan_fb = -1;
    int n_rtiles = 0, n_ftiles = 0;
    std::vector<int4> h_rtiles;
    std::vector<int2> h_ftiles;
    int rho_grid_per_sm[kMaxRhoThreads / 32 + 1] = {0};
    int force_grid_per_sm = 1;
    cudaEvent_t upload_ev = nullptr;  // after the last upload of the pinned descriptors
    bool upload_pending = false;
    std::string last_error;
};

namespace {

rbe_status bfail(rbe_batch b, rbe_status st, const std::string& msg)
{
    if (b) b->last_error = msg;
    return fail(nullptr, st, msg);
}

rbe_status bcuda(rbe_batch b, cudaError_t e, const char* what)
{
    return bfail(b, e == cudaErrorMemoryAllocation ? RBE_ENOMEM : RBE_ECUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

struct BatchDevice {
    int prev = -1;
    explicit BatchDevice(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~BatchDevice()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
cudaError_t grow(T** p, size_t* cap, size_t need, cudaStream_t s)
{
    if (need <= *cap) return cudaSuccess;
    if (*p) cudaFreeAsync(*p, s);
    *p = nullptr;
    *cap = 0;
    const size_t n = need + need / 4 + 64;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), sizeof(T) * n, s);
    if (e == cudaSuccess) *cap = n;
    return e;
}

bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

bool valid_tiles(int P, int rho_k, int rho_chunk, int force_block)
{
    return rho_k >= 32 && rho_k <= kMaxRhoThreads && rho_k % 32 == 0 && rho_chunk >= 32 && rho_chunk <= (1 << 24) &&
           force_block >= kForceRound && force_block % kForceRound == 0 && force_block <= (1 << 24) && P >= 1;
}

// The tile shapes the planner uses when none were set: the single-system planner's
// frequency tiles (whole warps, at most 256 frequencies) and chunks of 256 particles.
void default_tiles(rbe_batch b)
{
    const int ktiles = (b->P + kMaxRhoThreads - 1) / kMaxRhoThreads;
    const int per = (b->P + ktiles - 1) / ktiles;
    b->rho_k = std::min(kMaxRhoThreads, 32 * ((per + 31) / 32));
    b->rho_chunk = 256;
    b->force_block = 2 * kForceRound;
}

rbe_status validate_items(rbe_batch b, const rbe_batch_item* items, int n)
{
    if (n < 1 || n > b->max_items) return bfail(b, RBE_EINVAL, "item count must be 1..max_items");
    if (!items) return bfail(b, RBE_EINVAL, "items is NULL");
    for (int r = 0; r < n; ++r) {
        const rbe_batch_item& it = items[r];
        if (it.N < 1 || it.N > ((int64_t)1 << 31) - 256) return bfail(b, RBE_EINVAL, "item N out of range");
        if (!it.pos || !it.charge || !it.forces || !it.virial)
            return bfail(b, RBE_EINVAL, "item pos, charge, forces and virial must not be NULL");
        if ((reinterpret_cast<uintptr_t>(it.pos) | reinterpret_cast<uintptr_t>(it.charge) |
             reinterpret_cast<uintptr_t>(it.forces) | reinterpret_cast<uintptr_t>(it.virial) |
             reinterpret_cast<uintptr_t>(it.energy)) % 8)
            return bfail(b, RBE_EINVAL, "item buffers must be 8-byte aligned");
        if ((it.step >> 56) != 0) return bfail(b, RBE_EINVAL, "item step must be < 2^56");
        for (int t = 0; t < 3; ++t) {
            const double l = it.box[t];
            if (!std::isfinite(l) || !(l > 0.0)) return bfail(b, RBE_EINVAL, "item box lengths must be finite and > 0");
            const double c = (kPi * kPi) / (b->alpha * (l * l));
            if (!(c <= 600.0)) return bfail(b, RBE_EINVAL, "pi^2/(alpha l^2) > 600: degenerate frequency distribution");
            if (2 * host_axis_M(b->alpha, l) + 1 > b->cap)
                return bfail(b, RBE_EINVAL, "item box beyond the batch's table capacity (rbe_batch_create max_box)");
        }
    }
    return RBE_OK;
}

// Work lists and item descriptors for the current items and tile shapes (rebuilt only when
// the N of some item or a tile shape changed).
rbe_status plan(rbe_batch b, const rbe_batch_item* items, int n)
{
    bool same = (int)b->plan_N.size() == n && b->plan_k == b->rho_k && b->plan_chunk == b->rho_chunk &&
                b->plan_fb == b->force_block;
    for (int r = 0; same && r < n; ++r) same = b->plan_N[r] == items[r].N;
    if (!same) {
        if (capturing(b->stream))
            return bfail(b, RBE_ESTATE, "new item sizes or tiles during stream capture: evaluate these items once "
                                        "outside capture first");
        b->h_rtiles.clear();
        b->h_ftiles.clear();
        b->plan_N.assign(n, 0);
        const int ktiles = (b->P + b->rho_k - 1) / b->rho_k;
        int64_t part = 0;
        for (int r = 0; r < n; ++r) {
            const int64_t N = items[r].N;
            BItem& it = b->h_items[r];
            it.chunk_len = std::min<int64_t>(N, b->rho_chunk);
            it.nchunks = (int)((N + it.chunk_len - 1) / it.chunk_len);
            it.part_off = part;
            part += (int64_t)(b->P + 1) * it.nchunks;
            it.per_block = b->force_block;
            it.fblocks = (int)((N + it.per_block - 1) / it.per_block);
            for (int c = 0; c < it.nchunks; ++c)
                for (int kt = 0; kt < ktiles; ++kt) b->h_rtiles.push_back(make_int4(r, kt, c, 0));
            for (int f = 0; f < it.fblocks; ++f) b->h_ftiles.push_back(make_int2(r, f));
            b->plan_N[r] = N;
        }
        if (b->h_rtiles.size() > (size_t)INT32_MAX || b->h_ftiles.size() > (size_t)INT32_MAX)
            return bfail(b, RBE_EINVAL, "work list too long");
        cudaError_t e;
        if ((e = grow(&b->d_part, &b->part_cap, (size_t)part, b->stream)) != cudaSuccess ||
            (e = grow(&b->d_rtiles, &b->rtile_cap, b->h_rtiles.size(), b->stream)) != cudaSuccess ||
            (e = grow(&b->d_ftiles, &b->ftile_cap, b->h_ftiles.size(), b->stream)) != cudaSuccess)
            return bcuda(b, e, "batch work lists");
        if ((e = cudaMemcpyAsync(b->d_rtiles, b->h_rtiles.data(), sizeof(int4) * b->h_rtiles.size(),
                                 cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(b->d_ftiles, b->h_ftiles.data(), sizeof(int2) * b->h_ftiles.size(),
                                 cudaMemcpyHostToDevice, b->stream)) != cudaSuccess)
            return bcuda(b, e, "upload work lists");
        // the host vectors are read by those copies: keep them until the stream passes here
        if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return bcuda(b, e, "work lists");
        b->n_rtiles = (int)b->h_rtiles.size();
        b->n_ftiles = (int)b->h_ftiles.size();
        b->plan_k = b->rho_k;
        b->plan_chunk = b->rho_chunk;
        b->plan_fb = b->force_block;
    }
    for (int r = 0; r < n; ++r) {
        BItem& it = b->h_items[r];
        it.pos = items[r].pos;
        it.q = items[r].charge;
        it.F = items[r].forces;
        it.W = items[r].virial;
        it.E = items[r].energy;
        it.N = items[r].N;
        it.seed = items[r].seed;
        it.step = items[r].step;
    }
    return RBE_OK;
}

// The launches of one evaluation; which of the five passes run is given by the mask
// (1 tables, 2 sample, 4 rho, 8 reduce, 16 force) so that the tuner can time one pass.
rbe_status launch(rbe_batch b, int n, int mask)
{
    cudaStream_t s = b->stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->d_items, b->h_items, sizeof(BItem) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return bcuda(b, e, "upload items");
    const bool cap = capturing(s);
    const int P = b->P;
    if (mask & 1) {
        // tables of the items whose box changed since the last evaluation
        int nw = 0;
        for (int r = 0; r < n; ++r) {
            const double* bx = b->h_boxes + 3 * (size_t)r;
            const bool changed = b->last_boxes.size() < 3 * (size_t)(r + 1) || b->last_boxes[3 * r] != bx[0] ||
                                 b->last_boxes[3 * r + 1] != bx[1] || b->last_boxes[3 * r + 2] != bx[2];
            if (changed) b->h_which[nw++] = r;
        }
        if (nw > 0) {
            if ((e = cudaMemcpyAsync(b->d_boxes, b->h_boxes, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s)) !=
                    cudaSuccess ||
                (e = cudaMemcpyAsync(b->d_which, b->h_which, sizeof(int) * nw, cudaMemcpyHostToDevice, s)) !=
                    cudaSuccess)
                return bcuda(b, e, "upload boxes");
            k_btables<<<nw, kTableThreads, 0, s>>>(b->d_boxes, b->d_which, b->alpha, P, b->d_cum, b->cap, b->d_ks,
                                                   b->d_status);
            b->last_boxes.assign(b->h_boxes, b->h_boxes + 3 * (size_t)n);
        }
    }
    // the pinned descriptors (and boxes) may be overwritten once these copies have run
    if (!cap) {
        if ((e = cudaEventRecord(b->upload_ev, s)) != cudaSuccess) return bcuda(b, e, "cudaEventRecord");
        b->upload_pending = true;
    }
    if (mask & 2) {
        const int bpi = (P + kSampleBlock - 1) / kSampleBlock;
        const size_t smem = sizeof(unsigned long long) * 3 * (size_t)b->cap;
        const int smem_cap = smem <= 48 * 1024 ? b->cap : 0;
        k_bsample<<<n * bpi, kSampleBlock, smem_cap ? smem : 0, s>>>(b->d_items, P, bpi, b->d_cum, b->cap, smem_cap,
                                                                    b->d_ks, b->d_m, b->d_w, b->d_status);
    }
    if (mask & 4) {
        int& per_sm = b->rho_grid_per_sm[b->rho_k / 32];
        if (per_sm == 0) per_sm = resident_blocks(k_brho, b->rho_k, 0);
        const int grid = std::max(1, std::min(b->n_rtiles, b->num_sms * per_sm));
        k_brho<<<grid, b->rho_k, 0, s>>>(b->d_items, b->d_rtiles, b->n_rtiles, b->d_ks, b->d_m, P, b->d_part,
                                         b->d_status);
    }
    if (mask & 8)
        k_breduce<<<n * (P + 1), kReduceThreads, 0, s>>>(b->d_items, P, b->d_part, b->d_m, b->d_w, b->d_ks, b->d_rho,
                                                         b->d_terms, b->d_coef_m, b->d_coef_f, b->d_status);
    if (mask & 16) {
        const int kstage = std::min(P, kForceStageK);
        const int grid = std::max(1, std::min(b->n_ftiles + n, b->num_sms * b->force_grid_per_sm));
        k_bforce<<<grid, kForceThreads, (size_t)kForceSmemPerK * kstage, s>>>(b->d_items, b->d_ftiles, b->n_ftiles, n, b->d_ks,
                                                                 b->d_coef_m, b->d_coef_f, P, b->d_terms,
                                                                 b->d_status);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return bcuda(b, e, "batched k-space launch");
    return RBE_OK;
}

rbe_status prepare(rbe_batch b, const rbe_batch_item* items, int n)
{
    rbe_status st = validate_items(b, items, n);
    if (st != RBE_OK) return st;
    // the pinned descriptors may still be read by the previous evaluation's copies (during a
    // capture nothing executes, so nothing to wait for)
    if (b->upload_pending && !capturing(b->stream)) {
        cudaError_t e = cudaEventSynchronize(b->upload_ev);
        if (e != cudaSuccess) return bcuda(b, e, "cudaEventSynchronize");
        b->upload_pending = false;
    }
    for (int r = 0; r < n; ++r)
        for (int t = 0; t < 3; ++t) b->h_boxes[3 * r + t] = items[r].box[t];
    if ((int)b->last_boxes.size() > 3 * n) b->last_boxes.resize(3 * (size_t)n);
    return plan(b, items, n);
}

void free_batch(rbe_batch b)
{
    for (void* p : {(void*)b->d_items, (void*)b->d_boxes, (void*)b->d_which, (void*)b->d_ks, (void*)b->d_cum,
                    (void*)b->d_m, (void*)b->d_w, (void*)b->d_rho, (void*)b->d_terms, (void*)b->d_coef_m,
                    (void*)b->d_coef_f, (void*)b->d_status, (void*)b->d_part, (void*)b->d_rtiles,
                    (void*)b->d_ftiles})
        if (p) cudaFree(p);
    if (b->h_items) cudaFreeHost(b->h_items);
    if (b->h_boxes) cudaFreeHost(b->h_boxes);
    if (b->h_which) cudaFreeHost(b->h_which);
    if (b->upload_ev) cudaEventDestroy(b->upload_ev);
}

}  // namespace

extern "C" {

rbe_status rbe_batch_create(double alpha, int32_t P, int32_t max_items, double max_box, rbe_batch* out)
{
    if (!out) return fail(nullptr, RBE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!(alpha > 0.0) || !std::isfinite(alpha) || P < 1 || P > 65536 || max_items < 1 || max_items > 65536 ||
        !(max_box > 0.0) || !std::isfinite(max_box) || (int64_t)max_items * (P + 1) > INT32_MAX)
        return fail(nullptr, RBE_EINVAL, "invalid batch parameters");
    const int M = host_axis_M(alpha, max_box);
    if (M > (1 << 20)) return fail(nullptr, RBE_EINVAL, "alpha max_box^2 too large for the tables");
    rbe_batch b = new (std::nothrow) rbe_batch_s();
    if (!b) return fail(nullptr, RBE_ENOMEM, "host allocation failed");
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    b->alpha = alpha;
    b->P = P;
    b->max_items = max_items;
    b->cap = 2 * M + 1;
    default_tiles(b);
    const size_t R = (size_t)max_items;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    A((void**)&b->d_items, sizeof(BItem) * R);
    A((void**)&b->d_boxes, sizeof(double) * 3 * R);
    A((void**)&b->d_which, sizeof(int) * R);
    A((void**)&b->d_ks, sizeof(KState) * R);
    A((void**)&b->d_cum, sizeof(unsigned long long) * 3 * (size_t)b->cap * R);
    A((void**)&b->d_m, sizeof(int4) * P * R);
    A((void**)&b->d_w, sizeof(double) * P * R);
    A((void**)&b->d_rho, sizeof(double2) * P * R);
    A((void**)&b->d_terms, sizeof(double) * 8 * (size_t)(P + 1) * R);
    A((void**)&b->d_coef_m, sizeof(int4) * P * R);
    A((void**)&b->d_coef_f, sizeof(float4) * P * R);
    A((void**)&b->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_items, sizeof(BItem) * R);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_boxes, sizeof(double) * 3 * R);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_which, sizeof(int) * R);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->upload_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        cudaFuncSetAttribute(k_bforce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kForceSmemPerK * kForceStageK));
        b->force_grid_per_sm = resident_blocks(k_bforce, kForceThreads, (size_t)kForceSmemPerK * std::min(P, kForceStageK));
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        std::string msg = std::string("rbe_batch_create: ") + cudaGetErrorString(e);
        free_batch(b);
        delete b;
        return fail(nullptr, e == cudaErrorMemoryAllocation ? RBE_ENOMEM : RBE_ECUDA, msg);
    }
    *out = b;
    return RBE_OK;
}

rbe_status rbe_batch_destroy(rbe_batch b)
{
    if (!b) return RBE_OK;
    BatchDevice g(b->device);
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
    return RBE_OK;
}

rbe_status rbe_batch_set_stream(rbe_batch b, void* stream)
{
    if (!b) return RBE_EINVAL;
    BatchDevice g(b->device);
    cudaStreamSynchronize(b->stream);
    b->stream = static_cast<cudaStream_t>(stream);
    return RBE_OK;
}

rbe_status rbe_batch_set_tiles(rbe_batch b, int32_t rho_k, int32_t rho_chunk, int32_t force_block)
{
    if (!b) return RBE_EINVAL;
    if (rho_k == 0 && rho_chunk == 0 && force_block == 0) {
        default_tiles(b);
        return RBE_OK;
    }
    if (!valid_tiles(b->P, rho_k, rho_chunk, force_block))
        return bfail(b, RBE_EINVAL, "tiles: rho_k a multiple of 32 in [32, 256], rho_chunk >= 32, "
                                    "force_block a positive multiple of 128");
    b->rho_k = rho_k;
    b->rho_chunk = rho_chunk;
    b->force_block = force_block;
    return RBE_OK;
}

rbe_status rbe_batch_get_tiles(rbe_batch b, int32_t* rho_k, int32_t* rho_chunk, int32_t* force_block)
{
    if (!b) return RBE_EINVAL;
    if (rho_k) *rho_k = b->rho_k;
    if (rho_chunk) *rho_chunk = b->rho_chunk;
    if (force_block) *force_block = b->force_block;
    return RBE_OK;
}

rbe_status rbe_kspace_forces_virial_batched(rbe_batch b, const rbe_batch_item* items, int32_t n)
{
    if (!b) return RBE_EINVAL;
    BatchDevice g(b->device);
    rbe_status st = prepare(b, items, n);
    if (st != RBE_OK) return st;
    return launch(b, n, 31);
}

rbe_status rbe_batch_autotune(rbe_batch b, const rbe_batch_item* items, int32_t n, int32_t reps, double* best_ms)
{
    if (!b) return RBE_EINVAL;
    if (reps < 1 || reps > 1000) return bfail(b, RBE_EINVAL, "reps must be 1..1000");
    BatchDevice g(b->device);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return bfail(b, RBE_ECUDA, "cudaEventCreate");
    }
    auto time_pass = [&](int mask, float* ms) -> rbe_status {
        rbe_status st = launch(b, n, mask);  // warm-up (and the plan's first use)
        if (st != RBE_OK) return st;
        cudaEventRecord(e0, b->stream);
        for (int k = 0; k < reps && st == RBE_OK; ++k) st = launch(b, n, mask);
        cudaEventRecord(e1, b->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (st != RBE_OK) return st;
        if (e != cudaSuccess) return bcuda(b, e, "autotune timing");
        cudaEventElapsedTime(ms, e0, e1);
        *ms /= (float)reps;
        return RBE_OK;
    };
    const int rho_ks[] = {32, 64, 96, 128, 192, 256};
    const int chunks[] = {64, 128, 256, 512, 1024, 2048};
    const int fblocks[] = {128, 256, 512, 1024, 2048};
    rbe_status st = RBE_OK;
    float best_rho = 1e30f, best_force = 1e30f;
    int bk = b->rho_k, bc = b->rho_chunk, bf = b->force_block;
    // a full evaluation with the current shapes gives the frequencies and coefficients the
    // timed passes read
    st = prepare(b, items, n);
    if (st == RBE_OK) st = launch(b, n, 31);
    for (int k : rho_ks) {
        if (st != RBE_OK) break;
        const int ktiles = (b->P + k - 1) / k;
        if (k - ((b->P + ktiles - 1) / ktiles) >= 32) continue;  // a whole idle warp per tile
        for (int c : chunks) {
            b->rho_k = k;
            b->rho_chunk = c;
            b->force_block = bf;
            float ms = 0.f;
            if ((st = prepare(b, items, n)) != RBE_OK || (st = time_pass(4, &ms)) != RBE_OK) break;
            if (ms < best_rho) {
                best_rho = ms;
                bk = k;
                bc = c;
            }
        }
    }
    for (int f : fblocks) {
        if (st != RBE_OK) break;
        b->rho_k = bk;
        b->rho_chunk = bc;
        b->force_block = f;
        float ms = 0.f;
        if ((st = prepare(b, items, n)) != RBE_OK || (st = time_pass(16, &ms)) != RBE_OK) break;
        if (ms < best_force) {
            best_force = ms;
            bf = f;
        }
    }
    b->rho_k = bk;
    b->rho_chunk = bc;
    b->force_block = bf;
    float full = 0.f;
    if (st == RBE_OK && (st = prepare(b, items, n)) == RBE_OK) st = time_pass(31, &full);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == RBE_OK && best_ms) *best_ms = full;
    return st;
}

rbe_status rbe_batch_sync(rbe_batch b)
{
    if (!b) return RBE_EINVAL;
    BatchDevice g(b->device);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize");
    unsigned bits = 0;
    e = cudaMemcpy(&bits, b->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "read status");
    if (bits) {
        cudaMemset(b->d_status, 0, sizeof(unsigned));
        if (bits & kStatusSample) return bfail(b, RBE_ESAMPLE, "a frequency stayed m = 0 after 2^20 redraws");
        if (bits & kStatusTable) return bfail(b, RBE_ESTATE, "sampling table capacity exceeded");
        return bfail(b, RBE_ENONFINITE, "rho(k) or an output is not finite");
    }
    return RBE_OK;
}

const char* rbe_batch_last_error(rbe_batch b) { return b ? b->last_error.c_str() : ""; }

}  // extern "C"
