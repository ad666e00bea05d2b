// Batched RBE k-space evaluation: many systems of uneven N in one persistent launch.
//
// Each item is one system (its own positions, charges, box, Philox key and batch index) with
// the batch's alpha and P, on the FP32-phase path with compensated FP32 accumulation inside
// a staged tile (RBE_RHO_COMP32) and FP64 energy and virial terms.  One evaluation is one
// cooperative launch of k_batch whose blocks stay resident and run five passes, with a grid
// barrier (bounded wait) between consecutive passes (after the tables pass only when it has
// tables to rebuild):
//   tables   one unit per item whose box changed (or lives on the device): tables and box
//            constants                                                           (H1)
//   sample   units of 256 frequencies per item                                   (H2)
//   rho      the work list of (item, frequency tile, particle chunk) tiles: partial rho(k)
//            per chunk                                                           (H4)
//   reduce   groups of 32 (item, frequency) rows: rho(k), terms, force coefficients
//                                                                                (H3, H6)
//   force    the work list of (item, particle block) tiles, then one final-sum unit per item:
//            forces, virial, energies                                            (H5, H6)
// The tiles run the single-system kernels' bodies (rbe_kspace_tiles.cuh).  Tile shapes
// (frequencies per rho tile, particles per rho chunk, particles per force block) are the
// batch's, set by hand or by rbe_batch_autotune, which times the candidate shapes on the
// caller's items pass by pass.  An item's result depends only on its own inputs and the tile
// shapes, never on the other items (fixed-order sums inside the item's tiles).  With
// persistence off the five passes are five launches of kernels compiled one per pass (the
// same bodies, so the same results bit for bit): each needs fewer registers than the fused
// kernel, so more of its blocks stay resident.
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
    const double* box_dev;                // the item's box in device memory (read every evaluation), or NULL
    const unsigned long long* step_dev;   // the item's batch index in device memory, or NULL: `step`
    unsigned* status;                     // where the item's device errors are latched
    int64_t N;
    uint64_t seed, step;
    int64_t chunk_len, per_block;
    int64_t part_off;  // float4 offset of the item's (P + 1) x nchunks partials
    int nchunks, fblocks;
};

// Every batched kernel runs blocks of kBThreads threads; a sampling unit covers kSampleBlock
// frequencies of one item.
constexpr int kBThreads = kForceThreads;
constexpr int kForceTileUnit = 128;  // force tiles are multiples of this many particles
constexpr int kSampleBlock = kBThreads;
constexpr int kMinRhoK = 16;        // fewest frequency lanes of a rho tile (at most 16 sub-streams)
constexpr int kRhoKCandidates = 6;  // frequency-tile shapes the autotuner times
// Bounded wait of the grid barrier: one second by the GPU's global timer (and at most
// kBarrierSpins polls), then the block gives up and the evaluation reports RBE_ETIMEOUT.
constexpr unsigned long long kBarrierNs = 1000000000ull;
constexpr int kBarrierSpins = 1 << 24;
// unroll of the force pass's frequency loop in the batched kernel, whose registers are shared by
// all five passes
#ifndef RBE_BATCH_FORCE_LUNROLL
#define RBE_BATCH_FORCE_LUNROLL 2
#endif
constexpr int kBatchForceUnroll = RBE_BATCH_FORCE_LUNROLL;

struct GridBar {
    unsigned count;     // blocks arrived at the current barrier
    unsigned pad[31];   // (the count and the generation on lines of their own)
    unsigned gen;       // barriers completed
};

// Everything the five passes of one batched evaluation read and write.
struct BArgs {
    const BItem* items;
    int n, P;
    const double* boxes;        // host-given boxes (3 per item)
    const int* which;           // items whose tables are rebuilt
    int nw;
    double alpha;
    unsigned long long* cum;    // per item: 3 x cap cumulative weights
    int cap, smem_cap;
    KState* ks;
    int bpi;                    // sampling units per item
    int4* m;
    double* w;
    const int4* rtiles;         // (item, frequency tile, chunk)
    int nrt, S, T, F;           // rho tiles; particle sub-streams of a rho block (kBThreads / T),
                                // frequency lanes of each (T = rho_k) and frequencies per lane (rho_f)
    float4* part;
    double2* rho;
    double* terms;
    int4* coef_m;
    float4* coef_f;
    const int2* ftiles;         // (item, particle block)
    int nft;
    unsigned* status;
    GridBar* bar;
    int bar_extra;              // test hook: arrivals the barriers wait for beyond the grid (0)
};

// Grid-wide barrier of a cooperative launch with a bounded wait.  Thread 0 of each block reads
// the generation, then arrives with an acquire-release add on the count (its block's writes,
// ordered before it by the block barrier and a fence, are visible to whoever observes the
// arrival); the last block to arrive resets the count and advances the generation with an
// acquire-release add; the others poll the generation with acquire loads and a short back-off.
// Returns false, after latching kStatusTimeout, when the other blocks did not all arrive within
// kBarrierSpins polls: the caller then leaves the kernel, and the other blocks' later barriers
// time out in turn.  The words are zeroed before every launch.
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_sync(GridBar* bar, unsigned nblocks, unsigned* status)
{
    __shared__ unsigned ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned good = 1u;
        __threadfence();
        const unsigned g = ld_acquire(&bar->gen);
        if (atom_add_acq_rel(&bar->count, 1u) + 1u == nblocks) {
            bar->count = 0u;  // ordered before the release below
            atom_add_acq_rel(&bar->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            for (int it = 0; ld_acquire(&bar->gen) == g; ++it) {
                if (it >= kBarrierSpins || global_ns() - t0 > kBarrierNs) {
                    good = 0u;
                    atomicOr(status, kStatusTimeout);
                    break;
                }
                __nanosleep(32);
            }
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0u;
}

// The passes (Sec. 4.2 for each item), each a loop of units over the blocks of the grid.
__device__ __forceinline__ void pass_tables(const BArgs& a)
{
    for (int w = blockIdx.x; w < a.nw; w += gridDim.x) {
        const int r = a.which[w];
        const double* b = a.boxes + 3 * (size_t)r;
        tables_body(b[0], b[1], b[2], a.items[r].box_dev, a.alpha, a.P, a.cum + (size_t)r * 3 * a.cap, a.cap, a.ks + r,
                    a.items[r].status);
        __syncthreads();
    }
}

__device__ __forceinline__ void pass_sample(const BArgs& a)
{
    for (int u = blockIdx.x; u < a.n * a.bpi; u += gridDim.x) {
        const int r = u / a.bpi, lb = (u % a.bpi) * kSampleBlock;
        const BItem& it = a.items[r];
        sample_body(lb, it.seed, it.step, it.step_dev, a.P, a.P, a.cum + (size_t)r * 3 * a.cap, a.cap, a.smem_cap,
                    a.ks + r, a.m + (size_t)r * a.P, a.w + (size_t)r * a.P, it.status);
        __syncthreads();
    }
}

// F frequencies per lane (a.F): with two, one broadcast particle record feeds two pairs
template <int F>
__device__ __forceinline__ void pass_rho_f(const BArgs& a)
{
    for (int t = blockIdx.x; t < a.nrt; t += gridDim.x) {
        const int4 tl = a.rtiles[t];
        const BItem& it = a.items[tl.x];
        rho_f32_tile<RBE_RHO_COMP32, F, false, kBThreads>(tl.y, tl.z, it.pos, it.q, it.N, a.ks + tl.x,
                                                          a.m + (size_t)tl.x * a.P, a.P, it.chunk_len, it.nchunks,
                                                          a.part + it.part_off, it.status, a.S, a.T);
        __syncthreads();
    }
}

__device__ __forceinline__ void pass_rho(const BArgs& a)
{
    if (a.F == 2)  // the same for every block
        pass_rho_f<2>(a);
    else
        pass_rho_f<1>(a);
}

// (item, frequency) rows u = r (P + 1) + l in groups of 32 per block: each warp sums four rows
// (warp_row_sum), then the lanes of warp 0 form the 32 rows' FP64 terms and coefficients at
// once (GB300 issues a warp's FP64 instruction at about two lanes per clock, so one FP64 chain
// per row and warp would queue on the FP64 unit).
constexpr int kReduceRowsPerWarp = 4;
constexpr int kReduceGroup = kReduceRowsPerWarp * kBThreads / 32;
static_assert(kReduceGroup == 32, "one row per lane of the finishing warp");

// JOINT: a warp's rows summed together (the per-pass kernel, given the registers for it) or one
// after the other (the persistent kernel, whose registers all five passes share); the same bits.
template <bool JOINT>
__device__ __forceinline__ void pass_reduce(const BArgs& a)
{
    __shared__ double2 srho[kReduceGroup];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rows = a.n * (a.P + 1);
    for (int base = blockIdx.x * kReduceGroup; base < rows; base += gridDim.x * kReduceGroup) {
        // warp 0's lanes: the factors of their rows that do not depend on rho, meanwhile
        int4 mi = make_int4(0, 0, 0, 0);
        double c[8];
        const int uf = base + lane;
        if (warp == 0 && uf < rows) {
            const int r = uf / (a.P + 1), l = uf % (a.P + 1);
            if (l < a.P) {
                const size_t o = (size_t)r * a.P;
                mi = a.m[o + l];
                freq_pre(mi, a.w[o + l], a.ks + r, c);
            }
        }
        if (!JOINT) {  // the warp's rows one after the other
#pragma unroll 1
            for (int i = 0; i < kReduceRowsPerWarp; ++i) {
                const int j = warp * kReduceRowsPerWarp + i, u = base + j;
                if (u >= rows) break;
                const int r = u / (a.P + 1), l = u % (a.P + 1);
                const BItem& it = a.items[r];
                const double2 v = warp_row_sum(a.part + it.part_off + (size_t)l * it.nchunks, it.nchunks);
                if (lane == 0) srho[j] = v;
            }
        } else {
            // the warp's rows summed together, so that the loads of all of them are in flight at
            // once; each row's own order is warp_row_sum's (lane-strided float-float sums over the
            // chunks, then the same shuffle tree), so a row's sum does not depend on its neighbours
            const float4* rowp[kReduceRowsPerWarp];
            int nch[kReduceRowsPerWarp], nmax = 0;
            float rh[kReduceRowsPerWarp], rl[kReduceRowsPerWarp], ih[kReduceRowsPerWarp], il[kReduceRowsPerWarp];
#pragma unroll
            for (int i = 0; i < kReduceRowsPerWarp; ++i) {
                const int u = base + warp * kReduceRowsPerWarp + i;
                rowp[i] = a.part;
                nch[i] = 0;
                if (u < rows) {
                    const int r = u / (a.P + 1), l = u % (a.P + 1);
                    const BItem& it = a.items[r];
                    rowp[i] = a.part + it.part_off + (size_t)l * it.nchunks;
                    nch[i] = it.nchunks;
                }
                nmax = max(nmax, nch[i]);
                rh[i] = rl[i] = ih[i] = il[i] = 0.f;
            }
            for (int j = lane; j < nmax; j += 32) {
#pragma unroll
                for (int i = 0; i < kReduceRowsPerWarp; ++i) {
                    if (j < nch[i]) {
                        const float4 v = rowp[i][j];
                        ff_add2(rh[i], rl[i], v.x, v.y);
                        ff_add2(ih[i], il[i], v.z, v.w);
                    }
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                for (int i = 0; i < kReduceRowsPerWarp; ++i) {
                    const float x0 = __shfl_xor_sync(0xffffffffu, rh[i], off), x1 = __shfl_xor_sync(0xffffffffu, rl[i], off);
                    const float x2 = __shfl_xor_sync(0xffffffffu, ih[i], off), x3 = __shfl_xor_sync(0xffffffffu, il[i], off);
                    ff_add2(rh[i], rl[i], x0, x1);
                    ff_add2(ih[i], il[i], x2, x3);
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < kReduceRowsPerWarp; ++i)
                    if (nch[i] > 0)
                        srho[warp * kReduceRowsPerWarp + i] =
                            make_double2(ff_to_double(rh[i], rl[i]), ff_to_double(ih[i], il[i]));
            }
        }
        __syncthreads();
        if (warp == 0 && uf < rows) {
            const int r = uf / (a.P + 1), l = uf % (a.P + 1);
            const size_t o = (size_t)r * a.P;
            row_finish(l, a.P, srho[lane].x, srho[lane].y, mi, c, a.rho + o, a.terms + (size_t)r * (a.P + 1) * 8,
                       a.coef_m + o, a.coef_f + o, a.items[r].status);
        }
        __syncthreads();
    }
}

// tiles [0, nft) are (item, particle block); tiles [nft, nft + n) the per-item energy and
// virial sums
// LU: unroll of the frequency loop (the per-pass kernel takes the single-system unroll; the
// persistent kernel, whose registers all five passes share, a shorter one)
template <int LU>
__device__ __forceinline__ void pass_force(const BArgs& a)
{
    for (int t = blockIdx.x; t < a.nft + a.n; t += gridDim.x) {
        if (t < a.nft) {
            const int2 tl = a.ftiles[t];
            const BItem& it = a.items[tl.x];
            const size_t o = (size_t)tl.x * a.P;
            force_f32_block<false, LU>((int64_t)tl.y, it.pos, it.q, it.N, it.per_block, a.ks + tl.x,
                                                      a.coef_m + o, a.coef_f + o, a.P, it.F, it.status);
        } else {
            const int r = t - a.nft;
            const BItem& it = a.items[r];
            final_sums(a.terms + (size_t)r * (a.P + 1) * 8, a.P, a.ks + r, it.W, it.E, it.status);
        }
        __syncthreads();
    }
}

// The batched evaluation in one launch, the persistent form: a cooperative launch whose blocks
// all stay resident and run the five passes with a grid barrier between consecutive passes.
// Written as straight-line code (not a loop over the passes), the fused kernel fits three
// blocks of 256 threads per SM without spilling.
#ifndef RBE_BATCH_MINB
#define RBE_BATCH_MINB 3
#endif
__global__ void __launch_bounds__(kBThreads, RBE_BATCH_MINB) k_batch(BArgs a)
{
    const unsigned nb = gridDim.x + (unsigned)a.bar_extra;
    if (a.nw > 0) {  // tables to rebuild (the same for every block): the sampler waits for them
        pass_tables(a);
        if (!grid_sync(a.bar, nb, a.status)) return;
    }
    pass_sample(a);
    if (!grid_sync(a.bar, nb, a.status)) return;
    pass_rho(a);
    if (!grid_sync(a.bar, nb, a.status)) return;
    pass_reduce<false>(a);
    if (!grid_sync(a.bar, nb, a.status)) return;
    pass_force<kBatchForceUnroll>(a);
}

// The same passes as launches of their own (persistence off): each pass compiled alone needs 60
// to 86 registers (tables 86), not the fused kernel's 128, so four blocks of 256 threads stay
// resident per SM instead of two.
#ifndef RBE_BATCH_PASS_MINB
#define RBE_BATCH_PASS_MINB 4
#endif
__global__ void __launch_bounds__(kBThreads, 2) k_btables(BArgs a) { pass_tables(a); }
__global__ void __launch_bounds__(kBThreads, RBE_BATCH_PASS_MINB) k_bsample(BArgs a) { pass_sample(a); }
__global__ void __launch_bounds__(kBThreads, RBE_BATCH_PASS_MINB) k_brho(BArgs a) { pass_rho_f<1>(a); }
__global__ void __launch_bounds__(kBThreads, RBE_BATCH_PASS_MINB) k_brho2(BArgs a) { pass_rho_f<2>(a); }
__global__ void __launch_bounds__(kBThreads, 2) k_breduce(BArgs a) { pass_reduce<true>(a); }
__global__ void __launch_bounds__(kBThreads, RBE_BATCH_PASS_MINB) k_bforce(BArgs a) { pass_force<kForceLUnroll>(a); }

using PassKernel = void (*)(BArgs);
// the five passes in order, then the rho pass with two frequencies per lane
static const PassKernel kPassKernels[6] = {k_btables, k_bsample, k_brho, k_breduce, k_bforce, k_brho2};

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
    // tile shapes (rho_k frequency lanes of rho_f frequencies each per rho tile)
    int rho_k = 0, rho_f = 1, rho_chunk = 0, force_block = 0;
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
    int plan_k = -1, plan_f = -1, plan_chunk = -1, plan_fb = -1;
    int n_rtiles = 0, n_ftiles = 0;
    std::vector<int4> h_rtiles;
    std::vector<int2> h_ftiles;
    int grid_per_sm = 1;      // resident blocks of k_batch per SM (the persistent grid)
    int pass_per_sm[6] = {1, 1, 1, 1, 1, 1};  // resident blocks per SM of each pass kernel
    size_t pass_smem[6] = {0, 0, 0, 0, 0, 0};  // their dynamic shared memory
    GridBar* d_bar = nullptr;  // the grid barrier of the persistent launch
    bool persistent = true;    // one cooperative launch per evaluation (else one launch per pass)
    int bar_extra = 0;         // test hook of the barriers' timeout (rbe_batch_test_barrier_timeout)
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
    // a rho tile of rho_k frequencies fills a block of kBThreads threads with kBThreads / rho_k
    // particle sub-streams (the threads beyond them idle)
    return rho_k >= kMinRhoK && rho_k <= kBThreads && rho_chunk >= 32 && rho_chunk <= (1 << 24) &&
           force_block >= kForceTileUnit && force_block % kForceTileUnit == 0 && force_block <= (1 << 24) && P >= 1;
}

// Busy fraction of a rho block's lanes with frequency tiles of k lanes of f frequencies: the
// tiles' share of real frequencies times the share of the block's threads in whole sub-streams.
static double rho_lane_efficiency(int P, int k, int f)
{
    const int ktiles = (P + k * f - 1) / (k * f);
    const int S = kBThreads / k;
    return (double)P / ((double)ktiles * k * f) * (double)(S * k) / kBThreads;
}

// Frequency-tile candidates for the autotuner: P split evenly into 1 to 16 tiles (lane counts
// that need not be powers of two: P = 100 as two tiles of 50 lanes in five sub-streams keeps
// 250 of 256 threads on real frequencies) and the powers of two 32 to 256; at most
// kRhoKCandidates of them, ranked by lane efficiency less 0.01 per frequency tile (every tile
// stages and converts the particles again).  The pass is bound by instruction issue, so the
// busier lanes pay for the extra re-staging and sub-streams rather than run faster (measured
// at P = 100: 50-lane and 128-lane tiles equal); the timing decides.
static double rho_k_score(int P, int k, int f)
{
    return rho_lane_efficiency(P, k, f) - 0.01 * ((P + k * f - 1) / (k * f));
}

// Lane counts for tiles of f frequencies per lane (a tile covers k f frequencies).
static std::vector<int> rho_k_candidates(int P, int f = 1)
{
    std::vector<int> ks;
    for (int kt = 1; kt <= 16; ++kt) {
        const int k = (P + kt * f - 1) / (kt * f);
        if (k >= kMinRhoK && k <= kBThreads) ks.push_back(k);
    }
    for (int k : {32, 64, 128, 256}) ks.push_back(k);
    std::sort(ks.begin(), ks.end());
    ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
    std::stable_sort(ks.begin(), ks.end(), [P, f](int x, int y) {
        const double sx = rho_k_score(P, x, f), sy = rho_k_score(P, y, f);
        if (sx != sy) return sx > sy;
        return x > y;
    });
    if ((int)ks.size() > kRhoKCandidates) ks.resize(kRhoKCandidates);
    return ks;
}

// The tile shapes the planner uses when none were set: the frequency tile of the best lane
// efficiency, chunks of 256 particles.
void default_tiles(rbe_batch b)
{
    b->rho_f = 1;
    b->rho_k = rho_k_candidates(b->P, b->rho_f).front();
    b->rho_chunk = 256;
    b->force_block = 4 * kForceTileUnit;  // a round of kForceRound particles for each of the block's warps
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
        if ((reinterpret_cast<uintptr_t>(it.box_dev) | reinterpret_cast<uintptr_t>(it.step_dev)) % 8 ||
            reinterpret_cast<uintptr_t>(it.status_dev) % 4)
            return bfail(b, RBE_EINVAL, "item box_dev and step_dev must be 8-byte, status_dev 4-byte aligned");
    }
    return RBE_OK;
}

// Work lists and item descriptors for the current items and tile shapes (rebuilt only when
// the N of some item or a tile shape changed).
rbe_status plan(rbe_batch b, const rbe_batch_item* items, int n)
{
    bool same = (int)b->plan_N.size() == n && b->plan_k == b->rho_k && b->plan_f == b->rho_f &&
                b->plan_chunk == b->rho_chunk && b->plan_fb == b->force_block;
    for (int r = 0; same && r < n; ++r) same = b->plan_N[r] == items[r].N;
    if (!same) {
        if (capturing(b->stream))
            return bfail(b, RBE_ESTATE, "new item sizes or tiles during stream capture: evaluate these items once "
                                        "outside capture first");
        b->h_rtiles.clear();
        b->h_ftiles.clear();
        b->plan_N.assign(n, 0);
        const int ktiles = (b->P + b->rho_k * b->rho_f - 1) / (b->rho_k * b->rho_f);
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
        b->plan_f = b->rho_f;
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
        it.box_dev = items[r].box_dev;
        it.step_dev = reinterpret_cast<const unsigned long long*>(items[r].step_dev);
        it.status = items[r].status_dev ? reinterpret_cast<unsigned*>(items[r].status_dev) : b->d_status;
    }
    return RBE_OK;
}

// One evaluation: the passes in `mask` (1 tables, 2 sample, 4 rho, 8 reduce, 16 force; the
// tuner times one pass at a time).  All five: one persistent cooperative launch of k_batch
// (grid barriers between the passes), or, with persistence off, one launch per pass.
rbe_status launch(rbe_batch b, int n, int mask)
{
    cudaStream_t s = b->stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->d_items, b->h_items, sizeof(BItem) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return bcuda(b, e, "upload items");
    const bool cap = capturing(s);
    const int P = b->P;
    int nw = 0;
    if (mask & 1) {
        // tables of the items whose host box changed since the last evaluation, and of every item
        // whose box lives on the device
        for (int r = 0; r < n; ++r) {
            const double* bx = b->h_boxes + 3 * (size_t)r;
            const bool changed = b->last_boxes.size() < 3 * (size_t)(r + 1) || b->last_boxes[3 * r] != bx[0] ||
                                 b->last_boxes[3 * r + 1] != bx[1] || b->last_boxes[3 * r + 2] != bx[2];
            if (changed || b->h_items[r].box_dev) b->h_which[nw++] = r;
        }
        if (nw > 0 &&
            ((e = cudaMemcpyAsync(b->d_boxes, b->h_boxes, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s)) !=
                 cudaSuccess ||
             (e = cudaMemcpyAsync(b->d_which, b->h_which, sizeof(int) * nw, cudaMemcpyHostToDevice, s)) != cudaSuccess))
            return bcuda(b, e, "upload boxes");
        b->last_boxes.assign(b->h_boxes, b->h_boxes + 3 * (size_t)n);
    }
    // the pinned descriptors (and boxes) may be overwritten once these copies have run
    if (!cap) {
        if ((e = cudaEventRecord(b->upload_ev, s)) != cudaSuccess) return bcuda(b, e, "cudaEventRecord");
        b->upload_pending = true;
    }
    BArgs a;
    a.items = b->d_items;
    a.n = n;
    a.P = P;
    a.boxes = b->d_boxes;
    a.which = b->d_which;
    a.nw = nw;
    a.alpha = b->alpha;
    a.cum = b->d_cum;
    a.cap = b->cap;
    const size_t table_smem = sizeof(unsigned long long) * 3 * (size_t)b->cap;
    a.smem_cap = table_smem <= 48 * 1024 ? b->cap : 0;
    a.ks = b->d_ks;
    a.bpi = (P + kSampleBlock - 1) / kSampleBlock;
    a.m = b->d_m;
    a.w = b->d_w;
    a.rtiles = b->d_rtiles;
    a.nrt = b->n_rtiles;
    a.S = kBThreads / b->rho_k;
    a.T = b->rho_k;
    a.F = b->rho_f;
    a.part = b->d_part;
    a.rho = b->d_rho;
    a.terms = b->d_terms;
    a.coef_m = b->d_coef_m;
    a.coef_f = b->d_coef_f;
    a.ftiles = b->d_ftiles;
    a.nft = b->n_ftiles;
    a.status = b->d_status;
    a.bar = b->d_bar;
    a.bar_extra = b->bar_extra;
    const size_t smem = std::max(a.smem_cap ? table_smem : 0, (size_t)kForceSmemPerK * std::min(P, kForceStageK));
    const int resident = std::max(1, b->num_sms * b->grid_per_sm);
    if (mask == 31 && b->persistent) {
        // the barrier words start at zero for every launch (a launch that timed out leaves them set)
        if ((e = cudaMemsetAsync(b->d_bar, 0, sizeof(GridBar), s)) != cudaSuccess) return bcuda(b, e, "barrier reset");
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(resident);
        cfg.blockDim = dim3(kBThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if ((e = cudaLaunchKernelEx(&cfg, k_batch, a)) != cudaSuccess)
            return bcuda(b, e, "persistent batched k-space launch");
        return RBE_OK;
    }
    const int units[5] = {nw, n * a.bpi, a.nrt, (n * (P + 1) + kReduceGroup - 1) / kReduceGroup, a.nft + n};
    for (int k = 0; k < 5; ++k) {
        if (!(mask & (1 << k)) || units[k] == 0) continue;
        const int kk = k == 2 && a.F == 2 ? 5 : k;
        const int grid = std::max(1, std::min(units[k], b->num_sms * b->pass_per_sm[kk]));
        kPassKernels[kk]<<<grid, kBThreads, b->pass_smem[kk], s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return bcuda(b, e, "batched k-space pass");
    }
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
                    (void*)b->d_ftiles, (void*)b->d_bar})
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
    A((void**)&b->d_bar, sizeof(GridBar));
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_bar, 0, sizeof(GridBar));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_items, sizeof(BItem) * R);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_boxes, sizeof(double) * 3 * R);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_which, sizeof(int) * R);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->upload_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        // dynamic shared memory: the sampler's tables (when they fit 48 KB) or the force pass's
        // staged frequencies; the persistent grid is every block that fits at once
        const size_t tsm = sizeof(unsigned long long) * 3 * (size_t)b->cap;
        const size_t smem = std::max(tsm <= 48 * 1024 ? tsm : 0, (size_t)kForceSmemPerK * std::min(P, kForceStageK));
        cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        b->grid_per_sm = resident_blocks(k_batch, kBThreads, smem);
        // the pass kernels: the tables and the sampler take the tables' shared memory, the force
        // pass its staged frequencies
        const size_t ts = tsm <= 48 * 1024 ? tsm : 0;
        const size_t psm[6] = {ts, ts, 0, 0, (size_t)kForceSmemPerK * std::min(P, kForceStageK), 0};
        for (int k = 0; k < 6; ++k) {
            b->pass_smem[k] = psm[k];
            cudaFuncSetAttribute(kPassKernels[k], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm[k]);
            b->pass_per_sm[k] = resident_blocks(kPassKernels[k], kBThreads, psm[k]);
        }
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
        return bfail(b, RBE_EINVAL, "tiles: rho_k in [16, 256], rho_chunk >= 32, "
                                    "force_block a positive multiple of 128");
    b->rho_k = rho_k;
    b->rho_chunk = rho_chunk;
    b->force_block = force_block;
    return RBE_OK;
}

rbe_status rbe_batch_set_persistent(rbe_batch b, int32_t enable)
{
    if (!b) return RBE_EINVAL;
    if (enable != 0 && enable != 1) return bfail(b, RBE_EINVAL, "enable must be 0 or 1");
    b->persistent = enable == 1;
    return RBE_OK;
}

rbe_status rbe_batch_test_barrier_timeout(rbe_batch b, int32_t enable)
{
    if (!b) return RBE_EINVAL;
    if (enable != 0 && enable != 1) return bfail(b, RBE_EINVAL, "enable must be 0 or 1");
    b->bar_extra = enable;
    return RBE_OK;
}

rbe_status rbe_batch_set_rho_f(rbe_batch b, int32_t rho_f)
{
    if (!b) return RBE_EINVAL;
    if (rho_f != 1 && rho_f != 2) return bfail(b, RBE_EINVAL, "rho_f must be 1 or 2");
    b->rho_f = rho_f;
    return RBE_OK;
}

rbe_status rbe_batch_get_rho_f(rbe_batch b, int32_t* rho_f)
{
    if (!b || !rho_f) return RBE_EINVAL;
    *rho_f = b->rho_f;
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
    const int chunks[] = {64, 128, 256, 512, 1024, 2048};
    const int fblocks[] = {128, 256, 512, 1024, 2048};
    rbe_status st = RBE_OK;
    float best_rho = 1e30f, best_force = 1e30f;
    int bk = b->rho_k, bff = b->rho_f, bc = b->rho_chunk, bf = b->force_block;
    // a full evaluation with the current shapes gives the frequencies and coefficients the
    // timed passes read
    st = prepare(b, items, n);
    if (st == RBE_OK) st = launch(b, n, 31);
    for (int rf = 1; rf <= 2; ++rf) {
        for (int k : rho_k_candidates(b->P, rf)) {
            if (st != RBE_OK) break;
            // the chunk lengths, and whole multiples of the tile's staged particles (S sub-streams of
            // kRhoGroup-multiple shares of kRhoStage), whose chunks end on a full staged tile
            const int S = kBThreads / k, stage = S * (kRhoGroup * (kRhoStage / (kRhoGroup * S)));
            std::vector<int> cands(std::begin(chunks), std::end(chunks));
            for (int mlt : {1, 2, 4})
                if (stage * mlt >= 32 && stage * mlt <= 2048) cands.push_back(stage * mlt);
            std::sort(cands.begin(), cands.end());
            cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
            for (int c : cands) {
                b->rho_k = k;
                b->rho_f = rf;
                b->rho_chunk = c;
                b->force_block = bf;
                float ms = 0.f;
                if ((st = prepare(b, items, n)) != RBE_OK || (st = time_pass(4, &ms)) != RBE_OK) break;
                if (ms < best_rho) {
                    best_rho = ms;
                    bk = k;
                    bff = rf;
                    bc = c;
                }
            }
        }
    }
    for (int f : fblocks) {
        if (st != RBE_OK) break;
        b->rho_k = bk;
        b->rho_f = bff;
        b->rho_chunk = bc;
        b->force_block = f;
        float ms = 0.f;
        if ((st = prepare(b, items, n)) != RBE_OK || (st = time_pass(16, &ms)) != RBE_OK) break;
        if (ms < best_force) {
            best_force = ms;
            bf = f;
        }
    }
    if (b->persistent) {
        // the persistent launch runs every pass on its fewer resident blocks, where the force
        // tiles' count against the grid decides the balance: choose them on whole evaluations
        float best_full = 1e30f;
        const int bf_pass = bf;
        for (int f : fblocks) {
            if (st != RBE_OK) break;
            b->rho_k = bk;
            b->rho_f = bff;
            b->rho_chunk = bc;
            b->force_block = f;
            float ms = 0.f;
            if ((st = prepare(b, items, n)) != RBE_OK || (st = time_pass(31, &ms)) != RBE_OK) break;
            if (ms < best_full) {
                best_full = ms;
                bf = f;
            }
        }
        if (st != RBE_OK) bf = bf_pass;
    }
    b->rho_k = bk;
    b->rho_f = bff;
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
        if (bits & kStatusTimeout)
            return bfail(b, RBE_ETIMEOUT, "a grid barrier of the persistent launch gave up waiting (one second)");
        if (bits & kStatusTable) return bfail(b, RBE_ESTATE, "sampling table capacity exceeded");
        return bfail(b, RBE_ENONFINITE, "rho(k) or an output is not finite");
    }
    return RBE_OK;
}

const char* rbe_batch_last_error(rbe_batch b) { return b ? b->last_error.c_str() : ""; }

}  // extern "C"
