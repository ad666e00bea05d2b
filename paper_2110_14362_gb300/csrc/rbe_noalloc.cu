// An allocation-free variant of the frequency sampler.
//
// Some callers cannot allocate device memory at the time they need a batch: an MD engine
// that sized one device pool at start-up and forbids allocations afterwards, a plugin
// running inside a host application that owns all device memory, or a loop that must
// not call cudaMalloc because a device allocation can synchronise the whole device.
// rbe_sample_k_noalloc serves them: it needs no context, allocates nothing, and keeps
// its scratch (the three cumulative weight tables and a status word) in a file-scope
// __device__ array that every GPU which loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "rbe_context.h"
#include "rbe_device.cuh"

namespace rbe {

// Entries per axis table (2M + 1 <= kNoAllocTableCap, i.e. M <= 4095); 3 x 8191 64-bit
// integers plus a status word: 192 KB per device.
constexpr int kNoAllocTableCap = 8191;
constexpr int kNoAllocThreads = 256;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[3 * kNoAllocTableCap + 32];

// Smallest j in [0, 2M] with T < C_j, minus M.
__device__ __forceinline__ int search_int(const unsigned long long* __restrict__ row, int M, unsigned long long T)
{
    int lo = 0, hi = 2 * M;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (T < row[mid]) hi = mid;
        else lo = mid + 1;
    }
    return lo - M;
}

// One block: builds the three integer tables in the scratch array exactly as k_tables does
// (the same weights; integer prefix sums are exact in any order), then draws all P samples
// as k_sample does.  The status word at scratch[3 * cap] is cleared at the start of every
// call.
__global__ void __launch_bounds__(kNoAllocThreads)
k_sample_noalloc(unsigned long long* __restrict__ scratch, double bx, double by, double bz, double alpha, int P,
                 uint64_t seed, uint64_t step, int32_t* __restrict__ m_out, double* __restrict__ S_out)
{
    __shared__ int sM[3], sSh[3];
    __shared__ double sc[3];
    __shared__ unsigned long long wsum[kNoAllocThreads / 32];
    unsigned* status = reinterpret_cast<unsigned*>(scratch + 3 * kNoAllocTableCap);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) *status = 0u;  // the array keeps the previous call's contents
    __syncthreads();
    if (tid < 3) {
        const double ell = tid == 0 ? bx : (tid == 1 ? by : bz);
        const double c = axis_c(alpha, ell);
        bool bad;  // the host checked 2M + 1 <= kNoAllocTableCap; clamp all the same
        const int M = axis_M_capped(ell, c, kNoAllocTableCap, &bad);
        if (bad) atomicOr(status, kStatusTable);
        sc[tid] = c;
        sM[tid] = M;
        sSh[tid] = 62 - (32 - __clz((unsigned)(2 * M + 1)));
    }
    __syncthreads();
    for (int t = 0; t < 3; ++t) {
        const int M = sM[t];
        unsigned long long* row = scratch + (size_t)t * kNoAllocTableCap;
        for (int a = tid; a <= M; a += kNoAllocThreads) {
            const double v = table_exp(-__dmul_rn(sc[t], (double)a * (double)a));
            const unsigned long long W = (unsigned long long)__double2ll_rn(ldexp(v, sSh[t]));
            row[M + a] = W;
            row[M - a] = W;
        }
    }
    __syncthreads();
    for (int t = 0; t < 3; ++t) {
        const int n = 2 * sM[t] + 1;
        unsigned long long* row = scratch + (size_t)t * kNoAllocTableCap;
        const int per = (n + kNoAllocThreads - 1) / kNoAllocThreads;
        const int j0 = min(n, tid * per), j1 = min(n, j0 + per);
        unsigned long long local = 0;
        for (int j = j0; j < j1; ++j) local += row[j];
        unsigned long long incl = local;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long v = lane < kNoAllocThreads / 32 ? wsum[lane] : 0ull;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long o = __shfl_up_sync(0xffffffffu, v, off);
                if (lane >= off) v += o;
            }
            if (lane < kNoAllocThreads / 32) wsum[lane] = v;
        }
        __syncthreads();
        unsigned long long run = incl - local + (warp > 0 ? wsum[warp - 1] : 0ull);
        for (int j = j0; j < j1; ++j) {
            run += row[j];
            row[j] = run;
        }
        __syncthreads();
    }
    const unsigned long long* tx = scratch;
    const unsigned long long* ty = scratch + kNoAllocTableCap;
    const unsigned long long* tz = scratch + 2 * kNoAllocTableCap;
    const unsigned long long Cx = tx[2 * sM[0]], Cy = ty[2 * sM[1]], Cz = tz[2 * sM[2]];
    if (tid == 0) {
        const double Hx = ldexp((double)Cx, -sSh[0]), Hy = ldexp((double)Cy, -sSh[1]), Hz = ldexp((double)Cz, -sSh[2]);
        *S_out = __dsub_rn(__dmul_rn(__dmul_rn(Hx, Hy), Hz), 1.0);
    }
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t c2 = (uint32_t)step, c3 = (uint32_t)((step >> 32) & 0xFFFFFFu);
    for (int l = tid; l < P; l += kNoAllocThreads) {
        int mx = 0, my = 0, mz = 0;
        bool found = false;
        for (uint32_t attempt = 0; attempt < kMaxAttempts; ++attempt) {
            const uint4 w0 = philox4x32_10(make_uint4((uint32_t)l, 2u * attempt, c2, c3), k0, k1);
            const uint4 w1 = philox4x32_10(make_uint4((uint32_t)l, 2u * attempt + 1u, c2, c3), k0, k1);
            const unsigned long long Ux = ((unsigned long long)w0.x << 21) | (w0.y >> 11);
            const unsigned long long Uy = ((unsigned long long)w0.z << 21) | (w0.w >> 11);
            const unsigned long long Uz = ((unsigned long long)w1.x << 21) | (w1.y >> 11);
            mx = search_int(tx, sM[0], (__umul64hi(Ux, Cx) << 11) | ((Ux * Cx) >> 53));
            my = search_int(ty, sM[1], (__umul64hi(Uy, Cy) << 11) | ((Uy * Cy) >> 53));
            mz = search_int(tz, sM[2], (__umul64hi(Uz, Cz) << 11) | ((Uz * Cz) >> 53));
            if (mx != 0 || my != 0 || mz != 0) {
                found = true;
                break;
            }
        }
        if (!found) {
            atomicOr(status, kStatusSample);
            mx = 1;
            my = mz = 0;
        }
        m_out[3 * l] = mx;
        m_out[3 * l + 1] = my;
        m_out[3 * l + 2] = mz;
    }
}

// Device address of the scratch array in the CUDA context current on the calling thread
// (host code may not use the symbol itself as an address).  Looked up on every call: the
// address belongs to the context that loaded the module, and a caller may switch contexts
// (a plugin inside an application with its own driver context) or rebuild the primary
// context (cudaDeviceReset), after which an address kept from an earlier call would be stale.
// The lookup is a host-side query; it allocates nothing.
static rbe_status noalloc_scratch(unsigned long long** out, std::string& err)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        err = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
        return RBE_ECUDA;
    }
    *out = static_cast<unsigned long long*>(p);
    return RBE_OK;
}

}  // namespace rbe

using namespace rbe;

extern "C" rbe_status rbe_sample_k_noalloc(const double box[3], double alpha, int32_t P, uint64_t seed,
                                           uint64_t step, int32_t* m_out, double* S_out, void* stream)
{
    if (!box || !m_out || !S_out) return fail(nullptr, RBE_EINVAL, "box, m_out and S_out must not be NULL");
    if (!std::isfinite(alpha) || !(alpha > 0.0)) return fail(nullptr, RBE_EINVAL, "alpha must be finite and > 0");
    if (P < 1 || P > 65536) return fail(nullptr, RBE_EINVAL, "P must be in [1, 65536]");
    if ((step >> 56) != 0) return fail(nullptr, RBE_EINVAL, "step must be < 2^56");
    for (int t = 0; t < 3; ++t) {
        if (!std::isfinite(box[t]) || !(box[t] > 0.0)) return fail(nullptr, RBE_EINVAL, "box lengths must be finite and > 0");
        const double c = (kPi * kPi) / (alpha * (box[t] * box[t]));
        if (!(c <= 600.0))
            return fail(nullptr, RBE_EINVAL, "pi^2/(alpha l^2) > 600 on some axis: the frequency distribution is degenerate");
        // the device rounds the same quantities without contraction; allow one entry of slack
        if (2 * host_axis_M(alpha, box[t]) + 3 > kNoAllocTableCap)
            return fail(nullptr, RBE_EINVAL,
                        "rbe_sample_k_noalloc: alpha l^2 too large for the fixed scratch (needs |m| <= 4094 per axis; "
                        "use rbe_sample_k)");
    }
    if (reinterpret_cast<uintptr_t>(m_out) % 4 != 0 || reinterpret_cast<uintptr_t>(S_out) % 8 != 0)
        return fail(nullptr, RBE_EINVAL, "m_out must be 4-byte and S_out 8-byte aligned device memory");
    unsigned long long* scratch = nullptr;
    std::string err;
    rbe_status st = noalloc_scratch(&scratch, err);
    if (st != RBE_OK) return fail(nullptr, st, err);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_sample_noalloc<<<1, kNoAllocThreads, 0, s>>>(scratch, box[0], box[1], box[2], alpha, P, seed, step, m_out, S_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, RBE_ECUDA, std::string("k_sample_noalloc: ") + cudaGetErrorString(e));
    unsigned bits = 0;
    e = cudaMemcpyAsync(&bits, scratch + 3 * kNoAllocTableCap, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(nullptr, RBE_ECUDA, std::string("rbe_sample_k_noalloc: ") + cudaGetErrorString(e));
    if (bits & kStatusTable) return fail(nullptr, RBE_EINVAL, "rbe_sample_k_noalloc: table larger than the fixed scratch");
    if (bits & kStatusSample) return fail(nullptr, RBE_ESAMPLE, "a frequency stayed m = 0 after 2^20 redraws");
    return RBE_OK;
}
