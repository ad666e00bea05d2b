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
#include <mutex>
#include <string>

#include "rbe_context.h"
#include "rbe_device.cuh"

namespace rbe {

// Entries per axis table (2M + 1 <= kNoAllocTableCap, i.e. M <= 4095); 3 x 8191 doubles
// plus a status word: 192 KB per device.
constexpr int kNoAllocTableCap = 8191;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[3 * kNoAllocTableCap + 32];

// Smallest j in [0, 2M] with target < cdf[j], minus M, comparing the bit patterns of
// non-negative doubles (their order is the order of the values).
__device__ __forceinline__ int search_bits(const unsigned long long* __restrict__ row, int M, unsigned long long target)
{
    int lo = 0, hi = 2 * M;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (target < row[mid]) hi = mid;
        else lo = mid + 1;
    }
    return lo - M;
}

// One block: builds the three tables in the scratch array exactly as k_tables does (same
// operations in the same order, so the same bits), then draws all P samples as k_sample
// does.  The status word at scratch[3 * cap] is cleared at the start of every call.
__global__ void __launch_bounds__(256)
k_sample_noalloc(unsigned long long* __restrict__ scratch, double bx, double by, double bz, double alpha, int P,
                 uint64_t seed, uint64_t step, int32_t* __restrict__ m_out, double* __restrict__ S_out)
{
    __shared__ int sM[3];
    __shared__ double sc[3];
    __shared__ double sH[3];
    double* cdf = reinterpret_cast<double*>(scratch);
    unsigned* status = reinterpret_cast<unsigned*>(scratch + 3 * kNoAllocTableCap);
    const int tid = threadIdx.x;
    if (tid == 0) *status = 0u;  // the array keeps the previous call's contents
    __syncthreads();
    if (tid < 3) {
        const double ell = tid == 0 ? bx : (tid == 1 ? by : bz);
        const double c = axis_c(alpha, ell);
        sc[tid] = c;
        int M = axis_M(c);  // the host checked 2M + 1 <= kNoAllocTableCap; clamp all the same
        if (2 * M + 1 > kNoAllocTableCap) {
            atomicOr(status, kStatusTable);
            M = (kNoAllocTableCap - 1) / 2;
        }
        sM[tid] = M;
    }
    __syncthreads();
    for (int t = 0; t < 3; ++t) {
        const int M = sM[t];
        double* row = cdf + (size_t)t * kNoAllocTableCap;
        for (int a = tid; a <= M; a += blockDim.x) {
            const double v = table_exp(-__dmul_rn(sc[t], (double)a * (double)a));
            row[M + a] = v;
            row[M - a] = v;
        }
    }
    __syncthreads();
    if (tid < 3) {
        double* row = cdf + (size_t)tid * kNoAllocTableCap;
        double acc = 0.0;
        for (int j = 0; j <= 2 * sM[tid]; ++j) {
            acc = __dadd_rn(acc, row[j]);
            row[j] = acc;
        }
        sH[tid] = acc;
    }
    __syncthreads();
    if (tid == 0 && S_out) *S_out = __dsub_rn(__dmul_rn(__dmul_rn(sH[0], sH[1]), sH[2]), 1.0);
    const unsigned long long* tx = scratch;
    const unsigned long long* ty = scratch + kNoAllocTableCap;
    const unsigned long long* tz = scratch + 2 * kNoAllocTableCap;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t c2 = (uint32_t)step, c3 = (uint32_t)((step >> 32) & 0xFFFFFFu);
    for (int l = tid; l < P; l += blockDim.x) {
        int mx = 0, my = 0, mz = 0;
        bool found = false;
        for (uint32_t attempt = 0; attempt < kMaxAttempts; ++attempt) {
            const uint4 w0 = philox4x32_10(make_uint4((uint32_t)l, 2u * attempt, c2, c3), k0, k1);
            const uint4 w1 = philox4x32_10(make_uint4((uint32_t)l, 2u * attempt + 1u, c2, c3), k0, k1);
            const double ux = __longlong_as_double((long long)uniform53_bits(w0.x, w0.y));
            const double uy = __longlong_as_double((long long)uniform53_bits(w0.z, w0.w));
            const double uz = __longlong_as_double((long long)uniform53_bits(w1.x, w1.y));
            mx = search_bits(tx, sM[0], (unsigned long long)__double_as_longlong(__dmul_rn(ux, sH[0])));
            my = search_bits(ty, sM[1], (unsigned long long)__double_as_longlong(__dmul_rn(uy, sH[1])));
            mz = search_bits(tz, sM[2], (unsigned long long)__double_as_longlong(__dmul_rn(uz, sH[2])));
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

// Device address of the scratch array, looked up once per device (host code may not use
// the symbol itself as an address).
static std::mutex g_noalloc_mutex;
static unsigned long long* g_noalloc_ptr[64] = {nullptr};

static rbe_status noalloc_scratch(int device, unsigned long long** out, std::string& err)
{
    if (device < 0 || device >= 64) {
        err = "device ordinal out of range";
        return RBE_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
            return RBE_ECUDA;
        }
        g_noalloc_ptr[device] = static_cast<unsigned long long*>(p);
    }
    *out = g_noalloc_ptr[device];
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
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return fail(nullptr, RBE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    unsigned long long* scratch = nullptr;
    std::string err;
    rbe_status st = noalloc_scratch(device, &scratch, err);
    if (st != RBE_OK) return fail(nullptr, st, err);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_sample_noalloc<<<1, 256, 0, s>>>(scratch, box[0], box[1], box[2], alpha, P, seed, step, m_out, S_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, RBE_ECUDA, std::string("k_sample_noalloc: ") + cudaGetErrorString(e));
    unsigned bits = 0;
    e = cudaMemcpyAsync(&bits, scratch + 3 * kNoAllocTableCap, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(nullptr, RBE_ECUDA, std::string("rbe_sample_k_noalloc: ") + cudaGetErrorString(e));
    if (bits & kStatusTable) return fail(nullptr, RBE_EINVAL, "rbe_sample_k_noalloc: table larger than the fixed scratch");
    if (bits & kStatusSample) return fail(nullptr, RBE_ESAMPLE, "a frequency stayed m = 0 after 2^20 redraws");
    return RBE_OK;
}
