// The C ABI of librbe (declared in include/rbe.h): argument validation, context
// lifetime, device scratch, and the host-buffer variants.  The arithmetic lives in
// rbe_kspace.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rbe_context.h"
#include "rbe_device.cuh"

namespace rbe {

static thread_local std::string g_create_error;

rbe_status fail(rbe_ctx ctx, rbe_status st, const std::string& msg)
{
    if (ctx) ctx->last_error = msg;
    else g_create_error = msg;
    return st;
}

rbe_status cuda_fail(rbe_ctx ctx, cudaError_t err, const char* what)
{
    std::string msg = std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
    return fail(ctx, err == cudaErrorMemoryAllocation ? RBE_ENOMEM : RBE_ECUDA, msg);
}

int host_axis_M(double alpha, double ell)
{
    const double c = (kPi * kPi) / (alpha * (ell * ell));
    const double M = std::ceil(std::sqrt((60.0 * kLn2) / c));
    return M <= 1073741824.0 ? (int)M : 1073741824;  // clamped (also NaN) before the conversion
}

// Makes ctx->device current for the duration of a call and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static rbe_status check_box(rbe_ctx ctx, const double box[3], double alpha)
{
    if (!box) return fail(ctx, RBE_EINVAL, "box is NULL");
    for (int t = 0; t < 3; ++t) {
        if (!std::isfinite(box[t]) || !(box[t] > 0.0)) return fail(ctx, RBE_EINVAL, "box lengths must be finite and > 0");
        const double c = (kPi * kPi) / (alpha * (box[t] * box[t]));
        if (!(c <= 600.0))
            return fail(ctx, RBE_EINVAL, "pi^2/(alpha l^2) > 600 on some axis: the frequency distribution is degenerate");
        if (host_axis_M(alpha, box[t]) > (1 << 20))
            return fail(ctx, RBE_EINVAL, "alpha l^2 too large: per-axis table would exceed 2^21 entries");
    }
    return RBE_OK;
}

// A pointer the current device can read: device or managed memory.
static bool is_device_ptr(const void* p)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

rbe_status check_dev(rbe_ctx ctx, const void* p, const char* name, bool required)
{
    if (!p) return required ? fail(ctx, RBE_EINVAL, std::string(name) + " is NULL") : RBE_OK;
    if (reinterpret_cast<uintptr_t>(p) % 8 != 0) return fail(ctx, RBE_EINVAL, std::string(name) + " is not 8-byte aligned");
    if (!is_device_ptr(p)) return fail(ctx, RBE_EINVAL, std::string(name) + " is not device memory");
    return RBE_OK;
}

constexpr int64_t kMaxN = (int64_t(1) << 31) - 256;

// Non-finite values are reported first: they are the cause when a NaN or infinity has also
// carried the box out of its prepared range.
rbe_status status_from_bits(rbe_ctx ctx, unsigned bits)
{
    if (bits & kStatusSample) return fail(ctx, RBE_ESAMPLE, "a frequency stayed m = 0 after 2^20 redraws");
    if (bits & kStatusNonFinite) return fail(ctx, RBE_ENONFINITE, "rho(k) or an output is not finite");
    if (bits & kStatusTable) return fail(ctx, RBE_ESTATE, "sampling table capacity exceeded on the device");
    if (bits & kStatusList)
        return fail(ctx, RBE_ESTATE, "neighbour list capacity exceeded (the density rose far above its initial value)");
    if (bits & kStatusBox)
        return fail(ctx, RBE_ESTATE,
                    "the box left the range rbe_npt_init prepared (cell list capacity, or rc > l/2 on some axis)");
    if (bits & kStatusShake)
        return fail(ctx, RBE_ESTATE, "SHAKE did not converge within its sweep limit (a molecule was torn apart)");
    if (bits & kStatusTimeout) return fail(ctx, RBE_ETIMEOUT, "a bounded device wait gave up");
    return RBE_OK;
}

static rbe_status sync_and_status(rbe_ctx ctx)
{
    cudaError_t err = cudaStreamSynchronize(ctx->stream);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaStreamSynchronize");
    unsigned bits = 0;
    err = cudaMemcpy(&bits, ctx->d.status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaMemcpy(status)");
    if (bits) {
        err = cudaMemset(ctx->d.status, 0, sizeof(unsigned));
        if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaMemset(status)");
    }
    return status_from_bits(ctx, bits);
}

static void free_npt(NptBuffers& b)
{
    cudaFree(b.Fk); cudaFree(b.Fr); cudaFree(b.WEk); cudaFree(b.coef); cudaFree(b.cid); cudaFree(b.fill);
    cudaFree(b.sorted); cudaFree(b.spos32); cudaFree(b.spos64); cudaFree(b.mprop); cudaFree(b.cellc); cudaFree(b.cnt);
    cudaFree(b.nbr); cudaFree(b.nnb); cudaFree(b.sref); cudaFree(b.nls); cudaFree(b.start); cudaFree(b.cursor); cudaFree(b.partials);
    cudaFree(b.counter);
    b = NptBuffers{};
}

static void free_buffers(DeviceBuffers& d)
{
    cudaFree(d.cum); cudaFree(d.ks); cudaFree(d.m); cudaFree(d.w); cudaFree(d.rho); cudaFree(d.terms);
    cudaFree(d.coef_m); cudaFree(d.coef_f); cudaFree(d.coef_d); cudaFree(d.partials); cudaFree(d.counter);
    cudaFree(d.status); cudaFree(d.pos); cudaFree(d.q); cudaFree(d.F); cudaFree(d.WE);
    d = DeviceBuffers{};
}

}  // namespace rbe

using namespace rbe;

extern "C" {

rbe_status rbe_create(const double box[3], double alpha, int32_t P, uint64_t seed, rbe_ctx* out)
{
    if (!out) return fail(nullptr, RBE_EINVAL, "out is NULL");
    if (!std::isfinite(alpha) || !(alpha > 0.0)) return fail(nullptr, RBE_EINVAL, "alpha must be finite and > 0");
    if (P < 1 || P > 65536) return fail(nullptr, RBE_EINVAL, "P must be in [1, 65536]");
    rbe_status st = check_box(nullptr, box, alpha);
    if (st != RBE_OK) return st;
    rbe_ctx ctx = new (std::nothrow) rbe_ctx_s();
    if (!ctx) return fail(nullptr, RBE_ENOMEM, "host allocation failed");
    cudaError_t err = cudaGetDevice(&ctx->device);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (err != cudaSuccess) {
        std::string msg = std::string("no usable CUDA device: ") + cudaGetErrorString(err);
        delete ctx;
        return fail(nullptr, RBE_ECUDA, msg);
    }
    for (int t = 0; t < 3; ++t) ctx->box[t] = box[t];
    ctx->alpha = alpha;
    ctx->P = P;
    ctx->seed = seed;
    DeviceBuffers& d = ctx->d;
    if ((err = cudaMalloc(&d.ks, sizeof(KState))) != cudaSuccess ||
        (err = cudaMalloc(&d.counter, sizeof(unsigned))) != cudaSuccess ||
        (err = cudaMalloc(&d.status, sizeof(unsigned))) != cudaSuccess ||
        (err = cudaMemset(d.counter, 0, sizeof(unsigned))) != cudaSuccess ||
        (err = cudaMemset(d.status, 0, sizeof(unsigned))) != cudaSuccess) {
        std::string msg = std::string("device allocation failed: ") + cudaGetErrorString(err);
        free_buffers(d);
        delete ctx;
        return fail(nullptr, err == cudaErrorMemoryAllocation ? RBE_ENOMEM : RBE_ECUDA, msg);
    }
    // frequency buffers now; the tables are built by the first evaluation (tables_dirty), on
    // whatever stream the context uses by then.  Only the legacy default stream is waited for.
    st = ensure_k_capacity(ctx, P);
    if (st == RBE_OK && (err = cudaStreamSynchronize(nullptr)) != cudaSuccess) st = cuda_fail(ctx, err, "rbe_create");
    if (st != RBE_OK) {
        std::string msg = ctx->last_error;
        free_buffers(d);
        delete ctx;
        return fail(nullptr, st, msg);
    }
    *out = ctx;
    return RBE_OK;
}

rbe_status rbe_destroy(rbe_ctx ctx)
{
    if (!ctx) return RBE_OK;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    for (auto& e : ctx->pev)
        if (e) cudaEventDestroy(e);
    if (ctx->h_out) cudaFreeHost(ctx->h_out);
    free_npt(ctx->npt);
    free_buffers(ctx->d);
    if (ctx->chain) cudaFree(ctx->chain);
    if (ctx->m_all) cudaFree(ctx->m_all);
    if (ctx->gchain) cudaFree(ctx->gchain);
    if (ctx->gpos) cudaFree(ctx->gpos);
    if (ctx->flex_coef) cudaFree(ctx->flex_coef);
    if (ctx->gcell_dev) cudaFree(ctx->gcell_dev);
    if (ctx->flex_nls) cudaFree(ctx->flex_nls);
    if (ctx->flex_cpos32) cudaFree(ctx->flex_cpos32);
    if (ctx->flex_cpos64) cudaFree(ctx->flex_cpos64);
    if (ctx->flex_code) cudaFree(ctx->flex_code);
    delete ctx;
    return RBE_OK;
}

rbe_status rbe_set_stream(rbe_ctx ctx, void* stream)
{
    if (!ctx) return RBE_EINVAL;
    if (static_cast<cudaStream_t>(stream) != ctx->stream) {
        // scratch was allocated in the old stream's order: finish it before switching
        DeviceGuard g(ctx->device);
        cudaError_t err = cudaStreamSynchronize(ctx->stream);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "rbe_set_stream");
    }
    ctx->stream = static_cast<cudaStream_t>(stream);
    return RBE_OK;
}

rbe_status rbe_set_seed(rbe_ctx ctx, uint64_t seed)
{
    if (!ctx) return RBE_EINVAL;
    ctx->seed = seed;
    return RBE_OK;
}

rbe_status rbe_set_precision(rbe_ctx ctx, int32_t precision, int32_t rho_accum)
{
    if (!ctx) return RBE_EINVAL;
    if (precision != RBE_FP64 && precision != RBE_FP32_PHASE) return fail(ctx, RBE_EINVAL, "unknown precision");
    if (rho_accum != RBE_RHO_FP64 && rho_accum != RBE_RHO_COMP32 && rho_accum != RBE_RHO_FP32)
        return fail(ctx, RBE_EINVAL, "unknown rho accumulation");
    ctx->precision = precision;
    ctx->rho_accum = rho_accum;
    return RBE_OK;
}

rbe_status rbe_set_sampler(rbe_ctx ctx, int32_t sampler)
{
    if (!ctx) return RBE_EINVAL;
    if (sampler != RBE_SAMPLER_EXACT && sampler != RBE_SAMPLER_OFFLINE && sampler != RBE_SAMPLER_MH)
        return fail(ctx, RBE_EINVAL, "unknown sampler");
    DeviceGuard g(ctx->device);
    if (sampler == RBE_SAMPLER_MH && ctx->reuse > 1)
        return fail(ctx, RBE_EINVAL, "sample reuse and the Metropolis-Hastings chain exclude each other");
    if (sampler == RBE_SAMPLER_MH) {
        const int32_t need = ctx->P + ctx->Ptilde > 0 ? ctx->P + ctx->Ptilde : 1;
        cudaError_t e = cudaSuccess;
        if (ctx->chain_cap < need) {
            ctx_free(ctx, ctx->chain);
            ctx->chain = nullptr;
            ctx->chain_cap = 0;
            if ((e = ctx_alloc(ctx, &ctx->chain, sizeof(int4) * (size_t)need)) != cudaSuccess)
                return cuda_fail(ctx, e, "cudaMallocAsync(MH chain)");
            ctx->chain_cap = need;
        }
        // every slot starts again from the exact draw of its next sampling step
        if ((e = cudaMemsetAsync(ctx->chain, 0, sizeof(int4) * (size_t)ctx->chain_cap, ctx->stream)) != cudaSuccess)
            return cuda_fail(ctx, e, "cudaMemsetAsync(MH chain)");
    }
    if (ctx->gchain) {  // the general cell's chains restart too
        cudaError_t e = cudaMemsetAsync(ctx->gchain, 0, sizeof(int4) * (size_t)ctx->gchain_cap, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync(general chain)");
    }
    ctx->sampler = sampler;
    return RBE_OK;
}

rbe_status rbe_set_pressure_batch(rbe_ctx ctx, int32_t Ptilde)
{
    if (!ctx) return RBE_EINVAL;
    if (Ptilde < 0 || Ptilde > (1 << 20)) return fail(ctx, RBE_EINVAL, "Ptilde must be in [0, 2^20]");
    ctx->Ptilde = Ptilde;
    // an MH chain grows with the slots (and every slot restarts from the exact draw)
    return ctx->sampler == RBE_SAMPLER_MH ? rbe_set_sampler(ctx, RBE_SAMPLER_MH) : RBE_OK;
}

rbe_status rbe_set_sample_reuse(rbe_ctx ctx, int32_t M)
{
    if (!ctx) return RBE_EINVAL;
    if (M < 1 || M > 1024) return fail(ctx, RBE_EINVAL, "M must be in [1, 1024]");
    if (M > 1 && ctx->sampler == RBE_SAMPLER_MH)
        return fail(ctx, RBE_EINVAL, "sample reuse and the Metropolis-Hastings chain exclude each other");
    ctx->reuse = M;
    return RBE_OK;
}

rbe_status rbe_set_box(rbe_ctx ctx, const double box[3])
{
    if (!ctx) return RBE_EINVAL;
    rbe_status st = check_box(ctx, box, ctx->alpha);
    if (st != RBE_OK) return st;
    for (int t = 0; t < 3; ++t) {
        if (ctx->box[t] != box[t]) ctx->tables_dirty = true;
        ctx->box[t] = box[t];
    }
    return RBE_OK;
}

rbe_status rbe_sample_k(rbe_ctx ctx, uint64_t step, int32_t* m_out, double* S_out)
{
    if (!ctx) return RBE_EINVAL;
    if ((step >> 56) != 0) return fail(ctx, RBE_EINVAL, "step must be < 2^56");
    DeviceGuard g(ctx->device);
    rbe_status st = launch_sample(ctx, step, ctx->P);
    if (st != RBE_OK) return st;
    std::vector<int4> m(ctx->P);
    KState h;
    cudaError_t err = cudaMemcpyAsync(m.data(), ctx->d.m, sizeof(int4) * ctx->P, cudaMemcpyDeviceToHost, ctx->stream);
    if (err == cudaSuccess) err = cudaMemcpyAsync(&h, ctx->d.ks, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaMemcpyAsync(sample)");
    st = sync_and_status(ctx);
    if (st != RBE_OK) return st;
    if (m_out)
        for (int l = 0; l < ctx->P; ++l) {
            m_out[3 * l] = m[l].x;
            m_out[3 * l + 1] = m[l].y;
            m_out[3 * l + 2] = m[l].z;
        }
    if (S_out) *S_out = h.S;
    return RBE_OK;
}

rbe_status rbe_kspace_forces_virial(rbe_ctx ctx, int64_t N, const double* positions, const double* charges,
                                    uint64_t step, double* forces_out, double* virial_out, double* energy_out)
{
    if (!ctx) return RBE_EINVAL;
    if (N < 0 || N > kMaxN) return fail(ctx, RBE_EINVAL, "N out of range [0, 2^31 - 256]");
    if ((step >> 56) != 0) return fail(ctx, RBE_EINVAL, "step must be < 2^56");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, RBE_ECUDA, "cannot select the context's device");
    rbe_status st;
    if ((st = check_dev(ctx, positions, "positions", N > 0)) != RBE_OK) return st;
    if ((st = check_dev(ctx, charges, "charges", N > 0)) != RBE_OK) return st;
    if ((st = check_dev(ctx, forces_out, "forces_out", N > 0)) != RBE_OK) return st;
    if ((st = check_dev(ctx, virial_out, "virial_out", false)) != RBE_OK) return st;
    if ((st = check_dev(ctx, energy_out, "energy_out", false)) != RBE_OK) return st;
    st = launch_sample(ctx, step, ctx->P);
    if (st != RBE_OK) return st;
    return launch_rbe(ctx, N, positions, charges, ctx->P, forces_out, virial_out, energy_out);
}

rbe_status rbe_kspace_forces_virial_xyzq(rbe_ctx ctx, int64_t N, const float* xyzq, uint64_t step,
                                         double* forces_out, double* virial_out, double* energy_out)
{
    if (!ctx) return RBE_EINVAL;
    if (N < 0 || N > kMaxN) return fail(ctx, RBE_EINVAL, "N out of range [0, 2^31 - 256]");
    if ((step >> 56) != 0) return fail(ctx, RBE_EINVAL, "step must be < 2^56");
    if (ctx->precision != RBE_FP32_PHASE)
        return fail(ctx, RBE_EINVAL, "float4 xyzq positions need the RBE_FP32_PHASE precision");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, RBE_ECUDA, "cannot select the context's device");
    rbe_status st;
    if ((st = check_dev(ctx, xyzq, "xyzq", N > 0)) != RBE_OK) return st;
    if (N > 0 && reinterpret_cast<uintptr_t>(xyzq) % 16 != 0)
        return fail(ctx, RBE_EINVAL, "xyzq must be 16-byte aligned (one float4 per particle)");
    if ((st = check_dev(ctx, forces_out, "forces_out", N > 0)) != RBE_OK) return st;
    if ((st = check_dev(ctx, virial_out, "virial_out", false)) != RBE_OK) return st;
    if ((st = check_dev(ctx, energy_out, "energy_out", false)) != RBE_OK) return st;
    st = launch_sample(ctx, step, ctx->P);
    if (st != RBE_OK) return st;
    return launch_rbe(ctx, N, xyzq, nullptr, ctx->P, forces_out, virial_out, energy_out, true);
}

// The copy stream and events of the pipelined host-buffer call (created on first use).
static rbe_status ensure_copy_stream(rbe_ctx ctx)
{
    if (ctx->copy_stream) return RBE_OK;
    cudaError_t err = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    for (auto& e : ctx->pev)
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return err == cudaSuccess ? RBE_OK : cuda_fail(ctx, err, "copy stream");
}

// Pinned host words for the small outputs of the host-buffer call: virial (9), energy (2),
// status (in the 12th slot).
static rbe_status ensure_host_out(rbe_ctx ctx)
{
    if (ctx->h_out) return RBE_OK;
    cudaError_t err = cudaMallocHost(reinterpret_cast<void**>(&ctx->h_out), 16 * sizeof(double));
    return err == cudaSuccess ? RBE_OK : cuda_fail(ctx, err, "cudaMallocHost(outputs)");
}

rbe_status rbe_kspace_forces_virial_host(rbe_ctx ctx, int64_t N, const double* positions, const double* charges,
                                         uint64_t step, double* forces_out, double* virial_out,
                                         double* energy_out)
{
    if (!ctx) return RBE_EINVAL;
    if (N < 0 || N > kMaxN) return fail(ctx, RBE_EINVAL, "N out of range [0, 2^31 - 256]");
    if ((step >> 56) != 0) return fail(ctx, RBE_EINVAL, "step must be < 2^56");
    if (N > 0 && (!positions || !charges)) return fail(ctx, RBE_EINVAL, "positions/charges are NULL");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, RBE_ECUDA, "cannot select the context's device");
    DeviceBuffers& d = ctx->d;
    cudaError_t err;
    if (!d.WE && (err = ctx_alloc(ctx, &d.WE, 11 * sizeof(double))) != cudaSuccess)
        return cuda_fail(ctx, err, "cudaMalloc(host-call outputs)");
    if (N > d.ncap) {
        ctx_free(ctx, d.pos); ctx_free(ctx, d.q); ctx_free(ctx, d.F);
        d.pos = d.q = d.F = nullptr;
        d.ncap = 0;
        if ((err = ctx_alloc(ctx, &d.pos, sizeof(double) * 3 * N)) != cudaSuccess ||
            (err = ctx_alloc(ctx, &d.q, sizeof(double) * N)) != cudaSuccess ||
            (err = ctx_alloc(ctx, &d.F, sizeof(double) * 3 * N)) != cudaSuccess)
            return cuda_fail(ctx, err, "cudaMalloc(host-call staging)");
        d.ncap = N;
    }
    cudaStream_t s = ctx->stream;
    // pipelined on the FP32-phase path for systems large enough to split; plain copies else
    // four groups from 2^19 particles (an eighth, three eighths, three eighths, an eighth: the
    // exposed copies before the first pass and after the last shrink; N = 4e6, P = 2000: 7.24 ->
    // 6.99 ms per call), two from 2^17, one below
    const int pieces = N >= (1 << 19) ? 4 : (N >= (1 << 17) ? 2 : 1);
    const bool piped = ctx->precision == RBE_FP32_PHASE && pieces > 1 && ctx->Ptilde == 0;
    rbe_status st;
    if (piped) {
        // the copy stream starts after the main stream's earlier work (the staging buffers
        // may have been in use) and runs beside the sampler
        if ((st = ensure_copy_stream(ctx)) != RBE_OK) return st;
        if ((err = cudaEventRecord(ctx->pev[0], s)) != cudaSuccess ||
            (err = cudaStreamWaitEvent(ctx->copy_stream, ctx->pev[0], 0)) != cudaSuccess)
            return cuda_fail(ctx, err, "order the copy stream");
    }
    if ((st = launch_sample(ctx, step, ctx->P)) != RBE_OK) return st;
    if (piped) {
        st = launch_evaluate_staged(ctx, N, positions, charges, forces_out, d.pos, d.q, d.F, ctx->P, d.WE, d.WE + 9,
                                    pieces);
        if (st != RBE_OK) return st;
    } else {
        if (N > 0) {
            if ((err = cudaMemcpyAsync(d.pos, positions, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s)) !=
                    cudaSuccess ||
                (err = cudaMemcpyAsync(d.q, charges, sizeof(double) * N, cudaMemcpyHostToDevice, s)) != cudaSuccess)
                return cuda_fail(ctx, err, "cudaMemcpyAsync(H2D)");
        }
        st = launch_rbe(ctx, N, d.pos, d.q, ctx->P, d.F, d.WE, d.WE + 9);
        if (st != RBE_OK) return st;
        if (forces_out && N > 0 &&
            (err = cudaMemcpyAsync(forces_out, d.F, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(ctx, err, "cudaMemcpyAsync(D2H forces)");
    }
    // virial, energy and the status word into pinned host memory, then one wait
    if ((st = ensure_host_out(ctx)) != RBE_OK) return st;
    double* ho = ctx->h_out;
    if ((err = cudaMemcpyAsync(ho, d.WE, 11 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (err = cudaMemcpyAsync(ho + 11, d.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(ctx, err, "cudaMemcpyAsync(D2H virial)");
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ctx, err, "cudaStreamSynchronize");
    if (ctx->copy_stream && (err = cudaStreamSynchronize(ctx->copy_stream)) != cudaSuccess)
        return cuda_fail(ctx, err, "cudaStreamSynchronize(copy)");
    unsigned bits;
    std::memcpy(&bits, ho + 11, sizeof(unsigned));
    if (bits) {
        if ((err = cudaMemsetAsync(d.status, 0, sizeof(unsigned), s)) != cudaSuccess ||
            (err = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(ctx, err, "reset status");
        return status_from_bits(ctx, bits);
    }
    if (virial_out) std::memcpy(virial_out, ho, 9 * sizeof(double));
    if (energy_out) std::memcpy(energy_out, ho + 9, 2 * sizeof(double));
    return RBE_OK;
}

rbe_status rbe_kspace_weighted(rbe_ctx ctx, int64_t N, const double* positions, const double* charges, int32_t K,
                               const int32_t* m, const double* weights, double* forces_out, double* virial_out,
                               double* energy_out)
{
    if (!ctx) return RBE_EINVAL;
    if (N < 0 || N > kMaxN) return fail(ctx, RBE_EINVAL, "N out of range [0, 2^31 - 256]");
    if (K < 1 || K > (1 << 24)) return fail(ctx, RBE_EINVAL, "K must be in [1, 2^24]");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, RBE_ECUDA, "cannot select the context's device");
    rbe_status st;
    if ((st = check_dev(ctx, positions, "positions", N > 0)) != RBE_OK) return st;
    if ((st = check_dev(ctx, charges, "charges", N > 0)) != RBE_OK) return st;
    if ((st = check_dev(ctx, forces_out, "forces_out", N > 0)) != RBE_OK) return st;
    if ((st = check_dev(ctx, virial_out, "virial_out", false)) != RBE_OK) return st;
    if ((st = check_dev(ctx, energy_out, "energy_out", false)) != RBE_OK) return st;
    if (!m || (reinterpret_cast<uintptr_t>(m) % 4) != 0 || !is_device_ptr(m))
        return fail(ctx, RBE_EINVAL, "m must be 4-byte aligned device memory");
    if ((st = check_dev(ctx, weights, "weights", true)) != RBE_OK) return st;
    st = launch_weights_from_list(ctx, K, m, weights);
    if (st != RBE_OK) return st;
    return launch_evaluate(ctx, N, positions, charges, K, false, forces_out, virial_out, energy_out);
}

rbe_status rbe_get_rho(rbe_ctx ctx, double* rho_out, int32_t capacity)
{
    if (!ctx) return RBE_EINVAL;
    if (!rho_out) return fail(ctx, RBE_EINVAL, "rho_out is NULL");
    if (ctx->last_K <= 0) return fail(ctx, RBE_ESTATE, "no evaluation has run on this context");
    if (capacity < 2 * ctx->last_K) return fail(ctx, RBE_EINVAL, "capacity < 2 * K");
    DeviceGuard g(ctx->device);
    cudaError_t err = cudaMemcpyAsync(rho_out, ctx->d.rho, sizeof(double2) * ctx->last_K, cudaMemcpyDeviceToHost,
                                      ctx->stream);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaMemcpyAsync(rho)");
    return sync_and_status(ctx);
}

rbe_status rbe_npt_init(rbe_ctx ctx, rbe_system* sys, uint64_t batch)
{
    if (!ctx) return RBE_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, RBE_ECUDA, "cannot select the context's device");
    if (sys) {
        rbe_status st;
        const int64_t N = sys->N;
        if ((st = check_dev(ctx, sys->pos, "pos", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->mom, "mom", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->force, "force", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->charge, "charge", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->mass, "mass", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->cell, "cell", true)) != RBE_OK) return st;
    }
    return npt_init(ctx, sys, batch);
}

rbe_status rbe_npt_step(rbe_ctx ctx, rbe_system* sys, int32_t nsteps)
{
    if (!ctx) return RBE_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, RBE_ECUDA, "cannot select the context's device");
    return npt_run(ctx, sys, nsteps);
}

rbe_status rbe_flex_init(rbe_ctx ctx, rbe_flex_system* sys, uint64_t batch)
{
    if (!ctx) return RBE_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, RBE_ECUDA, "cannot select the context's device");
    if (sys) {
        rbe_status st;
        const int64_t N = sys->N;
        if ((st = check_dev(ctx, sys->pos, "pos", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->mom, "mom", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->force, "force", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->charge, "charge", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->mass, "mass", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->cell, "cell", true)) != RBE_OK) return st;
    }
    return flex_init(ctx, sys, batch);
}

rbe_status rbe_flex_step(rbe_ctx ctx, rbe_flex_system* sys, int32_t nsteps)
{
    if (!ctx) return RBE_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, RBE_ECUDA, "cannot select the context's device");
    return flex_run(ctx, sys, nsteps);
}

rbe_status rbe_water_init(rbe_ctx ctx, rbe_system* sys, const rbe_water_params* wp, uint64_t batch)
{
    if (!ctx) return RBE_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, RBE_ECUDA, "cannot select the context's device");
    if (sys) {
        rbe_status st;
        const int64_t N = sys->N;
        if ((st = check_dev(ctx, sys->pos, "pos", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->mom, "mom", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->force, "force", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->charge, "charge", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->mass, "mass", N > 0)) != RBE_OK) return st;
        if ((st = check_dev(ctx, sys->cell, "cell", true)) != RBE_OK) return st;
    }
    return water_init(ctx, sys, wp, batch);
}

rbe_status rbe_water_step(rbe_ctx ctx, rbe_system* sys, const rbe_water_params* wp, int32_t nsteps)
{
    if (!ctx) return RBE_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, RBE_ECUDA, "cannot select the context's device");
    return water_run(ctx, sys, wp, nsteps);
}

rbe_status rbe_set_kernel_timing(rbe_ctx ctx, int32_t enable)
{
    if (!ctx) return RBE_EINVAL;
    DeviceGuard g(ctx->device);
    if (enable && !ctx->ev[0])
        for (auto& e : ctx->ev) {
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaEventCreate");
        }
    ctx->timing = enable != 0;
    return RBE_OK;
}

rbe_status rbe_get_kernel_times(rbe_ctx ctx, float ms_out[4])
{
    if (!ctx || !ms_out) return RBE_EINVAL;
    if (!ctx->timing || ctx->last_K <= 0) return fail(ctx, RBE_ESTATE, "kernel timing is off or nothing ran");
    DeviceGuard g(ctx->device);
    cudaError_t err = cudaEventSynchronize(ctx->ev[4]);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaEventSynchronize");
    for (int j = 0; j < 4; ++j) {
        err = cudaEventElapsedTime(&ms_out[j], ctx->ev[j], ctx->ev[j + 1]);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaEventElapsedTime");
    }
    return RBE_OK;
}

rbe_status rbe_sync(rbe_ctx ctx)
{
    if (!ctx) return RBE_EINVAL;
    DeviceGuard g(ctx->device);
    return sync_and_status(ctx);
}

const char* rbe_status_string(rbe_status status)
{
    switch (status) {
    case RBE_OK: return "RBE_OK";
    case RBE_EINVAL: return "RBE_EINVAL: invalid argument";
    case RBE_ENOMEM: return "RBE_ENOMEM: allocation failed";
    case RBE_ECUDA: return "RBE_ECUDA: CUDA runtime error";
    case RBE_ETIMEOUT: return "RBE_ETIMEOUT: bounded device wait gave up";
    case RBE_ENONFINITE: return "RBE_ENONFINITE: non-finite rho or output";
    case RBE_ESAMPLE: return "RBE_ESAMPLE: frequency sampling did not find m != 0";
    case RBE_ESTATE: return "RBE_ESTATE: call not valid in this state";
    }
    return "unknown rbe_status";
}

const char* rbe_last_error(rbe_ctx ctx)
{
    return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

int32_t rbe_version(void) { return 100; }

}  // extern "C"
