// Serving loop for independent NPT replicas (continuous batching on one GPU).
//
// Requests (N charges, initial state, NPT parameters, number of steps) queue on the host.
// A request is admitted when a slot is free and its device memory fits the budget; its
// state then stays resident in HBM until it finishes.  Every resident replica runs on its
// own non-blocking stream with its own context, in chunks of `chunk_steps` steps; a chunk is
// the library's NPT step launches captured once per replica as a CUDA graph (the step index
// is device-resident, so one graph serves every chunk).  Chunks of different replicas run
// concurrently on the GPU and new requests are admitted while others run.  Latency of a
// chunk = host time from its launch to the observation of its completion event.
//
// Failures stay with their request: every chunk ends with a one-thread kernel that stores the
// slot's device status word into mapped pinned host memory (inside the chunk's graph; a store
// over the host link instead of a copy-engine transfer per chunk, which the copy engines shared
// by all slots' streams would serialise), before the completion event, so a replica that
// latched an error (non-finite values, a box outside its prepared range, a full neighbour
// list) is evicted at the end of that chunk with the error as its result, and its slot serves
// the next request; the other replicas run on untouched.  A request can also be cancelled,
// queued or resident (a resident one leaves at the end of its chunk in flight).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <memory>
#include <string>
#include <vector>

#include "rbe_context.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    rbe_request r;
    std::vector<double> pos, mom, q, m;  // copies of the caller's host inputs
    std::vector<double> out_pos, out_mom, out_cell;
    int state = 0;  // 0 queued, 1 resident, 2 done, 3 failed, 4 cancelled
    rbe_status error = RBE_OK;
    std::string error_msg;  // why the request failed
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
};

struct Slot {
    bool busy = false;
    int64_t req = -1;
    rbe_ctx ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    double *pos = nullptr, *mom = nullptr, *force = nullptr, *charge = nullptr, *mass = nullptr, *cell = nullptr;
    int64_t ncap = 0;
    rbe_system sys{};
    int32_t steps_left = 0;
    bool in_flight = false;
    int32_t chunk_in_flight = 0;
    double t_launch = 0.0;
    cudaGraphExec_t graph = nullptr;
    int32_t graph_steps = 0;
    int64_t bytes = 0;
    unsigned* h_status = nullptr;  // pinned, mapped: the context's device status word after the last chunk
    unsigned* h_status_dev = nullptr;  // the same word's device address
    bool cancel = false;           // leave at the end of the chunk in flight
};

// Stores up to kPublishMax device status words into their mapped host words (thread i: pair i).
constexpr int kPublishMax = 64;
struct StatusPairs {
    const unsigned* dev[kPublishMax];
    unsigned* host[kPublishMax];
    int n;
};

__global__ void k_publish_status(StatusPairs p)
{
    const int i = threadIdx.x;
    if (i < p.n) {
        *reinterpret_cast<volatile unsigned*>(p.host[i]) = *reinterpret_cast<const volatile unsigned*>(p.dev[i]);
        __threadfence_system();
    }
}

}  // namespace

struct rbe_server_s {
    rbe_server_config cfg;
    std::vector<std::unique_ptr<Request>> reqs;
    std::deque<int64_t> queue;
    std::vector<Slot> slots;
    int64_t mem_used = 0;
    std::vector<double> latencies;
    int64_t steps_done = 0;
    int64_t n_done = 0;
    Clock::time_point t0;
    double t_first_admit = -1.0, t_last_done = 0.0;
    std::string last_error;
    int device = 0;
    // lockstep groups (cfg.batched): the group's stream, the batched k-space, the chunk in flight
    rbe_batch batch = nullptr;
    double batch_box = 0.0;             // the batch's max_box
    bool tuned = false;                 // cfg.batched == 2: tiles chosen (once)
    cudaStream_t gstream = nullptr;
    cudaEvent_t gfork = nullptr, gk = nullptr, gdone = nullptr;
    std::vector<cudaEvent_t> ev_a, ev_b;  // per slot: after its move, after its finish
    std::vector<int> members;           // slots of the chunk in flight (slot order)
    std::vector<rbe_batch_item> items;
    bool group_in_flight = false;
    int32_t group_steps = 0;
    double group_t_launch = 0.0;
    std::vector<int64_t> last_key, graph_key;  // request ids of the last group and of the captured one
    cudaGraphExec_t ggraph = nullptr;
    int32_t ggraph_steps = 0;
};

namespace rbe {

static double now_s(const rbe_server_s* s)
{
    return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

static rbe_status sfail(rbe_server_s* s, rbe_status st, const std::string& msg)
{
    if (s) s->last_error = msg;
    return fail(nullptr, st, msg);
}

// Device bytes a replica of N particles holds while resident: its state (r, p, F: 72 B;
// q, m: 16 B), the context's NPT scratch (k-space and real-space forces 48 B, cell list
// 12 B, packed positions 16 B FP32 + 32 B FP64), the cell arrays (12 B per cell for edges
// up to twice the initial box), the neighbour list when the request uses one, and a fixed
// allowance for tables, frequency buffers and partial sums.
static int64_t replica_bytes(const rbe_request& r, int P)
{
    int64_t cells = 1;
    for (int t = 0; t < 3; ++t) {
        const double f = std::floor(2.0 * r.box[t] / r.params.rc);
        cells *= f >= 1.0 ? (f <= 4096.0 ? (int64_t)f : 4096) : 1;
    }
    int64_t list = 0;  // neighbour list (skin > 0): entries per particle as rbe_npt_init sizes them
    if (r.params.skin > 0.0) {
        const double rl = r.params.rc + r.params.skin, V = r.box[0] * r.box[1] * r.box[2];
        const double expect = 4.0 / 3.0 * 3.14159265358979323846 * rl * rl * rl * (double)r.N / V;
        const int64_t cap = (int64_t)(std::ceil((2.0 * expect + 64.0) / 32.0) * 32.0);
        list = r.N * (4 * cap + 4 + 16);
    }
    // frequency buffers of the force and pressure batches (each slot ~100 B) and the reused draws
    const int64_t Ptot = (int64_t)P + std::max(0, r.ptilde);
    const int64_t freq = Ptot * 112 + (r.reuse > 1 ? (int64_t)r.reuse * Ptot * 16 : 0) + Ptot * 16;
    return r.N * (72 + 16 + 48 + 12 + 48) + 12 * cells + list + (int64_t)(P + 1) * 16 * 2048 + freq + (4 << 20);
}

static void release_slot(rbe_server_s* s, Slot& sl)
{
    if (sl.graph) {
        cudaGraphExecDestroy(sl.graph);
        sl.graph = nullptr;
        sl.graph_steps = 0;
    }
    s->mem_used -= sl.bytes;
    sl.bytes = 0;
    sl.busy = false;
    sl.req = -1;
    sl.in_flight = false;
    sl.cancel = false;
}

// Publishes the status words of `n` slots on `stream` (kernel launches, capturable).
static cudaError_t publish_status(cudaStream_t stream, const Slot* const* sl, int n)
{
    for (int b = 0; b < n; b += kPublishMax) {
        StatusPairs p{};
        p.n = std::min(kPublishMax, n - b);
        for (int i = 0; i < p.n; ++i) {
            p.dev[i] = sl[b + i]->ctx->d.status;
            p.host[i] = sl[b + i]->h_status_dev;
        }
        k_publish_status<<<1, kPublishMax, 0, stream>>>(p);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static rbe_status ensure_slot_buffers(rbe_server_s* s, Slot& sl, int64_t N)
{
    if (!sl.stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaHostAlloc(reinterpret_cast<void**>(&sl.h_status), sizeof(unsigned), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&sl.h_status_dev), sl.h_status, 0);
        if (e != cudaSuccess) return sfail(s, RBE_ECUDA, std::string("slot stream: ") + cudaGetErrorString(e));
        *sl.h_status = 0u;
    }
    if (N > sl.ncap) {
        for (double** p : {&sl.pos, &sl.mom, &sl.force, &sl.charge, &sl.mass}) {
            if (*p) cudaFreeAsync(*p, sl.stream);
            *p = nullptr;
        }
        cudaError_t e = cudaSuccess;
        if ((e = cudaMallocAsync(&sl.pos, sizeof(double) * 3 * N, sl.stream)) != cudaSuccess ||
            (e = cudaMallocAsync(&sl.mom, sizeof(double) * 3 * N, sl.stream)) != cudaSuccess ||
            (e = cudaMallocAsync(&sl.force, sizeof(double) * 3 * N, sl.stream)) != cudaSuccess ||
            (e = cudaMallocAsync(&sl.charge, sizeof(double) * N, sl.stream)) != cudaSuccess ||
            (e = cudaMallocAsync(&sl.mass, sizeof(double) * N, sl.stream)) != cudaSuccess)
            return sfail(s, RBE_ENOMEM, std::string("slot buffers: ") + cudaGetErrorString(e));
        sl.ncap = N;
    }
    if (!sl.cell) {
        cudaError_t e = cudaMallocAsync(&sl.cell, sizeof(double) * RBE_CELL_DOUBLES, sl.stream);
        if (e != cudaSuccess) return sfail(s, RBE_ENOMEM, std::string("slot cell: ") + cudaGetErrorString(e));
    }
    return RBE_OK;
}

// Admit request `id` into slot `sl`: upload its state, initialise the forces, capture the
// chunk graph.  Everything runs on the slot's stream; no device-wide synchronisation.
static rbe_status admit(rbe_server_s* s, Slot& sl, int64_t id)
{
    Request& rq = *s->reqs[id];
    const int64_t N = rq.r.N;
    rbe_status st = ensure_slot_buffers(s, sl, N);
    if (st != RBE_OK) return st;
    if (!sl.ctx) {
        st = rbe_create(rq.r.box, s->cfg.alpha, s->cfg.P, rq.r.seed, &sl.ctx);
        if (st != RBE_OK) return sfail(s, st, std::string("slot context: ") + rbe_last_error(nullptr));
        rbe_set_precision(sl.ctx, s->cfg.precision, RBE_RHO_COMP32);
        if ((st = rbe_set_stream(sl.ctx, sl.stream)) != RBE_OK) return st;
    }
    rbe_set_seed(sl.ctx, rq.r.seed);
    if ((st = rbe_set_box(sl.ctx, rq.r.box)) != RBE_OK) return sfail(s, st, rbe_last_error(sl.ctx));
    // the request's sampling (a slot's context is reused: every admission sets all three, the
    // exact sampler first so that neither a previous MH chain nor a previous reuse excludes the
    // request's combination; an MH chain starts afresh)
    if ((st = rbe_set_sampler(sl.ctx, RBE_SAMPLER_EXACT)) != RBE_OK ||
        (st = rbe_set_sample_reuse(sl.ctx, rq.r.reuse > 1 ? rq.r.reuse : 1)) != RBE_OK ||
        (st = rbe_set_sampler(sl.ctx, rq.r.sampler)) != RBE_OK ||
        (st = rbe_set_pressure_batch(sl.ctx, rq.r.ptilde)) != RBE_OK)
        return sfail(s, st, rbe_last_error(sl.ctx));
    double cell[RBE_CELL_DOUBLES] = {0};
    for (int t = 0; t < 3; ++t) cell[t] = rq.r.box[t];
    cell[3] = rq.r.pV;
    for (int t = 0; t < 3; ++t) cell[12 + t] = rq.r.pc[t];
    cudaError_t e = cudaSuccess;
    if ((e = cudaMemcpyAsync(sl.pos, rq.pos.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, sl.stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sl.mom, rq.mom.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, sl.stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sl.charge, rq.q.data(), sizeof(double) * N, cudaMemcpyHostToDevice, sl.stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sl.mass, rq.m.data(), sizeof(double) * N, cudaMemcpyHostToDevice, sl.stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sl.cell, cell, sizeof(cell), cudaMemcpyHostToDevice, sl.stream)) != cudaSuccess)
        return sfail(s, RBE_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
    sl.sys = rbe_system{N, sl.pos, sl.mom, sl.force, sl.charge, sl.mass, sl.cell, 0, rq.r.params};
    if ((st = rbe_npt_init(sl.ctx, &sl.sys, 0)) != RBE_OK) return sfail(s, st, rbe_last_error(sl.ctx));
    if (sl.graph) {
        cudaGraphExecDestroy(sl.graph);
        sl.graph = nullptr;
    }
    sl.graph_steps = 0;
    if (s->cfg.use_graphs && !s->cfg.batched && rq.r.nsteps >= s->cfg.chunk_steps) {
        // one chunk of launches, captured; the device step index makes it replayable
        cudaGraph_t g = nullptr;
        rbe_system probe = sl.sys;
        e = cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = rbe_npt_step(sl.ctx, &probe, s->cfg.chunk_steps);
            const Slot* one = &sl;
            const cudaError_t ep = st == RBE_OK ? publish_status(sl.stream, &one, 1) : cudaSuccess;
            e = cudaStreamEndCapture(sl.stream, &g);
            if (e == cudaSuccess) e = ep;
            if (st != RBE_OK) {
                if (g) cudaGraphDestroy(g);
                return sfail(s, st, std::string("capture: ") + rbe_last_error(sl.ctx));
            }
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&sl.graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) return sfail(s, RBE_ECUDA, std::string("graph: ") + cudaGetErrorString(e));
        sl.graph_steps = s->cfg.chunk_steps;
    }
    sl.busy = true;
    sl.req = id;
    sl.steps_left = rq.r.nsteps;
    sl.in_flight = false;
    sl.bytes = replica_bytes(rq.r, s->cfg.P);
    s->mem_used += sl.bytes;
    rq.state = 1;
    rq.t_admit = now_s(s);
    if (s->t_first_admit < 0.0) s->t_first_admit = rq.t_admit;
    return RBE_OK;
}

static rbe_status launch_chunk(rbe_server_s* s, Slot& sl)
{
    const int32_t n = std::min(sl.steps_left, s->cfg.chunk_steps);
    rbe_status st = RBE_OK;
    if (sl.graph && n == sl.graph_steps) {
        cudaError_t e = cudaGraphLaunch(sl.graph, sl.stream);
        if (e != cudaSuccess) return sfail(s, RBE_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
        sl.sys.step += (uint64_t)n;
    } else {
        st = rbe_npt_step(sl.ctx, &sl.sys, n);
        if (st != RBE_OK) return sfail(s, st, rbe_last_error(sl.ctx));
        // the replica's latched device errors, read by progress() once the chunk is complete (the
        // captured chunk publishes them itself)
        const Slot* one = &sl;
        const cudaError_t ep = publish_status(sl.stream, &one, 1);
        if (ep != cudaSuccess) return sfail(s, RBE_ECUDA, std::string("chunk status: ") + cudaGetErrorString(ep));
    }
    cudaError_t e = cudaEventRecord(sl.done, sl.stream);
    if (e != cudaSuccess) return sfail(s, RBE_ECUDA, std::string("chunk status: ") + cudaGetErrorString(e));
    sl.in_flight = true;
    sl.chunk_in_flight = n;
    sl.t_launch = now_s(s);
    return RBE_OK;
}

static rbe_status retire(rbe_server_s* s, Slot& sl)
{
    Request& rq = *s->reqs[sl.req];
    const int64_t N = rq.r.N;
    rq.out_pos.resize(3 * N);
    rq.out_mom.resize(3 * N);
    rq.out_cell.resize(RBE_CELL_DOUBLES);
    cudaError_t e = cudaMemcpyAsync(rq.out_pos.data(), sl.pos, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rq.out_mom.data(), sl.mom, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rq.out_cell.data(), sl.cell, sizeof(double) * RBE_CELL_DOUBLES, cudaMemcpyDeviceToHost,
                            sl.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sl.stream);
    rbe_status st = e == cudaSuccess ? rbe_sync(sl.ctx) : RBE_ECUDA;
    rq.state = st == RBE_OK ? 2 : 3;
    rq.error = st;
    if (st != RBE_OK) rq.error_msg = e == cudaSuccess ? rbe_last_error(sl.ctx) : cudaGetErrorString(e);
    rq.t_done = now_s(s);
    s->t_last_done = rq.t_done;
    ++s->n_done;
    release_slot(s, sl);
    return RBE_OK;  // a failed request is reported through rbe_server_result, not here
}

// End a resident request before its last step: `state` 3 (failed with `st`, message from the
// slot's context) or 4 (cancelled).  Its chunk in flight has completed (or none was launched);
// the latched status word is cleared on the slot's stream for the slot's next request.
static void evict(rbe_server_s* s, Slot& sl, int state, rbe_status st, const std::string& msg)
{
    Request& rq = *s->reqs[sl.req];
    rq.state = state;
    rq.error = st;
    rq.error_msg = msg;
    rq.t_done = now_s(s);
    s->t_last_done = rq.t_done;
    ++s->n_done;
    if (sl.ctx) cudaMemsetAsync(sl.ctx->d.status, 0, sizeof(unsigned), sl.stream);
    *sl.h_status = 0u;
    release_slot(s, sl);
}

// ---------------------------------------------------------------------------------
// Lockstep groups (cfg.batched): every resident replica advances by the same chunk.  The group
// stream forks to the replicas' streams once per chunk; per step each replica moves (cell
// update and drift), the group stream joins the moves for one persistent batched k-space
// launch over the group (each item reads its box and step index from its replica's cell block
// and writes into its context's k-space buffers and status word), and the replicas run their
// real space beside it and their finishing kernels after it; the group stream joins them at
// the end of the chunk.

static rbe_status ensure_group_batch(rbe_server_s* s, int m)
{
    double need = 0.0;
    for (int k : s->members) {
        const Request& rq = *s->reqs[s->slots[k].req];
        for (int t = 0; t < 3; ++t) need = std::max(need, 2.05 * rq.r.box[t]);  // the NPT range: twice the box
    }
    if (s->batch && need <= s->batch_box && m <= s->cfg.max_slots) return RBE_OK;
    int32_t tk = 0, tc = 0, tf = 0, trf = 1;
    if (s->batch) {
        rbe_batch_get_tiles(s->batch, &tk, &tc, &tf);
        rbe_batch_get_rho_f(s->batch, &trf);
        rbe_batch_destroy(s->batch);
        s->batch = nullptr;
    }
    need = std::max(need, 2.0 * s->batch_box);  // grow geometrically
    rbe_status st = rbe_batch_create(s->cfg.alpha, s->cfg.P, s->cfg.max_slots, need, &s->batch);
    if (st != RBE_OK) return sfail(s, st, std::string("group batch: ") + rbe_last_error(nullptr));
    s->batch_box = need;
    if ((st = rbe_batch_set_stream(s->batch, s->gstream)) != RBE_OK) return sfail(s, st, "group batch stream");
    if (tk) {  // keep the tuned shapes
        rbe_batch_set_tiles(s->batch, tk, tc, tf);
        rbe_batch_set_rho_f(s->batch, trf);
    }
    if (s->ggraph) {
        cudaGraphExecDestroy(s->ggraph);  // it launched the old batch
        s->ggraph = nullptr;
        s->graph_key.clear();
    }
    return RBE_OK;
}

// The launches of `n` lockstep steps of the members (captured or direct).
static rbe_status enqueue_group_steps(rbe_server_s* s, int32_t n)
{
    const int m = (int)s->members.size();
    cudaError_t e = cudaSuccess;
    rbe_status st = RBE_OK;
    // fork once per chunk: a replica's next move follows its own finishing pass in stream order,
    // and that pass waited for the group's k-space, so the steps need no join of their own
    // beyond the k-space's (which needs every replica's moved positions and cell)
    if ((e = cudaEventRecord(s->gfork, s->gstream)) == cudaSuccess)
        for (int j = 0; j < m && e == cudaSuccess; ++j)
            e = cudaStreamWaitEvent(s->slots[s->members[j]].stream, s->gfork, 0);
    for (int32_t k = 0; k < n && e == cudaSuccess; ++k) {
        for (int j = 0; j < m && e == cudaSuccess; ++j) {
            Slot& sl = s->slots[s->members[j]];
            if ((st = npt_step_phase(sl.ctx, &sl.sys, kNptPhaseMove)) != RBE_OK) return sfail(s, st, rbe_last_error(sl.ctx));
            e = cudaEventRecord(s->ev_a[s->members[j]], sl.stream);
        }
        for (int j = 0; j < m && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(s->gstream, s->ev_a[s->members[j]], 0);
        if (e != cudaSuccess) break;
        if ((st = rbe_kspace_forces_virial_batched(s->batch, s->items.data(), m)) != RBE_OK)
            return sfail(s, st, std::string("group k-space: ") + rbe_batch_last_error(s->batch));
        if ((e = cudaEventRecord(s->gk, s->gstream)) != cudaSuccess) break;
        for (int j = 0; j < m && e == cudaSuccess; ++j) {
            Slot& sl = s->slots[s->members[j]];
            // the real space needs only this replica's moved positions: it runs beside the k-space
            if ((st = npt_step_phase(sl.ctx, &sl.sys, kNptPhaseReal)) != RBE_OK) return sfail(s, st, rbe_last_error(sl.ctx));
            if ((e = cudaStreamWaitEvent(sl.stream, s->gk, 0)) != cudaSuccess) break;
            if ((st = npt_step_phase(sl.ctx, &sl.sys, kNptPhaseFinish)) != RBE_OK)
                return sfail(s, st, rbe_last_error(sl.ctx));
        }
    }
    // join once per chunk
    for (int j = 0; j < m && e == cudaSuccess; ++j) {
        if ((e = cudaEventRecord(s->ev_b[s->members[j]], s->slots[s->members[j]].stream)) != cudaSuccess) break;
        e = cudaStreamWaitEvent(s->gstream, s->ev_b[s->members[j]], 0);
    }
    if (e != cudaSuccess) return sfail(s, RBE_ECUDA, std::string("group chunk: ") + cudaGetErrorString(e));
    return RBE_OK;
}

// Launch the next lockstep chunk of every resident replica: replayed from the group's graph
// when the group is the one captured, captured when the same group comes a second time,
// launched directly otherwise.
static rbe_status launch_group_chunk(rbe_server_s* s)
{
    s->members.clear();
    std::vector<int64_t> key;
    int32_t n = s->cfg.chunk_steps;
    for (int k = 0; k < (int)s->slots.size(); ++k)
        if (s->slots[k].busy && s->slots[k].steps_left > 0) {
            s->members.push_back(k);
            key.push_back(s->slots[k].req);
            n = std::min(n, s->slots[k].steps_left);
        }
    const int m = (int)s->members.size();
    if (m == 0) return RBE_OK;
    rbe_status st = ensure_group_batch(s, m);
    if (st != RBE_OK) return st;
    s->items.assign(m, rbe_batch_item{});
    for (int j = 0; j < m; ++j) {
        Slot& sl = s->slots[s->members[j]];
        const Request& rq = *s->reqs[sl.req];
        rbe_batch_item& it = s->items[j];
        it.N = rq.r.N;
        it.pos = sl.pos;
        it.charge = sl.charge;
        it.forces = sl.ctx->npt.Fk;
        it.virial = sl.ctx->npt.WEk;
        it.energy = sl.ctx->npt.WEk + 9;
        for (int t = 0; t < 3; ++t) it.box[t] = rq.r.box[t];
        it.seed = rq.r.seed;
        it.step = 0;
        it.box_dev = sl.cell;
        it.step_dev = reinterpret_cast<const uint64_t*>(sl.cell + 11);
        it.status_dev = sl.ctx->d.status;
    }
    cudaError_t e = cudaSuccess;
    const bool replay = s->cfg.use_graphs && s->ggraph && key == s->graph_key && n == s->ggraph_steps;
    if (!replay && s->ggraph) {
        // the captured graph reads the batch's descriptors as they were at capture: once another
        // group has run, it may not be replayed
        cudaGraphExecDestroy(s->ggraph);
        s->ggraph = nullptr;
        s->graph_key.clear();
    }
    if (replay) {
        if ((e = cudaGraphLaunch(s->ggraph, s->gstream)) != cudaSuccess)
            return sfail(s, RBE_ECUDA, std::string("group graph launch: ") + cudaGetErrorString(e));
        for (int k : s->members) s->slots[k].sys.step += (uint64_t)n;
    } else if (s->cfg.use_graphs && key == s->last_key && n == s->cfg.chunk_steps) {
        if (s->cfg.batched == 2 && !s->tuned) {
            // the tile shapes of the group, once; the items' k-space buffers are scratch between steps
            if ((st = rbe_batch_autotune(s->batch, s->items.data(), m, 2, nullptr)) != RBE_OK)
                return sfail(s, st, std::string("group autotune: ") + rbe_batch_last_error(s->batch));
            s->tuned = true;
        }
        // the batch plans its work lists outside capture: one direct chunk of these items first
        // has done that (the same group ran the chunk before)
        std::vector<rbe_system> saved;
        for (int k : s->members) saved.push_back(s->slots[k].sys);
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(s->gstream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return sfail(s, RBE_ECUDA, std::string("group capture: ") + cudaGetErrorString(e));
        st = enqueue_group_steps(s, n);
        e = cudaStreamEndCapture(s->gstream, &g);
        for (int j = 0; j < m; ++j) s->slots[s->members[j]].sys = saved[j];  // the capture ran nothing
        if (st != RBE_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&s->ggraph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) e = cudaGraphLaunch(s->ggraph, s->gstream);
        if (e != cudaSuccess) return sfail(s, RBE_ECUDA, std::string("group graph: ") + cudaGetErrorString(e));
        s->graph_key = key;
        s->ggraph_steps = n;
        for (int k : s->members) s->slots[k].sys.step += (uint64_t)n;
    } else {
        if ((st = enqueue_group_steps(s, n)) != RBE_OK) return st;
    }
    s->last_key = key;
    // every member's latched device errors, read once the chunk is complete
    std::vector<const Slot*> pub;
    for (int k : s->members) {
        Slot& sl = s->slots[k];
        pub.push_back(&sl);
        sl.in_flight = true;
        sl.chunk_in_flight = n;
    }
    if ((e = publish_status(s->gstream, pub.data(), (int)pub.size())) != cudaSuccess)
        return sfail(s, RBE_ECUDA, std::string("group status: ") + cudaGetErrorString(e));
    if ((e = cudaEventRecord(s->gdone, s->gstream)) != cudaSuccess)
        return sfail(s, RBE_ECUDA, std::string("group event: ") + cudaGetErrorString(e));
    s->group_in_flight = true;
    s->group_steps = n;
    s->group_t_launch = now_s(s);
    return RBE_OK;
}

// Whether a request can run in a lockstep group (the batched k-space samples exactly, without a
// pressure batch or reuse, on the FP32-phase path).
static bool group_eligible(const rbe_request& r)
{
    return r.sampler == RBE_SAMPLER_EXACT && r.ptilde == 0 && r.reuse <= 1 && r.params.kspace == 1;
}

}  // namespace rbe

using namespace rbe;

extern "C" {

rbe_status rbe_server_create(const rbe_server_config* cfg, rbe_server* out)
{
    if (!cfg || !out) return fail(nullptr, RBE_EINVAL, "cfg and out must not be NULL");
    if (!(cfg->alpha > 0.0) || cfg->P < 1 || cfg->P > 65536 || cfg->max_slots < 1 || cfg->max_slots > 4096 ||
        cfg->chunk_steps < 1 || cfg->mem_budget <= 0 ||
        (cfg->precision != RBE_FP64 && cfg->precision != RBE_FP32_PHASE) || cfg->batched < 0 || cfg->batched > 2)
        return fail(nullptr, RBE_EINVAL, "invalid server configuration");
    if (cfg->batched && cfg->precision != RBE_FP32_PHASE)
        return fail(nullptr, RBE_EINVAL, "lockstep groups run the batched FP32-phase k-space: precision RBE_FP32_PHASE");
    rbe_server s = new (std::nothrow) rbe_server_s();
    if (!s) return fail(nullptr, RBE_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    s->slots.resize(cfg->max_slots);
    s->t0 = Clock::now();
    cudaGetDevice(&s->device);
    if (cfg->batched) {
        cudaError_t e = cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->gfork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->gk, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->gdone, cudaEventDisableTiming);
        s->ev_a.assign(cfg->max_slots, nullptr);
        s->ev_b.assign(cfg->max_slots, nullptr);
        for (int k = 0; k < cfg->max_slots && e == cudaSuccess; ++k) {
            e = cudaEventCreateWithFlags(&s->ev_a[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_b[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            rbe_server_destroy(s);
            return fail(nullptr, RBE_ECUDA, std::string("server group stream: ") + cudaGetErrorString(e));
        }
    }
    *out = s;
    return RBE_OK;
}

rbe_status rbe_server_destroy(rbe_server s)
{
    if (!s) return RBE_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    if (s->gstream) cudaStreamSynchronize(s->gstream);
    if (s->ggraph) cudaGraphExecDestroy(s->ggraph);
    if (s->batch) rbe_batch_destroy(s->batch);
    for (cudaEvent_t ev : {s->gfork, s->gk, s->gdone})
        if (ev) cudaEventDestroy(ev);
    for (auto* v : {&s->ev_a, &s->ev_b})
        for (cudaEvent_t ev : *v)
            if (ev) cudaEventDestroy(ev);
    if (s->gstream) cudaStreamDestroy(s->gstream);
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.graph) cudaGraphExecDestroy(sl.graph);
        if (sl.ctx) rbe_destroy(sl.ctx);  // frees its scratch on the slot's stream
        for (double* p : {sl.pos, sl.mom, sl.force, sl.charge, sl.mass, sl.cell})
            if (p) cudaFreeAsync(p, sl.stream);
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_status) cudaFreeHost(sl.h_status);
    }
    if (cur >= 0 && cur != s->device) cudaSetDevice(cur);
    delete s;
    return RBE_OK;
}

rbe_status rbe_server_submit(rbe_server s, const rbe_request* req, int64_t* id)
{
    if (!s || !req || !id) return fail(nullptr, RBE_EINVAL, "NULL argument");
    const int64_t N = req->N;
    if (N < 1 || N > ((int64_t)1 << 31) - 256 || req->nsteps < 1 || !req->pos || !req->mom || !req->charge ||
        !req->mass)
        return sfail(s, RBE_EINVAL, "invalid request");
    for (int t = 0; t < 3; ++t)
        if (!(req->box[t] > 0.0)) return sfail(s, RBE_EINVAL, "box lengths must be > 0");
    if (req->sampler < 0 || req->sampler > 2 || req->ptilde < 0 || req->ptilde > 65536 || req->reuse < 0 ||
        req->reuse > 1024)
        return sfail(s, RBE_EINVAL, "invalid sampler, pressure batch or reuse");
    if (req->sampler == 2 && req->reuse > 1)
        return sfail(s, RBE_EINVAL, "sample reuse and the Metropolis-Hastings chain exclude each other");
    if (s->cfg.batched && !group_eligible(*req))
        return sfail(s, RBE_EINVAL, "lockstep groups serve requests with the exact sampler, no pressure batch, no "
                                    "sample reuse and the k-space on");
    if (replica_bytes(*req, s->cfg.P) > s->cfg.mem_budget)
        return sfail(s, RBE_ENOMEM, "request larger than the whole memory budget");
    auto rq = std::make_unique<Request>();
    rq->r = *req;
    rq->pos.assign(req->pos, req->pos + 3 * N);
    rq->mom.assign(req->mom, req->mom + 3 * N);
    rq->q.assign(req->charge, req->charge + N);
    rq->m.assign(req->mass, req->mass + N);
    rq->r.pos = rq->pos.data();
    rq->r.mom = rq->mom.data();
    rq->r.charge = rq->q.data();
    rq->r.mass = rq->m.data();
    rq->t_submit = now_s(s);
    *id = (int64_t)s->reqs.size();
    s->reqs.push_back(std::move(rq));
    s->queue.push_back(*id);
    return RBE_OK;
}

rbe_status rbe_server_progress(rbe_server s, int32_t wait, int32_t* n_queued, int32_t* n_active, int64_t* n_done)
{
    if (!s) return RBE_EINVAL;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    bool any_done = false;
    for (;;) {
        // 1. observe finished chunks (a lockstep group's chunk completes for all members at once)
        if (s->cfg.batched && s->group_in_flight) {
            const cudaError_t q = cudaEventQuery(s->gdone);
            if (q != cudaErrorNotReady) {
                if (q != cudaSuccess) return sfail(s, RBE_ECUDA, std::string("cudaEventQuery: ") + cudaGetErrorString(q));
                const double now = now_s(s);
                s->group_in_flight = false;
                any_done = true;
                for (int k : s->members) {
                    Slot& sl = s->slots[k];
                    s->latencies.push_back(now - s->group_t_launch);
                    sl.in_flight = false;
                    sl.steps_left -= sl.chunk_in_flight;
                    s->steps_done += sl.chunk_in_flight;
                    const unsigned bits = *static_cast<volatile unsigned*>(sl.h_status);
                    if (bits) {
                        const rbe_status st = status_from_bits(sl.ctx, bits);
                        evict(s, sl, 3, st, std::string("evicted after step ") + std::to_string(sl.sys.step) + ": " +
                                                rbe_last_error(sl.ctx));
                    } else if (sl.cancel) {
                        evict(s, sl, 4, RBE_ESTATE, "request cancelled");
                    } else if (sl.steps_left <= 0) {
                        retire(s, sl);
                    }
                }
            }
        }
        for (Slot& sl : s->slots) {
            if (s->cfg.batched || !sl.busy || !sl.in_flight) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return sfail(s, RBE_ECUDA, std::string("cudaEventQuery: ") + cudaGetErrorString(q));
            s->latencies.push_back(now_s(s) - sl.t_launch);
            sl.in_flight = false;
            sl.steps_left -= sl.chunk_in_flight;
            s->steps_done += sl.chunk_in_flight;
            any_done = true;
            const unsigned bits = *static_cast<volatile unsigned*>(sl.h_status);
            if (bits) {
                const rbe_status st = status_from_bits(sl.ctx, bits);
                evict(s, sl, 3, st, std::string("evicted after step ") + std::to_string(sl.sys.step) + ": " +
                                        rbe_last_error(sl.ctx));
            } else if (sl.cancel) {
                evict(s, sl, 4, RBE_ESTATE, "request cancelled");
            } else if (sl.steps_left <= 0) {
                retire(s, sl);
            }
        }
        // 2. admit while a slot is free and the budget allows (first come, first served); lockstep
        //    groups admit between chunks
        while (!s->queue.empty() && !(s->cfg.batched && s->group_in_flight)) {
            const int64_t id = s->queue.front();
            const int64_t need = replica_bytes(s->reqs[id]->r, s->cfg.P);
            if (s->mem_used + need > s->cfg.mem_budget) break;
            Slot* free_slot = nullptr;
            for (Slot& sl : s->slots)
                if (!sl.busy) {
                    free_slot = &sl;
                    break;
                }
            if (!free_slot) break;
            s->queue.pop_front();
            const rbe_status st = admit(s, *free_slot, id);
            if (st != RBE_OK) {
                s->reqs[id]->state = 3;
                s->reqs[id]->error = st;
                s->reqs[id]->error_msg = s->last_error;
                ++s->n_done;
                return st;
            }
        }
        // 3. next chunk of every resident replica that is idle (lockstep: of the whole group)
        if (s->cfg.batched) {
            if (!s->group_in_flight) {
                const rbe_status st = launch_group_chunk(s);
                if (st != RBE_OK) return st;
            }
        } else {
            for (Slot& sl : s->slots)
                if (sl.busy && !sl.in_flight && sl.steps_left > 0) {
                    const rbe_status st = launch_chunk(s, sl);
                    if (st != RBE_OK) return st;
                }
        }
        bool active = false;
        for (const Slot& sl : s->slots) active = active || sl.busy;
        if (!wait || any_done || (!active && s->queue.empty())) break;
    }
    int32_t na = 0;
    for (const Slot& sl : s->slots) na += sl.busy ? 1 : 0;
    if (n_queued) *n_queued = (int32_t)s->queue.size();
    if (n_active) *n_active = na;
    if (n_done) *n_done = s->n_done;
    return RBE_OK;
}

rbe_status rbe_server_cancel(rbe_server s, int64_t id)
{
    if (!s || id < 0 || id >= (int64_t)s->reqs.size()) return RBE_EINVAL;
    Request& rq = *s->reqs[id];
    if (rq.state == 0) {
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
            if (*it == id) {
                s->queue.erase(it);
                break;
            }
        rq.state = 4;
        rq.error = RBE_ESTATE;
        rq.error_msg = "request cancelled";
        ++s->n_done;
        return RBE_OK;
    }
    if (rq.state != 1) return sfail(s, RBE_ESTATE, "request already finished");
    for (Slot& sl : s->slots)
        if (sl.busy && sl.req == id) {
            if (sl.in_flight) {
                sl.cancel = true;  // progress() ends it when its chunk completes
            } else {
                int cur = -1;
                cudaGetDevice(&cur);
                if (cur != s->device) cudaSetDevice(s->device);
                evict(s, sl, 4, RBE_ESTATE, "request cancelled");
                if (cur >= 0 && cur != s->device) cudaSetDevice(cur);
            }
            return RBE_OK;
        }
    return sfail(s, RBE_ESTATE, "request not resident");
}

rbe_status rbe_server_request_state(rbe_server s, int64_t id, int32_t* state, rbe_status* error)
{
    if (!s || id < 0 || id >= (int64_t)s->reqs.size()) return RBE_EINVAL;
    const Request& rq = *s->reqs[id];
    if (state) *state = rq.state;
    if (error) *error = rq.state >= 3 ? rq.error : RBE_OK;
    return RBE_OK;
}

rbe_status rbe_server_result(rbe_server s, int64_t id, double* pos, double* mom, double* cell)
{
    if (!s || id < 0 || id >= (int64_t)s->reqs.size()) return RBE_EINVAL;
    const Request& rq = *s->reqs[id];
    if (rq.state == 4) return sfail(s, RBE_ESTATE, "request cancelled");
    if (rq.state == 3) return sfail(s, rq.error, "request failed: " + rq.error_msg);
    if (rq.state != 2) return sfail(s, RBE_ESTATE, "request not finished");
    const int64_t N = rq.r.N;
    if (pos) std::memcpy(pos, rq.out_pos.data(), sizeof(double) * 3 * N);
    if (mom) std::memcpy(mom, rq.out_mom.data(), sizeof(double) * 3 * N);
    if (cell) std::memcpy(cell, rq.out_cell.data(), sizeof(double) * RBE_CELL_DOUBLES);
    return RBE_OK;
}

rbe_status rbe_server_stats(rbe_server s, double* chunk_latency, int64_t capacity, int64_t* n_chunks,
                            int64_t* steps_done, double* span_seconds)
{
    if (!s) return RBE_EINVAL;
    const int64_t n = (int64_t)s->latencies.size();
    if (chunk_latency)
        std::memcpy(chunk_latency, s->latencies.data(), sizeof(double) * (size_t)std::min(n, std::max<int64_t>(capacity, 0)));
    if (n_chunks) *n_chunks = n;
    if (steps_done) *steps_done = s->steps_done;
    if (span_seconds) *span_seconds = s->t_first_admit >= 0.0 ? s->t_last_done - s->t_first_admit : 0.0;
    return RBE_OK;
}

const char* rbe_server_last_error(rbe_server s) { return s ? s->last_error.c_str() : ""; }

}  // extern "C"
