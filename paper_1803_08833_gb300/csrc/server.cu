// server.cu -- continuous-batching simulation server (host runtime).
//
// Requests (a network description and a number of time steps) queue with
// their arrival time.  Each tick admits queued requests in arrival order
// while their estimated device footprint fits the memory budget (the
// network's state then stays resident on the device), advances every
// resident network by up to one chunk of steps in a single batched
// persistent launch, and retires the networks that have finished: their
// counters, a hash of their spike raster and of their final membrane
// potentials are recorded, their memory is released and the freed budget is
// available to the next tick.  Requests that arrive while others run join
// at the next tick.  Retirement is pipelined: a network that finishes in one
// tick is read back (on a side stream) and released while the next tick's
// batch runs, so the host work of retiring overlaps the GPU.
#include "snn.h"
#include "snn_internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// FNV-1a over bytes.
uint64_t fnv(const void* p, size_t n, uint64_t h) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

struct Pending {
    uint64_t id;
    snn_config cfg;
    uint32_t steps;
    uint64_t arrival_ns;
    uint64_t bytes;
};

struct Active {
    Pending req;
    snn_net* net;
    uint32_t done;
    uint64_t admit_ns;
    uint64_t bytes;
    uint64_t finish_ns;  // end of the tick that ran its last chunk
};

snn_status sfail(snn_status s, const std::string& m) {
    snn::set_last_error(m.c_str());
    return s;
}

}  // namespace

struct snn_server {
    uint64_t budget = 0, used = 0;
    uint32_t chunk = 0, max_slots = 0;
    int32_t batch_mode = SNN_BATCH_GROUPS, batch_shape = 0;  // layout of every tick's batch
    uint64_t batch_budget = 0;                                // its ring budget (0: the batch's default)
    snn_alloc_fn alloc_fn = nullptr;
    snn_free_fn free_fn = nullptr;
    void* alloc_ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;  // read-back of finished networks while the next batch runs
    uint64_t next_id = 1;
    std::deque<Pending> queue;
    std::vector<Active> active;
    std::vector<Active> finished;  // ran their last chunk, not yet retired
    std::vector<snn_request_result> done;
    uint64_t ticks = 0, launches = 0;
    uint64_t rec_events = 0, ext_events = 0, steps = 0;
    uint64_t busy_ns = 0;  // host time spent inside ticks that ran networks
};

extern "C" {

uint64_t snn_now_ns(void) { return now_ns(); }

uint64_t snn_estimate_bytes(const snn_config* c) {
    if (!c) return 0;
    const uint64_t N = (uint64_t)c->grid_w * c->grid_h * c->neurons_per_module;
    const uint64_t Npad = (N + 1023) / 1024 * 1024;
    uint64_t K = c->K, temp = 0;
    if (c->conn_rule == SNN_RULE_PAIRWISE) {
        uint32_t mr = 0, st = 0;
        snn::pairwise_bounds(*c, &mr, &st);
        K = mr;
        temp = N * st * 2;  // per-entry counts, held during construction
    }
    const uint64_t Kpad = (K + 7) / 8 * 8;
    const uint64_t wb = c->weight_dtype == SNN_WEIGHT_BF16 ? 2 : 4;
    const uint64_t D = (uint64_t)std::max(c->d_exc_hi, c->d_inh) + 1;
    const double q = c->cutoff_um / (double)c->spacing_um;
    const uint64_t off = (uint64_t)(3.2 * q * q + 8 * q + 8);  // bound on the stencil size
    const uint64_t modules = (uint64_t)c->grid_w * c->grid_h;
    uint64_t b = N * Kpad * (4 + wb) + temp;          // synapse table (target | delay word, weight)
    b += Npad * (4 + 4 + 1 + 4 + 4) + D * Npad * 4;    // state, staging, ring
    b += c->raster_capacity * 8 + modules * off * 16;  // raster, tables
    if (c->table_layout == SNN_LAYOUT_GROUPED) b += N * (off + 1) * 2;
    return b + (4u << 20);                             // small buffers and rounding
}

snn_status snn_server_create(uint64_t budget_bytes, uint32_t chunk_steps, uint32_t max_slots, snn_alloc_fn alloc_fn,
                             snn_free_fn free_fn, void* alloc_ctx, void* stream, snn_server** out) {
    if (!out) return sfail(SNN_EINVAL, "out is NULL");
    *out = nullptr;
    if (budget_bytes == 0 || chunk_steps == 0 || max_slots == 0)
        return sfail(SNN_EINVAL, "budget, chunk and slots must be positive");
    if ((alloc_fn == nullptr) != (free_fn == nullptr))
        return sfail(SNN_EINVAL, "alloc_fn and free_fn must both be set or both be NULL");
    snn_server* s = new (std::nothrow) snn_server();
    if (!s) return sfail(SNN_ENOMEM, "host allocation failed");
    s->budget = budget_bytes;
    s->chunk = chunk_steps;
    s->max_slots = max_slots;
    s->alloc_fn = alloc_fn;
    s->free_fn = free_fn;
    s->alloc_ctx = alloc_ctx;
    s->stream = (cudaStream_t)stream;
    if (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return sfail(SNN_ECUDA, "cudaStreamCreateWithFlags failed");
    }
    *out = s;
    return SNN_OK;
}

snn_status snn_server_set_batch(snn_server* s, int32_t mode, int32_t shape, uint64_t ring_budget) {
    if (!s) return sfail(SNN_EINVAL, "server is NULL");
    if ((mode != SNN_BATCH_GROUPS && mode != SNN_BATCH_GLOBAL) || (shape != 0 && shape != 1))
        return sfail(SNN_EINVAL, "unknown batch layout or shape");
    s->batch_mode = mode;
    s->batch_shape = shape;
    s->batch_budget = ring_budget;
    return SNN_OK;
}

snn_status snn_server_submit(snn_server* s, const snn_config* cfg, uint32_t n_steps, uint64_t arrival_ns,
                             uint64_t* request_id) {
    if (!s || !cfg) return sfail(SNN_EINVAL, "server or config is NULL");
    if (cfg->stdp) return sfail(SNN_EINVAL, "the server runs static synapses (stdp = 0)");
    Pending p;
    p.id = s->next_id++;
    p.cfg = *cfg;
    p.steps = n_steps;
    p.arrival_ns = arrival_ns ? arrival_ns : now_ns();
    p.bytes = snn_estimate_bytes(cfg);
    if (p.bytes > s->budget)
        return sfail(SNN_EBUDGET, "request needs ~" + std::to_string(p.bytes >> 20) + " MiB, over the budget");
    s->queue.push_back(p);
    if (request_id) *request_id = p.id;
    return SNN_OK;
}

// Reads back a finished network's counters, raster and final potentials (on
// the side stream: its last batch has completed) and releases it.
static snn_status retire(snn_server* s, Active& a) {
    const uint64_t t_ns = a.finish_ns;
    cudaStream_t rs = s->side;
    snn_request_result r{};
    r.request_id = a.req.id;
    r.status = SNN_OK;
    snn_stats st{};
    snn_status e = snn_get_stats(a.net, &st, rs);
    if (e != SNN_OK) r.status = e;
    r.steps = st.steps;
    r.n_spikes = st.n_spikes;
    r.rec_events = st.rec_events;
    r.ext_events = st.ext_events;
    // hashes of the raster and of the final membrane potentials
    const size_t cap = (size_t)std::min<uint64_t>(st.raster_count, a.req.cfg.raster_capacity);
    std::vector<uint32_t> steps(cap), ids(cap);
    size_t got = 0;
    e = snn_read_spikes(a.net, steps.data(), ids.data(), cap, &got, rs);
    if (e == SNN_EOVERFLOW)
        r.raster_overflow = 1;  // the raster kept its first `cap` spikes; the counters are complete
    else if (e != SNN_OK && r.status == SNN_OK)
        r.status = e;
    uint64_t h = 1469598103934665603ull;
    h = fnv(steps.data(), got * 4, h);
    h = fnv(ids.data(), got * 4, h);
    r.raster_hash = h;
    uint32_t N = 0;
    snn_get_dims(a.net, &N, nullptr, nullptr, nullptr);
    std::vector<float> V(N);
    snn_get_state(a.net, V.data(), nullptr, nullptr, nullptr, nullptr, rs);
    r.state_hash = fnv(V.data(), (size_t)N * 4, 1469598103934665603ull);
    r.queue_ms = (double)(a.admit_ns - a.req.arrival_ns) / 1e6;
    r.latency_ms = (double)(t_ns - a.req.arrival_ns) / 1e6;
    s->rec_events += st.rec_events;
    s->ext_events += st.ext_events;
    s->steps += st.steps;
    snn_destroy(a.net);
    s->used -= a.bytes;
    s->done.push_back(r);
    return SNN_OK;
}

snn_status snn_server_tick(snn_server* s, uint32_t* n_active, uint32_t* n_queued) {
    if (!s) return sfail(SNN_EINVAL, "server is NULL");
    snn::NvtxRange range("snn_server_tick");
    s->ticks += 1;
    // admission: arrival order, while the footprint fits the budget
    while (!s->queue.empty() && s->active.size() < s->max_slots && s->used + s->queue.front().bytes <= s->budget) {
        Pending p = s->queue.front();
        s->queue.pop_front();
        snn_net* net = nullptr;
        snn_status e = snn_build_network(&p.cfg, s->alloc_fn, s->free_fn, s->alloc_ctx, s->stream, &net);
        if (e != SNN_OK) {
            snn_request_result r{};
            r.request_id = p.id;
            r.status = e;
            r.latency_ms = (double)(now_ns() - p.arrival_ns) / 1e6;
            s->done.push_back(r);
            continue;
        }
        snn_set_schedule(net, 2, 0);
        Active a{p, net, 0, now_ns(), p.bytes, 0};
        s->used += p.bytes;
        s->active.push_back(a);
    }
    if (!s->active.empty()) {
        const uint64_t t0 = now_ns();
        std::vector<snn_net*> nets;
        std::vector<uint32_t> steps;
        for (auto& a : s->active) {
            nets.push_back(a.net);
            steps.push_back(std::min(s->chunk, a.req.steps - a.done));
        }
        snn_batch* b = nullptr;
        snn_status e = snn_batch_create(nets.data(), (uint32_t)nets.size(), s->alloc_fn, s->free_fn, s->alloc_ctx, &b);
        if (e != SNN_OK) return e;
        // a non-default layout regroups the waves once (set_mode and set_shape
        // each regroup; the budget call regroups for both)
        if (s->batch_mode != SNN_BATCH_GROUPS || s->batch_shape != 0 || s->batch_budget) {
            uint64_t bud = 0;
            uint32_t waves = 0;
            snn_batch_waves(b, &waves, &bud);
            e = snn_batch_set_layout(b, s->batch_mode, s->batch_shape, s->batch_budget ? s->batch_budget : bud);
        }
        if (e == SNN_OK) e = snn_batch_step(b, steps.data(), s->stream);
        // while the batch runs: retire the networks that finished in the previous tick
        for (auto& a : s->finished) retire(s, a);
        s->finished.clear();
        if (e == SNN_OK && cudaStreamSynchronize(s->stream) != cudaSuccess)
            e = sfail(SNN_ECUDA, "stream synchronisation after the batch launch failed");
        snn_batch_destroy(b);
        if (e != SNN_OK) return e;
        s->launches += 1;
        const uint64_t t1 = now_ns();
        s->busy_ns += t1 - t0;
        std::vector<Active> keep;
        for (size_t i = 0; i < s->active.size(); ++i) {
            Active& a = s->active[i];
            a.done += steps[i];
            if (a.done >= a.req.steps) {
                a.finish_ns = t1;
                s->finished.push_back(a);
            } else {
                keep.push_back(a);
            }
        }
        s->active.swap(keep);
    } else {
        for (auto& a : s->finished) retire(s, a);  // nothing runs: retire at once
        s->finished.clear();
    }
    if (n_active) *n_active = (uint32_t)(s->active.size() + s->finished.size());
    if (n_queued) *n_queued = (uint32_t)s->queue.size();
    return SNN_OK;
}

snn_status snn_server_poll(snn_server* s, snn_request_result* out, uint32_t cap, uint32_t* n_out) {
    if (!s || !n_out) return sfail(SNN_EINVAL, "server or n_out is NULL");
    const uint32_t n = (uint32_t)std::min<size_t>(cap, s->done.size());
    if (out) std::copy(s->done.begin(), s->done.begin() + n, out);
    s->done.erase(s->done.begin(), s->done.begin() + n);
    *n_out = n;
    return SNN_OK;
}

snn_status snn_server_stats(snn_server* s, snn_server_stats_t* out) {
    if (!s || !out) return sfail(SNN_EINVAL, "server or out is NULL");
    out->ticks = s->ticks;
    out->launches = s->launches;
    out->rec_events = s->rec_events;
    out->ext_events = s->ext_events;
    out->steps = s->steps;
    out->busy_ns = s->busy_ns;
    out->used_bytes = s->used;
    out->active = (uint32_t)(s->active.size() + s->finished.size());
    out->queued = (uint32_t)s->queue.size();
    return SNN_OK;
}

void snn_server_destroy(snn_server* s) {
    if (!s) return;
    for (auto& a : s->active) snn_destroy(a.net);
    for (auto& a : s->finished) snn_destroy(a.net);
    if (s->side) cudaStreamDestroy(s->side);
    delete s;
}

}  // extern "C"
