// sw_server.cu -- serving loop: continuous batching of database searches
// against a device-resident database.
//
// The database (sorted by length) is cut into C chunks of subject pairs.
// Active requests sweep it circularly: one server step launches the packed
// 16-bit search over the current chunk for every active request at once
// (one job per request; blocks of all jobs run concurrently and share the
// chunk's residues through L2).  A request is admitted into a free slot as
// soon as one exists and its device memory fits the budget, joins the sweep
// at the next step, and retires after it has visited all C chunks: its
// flagged subjects are rescored exactly in 32 bits and its top-k hits are
// taken from its per-request score array, which lives on the device for the
// request's whole life.  A request's result does not depend on which other
// requests shared its steps.  Steps are pipelined: a step is enqueued before
// the host waits for the previous one, so a request's hits are ready after
// the step call that follows its last chunk's.
#include "sw.h"
#include "sw_ctx.h"
#include "dbsearch.cuh"
#include "wavefront.cuh"
#include "aux_kernels.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

using namespace swgb;

#define CU(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; } } while (0)
#define RC(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)


namespace {

constexpr double kOversub = 4.0;     // blocks per step, in units of the blocks resident at once

struct Slot {
    bool active = false;
    uint64_t ticket = 0;
    int64_t m = 0;
    int enq = 0;                     // chunks enqueued
    int visited = 0;                 // chunks completed
    DevBuf q, scores, ovf, ctr;      // ctr: [novf, next_pair of even steps, next_pair of odd steps]
};

struct Done {
    int status = SW_OK;
    std::vector<sw_dbhit> hits;
};

// The step on the device while the host prepares the next one: its requests, and how many
// tile-shape groups (streams) it launched.
struct InFlight {
    bool on = false;
    int parity = 0;
    int ngroups = 0;
    std::vector<Slot *> slots;
};

}  // namespace

struct sw_server {
    sw_ctx *c = nullptr;
    const sw_db *db = nullptr;
    DevScoring ds;
    int k = 20;
    size_t mem_budget = 0, mem_used = 0;
    int chunks = 16;
    int cur_chunk = 0;
    uint64_t next_ticket = 1;
    std::vector<Slot> slots;         // fixed at creation (in-flight steps hold pointers into it)
    std::map<uint64_t, Done> done;
    DbView view{};
    int64_t nseq = 0;
    int maxK = 0;
    long long cells_done = 0;        // cells of retired requests
    int64_t total_res = 0;
    // Steps are pipelined: step n is enqueued before the host waits for step n - 1, so the device
    // never idles between steps.  Each step's tile-shape groups run on streams of their own
    // (one group's tail fills with the others' blocks), with their own boundary-row scratch and
    // slot pools.  Whatever a step in flight reads or writes belongs to the server: job tables and
    // per-request work counters alternate between even and odd steps, and the scoring table and
    // error word are the server's, so the context's other calls may run meanwhile.
    DevBuf jobs[2];
    HostBuf hjobs[2];
    DevBuf dscore, derr;
    HostBuf herr;
    std::vector<cudaStream_t> gstreams;
    std::vector<cudaEvent_t> gdone[2];   // group g of an even / odd step done
    cudaEvent_t fork[2] = {nullptr, nullptr};
    std::deque<DevBuf> grows, gslots;
    long long nstep = 0;             // steps enqueued
    InFlight inflight;
    int failed = SW_OK;              // a device error of a step: every later request fails with it
    ~sw_server() {
        for (int p = 0; p < 2; ++p) {
            for (cudaEvent_t e : gdone[p]) if (e) cudaEventDestroy(e);
            if (fork[p]) cudaEventDestroy(fork[p]);
        }
        for (cudaStream_t t : gstreams) if (t) cudaStreamDestroy(t);
    }
};

namespace {

size_t slot_bytes(const sw_server *S, int64_t m) {
    return (size_t)m + 256 + 2 * (size_t)std::max<int64_t>(1, S->nseq) * sizeof(int32_t) + 256;
}

// Retire a request that has seen every chunk: exact rescoring, top-k; its
// slot (and the slot's device buffers, kept for the next request, since the
// database size fixes them) becomes free.  A request of a failed step
// retires with that step's status.
int retire_work(sw_server *S, Slot &s, Done &d);

int retire(sw_server *S, Slot &s, int status) {
    Done d;
    const int rc = status != SW_OK ? status : retire_work(S, s, d);
    if (rc != SW_OK) d = Done{rc, {}};        // the request fails, the slot is freed all the same
    S->done[s.ticket] = std::move(d);
    S->cells_done += (long long)s.m * S->total_res;
    S->mem_used -= slot_bytes(S, s.m);
    s.active = false;
    return rc;
}

int retire_work(sw_server *S, Slot &s, Done &d) {
    sw_ctx *c = S->c;
    int32_t nflag = 0;
    CU(cudaMemcpyAsync(c->stage3.p, s.ctr.p, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    std::memcpy(&nflag, c->stage3.p, sizeof(int32_t));
    if (nflag > 0) {
        // rescore the flagged subjects exactly: reuse the search path's rescoring on this slot
        std::vector<int32_t> flagged((size_t)nflag);
        CU(cudaMemcpyAsync(flagged.data(), s.ovf.p, (size_t)nflag * sizeof(int32_t), cudaMemcpyDeviceToHost,
                           c->stream));
        CU(cudaStreamSynchronize(c->stream));
        RC(db_rescore(c, S->db, static_cast<const uint8_t *>(s.q.p), s.m, S->ds, flagged,
                      static_cast<int32_t *>(s.scores.p)));
    }
    const int kk = (int)std::min<int64_t>(S->k, S->nseq);
    if (kk > 0) {
        RC(c->result.ensure(64 * sizeof(int4)));
        RC(db_topk(c, static_cast<const int32_t *>(s.scores.p), S->nseq, kk, static_cast<int2 *>(c->result.p)));
        CU(cudaMemcpyAsync(c->stage3.p, c->result.p, (size_t)kk * sizeof(int2), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        const int2 *h = static_cast<const int2 *>(c->stage3.p);
        for (int i = 0; i < kk; ++i) d.hits.push_back(sw_dbhit{(int64_t)h[i].x, h[i].y, 0});
    }
    return SW_OK;
}

// Wait for the step in flight; count its chunk for each of its requests and
// retire those that have seen every chunk.
int complete_inflight(sw_server *S) {
    InFlight &f = S->inflight;
    if (!f.on) return SW_OK;
    f.on = false;
    sw_ctx *c = S->c;
    int rc = SW_OK;
    for (int g = 0; g < f.ngroups; ++g)
        if (cudaEventSynchronize(S->gdone[f.parity][g]) != cudaSuccess) { cudaGetLastError(); rc = SW_ECUDA; }
    if (rc == SW_OK) {
        if (cudaMemcpyAsync(S->herr.p, S->derr.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            cudaGetLastError();
            rc = SW_ECUDA;
        } else {
            rc = map_kernel_error(*static_cast<const int *>(S->herr.p));
        }
    }
    if (rc != SW_OK && S->failed == SW_OK) S->failed = rc;
    int first = rc;
    for (Slot *s : f.slots)                  // every finished request retires, even after a failure
        if (++s->visited >= S->chunks) {
            const int r = retire(S, *s, S->failed);
            if (r != SW_OK && first == SW_OK) first = r;
        }
    f.slots.clear();
    return first;
}

// Enqueue one sweep step for the requests `act` (each has chunks left to
// enqueue) on the groups' streams; it becomes the step in flight in *next.
// *early receives the status of the step in flight if it had to be
// completed first (a group's scratch had to grow while it may be in use).
int enqueue_step(sw_server *S, const std::vector<Slot *> &act, InFlight *next, int *early) {
    sw_ctx *c = S->c;
    const int par = (int)(S->nstep & 1);
    // chunk c = pairs c, c + C, c + 2C, ...: every chunk mixes long and short subjects
    const int np = S->view.npairs;
    const int p0 = S->cur_chunk, p1 = np, stride = S->chunks;
    const int chunk_pairs = p0 < np ? (np - p0 + stride - 1) / stride : 0;
    // the requests of a step run in groups of one tile shape each, every query with the shape
    // that pads it least (one shape for all would pad a 100-residue query to a 512-row pass
    // next to a long one); one launch per group
    std::map<int, std::vector<Slot *>> groups;
    for (Slot *s : act) groups[db_shape(S->ds.K, (int)s->m)].push_back(s);
    std::vector<DbJob> jobs;
    struct Launch { int shape, job0, njobs, nblocks, maxm; };
    std::vector<Launch> launches;
    for (const auto &g : groups) {
        const int shape = g.first;
        int64_t maxm = 0;
        for (Slot *s : g.second) maxm = std::max(maxm, s->m);
        int resident = 0;
        RC(db_resident_blocks_shape(c, shape, S->ds.K, (int)maxm, &resident));
        const int W = db_shape_warps(shape), rows = db_shape_rows(shape);
        // a request's work is its query padded to whole passes of `rows` rows
        auto padded = [&](int64_t m) { return (double)((m + rows - 1) / rows) * rows; };
        double sumpad = 0;
        for (Slot *s : g.second) sumpad += padded(s->m);
        Launch L{shape, (int)jobs.size(), (int)g.second.size(), 0, (int)maxm};
        for (Slot *s : g.second) {
            DbJob j;
            j.q = static_cast<const uint8_t *>(s->q.p);
            j.m = (int32_t)s->m;
            j.scoring = 0;
            j.pair0 = p0; j.pair1 = p1; j.pair_stride = stride;
            // blocks in proportion to the request's share of the group's work, kOversub times what
            // fits at once: blocks of short jobs finish early and free their SMs for the others
            const int share = (int)std::ceil(kOversub * resident * padded(s->m) / std::max(1.0, sumpad));
            const int nb = std::max(1, std::min(share, (chunk_pairs + W - 1) / W));
            j.block0 = L.nblocks;
            L.nblocks += nb;
            j.scores = static_cast<int32_t *>(s->scores.p);
            j.ovf = static_cast<int32_t *>(s->ovf.p);
            j.novf = static_cast<int32_t *>(s->ctr.p);
            j.next_pair = static_cast<int32_t *>(s->ctr.p) + 1 + par;
            jobs.push_back(j);
        }
        launches.push_back(L);
    }
    const int ng = chunk_pairs > 0 ? (int)launches.size() : 0;
    DbView v = S->view;
    v.maxlen = std::max(1, db_chunk_maxlen(S->db, p0, p0 + 1));     // pairs are sorted longest first
    while ((int)S->gstreams.size() < ng) {
        cudaStream_t t = nullptr;
        CU(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking));
        S->gstreams.push_back(t);
    }
    for (int p = 0; p < 2; ++p)
        while ((int)S->gdone[p].size() < ng) {
            cudaEvent_t e = nullptr;
            CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            S->gdone[p].push_back(e);
        }
    while ((int)S->grows.size() < ng) {
        S->grows.emplace_back();
        S->gslots.emplace_back();
    }
    // a group's scratch that must grow may still be in use by the step in flight (the same
    // stream's previous launch): complete that step before the buffer is reallocated
    std::vector<size_t> rneed((size_t)ng), sneed((size_t)ng);
    bool grow = false;
    for (int g = 0; g < ng; ++g) {
        RC(db_scratch_shape(c, launches[g].shape, S->ds.K, launches[g].maxm, v.maxlen, &rneed[g], &sneed[g]));
        grow = grow || rneed[g] > S->grows[g].cap || sneed[g] > S->gslots[g].cap;
    }
    if (grow) *early = complete_inflight(S);
    for (int g = 0; g < ng; ++g) {
        RC(S->grows[g].ensure(rneed[g]));
        RC(S->gslots[g].ensure(sneed[g]));
    }
    // the job table and the work counters of this parity were last used by step nstep - 2,
    // which has completed
    const cudaStream_t home = c->stream;
    const size_t jb = std::max<size_t>(1, jobs.size()) * sizeof(DbJob);
    RC(S->jobs[par].ensure(jb));
    RC(S->hjobs[par].ensure(jb));
    if (!jobs.empty()) std::memcpy(S->hjobs[par].p, jobs.data(), jobs.size() * sizeof(DbJob));
    CU(cudaMemcpyAsync(S->jobs[par].p, S->hjobs[par].p, jobs.size() * sizeof(DbJob), cudaMemcpyHostToDevice, home));
    for (Slot *s : act) CU(cudaMemsetAsync(static_cast<int32_t *>(s->ctr.p) + 1 + par, 0, sizeof(int32_t), home));
    CU(cudaEventRecord(S->fork[par], home));
    const DbJob *djobs = static_cast<const DbJob *>(S->jobs[par].p);
    int rc = SW_OK;
    int launched = 0;
    for (int g = 0; g < ng && rc == SW_OK; ++g) {
        const Launch &L = launches[g];
        const cudaStream_t gs = S->gstreams[g];
        if (cudaStreamWaitEvent(gs, S->fork[par], 0) != cudaSuccess) { cudaGetLastError(); rc = SW_ECUDA; break; }
        DbBufs B{&S->grows[g], &S->gslots[g], static_cast<const DevScoring *>(S->dscore.p),
                 static_cast<int *>(S->derr.p)};
        c->stream = gs;
        rc = db_launch_shape(c, L.shape, djobs + L.job0, L.njobs, L.nblocks, v, S->ds.K, L.maxm, &B);
        c->stream = home;
        if (rc == SW_OK && cudaEventRecord(S->gdone[par][g], gs) != cudaSuccess) { cudaGetLastError(); rc = SW_ECUDA; }
        if (rc == SW_OK) ++launched;
    }
    c->stream = home;
    // (a partial step is still waited for: its groups that launched hold its requests' buffers)
    next->on = true;
    next->parity = par;
    next->ngroups = launched;
    next->slots = act;
    for (Slot *s : act) ++s->enq;
    S->cur_chunk = (S->cur_chunk + 1) % S->chunks;
    ++S->nstep;
    return rc;
}

}  // namespace

extern "C" int sw_server_create(sw_ctx *c, const sw_db *db, const sw_scoring *sc, size_t mem_budget, int32_t k,
                                int32_t max_slots, int32_t chunks, sw_server **out) {
    if (!c || !db || !out || k < 0 || k > 64 || max_slots < 1 || max_slots > 256 || chunks < 1) return SW_EINVAL;
    DevScoring ds;
    RC(check_scoring(sc, &ds));
    if (ds.alg != kAlgLocal) return SW_EINVAL;          // the server searches with the local algorithm
    if (!fold_open(ds) || ds.go > 16000 || ds.ge > 16000) return SW_ERANGE;   // needs the packed kernel
    sw_server *S = new (std::nothrow) sw_server();
    if (!S) return SW_ENOMEM;
    S->c = c;
    S->db = db;
    S->ds = ds;
    S->k = k;
    S->mem_budget = mem_budget;
    S->slots.resize((size_t)max_slots);
    int32_t max_code = 0;
    int dev = 0;
    db_view(db, &S->view, &S->nseq, &max_code, &dev);
    if (dev != c->device || max_code >= ds.K) { delete S; return SW_EINVAL; }
    S->chunks = std::max(1, std::min<int>(chunks, std::max(1, S->view.npairs)));
    S->total_res = db_total_residues(db);
    S->maxK = ds.K;
    DeviceGuard g(c->device);
    int rc = S->dscore.ensure(sizeof(DevScoring));
    if (!rc) rc = S->derr.ensure(256);
    if (!rc) rc = S->herr.ensure(std::max<size_t>(64, sizeof(DevScoring)));   // (staging of the scoring too)
    for (int p = 0; p < 2 && !rc; ++p)
        if (cudaEventCreateWithFlags(&S->fork[p], cudaEventDisableTiming) != cudaSuccess) rc = SW_ECUDA;
    if (!rc) {
        std::memcpy(S->herr.p, &ds, sizeof(DevScoring));
        if (cudaMemcpyAsync(S->dscore.p, S->herr.p, sizeof(DevScoring), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaMemsetAsync(S->derr.p, 0, 256, c->stream) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess)
            rc = SW_ECUDA;
    }
    if (rc) {
        cudaGetLastError();
        delete S;
        return rc;
    }
    *out = S;
    return SW_OK;
}

extern "C" int sw_server_submit(sw_server *S, const uint8_t *q, int64_t m, uint64_t *ticket) {
    if (!S || !ticket || m < 0 || (m > 0 && !q)) return SW_EINVAL;
    if (m > 8000) return SW_ERANGE;                  // the query profile must fit shared memory
    if (S->failed != SW_OK) return S->failed;
    Slot *free_slot = nullptr;
    for (Slot &s : S->slots) if (!s.active) { free_slot = &s; break; }
    const size_t need = slot_bytes(S, m);
    if (!free_slot || S->mem_used + need > S->mem_budget) return SW_EAGAIN;
    sw_ctx *c = S->c;
    DeviceGuard g(c->device);
    Slot &s = *free_slot;
    RC(s.q.ensure((size_t)m + 16));
    RC(s.scores.ensure((size_t)std::max<int64_t>(1, S->nseq) * sizeof(int32_t)));
    RC(s.ovf.ensure((size_t)std::max<int64_t>(1, S->nseq) * sizeof(int32_t)));
    RC(s.ctr.ensure(64));
    if (m > 0) CU(cudaMemcpyAsync(s.q.p, q, (size_t)m, is_device_ptr(q) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemsetAsync(s.scores.p, 0, (size_t)std::max<int64_t>(1, S->nseq) * sizeof(int32_t), c->stream));
    CU(cudaMemsetAsync(s.ctr.p, 0, 64, c->stream));
    RC(reset_err(c));
    if (m > 0) RC(validate_codes(c, static_cast<const uint8_t *>(s.q.p), m, S->ds.K));
    int e = 0;
    RC(read_err(c, &e));
    if (e) return map_kernel_error(e);
    s.active = true;
    s.ticket = S->next_ticket++;
    s.m = m;
    s.enq = 0;
    s.visited = (m == 0 || S->nseq == 0) ? S->chunks : 0;
    S->mem_used += need;
    *ticket = s.ticket;
    if (s.visited >= S->chunks) RC(retire(S, s, SW_OK));
    return SW_OK;
}

// One sweep step: every active request that has chunks left to visit takes
// the current chunk.  The step is enqueued before the previous one is waited
// for; requests whose last chunk that previous step was retire here.
extern "C" int sw_server_step(sw_server *S, int32_t *active) {
    if (!S) return SW_EINVAL;
    sw_ctx *c = S->c;
    DeviceGuard g(c->device);
    std::vector<Slot *> act;
    if (S->failed == SW_OK)
        for (Slot &s : S->slots) if (s.active && s.enq < S->chunks) act.push_back(&s);
    if (active) *active = (int32_t)act.size();
    InFlight next;
    int first = SW_OK;
    if (!act.empty()) {
        int early = SW_OK;
        const int rc = enqueue_step(S, act, &next, &early);
        first = early;
        if (rc != SW_OK) {
            // the step could not be enqueued whole: wait for everything, fail its requests
            for (cudaStream_t t : S->gstreams) cudaStreamSynchronize(t);
            cudaStreamSynchronize(c->stream);
            cudaGetLastError();
            if (S->failed == SW_OK) S->failed = rc;
            if (first == SW_OK) first = rc;
        }
    }
    const int rc = complete_inflight(S);    // the previous step (or, with nothing new, the last)
    if (first == SW_OK) first = rc;
    S->inflight = std::move(next);
    if (S->failed != SW_OK) {
        // a failed server keeps no step in flight, and every request it holds fails with it
        const int r = complete_inflight(S);
        if (first == SW_OK) first = r;
        for (Slot &s : S->slots) if (s.active) retire(S, s, S->failed);
    }
    return first;
}

extern "C" int sw_server_poll(sw_server *S, uint64_t ticket, sw_dbhit *hits, int32_t *nhits) {
    if (!S || !nhits) return SW_EINVAL;
    auto it = S->done.find(ticket);
    if (it == S->done.end()) {
        for (const Slot &s : S->slots) if (s.active && s.ticket == ticket) return SW_EAGAIN;
        return SW_EINVAL;                            // unknown or already collected
    }
    if (!it->second.hits.empty() && !hits) return SW_EINVAL;
    const int st = it->second.status;
    for (size_t i = 0; i < it->second.hits.size(); ++i) hits[i] = it->second.hits[i];
    *nhits = (int32_t)it->second.hits.size();
    S->done.erase(it);
    return st;
}

extern "C" int sw_server_stats(const sw_server *S, int32_t *active, size_t *mem_used, int64_t *cells_done) {
    if (!S) return SW_EINVAL;
    int a = 0;
    for (const Slot &s : S->slots) a += s.active ? 1 : 0;
    if (active) *active = a;
    if (mem_used) *mem_used = S->mem_used;
    if (cells_done) *cells_done = S->cells_done;
    return SW_OK;
}

extern "C" void sw_server_destroy(sw_server *S) {
    if (!S) return;
    DeviceGuard g(S->c->device);
    for (cudaStream_t t : S->gstreams) cudaStreamSynchronize(t);
    cudaStreamSynchronize(S->c->stream);
    delete S;
}
