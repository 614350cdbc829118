// sw_batch.cu -- many pairs of uneven lengths in one launch.
//
// Every pair is one task of the wavefront fill (its own scoring scheme:
// DNA and protein pairs mix freely).  Tasks are ordered by cell count,
// largest first, so the long pairs' strip pipelines start first and the
// short pairs fill the device at the end (longest-processing-time order);
// a strip only activates the warps that hold rows of its task.  A plan
// keeps its inputs and task table on the device; its run (counter resets,
// the fill, the per-task reduction and the scatter of results back to pair
// order, the copy to the host) can be captured once in a CUDA graph and
// replayed.  The tile shape is picked per plan from a small candidate set
// by timing the plan itself (autotuning), and the choice is cached in the
// context for plans of the same size class.
#include "sw.h"
#include "sw_ctx.h"
#include "wavefront.cuh"
#include "aux_kernels.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

using namespace swgb;

#define CU(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; } } while (0)
#define RC(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)

namespace {

// err = kErrBadCode if a residue of pair p is >= the alphabet of its scoring.
static __global__ void validate_pairs_kernel(const uint8_t *a, const int64_t *aoff, const uint8_t *b,
                                             const int64_t *boff, const int32_t *sidx, const int32_t *alph,
                                             int npairs, int *err) {
    for (int p = blockIdx.x; p < npairs; p += gridDim.x) {
        const int K = alph[sidx[p]];
        bool bad = false;
        for (long long k = aoff[p] + threadIdx.x; k < aoff[p + 1]; k += blockDim.x) bad |= a[k] >= K;
        for (long long k = boff[p] + threadIdx.x; k < boff[p + 1]; k += blockDim.x) bad |= b[k] >= K;
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(err, 0, kErrBadCode);
    }
}

// out[pair[k]] = res[k] for the tasks of the plan.
static __global__ void scatter_hits_kernel(const int4 *res, const int32_t *pair, int ntasks, int4 *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ntasks) out[pair[k]] = res[k];
}

const FillConfig kCandidates[] = {{8, 4}, {4, 4}, {16, 4}, {8, 8}};

}  // namespace

struct sw_batch {
    sw_ctx *c = nullptr;
    int64_t npairs = 0;
    std::vector<int64_t> m, n;
    std::vector<int32_t> sidx;
    std::vector<DevScoring> scorings;
    const uint8_t *da = nullptr, *db = nullptr;    // residues on the device
    std::vector<int64_t> aoff, boff;
    DevBuf a_own, b_own, tasks, prog, cand, res, hits, perm, bnd, ticket, meta;
    HostBuf host_hits;
    FillConfig cfg{8, 4};
    bool fold = true;
    int maxK = 1;
    int ntasks = 0;
    long long tickets = 0;
    int grid = 0;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = false;
    ~sw_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

// Tasks for tile shape cfg: pairs with cells, largest first.
int build_tasks(sw_batch *B, const FillConfig &cfg) {
    const int HC = fill_rows_per_strip(cfg);
    std::vector<int32_t> order;
    for (int64_t p = 0; p < B->npairs; ++p)
        if (B->m[(size_t)p] > 0 && B->n[(size_t)p] > 0) order.push_back((int32_t)p);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return (double)B->m[(size_t)x] * (double)B->n[(size_t)x] > (double)B->m[(size_t)y] * (double)B->n[(size_t)y];
    });
    std::vector<FillTask> tasks;
    tasks.reserve(order.size());
    long long tickets = 0;
    size_t bnd_need = 0;
    for (int32_t p : order) {
        const int ns = (int)((B->m[(size_t)p] + HC - 1) / HC);
        if (ns > 1) bnd_need += 2 * (size_t)B->n[(size_t)p] * sizeof(int2);
    }
    RC(B->bnd.ensure(std::max<size_t>(bnd_need, 16)));
    size_t boff = 0;
    for (int32_t p : order) {
        FillTask t{};
        t.a = B->da + B->aoff[(size_t)p];
        t.b = B->db + B->boff[(size_t)p];
        t.rows = (int32_t)B->m[(size_t)p];
        t.ncols = (int32_t)B->n[(size_t)p];
        t.nstrips = (t.rows + HC - 1) / HC;
        t.scoring = B->sidx[(size_t)p];
        t.ticket0 = tickets;
        t.nslot = 2;
        if (t.nstrips > 1) {
            t.bnd = reinterpret_cast<int2 *>(static_cast<char *>(B->bnd.p) + boff);
            boff += 2 * (size_t)t.ncols * sizeof(int2);
        }
        tickets += t.nstrips;
        tasks.push_back(t);
    }
    B->ntasks = (int)tasks.size();
    B->tickets = tickets;
    B->cfg = cfg;
    const size_t tb = std::max<size_t>(1, tasks.size()) * sizeof(FillTask);
    RC(B->tasks.ensure(tb));
    RC(B->prog.ensure(std::max<long long>(1, tickets) * sizeof(int)));
    RC(B->cand.ensure(std::max<long long>(1, tickets) * sizeof(int4)));
    RC(B->res.ensure(std::max<size_t>(1, tasks.size()) * sizeof(int4)));
    RC(B->perm.ensure(std::max<size_t>(1, order.size()) * sizeof(int32_t)));
    if (!tasks.empty()) {
        CU(cudaMemcpy(B->tasks.p, tasks.data(), tb, cudaMemcpyHostToDevice));
        CU(cudaMemcpy(B->perm.p, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    return SW_OK;
}

// Enqueue one run of the plan on B->stream (graph-capturable: no host sync,
// no allocation).
int enqueue_run(sw_batch *B) {
    sw_ctx *c = B->c;
    cudaStream_t st = B->stream;
    const size_t out_bytes = (size_t)std::max<int64_t>(1, B->npairs) * sizeof(int4);
    CU(cudaMemsetAsync(B->hits.p, 0, out_bytes, st));
    if (B->ntasks > 0) {
        CU(cudaMemsetAsync(B->prog.p, 0, (size_t)B->tickets * sizeof(int), st));
        CU(cudaMemsetAsync(B->ticket.p, 0, 256, st));            // ticket counter and error word
        FillLaunch L;
        L.tasks = static_cast<const FillTask *>(B->tasks.p);
        L.scorings = static_cast<const DevScoring *>(B->meta.p);
        L.ticket = static_cast<unsigned long long *>(B->ticket.p);
        L.prog = static_cast<int *>(B->prog.p);
        L.cand = static_cast<int4 *>(B->cand.p);
        L.err = reinterpret_cast<int *>(static_cast<char *>(B->ticket.p) + 64);
        L.total = B->tickets;
        L.spin_limit = c->spin_limit;
        L.ntasks = B->ntasks;
        cudaStream_t saved = c->stream;
        c->stream = st;
        const int rc = launch_fill(c, B->cfg, kModeScore, B->fold, L, B->maxK, B->tickets);
        c->stream = saved;
        RC(rc);
        reduce_candidates_kernel<<<(B->ntasks + 7) / 8, 256, 0, st>>>(L.tasks, B->ntasks, L.cand,
                                                                      static_cast<int4 *>(B->res.p));
        CU(cudaGetLastError());
        ++c->launches;
        scatter_hits_kernel<<<(B->ntasks + 255) / 256, 256, 0, st>>>(static_cast<const int4 *>(B->res.p),
                                                                      static_cast<const int32_t *>(B->perm.p),
                                                                      B->ntasks, static_cast<int4 *>(B->hits.p));
        CU(cudaGetLastError());
        ++c->launches;
    }
    CU(cudaMemcpyAsync(B->host_hits.p, B->hits.p, out_bytes, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(static_cast<char *>(B->host_hits.p) + out_bytes,
                       static_cast<char *>(B->ticket.p) + 64, sizeof(int), cudaMemcpyDeviceToHost, st));
    return SW_OK;
}

int finish_run(sw_batch *B, sw_hit *out) {
    CU(cudaStreamSynchronize(B->stream));
    const size_t out_bytes = (size_t)std::max<int64_t>(1, B->npairs) * sizeof(int4);
    int e;
    std::memcpy(&e, static_cast<char *>(B->host_hits.p) + out_bytes, sizeof(int));
    RC(map_kernel_error(e));
    const int4 *h = static_cast<const int4 *>(B->host_hits.p);
    for (int64_t p = 0; p < B->npairs; ++p) out[p] = sw_hit{h[p].x, 0, (int64_t)h[p].y, (int64_t)h[p].z};
    return SW_OK;
}

// Size class of a plan for the autotune cache: log2 of its cells and of its pair count.
long long size_class(const sw_batch *B) {
    double cells = 0;
    for (int64_t p = 0; p < B->npairs; ++p) cells += (double)B->m[(size_t)p] * (double)B->n[(size_t)p];
    const int lc = cells > 1 ? (int)std::log2(cells) : 0;
    const int lp = B->npairs > 1 ? (int)std::log2((double)B->npairs) : 0;
    return (long long)lc * 64 + lp + 4096LL * B->maxK;
}

}  // namespace

extern "C" int sw_batch_create(sw_ctx *c, int64_t npairs, const uint8_t *a_res, const int64_t *a_off,
                               const uint8_t *b_res, const int64_t *b_off, const int32_t *scoring_of_pair,
                               int32_t nscorings, const sw_scoring *scorings, int32_t flags, sw_batch **out) {
    if (!c || !out || npairs < 0 || npairs > (1 << 28) || nscorings < 1 || !scorings) return SW_EINVAL;
    if (npairs > 0 && (!a_off || !b_off || !scoring_of_pair)) return SW_EINVAL;
    sw_batch *B = new (std::nothrow) sw_batch();
    if (!B) return SW_ENOMEM;
    struct Guard { sw_batch *&b; bool keep = false; ~Guard() { if (!keep) delete b; } } guard{B};
    B->c = c;
    B->npairs = npairs;
    for (int k = 0; k < nscorings; ++k) {
        DevScoring d;
        RC(check_scoring(&scorings[k], &d));
        B->scorings.push_back(d);
        B->maxK = std::max(B->maxK, d.K);
    }
    B->fold = true;
    for (const DevScoring &d : B->scorings) B->fold &= fold_open(d);
    B->m.resize((size_t)npairs);
    B->n.resize((size_t)npairs);
    B->sidx.assign(scoring_of_pair, scoring_of_pair + npairs);
    B->aoff.assign(a_off, a_off + (npairs > 0 ? npairs + 1 : 0));
    B->boff.assign(b_off, b_off + (npairs > 0 ? npairs + 1 : 0));
    if (npairs > 0 && (a_off[0] != 0 || b_off[0] != 0)) return SW_EINVAL;
    for (int64_t p = 0; p < npairs; ++p) {
        const int64_t m = a_off[p + 1] - a_off[p], n = b_off[p + 1] - b_off[p];
        if (m < 0 || n < 0 || scoring_of_pair[p] < 0 || scoring_of_pair[p] >= nscorings) return SW_EINVAL;
        if (m > SW_MAX_LEN || n > SW_MAX_LEN) return SW_ERANGE;
        int mx = 0;
        const DevScoring &d = B->scorings[(size_t)scoring_of_pair[p]];
        for (int k = 0; k < d.K * d.K; ++k) mx = std::max(mx, (int)d.mat[k]);
        if ((double)std::min(m, n) * (double)mx >= (double)kMaxScoreBound) return SW_ERANGE;
        B->m[(size_t)p] = m;
        B->n[(size_t)p] = n;
    }
    DeviceGuard g(c->device);
    CU(cudaStreamSynchronize(c->stream));
    CU(cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking));
    const int64_t ta = npairs > 0 ? a_off[npairs] : 0, tbn = npairs > 0 ? b_off[npairs] : 0;
    if (ta > 0 && !a_res) return SW_EINVAL;
    if (tbn > 0 && !b_res) return SW_EINVAL;
    // inputs on the device (device inputs are used in place and must outlive the plan)
    if (ta > 0 && is_device_ptr(a_res)) B->da = a_res;
    else if (ta > 0) {
        RC(B->a_own.ensure((size_t)ta + 16));
        CU(cudaMemcpy(B->a_own.p, a_res, (size_t)ta, cudaMemcpyHostToDevice));
        B->da = static_cast<const uint8_t *>(B->a_own.p);
    }
    if (tbn > 0 && is_device_ptr(b_res)) B->db = b_res;
    else if (tbn > 0) {
        RC(B->b_own.ensure((size_t)tbn + 16));
        CU(cudaMemcpy(B->b_own.p, b_res, (size_t)tbn, cudaMemcpyHostToDevice));
        B->db = static_cast<const uint8_t *>(B->b_own.p);
    }
    RC(B->meta.ensure(B->scorings.size() * sizeof(DevScoring) + 4096));
    CU(cudaMemcpy(B->meta.p, B->scorings.data(), B->scorings.size() * sizeof(DevScoring), cudaMemcpyHostToDevice));
    RC(B->ticket.ensure(256));
    CU(cudaMemset(B->ticket.p, 0, 256));
    RC(B->hits.ensure((size_t)std::max<int64_t>(1, npairs) * sizeof(int4)));
    RC(B->host_hits.ensure((size_t)std::max<int64_t>(1, npairs) * sizeof(int4) + 64));
    // residue codes against each pair's alphabet
    if (npairs > 0 && ta + tbn > 0) {
        DevBuf offs;
        RC(offs.ensure((size_t)(2 * (npairs + 1) + npairs) * 8 + 256));
        int64_t *doa = static_cast<int64_t *>(offs.p);
        int64_t *dob = doa + (npairs + 1);
        int32_t *dsi = reinterpret_cast<int32_t *>(dob + (npairs + 1));
        std::vector<int32_t> alph;
        for (const DevScoring &d : B->scorings) alph.push_back(d.K);
        CU(cudaMemcpy(doa, a_off, (size_t)(npairs + 1) * 8, cudaMemcpyHostToDevice));
        CU(cudaMemcpy(dob, b_off, (size_t)(npairs + 1) * 8, cudaMemcpyHostToDevice));
        CU(cudaMemcpy(dsi, scoring_of_pair, (size_t)npairs * 4, cudaMemcpyHostToDevice));
        DevBuf al;
        RC(al.ensure(alph.size() * 4));
        CU(cudaMemcpy(al.p, alph.data(), alph.size() * 4, cudaMemcpyHostToDevice));
        int *err = reinterpret_cast<int *>(static_cast<char *>(B->ticket.p) + 64);
        validate_pairs_kernel<<<(unsigned)std::min<int64_t>(npairs, 4LL * c->nsm), 256, 0, B->stream>>>(
            B->da, doa, B->db, dob, dsi, static_cast<const int32_t *>(al.p), (int)npairs, err);
        CU(cudaGetLastError());
        ++c->launches;
        int e = 0;
        CU(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
        CU(cudaStreamSynchronize(B->stream));
        if (e) return map_kernel_error(e);
    }
    // tile shape: cached for the size class, else autotuned (or the context default)
    const long long cls = size_class(B);
    FillConfig cfg = c->bat;
    bool tuned = false;
    for (const auto &kv : c->batch_tune)
        if (kv.first == cls) { cfg = kv.second; tuned = true; }
    if (!tuned && (flags & SW_BATCH_AUTOTUNE)) {
        float best = 1e30f;
        cudaEvent_t e0, e1;
        CU(cudaEventCreate(&e0));
        CU(cudaEventCreate(&e1));
        for (const FillConfig &cand : kCandidates) {
            RC(build_tasks(B, cand));
            CU(cudaEventRecord(e0, B->stream));
            RC(enqueue_run(B));
            CU(cudaEventRecord(e1, B->stream));
            CU(cudaStreamSynchronize(B->stream));
            float ms = 0;
            CU(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; cfg = cand; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->batch_tune.push_back({cls, cfg});
    }
    RC(build_tasks(B, cfg));
    if (flags & SW_BATCH_GRAPH) {
        // one plain run first: kernel attributes are set outside the capture
        RC(enqueue_run(B));
        CU(cudaStreamSynchronize(B->stream));
        CU(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue_run(B);
        cudaGraph_t gph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(B->stream, &gph);
        if (rc) { if (gph) cudaGraphDestroy(gph); return rc; }
        if (ce != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; }
        B->graph = gph;
        CU(cudaGraphInstantiate(&B->exec, B->graph, 0));
        B->use_graph = true;
    }
    guard.keep = true;
    *out = B;
    return SW_OK;
}

extern "C" int sw_batch_run(sw_batch *B, sw_hit *out) {
    if (!B || (B->npairs > 0 && !out)) return SW_EINVAL;
    DeviceGuard g(B->c->device);
    if (B->use_graph) {
        CU(cudaGraphLaunch(B->exec, B->stream));
        B->c->launches += B->ntasks > 0 ? 3 : 0;
    } else {
        RC(enqueue_run(B));
    }
    return finish_run(B, out);
}

extern "C" void sw_batch_destroy(sw_batch *B) {
    if (!B) return;
    DeviceGuard g(B->c->device);
    if (B->stream) cudaStreamSynchronize(B->stream);
    delete B;
}

extern "C" int sw_batch_config(const sw_batch *B, int32_t *rows_per_lane, int32_t *warps) {
    if (!B || !rows_per_lane || !warps) return SW_EINVAL;
    *rows_per_lane = B->cfg.R;
    *warps = B->cfg.W;
    return SW_OK;
}

extern "C" int sw_score_batch(sw_ctx *c, int64_t npairs, const uint8_t *a_res, const int64_t *a_off,
                              const uint8_t *b_res, const int64_t *b_off, const int32_t *scoring_of_pair,
                              int32_t nscorings, const sw_scoring *scorings, sw_hit *out) {
    sw_batch *B = nullptr;
    RC(sw_batch_create(c, npairs, a_res, a_off, b_res, b_off, scoring_of_pair, nscorings, scorings, 0, &B));
    const int rc = sw_batch_run(B, out);
    sw_batch_destroy(B);
    return rc;
}
