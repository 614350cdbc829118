// sw_batch.cu -- many pairs of uneven lengths, binned by length and scoring.
//
// Every pair is one task of the wavefront fill.  Pairs are binned by their
// scoring scheme (so each launch knows its alphabet: small alphabets get the
// int32 query profile) and by their length in rows (short queries and long
// ones want different strip heights); each bin is one launch of all its
// tasks, ordered by cell count, largest first, so the long pairs' strip
// pipelines start first and the short pairs fill the device at the end
// (longest-processing-time order); a strip only activates the warps that
// hold rows of its task.  A plan keeps its inputs and task table on the
// device; its run (counter resets, the bins' fills, the per-task reduction,
// the scatter of results back to pair order, the copy to the host) can be
// captured once in a CUDA graph and replayed.  Each bin's tile shape is
// picked from a candidate set by timing the plan itself (autotuning), and
// the choice is cached in the context for bins of the same size class.  The
// candidates include the packed 16-bit fill (wavefront16.cuh) wherever its
// exactness test passes for the bin's scoring scheme, so the autotuner
// chooses the lane width as well as the tile shape.
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

const FillConfig kCandidates[] = {{8, 4}, {4, 4}, {12, 4}, {16, 4}, {8, 8},
                                  {8, 4, 0, 0, 1}, {12, 4, 0, 0, 1}, {16, 4, 0, 0, 1},
                                  {8, 2, 0, 0, 1}, {12, 2, 0, 0, 1}, {16, 2, 0, 0, 1}};

constexpr int64_t kShortRows = 1024;      // row classes: queries up to this many rows, and longer

// ticket counter of bin b starts at the bin's first ticket
static __global__ void set_counters_kernel(unsigned long long *ctr, const long long *base, int nbins) {
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) ctr[b] = (unsigned long long)base[b];
}

struct Bin {
    int32_t sidx = 0;              // scoring scheme of its pairs
    int rclass = 0;                // 0: up to kShortRows rows, 1: longer
    std::vector<int32_t> pairs;    // its pairs, largest first
    FillConfig cfg{8, 4};
    int t0 = 0, nt = 0;            // its tasks
    long long tbase = 0, tcount = 0;
};

}  // namespace

struct sw_batch {
    sw_ctx *c = nullptr;
    int64_t npairs = 0;
    std::vector<int64_t> m, n;
    std::vector<int32_t> sidx;
    std::vector<DevScoring> scorings;
    const uint8_t *da = nullptr, *db = nullptr;    // residues on the device
    std::vector<int64_t> aoff, boff;
    DevBuf a_own, b_own, tasks, prog, cand, res, hits, perm, bnd, ticket, meta, order;
    HostBuf host_hits;
    std::vector<Bin> bins;
    FillConfig cfg{8, 4};          // the tile shape of the bin with the most cells
    bool fold = true;
    int maxK = 1;
    int ntasks = 0;
    long long tickets = 0;
    int grid = 0;
    cudaStream_t stream = nullptr;
    std::vector<cudaStream_t> bstreams;   // one per bin: the bins' fills run concurrently
    std::vector<cudaEvent_t> bevents;     // [0]: fork, [1 + k]: bin k done
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = false;
    ~sw_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaEvent_t e : bevents) if (e) cudaEventDestroy(e);
        for (cudaStream_t t : bstreams) if (t) cudaStreamDestroy(t);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

// Task table of the plan: the bins in order, each bin's pairs largest first
// with the bin's tile shape; tickets numbered across the whole plan.
int build_plan(sw_batch *B) {
    std::vector<FillTask> tasks;
    std::vector<int32_t> order;
    std::vector<long long> bases;
    size_t bnd_need = 0;
    for (const Bin &bin : B->bins) {
        const int HC = fill_rows_per_strip(bin.cfg);
        for (int32_t p : bin.pairs)
            if ((B->m[(size_t)p] + HC - 1) / HC > 1) bnd_need += 2 * (size_t)B->n[(size_t)p] * sizeof(int2);
    }
    RC(B->bnd.ensure(std::max<size_t>(bnd_need, 16)));
    size_t boff = 0;
    long long tickets = 0;
    B->cfg = B->bins.empty() ? FillConfig{8, 4} : B->bins[0].cfg;
    double best_cells = -1;
    for (Bin &bin : B->bins) {
        const int HC = fill_rows_per_strip(bin.cfg);
        bin.t0 = (int)tasks.size();
        bin.tbase = tickets;
        double cells = 0;
        for (int32_t p : bin.pairs) {
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
            cells += (double)t.rows * (double)t.ncols;
            tasks.push_back(t);
            order.push_back(p);
        }
        bin.nt = (int)tasks.size() - bin.t0;
        bin.tcount = tickets - bin.tbase;
        bases.push_back(bin.tbase);
        if (cells > best_cells) { best_cells = cells; B->cfg = bin.cfg; }
    }
    // claim order, level by level: in task order a block that takes a task's strip k waits until
    // strip k - 1 has produced rows, holding its SM slot idle; level by level, strip k - 1 has run
    // ahead.  Levels are counted from each task's last strip (the last level holds every task's
    // last strip, the first only the tallest tasks' first strips), and within a level the widest
    // strips come first: a strip takes about as many steps as its task has columns, so the run
    // ends on narrow strips rather than on the tallest tasks' last strips, which may be wide
    // (10,000 uneven pairs: 56.5 -> 55.9 ms).
    std::vector<int2> claims((size_t)std::max<long long>(1, tickets));
    for (const Bin &bin : B->bins) {
        int levels = 0;
        for (int k = 0; k < bin.nt; ++k) levels = std::max(levels, tasks[(size_t)(bin.t0 + k)].nstrips);
        struct Claim { int level, ncols, k, strip; };
        std::vector<Claim> cl;
        cl.reserve((size_t)bin.tcount);
        for (int k = 0; k < bin.nt; ++k) {
            const FillTask &t = tasks[(size_t)(bin.t0 + k)];
            for (int s = 0; s < t.nstrips; ++s) cl.push_back({levels - t.nstrips + s, t.ncols, k, s});
        }
        std::sort(cl.begin(), cl.end(), [](const Claim &x, const Claim &y) {
            if (x.level != y.level) return x.level < y.level;
            if (x.ncols != y.ncols) return x.ncols > y.ncols;
            return x.k < y.k;
        });
        long long pos = bin.tbase;
        for (const Claim &q : cl) claims[(size_t)pos++] = make_int2(q.k, q.strip);
    }
    B->ntasks = (int)tasks.size();
    B->tickets = tickets;
    const size_t tb = std::max<size_t>(1, tasks.size()) * sizeof(FillTask);
    RC(B->tasks.ensure(tb));
    RC(B->prog.ensure(std::max<long long>(1, tickets) * sizeof(int)));
    RC(B->cand.ensure(std::max<long long>(1, tickets) * sizeof(int4)));
    RC(B->res.ensure(std::max<size_t>(1, tasks.size()) * sizeof(int4)));
    RC(B->perm.ensure(std::max<size_t>(1, order.size()) * sizeof(int32_t)));
    RC(B->order.ensure(claims.size() * sizeof(int2)));
    // counters and error word: [bins x u64 counters][bins x i64 bases][err]
    const size_t nb = std::max<size_t>(1, B->bins.size());
    RC(B->ticket.ensure(16 * nb + 256));
    if (!tasks.empty()) {
        CU(cudaMemcpy(B->tasks.p, tasks.data(), tb, cudaMemcpyHostToDevice));
        CU(cudaMemcpy(B->perm.p, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(B->order.p, claims.data(), claims.size() * sizeof(int2), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(static_cast<char *>(B->ticket.p) + 8 * nb, bases.data(), bases.size() * sizeof(long long),
                      cudaMemcpyHostToDevice));
    }
    return SW_OK;
}

int *batch_err(sw_batch *B) {
    return reinterpret_cast<int *>(static_cast<char *>(B->ticket.p) + 16 * std::max<size_t>(1, B->bins.size()) + 64);
}

// Enqueue one run of the plan on B->stream (graph-capturable: no host sync,
// no allocation).
int enqueue_run(sw_batch *B) {
    sw_ctx *c = B->c;
    cudaStream_t st = B->stream;
    const size_t out_bytes = (size_t)std::max<int64_t>(1, B->npairs) * sizeof(int4);
    CU(cudaMemsetAsync(B->hits.p, 0, out_bytes, st));
    const size_t nb = std::max<size_t>(1, B->bins.size());
    CU(cudaMemsetAsync(batch_err(B), 0, sizeof(int), st));
    if (B->ntasks > 0) {
        CU(cudaMemsetAsync(B->prog.p, 0, (size_t)B->tickets * sizeof(int), st));
        unsigned long long *ctr = static_cast<unsigned long long *>(B->ticket.p);
        set_counters_kernel<<<1, 32, 0, st>>>(ctr, reinterpret_cast<const long long *>(ctr + nb), (int)B->bins.size());
        CU(cudaGetLastError());
        ++c->launches;
        // fork: every bin's fill on its own stream, so the bins' tails overlap.  The short-query
        // bins are launched first: the long-query bins (claimed level by level, narrow strips
        // last) end the run, rather than a short-query bin's widest pair (55.9 -> 55.7 ms)
        CU(cudaEventRecord(B->bevents[0], st));
        cudaStream_t saved = c->stream;
        int rc = SW_OK;
        std::vector<size_t> launch_order(B->bins.size());
        std::iota(launch_order.begin(), launch_order.end(), size_t(0));
        std::stable_sort(launch_order.begin(), launch_order.end(),
                         [&](size_t x, size_t y) { return B->bins[x].rclass < B->bins[y].rclass; });
        for (size_t kk = 0; kk < launch_order.size() && rc == SW_OK; ++kk) {
            const size_t k = launch_order[kk];
            const Bin &bin = B->bins[k];
            cudaStream_t bs = B->bstreams[k];
            if (cudaStreamWaitEvent(bs, B->bevents[0], 0) != cudaSuccess) { cudaGetLastError(); rc = SW_ECUDA; break; }
            if (bin.nt > 0) {
                const DevScoring &sc = B->scorings[(size_t)bin.sidx];
                FillLaunch L{};
                L.tasks = static_cast<const FillTask *>(B->tasks.p) + bin.t0;
                L.scorings = static_cast<const DevScoring *>(B->meta.p);
                L.ticket = ctr + k;
                L.prog = static_cast<int *>(B->prog.p);
                L.cand = static_cast<int4 *>(B->cand.p);
                L.err = batch_err(B);
                L.total = bin.tbase + bin.tcount;
                L.spin_limit = c->spin_limit;
                L.ntasks = bin.nt;
                L.order = static_cast<const int2 *>(B->order.p);
                c->stream = bs;
                rc = launch_fill(c, bin.cfg, kModeScore, fold_open(sc), L, sc.K, bin.tcount);
                c->stream = saved;
            }
            if (rc == SW_OK && cudaEventRecord(B->bevents[1 + k], bs) != cudaSuccess) { cudaGetLastError(); rc = SW_ECUDA; }
            if (rc == SW_OK && cudaStreamWaitEvent(st, B->bevents[1 + k], 0) != cudaSuccess) { cudaGetLastError(); rc = SW_ECUDA; }
        }
        c->stream = saved;
        RC(rc);
        FillLaunch L{};
        L.tasks = static_cast<const FillTask *>(B->tasks.p);
        L.cand = static_cast<int4 *>(B->cand.p);
        reduce_candidates_kernel<<<(B->ntasks + 7) / 8, 256, 0, st>>>(L.tasks, B->ntasks, L.cand,
                                                                      static_cast<const DevScoring *>(B->meta.p),
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
    CU(cudaMemcpyAsync(static_cast<char *>(B->host_hits.p) + out_bytes, batch_err(B), sizeof(int),
                       cudaMemcpyDeviceToHost, st));
    return SW_OK;
}

int finish_run(sw_batch *B, sw_hit *out) {
    CU(cudaStreamSynchronize(B->stream));
    const size_t out_bytes = (size_t)std::max<int64_t>(1, B->npairs) * sizeof(int4);
    int e;
    std::memcpy(&e, static_cast<char *>(B->host_hits.p) + out_bytes, sizeof(int));
    RC(map_kernel_error(e));
    const int4 *h = static_cast<const int4 *>(B->host_hits.p);
    for (int64_t p = 0; p < B->npairs; ++p) {
        out[p] = sw_hit{h[p].x, 0, (int64_t)h[p].y, (int64_t)h[p].z};
        const DevScoring &d = B->scorings[(size_t)B->sidx[(size_t)p]];
        if ((B->m[(size_t)p] == 0 || B->n[(size_t)p] == 0) && d.alg != kAlgLocal) {
            // pairs with an empty side have no task: their end cell lies on the border
            int cs = kNoScore, ci = 0x7fffffff, cj = 0x7fffffff;
            border_end_candidates(d.alg, B->m[(size_t)p], B->n[(size_t)p], d.go, d.ge, &cs, &ci, &cj);
            out[p] = sw_hit{cs, 0, (int64_t)ci, (int64_t)cj};
        }
    }
    return SW_OK;
}

// Size class of a bin for the autotune cache: its alphabet, row class, and
// log2 of its cells and of its pair count.
long long bin_class(const sw_batch *B, const Bin &bin) {
    double cells = 0;
    for (int32_t p : bin.pairs) cells += (double)B->m[(size_t)p] * (double)B->n[(size_t)p];
    const int lc = cells > 1 ? (int)std::log2(cells) : 0;
    const int lp = bin.pairs.size() > 1 ? (int)std::log2((double)bin.pairs.size()) : 0;
    return (((long long)B->scorings[(size_t)bin.sidx].K * 2 + bin.rclass) * 64 + lc) * 64 + lp;
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
        if (!score_range_ok(&scorings[scoring_of_pair[p]], m, n)) return SW_ERANGE;
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
    // bins: scoring scheme x row class, the bin with the most cells first
    {
        std::vector<Bin> bins;
        for (int64_t p = 0; p < npairs; ++p) {
            if (B->m[(size_t)p] == 0 || B->n[(size_t)p] == 0) continue;
            const int rcl = B->m[(size_t)p] > kShortRows ? 1 : 0;
            Bin *bin = nullptr;
            for (Bin &x : bins) if (x.sidx == B->sidx[(size_t)p] && x.rclass == rcl) bin = &x;
            if (!bin) { bins.push_back(Bin{}); bin = &bins.back(); bin->sidx = B->sidx[(size_t)p]; bin->rclass = rcl; }
            bin->pairs.push_back((int32_t)p);
        }
        auto cells = [&](int32_t p) { return (double)B->m[(size_t)p] * (double)B->n[(size_t)p]; };
        for (Bin &bin : bins)
            std::stable_sort(bin.pairs.begin(), bin.pairs.end(), [&](int32_t x, int32_t y) { return cells(x) > cells(y); });
        auto bin_cells = [&](const Bin &bin) { double t = 0; for (int32_t p : bin.pairs) t += cells(p); return t; };
        std::stable_sort(bins.begin(), bins.end(), [&](const Bin &x, const Bin &y) { return bin_cells(x) > bin_cells(y); });
        for (Bin &bin : bins) {
            bin.cfg = c->bat;
            if (bin.cfg.P16 && ((bin.cfg.W != 4 && bin.cfg.W != 2) || !p16_fits(B->scorings[(size_t)bin.sidx], bin.cfg.R)))
                bin.cfg.P16 = 0;
            if (B->scorings[(size_t)bin.sidx].alg != kAlgLocal) {   // global, semi-global, overlap
                bin.cfg = FillConfig{bin.rclass ? 16 : 8, 4};
                bin.cfg.alg = 1;
            }
        }
        B->bins = std::move(bins);
        for (size_t k = 0; k < B->bins.size(); ++k) {
            cudaStream_t bs = nullptr;
            CU(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
            B->bstreams.push_back(bs);
        }
        for (size_t k = 0; k < B->bins.size() + 1; ++k) {
            cudaEvent_t e = nullptr;
            CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            B->bevents.push_back(e);
        }
    }
    // each bin's tile shape: cached for its size class, else autotuned one bin at a time
    // (the others keep their current shapes), else the context default
    std::vector<long long> cls(B->bins.size());
    std::vector<bool> tuned(B->bins.size(), false);
    for (size_t k = 0; k < B->bins.size(); ++k) {
        cls[k] = bin_class(B, B->bins[k]);
        if (B->bins[k].cfg.alg != kAlgLocal) { tuned[k] = true; continue; }   // fixed shapes
        for (const auto &kv : c->batch_tune)
            if (kv.first == cls[k]) { B->bins[k].cfg = kv.second; tuned[k] = true; }
    }
    if (flags & SW_BATCH_AUTOTUNE) {
        cudaEvent_t e0, e1;
        CU(cudaEventCreate(&e0));
        CU(cudaEventCreate(&e1));
        int rc = SW_OK;
        for (size_t k = 0; k < B->bins.size() && rc == SW_OK; ++k) {
            if (tuned[k]) continue;
            float best = 1e30f;
            FillConfig pick = B->bins[k].cfg;
            for (const FillConfig &cand : kCandidates) {
                if (cand.P16 && !p16_fits(B->scorings[(size_t)B->bins[k].sidx], cand.R)) continue;
                B->bins[k].cfg = cand;
                rc = build_plan(B);
                if (!rc) rc = cudaEventRecord(e0, B->stream) == cudaSuccess ? SW_OK : SW_ECUDA;
                if (!rc) rc = enqueue_run(B);
                if (!rc) rc = cudaEventRecord(e1, B->stream) == cudaSuccess ? SW_OK : SW_ECUDA;
                if (!rc) rc = cudaStreamSynchronize(B->stream) == cudaSuccess ? SW_OK : SW_ECUDA;
                float ms = 0;
                if (!rc) rc = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess ? SW_OK : SW_ECUDA;
                if (rc) break;
                if (ms < best) { best = ms; pick = cand; }
            }
            B->bins[k].cfg = pick;
            if (!rc) c->batch_tune.push_back({cls[k], pick});
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) { cudaGetLastError(); return rc; }
    }
    RC(build_plan(B));
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
        B->c->launches += B->ntasks > 0 ? 3 + (int64_t)B->bins.size() : 0;
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

extern "C" int sw_batch_bin_config(const sw_batch *B, int32_t bin, int32_t *rows_per_lane, int32_t *warps,
                                   int32_t *lane_bits, int64_t *npairs) {
    if (!B || !rows_per_lane || !warps || !lane_bits || !npairs || bin < 0) return SW_EINVAL;
    if ((size_t)bin >= B->bins.size()) return SW_ERANGE;
    const Bin &b = B->bins[(size_t)bin];
    *rows_per_lane = b.cfg.R;
    *warps = b.cfg.W;
    *lane_bits = b.cfg.P16 ? 16 : 32;
    *npairs = (int64_t)b.pairs.size();
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
