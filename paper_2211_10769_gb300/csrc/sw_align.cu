// sw_align.cu -- reconstruction phase (paper Section 2.2: resolution finds
// the best score, reconstruction recovers the path with space-efficient
// methods).
//
// 1. Forward fill over the whole matrix (score mode), keeping the bottom
//    row (H, F per column) of strips as checkpoint rows: every strip while
//    that fits the checkpoint budget, else every k-th strip.
// 2. The end cell (ie, je) comes from the per-strip candidates.
// 3. Blocks are the row ranges between consecutive checkpoint rows, cut at
//    row ie and column je.  Going upwards from the block holding ie, groups
//    of blocks whose decision bits fit the traceback budget are recomputed
//    from their checkpoint rows (traceback mode; the blocks of a group are
//    independent tasks of one launch) and the walk kernel follows the bits
//    through the group, carrying its cell and state to the next group.
// Memory is (rows / checkpoint spacing) x n checkpoint entries plus one
// group of bits, instead of the m x n matrix; the recomputation touches at
// most ie x je cells.
#include "sw.h"
#include "sw_ctx.h"
#include "wavefront.cuh"
#include "aux_kernels.cuh"

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace swgb;

#define CU(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; } } while (0)
#define RC(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)

namespace {

int launch_walk(sw_ctx *c, int R, const void *tb, long long ld, int G0) {
    WalkState *st = static_cast<WalkState *>(c->walk.p);
    int2 *runs = static_cast<int2 *>(c->runs.p);
    switch (R) {
        case 4: walk_kernel<uint16_t, 4><<<1, 32, 0, c->stream>>>(static_cast<const uint16_t *>(tb), ld, G0, st, runs); break;
        case 8: walk_kernel<uint32_t, 8><<<1, 32, 0, c->stream>>>(static_cast<const uint32_t *>(tb), ld, G0, st, runs); break;
        case 16: walk_kernel<unsigned long long, 16><<<1, 32, 0, c->stream>>>(static_cast<const unsigned long long *>(tb), ld, G0, st, runs); break;
        default: return SW_EINVAL;
    }
    CU(cudaGetLastError());
    ++c->launches;
    return SW_OK;
}

int tb_word_bytes(int R) { return R / 2; }

int empty_alignment(sw_alignment *out) {
    char *s = static_cast<char *>(std::malloc(1));
    if (!s) return SW_ENOMEM;
    s[0] = 0;
    *out = sw_alignment{0, 0, 0, 0, 0, 0, s, 0};
    return SW_OK;
}

}  // namespace

extern "C" int sw_align(sw_ctx *c, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                        const sw_scoring *sc, sw_alignment *out) {
    if (!c || !out) return SW_EINVAL;
    DevScoring ds;
    RC(check_scoring(sc, &ds));
    if (m < 0 || n < 0 || (m > 0 && !a) || (n > 0 && !b)) return SW_EINVAL;
    if (m > SW_MAX_LEN || n > SW_MAX_LEN) return SW_ERANGE;
    if ((double)std::min(m, n) * (double)max_pos_score(sc) >= (double)(1 << 30)) return SW_ERANGE;
    if (m == 0 || n == 0) return empty_alignment(out);
    DeviceGuard g(c->device);
    const uint8_t *da, *db;
    RC(stage_seq(c, a, m, c->seq_a, &da));
    RC(stage_seq(c, b, n, c->seq_b, &db));
    RC(reset_err(c));
    RC(validate_codes(c, da, m, ds.K));
    RC(validate_codes(c, db, n, ds.K));
    RC(upload_scorings(c, {ds}));

    // ---- 1. forward fill with checkpoint rows
    const int HC = fill_rows_per_strip(c->fwd);
    const int HT = fill_rows_per_strip(c->tbc);
    if (HC % HT != 0) return SW_EINVAL;
    FillTask t{};
    t.a = da; t.b = db;
    t.rows = (int32_t)m; t.ncols = (int32_t)n;
    t.nstrips = (int32_t)((m + HC - 1) / HC);
    t.scoring = 0; t.ticket0 = 0; t.top = nullptr; t.row0 = 0;
    const size_t row_bytes = (size_t)n * sizeof(int2);
    int every = 1;                                    // strips per checkpoint
    while ((size_t)(t.nstrips / every) * row_bytes > c->ckpt_budget && every < t.nstrips) every *= 2;
    if (every == 1) {
        t.nslot = t.nstrips;                          // every strip's bottom row stays
        RC(c->bnd.ensure((size_t)t.nslot * row_bytes));
        t.bnd = static_cast<int2 *>(c->bnd.p);
        t.ckpt_every = 0; t.ckpt = nullptr;
    } else {
        t.nslot = std::min(t.nstrips, 4);
        RC(c->bnd.ensure((size_t)t.nslot * row_bytes));
        t.bnd = static_cast<int2 *>(c->bnd.p);
        t.ckpt_every = every;
        RC(c->ckpt.ensure((size_t)std::max(1, t.nstrips / every) * row_bytes));
        t.ckpt = static_cast<int2 *>(c->ckpt.p);
    }
    RC(run_fill(c, c->fwd, false, {t}, t.nstrips, ds.K));
    RC(c->result.ensure(sizeof(int4)));
    reduce_candidates_kernel<<<1, 32, 0, c->stream>>>(static_cast<const FillTask *>(c->tasks.p), 1,
                                                       static_cast<const int4 *>(c->cand.p),
                                                       static_cast<int4 *>(c->result.p));
    CU(cudaGetLastError());
    ++c->launches;
    CU(cudaMemcpyAsync(c->stage3.p, c->result.p, sizeof(int4), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(static_cast<char *>(c->stage3.p) + 16, c->err.p, sizeof(int),
                       cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    int4 res;
    int e;
    std::memcpy(&res, c->stage3.p, sizeof(int4));
    std::memcpy(&e, static_cast<char *>(c->stage3.p) + 16, sizeof(int));
    RC(map_kernel_error(e));
    if (res.x <= 0) return empty_alignment(out);
    const int ie = res.y, je = res.z;

    // ---- 2. walk state
    RC(c->walk.ensure(sizeof(WalkState)));
    RC(c->runs.ensure((size_t)(ie + je + 2) * sizeof(int2)));
    WalkState w0{ie, je, 0, 0, 0, -1, 0};
    std::memcpy(c->stage2.p, &w0, sizeof(w0));
    CU(cudaMemcpyAsync(c->walk.p, c->stage2.p, sizeof(w0), cudaMemcpyHostToDevice, c->stream));

    // ---- 3. groups of checkpoint blocks, bottom-up
    const long long BR = (long long)HC * every;       // rows per block
    const int nblocks = (int)((ie + BR - 1) / BR);
    auto block_rows = [&](int bk) { return (int)std::min<long long>(BR, ie - bk * BR); };
    auto ckpt_row = [&](int bk) -> const int2 * {     // bottom row of block bk-1
        if (bk == 0) return nullptr;
        if (every == 1) return t.bnd + (size_t)(bk - 1) * n;
        return t.ckpt + (size_t)(bk - 1) * n;
    };
    const int wb = tb_word_bytes(c->tbc.R);
    WalkState w = w0;
    int hi = nblocks - 1;
    while (hi >= 0 && !w.done) {
        // largest group [lo, hi] whose bits fit the budget (at least one block)
        int lo = hi;
        auto group_bytes = [&](int l) {
            long long rows = (long long)(hi - l) * BR + ((block_rows(hi) + HT - 1) / HT) * (long long)HT;
            return (size_t)(rows / c->tbc.R) * (size_t)je * wb;
        };
        while (lo > 0 && group_bytes(lo - 1) <= c->tb_budget) --lo;
        RC(c->tb.ensure(group_bytes(lo)));
        std::vector<FillTask> tasks;
        long long tickets = 0;
        size_t bnd_need = 0;
        for (int bk = lo; bk <= hi; ++bk) {
            const int rows = block_rows(bk);
            const int ns = (rows + HT - 1) / HT;
            bnd_need += (size_t)std::min(ns, 2) * (size_t)je * sizeof(int2);
        }
        RC(c->tbbnd.ensure(bnd_need));
        size_t bnd_off = 0;
        for (int bk = lo; bk <= hi; ++bk) {
            FillTask u{};
            const int rows = block_rows(bk);
            u.a = da + (size_t)bk * BR;
            u.b = db;
            u.rows = rows;
            u.ncols = je;
            u.nstrips = (rows + HT - 1) / HT;
            u.scoring = 0;
            u.ticket0 = tickets;
            u.top = ckpt_row(bk);
            u.nslot = std::min(u.nstrips, 2);
            u.bnd = reinterpret_cast<int2 *>(static_cast<char *>(c->tbbnd.p) + bnd_off);
            bnd_off += (size_t)u.nslot * (size_t)je * sizeof(int2);
            u.ckpt_every = 0; u.ckpt = nullptr;
            u.row0 = (int32_t)(bk * BR);
            u.tb = static_cast<char *>(c->tb.p) + (size_t)((bk - lo) * BR / c->tbc.R) * (size_t)je * wb;
            u.tb_ld = je;
            tickets += u.nstrips;
            tasks.push_back(u);
        }
        RC(run_fill(c, c->tbc, true, tasks, tickets, ds.K));
        RC(launch_walk(c, c->tbc.R, c->tb.p, je, (int)(lo * BR)));
        CU(cudaMemcpyAsync(c->stage3.p, c->walk.p, sizeof(WalkState), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaMemcpyAsync(static_cast<char *>(c->stage3.p) + 64, c->err.p, sizeof(int),
                           cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        std::memcpy(&w, c->stage3.p, sizeof(w));
        std::memcpy(&e, static_cast<char *>(c->stage3.p) + 64, sizeof(int));
        RC(map_kernel_error(e));
        hi = lo - 1;
    }
    if (w.done != 1) return SW_ECUDA;     // the walk must end at a zero cell or the border

    // ---- 4. CIGAR text from the run records (stored end -> start)
    std::vector<int2> runs((size_t)w.nruns);
    if (w.nruns > 0) {
        CU(cudaMemcpy(runs.data(), c->runs.p, (size_t)w.nruns * sizeof(int2), cudaMemcpyDeviceToHost));
    }
    std::string cig;
    cig.reserve((size_t)w.nruns * 6);
    static const char opc[3] = {'M', 'I', 'D'};
    char buf[24];
    for (long long k = w.nruns - 1; k >= 0; --k) {
        const int2 r = runs[(size_t)k];
        if (r.x < 0 || r.x > 2) return SW_ECUDA;
        std::snprintf(buf, sizeof(buf), "%d%c", r.y, opc[r.x]);
        cig += buf;
    }
    char *s = static_cast<char *>(std::malloc(cig.size() + 1));
    if (!s) return SW_ENOMEM;
    std::memcpy(s, cig.c_str(), cig.size() + 1);
    *out = sw_alignment{res.x, 0, (int64_t)w.i, (int64_t)ie, (int64_t)w.j, (int64_t)je, s,
                        (int64_t)cig.size()};
    return SW_OK;
}
