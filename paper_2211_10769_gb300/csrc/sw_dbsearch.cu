// sw_dbsearch.cu -- database search (paper Section 2.1, one-to-many,
// inter-task): device-resident database, packed 16-bit search with exact
// 32-bit rescoring of saturating subjects, top-k hits.
#include "sw.h"
#include "sw_ctx.h"
#include "dbsearch.cuh"
#include "wavefront.cuh"
#include "aux_kernels.cuh"

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

using namespace swgb;

#define CU(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; } } while (0)
#define RC(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)

struct sw_db {
    int device = 0;
    int64_t nseq = 0;
    int32_t npairs = 0;
    int32_t maxlen = 0;
    int32_t max_code = -1;
    std::vector<int64_t> off;           // host copy of the offsets
    std::vector<int32_t> hpairs;        // host copy of the length-sorted pairs
    DevBuf res, doff, pairs, pres, poff;   // pres / poff: interleaved residues of every pair
};

namespace {

static __global__ void max_code_kernel(const uint8_t *s, long long len, int *out) {
    int mx = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += stride)
        mx = max(mx, (int)s[k]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

constexpr long long kMaxProfileSmem = 200 * 1024;

// Profile bytes of a query of m residues for tile shape (R, G) (whole passes
// of G lane slots of db_lane_slot(R) bytes, per residue code and padding).
template <int R, int G>
size_t db_profile_bytes(int K, int m) {
    constexpr int ROWS = G * R;
    const long long mpad = (long long)((m + ROWS - 1) / ROWS) * G * db_lane_slot(R);
    return (size_t)(K + 1) * (size_t)mpad;
}

// Scratch of one launch: boundary rows, one per wavefront (32 / G of them a
// warp) of every block that can be resident at once, and the slot pool's words.
template <int R, int W, int G>
int db_scratch(sw_ctx *c, int K, int m, int maxlen, int *nslots, size_t *row_bytes, size_t *slot_bytes) {
    const size_t smem = db_profile_bytes<R, G>(K, m);
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, db_s16x2_kernel<R, W, false, G>, W * 32, smem));
    int occ2 = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, db_s16x2_kernel<R, W, true, G>, W * 32, smem));
    occ = std::min(occ, occ2);
    if (occ < 1) return SW_ECUDA;
    *nslots = occ * c->nsm;
    *row_bytes = (size_t)*nslots * W * (32 / G) * (size_t)(maxlen + 1) * sizeof(uint2);
    *slot_bytes = (size_t)((*nslots + 31) / 32) * sizeof(unsigned);
    return SW_OK;
}

template <int R, int W, int G>
int launch_db(sw_ctx *c, const DbJob *jobs, int njobs, int nblocks, const DbView &D0, int K, int m,
              const DbBufs &B) {
    const size_t smem = db_profile_bytes<R, G>(K, m);
    // boundary rows: one per warp of every block that can be resident at once; a grid larger
    // than that (the server's steps) takes the kernel whose later blocks share the slots
    DbView D = D0;
    size_t row_bytes = 0, slot_bytes = 0;
    RC((db_scratch<R, W, G>(c, K, m, D.maxlen, &D.nslots, &row_bytes, &slot_bytes)));
    D.slot_words = (D.nslots + 31) / 32;
    const bool over = nblocks > D.nslots;
    RC(B.rows->ensure(row_bytes));
    RC(B.slots->ensure(slot_bytes));
    D.slot_pool = static_cast<unsigned *>(B.slots->p);
    D.err = B.err;
    D.spin_limit = c->spin_limit;
    if (over) {
        init_slot_pool_kernel<<<1, 64, 0, c->stream>>>(D.slot_pool, D.slot_words, D.nslots, D.nslots);
        CU(cudaGetLastError());
        ++c->launches;
    }
    auto kern = over ? db_s16x2_kernel<R, W, true, G> : db_s16x2_kernel<R, W, false, G>;
    const int kp = kt_begin(c, SW_KT_DB16);
    kern<<<(unsigned)nblocks, W * 32, smem, c->stream>>>(jobs, njobs, D, B.scorings,
                                                         static_cast<uint2 *>(B.rows->p));
    kt_end(c, kp);
    CU(cudaGetLastError());
    ++c->launches;
    return SW_OK;
}

template <int R, int W, int G>
int resident_blocks(sw_ctx *c, int K, int m, int *out) {
    const size_t smem = db_profile_bytes<R, G>(K, m);
    if ((long long)smem > kMaxProfileSmem) return SW_ERANGE;
    static int attr_set[64] = {0};
    if (c->device < 64 && !attr_set[c->device]) {
        CU(cudaFuncSetAttribute(db_s16x2_kernel<R, W, false, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kMaxProfileSmem));
        CU(cudaFuncSetAttribute(db_s16x2_kernel<R, W, true, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kMaxProfileSmem));
        attr_set[c->device] = 1;
    }
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, db_s16x2_kernel<R, W, false, G>, W * 32, smem));
    if (occ < 1) return SW_ECUDA;
    *out = occ * c->nsm;
    return SW_OK;
}

// Tile shapes of the packed search: rows a lane, warps a block and lanes a
// wavefront.  A query is padded to whole passes of G R rows, so short queries
// want few rows a pass: 144 residues take one 144-row pass in two 16-lane
// wavefronts a warp at R = 9 (in one 32-lane wavefront: 160 rows at R = 5, with
// a lane's fixed per-step cost shared by 5 rows instead of 9; measured 4,333
// against 3,476 GCUPS).  Long queries want R = 16, whose per-step overhead is
// shared by more rows.  Queries whose profile would not leave room for three
// blocks an SM take blocks of 16 warps (one per SM) at R = 16.  (Lanes of 4, 5,
// 6 and 12 rows in 32-lane wavefronts were measured too and never won.)
#define SWGB_DB_SHAPES(X)                                                                              \
    X(0, 8, 8, 32) X(1, 16, 8, 32) X(2, 4, 8, 16) X(3, 6, 8, 16) X(4, 9, 8, 16) X(5, 12, 8, 16)          \
    X(6, 16, 16, 32)
struct DbShape { int R, W, G; };
#define SWGB_DB_ROW(i, R, W, G) {R, W, G},
constexpr DbShape kDbShapes[] = {SWGB_DB_SHAPES(SWGB_DB_ROW)};
#undef SWGB_DB_ROW
constexpr int kDbWide = 6;                         // index of the one-block-an-SM shape
constexpr size_t kDbNarrowProfileMax = 96 * 1024;  // profile bytes of a three-blocks-an-SM shape at most
// cost model of a shape (db_shape), fitted to measured GCUPS of every shape at query lengths 144,
// 300, 464, 700, 1,000 and 2,005 (it picks the fastest at each): a lane's fixed per-step cost in
// rows' worth, a pass boundary in rows, and a typical subject length (a wavefront's skew of
// G - 1 steps costs about (G - 1) / 360 of a pair's sweep)
constexpr double kDbStepRows = 2.25, kDbPassRows = 16, kDbTypicalCols = 360;

size_t shape_profile_bytes(int s, int K, int m) {
    switch (s) {
#define SWGB_DB_CASE(i, R, W, G) case i: return db_profile_bytes<R, G>(K, m);
        SWGB_DB_SHAPES(SWGB_DB_CASE)
#undef SWGB_DB_CASE
        default: return 0;
    }
}

}  // namespace

// The shape for a query of m residues: the least padded work, counting the
// per-step overhead of a lane, a pass boundary and the wavefront's skew, among
// the shapes whose profile fits.
int swgb::db_shape(int K, int m) {
    // tuning override: SWGB_DB_SHAPE=<index into kDbShapes>, where its profile fits
    static const int forced = [] { const char *f = std::getenv("SWGB_DB_SHAPE"); return f ? std::atoi(f) : -1; }();
    if (forced >= 0 && forced < kDbWide && shape_profile_bytes(forced, K, m) <= kDbNarrowProfileMax) return forced;
    int best = kDbWide;
    double best_cost = 1e300;
    for (int s = 0; s < kDbWide; ++s) {
        if (shape_profile_bytes(s, K, m) > kDbNarrowProfileMax) continue;
        const int R = kDbShapes[s].R, G = kDbShapes[s].G, rows = G * R;
        const long long passes = (m + rows - 1) / rows;
        const double cost = (double)passes * rows * (R + kDbStepRows) / R * (1.0 + (G - 1) / kDbTypicalCols) +
                            kDbPassRows * (double)passes;
        if (cost < best_cost) { best_cost = cost; best = s; }
    }
    return best;
}

int swgb::db_resident_blocks_shape(sw_ctx *c, int shape, int K, int m, int *out) {
    switch (shape) {
#define SWGB_DB_CASE(i, R, W, G) case i: return resident_blocks<R, W, G>(c, K, m, out);
        SWGB_DB_SHAPES(SWGB_DB_CASE)
#undef SWGB_DB_CASE
        default: return SW_EINVAL;
    }
}

int swgb::db_resident_blocks(sw_ctx *c, int K, int m, int *out) {
    return db_resident_blocks_shape(c, db_shape(K, m), K, m, out);
}

int swgb::db_shape_warps(int shape) { return kDbShapes[shape].W; }
int swgb::db_shape_rows(int shape) { return kDbShapes[shape].G * kDbShapes[shape].R; }
int swgb::db_warps_per_block(int K, int m) { return db_shape_warps(db_shape(K, m)); }
int swgb::db_rows_per_pass(int K, int m) { return db_shape_rows(db_shape(K, m)); }

int swgb::db_launch_shape(sw_ctx *c, int shape, const DbJob *jobs, int njobs, int nblocks, const DbView &D, int K,
                          int m, const DbBufs *bufs) {
    DbBufs B{&c->dbscratch, &c->dbslots, static_cast<const DevScoring *>(c->scorings.p), static_cast<int *>(c->err.p)};
    if (bufs) B = *bufs;
    switch (shape) {
#define SWGB_DB_CASE(i, R, W, G) case i: return launch_db<R, W, G>(c, jobs, njobs, nblocks, D, K, m, B);
        SWGB_DB_SHAPES(SWGB_DB_CASE)
#undef SWGB_DB_CASE
        default: return SW_EINVAL;
    }
}

int swgb::db_scratch_shape(sw_ctx *c, int shape, int K, int m, int maxlen, size_t *row_bytes, size_t *slot_bytes) {
    int nslots = 0;
    switch (shape) {
#define SWGB_DB_CASE(i, R, W, G) case i: return db_scratch<R, W, G>(c, K, m, maxlen, &nslots, row_bytes, slot_bytes);
        SWGB_DB_SHAPES(SWGB_DB_CASE)
#undef SWGB_DB_CASE
        default: return SW_EINVAL;
    }
}

int swgb::db_launch(sw_ctx *c, const DbJob *jobs, int njobs, int nblocks, const DbView &D, int K, int m) {
    return db_launch_shape(c, db_shape(K, m), jobs, njobs, nblocks, D, K, m);
}

int swgb::db_view(const sw_db *db, DbView *v, int64_t *nseq, int32_t *max_code, int *device) {
    v->res = static_cast<const uint8_t *>(db->res.p);
    v->off = static_cast<const int64_t *>(db->doff.p);
    v->pairs = static_cast<const int32_t *>(db->pairs.p);
    v->pres = static_cast<const uint16_t *>(db->pres.p);
    v->poff = static_cast<const int64_t *>(db->poff.p);
    v->npairs = db->npairs;
    v->maxlen = db->maxlen;
    *nseq = db->nseq;
    *max_code = db->max_code;
    *device = db->device;
    return SW_OK;
}

int64_t swgb::db_total_residues(const sw_db *db) { return db->off.empty() ? 0 : db->off.back(); }

int swgb::db_chunk_maxlen(const sw_db *db, int32_t pair0, int32_t pair1) {
    int64_t mx = 0;
    for (int32_t p = pair0; p < pair1 && p < db->npairs; ++p)
        for (int h = 0; h < 2; ++h) {
            const int32_t s = db->hpairs[(size_t)(2 * p + h)];
            if (s >= 0) mx = std::max(mx, db->off[(size_t)s + 1] - db->off[(size_t)s]);
        }
    return (int)mx;
}

extern "C" int sw_db_create(sw_ctx *c, const uint8_t *residues, const int64_t *offsets, int64_t nseq,
                            sw_db **out) {
    if (!c || !out || !offsets || nseq < 0 || nseq > (int64_t)1 << 30) return SW_EINVAL;
    if (offsets[0] != 0) return SW_EINVAL;
    for (int64_t s = 0; s < nseq; ++s) {
        if (offsets[s + 1] < offsets[s]) return SW_EINVAL;
        if (offsets[s + 1] - offsets[s] > SW_MAX_LEN) return SW_ERANGE;
    }
    const int64_t total = offsets[nseq];
    if (total > 0 && !residues) return SW_EINVAL;
    DeviceGuard g(c->device);
    sw_db *db = new (std::nothrow) sw_db();
    if (!db) return SW_ENOMEM;
    db->device = c->device;
    db->nseq = nseq;
    db->off.assign(offsets, offsets + nseq + 1);
    int rc = db->res.ensure((size_t)total + 16);
    if (!rc) rc = db->doff.ensure((size_t)(nseq + 1) * sizeof(int64_t));
    if (rc) { delete db; return rc; }
    // length-sorted pairs, longest first (ties by index)
    std::vector<int32_t> order((size_t)nseq);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return offsets[x + 1] - offsets[x] > offsets[y + 1] - offsets[y];
    });
    db->npairs = (int32_t)((nseq + 1) / 2);
    std::vector<int32_t> pairs((size_t)db->npairs * 2, -1);
    for (int64_t k = 0; k < nseq; ++k) pairs[(size_t)k] = order[(size_t)k];
    int64_t maxlen = 0;
    for (int64_t s = 0; s < nseq; ++s) maxlen = std::max(maxlen, offsets[s + 1] - offsets[s]);
    db->maxlen = (int32_t)maxlen;
    db->hpairs = pairs;
    rc = db->pairs.ensure(std::max<size_t>(1, pairs.size()) * sizeof(int32_t));
    if (rc) { delete db; return rc; }
    // interleaved residues of the pairs: max(na, nb) columns plus one padding column each
    std::vector<int64_t> poff((size_t)db->npairs + 1, 0);
    for (int32_t p = 0; p < db->npairs; ++p) {
        const int32_t sa = pairs[2 * (size_t)p], sb = pairs[2 * (size_t)p + 1];
        const int64_t na = offsets[sa + 1] - offsets[sa];
        const int64_t nb = sb >= 0 ? offsets[sb + 1] - offsets[sb] : 0;
        poff[(size_t)p + 1] = poff[(size_t)p] + std::max(na, nb) + 1;
    }
    rc = db->pres.ensure(std::max<size_t>(1, (size_t)poff.back()) * sizeof(uint16_t));
    if (!rc) rc = db->poff.ensure(poff.size() * sizeof(int64_t));
    if (rc) { delete db; return rc; }
    const cudaMemcpyKind kind = is_device_ptr(residues) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    bool ok = true;
    if (total > 0) ok &= cudaMemcpyAsync(db->res.p, residues, (size_t)total, kind, c->stream) == cudaSuccess;
    ok &= cudaMemcpyAsync(db->doff.p, offsets, (size_t)(nseq + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
    if (!pairs.empty())
        ok &= cudaMemcpyAsync(db->pairs.p, pairs.data(), pairs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
    ok &= cudaMemcpyAsync(db->poff.p, poff.data(), poff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
    if (ok && db->npairs > 0) {
        pair_residues_kernel<<<(unsigned)std::min<long long>((db->npairs + 7) / 8, 16LL * c->nsm), 256, 0, c->stream>>>(
            static_cast<const uint8_t *>(db->res.p), static_cast<const int64_t *>(db->doff.p),
            static_cast<const int32_t *>(db->pairs.p), static_cast<const int64_t *>(db->poff.p), db->npairs,
            static_cast<uint16_t *>(db->pres.p));
        ok &= cudaGetLastError() == cudaSuccess;
        ++c->launches;
    }
    // largest residue code, checked against the alphabet at search time
    ok &= c->misc.ensure(sizeof(int)) == SW_OK;
    ok &= cudaMemsetAsync(c->misc.p, 0, sizeof(int), c->stream) == cudaSuccess;
    if (ok && total > 0) {
        max_code_kernel<<<(unsigned)std::min<long long>((total + 255) / 256, 8LL * c->nsm), 256, 0, c->stream>>>(
            static_cast<const uint8_t *>(db->res.p), total, static_cast<int *>(c->misc.p));
        ok &= cudaGetLastError() == cudaSuccess;
        ++c->launches;
    }
    int mc = 0;
    ok &= cudaMemcpyAsync(&mc, c->misc.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream) == cudaSuccess;
    ok &= cudaStreamSynchronize(c->stream) == cudaSuccess;
    if (!ok) { cudaGetLastError(); delete db; return SW_ECUDA; }
    db->max_code = total > 0 ? mc : -1;
    *out = db;
    return SW_OK;
}

extern "C" void sw_db_destroy(sw_db *db) {
    if (!db) return;
    DeviceGuard g(db->device);
    delete db;
}

extern "C" int64_t sw_db_size(const sw_db *db) { return db ? db->nseq : -1; }

// Score every subject of the database against query q (device array
// scores, int32 per subject), flagged subjects rescored exactly.
int swgb::db_score_all(sw_ctx *c, const sw_db *db, const uint8_t *dq, int64_t m, const DevScoring &ds,
                       int32_t *dscores) {
    const int K = ds.K;
    RC(c->dbovf.ensure((size_t)std::max<int64_t>(1, db->nseq) * sizeof(int32_t)));
    RC(c->dbjob.ensure(sizeof(DbJob) + 64));
    int32_t *novf = reinterpret_cast<int32_t *>(static_cast<char *>(c->dbjob.p) + sizeof(DbJob));
    int32_t *next = novf + 1;
    CU(cudaMemsetAsync(novf, 0, 2 * sizeof(int32_t), c->stream));
    DbJob job;
    job.q = dq; job.m = (int32_t)m; job.scoring = 0;
    job.pair0 = 0; job.pair1 = db->npairs; job.pair_stride = 1; job.block0 = 0;
    job.scores = dscores;
    job.ovf = static_cast<int32_t *>(c->dbovf.p);
    job.novf = novf; job.next_pair = next;
    RC(c->stage.ensure(sizeof(DbJob)));
    std::memcpy(c->stage.p, &job, sizeof(job));
    CU(cudaMemcpyAsync(c->dbjob.p, c->stage.p, sizeof(job), cudaMemcpyHostToDevice, c->stream));
    DbView D;
    D.res = static_cast<const uint8_t *>(db->res.p);
    D.off = static_cast<const int64_t *>(db->doff.p);
    D.pairs = static_cast<const int32_t *>(db->pairs.p);
    D.pres = static_cast<const uint16_t *>(db->pres.p);
    D.poff = static_cast<const int64_t *>(db->poff.p);
    D.npairs = db->npairs;
    D.maxlen = db->maxlen;
    int32_t nflag = 0;
    std::vector<int32_t> flagged;
    const bool packed_ok = fold_open(ds) && ds.go <= 16000 && ds.ge <= 16000;
    int rc = SW_ERANGE;
    if (packed_ok) {
        int nblk = 0;
        rc = db_resident_blocks(c, K, (int)m, &nblk);
        if (!rc) {
            const int W = db_warps_per_block(K, (int)m);
            nblk = std::max(1, std::min(nblk, (db->npairs + W - 1) / W));
            rc = db_launch(c, static_cast<const DbJob *>(c->dbjob.p), 1, nblk, D, K, (int)m);
        }
    }
    if (rc == SW_ERANGE) {
        // the packed kernel cannot take this query / scoring: score every subject in int32
        flagged.resize((size_t)db->nseq);
        std::iota(flagged.begin(), flagged.end(), 0);
    } else {
        RC(rc);
        CU(cudaMemcpyAsync(c->stage3.p, novf, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        std::memcpy(&nflag, c->stage3.p, sizeof(int32_t));
        if (nflag > 0) {
            flagged.resize((size_t)nflag);
            CU(cudaMemcpy(flagged.data(), c->dbovf.p, (size_t)nflag * sizeof(int32_t), cudaMemcpyDeviceToHost));
        }
    }
    if (flagged.empty()) return SW_OK;
    return db_rescore(c, db, dq, m, ds, flagged, dscores);
}

// Exact rescoring: one int32 wavefront task per flagged subject (query down
// the rows); scores[flagged[k]] receives the result.
int swgb::db_rescore(sw_ctx *c, const sw_db *db, const uint8_t *dq, int64_t m, const DevScoring &ds,
                     const std::vector<int32_t> &flagged, int32_t *dscores) {
    const int K = ds.K;
    RC(upload_scorings(c, {ds}));
    const int HC = fill_rows_per_strip(c->bat);
    std::vector<FillTask> tasks;
    tasks.reserve(flagged.size());
    long long tickets = 0;
    size_t bnd_need = 0;
    for (int32_t s : flagged) {
        const int64_t n = db->off[(size_t)s + 1] - db->off[(size_t)s];
        const int ns = (int)((m + HC - 1) / HC);
        bnd_need += (size_t)std::min(ns, 2) * (size_t)std::max<int64_t>(n, 1) * sizeof(int2);
    }
    RC(c->tbbnd.ensure(bnd_need));
    size_t boff = 0;
    for (int32_t s : flagged) {
        FillTask u{};
        const int64_t n = db->off[(size_t)s + 1] - db->off[(size_t)s];
        u.a = dq; u.rows = (int32_t)m;
        u.b = static_cast<const uint8_t *>(db->res.p) + db->off[(size_t)s];
        u.ncols = (int32_t)n;
        u.nstrips = (int32_t)((m + HC - 1) / HC);
        u.scoring = 0;
        u.ticket0 = tickets;
        u.nslot = std::min(u.nstrips, 2);
        u.bnd = reinterpret_cast<int2 *>(static_cast<char *>(c->tbbnd.p) + boff);
        boff += (size_t)u.nslot * (size_t)std::max<int64_t>(n, 1) * sizeof(int2);
        tickets += n > 0 ? u.nstrips : 0;
        if (n == 0) { u.nstrips = 0; }
        tasks.push_back(u);
    }
    RC(run_fill(c, c->bat, kModeScore, fold_open(ds), tasks, tickets, K));
    const int nt = (int)tasks.size();
    RC(c->result.ensure((size_t)nt * sizeof(int4)));
    reduce_candidates_kernel<<<(nt + 7) / 8, 256, 0, c->stream>>>(static_cast<const FillTask *>(c->tasks.p), nt,
                                                                  static_cast<const int4 *>(c->cand.p),
                                                                  static_cast<const DevScoring *>(c->scorings.p),
                                                                  static_cast<int4 *>(c->result.p));
    CU(cudaGetLastError());
    ++c->launches;
    RC(c->dbovf.ensure((size_t)nt * sizeof(int32_t)));
    CU(cudaMemcpyAsync(c->dbovf.p, flagged.data(), (size_t)nt * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    scatter_scores_kernel<<<(nt + 255) / 256, 256, 0, c->stream>>>(static_cast<const int32_t *>(c->dbovf.p),
                                                                   static_cast<const int4 *>(c->result.p), nt, dscores);
    CU(cudaGetLastError());
    ++c->launches;
    CU(cudaStreamSynchronize(c->stream));      // flagged is host memory used by the copy above
    return SW_OK;
}

// Top-k of a device score array: (subject, score) pairs, score descending,
// subject ascending.
int swgb::db_topk(sw_ctx *c, const int32_t *dscores, int64_t nseq, int k, int2 *dout) {
    const int nb = (int)((nseq + kTopkChunk - 1) / kTopkChunk);
    RC(c->topk.ensure((size_t)std::max(1, nb) * k * sizeof(unsigned long long)));
    topk_phase1_kernel<<<nb, kTopkThreads, 0, c->stream>>>(dscores, (int)nseq, k,
                                                           static_cast<unsigned long long *>(c->topk.p));
    CU(cudaGetLastError());
    ++c->launches;
    const size_t smem = (size_t)nb * k * sizeof(unsigned long long);
    static int attr_set = 0;
    if (!attr_set) {
        CU(cudaFuncSetAttribute(topk_phase2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr_set = 1;
    }
    if (smem > 200 * 1024) return SW_ERANGE;
    topk_phase2_kernel<<<1, kTopkThreads, smem, c->stream>>>(static_cast<const unsigned long long *>(c->topk.p),
                                                             nb * k, k, dout);
    CU(cudaGetLastError());
    ++c->launches;
    return SW_OK;
}

extern "C" int sw_dbsearch(sw_ctx *c, const sw_db *db, const uint8_t *q, int64_t m, const sw_scoring *sc,
                           int32_t k, sw_dbhit *hits, int32_t *nhits, int32_t *all_scores) {
    if (!c || !db || !nhits || k < 0 || k > 64 || (k > 0 && !hits)) return SW_EINVAL;
    if (db->device != c->device) return SW_EINVAL;
    DevScoring ds;
    RC(check_scoring(sc, &ds));
    if (ds.alg != kAlgLocal) return SW_EINVAL;          // database search: the local algorithm
    if (m < 0 || (m > 0 && !q)) return SW_EINVAL;
    if (m > SW_MAX_LEN) return SW_ERANGE;
    if (db->max_code >= ds.K) return SW_EINVAL;
    if ((double)std::min<int64_t>(m, db->maxlen) * (double)max_pos_score(sc) >= (double)kMaxScoreBound) return SW_ERANGE;
    DeviceGuard g(c->device);
    const int64_t nseq = db->nseq;
    RC(c->dbscores.ensure((size_t)std::max<int64_t>(1, nseq) * sizeof(int32_t)));
    int32_t *dscores = static_cast<int32_t *>(c->dbscores.p);
    if (nseq > 0) CU(cudaMemsetAsync(dscores, 0, (size_t)nseq * sizeof(int32_t), c->stream));
    if (m > 0 && nseq > 0) {
        const uint8_t *dq;
        RC(stage_seq(c, q, m, c->seq_a, &dq));
        RC(reset_err(c));
        RC(validate_codes(c, dq, m, ds.K));
        RC(upload_scorings(c, {ds}));
        RC(db_score_all(c, db, dq, m, ds, dscores));
    }
    const int kk = (int)std::min<int64_t>(k, nseq);
    if (kk > 0) {
        RC(c->result.ensure(64 * sizeof(int4)));
        RC(db_topk(c, dscores, nseq, kk, static_cast<int2 *>(c->result.p)));
        CU(cudaMemcpyAsync(c->stage3.p, c->result.p, (size_t)kk * sizeof(int2), cudaMemcpyDeviceToHost, c->stream));
    }
    CU(cudaMemcpyAsync(static_cast<char *>(c->stage3.p) + 1024, c->err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if (all_scores && nseq > 0) {
        CU(cudaMemcpyAsync(all_scores, dscores, (size_t)nseq * sizeof(int32_t),
                           is_device_ptr(all_scores) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    }
    CU(cudaStreamSynchronize(c->stream));
    int e;
    std::memcpy(&e, static_cast<char *>(c->stage3.p) + 1024, sizeof(int));
    RC(map_kernel_error(e));
    const int2 *h = static_cast<const int2 *>(c->stage3.p);
    for (int i = 0; i < kk; ++i) hits[i] = sw_dbhit{(int64_t)h[i].x, h[i].y, 0};
    *nhits = kk;
    return SW_OK;
}
