// sw_align.cu -- reconstruction phase (paper Section 2.2: resolution finds
// the best score, reconstruction recovers the path with space-efficient
// methods).
//
// 1. Forward fill over the whole matrix (score mode with checkpoints): the
//    H / F row at every BT-th row and the H / E column at every BT-th
//    column are kept.  BT is the smallest multiple of both fills' strip
//    heights (at least 1024) for which both sets of checkpoints fit the
//    checkpoint budget, so memory is O((m + n)^2 / BT) rather than m x n.
//    The columns are stored in staircase form (each lane of the fill one
//    column further left than the lane above it, all at one step, so the
//    sweep needs no per-step test); a tile entered from one first brings its
//    lanes to the straight column (see FillTask::left).
// 2. The end cell (ie, je) comes from the per-strip candidates.
// 3. With checkpoints on both sides, every BT x BT tile can be recomputed
//    on its own from its top row and left column.  The walk goes
//    in rounds: recompute the decision bits of a diagonal band of tiles
//    from the walk's current tile towards the upper left (traceback mode,
//    every tile an independent task of one launch), walk the path through
//    them, and start the next band where the walk left the computed tiles.
//    Only tiles near the path are recomputed.
// 4. The run records of the walk become the CIGAR text on the host.
#include "sw.h"
#include "sw_ctx.h"
#include "wavefront.cuh"
#include "walk.cuh"
#include "aux_kernels.cuh"

#include <algorithm>
#include <numeric>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace swgb;

#define CU(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; } } while (0)
#define RC(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)

namespace {

constexpr int kMinBandDepth = 16;         // tile rows per band at least
constexpr long long kWalkMaxIters = 1LL << 26;

int empty_alignment(sw_alignment *out) {
    char *s = static_cast<char *>(std::malloc(1));
    if (!s) return SW_ENOMEM;
    s[0] = 0;
    *out = sw_alignment{0, 0, 0, 0, 0, 0, s, 0};
    return SW_OK;
}

// The forced part of a path that reaches the matrix border at (i, j) in
// state H: the global algorithm continues from (i, 0) with i deletions and
// from (0, j) with j insertions to (0, 0), the semi-global one from (i, 0)
// with i deletions; the other border cells are free starts.  Returns the
// CIGAR text of that run ("" when none) and moves (i, j) to where the path
// starts.
std::string border_run(int alg, int64_t *i, int64_t *j) {
    char buf[32];
    if (*j == 0 && *i > 0 && (alg == kAlgGlobal || alg == kAlgSemiGlobal)) {
        std::snprintf(buf, sizeof(buf), "%lldD", (long long)*i);
        *i = 0;
        return buf;
    }
    if (*i == 0 && *j > 0 && alg == kAlgGlobal) {
        std::snprintf(buf, sizeof(buf), "%lldI", (long long)*j);
        *j = 0;
        return buf;
    }
    return "";
}

// An alignment whose end cell (ie, je) lies on the border: only the forced
// border run, if any.
int border_alignment(int alg, int score, int64_t ie, int64_t je, sw_alignment *out) {
    int64_t i = ie, j = je;
    const std::string cig = border_run(alg, &i, &j);
    char *s = static_cast<char *>(std::malloc(cig.size() + 1));
    if (!s) return SW_ENOMEM;
    std::memcpy(s, cig.c_str(), cig.size() + 1);
    *out = sw_alignment{score, 0, i, ie, j, je, s, (int64_t)cig.size()};
    return SW_OK;
}

// The alignment from the walk's run records (stored end -> start), after the
// forced run of a path that reached the border (the global and semi-global
// algorithms).
int finish_alignment(int alg, int score, int64_t ie, int64_t je, const WalkState &w, const int2 *runs,
                     sw_alignment *out) {
    int64_t bi = w.i, bj = w.j;
    std::string cig = border_run(alg, &bi, &bj);
    cig.reserve(cig.size() + (size_t)w.nruns * 6);
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
    *out = sw_alignment{score, 0, bi, ie, bj, je, s, (int64_t)cig.size()};
    return SW_OK;
}

template <typename Word, int R>
int launch_walk_t(sw_ctx *c, const void *const *table, int I0, int J0, int nI, int nJ, int BT) {
    if ((long long)nI * nJ > kWalkTableMax || BT < kWalkMinBT || BT % R != 0) return SW_EINVAL;
    TileTable<Word> T;
    T.bits = reinterpret_cast<const Word *const *>(table);
    T.I0 = I0; T.J0 = J0; T.nI = nI; T.nJ = nJ; T.BT = BT; T.R = R;
    T.win_groups = walk_window_groups(BT, R);
    const size_t smem = walk_window_bytes<R>(sizeof(Word));
    static int attr_set[64] = {0};                       // per instantiation and device
    if (c->device >= 64 || !attr_set[c->device]) {
        CU(cudaFuncSetAttribute(walk_kernel<Word, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (c->device < 64) attr_set[c->device] = 1;
    }
    const int kp = kt_begin(c, SW_KT_WALK);
    walk_kernel<Word, R><<<1, kWalkThreads, smem, c->stream>>>(T, static_cast<WalkState *>(c->walk.p),
                                                               static_cast<int2 *>(c->runs.p), kWalkMaxIters);
    kt_end(c, kp);
    CU(cudaGetLastError());
    ++c->launches;
    return SW_OK;
}

int launch_walk(sw_ctx *c, const void *const *table, int I0, int J0, int nI, int nJ, int BT, int R) {
    switch (R) {
        case 4: return launch_walk_t<uint16_t, 4>(c, table, I0, J0, nI, nJ, BT);
        case 8: return launch_walk_t<uint32_t, 8>(c, table, I0, J0, nI, nJ, BT);
        case 12: return launch_walk_t<unsigned long long, 12>(c, table, I0, J0, nI, nJ, BT);
        case 16: return launch_walk_t<unsigned long long, 16>(c, table, I0, J0, nI, nJ, BT);
        default: return SW_EINVAL;
    }
}

// Traceback band: the margin around the walk's diagonal, as a fraction of the tile side, and
// the tile columns a row of the walk's table keeps along the diagonal.
constexpr long long kBandMarginDiv = 8;
constexpr int kBandWidth = 5;

// Run records of paths up to this many bytes come back with every round's walk state.
constexpr size_t kRunsEachRoundBytes = 256 * 1024;

// One checkpoint level while its tile side stays within this; two levels above it.
constexpr long long kMaxOneLevelBT = 16384;
constexpr long long kSmallPairSide = 16384;   // pairs up to this side may take 512-row traceback tiles

// Two levels of checkpoints: fill the part of coarse tile (CI, CJ) above and left
// of (Wi0, Wj0) again, entered from the forward fill's checkpoint row above it and
// its staircase column left of it, keeping checkpoint rows and staircase columns
// every BT2 inside it: the forward fill's own kind (the packed fill enters its
// two-positions staircase as its state after step -1; the int32 fill its
// staircase through the prologue) with its rows per lane, so that the refill's
// staircase columns have the forward fill's form too.  Memory for the refill's
// checkpoints is about 16 BT1^2 / BT2 bytes, for any pair size.
int refill_coarse_tile(sw_ctx *c, const uint8_t *da, const uint8_t *db, int64_t n, const DevScoring &ds,
                       const FillConfig &fwd, bool fold, int aux_rows, const int2 *rowck, const int2 *colck,
                       const int2 *colaux, long long colck_ld, long long colaux_ld, long long CI, long long CJ,
                       long long R0c, long long C0c, long long Wi0, long long Wj0, long long BT2,
                       const int2 **rowck2, const int2 **colck2, const int2 **colaux2, long long *ld2, long long *N2) {
    FillConfig fc{fwd.R, 4};
    fc.alg = fwd.alg;
    fc.P16 = fwd.P16;
    fc.left = 1;
    const int HC2 = 4 * 32 * fc.R;
    const long long M2 = Wi0 - R0c, W2 = Wj0 - C0c;
    FillTask t{};
    t.a = da + R0c; t.b = db + C0c;
    t.rows = (int32_t)M2; t.ncols = (int32_t)W2;
    t.strip_warps = 4;
    t.nstrips = (int32_t)((M2 + HC2 - 1) / HC2);
    t.nslot = std::min(t.nstrips, 4);
    RC(c->bnd.ensure((size_t)t.nslot * (size_t)W2 * sizeof(int2)));
    t.bnd = static_cast<int2 *>(c->bnd.p);
    t.top = CI > 0 ? rowck + (size_t)(CI - 1) * n + C0c : nullptr;
    if (CJ > 0) {
        t.left = colck + (size_t)(CJ - 1) * colck_ld + R0c;
        t.left_aux = colaux + (size_t)(CJ - 1) * colaux_ld + R0c / aux_rows;
        t.left_split = fwd.P16 ? 1 : 0;
    }
    t.row0 = (int32_t)R0c;
    t.col0 = (int32_t)C0c;
    const long long nr = std::max<long long>(1, M2 / BT2), nc = std::max<long long>(1, W2 / BT2);
    t.ckpt_every = (int32_t)(BT2 / HC2);
    RC(c->ckpt2.ensure((size_t)nr * (size_t)W2 * sizeof(int2)));
    t.ckpt = static_cast<int2 *>(c->ckpt2.p);
    t.colck_every = (int32_t)BT2;
    t.colck_ld = (long long)t.nstrips * HC2;
    RC(c->colck2.ensure((size_t)nc * (size_t)t.colck_ld * sizeof(int2)));
    RC(c->colaux2.ensure((size_t)nc * (size_t)(t.colck_ld / aux_rows) * sizeof(int2)));
    // the fill writes column checkpoints at colck + k ld + (row0 + row) and their row-group
    // records at colck_aux + k ld / A + (row0 + row) / A (A = rows a record: R, or R / 2 for the
    // packed fill's half-groups): based so that row0 lands on 0
    t.colck = static_cast<int2 *>(c->colck2.p) - R0c;
    t.colck_aux = static_cast<int2 *>(c->colaux2.p) - R0c / aux_rows;
    RC(run_fill(c, fc, kModeScoreCk, fold, {t}, t.nstrips, ds.K));
    int e = 0;
    RC(read_err(c, &e));          // synchronises: the next fill reuses the staging buffer
    RC(map_kernel_error(e));
    *rowck2 = static_cast<const int2 *>(c->ckpt2.p);
    *colck2 = static_cast<const int2 *>(c->colck2.p);
    *colaux2 = static_cast<const int2 *>(c->colaux2.p);
    *ld2 = t.colck_ld;
    *N2 = W2;
    return SW_OK;
}

// Sides up to this many cells may take the one-round reconstruction below.
constexpr int64_t kOneRoundSide = 8192;

// Tile side of a small pair's reconstruction: a multiple of both fills' strip
// heights and of the chunk, at least kWalkMinBT, the smallest whose tiles fit
// one wave on the SMs (else the largest tried, up to the pair's side); 0 if
// none fits the chunk.
long long small_pair_tile(const sw_ctx *c, int64_t m, int64_t n, const DevScoring &ds, FillConfig *fwd_out,
                          FillConfig *tbc_out, int *sw_out, int *tsw_out) {
    const FillConfig fwd = pair_fill_config_for(c, m, ds);
    // strips of two compute warps (at R = 4: 256 rows) in both fills, so that a tile can be one
    // two-warp strip of 256 rows: a small pair's forward chain has as many warps either way, and
    // a tile recomputes in about half the steps of a 512-row one
    const int sw = c->fwd_auto ? std::min(2, fwd.W) : pair_strip_warps(c, fwd, m);
    const int HC = sw * 32 * fwd.R;
    // the traceback tiles continue the forward fill's staircase checkpoint columns lane by
    // lane, so both fills must give each lane the same rows (R)
    FillConfig tbc = (c->tbc.R == fwd.R && fwd.alg == kAlgLocal) ? c->tbc : FillConfig{fwd.R, 4};
    tbc.P16 = 0;
    tbc.alg = fwd.alg;
    const int tsw = c->tb_strip_warps > 0 ? std::min(c->tb_strip_warps, tbc.W) : std::min(2, tbc.W);
    const long long BL = std::lcm((long long)HC, (long long)tsw * 32 * tbc.R);
    long long BT = BL * ((kWalkMinBT + BL - 1) / BL);
    auto tiles = [&](long long bt) { return ((m + bt - 1) / bt) * ((n + bt - 1) / bt); };
    while (tiles(BT) > c->nsm && BT < std::max(m, n)) BT += BL;
    if (BT % kCH != 0) return 0;
    *fwd_out = fwd;
    *tbc_out = tbc;
    *sw_out = sw;
    *tsw_out = tsw;
    return BT;
}

// Reconstruction of a small pair in one round, with one host synchronisation:
// the forward fill with checkpoints every BT rows and columns, the end cell
// reduced on the device, every BT x BT traceback tile of the matrix
// recomputed from those checkpoints in one launch (independent tasks), the
// walk started from the end cell there (walk_start_kernel) through a table of
// all tiles, and every result copied back at once.  The banded path needs a
// host round trip between the end cell and its band; for a pair whose tiles
// fit one wave on the SMs, recomputing all of them costs no more time.
int align_one_round(sw_ctx *c, const uint8_t *da, int64_t m, const uint8_t *db, int64_t n, const DevScoring &ds,
                    bool fold, const FillConfig &fwd, const FillConfig &tbc, int sw, int tsw, long long BT,
                    sw_alignment *out) {
    const int HC = sw * 32 * fwd.R;
    const int R = tbc.R;
    const int aux_rows = fwd.P16 ? fwd.R / 2 : fwd.R;
    const int HS = tsw * 32 * R;
    if (BT % HC != 0 || BT % HS != 0) return SW_EINVAL;
    const int nI = (int)((m + BT - 1) / BT), nJ = (int)((n + BT - 1) / BT);
    // the walk's table: row ti keeps tile columns [ti + J0, ti + J0 + nJw) (its diagonal layout),
    // J0 = 1 - nI and nJw = nI + nJ - 1 columns, so that every row holds all of its tiles
    const int J0 = 1 - nI, nJw = nI + nJ - 1;
    if ((long long)nI * nJw > kWalkTableMax) return SW_EINVAL;
    const int ntiles = nI * nJ;
    const size_t tile_bytes = (size_t)(BT / R) * (size_t)BT * (size_t)tb_word_bytes(R);
    const long long nrowck = std::max<long long>(1, m / BT), ncolck = std::max<long long>(1, n / BT);

    FillTask t{};                                   // the forward fill, checkpoints every BT
    t.a = da; t.b = db;
    t.rows = (int32_t)m; t.ncols = (int32_t)n;
    t.strip_warps = sw;
    t.nstrips = (int32_t)((m + HC - 1) / HC);
    t.nslot = std::min(t.nstrips, 4);
    RC(c->bnd.ensure((size_t)t.nslot * (size_t)n * sizeof(int2)));
    t.bnd = static_cast<int2 *>(c->bnd.p);
    t.ckpt_every = (int32_t)(BT / HC);
    RC(c->ckpt.ensure((size_t)nrowck * (size_t)n * sizeof(int2)));
    t.ckpt = static_cast<int2 *>(c->ckpt.p);
    t.colck_every = (int32_t)BT;
    t.colck_ld = (long long)t.nstrips * HC;     // rows padded to whole strips (the padding is written)
    RC(c->colck.ensure((size_t)ncolck * (size_t)t.colck_ld * sizeof(int2)));
    RC(c->colaux.ensure((size_t)ncolck * (size_t)(t.colck_ld / aux_rows) * sizeof(int2)));
    t.colck = static_cast<int2 *>(c->colck.p);
    t.colck_aux = static_cast<int2 *>(c->colaux.p);
    const int2 *rowck = t.ckpt, *colck = t.colck, *colaux = t.colck_aux;
    const long long colck_ld = t.colck_ld, colaux_ld = t.colck_ld / aux_rows;

    RC(c->tb.ensure((size_t)ntiles * tile_bytes));
    RC(c->tbbnd.ensure((size_t)ntiles * 2 * (size_t)BT * sizeof(int2)));
    std::vector<FillTask> tasks;                    // [0]: the forward fill; then every tile
    tasks.reserve((size_t)ntiles + 1);
    tasks.push_back(t);
    std::vector<const void *> table((size_t)nI * nJw, nullptr);
    long long tickets = 0;
    for (int ti = 0; ti < nI; ++ti)
        for (int tj = 0; tj < nJ; ++tj) {
            FillTask u{};
            const long long r0 = (long long)ti * BT, c0 = (long long)tj * BT;
            u.a = da + r0;
            u.b = db + c0;
            u.rows = (int32_t)std::min<long long>(BT, m - r0);
            u.ncols = (int32_t)std::min<long long>(BT, n - c0);
            u.strip_warps = tsw;
            u.nstrips = (u.rows + HS - 1) / HS;
            u.ticket0 = tickets;
            u.top = r0 == 0 ? nullptr : rowck + (size_t)(r0 / BT - 1) * n + c0;
            if (c0 > 0) {
                u.left = colck + (size_t)(c0 / BT - 1) * colck_ld + r0;
                u.left_aux = colaux + (size_t)(c0 / BT - 1) * colaux_ld + r0 / aux_rows;
                u.left_split = fwd.P16 ? 1 : 0;
            }
            const size_t k = tasks.size() - 1;
            u.nslot = std::min(u.nstrips, 2);
            u.bnd = static_cast<int2 *>(c->tbbnd.p) + k * 2 * (size_t)BT;
            u.row0 = (int32_t)r0;
            u.col0 = (int32_t)c0;
            u.tb = static_cast<char *>(c->tb.p) + k * tile_bytes;
            u.tb_ld = BT;
            tickets += u.nstrips;
            tasks.push_back(u);
            table[(size_t)ti * nJw + (size_t)(tj - J0 - ti)] = u.tb;
        }
    const long long all = (long long)t.nstrips + tickets;
    RC(c->tasks.ensure(tasks.size() * sizeof(FillTask)));
    RC(c->prog.ensure((size_t)all * sizeof(int)));
    RC(c->cand.ensure((size_t)all * sizeof(int4)));
    RC(c->ticket.ensure(2 * sizeof(unsigned long long)));
    RC(c->result.ensure(sizeof(int4)));
    RC(c->walk.ensure(sizeof(WalkState)));
    RC(c->runs.ensure((size_t)(m + n + 2) * sizeof(int2)));
    RC(c->misc.ensure(table.size() * sizeof(void *)));
    // host staging: the tasks and the tile table go down in two copies
    const size_t task_bytes = tasks.size() * sizeof(FillTask);
    const size_t tab_off = (task_bytes + 15) / 16 * 16;
    RC(c->stage.ensure(tab_off + table.size() * sizeof(void *)));
    std::memcpy(c->stage.p, tasks.data(), task_bytes);
    std::memcpy(static_cast<char *>(c->stage.p) + tab_off, table.data(), table.size() * sizeof(void *));
    CU(cudaMemcpyAsync(c->tasks.p, c->stage.p, task_bytes, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->misc.p, static_cast<char *>(c->stage.p) + tab_off, table.size() * sizeof(void *),
                       cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemsetAsync(c->prog.p, 0, (size_t)all * sizeof(int), c->stream));
    CU(cudaMemsetAsync(c->ticket.p, 0, 2 * sizeof(unsigned long long), c->stream));

    const FillTask *dtasks = static_cast<const FillTask *>(c->tasks.p);
    FillLaunch L{};
    L.tasks = dtasks;
    L.scorings = static_cast<const DevScoring *>(c->scorings.p);
    L.ticket = static_cast<unsigned long long *>(c->ticket.p);
    L.prog = static_cast<int *>(c->prog.p);
    L.cand = static_cast<int4 *>(c->cand.p);
    L.err = static_cast<int *>(c->err.p);
    L.total = t.nstrips;
    L.spin_limit = c->spin_limit;
    L.ntasks = 1;
    RC(launch_fill(c, fwd, kModeScoreCk, fold, L, ds.K, t.nstrips));
    reduce_candidates_kernel<<<1, 32, 0, c->stream>>>(dtasks, 1, static_cast<const int4 *>(c->cand.p),
                                                       static_cast<const DevScoring *>(c->scorings.p),
                                                       static_cast<int4 *>(c->result.p));
    CU(cudaGetLastError());
    ++c->launches;
    FillLaunch Lt = L;                              // the tiles: their own tickets and progress
    Lt.tasks = dtasks + 1;
    Lt.ticket = static_cast<unsigned long long *>(c->ticket.p) + 1;
    Lt.prog = static_cast<int *>(c->prog.p) + t.nstrips;
    Lt.cand = static_cast<int4 *>(c->cand.p) + t.nstrips;
    Lt.total = tickets;
    Lt.ntasks = ntiles;
    RC(launch_fill(c, tbc, kModeTb, fold, Lt, ds.K, tickets));
    walk_start_kernel<<<1, 32, 0, c->stream>>>(static_cast<const int4 *>(c->result.p), ds.alg == kAlgLocal ? 1 : 0,
                                               static_cast<WalkState *>(c->walk.p));
    CU(cudaGetLastError());
    ++c->launches;
    RC(launch_walk(c, static_cast<const void *const *>(c->misc.p), 0, J0, nI, nJw, (int)BT, R));

    // everything back at once: end cell, walk state, error word, run records
    const size_t runs_off = 128;
    const size_t runs_bytes = (size_t)(m + n + 2) * sizeof(int2);
    RC(c->stage3.ensure(runs_off + runs_bytes));
    char *h = static_cast<char *>(c->stage3.p);
    CU(cudaMemcpyAsync(h, c->result.p, sizeof(int4), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(h + 16, c->err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(h + 32, c->walk.p, sizeof(WalkState), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(h + runs_off, c->runs.p, runs_bytes, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    int4 res;
    int e;
    WalkState w;
    std::memcpy(&res, h, sizeof(int4));
    std::memcpy(&e, h + 16, sizeof(int));
    std::memcpy(&w, h + 32, sizeof(WalkState));
    RC(map_kernel_error(e));
    if (ds.alg == kAlgLocal && res.x <= 0) return empty_alignment(out);
    if (res.y == 0 || res.z == 0) return border_alignment(ds.alg, res.x, res.y, res.z, out);
    if (w.done != 1 || w.nruns < 0 || w.nruns > m + n) return SW_ECUDA;   // every tile is in the table
    return finish_alignment(ds.alg, res.x, res.y, res.z, w, reinterpret_cast<const int2 *>(h + runs_off), out);
}

}  // namespace

extern "C" int sw_align(sw_ctx *c, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                        const sw_scoring *sc, sw_alignment *out) {
    if (!c || !out) return SW_EINVAL;
    DevScoring ds;
    RC(check_scoring(sc, &ds));
    if (m < 0 || n < 0 || (m > 0 && !a) || (n > 0 && !b)) return SW_EINVAL;
    if (m > SW_MAX_LEN || n > SW_MAX_LEN) return SW_ERANGE;
    if (!score_range_ok(sc, m, n)) return SW_ERANGE;
    if (m == 0 || n == 0) {
        if (ds.alg == kAlgLocal) return empty_alignment(out);
        int cs = kNoScore, ci = 0x7fffffff, cj = 0x7fffffff;
        border_end_candidates(ds.alg, m, n, ds.go, ds.ge, &cs, &ci, &cj);
        return border_alignment(ds.alg, cs, ci, cj, out);
    }
    DeviceGuard g(c->device);
    const uint8_t *da, *db;
    RC(stage_seq(c, a, m, c->seq_a, &da));
    RC(stage_seq(c, b, n, c->seq_b, &db));
    RC(reset_err(c));
    RC(validate_codes(c, da, m, ds.K));
    RC(validate_codes(c, db, n, ds.K));
    RC(upload_scorings(c, {ds}));
    const bool fold = fold_open(ds);
    if (c->one_round != 0 && std::max(m, n) <= kOneRoundSide) {
        // one round: forced (one_round > 0), or by default where every tile fits one wave on the SMs
        FillConfig f1{8, 4}, t1{8, 4};
        int sw1 = 4, tsw1 = 4;
        const long long bt = small_pair_tile(c, m, n, ds, &f1, &t1, &sw1, &tsw1);
        const long long tiles = bt > 0 ? ((m + bt - 1) / bt) * ((n + bt - 1) / bt) : 0;
        if (bt > 0 && (c->one_round > 0 || tiles <= c->nsm))
            return align_one_round(c, da, m, db, n, ds, fold, f1, t1, sw1, tsw1, bt, out);
    }

    // ---- tile side: both checkpoint sets within the budget
    // tiles are BT x BT; BT is a multiple of both fills' strip heights, so
    // checkpoint rows fall on forward-strip bottoms and tiles hold whole
    // traceback strips
    const FillConfig fwd = pair_fill_config_for(c, m, ds);
    const int sw = pair_strip_warps(c, fwd, m);
    const int HC = sw * 32 * fwd.R;
    // the traceback tiles continue the forward fill's staircase checkpoint columns lane by
    // lane, so both fills must give each lane the same rows (R)
    FillConfig tbc = (c->tbc.R == fwd.R && fwd.alg == kAlgLocal) ? c->tbc : FillConfig{fwd.R, 4};
    tbc.P16 = 0;                                  // traceback bits come from the int32 fill
    tbc.alg = fwd.alg;
    // the packed forward fill stores its checkpoint columns with two positions per lane and
    // one auxiliary record per half-group of R/2 rows
    const int aux_rows = fwd.P16 ? fwd.R / 2 : fwd.R;
    const int HT = fill_rows_per_strip(tbc);
    const int HC2 = 4 * 32 * fwd.R;                // strip height of a coarse tile's refill (int32, 4 warps)
    const long long BL = std::lcm((long long)HC, (long long)HT);
    const long long BL2 = std::lcm((long long)HC2, (long long)HT);
    auto ck_bytes = [&](long long bt) {
        return (size_t)((m / bt) * n + (n / bt) * m) * sizeof(int2);
    };
    // BT1: the forward fill's checkpoint spacing; BT2: the traceback tiles' side.  One level
    // (BT1 = BT2) while the checkpoints fit the budget at a tile side up to kMaxOneLevelBT;
    // else two: coarse checkpoints every BT1 (half the budget), and each coarse tile the
    // path enters is filled again from them with fine checkpoints every BT2 (the other half)
    // pairs up to kSmallPairSide take tiles from 512 (a traceback tile is one strip of its
    // fill, half the chain of a 1,024 tile; 2 kbp: 0.22 -> ~0.11 ms of tile recompute)
    const long long min_side = std::max(m, n) <= kSmallPairSide ? 512 : 1024;
    long long BT1 = BL * ((min_side + BL - 1) / BL);
    while (ck_bytes(BT1) > c->ckpt_budget && BT1 < (1LL << 30)) BT1 *= 2;
    long long BT2 = BT1;
    if (c->two_level_bt1 > 0) {                     // SWGB_TWO_LEVEL: the sides, checked below
        BT1 = c->two_level_bt1;
        BT2 = c->two_level_bt2;
    } else if (BT1 > kMaxOneLevelBT) {
        // level-1 checkpoints ~ 16 m n / BT1 bytes, a refill's ~ 16 BT1^2 / BT2: each within half
        // the budget, BT2 doubled until the second fits
        for (BT2 = BL2 * ((1024 + BL2 - 1) / BL2);; BT2 *= 2) {
            const long long step = std::lcm(BT2, BL);
            BT1 = step * std::max<long long>(2, (4 * BT2 + step - 1) / step);
            while (ck_bytes(BT1) > c->ckpt_budget / 2 && BT1 < (1LL << 30)) BT1 += step;
            if ((double)2 * (double)(BT1 / BT2) * (double)BT1 * sizeof(int2) <= (double)(c->ckpt_budget / 2) ||
                BT2 >= kMaxOneLevelBT)
                break;
        }
    }
    const bool two = BT2 != BT1;
    // checkpoint columns are stored at chunk ends: the sides must be multiples of the chunk
    if (BT1 % HC != 0 || BT2 % HT != 0 || BT1 % kCH != 0 || BT2 % kCH != 0 || BT1 % BT2 != 0 ||
        (two && BT2 % HC2 != 0) || BT1 > (1LL << 30))
        return SW_EINVAL;
    const long long BT = BT2;
    const long long nrowck = std::max<long long>(1, m / BT1), ncolck = std::max<long long>(1, n / BT1);

    // ---- 1. forward fill with row and column checkpoints
    FillTask t{};
    t.a = da; t.b = db;
    t.rows = (int32_t)m; t.ncols = (int32_t)n;
    t.strip_warps = sw;
    t.nstrips = (int32_t)((m + HC - 1) / HC);
    t.scoring = 0; t.ticket0 = 0; t.top = nullptr; t.left = nullptr; t.left_aux = nullptr; t.row0 = 0;
    t.nslot = std::min(t.nstrips, 4);
    RC(c->bnd.ensure((size_t)t.nslot * (size_t)n * sizeof(int2)));
    t.bnd = static_cast<int2 *>(c->bnd.p);
    t.ckpt_every = (int32_t)(BT1 / HC);
    RC(c->ckpt.ensure((size_t)nrowck * (size_t)n * sizeof(int2)));
    t.ckpt = static_cast<int2 *>(c->ckpt.p);
    t.colck_every = (int32_t)BT1;
    t.colck_ld = (long long)t.nstrips * HC;     // rows padded to whole strips (the padding is written)
    RC(c->colck.ensure((size_t)ncolck * (size_t)t.colck_ld * sizeof(int2)));
    RC(c->colaux.ensure((size_t)ncolck * (size_t)(t.colck_ld / aux_rows) * sizeof(int2)));
    t.colck = static_cast<int2 *>(c->colck.p);
    t.colck_aux = static_cast<int2 *>(c->colaux.p);
    RC(run_fill(c, fwd, kModeScoreCk, fold, {t}, t.nstrips, ds.K));
    RC(c->result.ensure(sizeof(int4)));
    reduce_candidates_kernel<<<1, 32, 0, c->stream>>>(static_cast<const FillTask *>(c->tasks.p), 1,
                                                       static_cast<const int4 *>(c->cand.p),
                                                       static_cast<const DevScoring *>(c->scorings.p),
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
    if (ds.alg == kAlgLocal && res.x <= 0) return empty_alignment(out);
    const int ie = res.y, je = res.z;
    if (ie == 0 || je == 0) return border_alignment(ds.alg, res.x, ie, je, out);   // other algorithms only

    // ---- 2. walk state
    RC(c->walk.ensure(sizeof(WalkState)));
    RC(c->runs.ensure((size_t)(ie + je + 2) * sizeof(int2)));
    WalkState w{ie, je, 0, 0, 0, -1, 0};
    // the band's traceback bits within the budget (at most three tiles a row)
    const size_t tile_bytes = (size_t)(BT / tbc.R) * (size_t)BT * (size_t)tb_word_bytes(tbc.R);
    // tile rows per band: two or three tiles a row, about one tile per SM (measured at 200 kbp: a
    // band as deep as the SM count, 228 tiles in one round, took 1.18 ms against 1.00 ms for two
    // rounds of one tile per SM)
    int band = c->tb_band > 0 ? std::min(c->tb_band, 800) : std::max(kMinBandDepth, c->nsm / 2);
    band = (int)std::max<long long>(1, std::min<long long>(band, (long long)(c->tb_budget / (3 * tile_bytes))));
    const int tsw = c->tb_strip_warps > 0 ? std::min(c->tb_strip_warps, tbc.W) : tbc.W;
    const int HS = tsw * 32 * tbc.R;                     // rows per traceback strip
    const size_t table_cap = (size_t)(band + 1) * kBandWidth;
    // staging: the rounds' tile tables, then the walk's start (its own slot, so that no
    // synchronisation is needed before the first table is written)
    const size_t w_off = (table_cap * sizeof(void *) + 15) / 16 * 16;
    RC(c->stage2.ensure(w_off + sizeof(WalkState)));
    std::memcpy(static_cast<char *>(c->stage2.p) + w_off, &w, sizeof(w));
    CU(cudaMemcpyAsync(c->walk.p, static_cast<char *>(c->stage2.p) + w_off, sizeof(w), cudaMemcpyHostToDevice,
                       c->stream));
    // short paths: the run records come back with every round's walk state, which saves the
    // copy (and its synchronisation) after the last round
    const size_t runs_max = (size_t)(ie + je + 2) * sizeof(int2);
    const bool runs_each_round = runs_max <= kRunsEachRoundBytes;
    if (runs_each_round) RC(c->stage3.ensure(128 + runs_max));

    // ---- 3. rounds: recompute a band of tiles, walk through it
    const int R = tbc.R;
    const int maxtiles = 3 * band;
    RC(c->tb.ensure(tile_bytes * maxtiles));
    RC(c->tbbnd.ensure((size_t)maxtiles * 2 * (size_t)BT * sizeof(int2)));
    RC(c->misc.ensure(table_cap * sizeof(void *)));
    // level 1: the forward fill's checkpoints (every BT1); level 2 (two levels only): those of
    // the current coarse tile's refill (every BT2 inside it), over rows [R0c, Wi0) and
    // columns [C0c, Wj0), the part of the coarse tile above and left of where the walk entered
    const int2 *rowck = t.ckpt, *colck = t.colck, *colaux = t.colck_aux;
    const long long colck_ld = t.colck_ld, colaux_ld = t.colck_ld / aux_rows;
    long long CIc = -1, CJc = -1, R0c = 0, C0c = 0, Wi0 = m, Wj0 = n, ld2 = 0, N2 = 0;
    const int2 *rowck2 = nullptr, *colck2 = nullptr, *colaux2 = nullptr;

    // A band: the tiles of tile rows I0..I along the diagonal through the cell (wi, wj), ending
    // at that cell's tile row, in the buffers of slot s (0: the context's, 1: the look-ahead's).
    // A tile depends only on the checkpoints, never on the walk, so a band may be recomputed
    // ahead of the walk from a predicted cell; the walk stops at a tile missing from its table.
    struct Band {
        int slot = 0, I = 0, I0 = 0, nI = 0, nJ = 0, kd = 0;
        int Itop = 0;                     // the band's top tile row with tiles (rows above it: cut by the cap)
        std::vector<const void *> table;
        std::vector<FillTask> tasks;
        long long tickets = 0;
    };
    auto build_band = [&](long long wi, long long wj, int slot, Band &bd) {
        bd = Band{};
        bd.slot = slot;
        char *tbp = static_cast<char *>(slot ? c->tb_b.p : c->tb.p);
        int2 *bndp = static_cast<int2 *>(slot ? c->tbbnd_b.p : c->tbbnd.p);
        const int I = (int)((wi - 1) / BT), J = (int)((wj - 1) / BT);
        const int It0 = (int)(R0c / BT), Jt0 = (int)(C0c / BT);       // the region's first tile row, column
        const int I0 = std::max(It0, I - band + 1);
        // the walk's table keeps kBandWidth tile columns a row along the diagonal: row ti holds
        // columns [ti + kd, ti + kd + kBandWidth), which contain every tile chosen below
        const int nI = I - I0 + 1, nJ = kBandWidth, kd = J - I - (kBandWidth - 2);
        bd.I = I; bd.I0 = I0; bd.nI = nI; bd.nJ = nJ; bd.kd = kd;
        bd.table.assign((size_t)nI * nJ, nullptr);
        // tiles of each tile row: the columns that the diagonal through the cell crosses in that
        // row, widened by BT / kBandMarginDiv on each side (two tiles a row, a third where the
        // diagonal runs near a tile edge); a path that drifts further ends the round early
        const long long margin = BT / kBandMarginDiv;
        int rows = 0;
        for (int d = 0; d < band && I - d >= It0; ++d) {
            const int ti = I - d;
            // one tile per SM at most (a second wave would double the round's time); whole rows
            if (d > 0 && (int)bd.tasks.size() + kBandWidth - 2 > c->nsm) break;
            ++rows;
            const long long rlo = (long long)ti * BT, rhi = std::min<long long>((long long)(ti + 1) * BT, wi) - 1;
            const long long clo = (wj - 1) - ((wi - 1) - rlo) - margin;
            const long long chi = (wj - 1) - ((wi - 1) - rhi) + margin;
            const int wlo = ti + kd, whi = wlo + kBandWidth - 1;             // the table's window
            const int tlo = (int)std::min<long long>(J, std::max<long long>(std::max(Jt0, wlo), clo < 0 ? 0 : clo / BT));
            const int thi = (int)std::min<long long>(std::min(J, whi), std::max<long long>(tlo, chi < 0 ? 0 : chi / BT));
            for (int tj = tlo; tj <= thi; ++tj) {
                FillTask u{};
                const long long r0 = (long long)ti * BT, c0 = (long long)tj * BT;
                u.a = da + r0;
                u.b = db + c0;
                u.rows = (int32_t)std::min<long long>(BT, Wi0 - r0);
                u.ncols = (int32_t)std::min<long long>(BT, Wj0 - c0);
                u.strip_warps = tsw;
                u.nstrips = (u.rows + HS - 1) / HS;
                u.scoring = 0;
                u.ticket0 = bd.tickets;
                // the row above the tile and the column left of it: the matrix border, a
                // forward-fill checkpoint (on a coarse boundary) or a refill checkpoint
                if (r0 == 0) u.top = nullptr;
                else if (r0 % BT1 == 0) u.top = rowck + (size_t)(r0 / BT1 - 1) * n + c0;
                else u.top = rowck2 + (size_t)((r0 - R0c) / BT - 1) * N2 + (c0 - C0c);
                if (c0 == 0) {
                    u.left = nullptr; u.left_aux = nullptr;
                } else if (c0 % BT1 == 0) {
                    u.left = colck + (size_t)(c0 / BT1 - 1) * colck_ld + r0;
                    u.left_aux = colaux + (size_t)(c0 / BT1 - 1) * colaux_ld + r0 / aux_rows;
                    u.left_split = fwd.P16 ? 1 : 0;
                } else {
                    u.left = colck2 + (size_t)((c0 - C0c) / BT - 1) * ld2 + (r0 - R0c);
                    u.left_aux = colaux2 + (size_t)((c0 - C0c) / BT - 1) * (ld2 / aux_rows) + (r0 - R0c) / aux_rows;
                    u.left_split = fwd.P16 ? 1 : 0;
                }
                const size_t k = bd.tasks.size();
                u.nslot = std::min(u.nstrips, 2);
                u.bnd = bndp + k * 2 * (size_t)BT;
                u.ckpt_every = 0; u.ckpt = nullptr; u.colck = nullptr; u.colck_every = 0;
                u.row0 = (int32_t)r0;
                u.col0 = (int32_t)c0;
                u.tb = tbp + k * tile_bytes;
                u.tb_ld = BT;
                bd.tickets += u.nstrips;
                bd.tasks.push_back(u);
                bd.table[(size_t)(ti - I0) * nJ + (tj - (kd + I0) - (ti - I0))] = u.tb;
            }
        }
        bd.Itop = I - rows + 1;
    };
    const FillBufs main_bufs{&c->tasks, &c->prog, &c->cand, &c->ticket, &c->stage};
    const FillBufs side_bufs{&c->tasks_b, &c->prog_b, &c->cand_b, &c->ticket_b, &c->stage_b};
    // the look-ahead band (one level only: a refill changes the checkpoints under the bands)
    const bool ahead = c->lookahead && !two;
    if (ahead) {
        RC(c->tb_b.ensure(tile_bytes * maxtiles));
        RC(c->tbbnd_b.ensure((size_t)maxtiles * 2 * (size_t)BT * sizeof(int2)));
        RC(c->misc_b.ensure(table_cap * sizeof(void *)));
        if (!c->side) CU(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        if (!c->side_go) CU(cudaEventCreateWithFlags(&c->side_go, cudaEventDisableTiming));
        if (!c->side_done) CU(cudaEventCreateWithFlags(&c->side_done, cudaEventDisableTiming));
    }
    Band cur, spec;
    bool have_spec = false;
    // whatever happens below, the look-ahead fill is finished before this call returns
    struct SideSync {
        sw_ctx *c;
        bool *on;
        ~SideSync() { if (*on && c->side) cudaStreamSynchronize(c->side); }
    } side_sync{c, &have_spec};
    int prev_i = -1, prev_j = -1, prev_state = -1;
    while (true) {
        if (two && ((w.i - 1) / BT1 != CIc || (w.j - 1) / BT1 != CJc)) {
            CIc = (w.i - 1) / BT1;
            CJc = (w.j - 1) / BT1;
            R0c = CIc * BT1; C0c = CJc * BT1;
            Wi0 = w.i; Wj0 = w.j;
            RC(refill_coarse_tile(c, da, db, n, ds, fwd, fold, aux_rows, rowck, colck, colaux, colck_ld, colaux_ld,
                                  CIc, CJc, R0c, C0c, Wi0, Wj0, BT2, &rowck2, &colck2, &colaux2, &ld2, &N2));
        }
        const int Iw = (w.i - 1) / (int)BT, Jw = (w.j - 1) / (int)BT;
        bool use_spec = false;
        if (have_spec) {
            // the look-ahead band serves if it holds the tile the walk is in
            const int tj = Jw - (spec.kd + spec.I0) - (Iw - spec.I0);
            use_spec = Iw <= spec.I && Iw >= spec.I0 && tj >= 0 && tj < spec.nJ &&
                       spec.table[(size_t)(Iw - spec.I0) * spec.nJ + tj] != nullptr;
            if (use_spec) {
                CU(cudaStreamWaitEvent(c->stream, c->side_done, 0));
                cur = std::move(spec);
            } else {
                CU(cudaStreamSynchronize(c->side));   // its buffers may be needed again
            }
            have_spec = false;
        }
        if (!use_spec) {
            build_band(w.i, w.j, 0, cur);
            RC(run_fill_with(c, main_bufs, c->stream, tbc, kModeTb, fold, cur.tasks, cur.tickets, ds.K));
        }
        const size_t tbytes = cur.table.size() * sizeof(void *);
        if (tbytes > c->stage2.cap) return SW_EINVAL;
        std::memcpy(c->stage2.p, cur.table.data(), tbytes);
        void *dtab = cur.slot ? c->misc_b.p : c->misc.p;
        CU(cudaMemcpyAsync(dtab, c->stage2.p, tbytes, cudaMemcpyHostToDevice, c->stream));
        if (ahead) CU(cudaEventRecord(c->side_go, c->stream));   // the band's tiles are done
        RC(launch_walk(c, static_cast<const void *const *>(dtab), cur.I0, cur.kd + cur.I0, cur.nI, cur.nJ,
                       (int)BT, R));
        // the next band up the same diagonal, recomputed on the side stream while the walk runs
        if (ahead && cur.Itop > 0) {
            const long long pi = (long long)cur.Itop * BT, pj = (long long)w.j - ((long long)w.i - pi);
            if (pj >= 1) {
                build_band(pi, pj, 1 - cur.slot, spec);
                if (!spec.tasks.empty()) {
                    CU(cudaStreamWaitEvent(c->side, c->side_go, 0));
                    RC(run_fill_with(c, spec.slot ? side_bufs : main_bufs, c->side, tbc, kModeTb, fold, spec.tasks,
                                     spec.tickets, ds.K));
                    CU(cudaEventRecord(c->side_done, c->side));
                    have_spec = true;
                }
            }
        }
        CU(cudaMemcpyAsync(c->stage3.p, c->walk.p, sizeof(WalkState), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaMemcpyAsync(static_cast<char *>(c->stage3.p) + 64, c->err.p, sizeof(int),
                           cudaMemcpyDeviceToHost, c->stream));
        if (runs_each_round)
            CU(cudaMemcpyAsync(static_cast<char *>(c->stage3.p) + 128, c->runs.p, runs_max, cudaMemcpyDeviceToHost,
                               c->stream));
        CU(cudaStreamSynchronize(c->stream));
        std::memcpy(&w, c->stage3.p, sizeof(w));
        std::memcpy(&e, static_cast<char *>(c->stage3.p) + 64, sizeof(int));
        RC(map_kernel_error(e));
        if (w.done != 0) break;
        if (w.i == prev_i && w.j == prev_j && w.state == prev_state) return SW_ECUDA;   // no progress
        prev_i = w.i; prev_j = w.j; prev_state = w.state;
    }
    if (have_spec) {
        CU(cudaStreamSynchronize(c->side));
        have_spec = false;
    }
    if (w.done != 1) return SW_ECUDA;     // the walk must end at a zero cell or the border
    if (w.nruns < 0 || (size_t)w.nruns * sizeof(int2) > runs_max) return SW_ECUDA;

    // ---- 4. CIGAR text from the run records
    if (runs_each_round)
        return finish_alignment(ds.alg, res.x, ie, je, w,
                                reinterpret_cast<const int2 *>(static_cast<char *>(c->stage3.p) + 128), out);
    std::vector<int2> runs((size_t)w.nruns);
    if (w.nruns > 0) {
        CU(cudaMemcpy(runs.data(), c->runs.p, (size_t)w.nruns * sizeof(int2), cudaMemcpyDeviceToHost));
    }
    return finish_alignment(ds.alg, res.x, ie, je, w, runs.data(), out);
}
