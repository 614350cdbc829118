// sw_ctx.h -- internal host-side declarations of libswgb: the context,
// device/pinned buffers and the helpers the ABI translation units share.
#pragma once
#include "sw.h"
#include "sw_device.cuh"
#include "wavefront.cuh"

#include <cstddef>
#include <utility>
#include <vector>

namespace swgb {

// Grow-only device allocation.
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    int ensure(size_t bytes);
    void release();
    ~DevBuf() { release(); }
};

// Grow-only pinned host allocation (staging for asynchronous copies).
struct HostBuf {
    void *p = nullptr;
    size_t cap = 0;
    int ensure(size_t bytes);
    void release();
    ~HostBuf() { release(); }
};

struct DeviceGuard {
    int prev = 0, now = 0;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};

// Tile shape of the wavefront fill: R rows per lane, W compute warps per
// block; S fixes the compute warps per strip of a single-pair fill (0 = chosen
// from the pair's length); B caps the resident blocks per SM (0 = as many as
// fit).
struct FillConfig {
    int R;
    int W;
    int S = 0;
    int B = 0;
    int P16 = 0;   // packed 16-bit fill (wavefront16.cuh) instead of the int32 one
    int alg = 0;   // not kAlgLocal: the int32 fill without the zero floor (fill_variants.cu)
    int left = 0;  // packed fill whose tasks may start right of its own checkpoint column
};

// Device time per kernel kind (sw_ctx_timing): event pairs recorded around
// launches, folded into totals when read or when the pool is full.
struct KernelTimer {
    static constexpr int kPairs = 4096;
    bool on = false;
    std::vector<cudaEvent_t> ev;      // 2 * kPairs, created on first use
    std::vector<int> kind;            // kind of each recorded pair
    double ms[SW_KT_COUNT] = {};
    long long n[SW_KT_COUNT] = {};
    void destroy();
    ~KernelTimer() { destroy(); }
};

}  // namespace swgb

struct sw_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int nsm = 0;
    long long spin_limit = 0;
    long long launches = 0;           // kernels launched by this context
    swgb::FillConfig fwd{8, 4, 0, 2}; // score / forward pass (when fwd_auto is false)
    bool fwd_auto = true;             // choose R per pair (pair_fill_config)
    swgb::FillConfig tbc{8, 4};       // traceback recompute
    swgb::FillConfig bat{8, 4};       // batches of pairs (unless autotuned)
    bool prof32 = true;               // int32 query profiles where they fit (small alphabets)
    bool p16 = true;                  // packed 16-bit pair fill where it is exact (p16_fits)
    int tb_band = 0;                  // tile rows per traceback band (0 = about one tile per SM)
    int one_round = -1;               // sw_align of small pairs in one round: 1 forced, 0 off, -1 where the tiles fit one wave
    long long two_level_bt1 = 0;      // sw_align: forced coarse / fine checkpoint sides (0 = by budget)
    long long two_level_bt2 = 0;
    int tb_strip_warps = 0;           // compute warps per traceback strip (0 = all)
    size_t ckpt_budget = 0;           // bytes of checkpoint rows kept by sw_align
    size_t tb_budget = 0;             // bytes of traceback bits per row group
    swgb::DevBuf seq_a, seq_b, tasks, scorings, ticket, prog, cand, result, err, bnd, ckpt, colck, colaux, tb,
        ckpt2, colck2, colaux2,
        tbbnd, runs, walk, misc, dbscratch, dbslots, dbovf, dbjob, dbscores, topk;
    swgb::HostBuf stage, stage2, stage3;
    // sw_align's look-ahead band: a second set of traceback-fill buffers and a stream of their
    // own, so that the next band's tiles are recomputed while the walk goes through the current one
    swgb::DevBuf tb_b, tbbnd_b, tasks_b, prog_b, cand_b, ticket_b, misc_b;
    swgb::HostBuf stage_b;
    cudaStream_t side = nullptr;
    cudaEvent_t side_go = nullptr, side_done = nullptr;
    bool lookahead = true;
    std::vector<std::pair<long long, swgb::FillConfig>> batch_tune;   // autotuned tile shape per size class
    swgb::KernelTimer timer;
};

namespace swgb {

bool is_device_ptr(const void *p);
int check_scoring(const sw_scoring *sc, DevScoring *out);
int max_pos_score(const sw_scoring *sc);
int stage_seq(sw_ctx *c, const uint8_t *p, int64_t len, DevBuf &buf, const uint8_t **dptr);
int map_kernel_error(int e);
int fill_rows_per_strip(const FillConfig &cfg);
int pair_strip_warps(const sw_ctx *c, const FillConfig &cfg, int64_t rows);
FillConfig pair_fill_config(const sw_ctx *c, int64_t rows);
FillConfig pair_fill_config_for(const sw_ctx *c, int64_t rows, const DevScoring &s);   // picks P16 where exact
bool p16_fits(const DevScoring &s, int R);
int launch_fill16(sw_ctx *c, const FillConfig &cfg, int mode, const FillLaunch &L, int K, long long tickets);
// the global, semi-global and overlap algorithms: 8 or 16 rows a lane, four compute warps
FillConfig variant_fill_config(const sw_ctx *c, int64_t rows);
int launch_fill_variant(sw_ctx *c, const FillConfig &cfg, int mode, bool fold, const FillLaunch &L, int K,
                        long long tickets);
// the largest |score| the int32 fill keys without overflow, for a pair of these lengths
bool score_range_ok(const sw_scoring *sc, int64_t m, int64_t n);
int tb_word_bytes(int R);
bool fold_open(const DevScoring &s);   // S + open fits the int8 profile
int launch_fill(sw_ctx *c, const FillConfig &cfg, int mode, bool fold, const FillLaunch &L, int K,
                long long tickets);
// the buffers a fill's launch uses: its task table, progress counters, candidates, ticket
// counter and host staging (run_fill: the context's)
struct FillBufs {
    DevBuf *tasks, *prog, *cand, *ticket;
    HostBuf *stage;
};
int run_fill_with(sw_ctx *c, const FillBufs &b, cudaStream_t st, const FillConfig &cfg, int mode, bool fold,
                  const std::vector<FillTask> &tasks, long long tickets, int K);
int run_fill(sw_ctx *c, const FillConfig &cfg, int mode, bool fold, const std::vector<FillTask> &tasks,
             long long tickets, int K);
int upload_scorings(sw_ctx *c, const std::vector<DevScoring> &s);
int kt_begin(sw_ctx *c, int kind);         // -1 when not timing; else the pair to close with kt_end
void kt_end(sw_ctx *c, int pair);
int reset_err(sw_ctx *c);
int validate_codes(sw_ctx *c, const uint8_t *d, int64_t len, int K);
int read_err(sw_ctx *c, int *e);
// database search pieces shared with the serving loop
struct DbJob;
struct DbView;
int db_score_all(sw_ctx *c, const sw_db *db, const uint8_t *dq, int64_t m, const DevScoring &ds,
                 int32_t *dscores);
int db_rescore(sw_ctx *c, const sw_db *db, const uint8_t *dq, int64_t m, const DevScoring &ds,
               const std::vector<int32_t> &flagged, int32_t *dscores);
int db_topk(sw_ctx *c, const int32_t *dscores, int64_t nseq, int k, int2 *dout);
int db_shape(int K, int m);                // tile shape (index) for a query of m residues
int db_shape_warps(int shape);
int db_shape_rows(int shape);              // query rows per pass
int db_resident_blocks_shape(sw_ctx *c, int shape, int K, int m, int *out);
// Buffers of a database launch: boundary-row scratch, slot pool, scoring table and error word.
// Default: the context's; launches that may run while other calls use the context (the
// server's steps on their own streams) bring their own.
struct DbBufs {
    DevBuf *rows, *slots;
    const DevScoring *scorings;
    int *err;
};
int db_launch_shape(sw_ctx *c, int shape, const DbJob *jobs, int njobs, int nblocks, const DbView &D, int K, int m,
                    const DbBufs *bufs = nullptr);
// the scratch bytes db_launch_shape ensures for that launch (subjects up to maxlen residues)
int db_scratch_shape(sw_ctx *c, int shape, int K, int m, int maxlen, size_t *row_bytes, size_t *slot_bytes);
int db_resident_blocks(sw_ctx *c, int K, int m, int *out);
int db_warps_per_block(int K, int m);
int db_rows_per_pass(int K, int m);      // query rows per pass of the packed kernel for this launch shape
int db_launch(sw_ctx *c, const DbJob *jobs, int njobs, int nblocks, const DbView &D, int K, int m);
int db_view(const sw_db *db, DbView *v, int64_t *nseq, int32_t *max_code, int *device);
int db_chunk_maxlen(const sw_db *db, int32_t pair0, int32_t pair1);
int64_t db_total_residues(const sw_db *db);

}  // namespace swgb
