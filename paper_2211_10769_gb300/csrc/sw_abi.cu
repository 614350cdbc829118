// sw_abi.cu -- host runtime behind the C ABI declared in include/sw.h:
// argument checking, device scratch management, staging of host inputs,
// launch of the fill / reduction / traceback kernels and assembly of the
// results.  Every arithmetic step of the alignment runs in the kernels;
// the host only moves data and formats the CIGAR text.
#include "sw.h"
#include "sw_ctx.h"
#include "wavefront.cuh"
#include "aux_kernels.cuh"

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace swgb;

// ------------------------------------------------------------------ helpers

int swgb::DevBuf::ensure(size_t bytes) {
    if (bytes <= cap) return SW_OK;
    release();
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        return SW_ENOMEM;
    }
    cap = bytes;
    return SW_OK;
}

void swgb::DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
}

int swgb::HostBuf::ensure(size_t bytes) {
    if (bytes <= cap) return SW_OK;
    release();
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        return SW_ENOMEM;
    }
    cap = bytes;
    return SW_OK;
}

void swgb::HostBuf::release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
}

swgb::DeviceGuard::DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    now = dev;
}

swgb::DeviceGuard::~DeviceGuard() {
    if (prev != now) cudaSetDevice(prev);
}

bool swgb::is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int swgb::check_scoring(const sw_scoring *sc, DevScoring *out) {
    if (!sc || !sc->matrix) return SW_EINVAL;
    if (sc->alphabet < 1 || sc->alphabet > kMaxAlphabet) return SW_EINVAL;
    if (sc->gap_extend < 0 || sc->gap_open < sc->gap_extend || sc->gap_open > 1000000) return SW_EINVAL;
    if (sc->algorithm < SW_ALG_LOCAL || sc->algorithm > SW_ALG_OVERLAP) return SW_EINVAL;
    if (out) {
        std::memset(out, 0, sizeof(*out));
        const int K = sc->alphabet;
        std::memcpy(out->mat, sc->matrix, (size_t)K * K);
        out->K = K;
        out->go = sc->gap_open;
        out->ge = sc->gap_extend;
        out->alg = sc->algorithm;
    }
    return SW_OK;
}

int swgb::max_pos_score(const sw_scoring *sc) {
    int mx = 0;
    for (int k = 0; k < sc->alphabet * sc->alphabet; ++k) mx = std::max(mx, (int)sc->matrix[k]);
    return mx;
}

int swgb::stage_seq(sw_ctx *c, const uint8_t *p, int64_t len, DevBuf &buf, const uint8_t **dptr) {
    if (len == 0) { *dptr = nullptr; return SW_OK; }
    if (is_device_ptr(p)) { *dptr = p; return SW_OK; }
    int rc = buf.ensure((size_t)len + 16);
    if (rc) return rc;
    if (cudaMemcpyAsync(buf.p, p, (size_t)len, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return SW_ECUDA;
    *dptr = static_cast<const uint8_t *>(buf.p);
    return SW_OK;
}

int swgb::map_kernel_error(int e) {
    switch (e) {
        case 0: return SW_OK;
        case kErrBadCode: return SW_EINVAL;
        case kErrTimeout: return SW_ETIMEOUT;
        case kErrOverflow: return SW_ERANGE;
        default: return SW_ECUDA;
    }
}

#define CU(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; } } while (0)
#define RC(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)

// ------------------------------------------------------------- fill launches

namespace {

// shared memory of an int32 query profile, at most (so that two blocks still fit an SM)
constexpr size_t kProf32MaxBytes = 64 * 1024;

template <int R, int W, int MODE, int PK>
int launch_fill_cfg(sw_ctx *c, const FillLaunch &L, int K, long long tickets, int max_blocks) {
    auto kern = wavefront_kernel<R, W, MODE, PK>;
    constexpr int HC = W * 32 * R;
    constexpr size_t PB = PK == kProf32 ? 4 : 1;
    const size_t smem = (size_t)(K + 1) * HC * PB;
    static int attr_set[64] = {0};
    if (c->device < 64 && !attr_set[c->device]) {
        const size_t cap = PK == kProf32 ? kProf32MaxBytes : (size_t)(kMaxAlphabet + 1) * HC;
        CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
        attr_set[c->device] = 1;
    }
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (W + 2) * 32, smem));
    if (occ < 1) return SW_ECUDA;
    if (max_blocks > 0) occ = std::min(occ, max_blocks);
    const long long grid = std::min<long long>(tickets, (long long)occ * c->nsm);
    const int kp = kt_begin(c, MODE == kModeTb ? SW_KT_FILL_TB : SW_KT_FILL);
    kern<<<(unsigned)grid, (W + 2) * 32, smem, c->stream>>>(L);
    kt_end(c, kp);
    CU(cudaGetLastError());
    ++c->launches;
    return SW_OK;
}

template <int R, int W, int MODE>
int launch_fill_pk(sw_ctx *c, int pk, const FillLaunch &L, int K, long long tickets, int B) {
    switch (pk) {
        case kProf8: return launch_fill_cfg<R, W, MODE, kProf8>(c, L, K, tickets, B);
        case kProf8Fold: return launch_fill_cfg<R, W, MODE, kProf8Fold>(c, L, K, tickets, B);
        default: return launch_fill_cfg<R, W, MODE, kProf32>(c, L, K, tickets, B);
    }
}

template <int R, int W>
int launch_fill_rw(sw_ctx *c, int mode, bool fold, const FillLaunch &L, int K, long long tickets, int B) {
    // int32 profile when it is small (DNA-like alphabets), else int8 (+ open when it fits)
    const bool p32 = c->prof32 && (size_t)(K + 1) * (size_t)(W * 32 * R) * 4 <= kProf32MaxBytes;
    const int pk = p32 ? kProf32 : (fold ? kProf8Fold : kProf8);
    switch (mode) {
        case kModeScore: return launch_fill_pk<R, W, kModeScore>(c, pk, L, K, tickets, B);
        case kModeScoreCk: return launch_fill_pk<R, W, kModeScoreCk>(c, pk, L, K, tickets, B);
        case kModeTb: return launch_fill_pk<R, W, kModeTb>(c, pk, L, K, tickets, B);
        default: return SW_EINVAL;
    }
}

}  // namespace

// ------------------------------------------------------------- kernel timing

void swgb::KernelTimer::destroy() {
    for (cudaEvent_t e : ev) if (e) cudaEventDestroy(e);
    ev.clear();
    kind.clear();
}

namespace {

// Adds the recorded pairs to the totals; waits for the last recorded event.
int kt_fold(sw_ctx *c) {
    KernelTimer &T = c->timer;
    const size_t np = T.kind.size();
    if (np == 0) return SW_OK;
    CU(cudaEventSynchronize(T.ev[2 * (np - 1) + 1]));
    for (size_t k = 0; k < np; ++k) {
        float ms = 0;
        CU(cudaEventElapsedTime(&ms, T.ev[2 * k], T.ev[2 * k + 1]));
        T.ms[T.kind[k]] += ms;
        T.n[T.kind[k]] += 1;
    }
    T.kind.clear();
    return SW_OK;
}

}  // namespace

int swgb::kt_begin(sw_ctx *c, int kind) {
    KernelTimer &T = c->timer;
    if (!T.on) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess) { cudaGetLastError(); return -1; }
    if (cs != cudaStreamCaptureStatusNone) return -1;
    if (T.ev.empty()) {
        T.ev.assign(2 * KernelTimer::kPairs, nullptr);
        for (cudaEvent_t &e : T.ev)
            if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); T.destroy(); T.on = false; return -1; }
    }
    if ((int)T.kind.size() == KernelTimer::kPairs && kt_fold(c) != SW_OK) return -1;
    const int p = (int)T.kind.size();
    if (cudaEventRecord(T.ev[2 * p], c->stream) != cudaSuccess) { cudaGetLastError(); return -1; }
    T.kind.push_back(kind);
    return p;
}

void swgb::kt_end(sw_ctx *c, int p) {
    if (p < 0) return;
    if (cudaEventRecord(c->timer.ev[2 * p + 1], c->stream) != cudaSuccess) cudaGetLastError();
}

// ------------------------------------------------------------- tile shapes

int swgb::fill_rows_per_strip(const FillConfig &cfg) { return cfg.W * 32 * cfg.R; }

int swgb::tb_word_bytes(int R) { return R <= 4 ? 2 : (R <= 8 ? 4 : 8); }

// Tile shape of a single-pair fill of `rows` rows.  A pair's strips form one
// chain (each waits on the bottom row of the one above), so the chain runs
// at the pace of its slowest strip, and a strip that shares an SM with
// another runs at about half its pace.  Four compute warps (one per SM
// sub-partition) with the fewest rows per lane R that still give at most one
// strip per SM: a smaller R shortens the step's dependency chain.  Pairs too
// tall for that take R = 16 and two strips per SM.
FillConfig swgb::pair_fill_config(const sw_ctx *c, int64_t rows) {
    if (!c->fwd_auto) return c->fwd;
    for (int R : {4, 8, 12, 16}) {
        const int64_t sh = 4LL * 32 * R;
        if ((rows + sh - 1) / sh <= (int64_t)c->nsm) return FillConfig{R, 4, 0, 2};
    }
    return FillConfig{16, 4, 0, 2};
}

// Tile shape of a single-pair fill with scoring s: the packed 16-bit fill
// (two cells per lane operation) where it is exact for the shape, with the
// fewest rows per lane in {8, 12, 16} that give at most one strip per SM;
// else the int32 fill of pair_fill_config.
FillConfig swgb::pair_fill_config_for(const sw_ctx *c, int64_t rows, const DevScoring &s) {
    if (s.alg != kAlgLocal) {
        FillConfig f = variant_fill_config(c, rows);
        if (!c->fwd_auto && (c->fwd.R == 8 || c->fwd.R == 12 || c->fwd.R == 16)) f.R = c->fwd.R;   // SWGB_FWD
        return f;
    }
    if (!c->fwd_auto) {
        FillConfig f = c->fwd;
        f.P16 = f.P16 && p16_fits(s, f.R) && f.W == 4;
        return f;
    }
    // Up to one 512-row strip per SM the int32 fill's 4-row lanes use twice the SMs of the packed
    // fill's 8-row lanes, which outweighs the packed fill's cheaper cells (2 kbp: 0.170 against
    // 0.190 ms); above that both take the same SM count and the packed fill wins (200 kbp: 19.8
    // against 24.0 ms)
    if (c->p16 && rows > (int64_t)c->nsm * 4 * 32 * 4) {
        for (int R : {8, 12, 16}) {
            const int64_t sh = 4LL * 32 * R;
            if ((rows + sh - 1) / sh <= (int64_t)c->nsm || R == 16) {
                if (p16_fits(s, R)) return FillConfig{R, 4, 0, 2, 1};
                break;
            }
        }
    }
    return pair_fill_config(c, rows);
}

// Compute warps per strip for a fill of one pair with `rows` rows.  The strips
// of a pair form a chain (each waits on the bottom row of the one above), so
// the chain runs at the pace of its slowest strip: two strips sharing an SM
// slow the whole pair.  Take the fewest warps (at least 4, where a strip's
// step is still latency-bound) that give at most one strip per SM; all W
// when even that many strips outnumber the SMs.
int swgb::pair_strip_warps(const sw_ctx *c, const FillConfig &cfg, int64_t rows) {
    if (cfg.S > 0) return std::min(cfg.S, cfg.W);
    for (int w = std::min(4, cfg.W); w < cfg.W; ++w) {
        const int64_t sh = (int64_t)w * 32 * cfg.R;
        if ((rows + sh - 1) / sh <= (int64_t)c->nsm) return w;
    }
    return cfg.W;
}

bool swgb::fold_open(const DevScoring &s) {
    int lo = 127, hi = -128;
    for (int k = 0; k < s.K * s.K; ++k) { lo = std::min(lo, (int)s.mat[k]); hi = std::max(hi, (int)s.mat[k]); }
    return hi + s.go <= 127 && lo + s.go >= -128;
}

int swgb::launch_fill(sw_ctx *c, const FillConfig &cfg, int mode, bool fold, const FillLaunch &L, int K,
                      long long tickets) {
    if (tickets <= 0) return SW_OK;
    if (cfg.P16) return launch_fill16(c, cfg, mode, L, K, tickets);
    if (cfg.alg != kAlgLocal) return launch_fill_variant(c, cfg, mode, fold, L, K, tickets);
    if (cfg.R == 4 && cfg.W == 4) return launch_fill_rw<4, 4>(c, mode, fold, L, K, tickets, cfg.B);
    if (cfg.R == 8 && cfg.W == 4) return launch_fill_rw<8, 4>(c, mode, fold, L, K, tickets, cfg.B);
    if (cfg.R == 8 && cfg.W == 8) return launch_fill_rw<8, 8>(c, mode, fold, L, K, tickets, cfg.B);
    if (cfg.R == 12 && cfg.W == 4) return launch_fill_rw<12, 4>(c, mode, fold, L, K, tickets, cfg.B);
    if (cfg.R == 16 && cfg.W == 4) return launch_fill_rw<16, 4>(c, mode, fold, L, K, tickets, cfg.B);
    return SW_EINVAL;
}

// Runs the fill over `tasks` (already in host memory, ticket0 assigned) on
// stream st with buffers b, and leaves the per-strip candidates in b.cand.
int swgb::run_fill_with(sw_ctx *c, const FillBufs &b, cudaStream_t st, const FillConfig &cfg, int mode, bool fold,
                        const std::vector<FillTask> &tasks, long long tickets, int K) {
    const size_t tbytes = tasks.size() * sizeof(FillTask);
    RC(b.tasks->ensure(tbytes));
    RC(b.prog->ensure((size_t)tickets * sizeof(int)));
    RC(b.cand->ensure((size_t)tickets * sizeof(int4)));
    RC(b.ticket->ensure(sizeof(unsigned long long)));
    RC(b.stage->ensure(tbytes));
    std::memcpy(b.stage->p, tasks.data(), tbytes);
    CU(cudaMemcpyAsync(b.tasks->p, b.stage->p, tbytes, cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(b.prog->p, 0, (size_t)tickets * sizeof(int), st));
    CU(cudaMemsetAsync(b.ticket->p, 0, sizeof(unsigned long long), st));
    FillLaunch L{};
    L.tasks = static_cast<const FillTask *>(b.tasks->p);
    L.scorings = static_cast<const DevScoring *>(c->scorings.p);
    L.ticket = static_cast<unsigned long long *>(b.ticket->p);
    L.prog = static_cast<int *>(b.prog->p);
    L.cand = static_cast<int4 *>(b.cand->p);
    L.err = static_cast<int *>(c->err.p);
    L.total = tickets;
    L.spin_limit = c->spin_limit;
    L.ntasks = (int)tasks.size();
    // the staging buffer is pinned and copied asynchronously: callers synchronise the stream
    // before they stage another fill on the same buffers (every ABI call ends with a sync)
    const cudaStream_t home = c->stream;
    c->stream = st;
    const int rc = launch_fill(c, cfg, mode, fold, L, K, tickets);
    c->stream = home;
    return rc;
}

// Runs the fill over `tasks` on the context's stream and buffers; the
// per-strip candidates are left in c->cand.
int swgb::run_fill(sw_ctx *c, const FillConfig &cfg, int mode, bool fold,
                   const std::vector<FillTask> &tasks, long long tickets, int K) {
    const FillBufs b{&c->tasks, &c->prog, &c->cand, &c->ticket, &c->stage};
    return run_fill_with(c, b, c->stream, cfg, mode, fold, tasks, tickets, K);
}

// Upload one or more scoring tables into c->scorings.
int swgb::upload_scorings(sw_ctx *c, const std::vector<DevScoring> &s) {
    const size_t bytes = s.size() * sizeof(DevScoring);
    RC(c->scorings.ensure(bytes));
    RC(c->stage2.ensure(bytes));
    std::memcpy(c->stage2.p, s.data(), bytes);
    CU(cudaMemcpyAsync(c->scorings.p, c->stage2.p, bytes, cudaMemcpyHostToDevice, c->stream));
    return SW_OK;
}

int swgb::reset_err(sw_ctx *c) {
    CU(cudaMemsetAsync(c->err.p, 0, sizeof(int), c->stream));
    return SW_OK;
}

int swgb::validate_codes(sw_ctx *c, const uint8_t *d, int64_t len, int K) {
    if (len <= 0) return SW_OK;
    const int threads = 256;
    const long long blocks = std::min<long long>((len + threads - 1) / threads, 4LL * c->nsm);
    validate_codes_kernel<<<(unsigned)blocks, threads, 0, c->stream>>>(d, len, K, static_cast<int *>(c->err.p));
    CU(cudaGetLastError());
    ++c->launches;
    return SW_OK;
}

int swgb::read_err(sw_ctx *c, int *e) {
    RC(c->stage3.ensure(64));
    CU(cudaMemcpyAsync(c->stage3.p, c->err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    *e = *static_cast<int *>(c->stage3.p);
    return SW_OK;
}

// ---------------------------------------------------------------- the ABI

extern "C" {

const char *sw_strerror(int s) {
    switch (s) {
        case SW_OK: return "ok";
        case SW_EINVAL: return "invalid argument";
        case SW_ENOMEM: return "out of memory";
        case SW_ECUDA: return "CUDA error";
        case SW_ETIMEOUT: return "bounded device wait gave up";
        case SW_EAGAIN: return "resource busy or result not ready";
        case SW_ERANGE: return "size or score out of range";
        default: return "unknown status";
    }
}

int sw_ctx_create(int device, void *cuda_stream, sw_ctx **out) {
    if (!out) return SW_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; }
    if (device < 0 || device >= ndev) return SW_EINVAL;
    DeviceGuard g(device);
    sw_ctx *c = new (std::nothrow) sw_ctx();
    if (!c) return SW_ENOMEM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return SW_ECUDA;
    }
    int rc = c->err.ensure(256);
    if (!rc) rc = c->stage3.ensure(4096);
    if (rc) { delete c; return rc; }
    if (cudaMemsetAsync(c->err.p, 0, 256, c->stream) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return SW_ECUDA;
    }
    const char *ev = std::getenv("SWGB_SPIN_LIMIT");
    c->spin_limit = ev ? std::atoll(ev) : (1LL << 26);
    c->fwd = FillConfig{8, 4, 0, 2};
    c->tbc = FillConfig{8, 4};
    c->bat = FillConfig{8, 4};
    // tuning overrides: SWGB_FWD="R,W[,S[,B[,P16]]]", SWGB_TB="R,W" and SWGB_BATCH="R,W[,P16]" (tile shapes
    // and lane widths of the fills)
    if (const char *f = std::getenv("SWGB_FWD")) {
        std::sscanf(f, "%d,%d,%d,%d,%d", &c->fwd.R, &c->fwd.W, &c->fwd.S, &c->fwd.B, &c->fwd.P16);
        c->fwd_auto = false;
    }
    if (const char *f = std::getenv("SWGB_TB")) std::sscanf(f, "%d,%d", &c->tbc.R, &c->tbc.W);
    if (const char *f = std::getenv("SWGB_BATCH")) std::sscanf(f, "%d,%d,%d", &c->bat.R, &c->bat.W, &c->bat.P16);
    if (const char *f = std::getenv("SWGB_PROF32")) c->prof32 = std::atoi(f) != 0;
    if (const char *f = std::getenv("SWGB_ONE_ROUND")) c->one_round = std::atoi(f) != 0 ? 1 : 0;
    if (const char *f = std::getenv("SWGB_LOOKAHEAD")) c->lookahead = std::atoi(f) != 0;
    if (const char *f = std::getenv("SWGB_TWO_LEVEL")) std::sscanf(f, "%lld,%lld", &c->two_level_bt1, &c->two_level_bt2);
    if (const char *f = std::getenv("SWGB_P16")) c->p16 = std::atoi(f) != 0;
    if (const char *f = std::getenv("SWGB_TB_BAND")) c->tb_band = std::atoi(f);
    if (const char *f = std::getenv("SWGB_TB_SW")) c->tb_strip_warps = std::atoi(f);
    // checkpoint memory of sw_align: 40% of the device memory free now (at least 4 GB), so that
    // the tiles stay small on long pairs (5 Mbp x 5 Mbp needs about 100 GB for 4096-cell tiles);
    // traceback bits of one band: 4 GB
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); free_b = 0; }
    c->ckpt_budget = std::max<size_t>((size_t)4 << 30, (size_t)((double)free_b * 0.4));
    c->tb_budget = (size_t)4 << 30;
    if (const char *f = std::getenv("SWGB_CKPT_BUDGET_MB")) c->ckpt_budget = (size_t)std::atoll(f) << 20;
    *out = c;
    return SW_OK;
}

void sw_ctx_destroy(sw_ctx *c) {
    if (!c) return;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->side_go) cudaEventDestroy(c->side_go);
    if (c->side_done) cudaEventDestroy(c->side_done);
    delete c;
}

int sw_encode(sw_ctx *c, const char *alphabet, const char *text, int64_t len, uint8_t *codes) {
    if (!c || !alphabet || len < 0 || (len > 0 && (!text || !codes))) return SW_EINVAL;
    const size_t K = std::strlen(alphabet);
    if (K < 1 || K > (size_t)kMaxAlphabet) return SW_EINVAL;
    uint8_t table[256];
    std::memset(table, 255, sizeof(table));
    for (size_t k = 0; k < K; ++k) {
        const unsigned char ch = (unsigned char)alphabet[k];
        if (table[ch] != 255) return SW_EINVAL;     // repeated letter
        table[ch] = (uint8_t)k;
        if (ch >= 'A' && ch <= 'Z') table[ch - 'A' + 'a'] = (uint8_t)k;
    }
    if (len == 0) return SW_OK;
    DeviceGuard g(c->device);
    const uint8_t *dtext = nullptr;
    RC(stage_seq(c, reinterpret_cast<const uint8_t *>(text), len, c->seq_a, &dtext));
    const bool dev_out = is_device_ptr(codes);
    uint8_t *dcodes = codes;
    if (!dev_out) {
        RC(c->seq_b.ensure((size_t)len + 16));
        dcodes = static_cast<uint8_t *>(c->seq_b.p);
    }
    RC(c->misc.ensure(256 + 16));
    RC(c->stage2.ensure(256 + 16));
    std::memcpy(c->stage2.p, table, 256);
    const unsigned long long none = ~0ULL;
    std::memcpy(static_cast<char *>(c->stage2.p) + 256, &none, 8);
    CU(cudaMemcpyAsync(c->misc.p, c->stage2.p, 264, cudaMemcpyHostToDevice, c->stream));
    uint8_t *dtable = static_cast<uint8_t *>(c->misc.p);
    unsigned long long *dbad = reinterpret_cast<unsigned long long *>(dtable + 256);
    const long long blocks = std::min<long long>((len + 255) / 256, 8LL * c->nsm);
    encode_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(dtext, len, dtable, dcodes, dbad);
    CU(cudaGetLastError());
    ++c->launches;
    CU(cudaMemcpyAsync(c->stage3.p, dbad, 8, cudaMemcpyDeviceToHost, c->stream));
    if (!dev_out) CU(cudaMemcpyAsync(codes, dcodes, (size_t)len, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    unsigned long long bad;
    std::memcpy(&bad, c->stage3.p, 8);
    return bad == ~0ULL ? SW_OK : SW_EINVAL;
}

int sw_score(sw_ctx *c, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
             const sw_scoring *sc, sw_hit *out) {
    if (!c || !out) return SW_EINVAL;
    DevScoring ds;
    RC(check_scoring(sc, &ds));
    if (m < 0 || n < 0 || (m > 0 && !a) || (n > 0 && !b)) return SW_EINVAL;
    if (m > SW_MAX_LEN || n > SW_MAX_LEN) return SW_ERANGE;
    if (!score_range_ok(sc, m, n)) return SW_ERANGE;
    if (m == 0 || n == 0) {
        // an empty side: the local score is 0; the other algorithms end on the border
        int cs = kNoScore, ci = 0x7fffffff, cj = 0x7fffffff;
        if (ds.alg != kAlgLocal) border_end_candidates(ds.alg, m, n, ds.go, ds.ge, &cs, &ci, &cj);
        *out = ds.alg == kAlgLocal ? sw_hit{0, 0, 0, 0} : sw_hit{cs, 0, (int64_t)ci, (int64_t)cj};
        return SW_OK;
    }
    DeviceGuard g(c->device);
    const uint8_t *da, *db;
    RC(stage_seq(c, a, m, c->seq_a, &da));
    RC(stage_seq(c, b, n, c->seq_b, &db));
    RC(reset_err(c));
    RC(validate_codes(c, da, m, ds.K));
    RC(validate_codes(c, db, n, ds.K));
    RC(upload_scorings(c, {ds}));

    const FillConfig fwd = pair_fill_config_for(c, m, ds);
    const int sw = pair_strip_warps(c, fwd, m);
    const int SH = sw * 32 * fwd.R;
    FillTask t{};
    t.a = da; t.b = db;
    t.rows = (int32_t)m; t.ncols = (int32_t)n;
    t.strip_warps = sw;
    t.nstrips = (int32_t)((m + SH - 1) / SH);
    t.scoring = 0; t.ticket0 = 0;
    t.top = nullptr;
    t.nslot = std::min(t.nstrips, 4);
    RC(c->bnd.ensure((size_t)t.nslot * (size_t)n * sizeof(int2)));
    t.bnd = static_cast<int2 *>(c->bnd.p);
    t.ckpt_every = 0; t.ckpt = nullptr; t.row0 = 0; t.tb = nullptr; t.tb_ld = 0;
    RC(run_fill(c, fwd, kModeScore, fold_open(ds), {t}, t.nstrips, ds.K));

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
    *out = sw_hit{res.x, 0, (int64_t)res.y, (int64_t)res.z};
    return SW_OK;
}

int64_t sw_ctx_launches(const sw_ctx *c) { return c ? c->launches : -1; }

int sw_ctx_timing(sw_ctx *c, int32_t enable) {
    if (!c) return SW_EINVAL;
    KernelTimer &T = c->timer;
    T.kind.clear();
    for (int k = 0; k < SW_KT_COUNT; ++k) { T.ms[k] = 0; T.n[k] = 0; }
    T.on = enable != 0;
    return SW_OK;
}

int sw_ctx_kernel_time(sw_ctx *c, int32_t kind, double *ms, int64_t *launches) {
    if (!c || kind < 0 || kind >= SW_KT_COUNT || !ms || !launches) return SW_EINVAL;
    DeviceGuard g(c->device);
    RC(kt_fold(c));
    *ms = c->timer.ms[kind];
    *launches = c->timer.n[kind];
    return SW_OK;
}

void sw_alignment_free(sw_alignment *aln) {
    if (!aln) return;
    std::free(aln->cigar);
    aln->cigar = nullptr;
    aln->cigar_len = 0;
}

}  // extern "C"
