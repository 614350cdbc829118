// wavefront.cuh -- intra-task Smith-Waterman/Gotoh fill (paper Section 2.1:
// one matrix, all processing elements cooperate and pass border elements to
// their neighbours).
//
// A "task" is a rectangle of one pair: rows [0, rows) of its `a` slice
// against columns [0, ncols) of its `b` slice, entered from a top boundary
// row (H, F per column; the matrix border when null) and a left boundary
// column (H, E per row; the matrix border when null).  It is cut into
// strips of strip_warps*32*R rows (at most HC = W*32*R); one thread block
// computes one strip at a time.
//
//   * Each of the W compute warps owns 32*R consecutive rows, each lane R
//     of them in registers.  Lanes form an anti-diagonal wavefront: at warp
//     step s lane t computes column s - t and receives the bottom H / F of
//     lane t-1 for that column by warp shuffle.
//   * Warps hand their bottom row to the next warp through shared-memory
//     rings guarded by acquire/release counters (no block barriers in the
//     sweep); every wait is bounded.
//   * Two I/O warps move data between global and shared memory: the input
//     warp streams the strip's top boundary row and the column residues
//     ahead of warp 0; the output warp drains the strip's bottom row to
//     global memory and publishes how many columns are stored with
//     st.release.gpu, which the next strip's input warp reads with
//     ld.acquire.gpu.  Keeping them apart means polling for input never
//     delays the output the next strip is waiting for.
//   * Strips are claimed from a global ticket counter in order, so a strip
//     only waits on strips already held by running blocks.
//
// Cell update (R rows of one column).  With e <= o the vertical gap obeys
//   F(i+1,j) = max(F(i,j) - e, X(i,j) - o),  X = max(0, H(i-1,j-1)+S, E)
// because H = max(X, F) and F - o <= F - e; so the dependency from one row
// to the next is a single max-add, and H = max(X, F), H - o = max(F - o,
// X - o) follow off that chain.  Scores come from a per-strip query profile
// in shared memory, prof[c*HC + r] = S(a_r, c) (int8 with one prmt per
// cell, or int32 for small alphabets; padding residue c = K at -128), one
// vector load per step.
//
// Modes: score (TB = false) keeps, per lane, the best H with its first
// row, then first column (a branch-free row key, see row_key), and writes
// one end-cell candidate per strip; it can also store the strip's bottom row
// as a checkpoint row and, every `colck_every` columns, a checkpoint column
// in staircase form (all lanes store at one step, so lane l's rows hold
// column c - l; a task entered from such a column first brings every lane to
// column c, see FillTask::left).
// Traceback (TB = true) writes, for every cell, four decision bits
// {H source: 0 zero, 1 diagonal, 2 E, 3 F; E opened; F opened} packed R
// nibbles per word, for the walk.
#pragma once
#include "sw_device.cuh"

namespace swgb {

struct FillTask {
    const uint8_t *a;      // the task's rows: a[0 .. rows)
    const uint8_t *b;      // the task's columns: b[0 .. ncols)
    int32_t rows;
    int32_t ncols;
    int32_t nstrips;
    int32_t scoring;       // index into the scoring table
    int64_t ticket0;       // global ticket of strip 0
    const int2 *top;       // (H, F) per column of the row above, or null (matrix border)
    const int2 *left;      // staircase left boundary, or null (matrix border): row i of 32-lane
                           // group lane l = (i / R) % 32 holds (H - open, E) at column c - l,
                           // c = the column left of the task (written by a kModeScoreCk fill)
    const int2 *left_aux;  // per row group of left: (H - open of the row above at column c - l,
                           // F of the group's last row at column c - l)
    int2 *bnd;             // bottom rows of the strips: slot (strip % nslot) * ncols (not
                           // written by the last strip; may be null for one-strip tasks)
    int32_t nslot;
    int32_t ckpt_every;    // also copy every ckpt_every-th strip's bottom row to ckpt (0 = never);
                           // only strips whose bottom row is inside the task: rows / (strip rows * ckpt_every) rows
    int2 *ckpt;            // checkpoint rows: ((strip+1)/ckpt_every - 1) * ncols
    int2 *colck;           // checkpoint columns, staircase form (see left): checkpoint k = (c+1)/colck_every - 1
                           // at colck + k * colck_ld + row; colck_ld covers the last strip's padding rows
    int2 *colck_aux;       // the matching left_aux rows: colck_aux + k * (colck_ld / R) + row / R
    int32_t colck_every;   // 0 = none; else store after every colck_every-th column
    int32_t row0;          // row index (0-based, in the whole pair) of the task's first row
    int32_t col0;          // column index (0-based, in the whole pair) of the task's first column
    int64_t colck_ld;
    void *tb;              // traceback words, TB mode: [row group][tb_ld]
    int64_t tb_ld;
    int32_t strip_warps;   // compute warps per strip (rows per strip = strip_warps * 32 * R);
                           // 0 = all W warps of the block
    int32_t left_split;    // left / left_aux in the two-positions-per-lane form of the packed
                           // fill (wavefront16.cuh): the first R/2 rows of lane l sit at column
                           // c - 2l, the other R/2 at c - 2l - 1, and left_aux holds one record
                           // per half-group of R/2 rows (first the top half's, then the bottom's)
};

struct FillLaunch {
    const FillTask *tasks;
    const DevScoring *scorings;
    unsigned long long *ticket;   // zeroed before launch
    int *prog;                    // per ticket: columns published; zeroed before launch
    int4 *cand;                   // per ticket: (score, i, j, valid) end-cell candidate
    int *err;                     // error word (kErr*)
    long long total;              // total tickets
    long long spin_limit;         // polls before a wait gives up
    int ntasks;
    // claim order (optional): claim k takes strip order[k].y of task order[k].x, so that a
    // plan can hand out every task's first strip before any second one; nullptr: tickets in
    // task order, each task's strips consecutive (task = last with ticket0 <= k).  Either way a
    // strip's predecessor is claimed before it, and progress and candidates are kept per
    // (task, strip) at ticket0 + strip.
    const int2 *order;
};

template <int R> struct TbWord;
template <> struct TbWord<4> { using T = uint16_t; };
template <> struct TbWord<8> { using T = uint32_t; };
template <> struct TbWord<12> { using T = unsigned long long; };
template <> struct TbWord<16> { using T = unsigned long long; };

// Query profile kinds: int8 scores S, int8 scores S + open ("folded", the
// open penalty is then free in the cell update), or int32 scores S + open
// (no byte extraction per cell; four times the shared memory, so only for
// small alphabets).
enum ProfKind { kProf8 = 0, kProf8Fold = 1, kProf32 = 2 };

template <int R, int PK>
struct ProfWords { static constexpr int N = PK == kProf32 ? R : R / 4; };   // 32-bit words per lane

// int32 profiles are stored chunk-major so that every 16-byte load of a warp
// is conflict-free: residue c, lane g (of the strip's NL = W*32 lanes), rows
// 4q .. 4q+3 of the lane sit at int32 index ((c*(R/4) + q)*NL + g)*4.  A lane
// passes p = its first chunk of residue c; chunk q is NL*16 bytes further on.
template <int R, int PK, int NL = 0>
__device__ __forceinline__ void load_profile(const int8_t *p, uint32_t (&w)[ProfWords<R, PK>::N]) {
    if constexpr (PK == kProf32) {
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const uint4 v = *reinterpret_cast<const uint4 *>(p + (size_t)q * NL * 16);
            w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
        }
    } else if constexpr (R == 4) {
        w[0] = *reinterpret_cast<const uint32_t *>(p);
    } else if constexpr (R == 8) {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        w[0] = v.x; w[1] = v.y;
    } else if constexpr (R == 12) {           // 12-byte lane stride: 4-byte aligned only
        const uint32_t *q = reinterpret_cast<const uint32_t *>(p);
        w[0] = q[0]; w[1] = q[1]; w[2] = q[2];
    } else {
        const uint4 v = *reinterpret_cast<const uint4 *>(p);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
}

__device__ __forceinline__ int score_byte(const uint32_t *w, int r) {
    switch (r & 3) {            // r is a constant after unrolling: one prmt
        case 0: return sext8<0>(w[r >> 2]);
        case 1: return sext8<1>(w[r >> 2]);
        case 2: return sext8<2>(w[r >> 2]);
        default: return sext8<3>(w[r >> 2]);
    }
}

template <int PK>
__device__ __forceinline__ int score_at(const uint32_t *w, int r) {
    if constexpr (PK == kProf32) return (int)w[r];
    else return score_byte(w, r);
}

__device__ __forceinline__ int lds_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.b32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}

__device__ __forceinline__ void sts_release(int *p, int v) {
    asm volatile("st.release.cta.shared.b32 [%0], %1;" :: "r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}

// Thread 0 of a fill block claims its next strip: *s_tk = the claim (L.total once all are taken
// or after an error), and the task and strip it stands for (FillLaunch::order).
__device__ __forceinline__ void claim_strip(const FillLaunch &L, long long *s_tk, int *s_task, int *s_strip) {
    long long tk = (long long)atomicAdd(L.ticket, 1ULL);
    if (ld_volatile(L.err) != 0) tk = L.total;           // stop early after an error
    *s_tk = tk;
    if (tk >= L.total) return;
    if (L.order) {
        const int2 o = L.order[tk];
        *s_task = o.x;
        *s_strip = o.y;
        return;
    }
    int lo = 0, hi = L.ntasks - 1;                       // last task with ticket0 <= tk
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.tasks[mid].ticket0 <= tk) lo = mid; else hi = mid - 1;
    }
    *s_task = lo;
    *s_strip = (int)(tk - L.tasks[lo].ticket0);
}

// The warp waits until *ctr >= want (bounded).  Every lane reads the counter
// with acquire semantics, so the common case (already there) is one uniform
// check; false on timeout or when the block is aborting.
__device__ __forceinline__ bool warp_wait_geq(const int *ctr, int want, const volatile int *abort_flag,
                                              long long limit, int *err) {
    if (lds_acquire(ctr) >= want) return true;
    long long it = 0;
    while (lds_acquire(ctr) < want) {
        if (*abort_flag) return false;
        if (++it > limit) { atomicCAS(err, 0, kErrTimeout); return false; }
        if (it > 64) __nanosleep(20);              // spin first: the producer is usually a step away
    }
    return true;
}

enum FillMode { kModeScore = 0, kModeScoreCk = 1, kModeTb = 2 };

constexpr int kCH = 32;       // steps between the warps' counter updates: fewer hand-offs against
                              // more lag between warps (32 measured best of 8..64 on GB300)
// Steps per unrolled body of the steady loop.  Measured on GB300 (2, 4, 8, 16): the
// traceback fill, whose body also packs decision words, runs best at 4; the score
// fills at 8, and at 16 when a lane holds only 4 rows (a short body).
constexpr int fill_unroll(int R, int MODE) { return MODE == kModeTb ? 4 : (R <= 4 ? 16 : 8); }
constexpr int kQS = 256;      // boundary-ring columns per channel
constexpr int kQB = 1024;     // residue-ring columns
constexpr int kIOB = 64;      // columns per I/O batch

// Per-lane state of the sweep.  U = H - open and E of the lane's R rows at
// the previous column; ub / fb the bottom row's U and F of the previous step
// (shuffled to the next lane); udiag0 = U of the row above the first row at
// the previous column (the first row's diagonal); bk / bj the lane's best
// cell as a row key (below) and its column.
template <int R>
struct LaneState {
    int U[R], E[R];
    int ub, fb, udiag0;
    int bk, bj;
    int rlast;        // the other algorithms: the lane's row holding the task's last row, or -1
    unsigned track;   // ... as a bit mask (1 << rlast) where that row is an end row at every column
                      // (semi-global, overlap), else 0.  A mask, not a comparison with rlast: a
                      // chain of selects on r == rlast is turned into an indexed load of U by the
                      // compiler, which moves the lane state to local memory.
};

// The lane's end cell is the first of its cells in row-major order holding
// its maximum.  Each row r of a column gets the key U * kKeyRows + (R-1-r):
// one integer maximum over the rows then picks the largest U and, among
// equal ones, the smallest row.  Columns arrive in order, so a column
// replaces the lane's best exactly when its key is strictly larger (a larger
// score, or an equal one in an earlier row): one compare and two selects per
// step, no branch.  Keys need |U| < 2^31 / kKeyRows (callers bound scores by
// kMaxScoreBound).
constexpr int kKeyRows = 16;
static_assert(kKeyRows * kMaxScoreBound <= (1LL << 30), "row keys overflow");

template <int R>
__device__ __forceinline__ int row_key(int u, int r) { return u * kKeyRows + (R - 1 - r); }

// One column of one lane's R rows (Gotoh recurrence, paper Section 2.1.2),
// entered with uup / fup = H - open and F of the row above at this column;
// st.udiag0 holds H - open of the row above at the previous column.  TB
// collects the four decision bits of every cell into word.
// LOCAL: the Smith-Waterman zero floor; without it (the global, semi-global and
// overlap algorithms) H has no floor and no cell has the "zero" source.
template <int R, int PK, bool TB, bool LOCAL = true>
__device__ __forceinline__ void column_update(LaneState<R> &st, const uint32_t (&pw)[ProfWords<R, PK>::N], int uup, int fup,
                                              int go, int ge, typename TbWord<R>::T &word)
{
    int udiag = st.udiag0;
    st.udiag0 = uup;
    int f = __viaddmax_s32(fup, -ge, uup);                 // F of the first row
    int fopen_ref = uup;                                   // H(i-1,j) - open
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int sp = score_at<PK>(pw, r);                      // S (+ open when folded)
        if constexpr (PK == kProf8) sp += go;
        const int uold = st.U[r];                          // H(i,j-1) - open
        const int e = __viaddmax_s32(st.E[r], -ge, uold);
        const int x = LOCAL ? __viaddmax_s32_relu(udiag, sp, e)  // max(H(i-1,j-1) + S, E, 0)
                            : __viaddmax_s32(udiag, sp, e);
        const int xgo = x - go;
        const int u = __viaddmax_s32(f, -go, xgo);         // H(i,j) - open
        if constexpr (TB) {
            const int h = u + go, diag = udiag + sp;
            const unsigned src = (LOCAL && h == 0) ? 0u : (h == diag ? 1u : (h == e ? 2u : 3u));
            const unsigned nib = src | (e == uold ? 4u : 0u) | (f == fopen_ref ? 8u : 0u);
            word |= (typename TbWord<R>::T)nib << (4 * r);
            fopen_ref = u;
        }
        st.E[r] = e;
        udiag = uold;
        st.U[r] = u;
        if (r + 1 < R) f = __viaddmax_s32(f, -ge, xgo);    // F of the next row
    }
    st.ub = st.U[R - 1];
    st.fb = f;
}

// One wavefront step of one lane: column j = s - lane of its R rows.
// CHECK handles columns outside [0, n) (the first 31 and last 31 steps of
// a sweep) where no padding stands in for them (traceback tiles, tasks with
// a left boundary); every other step skips those tests.
template <int R, int MODE, int PK, bool CHECK, bool LOCAL = true>
__device__ __forceinline__ void lane_step(LaneState<R> &st, const uint32_t (&pw)[ProfWords<R, PK>::N], int2 top,
                                          int s, int lane, int n, int go, int ge,
                                          int2 *ring_out, typename TbWord<R>::T *tbw)
{
    const int j = s - lane;
    int uup = __shfl_up_sync(kFull, st.ub, 1);
    int fup = __shfl_up_sync(kFull, st.fb, 1);
    if (lane == 0) { uup = top.x; fup = top.y; }
    if (CHECK && (j < 0 || j >= n)) return;
    typename TbWord<R>::T word = 0;
    column_update<R, PK, MODE == kModeTb, LOCAL>(st, pw, uup, fup, go, ge, word);
    if (lane == 31) ring_out[j & (kQS - 1)] = make_int2(st.ub, st.fb);
    if constexpr (MODE == kModeTb) {
        tbw[j] = word;
    } else if constexpr (!LOCAL) {
        // semi-global and overlap: the task's last row is an end row at every column
        int ck = st.bk;
#pragma unroll
        for (int r = 0; r < R; ++r) ck = ((st.track >> r) & 1u) ? row_key<R>(st.U[r], r) : ck;
        st.bj = ck > st.bk ? j : st.bj;
        st.bk = max(st.bk, ck);
    } else {
        int ck = row_key<R>(st.U[0], 0);
#pragma unroll
        for (int r = 1; r + 1 < R; r += 2)
            ck = __vimax3_s32(ck, row_key<R>(st.U[r], r), row_key<R>(st.U[r + 1], r + 1));
        if constexpr (R % 2 == 0) ck = max(ck, row_key<R>(st.U[R - 1], R - 1));
        st.bj = ck > st.bk ? j : st.bj;
        st.bk = max(st.bk, ck);
    }
}

// Rows [r0, r1) of one lane advanced by one column (the Gotoh update of
// column_update restricted to a range of the lane's rows), entered with the
// row above's H - open and F at this column; udiag = H - open of the row
// above at the previous column.  Returns the last row's F in *fout.
template <int R, int PK, bool LOCAL>
__device__ __forceinline__ void rows_update(LaneState<R> &st, const uint32_t (&pw)[ProfWords<R, PK>::N], int r0,
                                            int r1, int uup, int fup, int udiag, int go, int ge, int *fout)
{
    int f = __viaddmax_s32(fup, -ge, uup);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r < r0 || r >= r1) continue;
        int sp = score_at<PK>(pw, r);
        if constexpr (PK == kProf8) sp += go;
        const int uold = st.U[r];
        const int e = __viaddmax_s32(st.E[r], -ge, uold);
        const int x = LOCAL ? __viaddmax_s32_relu(udiag, sp, e) : __viaddmax_s32(udiag, sp, e);
        const int xgo = x - go;
        st.U[r] = __viaddmax_s32(f, -go, xgo);
        st.E[r] = e;
        udiag = uold;
        if (r + 1 < r1) f = __viaddmax_s32(f, -ge, xgo);
    }
    *fout = f;
}

// A task entered from a checkpoint column written by the packed fill, whose
// lanes hold two wavefront positions each: lane l's top half (rows
// [0, R/2)) sits at column c - 2l, its bottom half at c - 2l - 1, where c is
// the column left of the task.  Position v = 2l (top) or 2l + 1 (bottom)
// advances v columns, in step with its neighbours -- the top half's k-th
// column needs lane l-1's bottom half after its (k-1)-th, the bottom half's
// needs this lane's top half after its (k-1)-th -- so that every row ends at
// column c: a 63-step wavefront inside the warp.  Leaves st as the straight
// boundary column the sweep starts from (U, E per row; ub / fb the last
// row's H - open and F at c; udiag0 the row above at c for lane 0).
template <int R, int W, int PK, bool LOCAL>
__device__ __forceinline__ void split_staircase_prologue(const FillTask &T, LaneState<R> &st, const int8_t *prow,
                                                         int grow, int lane, int K, int go, int ge)
{
    constexpr int H = R / 2;
    constexpr int HC = W * 32 * R;
    constexpr size_t PB = PK == kProf32 ? 4 : 1;
    constexpr int NPW = ProfWords<R, PK>::N;
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (grow + r < T.rows) { const int2 v = __ldcg(T.left + grow + r); st.U[r] = v.x; st.E[r] = v.y; }
    const bool in = grow < T.rows;
    const int2 at = in ? __ldcg(T.left_aux + grow / H) : make_int2(-go, kNeg);       // top half
    const int2 ab = in ? __ldcg(T.left_aux + grow / H + 1) : make_int2(-go, kNeg);   // bottom half
    int udT = at.x, fT = at.y;        // row above the top half at its column; F of its last row
    int udB = ab.x, fB = ab.y;        // the same for the bottom half
    for (int k = 1; k < 64; ++k) {
        // lane l-1's bottom half after its (k-1)-th column: the row above this lane's top half
        const int uupT = __shfl_up_sync(kFull, st.U[R - 1], 1);
        const int fupT = __shfl_up_sync(kFull, fB, 1);
        // the bottom half moves first: its row above is the top half before this step
        if (k <= 2 * lane + 1) {
            const int cb = min((int)T.b[k - 2 * lane - 2], K);   // column c - 2l - 1 + k
            uint32_t pwk[NPW];
            load_profile<R, PK, W * 32>(prow + cb * HC * PB, pwk);
            const int uup = st.U[H - 1];
            rows_update<R, PK, LOCAL>(st, pwk, H, R, uup, fT, udB, go, ge, &fB);
            udB = uup;
        }
        if (k <= 2 * lane) {
            const int cb = min((int)T.b[k - 2 * lane - 1], K);   // column c - 2l + k
            uint32_t pwk[NPW];
            load_profile<R, PK, W * 32>(prow + cb * HC * PB, pwk);
            rows_update<R, PK, LOCAL>(st, pwk, 0, H, uupT, fupT, udT, go, ge, &fT);
            udT = uupT;
        }
    }
    st.ub = st.U[R - 1];
    st.fb = fB;
    // the diagonal of the task's first column: the row above at column c
    const int up = __shfl_up_sync(kFull, st.ub, 1);
    st.udiag0 = lane > 0 ? up : udT;
}

// Input warp of a fill block: streams the strip's top boundary row (the
// matrix border, the task's top row or the previous strip's bottom row, as
// (H - open, F), multiplied by 2^SHIFT) into channel 0 of the boundary ring and the column residues
// into the residue ring, ahead of the first compute warp.  Room in channel 0
// is bounded by what warp 0 consumed, room in the residue ring by what the
// last active warp (whose lanes read furthest back, `lag` columns behind its
// published count) has published.
template <int QS, int QB, int IOB, int SHIFT = 0>
__device__ __forceinline__ void fill_input_warp(const FillTask &T, const FillLaunch &L, int strip, long long slot,
                                                int n, int go, int K, int Wa, int lag, int2 *ring0,
                                                uint8_t *bring, int *prod, const int *cons,
                                                volatile int *s_abort, int lane, int alg = kAlgLocal, int ge = 0,
                                                int *poff = nullptr, int pk1 = 0, int pstride = 0)
{
    int in_next = 0;
    long long idle = 0;
    const int2 *src = strip == 0 ? T.top : T.bnd + (size_t)((strip - 1) % T.nslot) * n;
    const int *pprev = L.prog + (slot - 1);
    int avail_prev = strip == 0 ? n : 0;
    while (in_next < n) {
        const int room0 = lds_acquire(&cons[0]) + QS;
        const int roomb = lds_acquire(&prod[Wa]) + QB - lag;
        int target = min(n, min(in_next + IOB, min(room0, roomb)));
        if (target > in_next && strip > 0 && avail_prev < target)
            avail_prev = ld_acquire(pprev);              // every lane: acquire for its own loads
        target = min(target, avail_prev);
        if (target > in_next) {
            for (int col = in_next + lane; col < target; col += 32) {
                // the matrix's top border: H(0, j) of the algorithm, F = -infinity
                const int2 v = src ? __ldcg(src + col)
                                   : make_int2((int)top_border_h(alg, (long long)T.col0 + col + 1, go, ge), kNeg);
                if constexpr (SHIFT == 0)
                    ring0[col & (QS - 1)] = make_int2(v.x - go, v.y);
                else     // scaled values; -infinity stays far below every real value, without overflow
                    ring0[col & (QS - 1)] = make_int2((v.x - go) * (1 << SHIFT), max(v.y, kNeg >> SHIFT) * (1 << SHIFT));
                const int c = min((int)T.b[col], K);
                bring[col & (QB - 1)] = (uint8_t)c;
                // pair profile (packed fill): the byte offset of the entry for (b[col], b[col - 1])
                if (poff)   // (column -1 is real for a task entered from a checkpoint column)
                    poff[col & (QB - 1)] = (c * pk1 + ((col > 0 || T.left) ? min((int)T.b[col - 1], K) : K)) * pstride;
            }
            __syncwarp();
            if (lane == 0) sts_release(&prod[0], target);
            in_next = target;
            idle = 0;
        } else {
            if (*s_abort) break;
            if (++idle > L.spin_limit) {
                if (lane == 0) atomicCAS(L.err, 0, kErrTimeout);
                *s_abort = 1;
                break;
            }
            // far ahead of warp 0 (more than two batches buffered): poll rarely, so that the
            // compute warp sharing this SM sub-partition keeps its issue slots
            if (in_next - lds_acquire(&cons[0]) > 2 * IOB) __nanosleep(256);
            else if (idle > 32) __nanosleep(32);
        }
    }
}

// Output warp of a fill block: drains the strip's bottom row (H - open, F),
// multiplied by 2^SHIFT, from the last active warp's channel to global memory as (H, F) -- the next
// strip's input and, every ckpt_every-th strip, a checkpoint row -- and
// publishes the stored column count with a release store.
template <int QS, int SHIFT = 0>
__device__ __forceinline__ void fill_output_warp(const FillTask &T, const FillLaunch &L, int strip, long long slot,
                                                 int n, int go, int SH, int Wa, const int2 *ringW,
                                                 const int *prod, int *cons, volatile int *s_abort, int lane)
{
    int out_next = 0;
    long long idle = 0;
    // a checkpoint row only where the strip's bottom row lies inside the task
    // (the last strip may be partial)
    const bool ck = T.ckpt_every > 0 && ((strip + 1) % T.ckpt_every) == 0 &&
                    (long long)(strip + 1) * SH <= (long long)T.rows;
    int2 *cdst = ck ? T.ckpt + (size_t)((strip + 1) / T.ckpt_every - 1) * n : nullptr;
    // the last strip's bottom row feeds no other strip
    const bool store = strip + 1 < T.nstrips;
    int2 *dst = store ? T.bnd + (size_t)(strip % T.nslot) * n : nullptr;
    while (out_next < n) {
        const int avail_out = lds_acquire(&prod[Wa]);
        if (avail_out > out_next) {
            if (store || ck) {
                for (int col = out_next + lane; col < avail_out; col += 32) {
                    const int2 u = ringW[col & (QS - 1)];
                    const int2 v = make_int2((u.x >> SHIFT) + go, u.y >> SHIFT);
                    if (store) dst[col] = v;
                    if (ck) cdst[col] = v;
                }
            }
            // the lanes' stores are ordered before lane 0's release by the warp
            // barrier; the release (gpu scope) publishes them cumulatively
            __syncwarp();
            if (lane == 0) {
                if (store) st_release(L.prog + slot, avail_out);
                sts_release(&cons[Wa], avail_out);
            }
            out_next = avail_out;
            idle = 0;
        } else {
            if (*s_abort) break;
            if (++idle > L.spin_limit) {
                if (lane == 0) atomicCAS(L.err, 0, kErrTimeout);
                *s_abort = 1;
                break;
            }
            if (idle > 32) __nanosleep(32);
        }
    }
}

// LOCAL = false: the global, semi-global and overlap algorithms (DevScoring::alg)
template <int R, int W, int MODE, int PK, bool LOCAL = true>
__global__ void __launch_bounds__((W + 2) * 32) __maxnreg__(R >= 12 ? 128 : (W > 4 ? 96 : 104))
wavefront_kernel(const FillLaunch L)
{
    constexpr int HC = W * 32 * R;
    constexpr int CH = kCH, QS = kQS, QB = kQB, IOB = kIOB;
    static_assert(QS >= 2 * IOB + 2 * CH + 64, "ring too small");
    constexpr int UNR = fill_unroll(R, MODE);
    // the unchecked tail below pays off where strips are few and their ends sit on the
    // critical path; with 16-row lanes its extra unrolled body slowed the steady state of
    // long sweeps (measured on GB300), so those keep the bounds-checked tail
    constexpr bool kEdgeFast = R <= 12;
    static_assert(CH % UNR == 0, "chunks are whole unrolled groups");

    extern __shared__ __align__(16) int8_t prof[];   // (K + 1) * HC scores of PB bytes
    constexpr int PB = PK == kProf32 ? 4 : 1;
    constexpr int NPW = ProfWords<R, PK>::N;
    __shared__ int2 ring[W + 1][QS];                 // channel k: producer k-1 (I/O for k=0), consumer k (I/O for k=W); (H - open, F)
    __shared__ uint8_t bring[QB];
    __shared__ int prod[W + 1];                      // columns available in channel k
    __shared__ int cons[W + 1];                      // columns consumed from channel k
    __shared__ long long s_tk;
    __shared__ int s_task, s_strip;
    __shared__ volatile int s_abort;
    __shared__ int4 s_cand[W];

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    for (;;) {
        if (threadIdx.x == 0) {
            claim_strip(L, &s_tk, &s_task, &s_strip);
            s_abort = 0;
        }
        if (threadIdx.x <= W) { prod[threadIdx.x] = 0; cons[threadIdx.x] = 0; }
        __syncthreads();
        const long long tk = s_tk;
        if (tk >= L.total) return;
        const FillTask &T = L.tasks[s_task];
        const DevScoring &SC = L.scorings[T.scoring];
        const int K = SC.K, go = SC.go, ge = SC.ge;
        const int strip = s_strip;
        const long long slot = T.ticket0 + strip;        // progress and candidate of (task, strip)
        const int SW = (T.strip_warps > 0 && T.strip_warps < W) ? T.strip_warps : W;
        const int SH = SW * 32 * R;                     // rows per strip of this task
        const int rbase = strip * SH;                   // first row of the strip within the task
        const int n = T.ncols;
        // warps holding at least one row of the task; the others sit the strip out
        const int Wa = min(SW, (T.rows - rbase + 32 * R - 1) / (32 * R));

        // ---- query profile of the strip's rows: S(a_r, c) (+ open when folded)
        for (int lr = threadIdx.x; lr < SH; lr += blockDim.x) {
            const int r = rbase + lr;
            const bool ok = r < T.rows;
            const int av = ok ? min((int)T.a[r], K - 1) : 0;
            for (int c = 0; c <= K; ++c) {
                const int v = (ok && c < K) ? SC.mat[av * K + c] + (PK != kProf8 ? go : 0) : kPadScore;
                if constexpr (PK == kProf32)
                    reinterpret_cast<int32_t *>(prof)[((c * (R / 4) + (lr % R) / 4) * (W * 32) + lr / R) * 4 + (lr & 3)] = v;
                else prof[c * HC + lr] = (int8_t)v;
            }
        }
        // the residue ring's last 32 slots read as padding: lanes may prefetch the columns
        // left of the task (index -31 .. -1) during their first chunk (see virt_ok below);
        // the input warp reaches those slots only after every warp has left its first chunk
        if (threadIdx.x < 32) bring[QB - 32 + threadIdx.x] = (uint8_t)K;
        __syncthreads();

        if (warp == W) {
            // ================= input warp: top boundary row and residues =================
            fill_input_warp<QS, QB, IOB>(T, L, strip, slot, n, go, K, Wa, 64, ring[0], bring, prod, cons,
                                         &s_abort, lane, LOCAL ? kAlgLocal : SC.alg, ge);
        } else if (warp == W + 1) {
            // ================= output warp: bottom row to global memory =================
            fill_output_warp<QS>(T, L, strip, slot, n, go, SH, Wa, ring[Wa], prod, cons, &s_abort, lane);
        } else if (warp >= Wa) {
            if constexpr (MODE != kModeTb)
                if (lane == 0) s_cand[warp] = make_int4(LOCAL ? 0 : kNoScore, 0x7fffffff, 0x7fffffff, 0);
        } else {
            // ================= compute warp =================
            const int lrow = (warp * 32 + lane) * R;        // first row of this lane within the strip
            const int grow = rbase + lrow;                  // ... within the task
            // this lane's first profile entry (int8: its R rows are contiguous; int32: chunk-major)
            const int8_t *prow = PK == kProf32 ? prof + (warp * 32 + lane) * 16 : prof + lrow;
            LaneState<R> st;
#pragma unroll
            for (int r = 0; r < R; ++r) { st.U[r] = -go; st.E[r] = kNeg; }
            st.udiag0 = -go;                                // matrix border: H = 0
            if constexpr (!LOCAL) {                         // the algorithm's left border H(i, 0)
#pragma unroll
                for (int r = 0; r < R; ++r)
                    st.U[r] = (int)left_border_h(SC.alg, (long long)T.row0 + grow + r + 1, go, ge) - go;
                st.udiag0 = (int)left_border_h(SC.alg, (long long)T.row0 + grow, go, ge) - go;
                st.rlast = (T.rows - 1 >= grow && T.rows - 1 < grow + R) ? T.rows - 1 - grow : -1;
                st.track = ((SC.alg == kAlgSemiGlobal || SC.alg == kAlgOverlap) && st.rlast >= 0) ? 1u << st.rlast : 0u;
            }
            st.ub = st.U[R - 1];
            st.fb = kNeg;
            if (T.left && T.left_split) {
                split_staircase_prologue<R, W, PK, LOCAL>(T, st, prow, grow, lane, K, go, ge);
            } else if (T.left) {
                // Staircase left boundary: lane l's rows hold column c - l (c = the column
                // left of the task).  Lane l advances l columns, in step with its neighbours
                // (lane l's k-th column needs lane l-1's (k-1)-th), so that every lane ends at
                // column c: a 31-step wavefront inside the warp.
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (grow + r < T.rows) { const int2 v = __ldcg(T.left + grow + r); st.U[r] = v.x; st.E[r] = v.y; }
                const int2 ax = grow < T.rows ? __ldcg(T.left_aux + grow / R) : make_int2(-go, kNeg);
                st.udiag0 = ax.x;
                st.ub = st.U[R - 1];
                st.fb = ax.y;
                for (int k = 1; k < 32; ++k) {
                    const int uup = __shfl_up_sync(kFull, st.ub, 1);
                    const int fup = __shfl_up_sync(kFull, st.fb, 1);
                    if (k <= lane) {
                        const int cb = min((int)T.b[k - lane - 1], K);   // column c - lane + k
                        uint32_t pwk[NPW];
                        load_profile<R, PK, W * 32>(prow + cb * HC * PB, pwk);
                        typename TbWord<R>::T unused = 0;
                        column_update<R, PK, false, LOCAL>(st, pwk, uup, fup, go, ge, unused);
                    }
                }
                // the diagonal of the task's first column: the row above at column c
                const int up = __shfl_up_sync(kFull, st.ub, 1);
                if (lane > 0) st.udiag0 = up;
            }
            // local: score 0 never becomes the best; the other algorithms: any cell of an end row
            st.bk = LOCAL ? row_key<R>(-go, 0) : kNoScore; st.bj = -1;
            // checkpoint columns (kModeScoreCk): every lane stores at the end of the chunk whose
            // last step is column next_ck for lane 0, so lane l stores column next_ck - l
            int next_ck = (MODE == kModeScoreCk && T.colck && T.colck_every > 0) ? T.colck_every - 1 : 0x7fffffff;
            typename TbWord<R>::T *tbw = nullptr;
            if constexpr (MODE == kModeTb)
                tbw = reinterpret_cast<typename TbWord<R>::T *>(T.tb) + (size_t)(grow / R) * (size_t)T.tb_ld;
            int2 *rin = ring[warp];
            int2 *rout = ring[warp + 1];

            int seen_in = 0;
            bool loaded = false;             // inputs of step s0 were prefetched by the previous step
            // columns left of the task may be computed (first chunk) only from a border state,
            // and never in traceback mode (their decision words would land outside the tile)
            const bool virt_ok = LOCAL && MODE != kModeTb && T.left == nullptr;
            int c;
            uint32_t pw[NPW];
            int2 top;
            for (int s0 = 0; s0 < n + 31; s0 += CH) {
                const int need_in = min(n, s0 + CH + 1);   // this chunk plus the next step's prefetch
                if (need_in > seen_in) {
                    if (!warp_wait_geq(&prod[warp], need_in, &s_abort, L.spin_limit, L.err)) { s_abort = 1; break; }
                    seen_in = need_in;
                }
                // lane 31 writes columns below s0 + CH - 31 to the ring this chunk (past n only
                // on the padded path below); out_hi of them are real and get published
                const int ring_hi = max(0, s0 + CH - 31);
                const int out_hi = min(n, ring_hi);
                if (ring_hi > 0 && !warp_wait_geq(&cons[warp + 1], ring_hi - QS, &s_abort, L.spin_limit, L.err)) { s_abort = 1; break; }
                if (!loaded) {
                    // inputs of the sweep's first step (later steps prefetch the next one)
                    const int j = s0 - lane;
                    c = ((unsigned)j < (unsigned)n) ? min((int)bring[j & (QB - 1)], K) : K;
                    load_profile<R, PK, W * 32>(prow + c * HC * PB, pw);
                    top = rin[s0 & (QS - 1)];
                    loaded = true;
                }
                // steady state: every lane's column and the prefetched one are in [0, n); a task
                // entered from the matrix border also takes the first chunk this way, computing
                // the columns left of the task with the padding residue: that keeps a lane at the
                // border state (H = 0, E and F at -open, which give column 0 the same values)
                if ((s0 >= 31 || virt_ok) && s0 + CH + 1 <= n) {
                    // steady state: every lane's column and the prefetched one are in [0, n)
#pragma unroll UNR
                    for (int k = 0; k < CH; ++k) {
                        const int s = s0 + k;
                        const int cn = min((int)bring[(s + 1 - lane) & (QB - 1)], K);
                        const int2 topn = rin[(s + 1) & (QS - 1)];
                        uint32_t pwn[NPW];
                        load_profile<R, PK, W * 32>(prow + cn * HC * PB, pwn);
                        lane_step<R, MODE, PK, false, LOCAL>(st, pw, top, s, lane, n, go, ge, rout, tbw);
#pragma unroll
                        for (int q = 0; q < NPW; ++q) pw[q] = pwn[q];
                        top = topn;
                    }
                } else if (kEdgeFast && virt_ok) {
                    // the sweep's last steps (and short sweeps): a lane right of the task reads
                    // the padding residue and lane 0 an -inf row above, so every value such a
                    // lane computes stays below the task's best cell and never reaches a real
                    // one (lane l + 1 only reads lane l's column when it is its own); the steps
                    // need no per-lane bounds test.  Steps go in whole unrolled groups (a test
                    // inside the unrolled body would keep it from unrolling), so up to
                    // UNR - 1 steps run past the last one (n + 30) and lane 31 may write
                    // columns n .. n + UNR - 2 to the ring: the wait on the consumer above
                    // covers them.
                    for (int g = 0; g < CH; g += UNR) {
                        if (s0 + g >= n + 31) break;
#pragma unroll
                        for (int k = 0; k < UNR; ++k) {
                            const int s = s0 + g + k;
                            const int jn = s + 1 - lane;
                            const int cn = jn < n ? min((int)bring[jn & (QB - 1)], K) : K;
                            const int2 topn = s + 1 < n ? rin[(s + 1) & (QS - 1)] : make_int2(kNeg, kNeg);
                            uint32_t pwn[NPW];
                            load_profile<R, PK, W * 32>(prow + cn * HC * PB, pwn);
                            lane_step<R, MODE, PK, false, LOCAL>(st, pw, top, s, lane, n, go, ge, rout, tbw);
#pragma unroll
                            for (int q = 0; q < NPW; ++q) pw[q] = pwn[q];
                            top = topn;
                        }
                    }
                } else {
                    // traceback tiles and tasks with a left boundary: the first and last 31
                    // steps with the same prefetch, bounds-checked
#pragma unroll 1
                    for (int k = 0; k < CH; ++k) {
                        const int s = s0 + k;
                        if (s >= n + 31) break;
                        const int jn = s + 1 - lane;
                        const int cn = ((unsigned)jn < (unsigned)n) ? min((int)bring[jn & (QB - 1)], K) : K;
                        const int2 topn = rin[(s + 1) & (QS - 1)];   // stale when s + 1 >= n: lane 0 skips that column
                        uint32_t pwn[NPW];
                        load_profile<R, PK, W * 32>(prow + cn * HC * PB, pwn);
                        lane_step<R, MODE, PK, true, LOCAL>(st, pw, top, s, lane, n, go, ge, rout, tbw);
#pragma unroll
                        for (int q = 0; q < NPW; ++q) pw[q] = pwn[q];
                        top = topn;
                    }
                }
                if constexpr (MODE == kModeScoreCk) {
                    if (s0 + CH - 1 == next_ck && next_ck < n) {   // the same for every lane
                        const long long kk = (next_ck + 1) / T.colck_every - 1;
                        int2 *cc = T.colck + kk * T.colck_ld + (T.row0 + grow);
#pragma unroll
                        for (int r = 0; r < R; r += 2)
                            *reinterpret_cast<int4 *>(cc + r) = make_int4(st.U[r], st.E[r], st.U[r + 1], st.E[r + 1]);
                        T.colck_aux[kk * (T.colck_ld / R) + (T.row0 + grow) / R] = make_int2(st.udiag0, st.fb);
                        next_ck += T.colck_every;
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    sts_release(&cons[warp], min(n, s0 + CH));
                    if (out_hi > 0) sts_release(&prod[warp + 1], out_hi);
                }
            }

            if constexpr (MODE != kModeTb) {
                static_assert(kKeyRows == 16, "key decode assumes 4 row bits");
                int cs, cj, ci;
                if constexpr (LOCAL) {
                    const int br = R - 1 - (st.bk & (kKeyRows - 1));
                    cs = (st.bk >> 4) + go; cj = st.bj + 1; ci = T.row0 + grow + br + 1;
                    if (cs <= 0 || grow + br >= T.rows) { cs = 0; cj = 0x7fffffff; ci = 0x7fffffff; }
                } else {
                    // the best of the task's last row (semi-global, overlap), then the last
                    // column: every row for the overlap algorithm, the last row for the global one
                    cs = kNoScore; cj = 0x7fffffff; ci = 0x7fffffff;
                    if (st.track && st.bj >= 0) {
                        cs = (st.bk >> 4) + go; cj = st.bj + 1; ci = T.row0 + grow + st.rlast + 1;
                    }
                    const unsigned lastbit = st.rlast >= 0 ? 1u << st.rlast : 0u;
                    if (n > 0 && (SC.alg == kAlgOverlap || SC.alg == kAlgGlobal)) {
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            const bool end = SC.alg == kAlgOverlap ? grow + r < T.rows : ((lastbit >> r) & 1u);
                            const int sc = st.U[r] + go, ii = T.row0 + grow + r + 1;
                            if (end && cand_better(sc, n, ii, cs, cj, ci)) { cs = sc; cj = n; ci = ii; }
                        }
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const int os = __shfl_xor_sync(kFull, cs, off);
                    const int oj = __shfl_xor_sync(kFull, cj, off);
                    const int oi = __shfl_xor_sync(kFull, ci, off);
                    if (cand_better(os, oj, oi, cs, cj, ci)) { cs = os; cj = oj; ci = oi; }
                }
                if (lane == 0) s_cand[warp] = make_int4(cs, ci, cj, 0);
            }
        }
        __syncthreads();
        if constexpr (MODE != kModeTb) {
            if (threadIdx.x == 0) {
                int4 b = s_cand[0];
                for (int w = 1; w < W; ++w) {
                    const int4 o = s_cand[w];
                    if (cand_better(o.x, o.z, o.y, b.x, b.z, b.y)) b = o;
                }
                b.w = LOCAL ? (b.x > 0 ? 1 : 0) : (b.x != kNoScore ? 1 : 0);
                L.cand[slot] = b;
            }
        }
        __syncthreads();
    }
}

// Reduce the per-strip candidates of every task to one end cell:
// out[k] = (score, a_end, b_end, 0) with a_end/b_end the 1-based cell
// (= exclusive 0-based ends); local: all zero when the best score is 0;
// the other algorithms: the end cells on the matrix border are candidates
// too (a task is a whole pair there).
static __global__ void reduce_candidates_kernel(const FillTask *tasks, int ntasks, const int4 *cand,
                                                const DevScoring *scorings, int4 *out)
{
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= ntasks) return;
    const FillTask &T = tasks[k];
    const DevScoring &SC = scorings[T.scoring];
    const bool local = SC.alg == kAlgLocal;
    int cs = local ? 0 : kNoScore, cj = 0x7fffffff, ci = 0x7fffffff;
    for (int s = lane; s < T.nstrips; s += 32) {
        const int4 c = cand[T.ticket0 + s];
        if (c.w && cand_better(c.x, c.z, c.y, cs, cj, ci)) { cs = c.x; cj = c.z; ci = c.y; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const int os = __shfl_xor_sync(kFull, cs, off);
        const int oj = __shfl_xor_sync(kFull, cj, off);
        const int oi = __shfl_xor_sync(kFull, ci, off);
        if (cand_better(os, oj, oi, cs, cj, ci)) { cs = os; cj = oj; ci = oi; }
    }
    if (lane != 0) return;
    if (local) {
        out[k] = cs > 0 ? make_int4(cs, ci, cj, 0) : make_int4(0, 0, 0, 0);
    } else {
        border_end_candidates(SC.alg, T.rows, T.ncols, SC.go, SC.ge, &cs, &ci, &cj);
        out[k] = make_int4(cs, ci, cj, 0);
    }
}

}  // namespace swgb
