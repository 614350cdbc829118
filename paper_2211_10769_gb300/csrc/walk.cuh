// walk.cuh -- the traceback walk over recomputed decision bits (paper
// Section 2.2, reconstruction phase).
//
// The matrix is cut into square tiles of BT x BT cells.  A round of the
// reconstruction recomputes the decision bits of a set of tiles (a band
// around the path) and this kernel walks the canonical path through them:
//
//   state H: stop if the H source is zero; diagonal -> emit M, go up-left;
//            source E -> state E; source F -> state F;
//   state E: emit I, go left; back to H if the E-opened bit is set;
//   state F: emit D, go up; back to H if the F-opened bit is set.
//
// The walk is a chain of dependent lookups, so it reads them from shared
// memory: a window of the decision words that follows the diagonal through
// the walk's cell (kWinRows rows above it, kWinCols columns per row group,
// kWinRight of them right of the diagonal).  Warp 0 walks inside one window
// while warps 1..8 stage the next one in a second buffer: the same band
// continued above the first, which is where a walk that follows the
// diagonal leaves it.  Where the walk left the window elsewhere (a long
// gap drifts it off the diagonal), the next window is staged at its cell
// while it waits.
//
// One warp walks.  Runs are taken 64 cells at a time: in state H the lanes
// read the cells of the diagonal ahead and the walk jumps over the leading
// cells whose source is "diagonal"; in state E (F) they read the cells to
// the left (above) and the walk jumps to the first one whose opened bit is
// set.  Only the run-ending cell is handled one at a time.
// The walk stops when it reaches a zero cell or the border (done = 1), or
// when its next cell lies in a tile that was not recomputed this round
// (done = 0, the host computes that tile next).
#pragma once
#include "sw_device.cuh"

namespace swgb {

struct WalkState {
    int32_t i, j;          // current cell (1-based rows / columns; 0 = border)
    int32_t state;         // 0 = H, 1 = E, 2 = F
    int32_t done;          // 0 running / needs tiles, 1 finished, 2 inconsistent bits
    int64_t nruns;         // run records written so far
    int32_t cur_op;        // op of the open run (0 = M, 1 = I, 2 = D, -1 = none)
    int32_t cur_len;
};

// The tiles recomputed in one round: for each tile row I in [I0, I0 + nI), a
// window of nJ tile columns that follows the diagonal, [J0 + (I - I0),
// J0 + (I - I0) + nJ); a null entry means the tile was not computed.  Words of
// a tile: [local row / R][local column], ld = BT.
template <typename Word>
struct TileTable {
    const Word *const *bits;   // nI * nJ entries
    int32_t I0, J0, nI, nJ;
    int32_t BT;                // tile side
    int32_t R;                 // rows per word
    int32_t win_groups;        // row groups of a window (walk_window_groups)
};

constexpr int kLook = 2;              // groups of 32 cells each lane reads ahead per iteration
constexpr int kWalkTableMax = 4096;   // tile-table entries cached in shared memory
constexpr int kWinRows = 768;         // rows of a window (a multiple of every R)
constexpr int kWinCols = 128;         // columns a window keeps per row group
constexpr int kWinRight = 64;         // ... of them right of the diagonal through the walk's cell
constexpr int kStageThreads = 256;    // threads staging a window (warps 1..8)
constexpr int kWalkThreads = 32 + kStageThreads;   // warp 0 walks
constexpr int kStage = 16;            // window words a thread loads at once
constexpr int kWinMargin = 16;        // columns a staged window must leave either side of the walk's cell
constexpr int kWalkMinBT = 256;       // tiles at least this side

// Row groups of a window on tiles of side BT: its rows, and its band of
// columns ((groups - 1) R + kWinCols wide), each within BT, so that a window
// meets 2 x 2 tiles at most (768 rows on tiles of 1,024 and more).
__host__ __device__ constexpr int walk_min3(int a, int b, int c) { return a < b ? (a < c ? a : c) : (b < c ? b : c); }
__host__ __device__ constexpr int walk_window_groups(int BT, int R) {
    return walk_min3(kWinRows / R, BT / R, (BT - kWinCols) / R + 1);
}

template <int R>
constexpr size_t walk_window_bytes(size_t word_bytes) { return 2 * (size_t)(kWinRows / R) * kWinCols * word_bytes; }

// Where a window lies (all coordinates 0-based).  Row groups g = 0 .. ng-1
// hold rows r_lo + g*R .. r_lo + g*R + R - 1 (r_lo a multiple of R); group
// g keeps columns [clo(g), clo(g) + kWinCols) with clo(g) = chi - (ng-1-g)*R,
// so the kept band slides along the diagonal.  The window meets at most two
// tile rows (the second from window row lrb on) and two tile columns (the
// second from column cb on); tile (x, y) starts at row rbase[x], column
// cbase[y], its words are tp[2x + y] and bit 2x + y of pres says whether it
// was recomputed.
struct WalkWindow {
    int r_lo, ng, chi;
    int lrb, cb;
    int rbase[2], cbase[2];
    int pres;
    const void *tp[4];
};

template <typename Word>
__device__ __forceinline__ const Word *tile_ptr(const TileTable<Word> &T, const Word *const *tiles, int I, int J) {
    const int ti = I - T.I0, tj = J - (T.J0 + ti);
    return (ti >= 0 && tj >= 0 && ti < T.nI && tj < T.nJ) ? tiles[ti * T.nJ + tj] : nullptr;
}

// The window whose last row group is ghi (>= 0) and keeps columns from chi
// on in that group.
template <typename Word, int R>
__device__ WalkWindow make_window_g(const TileTable<Word> &T, const Word *const *tiles, int ghi, int chi) {
    const int RG = T.win_groups;
    constexpr int kNone = 0x7fffffff;
    WalkWindow m;
    const int glo = max(0, ghi - (RG - 1));
    m.ng = ghi - glo + 1;
    m.r_lo = glo * R;
    m.chi = chi;
    const int BT = T.BT;
    const int ia = m.r_lo / BT, ib = (ghi * R + R - 1) / BT;
    m.lrb = ib > ia ? ib * BT - m.r_lo : kNone;
    const int cmin = max(0, m.chi - (m.ng - 1) * R), cmax = max(0, m.chi + kWinCols - 1);
    const int ja = cmin / BT, jb = cmax / BT;
    m.cb = jb > ja ? jb * BT : kNone;
    m.rbase[0] = ia * BT; m.rbase[1] = ib * BT;
    m.cbase[0] = ja * BT; m.cbase[1] = jb * BT;
    m.pres = 0;
    for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) {
            const Word *b = tile_ptr(T, tiles, x ? ib : ia, y ? jb : ja);
            m.tp[2 * x + y] = b;
            if (b) m.pres |= 1 << (2 * x + y);
        }
    return m;
}

// The window whose last row group holds the walk's cell (r0, c0), with that
// cell kWinRight columns left of the group's last kept column.
template <typename Word, int R>
__device__ WalkWindow make_window(const TileTable<Word> &T, const Word *const *tiles, int r0, int c0) {
    r0 = max(r0, 0);
    c0 = max(c0, 0);
    return make_window_g<Word, R>(T, tiles, r0 / R, c0 - (kWinCols - 1 - kWinRight));
}

// Whether window m holds the cell (r0, c0) at least kWinMargin columns from
// either side of its band.
template <int R>
__device__ __forceinline__ bool window_holds(const WalkWindow &m, int r0, int c0) {
    const int rr = r0 - m.r_lo;
    if (m.ng <= 0 || rr < 0 || rr >= m.ng * R) return false;
    const int k = c0 - m.chi + (m.ng - 1 - rr / R) * R;
    return k >= kWinMargin && k < kWinCols - kWinMargin;
}

// Stage window m into win: staging thread t (of kStageThreads) takes column
// k = t % kWinCols of every kStageThreads / kWinCols-th row group, kStage
// independent loads in flight at a time.
template <typename Word, int R>
__device__ __forceinline__ void stage_window(const TileTable<Word> &T, const WalkWindow &m, Word *win, int t) {
    constexpr int kGroupsPerPass = kStageThreads / kWinCols;
    static_assert(kStageThreads % kWinCols == 0, "whole row groups per pass");
    const int k = t % kWinCols;
    for (int g0 = t / kWinCols; g0 < m.ng; g0 += kStage * kGroupsPerPass) {
        Word v[kStage];
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const int g = g0 + u * kGroupsPerPass;
            const int c = m.chi - (m.ng - 1 - g) * R + k;
            const int x = g * R >= m.lrb, y = c >= m.cb;
            const Word *b = static_cast<const Word *>(x ? (y ? m.tp[3] : m.tp[2]) : (y ? m.tp[1] : m.tp[0]));
            const int rb = x ? m.rbase[1] : m.rbase[0], cbs = y ? m.cbase[1] : m.cbase[0];
            v[u] = 0;
            if (g < m.ng && c >= 0 && b)              // a row group never straddles tiles (BT % R == 0)
                v[u] = __ldcg(b + (size_t)((m.r_lo + g * R - rb) / R) * (size_t)T.BT + (size_t)(c - cbs));
        }
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const int g = g0 + u * kGroupsPerPass;
            if (g < m.ng) win[g * kWinCols + k] = v[u];
        }
    }
}

// Decision nibble of the cell p steps back along (di, dj) from the walk's
// cell (r0, c0) = (i - 1, j - 1): -2 at the matrix border, -3 outside the
// window, -1 in a tile that was not recomputed.  lr0 = r0 - m.r_lo.  Without
// branches: early returns made the lanes of the walker's warp diverge on its
// dependency chain (2.01 -> 1.53 ms a 200 kbp alignment without them).
template <typename Word, int R>
__device__ __forceinline__ int window_nibble(const WalkWindow &m, const Word *win, int lr0, int c0, int di, int dj, int p) {
    // every lane loads a word, clamped into the window (rr < ng R always: the walk starts
    // inside the window and only moves up), and the special cases are selected after
    const int rr = lr0 - di * p, c = c0 - dj * p;
    const int rrc = max(rr, 0);
    const int g = (int)((unsigned)rrc / R);
    const int k = c - m.chi + (m.ng - 1 - g) * R;
    const bool border = rr + m.r_lo < 0 || c < 0;
    const bool outside = rr < 0 || (unsigned)k >= (unsigned)kWinCols;
    const bool missing = !((m.pres >> (2 * (rrc >= m.lrb) + (c >= m.cb))) & 1);
    const int kc = min(max(k, 0), kWinCols - 1);
    const Word w = win[g * kWinCols + kc];
    const int nib = (int)((unsigned long long)w >> (4 * (rrc - g * R))) & 15;
    return border ? -2 : (outside ? -3 : (missing ? -1 : nib));
}

// The walk's start taken from the end cell reduced on the device (res: score,
// row, column), for an alignment done in one round without a round trip to
// the host: the end cell in state H, or nothing to walk (done = 3, parked at
// cell (1, 1), a cell every window can hold) when the local score is 0 or the
// end cell lies on the border.
static __global__ void walk_start_kernel(const int4 *res, int local, WalkState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int4 r = *res;
    WalkState w{r.y, r.z, 0, 0, 0, -1, 0};
    if ((local && r.x <= 0) || r.y <= 0 || r.z <= 0) { w.i = 1; w.j = 1; w.done = 3; }
    *st = w;
}

template <typename Word, int R>
__global__ void __launch_bounds__(kWalkThreads, 1) walk_kernel(const TileTable<Word> T, WalkState *st, int2 *runs,
                                                          long long max_iters)
{
    static_assert(kWinRows % R == 0, "a window holds whole row groups");
    constexpr int kWinWords = (kWinRows / R) * kWinCols;
    extern __shared__ __align__(16) unsigned char walk_smem[];
    Word *s_buf = reinterpret_cast<Word *>(walk_smem);   // two windows
    __shared__ const Word *s_tiles[kWalkTableMax];
    __shared__ WalkState s_w;
    __shared__ WalkWindow s_mw[2];
    __shared__ int s_stop, s_redo;
    if (blockIdx.x != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntab = T.nI * T.nJ;
    if (ntab > kWalkTableMax || T.BT < kWalkMinBT || T.win_groups < 1 || T.win_groups > kWinRows / R ||
        T.win_groups != walk_window_groups(T.BT, R)) {   // the host keeps bands, tiles and windows within these
        if (threadIdx.x == 0) st->done = 2;
        return;
    }
    for (int k = threadIdx.x; k < ntab; k += blockDim.x) s_tiles[k] = T.bits[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        s_w = *st;
        s_stop = s_w.done != 0;
        s_mw[0] = make_window<Word, R>(T, s_tiles, s_w.i - 1, s_w.j - 1);
    }
    __syncthreads();
    if (warp > 0 && !s_stop) stage_window<Word, R>(T, s_mw[0], s_buf, threadIdx.x - 32);
    __syncthreads();
    long long it = 0;                                    // walk iterations (warp 0)
    int cur = 0;
    while (!s_stop) {
        const int nxt = cur ^ 1;
        if (threadIdx.x == 0) {
            // the band continued above the current window (none above the first row)
            const WalkWindow &m = s_mw[cur];
            WalkWindow p{};
            if (m.r_lo > 0) p = make_window_g<Word, R>(T, s_tiles, m.r_lo / R - 1, m.chi - m.ng * R);
            else p.ng = 0;
            s_mw[nxt] = p;
        }
        __syncthreads();
        if (warp > 0) {
            if (s_mw[nxt].ng > 0) stage_window<Word, R>(T, s_mw[nxt], s_buf + nxt * kWinWords, threadIdx.x - 32);
        } else {
            const Word *s_win = s_buf + cur * kWinWords;
            const WalkWindow m = s_mw[cur];
            WalkState w = s_w;
            // every lane keeps the same (uniform) run state; lane 0 stores the records
            auto emit = [&](int op, int cnt) {
                if (op == w.cur_op) { w.cur_len += cnt; return; }
                if (w.cur_len > 0) {
                    if (lane == 0) runs[w.nruns] = make_int2(w.cur_op, w.cur_len);
                    ++w.nruns;
                }
                w.cur_op = op;
                w.cur_len = cnt;
            };
            bool stop = false;                           // back to the host (or finished)
            while (true) {                               // (w.done is 0 here: every exit that sets it breaks)
                if (++it >= max_iters) { w.done = 2; stop = true; break; }
                if (w.state == 0 && (w.i == 0 || w.j == 0)) { w.done = 1; stop = true; break; }
                // the next 32 * kLook cells of the run: the diagonal in state H, the row to
                // the left in state E, the column above in state F
                const int di = w.state == 1 ? 0 : 1, dj = w.state == 2 ? 0 : 1;
                const int mask = w.state == 0 ? 3 : (w.state == 1 ? 4 : 8);
                const int lr0 = w.i - 1 - m.r_lo, c0 = w.j - 1;
                int nb[kLook];
#pragma unroll
                for (int q = 0; q < kLook; ++q)
                    nb[q] = window_nibble<Word, R>(m, s_win, lr0, c0, di, dj, q * 32 + lane);
                // first cell that ends the run: in H a source other than "diagonal", in E / F
                // the opened bit; the window's edge, a missing tile or the border ends it too.
                // Both votes at once, one 64-bit scan, one shuffle: no loop, no divergence.
                static_assert(kLook == 2, "the scan below reads two groups of 32 cells");
                const bool end0 = nb[0] < 0 || (w.state == 0 ? (nb[0] & 3) != 1 : (nb[0] & mask) != 0);
                const bool end1 = nb[1] < 0 || (w.state == 0 ? (nb[1] & 3) != 1 : (nb[1] & mask) != 0);
                const unsigned long long ends = (unsigned long long)__ballot_sync(kFull, end0) |
                                                ((unsigned long long)__ballot_sync(kFull, end1) << 32);
                const int pos = ends ? __ffsll((long long)ends) - 1 : 64;
                const int nbk = __shfl_sync(kFull, pos >= 32 ? nb[1] : nb[0], pos & 31);
                const int op = w.state;                  // M, I or D runs of states H, E, F
                if (pos == 64) {                         // the whole look-ahead continues the run
                    emit(op, pos);
                    w.i -= di * pos;
                    w.j -= dj * pos;
                    continue;
                }
                if (nbk == -3) {                         // the window's edge: take what was read
                    if (pos > 0) emit(op, pos);
                    w.i -= di * pos;
                    w.j -= dj * pos;
                    break;                               // the next window starts here
                }
                if (w.state == 0) {
                    if (pos > 0) emit(0, pos);
                    w.i -= pos;
                    w.j -= pos;
                    if (nbk == -2) { w.done = 1; stop = true; break; }   // reached the border
                    if (nbk == -1) { stop = true; break; }              // tile not computed: ask the host
                    const int src = nbk & 3;
                    if (src == 0) { w.done = 1; stop = true; break; }
                    w.state = (src == 2) ? 1 : 2;
                } else {
                    if (nbk == -1) {                     // missing tile: consume what was read
                        if (pos > 0) emit(op, pos);
                        w.i -= di * pos;
                        w.j -= dj * pos;
                        stop = true;
                        break;
                    }
                    if (nbk == -2) { w.done = 2; stop = true; break; }  // a gap cannot reach the border
                    emit(op, pos + 1);                   // the extensions and the opening cell
                    w.i -= di * (pos + 1);
                    w.j -= dj * (pos + 1);
                    w.state = 0;
                }
            }
            if (lane == 0) {
                s_w = w;
                s_stop = stop;
            }
        }
        __syncthreads();
        if (s_stop) break;
        // the staged window serves if it holds the walk's cell with room to both sides
        if (threadIdx.x == 0) {
            s_redo = !window_holds<R>(s_mw[nxt], s_w.i - 1, s_w.j - 1);
            if (s_redo) s_mw[nxt] = make_window<Word, R>(T, s_tiles, s_w.i - 1, s_w.j - 1);
        }
        __syncthreads();
        if (s_redo) {
            if (warp > 0) stage_window<Word, R>(T, s_mw[nxt], s_buf + nxt * kWinWords, threadIdx.x - 32);
            __syncthreads();
        }
        cur = nxt;
    }
    if (threadIdx.x == 0) {
        WalkState w = s_w;
        if (w.done == 1 && w.cur_len > 0) {
            runs[w.nruns++] = make_int2(w.cur_op, w.cur_len);
            w.cur_len = 0;
            w.cur_op = -1;
        }
        *st = w;
    }
}

}  // namespace swgb
