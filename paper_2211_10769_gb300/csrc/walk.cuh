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
// One warp walks.  Runs are taken 32 cells at a time: in state H the lanes
// read the 32 cells of the diagonal ahead and the walk jumps over the
// leading cells whose source is "diagonal"; in state E (F) they read the
// 32 cells to the left (above) and the walk jumps to the first one whose
// opened bit is set.  Only the run-ending cell is handled one at a time.
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

// The tiles recomputed in one round: a dense table over tile rows
// [I0, I0 + nI) and tile columns [J0, J0 + nJ); a null entry means the tile
// was not computed.  Words of a tile: [local row / R][local column], ld = BT.
template <typename Word>
struct TileTable {
    const Word *const *bits;   // nI * nJ entries
    int32_t I0, J0, nI, nJ;
    int32_t BT;                // tile side
    int32_t R;                 // rows per word
};

template <typename Word>
__device__ __forceinline__ const Word *tile_of(const TileTable<Word> &T, int i, int j) {
    const int I = (i - 1) / T.BT - T.I0, J = (j - 1) / T.BT - T.J0;
    if (I < 0 || J < 0 || I >= T.nI || J >= T.nJ) return nullptr;
    return T.bits[I * T.nJ + J];
}

// Decision nibble of cell (i, j) (1-based) inside its tile, or -1 if the tile is missing.
template <typename Word>
__device__ __forceinline__ int nibble_at(const TileTable<Word> &T, int i, int j) {
    const Word *b = tile_of(T, i, j);
    if (!b) return -1;
    const int li = (i - 1) % T.BT, lj = (j - 1) % T.BT;
    const Word w = __ldcg(b + (size_t)(li / T.R) * (size_t)T.BT + lj);
    return (int)((unsigned long long)w >> (4 * (li % T.R))) & 15;
}

template <typename Word>
__global__ void walk_kernel(const TileTable<Word> T, WalkState *st, int2 *runs, long long max_iters)
{
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    WalkState w = *st;
    auto emit = [&](int op, int cnt) {          // lane 0 only
        if (op == w.cur_op) { w.cur_len += cnt; return; }
        if (w.cur_len > 0) runs[w.nruns++] = make_int2(w.cur_op, w.cur_len);
        w.cur_op = op;
        w.cur_len = cnt;
    };
    long long it = 0;
    while (w.done == 0 && ++it < max_iters) {
        if (w.state == 0) {
            if (w.i == 0 || w.j == 0) { w.done = 1; break; }
            // lanes look at the diagonal (i - l, j - l)
            const int ci = w.i - lane, cj = w.j - lane;
            const int nb = (ci > 0 && cj > 0) ? nibble_at(T, ci, cj) : -2;   // -2: border
            const unsigned notdiag = __ballot_sync(kFull, nb < 0 || (nb & 3) != 1);
            const int k = notdiag ? __ffs(notdiag) - 1 : 32;   // leading diagonal cells
            const int nbk = __shfl_sync(kFull, nb, k & 31);
            if (lane == 0 && k > 0) emit(0, k);
            w.i -= k;
            w.j -= k;
            if (k == 32) continue;
            if (nbk == -2) { w.done = 1; break; }              // reached the border
            if (nbk == -1) break;                              // tile not computed: ask the host
            const int src = nbk & 3;
            if (src == 0) { w.done = 1; break; }
            w.state = (src == 2) ? 1 : 2;
        } else if (w.state == 1) {
            // lanes look left along the row: cells (i, j - l)
            const int cj = w.j - lane;
            const int nb = cj > 0 ? nibble_at(T, w.i, cj) : -2;
            const unsigned stop = __ballot_sync(kFull, nb < 0 || (nb & 4));
            const int k = stop ? __ffs(stop) - 1 : 32;          // cells that extend the gap
            const int nbk = __shfl_sync(kFull, nb, k & 31);
            if (k == 32) {
                if (lane == 0) emit(1, 32);
                w.j -= 32;
                continue;
            }
            if (nbk == -1) {                                   // missing tile: consume what was read
                if (lane == 0 && k > 0) emit(1, k);
                w.j -= k;
                break;
            }
            if (nbk == -2) { w.done = 2; break; }              // a gap cannot reach column 0
            if (lane == 0) emit(1, k + 1);                     // k extensions and the opening cell
            w.j -= k + 1;
            w.state = 0;
        } else {
            const int ci = w.i - lane;
            const int nb = ci > 0 ? nibble_at(T, ci, w.j) : -2;
            const unsigned stop = __ballot_sync(kFull, nb < 0 || (nb & 8));
            const int k = stop ? __ffs(stop) - 1 : 32;
            const int nbk = __shfl_sync(kFull, nb, k & 31);
            if (k == 32) {
                if (lane == 0) emit(2, 32);
                w.i -= 32;
                continue;
            }
            if (nbk == -1) {
                if (lane == 0 && k > 0) emit(2, k);
                w.i -= k;
                break;
            }
            if (nbk == -2) { w.done = 2; break; }
            if (lane == 0) emit(2, k + 1);
            w.i -= k + 1;
            w.state = 0;
        }
    }
    if (w.done == 0 && it >= max_iters) w.done = 2;
    if (lane == 0) {
        if (w.done == 1 && w.cur_len > 0) {
            runs[w.nruns++] = make_int2(w.cur_op, w.cur_len);
            w.cur_len = 0;
            w.cur_op = -1;
        }
        *st = w;
    }
}

}  // namespace swgb
