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
// One warp walks.  Runs are taken 64 cells at a time (each lane issues
// two loads at once, so their latencies overlap): in state H the lanes
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

constexpr int kLook = 2;           // groups of 32 cells each lane reads ahead per iteration (2 measured
                                   // best of 1..16: runs are short, wasted look-ahead costs issue time)
constexpr int kWalkTableMax = 4096;   // tile-table entries cached in shared memory

// Where the walk is: its cell's tile (absolute tile row / column) and the
// cell's offsets inside that tile.  One division per iteration.
struct WalkPos {
    int I, J, li, lj;
};

// Decision nibble of the cell p steps back along (di, dj) from the walk's
// cell, -2 at the matrix border, -1 in a tile that was not computed.  The
// look-ahead (< BT) crosses at most one tile edge per direction.  The load
// is unconditional (a cell without bits reads the valid word `dummy`
// instead), so the loads of all look-ahead cells can be in flight together.
template <typename Word, int R>
__device__ __forceinline__ int nibble_back(const TileTable<Word> &T, const Word *const *tiles, const WalkPos &P,
                                           int i, int j, int di, int dj, int p, const Word *dummy) {
    const int ci = i - di * p, cj = j - dj * p;
    int I = P.I, J = P.J, li = P.li - di * p, lj = P.lj - dj * p;
    if (li < 0) { li += T.BT; --I; }
    if (lj < 0) { lj += T.BT; --J; }
    I -= T.I0;
    J -= T.J0;
    const bool border = ci <= 0 || cj <= 0;
    const bool inside = !border && I >= 0 && J >= 0 && I < T.nI && J < T.nJ;
    const Word *b = inside ? tiles[I * T.nJ + J] : nullptr;
    const bool have = b != nullptr;
    const int lr = have ? li : 0;
    const Word *addr = have ? b + (size_t)(lr / R) * (size_t)T.BT + lj : dummy;
    const Word w = __ldcg(addr);
    const int nib = (int)((unsigned long long)w >> (4 * (lr % R))) & 15;
    return border ? -2 : (have ? nib : -1);
}

template <typename Word, int R>
__global__ void walk_kernel(const TileTable<Word> T, WalkState *st, int2 *runs, long long max_iters)
{
    __shared__ const Word *s_tiles[kWalkTableMax];
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const int ntab = T.nI * T.nJ;
    if (ntab > kWalkTableMax) {                          // the host keeps bands smaller than this
        if (lane == 0) st->done = 2;
        return;
    }
    for (int k = lane; k < ntab; k += 32) s_tiles[k] = T.bits[k];
    __syncwarp();
    WalkState w = *st;
    auto emit = [&](int op, int cnt) {          // lane 0 only
        if (op == w.cur_op) { w.cur_len += cnt; return; }
        if (w.cur_len > 0) runs[w.nruns++] = make_int2(w.cur_op, w.cur_len);
        w.cur_op = op;
        w.cur_len = cnt;
    };
    long long it = 0;
    while (w.done == 0 && ++it < max_iters) {
        if (w.state == 0 && (w.i == 0 || w.j == 0)) { w.done = 1; break; }
        // the next 32 * kLook cells of the run: the diagonal in state H, the row to the
        // left in state E, the column above in state F; all loads are issued at once
        const int di = w.state == 1 ? 0 : 1, dj = w.state == 2 ? 0 : 1;
        const int mask = w.state == 0 ? 3 : (w.state == 1 ? 4 : 8);
        WalkPos P;
        P.I = (max(w.i, 1) - 1) / T.BT;
        P.J = (max(w.j, 1) - 1) / T.BT;
        P.li = (w.i - 1) - P.I * T.BT;
        P.lj = (w.j - 1) - P.J * T.BT;
        int nb[kLook];
#pragma unroll
        for (int q = 0; q < kLook; ++q)
            nb[q] = nibble_back<Word, R>(T, s_tiles, P, w.i, w.j, di, dj, q * 32 + lane,
                                         reinterpret_cast<const Word *>(st));
        // first cell that ends the run: in H a source other than "diagonal", in E / F
        // the opened bit; a missing tile or the border ends it too
        int pos = 32 * kLook, nbk = 0;
#pragma unroll
        for (int q = 0; q < kLook; ++q) {
            const bool end = nb[q] < 0 || (w.state == 0 ? (nb[q] & 3) != 1 : (nb[q] & mask) != 0);
            const unsigned ends = __ballot_sync(kFull, end);
            if (ends) {
                const int k = __ffs(ends) - 1;
                pos = q * 32 + k;
                nbk = __shfl_sync(kFull, nb[q], k);
                break;
            }
        }
        const int op = w.state;                          // M, I or D runs of states H, E, F
        if (pos == 32 * kLook) {                         // the whole look-ahead continues the run
            if (lane == 0) emit(op, pos);
            w.i -= di * pos;
            w.j -= dj * pos;
            continue;
        }
        if (w.state == 0) {
            if (lane == 0 && pos > 0) emit(0, pos);
            w.i -= pos;
            w.j -= pos;
            if (nbk == -2) { w.done = 1; break; }        // reached the border
            if (nbk == -1) break;                        // tile not computed: ask the host
            const int src = nbk & 3;
            if (src == 0) { w.done = 1; break; }
            w.state = (src == 2) ? 1 : 2;
        } else {
            if (nbk == -1) {                             // missing tile: consume what was read
                if (lane == 0 && pos > 0) emit(op, pos);
                w.i -= di * pos;
                w.j -= dj * pos;
                break;
            }
            if (nbk == -2) { w.done = 2; break; }        // a gap cannot reach the border
            if (lane == 0) emit(op, pos + 1);            // the extensions and the opening cell
            w.i -= di * (pos + 1);
            w.j -= dj * (pos + 1);
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
