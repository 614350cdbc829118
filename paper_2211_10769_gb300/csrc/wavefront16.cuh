// wavefront16.cuh -- intra-task Smith-Waterman/Gotoh fill of one pair in
// packed 16-bit lanes (paper Section 2.1: one matrix, all processing
// elements cooperate and pass border elements to their neighbours).
//
// The block layout is the one of wavefront.cuh (W compute warps per strip of
// W*32*R rows, an input and an output warp, strips chained through a global
// boundary-row ring), but every lane holds two wavefront positions, packed
// into the two 16-bit halves of its registers:
//
//   * lane t owns rows [tR, tR + R) of its warp; the top half, rows
//     [tR, tR + R/2), lives in the low 16 bits and at step s computes column
//     s - 2t; the bottom half, rows [tR + R/2, tR + R), lives in the high
//     16 bits and computes column s - 2t - 1;
//   * the bottom half's row above is this lane's top half one step earlier
//     (a register); the top half's is lane t-1's bottom half one step
//     earlier (a shuffle), or the strip's boundary row for lane 0;
//   * so one __viaddmax_s16x2 advances two cells, and the vertical
//     dependency chain of a step is R/2 packed operations long.
//
// Values are kept multiplied by 8 (scores and penalties scaled by 8: the
// recurrence is linear, so every H, E and F is scaled by 8 too), which frees
// the low 3 bits of every value for a row tag when the end cell is tracked.
//
// Exact 16-bit values.  H is Lipschitz along rows and columns:
// H(i-1,j) - o <= H(i,j) <= H(i-1,j) + o + max(S, 0) (the same along j), and
// E, F and H + S stay within o + e + |S| of a neighbouring H.  Every value a
// lane touches during one chunk of kP16CH steps sits within D = R + kP16CH + 6 rows
// plus columns of its top half's first row, so all of them lie within
// 8 (D (o + max S) + o + e + |min S| + max S) of that reference, in scaled
// units (p16_spread).  Each lane keeps a base B (a multiple of 8; absolute =
// B + stored value) and, at every chunk boundary, sets B = max(0, ref -
// kP16Center) rounded down to a multiple of 8, shifting its registers by the
// change.  With the spread below kP16Span:
//   * B = 0: values are absolute, the 0 floor of H is the hardware relu;
//   * B > 0: every value of the lane lies in (0, 32767 - 8), so the relu
//     never fires -- as in the true recurrence, where every such H is above
//     B > 0.
// A value shuffled in from lane t-1 is moved from its base to this lane's by
// one packed add; lane 0 converts the absolute boundary row; lane 31 writes
// absolute values.  The strips exchange absolute rows (scaled in shared
// memory, plain int32 in global memory), so the result does not depend on
// the bases.
//
// End cell without branches.  The key of packed row k is its value OR a
// tag 7 - k in the low 3 bits: the maximum key of a column is the largest
// value and, among equal ones, the earliest row.  Each half keeps its best
// key and the column where that key first appeared (a strictly larger key
// replaces it: a larger score, or the same score in an earlier row); the
// best is kept absolute in int32 across chunk boundaries, so a base change
// never loses it.
//
// Query profile: for small alphabets a pair profile, one packed word per
// (residue of the top half, residue of the bottom half) and packed row; else
// an int16 profile whose two words per packed row are merged with one prmt.
//
// Modes: score (end-cell candidate per strip) and score with checkpoints
// (strip bottom rows, and staircase checkpoint columns in the two-positions
// form that FillTask::left_split describes).
#pragma once
#include "wavefront.cuh"

namespace swgb {

constexpr int kNeg16p = -16384;     // -infinity of a packed 16-bit lane
constexpr int kP16Center = 16384;   // stored value of a lane's reference once B > 0
constexpr int kP16Span = 16000;     // largest scaled value spread (p16_spread) the packed fill accepts
constexpr int kP16QS = 512;         // boundary-ring columns per channel
constexpr int kP16Pos = 64;         // wavefront positions per warp (two per lane)
constexpr int kP16Shift = 3;        // values are multiplied by 2^3
constexpr int kP16CH = 32;          // steps per chunk (hand-off, base change; 16 measured slower)

// Profile kinds of the packed fill.
enum P16Prof { kP16Pair = 0, kP16Int16 = 1 };

// Bound on the spread, in scaled units, of all values a lane touches during
// one chunk (see the header); the packed fill is exact when it is below
// kP16Span.
inline long long p16_spread(int R, int go, int ge, int max_s, int min_s) {
    const long long L = (long long)go + (max_s > 0 ? max_s : 0);
    const long long D = (long long)R + kP16CH + 6;
    const long long neg = -min_s > 128 ? -min_s : 128;          // padding residues score -128
    return 8 * (D * L + go + ge + neg + (max_s > 0 ? max_s : 0));
}

// Bytes of the packed fill's query profile for K residue codes.
inline size_t p16_profile_bytes(int R, int W, int K, int pk) {
    const size_t HC = (size_t)W * 32 * R;
    return pk == kP16Pair ? (size_t)(K + 1) * (K + 1) * (HC / 2) * 4 : (size_t)(K + 1) * HC * 2;
}

__device__ __forceinline__ unsigned p16_pack(int lo, int hi) {
    return (unsigned)(lo & 0xffff) | ((unsigned)hi << 16);
}
__device__ __forceinline__ int p16_lo(unsigned v) { return (int)(short)(v & 0xffffu); }
__device__ __forceinline__ int p16_hi(unsigned v) { return (int)v >> 16; }

__device__ __forceinline__ unsigned prmt_r(unsigned a, unsigned b, unsigned sel) {
    unsigned d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// low half = 16-bit half ha of a, high half = 16-bit half hb of b
template <int ha, int hb>
__device__ __forceinline__ unsigned p16_halves(uint32_t a, uint32_t b) {
    constexpr uint32_t sel = (2 * ha) | ((2 * ha + 1) << 4) | ((4 + 2 * hb) << 8) | ((5 + 2 * hb) << 12);
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "n"(sel));
    return d;
}

// Profile words of one step, R/2 per lane.  Pair profile: the lane's packed
// words for (top residue, bottom residue).  int16 profile: the lane's R
// scores at the top half's residue; the bottom half uses the previous step's.
//
// Pair profile layout: combination cc = c_top * (K + 1) + c_bottom, lane g of
// NL, packed rows 2q, 2q+1 as one 8-byte chunk at word ((cc*(R/4) + q)*NL + g)*2
// (conflict-free 8-byte loads).  int16 layout: row r of the strip at
// prof16[c * HC + r].
template <int R, int PK, int NL>
__device__ __forceinline__ void p16_load(const int8_t *p, uint32_t (&w)[R / 2]) {
    if constexpr (PK == kP16Pair) {
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const uint2 v = *reinterpret_cast<const uint2 *>(p + (size_t)q * NL * 8);
            w[2 * q] = v.x; w[2 * q + 1] = v.y;
        }
    } else if constexpr (R == 8 || R == 16) {
#pragma unroll
        for (int q = 0; q < R / 8; ++q) {
            const uint4 v = *reinterpret_cast<const uint4 *>(p + 16 * q);
            w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const uint2 v = *reinterpret_cast<const uint2 *>(p + 8 * q);
            w[2 * q] = v.x; w[2 * q + 1] = v.y;
        }
    }
}

// Scaled score pair 8 (S + open) of packed row k.
template <int R, int PK>
__device__ __forceinline__ unsigned p16_score(const uint32_t (&cur)[R / 2], const uint32_t (&prev)[R / 2], int k) {
    if constexpr (PK == kP16Pair) {
        return cur[k];
    } else {
        constexpr int H = R / 2;
        const int kb = H + k;        // bottom half's row k is lane row R/2 + k
        switch ((k & 1) * 2 + (kb & 1)) {   // constants after unrolling: one prmt
            case 0: return p16_halves<0, 0>(cur[k >> 1], prev[kb >> 1]);
            case 1: return p16_halves<0, 1>(cur[k >> 1], prev[kb >> 1]);
            case 2: return p16_halves<1, 0>(cur[k >> 1], prev[kb >> 1]);
            default: return p16_halves<1, 1>(cur[k >> 1], prev[kb >> 1]);
        }
    }
}

// Per-lane state.  U = 8 (H - open) and E (scaled) of the lane's R/2 packed
// rows relative to the lane base B; ub the last packed row's U after the
// previous step and fb the F of the row below it, max(F - extend, U) (the
// first row's F of the half below, so the next step starts its F chain from
// it); udiag0 the packed row above the two halves at their previous columns.  Tracking: the best key per half relative to B
// (packed, valid inside a chunk) and absolute (int32, across chunks), and the
// column where it first appeared.
template <int R>
struct P16Lane {
    unsigned U[R / 2], E[R / 2];
    unsigned ub, fb, udiag0;
    unsigned flast;                 // F of each half's last row (fb is the F of the row below)
    unsigned kbest;
    int B;                          // lane base
    unsigned din2;                  // (lane t-1's base minus this one, 0); (0, 0) for lane 0
    int best[2], bcol[2];
};

// One step of one lane: column j = s - 2 lane (top half) and j - 1 (bottom
// half).  TAIL drops the keys of columns at or past n (the sweep's last steps
// run on padding residues); the first steps need no mask because columns
// left of the task hold the border state (H = 0), which is never a best.
template <int R, int PK, int QS, bool TAIL>
__device__ __forceinline__ void p16_step(P16Lane<R> &st, const uint32_t (&pw)[R / 2], const uint32_t (&pwp)[R / 2],
                                         uint2 top, int s, int lane, int n, unsigned nge2, unsigned ngo2,
                                         unsigned neg2, int2 *rout)
{
    constexpr int H = R / 2;
    const int j = s - 2 * lane;
    const unsigned su = __shfl_up_sync(kFull, st.ub, 1);
    const unsigned sf = __shfl_up_sync(kFull, st.fb, 1);
    // lane 0: the row above is the strip's boundary row, already in lane 0's base and in the
    // high halves (p16_top_row)
    const unsigned srcu = lane == 0 ? top.x : su;
    const unsigned srcf = lane == 0 ? top.y : sf;
    // low half: the row above the top half at j (the high half of the source, moved from
    // lane t-1's base to this one); high half: this lane's top half's last row at j - 1.
    // fb carries F of the row below a half's last row, so f is already the first row's F.
    const unsigned uup = __viaddmax_s16x2(prmt_r(srcu, st.ub, 0x5432u), st.din2, neg2);
    unsigned f = __viaddmax_s16x2(prmt_r(srcf, st.fb, 0x5432u), st.din2, neg2);
    unsigned udiag = st.udiag0;
    st.udiag0 = uup;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        const unsigned sp = p16_score<R, PK>(pw, pwp, k);           // 8 (S + open) of both cells
        const unsigned uold = st.U[k];
        const unsigned e = __viaddmax_s16x2(st.E[k], nge2, uold);
        const unsigned x = __viaddmax_s16x2_relu(udiag, sp, e);    // max(H(i-1,j-1) + S, E, 0)
        const unsigned xgo = __viaddmax_s16x2(x, ngo2, neg2);      // x - open
        const unsigned u = __viaddmax_s16x2(f, ngo2, xgo);         // H - open
        st.E[k] = e;
        udiag = uold;
        st.U[k] = u;
        if (k + 1 < H) f = __viaddmax_s16x2(f, nge2, xgo);         // F of the next row
        else st.fb = __viaddmax_s16x2(f, nge2, xgo);                // F of the row below the half
    }
    st.ub = st.U[H - 1];
    st.flast = f;
    if (lane == 31)      // the warp's bottom row (H - open, F) at column s - 63, scaled absolute
        rout[(j - 1) & (QS - 1)] = make_int2(p16_hi(st.ub) + st.B, p16_hi(f) + st.B);
    // keys: value | (7 - k) in both halves; the column's largest key
    // (the low 3 bits of a scaled value are 0, so adding the tag sets them without a carry: an
    // integer add, which the FMA pipe takes, instead of an OR on the busier ALU pipe)
    unsigned ck = __vimax3_s16x2(st.U[0] + 0x00070007u, st.U[1] + 0x00060006u, st.U[2] + 0x00050005u);
#pragma unroll
    for (int k = 3; k < H; k += 2) {
        const unsigned t0 = (unsigned)(7 - k) * 0x00010001u;
        const int k1 = k + 1 < H ? k + 1 : k;
        const unsigned t1 = (unsigned)(7 - k1) * 0x00010001u;
        ck = __vimax3_s16x2(ck, st.U[k] + t0, st.U[k1] + t1);
    }
    if (TAIL) ck = p16_pack(j < n ? p16_lo(ck) : -32768, j - 1 < n ? p16_hi(ck) : -32768);
    bool ph, pl;
    st.kbest = __vibmax_s16x2(st.kbest, ck, &ph, &pl);             // kept where best >= key
    st.bcol[0] = pl ? st.bcol[0] : j;
    st.bcol[1] = ph ? st.bcol[1] : j - 1;
}

// A task that starts right of a checkpoint column written by this fill (the
// two-positions staircase of the checkpoint mode, FillTask::left_split):
// lane l's top half holds its rows at column -1 - 2l and its bottom half at
// -2 - 2l (task columns), which is exactly the wavefront's state after step
// -1.  The lane takes that state (scaled by 8, in a base of its own) and the
// sweep goes on from step 0; its first steps recompute real columns left of
// the task from real residues (the residue ring's slots left of column 0).
template <int R>
__device__ __forceinline__ void p16_enter_staircase(const FillTask &T, P16Lane<R> &st, int grow, int lane, int go,
                                                    int ge) {
    constexpr int H = R / 2;
    int vU[R], vE[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int2 v = make_int2(-go, kNeg);
        if (grow + r < T.rows) v = __ldcg(T.left + grow + r);
        vU[r] = v.x;
        vE[r] = v.y;
    }
    const bool in = grow < T.rows;
    const int2 at = in ? __ldcg(T.left_aux + grow / H) : make_int2(-go, kNeg);       // top half
    const int2 ab = in ? __ldcg(T.left_aux + grow / H + 1) : make_int2(-go, kNeg);   // bottom half
    // absolute values scaled by 8 (-infinity clamped first so that scaling cannot overflow), then
    // relative to the lane's base, -infinity at kNeg16p
    auto scaled = [](int v) { return max(v, -(1 << 20)) * 8; };
    const int B = max(0, scaled(vU[0]) - kP16Center) & ~7;
    auto rel = [&](int v) { return max(scaled(v) - B, kNeg16p); };
#pragma unroll
    for (int k = 0; k < H; ++k) {
        st.U[k] = p16_pack(rel(vU[k]), rel(vU[H + k]));
        st.E[k] = p16_pack(rel(vE[k]), rel(vE[H + k]));
    }
    st.udiag0 = p16_pack(rel(at.x), rel(ab.x));
    st.flast = p16_pack(rel(at.y), rel(ab.y));
    st.ub = st.U[H - 1];
    // F of the row below each half's last row: max(F - extend, H - open) of that row
    st.fb = __viaddmax_s16x2(st.flast, p16_pack(-8 * ge, -8 * ge), st.U[H - 1]);
    st.B = B;
    const int bup = __shfl_up_sync(kFull, B, 1);
    st.din2 = lane == 0 ? 0u : p16_pack(bup - B, 0);
    // the best keys in the new base (H = 0 with the largest tag, never a best), kept above -32768
    st.kbest = p16_pack(max(st.best[0] - B, -32768), max(st.best[1] - B, -32768));
}

// Lane 0's row above at one step, from the strip's boundary row v (scaled,
// absolute: H - open and F): both taken to lane 0's base B0 and into the high
// halves, the F as the first row's F, max(F - extend, H - open).
__device__ __forceinline__ uint2 p16_top_row(int2 v, int B0, int ge8) {
    const int tu = __viaddmax_s32(v.x, -B0, kNeg16p);
    const int tf = __viaddmax_s32(__viaddmax_s32(v.y, -ge8, v.x), -B0, kNeg16p);
    return make_uint2((unsigned)tu << 16, (unsigned)tf << 16);
}

// Steps per unrolled body of the steady loop, measured on GB300 (2, 4, 8, 16, 32 at 12 rows a lane): 8 for
// the score fill; 16 with checkpoints above 8 rows a lane (its chunk-end code runs once per 16 steps); 32
// is much slower (a body that large no longer stays in the instruction cache).
constexpr int fill16_unroll(int R, int MODE) { return (R <= 8 || MODE == kModeScore) ? 8 : 16; }

// LEFT: the tasks may start right of a checkpoint column written by this fill
// (p16_enter_staircase; the coarse-tile refills of a two-level reconstruction).
// A separate instantiation, so that the others compile exactly without it.
template <int R, int W, int MODE, int PK, bool LEFT = false>
__global__ void __launch_bounds__((W + 2) * 32, 1)
wavefront16_kernel(const FillLaunch L)
{
    static_assert(R % 4 == 0 && R >= 8 && R <= 16, "two halves of at most 8 rows (3-bit tags)");
    static_assert(MODE == kModeScore || MODE == kModeScoreCk, "score modes only");
    constexpr int H = R / 2;
    constexpr int HC = W * 32 * R;
    constexpr int NL = W * 32;
    constexpr int CH = kP16CH, QS = kP16QS, QB = kQB, IOB = kIOB;
    constexpr int LAG = kP16Pos - 1;                 // lane 31's bottom half trails lane 0's top half
    static_assert(QS >= 2 * IOB + 2 * CH + 2 * kP16Pos, "ring too small");
    constexpr int UNR = fill16_unroll(R, MODE);
    static_assert(CH % UNR == 0, "chunks are whole unrolled groups");

    extern __shared__ __align__(16) int8_t prof[];   // p16_profile_bytes
    __shared__ int2 ring[W + 1][QS];                 // (8 (H - open), 8 F), absolute
    __shared__ uint8_t bring[QB];
    __shared__ int s_poff[PK == kP16Pair ? QB : 1];   // pair profile: byte offset per column (fill_input_warp)
    __shared__ int prod[W + 1];
    __shared__ int cons[W + 1];
    __shared__ long long s_tk;
    __shared__ int s_task, s_strip;
    __shared__ volatile int s_abort;
    __shared__ int4 s_cand[W];
    __shared__ uint2 s_top[W][CH];                   // lane 0's rows above for one chunk (p16_top_row)
    static_assert(CH <= 32 && (CH & (CH - 1)) == 0, "one boundary entry a lane, a power of two");

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
        const int SH = SW * 32 * R;
        const int rbase = strip * SH;
        const int n = T.ncols;
        const int Wa = min(SW, (T.rows - rbase + 32 * R - 1) / (32 * R));

        // ---- query profile of the strip's rows: 8 (S(a_r, c) + open), padding at 8 * -128
        if constexpr (PK == kP16Pair) {
            const int ncc = (K + 1) * (K + 1);
            uint32_t *pw32 = reinterpret_cast<uint32_t *>(prof);
            for (int idx = threadIdx.x; idx < ncc * NL * H; idx += blockDim.x) {
                const int k = idx % H, g = (idx / H) % NL, cc = idx / (H * NL);
                const int ct = cc / (K + 1), cb = cc % (K + 1);
                const int rt = g * R + k, rb = g * R + H + k;
                const bool okt = rt < SH && rbase + rt < T.rows && ct < K;
                const bool okb = rb < SH && rbase + rb < T.rows && cb < K;
                const int vt = okt ? 8 * (SC.mat[min((int)T.a[rbase + rt], K - 1) * K + ct] + go) : 8 * kPadScore;
                const int vb = okb ? 8 * (SC.mat[min((int)T.a[rbase + rb], K - 1) * K + cb] + go) : 8 * kPadScore;
                pw32[((cc * (R / 4) + (k >> 1)) * NL + g) * 2 + (k & 1)] = p16_pack(vt, vb);
            }
        } else {
            int16_t *p16 = reinterpret_cast<int16_t *>(prof);
            for (int idx = threadIdx.x; idx < (K + 1) * HC; idx += blockDim.x) {
                const int lr = idx % HC, c = idx / HC;
                const bool ok = lr < SH && rbase + lr < T.rows && c < K;
                p16[idx] = (int16_t)(ok ? 8 * (SC.mat[min((int)T.a[rbase + lr], K - 1) * K + c] + go) : 8 * kPadScore);
            }
        }
        // the residue ring's last kP16Pos slots hold the columns left of the task (down to -64),
        // which lanes compute during their first two chunks: padding at the matrix border;
        // the input warp reaches those slots only after the last warp has published a column,
        // i.e. left those chunks
        // bytes per profile entry: pair, per residue combination; int16, per residue
        const int pstride = PK == kP16Pair ? (R / 4) * NL * 8 : 2 * HC;
        // (a task entered from a checkpoint column: the real residues of those columns)
        if (threadIdx.x < kP16Pos) {
            const int j = (int)threadIdx.x - kP16Pos;                       // column -64 .. -1
            const bool real = LEFT && T.left;
            const int cj = real ? min((int)T.b[j], K) : K;
            bring[QB - kP16Pos + threadIdx.x] = (uint8_t)cj;
            if constexpr (PK == kP16Pair) {
                const int cjm = real ? min((int)T.b[j - 1], K) : K;
                s_poff[QB - kP16Pos + threadIdx.x] = (cj * (K + 1) + cjm) * pstride;
            }
        }
        __syncthreads();

        if (warp == W) {
            fill_input_warp<QS, QB, IOB, kP16Shift>(T, L, strip, slot, n, go, K, Wa, kP16Pos + 1, ring[0], bring,
                                                    prod, cons, &s_abort, lane, kAlgLocal, 0,
                                                    PK == kP16Pair ? s_poff : nullptr, K + 1, pstride);
        } else if (warp == W + 1) {
            fill_output_warp<QS, kP16Shift>(T, L, strip, slot, n, go, SH, Wa, ring[Wa], prod, cons, &s_abort, lane);
        } else if (warp >= Wa) {
            if (lane == 0) s_cand[warp] = make_int4(0, 0x7fffffff, 0x7fffffff, 0);
        } else {
            // ================= compute warp =================
            const int g = warp * 32 + lane;
            const int grow = rbase + g * R;
            // this lane's profile base (pair: its first chunk of combination 0; int16: its rows)
            const int8_t *prow = PK == kP16Pair ? prof + g * 8 : prof + 2 * g * R;
            const unsigned ngo2 = p16_pack(-8 * go, -8 * go), nge2 = p16_pack(-8 * ge, -8 * ge);
            const unsigned neg2 = p16_pack(kNeg16p, kNeg16p);
            P16Lane<R> st;
#pragma unroll
            for (int k = 0; k < H; ++k) { st.U[k] = ngo2; st.E[k] = neg2; }
            st.ub = ngo2; st.fb = ngo2; st.flast = neg2; st.udiag0 = ngo2;   // matrix border: H = 0
            st.B = 0; st.din2 = 0;
            // H = 0 with the largest tag: never replaced by H = 0, always by H > 0
            st.best[0] = st.best[1] = -8 * go + 7;
            st.bcol[0] = st.bcol[1] = -1;
            st.kbest = p16_pack(st.best[0], st.best[1]);
            if constexpr (LEFT)
                if (T.left) p16_enter_staircase<R>(T, st, grow, lane, go, ge);   // (a two-positions staircase)
            int next_ck = (MODE == kModeScoreCk && T.colck && T.colck_every > 0) ? T.colck_every - 1 : 0x7fffffff;
            int2 *rin = ring[warp];
            int2 *rout = ring[warp + 1];
            int seen_in = 0;
            bool loaded = false;
            uint32_t pw[R / 2], pwp[R / 2];
            if constexpr (PK == kP16Pair || !LEFT) {
#pragma unroll
                for (int q = 0; q < R / 2; ++q) pwp[q] = p16_pack(8 * kPadScore, 8 * kPadScore);
            } else {
                // the int16 profile's bottom half takes the previous step's words: at step 0 those
                // of column -1 - 2 lane (padding, or a real residue left of a checkpoint column)
                p16_load<R, PK, NL>(prow + min((int)bring[(-1 - 2 * lane) & (QB - 1)], K) * pstride, pwp);
            }
            uint2 top;
            for (int s0 = 0; s0 < n + LAG; s0 += CH) {
                const int need_in = min(n, s0 + CH + 1);
                if (need_in > seen_in) {
                    if (!warp_wait_geq(&prod[warp], need_in, &s_abort, L.spin_limit, L.err)) { s_abort = 1; break; }
                    seen_in = need_in;
                }
                const int ring_hi = max(0, s0 + CH - LAG);
                const int out_hi = min(n, ring_hi);
                if (ring_hi > 0 && !warp_wait_geq(&cons[warp + 1], ring_hi - QS, &s_abort, L.spin_limit, L.err)) { s_abort = 1; break; }
                if (!loaded) {
                    const int c = min((int)bring[(s0 - 2 * lane) & (QB - 1)], K);
                    if constexpr (PK == kP16Pair) {
                        // the bottom halves' column is left of the task: padding, or (LEFT) a real residue
                        if constexpr (LEFT) p16_load<R, PK, NL>(prow + s_poff[(s0 - 2 * lane) & (QB - 1)], pw);
                        else p16_load<R, PK, NL>(prow + (c * (K + 1) + K) * pstride, pw);
                    } else {
                        p16_load<R, PK, NL>(prow + c * pstride, pw);
                    }
                    loaded = true;
                }
                {   // new lane base from the top half's first row at its last column; the best
                    // keys go through their absolute copies
                    const int oldB = st.B;
                    if constexpr (LEFT) {   // (-32768: no key since the staircase entry put the best below the base)
                        if (p16_lo(st.kbest) > -32768) st.best[0] = max(st.best[0], p16_lo(st.kbest) + oldB);
                        if (p16_hi(st.kbest) > -32768) st.best[1] = max(st.best[1], p16_hi(st.kbest) + oldB);
                    } else {
                        st.best[0] = max(st.best[0], p16_lo(st.kbest) + oldB);
                        st.best[1] = max(st.best[1], p16_hi(st.kbest) + oldB);
                    }
                    const int ref = p16_lo(st.U[0]) + oldB;
                    const int Bn = max(0, ref - kP16Center) & ~7;
                    const unsigned d2 = p16_pack(oldB - Bn, oldB - Bn);
#pragma unroll
                    for (int k = 0; k < H; ++k) {
                        st.U[k] = __viaddmax_s16x2(st.U[k], d2, neg2);
                        st.E[k] = __viaddmax_s16x2(st.E[k], d2, neg2);
                    }
                    st.ub = __viaddmax_s16x2(st.ub, d2, neg2);
                    st.fb = __viaddmax_s16x2(st.fb, d2, neg2);
                    st.flast = __viaddmax_s16x2(st.flast, d2, neg2);
                    st.udiag0 = __viaddmax_s16x2(st.udiag0, d2, neg2);
                    st.B = Bn;
                    const int bup = __shfl_up_sync(kFull, Bn, 1);
                    st.din2 = lane == 0 ? 0u : p16_pack(bup - Bn, 0);
                    if constexpr (LEFT)
                        st.kbest = p16_pack(max(min(st.best[0] - Bn, 32767), -32768), max(min(st.best[1] - Bn, 32767), -32768));
                    else
                        st.kbest = p16_pack(min(st.best[0] - Bn, 32767), min(st.best[1] - Bn, 32767));
                }
                {   // lane 0's rows above for the chunk's steps, taken to its new base once per
                    // chunk (one entry a lane) rather than once per step; entries at or past n
                    // read as -infinity.  The wait above made entries below s0 + CH + 1 ready.
                    const int B0 = __shfl_sync(kFull, st.B, 0);
                    __syncwarp();
                    if (lane < CH) {
                        const int sk = s0 + lane;
                        const int2 v = sk < n ? rin[sk & (QS - 1)] : make_int2(kNeg, kNeg);
                        s_top[warp][lane] = p16_top_row(v, B0, -p16_lo(nge2));
                    }
                    __syncwarp();
                    top = s_top[warp][0];
                }
                if (s0 + CH + 1 <= n) {
                    // steady state: lane 0's prefetched column stays inside the task; columns
                    // left of the task (first chunks) compute the border state on padding
#pragma unroll UNR
                    for (int k = 0; k < CH; ++k) {
                        const int s = s0 + k;
                        const uint2 topn = s_top[warp][(k + 1) & (CH - 1)];   // (unused after the last step)
                        uint32_t pwn[R / 2];
                        if constexpr (PK == kP16Pair) {
                            p16_load<R, PK, NL>(prow + s_poff[(s + 1 - 2 * lane) & (QB - 1)], pwn);
                        } else {
                            const int cn = min((int)bring[(s + 1 - 2 * lane) & (QB - 1)], K);
                            p16_load<R, PK, NL>(prow + cn * pstride, pwn);
                        }
                        p16_step<R, PK, QS, false>(st, pw, pwp, top, s, lane, n, nge2, ngo2, neg2, rout);
#pragma unroll
                        for (int q = 0; q < R / 2; ++q) { pwp[q] = pw[q]; pw[q] = pwn[q]; }
                        top = topn;
                    }
                } else {
                    // the sweep's last steps: columns past n read the padding residue and lane 0
                    // an -inf row above; their keys are dropped.  Whole unrolled groups: up to
                    // UNR - 1 steps past the last one (n + 62), whose ring writes past n the
                    // wait on the consumer above covers.
                    for (int gs = 0; gs < CH; gs += UNR) {
                        if (s0 + gs >= n + LAG) break;
#pragma unroll
                        for (int k = 0; k < UNR; ++k) {
                            const int s = s0 + gs + k;
                            const int jn = s + 1 - 2 * lane;
                            const int cn = jn < n ? min((int)bring[jn & (QB - 1)], K) : K;
                            const uint2 topn = s_top[warp][(gs + k + 1) & (CH - 1)];
                            uint32_t pwn[R / 2];
                            if constexpr (PK == kP16Pair) {   // the bottom half's residue: column jn - 1
                                const int cb = jn - 1 < n ? min((int)bring[(jn - 1) & (QB - 1)], K) : K;
                                p16_load<R, PK, NL>(prow + (cn * (K + 1) + cb) * pstride, pwn);
                            } else {
                                p16_load<R, PK, NL>(prow + cn * pstride, pwn);
                            }
                            p16_step<R, PK, QS, true>(st, pw, pwp, top, s, lane, n, nge2, ngo2, neg2, rout);
#pragma unroll
                            for (int q = 0; q < R / 2; ++q) { pwp[q] = pw[q]; pw[q] = pwn[q]; }
                            top = topn;
                        }
                    }
                }
                if constexpr (MODE == kModeScoreCk) {
                    if (s0 + CH - 1 == next_ck && next_ck < n) {   // the same for every lane
                        // staircase in the two-positions form: the top half's rows at column
                        // next_ck - 2 lane, the bottom half's at next_ck - 2 lane - 1; unscaled
                        const long long kk = (next_ck + 1) / T.colck_every - 1;
                        int2 *cc = T.colck + kk * T.colck_ld + (T.row0 + grow);
                        const int B = st.B;
#pragma unroll
                        for (int k = 0; k < H; k += 2) {
                            *reinterpret_cast<int4 *>(cc + k) =
                                make_int4((p16_lo(st.U[k]) + B) >> 3, (p16_lo(st.E[k]) + B) >> 3,
                                          (p16_lo(st.U[k + 1]) + B) >> 3, (p16_lo(st.E[k + 1]) + B) >> 3);
                            *reinterpret_cast<int4 *>(cc + H + k) =
                                make_int4((p16_hi(st.U[k]) + B) >> 3, (p16_hi(st.E[k]) + B) >> 3,
                                          (p16_hi(st.U[k + 1]) + B) >> 3, (p16_hi(st.E[k + 1]) + B) >> 3);
                        }
                        int2 *ca = T.colck_aux + kk * (T.colck_ld / H) + (T.row0 + grow) / H;
                        ca[0] = make_int2((p16_lo(st.udiag0) + B) >> 3, (p16_lo(st.flast) + B) >> 3);
                        ca[1] = make_int2((p16_hi(st.udiag0) + B) >> 3, (p16_hi(st.flast) + B) >> 3);
                        next_ck += T.colck_every;
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    sts_release(&cons[warp], min(n, s0 + CH));
                    if (out_hi > 0) sts_release(&prod[warp + 1], out_hi);
                }
            }
            if (!LEFT || p16_lo(st.kbest) > -32768) st.best[0] = max(st.best[0], p16_lo(st.kbest) + st.B);
            if (!LEFT || p16_hi(st.kbest) > -32768) st.best[1] = max(st.best[1], p16_hi(st.kbest) + st.B);

            // the lane's candidate: the better of its halves (top rows come first)
            int cs = 0, cj = 0x7fffffff, ci = 0x7fffffff;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int key = st.best[h];
                const int row = grow + h * H + (7 - (key & 7));      // tag 7 - k gives row k of the half
                const int sc = (key >> 3) + go;                      // the value's multiple of 8, unscaled
                if (sc > 0 && row < T.rows && cand_better(sc, st.bcol[h] + 1, T.row0 + row + 1, cs, cj, ci)) {
                    cs = sc; cj = st.bcol[h] + 1; ci = T.row0 + row + 1;
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
        __syncthreads();
        if (threadIdx.x == 0) {
            int4 b = s_cand[0];
            for (int w = 1; w < W; ++w) {
                const int4 o = s_cand[w];
                if (cand_better(o.x, o.z, o.y, b.x, b.z, b.y)) b = o;
            }
            b.w = b.x > 0 ? 1 : 0;
            L.cand[slot] = b;
        }
        __syncthreads();
    }
}

}  // namespace swgb
