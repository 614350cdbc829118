// wavefront.cuh -- intra-task Smith-Waterman/Gotoh fill (paper Section 2.1:
// one matrix, all processing elements cooperate and pass border elements to
// their neighbours).
//
// Layout of the work.  A "task" is a range of rows of one pair (sequence a
// down the rows, b across the columns) swept over all of its columns.  It is
// cut into strips of HC = W*32*R rows; one thread block computes one strip
// at a time:
//   * each of its W compute warps owns 32*R consecutive rows, each lane R of
//     them, held in registers (H, H - open, E per row);
//   * lanes form an anti-diagonal wavefront: at warp step s lane t computes
//     column s - t, receiving the bottom H/F of lane t-1 for that column
//     by warp shuffle;
//   * warps hand their bottom row to the next warp through a shared-memory
//     ring, advancing in phases of CH steps separated by one block barrier;
//     warp w runs D = CH + 32 steps behind warp w-1, which is exactly what
//     the ring needs;
//   * an extra I/O warp moves the strip's top boundary row (H, F per column)
//     from global memory into the ring and the strip's bottom row out to
//     global memory, publishing its progress through a per-strip counter
//     with release/acquire semantics; the next strip polls that counter
//     (bounded spin) before reading.
// Strips are claimed in order from a global ticket counter, so a strip only
// ever waits on strips already held by running blocks.
//
// The substitution scores of the strip's rows are staged once per strip as
// a query profile in shared memory: prof[c*HC + r] = S(a_r, c), int8, with
// one extra padding residue c = K scoring -128 (used for columns outside
// the matrix; rows beyond the task also score -128).
//
// Modes: score (TB = false) tracks, per lane, the best H and its first
// column (then first row) and writes one end-cell candidate per strip;
// traceback (TB = true) writes, for every cell, four decision bits
// {H source: 0 zero, 1 diagonal, 2 E, 3 F; E opened; F opened} packed R
// nibbles per word, which a later walk follows.
#pragma once
#include "sw_device.cuh"

namespace swgb {

struct FillTask {
    const uint8_t *a;      // the task's rows: a[0 .. rows)
    const uint8_t *b;      // columns b[0 .. ncols)
    int32_t rows;
    int32_t ncols;
    int32_t nstrips;
    int32_t scoring;       // index into the scoring table
    int64_t ticket0;       // global ticket of strip 0
    const int2 *top;       // top boundary (H, F) per column, or null for the matrix border
    int2 *bnd;             // bottom rows of the strips: slot (strip % nslot) * ncols
    int32_t nslot;
    int32_t ckpt_every;    // also copy every ckpt_every-th strip's bottom row to ckpt (0 = never)
    int2 *ckpt;            // checkpoint rows: ((strip+1)/ckpt_every - 1) * ncols
    int32_t row0;          // row index (0-based, in the whole pair) of the task's first row
    int32_t pad_;
    void *tb;              // traceback words, TB mode: [row group][tb_ld]
    int64_t tb_ld;
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
};

template <int R> struct TbWord;
template <> struct TbWord<4> { using T = uint16_t; };
template <> struct TbWord<8> { using T = uint32_t; };
template <> struct TbWord<16> { using T = unsigned long long; };

template <int R>
__device__ __forceinline__ void load_profile(const int8_t *p, uint32_t (&w)[R / 4]) {
    if constexpr (R == 4) {
        w[0] = *reinterpret_cast<const uint32_t *>(p);
    } else if constexpr (R == 8) {
        uint2 v = *reinterpret_cast<const uint2 *>(p);
        w[0] = v.x; w[1] = v.y;
    } else {
        uint4 v = *reinterpret_cast<const uint4 *>(p);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
}

template <int r>
__device__ __forceinline__ int prof_score(const uint32_t *w) {
    return sext8<r % 4>(w[r / 4]);
}

template <int R, int W, bool TB>
__global__ void __launch_bounds__((W + 1) * 32)
wavefront_kernel(const FillLaunch L)
{
    constexpr int HC = W * 32 * R;
    constexpr int CH = 16;
    constexpr int D = CH + 32;
    constexpr int QS = 64;
    static_assert(QS >= 2 * CH + 1, "ring too small");

    extern __shared__ __align__(16) int8_t prof[];   // (K + 1) * HC
    __shared__ int2 chan[W + 1][QS];
    __shared__ long long s_tk;
    __shared__ int s_task;
    __shared__ int s_abort;
    __shared__ int4 s_cand[W];

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const bool io = (warp == W);

    int H[R], U[R], E[R];

    for (;;) {
        if (threadIdx.x == 0) {
            long long tk = (long long)atomicAdd(L.ticket, 1ULL);
            if (ld_volatile(L.err) != 0) tk = L.total;       // stop early after an error
            s_tk = tk;
            s_abort = 0;
            if (tk < L.total) {
                int lo = 0, hi = L.ntasks - 1;               // last task with ticket0 <= tk
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (L.tasks[mid].ticket0 <= tk) lo = mid; else hi = mid - 1;
                }
                s_task = lo;
            }
        }
        __syncthreads();
        const long long tk = s_tk;
        if (tk >= L.total) return;
        const FillTask &T = L.tasks[s_task];
        const DevScoring &SC = L.scorings[T.scoring];
        const int K = SC.K, go = SC.go, ge = SC.ge;
        const int strip = (int)(tk - T.ticket0);
        const int rbase = strip * HC;                   // first row of the strip within the task
        const int n = T.ncols;
        const uint8_t *__restrict__ bseq = T.b;

        // ---- query profile of the strip's rows
        for (int lr = threadIdx.x; lr < HC; lr += blockDim.x) {
            const int r = rbase + lr;
            const bool ok = r < T.rows;
            const int av = ok ? min((int)T.a[r], K - 1) : 0;
            for (int c = 0; c <= K; ++c)
                prof[c * HC + lr] = (ok && c < K) ? SC.mat[av * K + c] : (int8_t)kPadScore;
        }

        // ---- per-lane state
        int hb = 0, fb = kNeg, hprev = 0;
        int best = 0, bj = -1, br = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) { H[r] = 0; U[r] = -go; E[r] = kNeg; }
        const int lrow = (warp * 32 + lane) * R;            // first row of this lane within the strip
        const int8_t *prow = prof + lrow;

        // I/O helpers
        auto load_cols = [&](int lo2, int hi2) -> bool {
            if (hi2 <= lo2) return true;
            if (strip == 0) {
                for (int col = lo2 + lane; col < hi2; col += 32)
                    chan[0][col & (QS - 1)] = T.top ? __ldcg(T.top + col) : make_int2(0, kNeg);
                return true;
            }
            bool ok = true;
            if (lane == 0) {
                const int *pf = L.prog + (tk - 1);
                long long it = 0;
                while (ld_acquire(pf) < hi2) {
                    if (++it > L.spin_limit || ld_volatile(L.err) != 0) {
                        atomicCAS(L.err, 0, kErrTimeout);
                        ok = false;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            ok = __shfl_sync(kFull, ok ? 1 : 0, 0) != 0;
            if (!ok) return false;
            const int2 *src = T.bnd + (size_t)((strip - 1) % T.nslot) * n;
            for (int col = lo2 + lane; col < hi2; col += 32)
                chan[0][col & (QS - 1)] = __ldcg(src + col);
            return true;
        };

        if (io) {
            if (!load_cols(0, min(n, CH))) s_abort = 1;
        }
        __syncthreads();

        const int nphase = (n + 30 + (W - 1) * D) / CH + 2;
        for (int p = 0; p < nphase && !s_abort; ++p) {
            if (!io) {
                const int s0 = p * CH - warp * D;
#pragma unroll 2
                for (int k = 0; k < CH; ++k) {
                    const int s = s0 + k;
                    if (s < 0 || s >= n + 31) continue;         // warp-uniform
                    const int j = s - lane;
                    const bool colok = (unsigned)j < (unsigned)n;
                    int hup = __shfl_up_sync(kFull, hb, 1);
                    int fup = __shfl_up_sync(kFull, fb, 1);
                    if (lane == 0) {
                        const int2 v = chan[warp][j & (QS - 1)];
                        hup = v.x; fup = v.y;
                    }
                    const int c = colok ? min((int)bseq[j], K) : K;   // codes >= K are flagged by the validation kernel
                    uint32_t pw[R / 4];
                    load_profile<R>(prow + c * HC, pw);
                    int hdiag = hprev;
                    hprev = hup;
                    int f = fup;
                    int uu = hup - go;
                    typename TbWord<R>::T word = 0;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        int sr;
                        switch (r % 4) {
                            case 0: sr = sext8<0>(pw[r / 4]); break;
                            case 1: sr = sext8<1>(pw[r / 4]); break;
                            case 2: sr = sext8<2>(pw[r / 4]); break;
                            default: sr = sext8<3>(pw[r / 4]); break;
                        }   // r is a constant after unrolling, so this folds to one prmt
                        const int eopen = U[r];                    // H(i,j-1) - open
                        const int e = __viaddmax_s32(E[r], -ge, eopen);
                        const int fopen = uu;                      // H(i-1,j) - open
                        f = __viaddmax_s32(f, -ge, fopen);
                        const int hn = __viaddmax_s32_relu(hdiag, sr, max(e, f));
                        if constexpr (TB) {
                            const int diag = hdiag + sr;
                            unsigned src = hn == 0 ? 0u : (hn == diag ? 1u : (hn == e ? 2u : 3u));
                            unsigned nib = src | ((e == eopen) ? 4u : 0u) | ((f == fopen) ? 8u : 0u);
                            word |= (typename TbWord<R>::T)nib << (4 * r);
                        }
                        E[r] = e;
                        hdiag = H[r];
                        H[r] = hn;
                        uu = hn - go;
                        U[r] = uu;
                    }
                    hb = H[R - 1];
                    fb = f;
                    if (lane == 31 && colok) chan[warp + 1][j & (QS - 1)] = make_int2(hb, fb);
                    if constexpr (TB) {
                        if (colok) {
                            auto *tbw = reinterpret_cast<typename TbWord<R>::T *>(T.tb);
                            tbw[(size_t)((rbase + lrow) / R) * (size_t)T.tb_ld + j] = word;
                        }
                    } else {
                        int cm = H[0];
#pragma unroll
                        for (int r = 1; r + 1 < R; r += 2) cm = __vimax3_s32(cm, H[r], H[r + 1]);
                        if constexpr (R % 2 == 0) cm = max(cm, H[R - 1]);
                        if (colok && cm > best) {
                            best = cm;
                            bj = j;
                            int rr = R - 1;
#pragma unroll
                            for (int r = R - 1; r >= 0; --r) if (H[r] == cm) rr = r;
                            br = rr;
                        }
                    }
                }
            } else {
                // store the bottom-row columns warp W-1 produced in the previous phase
                if (p >= 1) {
                    const int lo = min(n, max(0, (p - 1) * CH - (W - 1) * D - 31));
                    const int hi = min(n, max(0, p * CH - (W - 1) * D - 31));
                    if (hi > lo) {
                        int2 *dst = T.bnd + (size_t)(strip % T.nslot) * n;
                        const bool ck = T.ckpt_every > 0 && ((strip + 1) % T.ckpt_every) == 0;
                        int2 *cdst = ck ? T.ckpt + (size_t)((strip + 1) / T.ckpt_every - 1) * n : nullptr;
                        for (int col = lo + lane; col < hi; col += 32) {
                            const int2 v = chan[W][col & (QS - 1)];
                            dst[col] = v;
                            if (ck) cdst[col] = v;
                        }
                        __threadfence();
                        __syncwarp();
                        if (lane == 0) st_release(L.prog + tk, hi);
                    }
                }
                // fetch warp 0's top-boundary columns for the next phase
                if (!load_cols(min(n, (p + 1) * CH), min(n, (p + 2) * CH))) s_abort = 1;
            }
            __syncthreads();
        }

        if constexpr (!TB) {
            // ---- end-cell candidate of the strip: best score, then first column, then first row
            int cs = best, cj = bj + 1, ci = T.row0 + rbase + lrow + br + 1;
            if (io || best <= 0 || rbase + lrow + br >= T.rows) { cs = 0; cj = 0x7fffffff; ci = 0x7fffffff; }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const int os = __shfl_xor_sync(kFull, cs, off);
                const int oj = __shfl_xor_sync(kFull, cj, off);
                const int oi = __shfl_xor_sync(kFull, ci, off);
                if (cand_better(os, oj, oi, cs, cj, ci)) { cs = os; cj = oj; ci = oi; }
            }
            if (lane == 0 && !io) s_cand[warp] = make_int4(cs, ci, cj, 0);
            __syncthreads();
            if (threadIdx.x == 0) {
                int4 b = s_cand[0];
                for (int w = 1; w < W; ++w) {
                    const int4 o = s_cand[w];
                    if (cand_better(o.x, o.z, o.y, b.x, b.z, b.y)) b = o;
                }
                b.w = b.x > 0 ? 1 : 0;
                L.cand[tk] = b;
            }
        }
        __syncthreads();
    }
}

// Reduce the per-strip candidates of every task to one end cell:
// out[k] = (score, a_end, b_end, 0) with a_end/b_end the 1-based cell
// (= exclusive 0-based ends), all zero when the best score is 0.
static __global__ void reduce_candidates_kernel(const FillTask *tasks, int ntasks, const int4 *cand,
                                         int4 *out)
{
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= ntasks) return;
    const FillTask &T = tasks[k];
    int cs = 0, cj = 0x7fffffff, ci = 0x7fffffff;
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
    if (lane == 0) out[k] = cs > 0 ? make_int4(cs, ci, cj, 0) : make_int4(0, 0, 0, 0);
}

}  // namespace swgb
