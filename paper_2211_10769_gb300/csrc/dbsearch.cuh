// dbsearch.cuh -- inter-task database search (paper Section 2.1: many
// matrices at once, no communication between processing elements), packed
// 16-bit lanes with exact 32-bit rescoring of saturating subjects, and the
// top-k selection of the hits.
//
// One warp aligns the query against two database subjects at once: the low
// 16 bits of every register belong to subject A, the high 16 bits to
// subject B (the database is sorted by length, so the two have nearly the
// same length).  The query runs down the warp: lane t owns R query rows of
// the current pass of 32*R rows; lanes form an anti-diagonal wavefront over
// the subjects' columns exactly as in the pairwise fill (bottom H / F to the
// next lane by shuffle), and longer queries take several passes, the bottom
// row of one pass feeding the next through a per-warp boundary row in
// global memory.  Short queries may instead run two independent 16-lane
// wavefronts per warp (G = 16), each over its own pair of subjects, so that a
// lane holds more rows of a short query and the skew of a wavefront is 15
// steps rather than 31.  The query profile (int8, S + open, all passes) sits in
// shared memory; the two residues' score bytes are merged into one packed
// register with a single prmt.  The cell update is the pairwise one in
// __viaddmax_s16x2 / __viaddmax_s16x2_relu form.
//
// Exactness of 16-bit lanes: every H value is exact while all H values of
// the subject stay <= T = 32767 - max(S) (the largest intermediate is
// H + S, E and F never drop below -open - extend - 16384).  The first cell
// whose H exceeds T is still exact and raises the running maximum above T,
// so a subject whose maximum exceeds T is flagged and rescored in 32 bits;
// all other scores are exact.
#pragma once
#include "sw_device.cuh"

namespace swgb {

constexpr int kNeg16 = -16384;

struct DbJob {
    const uint8_t *q;          // query codes (device)
    int32_t m;                 // query length
    int32_t scoring;           // index into the scoring table
    int32_t pair0, pair1;      // pairs pair0, pair0 + stride, ... below pair1 of the sorted database
    int32_t pair_stride;
    int32_t block0;            // first block of the launch working on this job (prefix over jobs)
    int32_t *scores;           // per subject (original index): score, or -1 when flagged
    int32_t *ovf;              // flagged subject ids
    int32_t *novf;             // their count
    int32_t *next_pair;        // work counter (zeroed before launch)
};

struct DbView {
    const uint8_t *res;        // all residues
    const int64_t *off;        // subject s = res[off[s] .. off[s+1])
    const int32_t *pairs;      // pair p = subjects pairs[2p], pairs[2p+1] (-1 = none)
    const uint16_t *pres;      // pair p's residues interleaved, column j at pres[poff[p] + j]:
    const int64_t *poff;       // low byte subject A, high byte subject B, 0xff past a subject's end;
                               // n_p = poff[p+1] - poff[p] - 1 columns plus one padding column
    int32_t npairs;
    int32_t maxlen;            // longest subject (scratch rows hold maxlen + 1 entries)
    // scratch slots: one per block that can be resident at a time (nslots = SMs x blocks per
    // SM); block b < nslots uses slot b, a later block (an oversubscribed grid) takes a slot a
    // finished block has released
    unsigned *slot_pool;       // bit set = slot taken; slots < min(grid, nslots) and >= nslots preset
    int32_t slot_words;
    int32_t nslots;
    long long spin_limit;      // bound of the wait for a free slot
    int *err;                  // error word (kErr*)
};

// Interleaved residues of every pair (see DbView::pres): one warp per pair.
static __global__ void pair_residues_kernel(const uint8_t *res, const int64_t *off, const int32_t *pairs,
                                            const int64_t *poff, int npairs, uint16_t *pres) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int p = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); p < npairs; p += nw) {
        const int sa = pairs[2 * p], sb = pairs[2 * p + 1];
        const int64_t a0 = off[sa], na = off[sa + 1] - a0;
        const int64_t b0 = sb >= 0 ? off[sb] : 0, nb = sb >= 0 ? off[sb + 1] - b0 : 0;
        const int64_t base = poff[p], cols = poff[p + 1] - base;   // n_p + 1
        for (int64_t j = lane; j < cols; j += 32) {
            const unsigned ca = j < na ? res[a0 + j] : 0xffu;
            const unsigned cb = j < nb ? res[b0 + j] : 0xffu;
            pres[base + j] = (uint16_t)(ca | (cb << 8));
        }
    }
}

// Presets the slot pool: the first wave's slots are taken, slots that do not exist too.
static __global__ void init_slot_pool_kernel(unsigned *pool, int words, int nslots, int first_wave) {
    for (int w = threadIdx.x; w < words; w += blockDim.x) {
        const int lo = w * 32;
        unsigned v = 0;
        for (int b = 0; b < 32; ++b) if (lo + b >= nslots || lo + b < first_wave) v |= 1u << b;
        pool[w] = v;
    }
}

// Acquires a scratch slot for this block (thread 0); -1 after a bounded wait.
__device__ __forceinline__ int db_acquire_slot(const DbView &D) {
    if ((int)blockIdx.x < D.nslots) return (int)blockIdx.x;
    for (long long t = 0; t < D.spin_limit; ++t) {
        const int w = (int)((blockIdx.x + t) % D.slot_words);
        const unsigned cur = *reinterpret_cast<volatile unsigned *>(D.slot_pool + w);
        if (cur != 0xffffffffu) {
            const int b = __ffs(~cur) - 1;
            if (!(atomicOr(D.slot_pool + w, 1u << b) & (1u << b))) {
                __threadfence();                  // after the previous holder's release
                return w * 32 + b;
            }
        } else if (t >= D.slot_words) {
            __nanosleep(64);
        }
    }
    atomicCAS(D.err, 0, kErrTimeout);
    return -1;
}

__device__ __forceinline__ unsigned pack2(int lo, int hi) {
    return (unsigned)(lo & 0xffff) | ((unsigned)hi << 16);
}

__device__ __forceinline__ int lo16(unsigned v) { return (int)(short)(v & 0xffff); }
__device__ __forceinline__ int hi16(unsigned v) { return (int)(short)(v >> 16); }

// Packed profile pair for row byte k of two profile words (sign-extended bytes).
template <int k>
__device__ __forceinline__ unsigned merge_bytes(uint32_t a, uint32_t b) {
    constexpr uint32_t sel = k | ((8 | k) << 4) | ((4 + k) << 8) | ((8 | (4 + k)) << 12);
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "n"(sel));
    return d;
}

__device__ __forceinline__ unsigned merge_row(const uint32_t *wa, const uint32_t *wb, int r) {
    switch (r & 3) {                 // r is a constant after unrolling
        case 0: return merge_bytes<0>(wa[r >> 2], wb[r >> 2]);
        case 1: return merge_bytes<1>(wa[r >> 2], wb[r >> 2]);
        case 2: return merge_bytes<2>(wa[r >> 2], wb[r >> 2]);
        default: return merge_bytes<3>(wa[r >> 2], wb[r >> 2]);
    }
}

// Profile bytes a lane owns per pass: its R rows rounded up to whole 32-bit
// words, so that every lane's profile load is aligned (R = 5 or 6 gives
// 160- or 192-row passes, which pad a short query far less than 256).
constexpr int db_lane_slot(int R) { return ((R + 3) / 4) * 4; }

template <int R>
__device__ __forceinline__ void load_prof_words(const int8_t *p, uint32_t (&w)[db_lane_slot(R) / 4]) {
    constexpr int LS = db_lane_slot(R);
    if constexpr (LS == 4) {
        w[0] = *reinterpret_cast<const uint32_t *>(p);
    } else if constexpr (LS == 8) {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        w[0] = v.x; w[1] = v.y;
    } else if constexpr (LS == 12) {             // 12-byte lane slots: 4-byte aligned only
        const uint32_t *q = reinterpret_cast<const uint32_t *>(p);
        w[0] = q[0]; w[1] = q[1]; w[2] = q[2];
    } else {
        const uint4 v = *reinterpret_cast<const uint4 *>(p);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
}

// grid: 1D; blocks [jobs[j].block0, jobs[j+1].block0) start on job j (the
// host gives each job blocks in proportion to its work); block: W warps.  A
// block whose job has no pairs left moves on to the job of the launch with
// the most work left (same scoring), so that the launch ends balanced.
// Dynamic shared memory: the query profile, (K + 1) * mpad bytes,
// mpad = passes * 32 * db_lane_slot(R) (lane slots of whole words).
constexpr int kDbCH = 8;      // steps per chunk of the packed fill (steady chunks skip all range tests)

// Per-lane state of the packed fill: U = H - open and E of the lane's R query
// rows for both subjects (16-bit halves), the bottom row's (U, F) of the
// previous step, the diagonal, the running maximum, and the prefetched
// residue pair / top cell of the next step.
template <int R>
struct DbLane {
    unsigned U[R], E[R];
    unsigned ub, fb, udiag0, cmax;
    unsigned cp;                 // residue pair of this step's column
    uint2 topv;                  // (U, F) of the row above, lane 0 (passes after the first)
    const int8_t *prow;          // this lane's profile rows of the current pass
};

// One step of the packed fill: column j = s - gl of both subjects, gl = the
// lane's index in its wavefront of G lanes.  CHECK handles columns outside the
// pair (the first and last G - 1 steps).
template <int R, int G, bool CHECK>
__device__ __forceinline__ void db_step(DbLane<R> &st, int s, int gl, int n, const uint16_t *pr, uint2 *bnd,
                                        bool tops, bool last, int K, int mpad,
                                        unsigned nge2, unsigned ngo2, unsigned neg2)
{
    const int j = s - gl;
    unsigned uup = __shfl_up_sync(kFull, st.ub, 1, G);
    unsigned fup = __shfl_up_sync(kFull, st.fb, 1, G);
    if (gl == 0) { uup = st.topv.x; fup = st.topv.y; }
    // inputs of the next step
    const int jn = j + 1;
    unsigned cpn;
    uint2 topn = make_uint2(ngo2, neg2);
    if (CHECK) {
        cpn = (jn >= 0 && jn <= n) ? pr[jn] : 0xffffu;
        if (tops && s + 1 < n) topn = bnd[s + 1];
    } else {
        cpn = pr[jn];                                   // jn <= n: at most the padding column
        if (tops) topn = bnd[s + 1];                    // s + 1 <= n: inside the scratch row
    }
    if (!CHECK || (j >= 0 && j < n)) {
        uint32_t wa[db_lane_slot(R) / 4], wb[db_lane_slot(R) / 4];
        load_prof_words<R>(st.prow + min((int)(st.cp & 0xffu), K) * mpad, wa);
        load_prof_words<R>(st.prow + min((int)(st.cp >> 8), K) * mpad, wb);
        unsigned udiag = st.udiag0;
        st.udiag0 = uup;
        unsigned f = __viaddmax_s16x2(fup, nge2, uup);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const unsigned sp = merge_row(wa, wb, r);
            const unsigned uold = st.U[r];
            const unsigned e = __viaddmax_s16x2(st.E[r], nge2, uold);
            const unsigned x = __viaddmax_s16x2_relu(udiag, sp, e);
            const unsigned xgo = __viaddmax_s16x2(x, ngo2, neg2);   // x - open
            const unsigned u = __viaddmax_s16x2(f, ngo2, xgo);      // H - open
            st.E[r] = e;
            udiag = uold;
            st.U[r] = u;
            if (r + 1 < R) f = __viaddmax_s16x2(f, nge2, xgo);
        }
        st.ub = st.U[R - 1];
        st.fb = f;
#pragma unroll
        for (int r = 0; r + 1 < R; r += 2) st.cmax = __vimax3_s16x2(st.cmax, st.U[r], st.U[r + 1]);
        if constexpr (R % 2 == 1) st.cmax = __vimax3_s16x2(st.cmax, st.U[R - 1], st.U[R - 1]);
        if (!last && gl == G - 1) bnd[j] = make_uint2(st.ub, st.fb);
    }
    st.cp = cpn;
    st.topv = topn;
}

template <int R, int W, bool OVERSUB, int G = 32>
__global__ void __launch_bounds__(W * 32, W >= 16 ? 1 : (R >= 12 ? 3 : 4))
db_s16x2_kernel(const DbJob *__restrict__ jobs, int njobs, const DbView D,
                const DevScoring *__restrict__ scorings, uint2 *__restrict__ scratch)
{
    static_assert(G == 32 || G == 16, "one or two wavefronts a warp");
    constexpr int NG = 32 / G;                    // wavefronts (pairs of subjects) a warp
    extern __shared__ __align__(16) int8_t prof[];
    // OVERSUB: the grid may exceed the blocks that fit at once (the server's steps); blocks
    // beyond the first wave share the scratch slots
    int slot = (int)blockIdx.x;
    if constexpr (OVERSUB) {
        __shared__ int s_slot;
        if (threadIdx.x == 0) s_slot = db_acquire_slot(D);
        __syncthreads();
        slot = s_slot;
        if (slot < 0) return;
    }
    int jlo = 0, jhi = njobs - 1;                 // last job with block0 <= blockIdx.x
    while (jlo < jhi) {
        const int mid = (jlo + jhi + 1) >> 1;
        if (jobs[mid].block0 <= (int)blockIdx.x) jlo = mid; else jhi = mid - 1;
    }
    __shared__ int s_job;
    for (int job = jlo; job >= 0;) {
        const DbJob &J = jobs[job];
        const DevScoring &SC = scorings[J.scoring];
        const int K = SC.K, go = SC.go, ge = SC.ge;
        const int m = J.m;
        constexpr int ROWS = G * R;
        constexpr int LS = db_lane_slot(R), PROWS = G * LS;    // profile bytes per lane and per pass
        const int passes = (m + ROWS - 1) / ROWS;
        const int mpad = passes * PROWS;
        for (int i = threadIdx.x; i < mpad; i += blockDim.x) {
            const int r = i % LS, row = (i / PROWS) * ROWS + ((i % PROWS) / LS) * R + r;
            const bool ok = r < R && row < m;
            const int qc = ok ? min((int)J.q[row], K - 1) : 0;
            for (int c = 0; c <= K; ++c)
                prof[c * mpad + i] = (ok && c < K) ? (int8_t)(SC.mat[qc * K + c] + go) : (int8_t)kPadScore;
        }
        __syncthreads();

        int maxs = 0;
        for (int k = 0; k < K * K; ++k) maxs = max(maxs, (int)SC.mat[k]);
        const int tmax_u = 32767 - maxs - go;            // overflow threshold on H - open
        const int lane = threadIdx.x & 31;
        const int gl = lane & (G - 1), grp = lane / G;          // the lane's wavefront and its place there
        const int gwarp = slot * W + (threadIdx.x >> 5);
        uint2 *bnd = scratch + ((size_t)gwarp * NG + grp) * (size_t)(D.maxlen + 1);
        const unsigned go2 = pack2(go, go), ge2 = pack2(ge, ge);
        const unsigned ngo2 = pack2(-go, -go), nge2 = pack2(-ge, -ge), neg2 = pack2(kNeg16, kNeg16);

        for (;;) {
            // the warp takes NG consecutive pairs (similar lengths: the pairs are sorted), one per wavefront
            int base = 0;
            if (lane == 0) base = atomicAdd(J.next_pair, NG);
            base = __shfl_sync(kFull, base, 0);
            const int p = J.pair0 + (base + grp) * J.pair_stride;
            const bool live = p < J.pair1;
            if constexpr (NG == 1) {
                if (!live) break;
            } else {
                if (!__any_sync(kFull, live)) break;
            }
            // a wavefront without a pair steps through no columns (its lanes still take part in the
            // warp's shuffles); its residue pointer only has to be readable
            int sa = -1, sb = -1, n = 0;
            const uint16_t *pr = D.pres;
            if (NG == 1 || live) {
                sa = D.pairs[2 * p];
                sb = D.pairs[2 * p + 1];
                pr = D.pres + D.poff[p];
                n = (int)(D.poff[p + 1] - D.poff[p]) - 1;           // columns (pr[n]: padding)
            }
            int nmax = n, nmin = n;                                  // over the warp's wavefronts
            if constexpr (NG > 1) {
                const int o = __shfl_xor_sync(kFull, n, G);
                nmax = max(n, o);
                nmin = min(n, o);
            }
            unsigned cmax = ngo2;                                   // running max of H - open (H = 0)
            for (int pass = 0; pass < passes; ++pass) {
                DbLane<R> st;
                st.prow = prof + pass * PROWS + gl * LS;
    #pragma unroll
                for (int r = 0; r < R; ++r) { st.U[r] = ngo2; st.E[r] = neg2; }
                st.ub = ngo2; st.fb = neg2; st.udiag0 = ngo2;
                st.cmax = cmax;
                const bool last = pass + 1 == passes;
                const bool tops = pass > 0;
                // prefetched inputs of this lane's first column and of lane 0's first top cell
                st.cp = gl == 0 && n > 0 ? pr[0] : 0xffffu;
                st.topv = (tops && n > 0) ? bnd[0] : make_uint2(ngo2, neg2);
                for (int s0 = 0; s0 < nmax + G - 1; s0 += kDbCH) {
                    if (s0 >= G - 1 && s0 + kDbCH <= nmin) {
                        // steady state: every lane's column is inside its pair, the prefetched
                        // column at most the padding column n
    #pragma unroll
                        for (int k = 0; k < kDbCH; ++k)
                            db_step<R, G, false>(st, s0 + k, gl, n, pr, bnd, tops, last, K, mpad, nge2, ngo2, neg2);
                    } else {
                        for (int k = 0; k < kDbCH && s0 + k < nmax + G - 1; ++k)
                            db_step<R, G, true>(st, s0 + k, gl, n, pr, bnd, tops, last, K, mpad, nge2, ngo2, neg2);
                    }
                }
                cmax = st.cmax;
                __syncwarp();
            }
            // each wavefront's maximum of each half
            int ma = lo16(cmax), mb = hi16(cmax);
    #pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                ma = max(ma, __shfl_xor_sync(kFull, ma, off));
                mb = max(mb, __shfl_xor_sync(kFull, mb, off));
            }
            if (gl == 0 && (NG == 1 || live)) {
                const int outs[2] = {sa, sb};
                const int mx[2] = {ma, mb};
                for (int h = 0; h < 2; ++h) {
                    const int s = outs[h];
                    if (s < 0) continue;
                    if (mx[h] > tmax_u) {
                        J.scores[s] = -1;
                        const int slot = atomicAdd(J.novf, 1);
                        J.ovf[slot] = s;
                    } else {
                        J.scores[s] = max(0, mx[h] + go);
                    }
                }
            }
        }
        // this job has no pairs left: every warp is done with the profile; take the job of the
        // launch with the most work left (pairs not yet claimed x passes), if any
        __syncthreads();
        if (threadIdx.x == 0) {
            long long best = 0;
            int pick = -1;
            for (int k = 0; k < njobs; ++k) {
                const DbJob &O = jobs[k];
                if (O.scoring != J.scoring) continue;
                const int npairs = (O.pair1 - O.pair0 + O.pair_stride - 1) / O.pair_stride;
                const int left = npairs - *(volatile const int32_t *)O.next_pair;
                const long long work = (long long)left * ((O.m + ROWS - 1) / ROWS);
                if (left > 0 && work > best) { best = work; pick = k; }
            }
            s_job = pick;
        }
        __syncthreads();
        job = s_job;
    }
    if constexpr (OVERSUB) {                      // hand the slot to a later block
        __syncthreads();                          // every warp is done with the slot's scratch
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAnd(D.slot_pool + slot / 32, ~(1u << (slot % 32)));
        }
    }
}

// Write rescored (int32) results into the score array: scores[subject[k]] = res[k].x.
static __global__ void scatter_scores_kernel(const int32_t *subject, const int4 *res, int count,
                                             int32_t *scores) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) scores[subject[k]] = res[k].x;
}

// ---- top-k: key = (score << 32) | (0xffffffff - subject), larger is better
__device__ __forceinline__ unsigned long long topk_key(int score, int s) {
    return ((unsigned long long)(unsigned)score << 32) | (unsigned long long)(0xffffffffu - (unsigned)s);
}

// Block-wide top-k by k rounds of arg-max over a chunk held in shared
// memory.  Phase 1: every block takes TOPK_CHUNK keys and writes its k
// best; phase 2: one block does the same over all block winners.
constexpr int kTopkThreads = 256;
constexpr int kTopkChunk = 2048;

static __device__ void block_topk(unsigned long long *keys, int count, int k, unsigned long long *out) {
    __shared__ unsigned long long red[kTopkThreads / 32];
    __shared__ int redi[kTopkThreads / 32];
    for (int it = 0; it < k; ++it) {
        unsigned long long best = 0;
        int bi = -1;
        for (int i = threadIdx.x; i < count; i += blockDim.x)
            if (bi < 0 || keys[i] > best) { best = keys[i]; bi = i; }
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(kFull, best, off);
            const int oi = __shfl_xor_sync(kFull, bi, off);
            if (ob > best || (bi < 0 && oi >= 0)) { best = ob; bi = oi; }
        }
        if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = best; redi[threadIdx.x >> 5] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long b = 0;
            int i0 = -1;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (redi[w] >= 0 && (red[w] > b || i0 < 0)) { b = red[w]; i0 = redi[w]; }
            out[it] = i0 >= 0 ? b : 0;
            if (i0 >= 0) keys[i0] = 0;          // taken
        }
        __syncthreads();
    }
}

static __global__ void __launch_bounds__(kTopkThreads)
topk_phase1_kernel(const int32_t *scores, int nseq, int k, unsigned long long *winners) {
    __shared__ unsigned long long keys[kTopkChunk];
    const int base = blockIdx.x * kTopkChunk;
    const int cnt = min(kTopkChunk, nseq - base);
    for (int i = threadIdx.x; i < kTopkChunk; i += blockDim.x)
        keys[i] = i < cnt ? topk_key(max(scores[base + i], 0), base + i) : 0;
    __syncthreads();
    block_topk(keys, cnt, k, winners + (size_t)blockIdx.x * k);
}

static __global__ void __launch_bounds__(kTopkThreads)
topk_phase2_kernel(const unsigned long long *winners, int count, int k, int2 *out) {
    extern __shared__ unsigned long long keys2[];
    for (int i = threadIdx.x; i < count; i += blockDim.x) keys2[i] = winners[i];
    __syncthreads();
    __shared__ unsigned long long best[64];
    block_topk(keys2, count, k, best);
    if (threadIdx.x < k) {
        const unsigned long long b = best[threadIdx.x];
        out[threadIdx.x] = make_int2((int)(0xffffffffu - (unsigned)(b & 0xffffffffu)), (int)(b >> 32));
    }
}

}  // namespace swgb
