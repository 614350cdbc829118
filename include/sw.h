/*
 * sw.h -- C ABI of the GB300 Smith-Waterman / Gotoh library (libswgb.so).
 *
 * The library computes optimal local alignments (Smith-Waterman, paper
 * Section 2.1.2) with affine gap penalties (gap open / gap extension, paper
 * Section 2.2; values used in the experiments, Section 3.2) on one NVIDIA
 * GB300 GPU.  It offers the two uses the paper distinguishes in Section
 * 2.1: pairwise alignment of two (long) sequences, where all threads work on
 * one matrix (intra-task parallelism), and database search, where many
 * matrices are computed at once (inter-task parallelism); plus the
 * resolution (score) and reconstruction (alignment path) phases the paper
 * describes for SW# in Section 2.2.
 *
 * Recurrence (the paper names the method without printing it; this is the
 * textbook Gotoh form).  Sequence a (length m) indexes rows i, sequence b
 * (length n) indexes columns j, S is the substitution matrix, o = gap_open,
 * e = gap_extend, a gap of k letters costs o + (k-1)*e:
 *
 *   E(i,j) = max(E(i,j-1) - e, H(i,j-1) - o)     gap in a, consumes b_j  (I)
 *   F(i,j) = max(F(i-1,j) - e, H(i-1,j) - o)     gap in b, consumes a_i  (D)
 *   H(i,j) = max(0, H(i-1,j-1) + S(a_i,b_j), E(i,j), F(i,j))
 *   H(0,*) = H(*,0) = 0
 *
 * Canonical results (the paper is silent on ties):
 *   - end cell: the maximum H; among equal maxima the smallest row (a_end)
 *     and then the smallest column (b_end), i.e. the first in row-major order;
 *   - traceback from the end cell: in H prefer the diagonal, then E, then F,
 *     stop where H = 0; inside a gap leave it (open) before extending it;
 *   - coordinates are 0-based, begin inclusive, end exclusive; score 0 means
 *     an empty alignment with all coordinates 0;
 *   - CIGAR is run-length M/I/D; D consumes a only, I consumes b only.
 *
 * Conventions for every call:
 *   - returns SW_OK (0) or a negative SW_E* code; outputs are untouched on
 *     error; no C++ exception crosses the ABI;
 *   - residues are pre-encoded codes 0 .. alphabet-1 (see sw_encode);
 *   - sequence pointers may be host or device memory (the library asks the
 *     CUDA driver which); host data is copied to the device inside the call;
 *   - input buffers are borrowed and not retained after the call returns,
 *     except by sw_db_create, which copies the database;
 *   - output structs are caller-owned host memory, except the CIGAR string
 *     of sw_alignment, which the library allocates and sw_alignment_free
 *     releases;
 *   - calls on one context are serialised on its CUDA stream and return
 *     after the stream work they issued is complete; a context must not be
 *     used from two host threads at once.
 */
#ifndef SWGB_SW_H
#define SWGB_SW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SW_OK        0
#define SW_EINVAL   (-1)   /* bad argument: null pointer, negative length, code >= alphabet, bad penalties */
#define SW_ENOMEM   (-2)   /* device or host allocation failed */
#define SW_ECUDA    (-3)   /* a CUDA runtime call failed */
#define SW_ETIMEOUT (-4)   /* a bounded device-side wait gave up (see sw_ctx_create) */
#define SW_EAGAIN   (-5)   /* resource busy / result not ready yet (serving calls) */
#define SW_ERANGE   (-6)   /* a size or score beyond the documented limits */

/* Largest sequence length accepted by the pairwise calls. */
#define SW_MAX_LEN  ((int64_t)2000000000)

typedef struct sw_ctx sw_ctx;   /* device, stream, scratch memory, tuning state */
typedef struct sw_db  sw_db;    /* device-resident, length-sorted protein database */

/*
 * Algorithms (paper Section 2.1: SW# computes local, global, semi-global
 * and overlap alignments; Sections 2.1.1-2.1.4 name them NW, SW, HW, OV).
 * The paper describes them in words; this library takes these readings,
 * with H(0,0) = 0, E(i,0) = F(0,j) = -infinity and the Gotoh recurrence
 * above in every interior cell:
 *   SW_ALG_LOCAL       Smith-Waterman: zero floor, best cell anywhere, the
 *                      traceback stops at H = 0.
 *   SW_ALG_GLOBAL      Needleman-Wunsch: H(i,0) = -(o + (i-1)e),
 *                      H(0,j) = -(o + (j-1)e), no zero floor; end cell
 *                      (m, n), the path starts at (0, 0).
 *   SW_ALG_SEMIGLOBAL  all of a against a substring of b: H(0,j) = 0,
 *                      H(i,0) = -(o + (i-1)e), no floor; end cell the best
 *                      of the last row (j = 0 .. n), the path starts in row 0.
 *   SW_ALG_OVERLAP     leading and trailing gaps of both sequences free:
 *                      H(0,j) = H(i,0) = 0, no floor; end cell the best of
 *                      the last row and the last column, the path starts in
 *                      row 0 or column 0.
 * Among equal maxima the end cell is the first in row-major order.  Scores
 * of the other algorithms may be zero or negative; every coordinate and
 * CIGAR follows the same conventions as the local one (a path that reaches
 * column 0 below row 0 in the global or semi-global algorithm, or row 0
 * right of column 0 in the global one, continues as one deletion or
 * insertion run to (0, 0)).
 */
#define SW_ALG_LOCAL       0
#define SW_ALG_GLOBAL      1
#define SW_ALG_SEMIGLOBAL  2
#define SW_ALG_OVERLAP     3

/*
 * Scoring scheme (paper Sections 2.2 and 3.2: a substitution matrix plus gap
 * open and gap extension penalties, and the algorithm of Section 2.1).
 * matrix is alphabet x alphabet int8, row-major, matrix[x*alphabet + y] =
 * score of residue x of a (rows) against residue y of b (columns); it is
 * copied at call time.  Penalties are given as non-negative numbers that are
 * subtracted; 0 <= gap_extend <= gap_open <= 1,000,000 (with gap_extend >
 * gap_open the Gotoh recurrence would not score maximal gap runs as
 * open + (k-1)*extend).  1 <= alphabet <= 32.  algorithm is one of SW_ALG_*
 * (a zero-initialised struct is the local algorithm); the pairwise calls
 * (sw_score, sw_align) and the batch accept all four, the database search,
 * the server and sw_score_noalloc the local one only (else SW_EINVAL).
 */
typedef struct {
    int32_t alphabet;
    const int8_t *matrix;
    int32_t gap_open;
    int32_t gap_extend;
    int32_t algorithm;
} sw_scoring;

/* Score and canonical end cell of one pair. */
typedef struct {
    int32_t score;
    uint32_t flags;        /* reserved, 0 */
    int64_t a_end;         /* exclusive end in a (rows) */
    int64_t b_end;         /* exclusive end in b (columns) */
} sw_hit;

/* Canonical alignment of one pair; cigar is owned by the library. */
typedef struct {
    int32_t score;
    uint32_t flags;        /* reserved, 0 */
    int64_t a_begin, a_end;
    int64_t b_begin, b_end;
    char *cigar;           /* NUL-terminated, run-length M/I/D; "" for score 0 */
    int64_t cigar_len;     /* strlen(cigar) */
} sw_alignment;

/* One database hit. */
typedef struct {
    int64_t subject;       /* index of the subject in the database */
    int32_t score;
    uint32_t flags;        /* reserved, 0 */
} sw_dbhit;

/*
 * Create a context on CUDA device `device`.  cuda_stream is a cudaStream_t
 * (NULL = the legacy default stream) on which every call of this context
 * runs.  Device-side waits between thread blocks are bounded; a wait that
 * gives up makes the call fail with SW_ETIMEOUT and leaves the context
 * usable.
 */
int sw_ctx_create(int device, void *cuda_stream, sw_ctx **out);
void sw_ctx_destroy(sw_ctx *ctx);

/* Human-readable text for a status code (static storage). */
const char *sw_strerror(int status);

/*
 * Encode residue letters (step "encode" of the path): codes[k] = index of
 * toupper(text[k]) in `alphabet` (a NUL-terminated string of at most 32
 * distinct upper-case ASCII letters or '*', e.g. "ACGT" or
 * "ARNDCQEGHILKMFPSTWYVBZX*").  text and codes may be host or device
 * memory, len >= 0.  A character outside the alphabet gives SW_EINVAL and
 * leaves codes unspecified.
 */
int sw_encode(sw_ctx *ctx, const char *alphabet, const char *text, int64_t len, uint8_t *codes);

/*
 * Resolution phase for one pair (paper Section 2.2): best score of the
 * scoring's algorithm and its canonical end cell.  0 <= m, n <= SW_MAX_LEN;
 * every code < alphabet.  Scores are bounded by min(m, n) * max S(x, y),
 * which must be below 2^26 (67,108,864), else SW_ERANGE (the int32 fill tags
 * row indices into the low bits of its scores to pick the canonical end cell
 * without branches); for the algorithms other than the local one the most
 * negative value, gap_open + (m + n) * gap_extend, must stay below it too.
 */
int sw_score(sw_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
             const sw_scoring *sc, sw_hit *out);

/*
 * Resolution and reconstruction for one pair (paper Section 2.2): score,
 * canonical alignment path and coordinates.  Same limits as sw_score.  The
 * path is reconstructed from traceback bits recomputed on the device from
 * checkpoint rows, so device memory stays far below the m*n matrix.  A pair
 * whose traceback tiles fit one wave on the SMs (sides up to 8,192) is
 * reconstructed with one host synchronisation; larger pairs take bands of
 * tiles along the path, one synchronisation per band.
 * *out is written only on success; release it with sw_alignment_free.
 */
int sw_align(sw_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
             const sw_scoring *sc, sw_alignment *out);

/* Free the CIGAR of an alignment filled by sw_align (NULL-safe). */
void sw_alignment_free(sw_alignment *aln);

/*
 * sw_score without any device allocation (the paper has no counterpart; it
 * exists for callers of this library that cannot call cudaMalloc, such as a
 * serving process whose own caching allocator owns the device memory
 * budget, or a latency-critical pipeline that must avoid the implicit
 * device synchronisation of cudaMalloc / cudaFree).
 *
 * Same result as sw_score (score and canonical end cell).  No context is
 * needed: it runs on the current CUDA device, on cuda_stream (a
 * cudaStream_t, NULL = legacy default stream).  a and b must be device
 * memory (else SW_EINVAL); out is host memory.  All scratch lives in one
 * fixed array of about 4.3 MB inside the library, which every GPU that
 * loads the library holds until the process exits.  Limits: n <= 262,144
 * columns and m <= 16,384 * 1,024 = 16,777,216 rows; larger inputs are
 * rejected with SW_ERANGE.  Every call looks up the array's device address
 * in the current context (so a device reset between calls is safe); the
 * first call in a context loads the library's device code and should come
 * before any stream capture.  Calls share the array: calls whose GPU work could
 * overlap (other streams, other host threads) race and must be serialised
 * by the caller.  Synchronous: returns after the result is on the host.
 */
int sw_score_noalloc(void *cuda_stream, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                     const sw_scoring *sc, sw_hit *out);

/*
 * Batched pairwise scores (many pairs of uneven lengths; the paper's Section
 * 3.1 replaces SW#'s static block sizes by sizes derived from the sequence
 * lengths, which this batch planner does per length bin).  Pairs are binned
 * by scoring scheme and by query length (up to 1024 rows, longer); each bin
 * is one launch with its own tile shape, and the bins' launches run
 * concurrently.  Pair p is
 * a = a_res[a_off[p] .. a_off[p+1]) against b = b_res[b_off[p] .. b_off[p+1])
 * scored with scorings[scoring_of_pair[p]]; a_off / b_off are host arrays of
 * npairs + 1 entries starting at 0; residues may be host or device memory
 * (device residues are used in place and must outlive the plan).  Results
 * are the same as sw_score on each pair.
 *
 * A plan keeps the inputs and the task table on the device:
 *   SW_BATCH_GRAPH     capture each run in a CUDA graph once and replay it;
 *   SW_BATCH_AUTOTUNE  time the candidate tile shapes of every bin on this plan
 *                      and keep the fastest (cached in the context per bin
 *                      size class).  The candidates are int32 lanes of 4-16
 *                      rows and, for local bins whose scoring keeps it exact,
 *                      packed 16-bit lanes of 8, 12 or 16 rows.
 * sw_batch_run writes npairs hits (host memory).  A plan belongs to its
 * context and must be destroyed before it.
 */
typedef struct sw_batch sw_batch;
#define SW_BATCH_GRAPH     1
#define SW_BATCH_AUTOTUNE  2
int sw_batch_create(sw_ctx *ctx, int64_t npairs, const uint8_t *a_res, const int64_t *a_off,
                    const uint8_t *b_res, const int64_t *b_off, const int32_t *scoring_of_pair,
                    int32_t nscorings, const sw_scoring *scorings, int32_t flags, sw_batch **out);
int sw_batch_run(sw_batch *plan, sw_hit *out);
void sw_batch_destroy(sw_batch *plan);
/* Tile shape of the plan's largest bin (by cells): rows per lane and compute
 * warps per block. */
int sw_batch_config(const sw_batch *plan, int32_t *rows_per_lane, int32_t *warps);
/* Configuration of bin `bin` of the plan (bins: scoring scheme x row class,
 * the bin with the most cells first): rows per lane, compute warps per block,
 * lane width in bits (32, or 16 for the packed fill) and its pair count.
 * SW_ERANGE once bin is past the last bin; SW_EINVAL on a null pointer. */
int sw_batch_bin_config(const sw_batch *plan, int32_t bin, int32_t *rows_per_lane, int32_t *warps,
                        int32_t *lane_bits, int64_t *npairs);
/* One-shot: create (no graph, no autotuning), run, destroy. */
int sw_score_batch(sw_ctx *ctx, int64_t npairs, const uint8_t *a_res, const int64_t *a_off,
                   const uint8_t *b_res, const int64_t *b_off, const int32_t *scoring_of_pair,
                   int32_t nscorings, const sw_scoring *scorings, sw_hit *out);

/*
 * Database of subject sequences for one-to-many search (paper Section 2.1,
 * database similarity search; Section 3.2 searches UniProtKB/Swiss-Prot).
 * residues holds all subjects back to back (codes, host or device memory),
 * offsets (host memory, nseq + 1 entries, offsets[0] = 0, non-decreasing)
 * delimits subject s = residues[offsets[s] .. offsets[s+1]).  The database
 * is copied to the device of ctx and sorted by length there once; the
 * caller's buffers are not retained.  nseq <= 2^30.  Codes are checked
 * against the alphabet of each search (SW_EINVAL if one is too large).
 */
int sw_db_create(sw_ctx *ctx, const uint8_t *residues, const int64_t *offsets, int64_t nseq, sw_db **out);
void sw_db_destroy(sw_db *db);

/* Number of subjects of a database (-1 for NULL). */
int64_t sw_db_size(const sw_db *db);

/*
 * Search the database with query q (length m, host or device memory):
 * the local alignment score of q against every subject, and the k best
 * hits (0 <= k <= 64) ordered by score descending, then subject index
 * ascending; subjects with score 0 are ranked too.  hits (host, k entries)
 * receives min(k, nseq) hits and *nhits their count.  all_scores, when not
 * NULL, receives every subject's score (nseq int32, host or device memory).
 * Scores are computed in packed 16-bit lanes; a subject whose score could
 * saturate them is rescored exactly in 32 bits, so every score is exact.
 */
int sw_dbsearch(sw_ctx *ctx, const sw_db *db, const uint8_t *q, int64_t m, const sw_scoring *sc,
                int32_t k, sw_dbhit *hits, int32_t *nhits, int32_t *all_scores);

/*
 * Serving loop over a device-resident database: continuous batching of
 * searches (same results as sw_dbsearch for every request).
 *
 * The database is swept circularly in `chunks` pieces; every sw_server_step
 * runs the current piece for all admitted requests at once, so requests
 * that arrive while others are on the GPU share the device with them.
 * Steps are pipelined: a step call enqueues its piece and then waits for
 * the previous call's, so the device does not idle while the host admits
 * and retires requests.  A request is admitted by sw_server_submit when one
 * of max_slots slots (1..256) is free and its device memory (about 8 bytes
 * per database subject plus its query) fits mem_budget bytes, else
 * SW_EAGAIN; it joins the sweep at the next step call, and its hits are
 * ready after `chunks` + 1 step calls, the last of which completes its last
 * piece (sw_server_poll: SW_EAGAIN while pending; a collected ticket is
 * forgotten).  The scoring must allow the packed 16-bit search (every
 * S + gap_open within int8, penalties <= 16000), else SW_ERANGE at
 * creation; queries longer than 8000 give SW_ERANGE.  k <= 64.  A step runs
 * its requests in groups of one tile shape each (every query padded to the
 * passes that fit it best).  A slot keeps its device buffers for the next
 * request, so the server holds at most max_slots of them; mem_used counts
 * the active requests' share.  A request whose retirement fails is
 * retired with that status (sw_server_poll returns it); a device error in
 * a step fails every request the server holds and every later call.  The
 * server enqueues its admissions and retirements on its context's stream
 * and its steps on streams of its own, with its own scoring table, error
 * word and scratch, so the context's other calls may run between steps.
 * It must be destroyed before the context and the database (destroying
 * waits for a step in flight).
 */
typedef struct sw_server sw_server;
int sw_server_create(sw_ctx *ctx, const sw_db *db, const sw_scoring *sc, size_t mem_budget, int32_t k,
                     int32_t max_slots, int32_t chunks, sw_server **out);
int sw_server_submit(sw_server *srv, const uint8_t *q, int64_t m, uint64_t *ticket);
/* Enqueue one sweep step, then complete the previous one (its finished
 * requests retire); *active = requests in the enqueued step. */
int sw_server_step(sw_server *srv, int32_t *active);
int sw_server_poll(sw_server *srv, uint64_t ticket, sw_dbhit *hits, int32_t *nhits);
/* Requests in flight, device bytes they hold, cells of retired requests. */
int sw_server_stats(const sw_server *srv, int32_t *active, size_t *mem_used, int64_t *cells_done);
void sw_server_destroy(sw_server *srv);

/*
 * Number of kernels this context has launched since it was created
 * (diagnostics: lets a caller count device launches per call).  Returns -1
 * for a null context.
 */
int64_t sw_ctx_launches(const sw_ctx *ctx);

/*
 * Kernel timing (instrumentation; the paper has no counterpart).  While
 * enabled, the context records a CUDA event pair on its stream around every
 * launch of the kernels below and accumulates their device time, so a
 * caller can time one kernel class inside a longer call (for example the
 * forward fill inside sw_align) without a profiler.  Launches issued while
 * the stream is being captured into a CUDA graph are not timed.
 *
 * sw_ctx_timing: enable (1) or disable (0); either clears the totals.
 * sw_ctx_kernel_time: total device milliseconds and launch count of one
 *   kind since timing was enabled; waits for the recorded events.
 *   SW_EINVAL for a null context, a bad kind or null outputs.
 */
#define SW_KT_FILL     0   /* wavefront fill, score and checkpoint modes (sw_score, sw_align forward, rescoring) */
#define SW_KT_FILL_TB  1   /* wavefront fill, traceback mode (sw_align recompute) */
#define SW_KT_WALK     2   /* traceback walk (sw_align) */
#define SW_KT_DB16     3   /* packed 16-bit database fill (sw_dbsearch, server) */
#define SW_KT_COUNT    4
int sw_ctx_timing(sw_ctx *ctx, int32_t enable);
int sw_ctx_kernel_time(sw_ctx *ctx, int32_t kind, double *ms, int64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* SWGB_SW_H */
