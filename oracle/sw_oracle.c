/*
 * sw_oracle.c -- plain scalar CPU oracle for Smith-Waterman local alignment
 * with Gotoh affine gaps.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file.  It exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA library against an
 * obviously correct reference.  It shares no code, header, table or constant
 * with the CUDA library.
 *
 * What it computes (Smith-Waterman local alignment, paper Section 2.1.2; gap
 * open / gap extension penalties and substitution matrices, Section 2.2 and
 * Section 3.2; the paper names the method but prints no recurrence, so the
 * textbook Gotoh form is written out here):
 *
 *   a = rows (length m), b = columns (length n), S = K x K substitution
 *   matrix (row-major, S[x*K+y] = score of residue x against residue y),
 *   o = gap open >= 0, e = gap extend >= 0, a gap of length k costs
 *   o + (k-1)*e.
 *
 *   E(i,j) = max(E(i,j-1) - e, H(i,j-1) - o)        gap consuming b_j  ("I")
 *   F(i,j) = max(F(i-1,j) - e, H(i-1,j) - o)        gap consuming a_i  ("D")
 *   H(i,j) = max(0, H(i-1,j-1) + S(a_i,b_j), E(i,j), F(i,j))
 *   H(0,*) = H(*,0) = 0,  E(i,0) = F(0,j) = -infinity.
 *
 * Canonical outputs (the paper is silent on ties; these are this project's
 * readings):
 *   end cell   : the maximum H; among equal maxima the smallest row i
 *                (a_end), then the smallest column j (b_end): the first in
 *                row-major order, a down the rows.  Score 0 gives an
 *                empty alignment with every coordinate 0.
 *   traceback  : from the end cell in state H:
 *                  state H: stop if H(i,j) == 0; else diagonal if
 *                           H(i,j) == H(i-1,j-1)+S; else state E if
 *                           H(i,j) == E(i,j); else state F.
 *                  state E: emit I, move left; return to state H if
 *                           E(i,j) == H(i,j-1) - o (open before extend).
 *                  state F: emit D, move up; return to state H if
 *                           F(i,j) == H(i-1,j) - o.
 *   coordinates: 0-based, begin inclusive, end exclusive.
 *   CIGAR      : run-length M/I/D; D consumes a only, I consumes b only.
 *
 * Error behaviour: every function returns 0 on success, -1 on bad arguments
 * and -2 when memory cannot be allocated.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_NEG_INF ((int64_t)-1 << 40)

static int64_t max2(int64_t x, int64_t y) { return x > y ? x : y; }

static int args_ok(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                   const int8_t *S, int K, int o, int e)
{
    if (m < 0 || n < 0 || K <= 0 || !S || o < 0 || e < 0 || e > o) return 0;
    if ((m > 0 && !a) || (n > 0 && !b)) return 0;
    for (int64_t i = 0; i < m; i++) if (a[i] >= K) return 0;
    for (int64_t j = 0; j < n; j++) if (b[j] >= K) return 0;
    return 1;
}

/* Is (i,j) with value h a better end cell than the current best? */
static int better_end(int64_t h, int64_t i, int64_t j,
                      int64_t best, int64_t bi, int64_t bj)
{
    if (h != best) return h > best;
    if (i != bi) return i < bi;
    return j < bj;
}

/*
 * Global (end-to-end) Gotoh score of a against b: the best alignment that
 * consumes all of a and all of b, with the same gap cost o + (k-1)e and no
 * zero floor.  It is used to check pieces of a local alignment: a piece of
 * an optimal path that starts and ends next to M columns is itself an
 * optimal global alignment of the sub-block it spans (otherwise splicing the
 * better one in would improve the whole path).
 *   H(0,0) = 0; H(i,0) = -(o + (i-1)e) and H(0,j) = -(o + (j-1)e) for i, j >= 1
 *   E(i,j) = max(E(i,j-1) - e, H(i,j-1) - o), F likewise down the column,
 *   H(i,j) = max(H(i-1,j-1) + S(a_i,b_j), E(i,j), F(i,j)); the score is H(m,n).
 */
int oracle_nw_score(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                    const int8_t *S, int K, int o, int e, int64_t *score)
{
    if (!args_ok(a, m, b, n, S, K, o, e) || !score) return -1;
    int64_t *Hrow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *Frow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!Hrow || !Frow) { free(Hrow); free(Frow); return -2; }
    Hrow[0] = 0;
    Frow[0] = ORACLE_NEG_INF;
    for (int64_t j = 1; j <= n; j++) { Hrow[j] = -(o + (j - 1) * (int64_t)e); Frow[j] = ORACLE_NEG_INF; }
    for (int64_t i = 1; i <= m; i++) {
        int64_t E = ORACLE_NEG_INF;                      /* E(i,0) */
        int64_t Hleft = -(o + (i - 1) * (int64_t)e);     /* H(i,0) */
        int64_t Hdiag = Hrow[0];                          /* H(i-1,0) */
        for (int64_t j = 1; j <= n; j++) {
            int64_t Hup = Hrow[j];
            E = max2(E - e, Hleft - o);
            int64_t F = max2(Frow[j] - e, Hup - o);
            int64_t H = Hdiag + S[a[i - 1] * K + b[j - 1]];
            H = max2(H, E);
            H = max2(H, F);
            Frow[j] = F;
            Hdiag = Hup;
            Hrow[j] = H;
            Hleft = H;
        }
        Hrow[0] = -(o + (i - 1) * (int64_t)e);
    }
    *score = Hrow[n];
    if (m == 0) *score = n == 0 ? 0 : -(o + (n - 1) * (int64_t)e);
    free(Hrow); free(Frow);
    return 0;
}

/*
 * Score and canonical end cell, linear memory.  One row of H and F is kept;
 * the loops visit every cell of the (m+1) x (n+1) table once.
 */
int oracle_sw_score(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                    const int8_t *S, int K, int o, int e,
                    int64_t *score, int64_t *a_end, int64_t *b_end)
{
    if (!args_ok(a, m, b, n, S, K, o, e) || !score || !a_end || !b_end) return -1;
    int64_t *Hrow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *Frow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!Hrow || !Frow) { free(Hrow); free(Frow); return -2; }
    for (int64_t j = 0; j <= n; j++) { Hrow[j] = 0; Frow[j] = ORACLE_NEG_INF; }

    int64_t best = 0, bi = 0, bj = 0;
    for (int64_t i = 1; i <= m; i++) {
        int64_t E = ORACLE_NEG_INF;   /* E(i,0) */
        int64_t Hleft = 0;            /* H(i,0) */
        int64_t Hdiag = Hrow[0];      /* H(i-1,0) */
        for (int64_t j = 1; j <= n; j++) {
            int64_t Hup = Hrow[j];                      /* H(i-1,j) */
            E = max2(E - e, Hleft - o);                 /* E(i,j) */
            int64_t F = max2(Frow[j] - e, Hup - o);     /* F(i,j) */
            int64_t H = Hdiag + S[a[i - 1] * K + b[j - 1]];
            H = max2(H, E);
            H = max2(H, F);
            H = max2(H, 0);
            Frow[j] = F;
            Hdiag = Hup;
            Hrow[j] = H;
            Hleft = H;
            if (H > 0 && better_end(H, i, j, best, bi, bj)) { best = H; bi = i; bj = j; }
        }
    }
    free(Hrow); free(Frow);
    *score = best;
    *a_end = best > 0 ? bi : 0;
    *b_end = best > 0 ? bj : 0;
    return 0;
}

/*
 * Full-matrix alignment: H, E and F are stored for every cell and the
 * traceback compares stored values.  Memory is 24 bytes per cell, so it is
 * meant for small problems.
 *
 * ops: caller buffer of at least m+n bytes; receives the operations in
 * forward order as the characters 'M', 'I', 'D'.  *n_ops gets their count.
 */
int oracle_sw_align_full(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                         const int8_t *S, int K, int o, int e,
                         int64_t *score, int64_t *a_begin, int64_t *a_end,
                         int64_t *b_begin, int64_t *b_end,
                         char *ops, int64_t *n_ops)
{
    if (!args_ok(a, m, b, n, S, K, o, e) || !score || !a_begin || !a_end ||
        !b_begin || !b_end || !n_ops || (m + n > 0 && !ops)) return -1;
    const int64_t W = n + 1;
    const size_t cells = (size_t)(m + 1) * (size_t)W;
    int64_t *H = (int64_t *)malloc(sizeof(int64_t) * cells);
    int64_t *E = (int64_t *)malloc(sizeof(int64_t) * cells);
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * cells);
    char *rev = (char *)malloc((size_t)(m + n + 1));
    if (!H || !E || !F || !rev) { free(H); free(E); free(F); free(rev); return -2; }
#define AT(X, i, j) X[(size_t)(i) * (size_t)W + (size_t)(j)]
    for (int64_t j = 0; j <= n; j++) { AT(H, 0, j) = 0; AT(E, 0, j) = ORACLE_NEG_INF; AT(F, 0, j) = ORACLE_NEG_INF; }
    for (int64_t i = 0; i <= m; i++) { AT(H, i, 0) = 0; AT(E, i, 0) = ORACLE_NEG_INF; AT(F, i, 0) = ORACLE_NEG_INF; }

    int64_t best = 0, bi = 0, bj = 0;
    for (int64_t i = 1; i <= m; i++) {
        for (int64_t j = 1; j <= n; j++) {
            AT(E, i, j) = max2(AT(E, i, j - 1) - e, AT(H, i, j - 1) - o);
            AT(F, i, j) = max2(AT(F, i - 1, j) - e, AT(H, i - 1, j) - o);
            int64_t h = AT(H, i - 1, j - 1) + S[a[i - 1] * K + b[j - 1]];
            h = max2(h, AT(E, i, j));
            h = max2(h, AT(F, i, j));
            h = max2(h, 0);
            AT(H, i, j) = h;
            if (h > 0 && better_end(h, i, j, best, bi, bj)) { best = h; bi = i; bj = j; }
        }
    }

    int64_t i = bi, j = bj, k = 0;
    int state = 0; /* 0 = H, 1 = E, 2 = F */
    if (best > 0) {
        for (;;) {
            if (state == 0) {
                int64_t h = AT(H, i, j);
                if (h == 0) break;
                if (h == AT(H, i - 1, j - 1) + S[a[i - 1] * K + b[j - 1]]) {
                    rev[k++] = 'M'; i--; j--;
                } else if (h == AT(E, i, j)) {
                    state = 1;
                } else {
                    state = 2;
                }
            } else if (state == 1) {
                rev[k++] = 'I';
                if (AT(E, i, j) == AT(H, i, j - 1) - o) state = 0;
                j--;
            } else {
                rev[k++] = 'D';
                if (AT(F, i, j) == AT(H, i - 1, j) - o) state = 0;
                i--;
            }
        }
    }
#undef AT
    for (int64_t t = 0; t < k; t++) ops[t] = rev[k - 1 - t];
    *n_ops = k;
    *score = best;
    *a_end = best > 0 ? bi : 0;
    *b_end = best > 0 ? bj : 0;
    *a_begin = best > 0 ? i : 0;
    *b_begin = best > 0 ? j : 0;
    free(H); free(E); free(F); free(rev);
    return 0;
}

/*
 * Same alignment, stored as traceback pointers instead of values (the usual
 * Gotoh pointer formulation): for every cell one byte holds
 *   bits 0-1  source of H: 0 zero, 1 diagonal, 2 E, 3 F  (first match in that order)
 *   bit  2    E(i,j) came from opening, E(i,j) == H(i,j-1) - o
 *   bit  3    F(i,j) came from opening, F(i,j) == H(i-1,j) - o
 * and the walk follows the bits with the same rules as the value version.
 * Memory is one byte per cell plus two rows, so it handles much larger
 * problems than oracle_sw_align_full.
 */
int oracle_sw_align_ptr(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                        const int8_t *S, int K, int o, int e,
                        int64_t *score, int64_t *a_begin, int64_t *a_end,
                        int64_t *b_begin, int64_t *b_end,
                        char *ops, int64_t *n_ops)
{
    if (!args_ok(a, m, b, n, S, K, o, e) || !score || !a_begin || !a_end ||
        !b_begin || !b_end || !n_ops || (m + n > 0 && !ops)) return -1;
    const int64_t W = n + 1;
    uint8_t *P = (uint8_t *)malloc((size_t)(m + 1) * (size_t)W);
    int64_t *Hrow = (int64_t *)malloc(sizeof(int64_t) * (size_t)W);
    int64_t *Frow = (int64_t *)malloc(sizeof(int64_t) * (size_t)W);
    char *rev = (char *)malloc((size_t)(m + n + 1));
    if (!P || !Hrow || !Frow || !rev) { free(P); free(Hrow); free(Frow); free(rev); return -2; }
    for (int64_t j = 0; j <= n; j++) { Hrow[j] = 0; Frow[j] = ORACLE_NEG_INF; }
    /* row 0 and column 0 hold H = 0: source "zero", the walk stops there */
    for (int64_t j = 0; j <= n; j++) P[j] = 0;
    for (int64_t i = 0; i <= m; i++) P[(size_t)i * (size_t)W] = 0;

    int64_t best = 0, bi = 0, bj = 0;
    for (int64_t i = 1; i <= m; i++) {
        int64_t Ecur = ORACLE_NEG_INF, Hleft = 0, Hdiag = Hrow[0];
        for (int64_t j = 1; j <= n; j++) {
            int64_t Hup = Hrow[j];
            int64_t e_ext = Ecur - e, e_open = Hleft - o;
            Ecur = max2(e_ext, e_open);
            int64_t f_ext = Frow[j] - e, f_open = Hup - o;
            int64_t Fcur = max2(f_ext, f_open);
            int64_t diag = Hdiag + S[a[i - 1] * K + b[j - 1]];
            int64_t h = max2(max2(max2(diag, Ecur), Fcur), 0);
            uint8_t src;
            if (h == 0) src = 0;
            else if (h == diag) src = 1;
            else if (h == Ecur) src = 2;
            else src = 3;
            uint8_t p = src;
            if (Ecur == e_open) p |= 4;
            if (Fcur == f_open) p |= 8;
            P[(size_t)i * (size_t)W + (size_t)j] = p;
            Frow[j] = Fcur;
            Hdiag = Hup;
            Hrow[j] = h;
            Hleft = h;
            if (h > 0 && better_end(h, i, j, best, bi, bj)) { best = h; bi = i; bj = j; }
        }
    }

    int64_t i = bi, j = bj, k = 0;
    int state = 0;
    if (best > 0) {
        for (;;) {
            uint8_t p = P[(size_t)i * (size_t)W + (size_t)j];
            if (state == 0) {
                uint8_t src = p & 3;
                if (src == 0) break;
                if (src == 1) { rev[k++] = 'M'; i--; j--; }
                else if (src == 2) state = 1;
                else state = 2;
            } else if (state == 1) {
                rev[k++] = 'I';
                if (p & 4) state = 0;
                j--;
            } else {
                rev[k++] = 'D';
                if (p & 8) state = 0;
                i--;
            }
        }
    }
    for (int64_t t = 0; t < k; t++) ops[t] = rev[k - 1 - t];
    *n_ops = k;
    *score = best;
    *a_end = best > 0 ? bi : 0;
    *b_end = best > 0 ? bj : 0;
    *a_begin = best > 0 ? i : 0;
    *b_begin = best > 0 ? j : 0;
    free(P); free(Hrow); free(Frow); free(rev);
    return 0;
}

/*
 * The four algorithms of the paper's Section 2.1 (SW, NW, HW, OV), written
 * out as one full-matrix dynamic programme per algorithm.  The paper
 * describes them in words only; this file takes these readings:
 *
 *   SW (alg 0)  local: the Smith-Waterman recurrence above (zero floor,
 *               best cell anywhere).
 *   NW (alg 1)  global: every residue of a and of b is aligned.  Borders
 *               H(0,0) = 0, H(i,0) = -(o + (i-1)e), H(0,j) = -(o + (j-1)e);
 *               no zero floor; the end cell is (m, n).
 *   HW (alg 2)  semi-global: all of a is aligned against a substring of b,
 *               so gaps before and after it in b are free.  Borders
 *               H(0,j) = 0, H(i,0) = -(o + (i-1)e); no zero floor; the end
 *               cell is the best of the last row H(m, j), j = 0 .. n.
 *   OV (alg 3)  overlap: leading and trailing gaps of both sequences are
 *               free.  Borders H(0,j) = H(i,0) = 0; no zero floor; the end
 *               cell is the best of the last row and the last column.
 *
 * In every algorithm E(i,0) = F(0,j) = -infinity and the interior cells
 * follow the Gotoh recurrence (E, F as above; H the maximum of diagonal, E
 * and F, plus 0 for SW only).  Among equal maxima the end cell is the
 * first in row-major order (smallest row, then smallest column).  The
 * traceback starts at the end cell in state H with the SW priorities
 * (diagonal, then E, then F; inside a gap leave it before extending it)
 * and stops where the algorithm lets an alignment start: SW at a cell with
 * H = 0 (or the border), NW at (0, 0), HW at row 0, OV at row 0 or column
 * 0.  At a border cell that is not a free start the rest of the path is
 * forced: (i, 0) is reached by i deletions from (0, 0) and (0, j) by j
 * insertions.
 *
 * oracle_align_alg stores H, E and F for every cell (24 bytes per cell);
 * oracle_score_alg keeps two rows and returns the score and end cell only.
 * alg outside 0..3 is an argument error.
 */
static int64_t border_gap(int64_t k, int o, int e) { return k == 0 ? 0 : -((int64_t)o + (k - 1) * (int64_t)e); }

static int64_t left_border(int alg, int64_t i, int o, int e) {   /* H(i, 0) */
    return (alg == 1 || alg == 2) ? border_gap(i, o, e) : 0;
}

static int64_t top_border(int alg, int64_t j, int o, int e) {    /* H(0, j) */
    return alg == 1 ? border_gap(j, o, e) : 0;
}

/* Is (i, j) a cell where an alignment of algorithm alg may end? */
static int end_allowed(int alg, int64_t i, int64_t j, int64_t m, int64_t n) {
    switch (alg) {
        case 0: return i > 0 && j > 0;
        case 1: return i == m && j == n;
        case 2: return i == m;
        default: return i == m || j == n;
    }
}

int oracle_align_alg(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                     const int8_t *S, int K, int o, int e, int alg,
                     int64_t *score, int64_t *a_begin, int64_t *a_end,
                     int64_t *b_begin, int64_t *b_end, char *ops, int64_t *n_ops)
{
    if (!args_ok(a, m, b, n, S, K, o, e) || alg < 0 || alg > 3 || !score || !a_begin || !a_end ||
        !b_begin || !b_end || !n_ops || (m + n > 0 && !ops)) return -1;
    const int64_t W = n + 1;
    const size_t cells = (size_t)(m + 1) * (size_t)W;
    int64_t *H = (int64_t *)malloc(sizeof(int64_t) * cells);
    int64_t *E = (int64_t *)malloc(sizeof(int64_t) * cells);
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * cells);
    char *rev = (char *)malloc((size_t)(m + n + 1));
    if (!H || !E || !F || !rev) { free(H); free(E); free(F); free(rev); return -2; }
#define AT(X, i, j) X[(size_t)(i) * (size_t)W + (size_t)(j)]
    for (int64_t j = 0; j <= n; j++) { AT(H, 0, j) = top_border(alg, j, o, e); AT(E, 0, j) = ORACLE_NEG_INF; AT(F, 0, j) = ORACLE_NEG_INF; }
    for (int64_t i = 0; i <= m; i++) { AT(H, i, 0) = left_border(alg, i, o, e); AT(E, i, 0) = ORACLE_NEG_INF; AT(F, i, 0) = ORACLE_NEG_INF; }
    for (int64_t i = 1; i <= m; i++) {
        for (int64_t j = 1; j <= n; j++) {
            AT(E, i, j) = max2(AT(E, i, j - 1) - e, AT(H, i, j - 1) - o);
            AT(F, i, j) = max2(AT(F, i - 1, j) - e, AT(H, i - 1, j) - o);
            int64_t h = AT(H, i - 1, j - 1) + S[a[i - 1] * K + b[j - 1]];
            h = max2(h, AT(E, i, j));
            h = max2(h, AT(F, i, j));
            if (alg == 0) h = max2(h, 0);
            AT(H, i, j) = h;
        }
    }
    /* end cell: the first maximum in row-major order among the allowed cells
       (SW: only positive scores; score 0 means the empty alignment) */
    int found = 0;
    int64_t best = 0, bi = 0, bj = 0;
    for (int64_t i = 0; i <= m; i++)
        for (int64_t j = 0; j <= n; j++) {
            if (!end_allowed(alg, i, j, m, n)) continue;
            const int64_t h = AT(H, i, j);
            if (alg == 0 && h <= 0) continue;
            if (!found || h > best) { best = h; bi = i; bj = j; found = 1; }
        }
    int64_t i = bi, j = bj, k = 0;
    if (found) {
        int state = 0;      /* 0 = H, 1 = E, 2 = F */
        for (;;) {
            if (state == 0) {
                const int64_t h = AT(H, i, j);
                if (alg == 0 && h == 0) break;
                if (i == 0 && j == 0) break;
                if (i == 0) {                              /* top border */
                    if (alg != 1) break;                   /* a free start for HW and OV */
                    while (j > 0) { rev[k++] = 'I'; j--; }
                    break;
                }
                if (j == 0) {                              /* left border */
                    if (alg == 0 || alg == 3) break;       /* a free start for SW and OV */
                    while (i > 0) { rev[k++] = 'D'; i--; }
                    break;
                }
                if (h == AT(H, i - 1, j - 1) + S[a[i - 1] * K + b[j - 1]]) {
                    rev[k++] = 'M'; i--; j--;
                } else if (h == AT(E, i, j)) {
                    state = 1;
                } else {
                    state = 2;
                }
            } else if (state == 1) {
                rev[k++] = 'I';
                if (AT(E, i, j) == AT(H, i, j - 1) - o) state = 0;
                j--;
            } else {
                rev[k++] = 'D';
                if (AT(F, i, j) == AT(H, i - 1, j) - o) state = 0;
                i--;
            }
        }
    }
#undef AT
    for (int64_t t = 0; t < k; t++) ops[t] = rev[k - 1 - t];
    *n_ops = k;
    *score = found ? best : 0;
    *a_end = found ? bi : 0;
    *b_end = found ? bj : 0;
    *a_begin = found ? i : 0;
    *b_begin = found ? j : 0;
    free(H); free(E); free(F); free(rev);
    return 0;
}

int oracle_score_alg(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                     const int8_t *S, int K, int o, int e, int alg,
                     int64_t *score, int64_t *a_end, int64_t *b_end)
{
    if (!args_ok(a, m, b, n, S, K, o, e) || alg < 0 || alg > 3 || !score || !a_end || !b_end) return -1;
    int64_t *Hrow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *Frow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!Hrow || !Frow) { free(Hrow); free(Frow); return -2; }
    int found = 0;
    int64_t best = 0, bi = 0, bj = 0;
    for (int64_t j = 0; j <= n; j++) {
        Hrow[j] = top_border(alg, j, o, e);
        Frow[j] = ORACLE_NEG_INF;
        if (end_allowed(alg, 0, j, m, n) && (alg != 0) && (!found || Hrow[j] > best)) {
            best = Hrow[j]; bi = 0; bj = j; found = 1;
        }
    }
    for (int64_t i = 1; i <= m; i++) {
        int64_t Ecur = ORACLE_NEG_INF;
        int64_t Hleft = left_border(alg, i, o, e);
        int64_t Hdiag = Hrow[0];
        Hrow[0] = Hleft;
        if (alg != 0 && end_allowed(alg, i, 0, m, n) && (!found || Hleft > best)) {
            best = Hleft; bi = i; bj = 0; found = 1;
        }
        for (int64_t j = 1; j <= n; j++) {
            const int64_t Hup = Hrow[j];
            Ecur = max2(Ecur - e, Hleft - o);
            const int64_t Fcur = max2(Frow[j] - e, Hup - o);
            int64_t h = Hdiag + S[a[i - 1] * K + b[j - 1]];
            h = max2(h, Ecur);
            h = max2(h, Fcur);
            if (alg == 0) h = max2(h, 0);
            Frow[j] = Fcur;
            Hdiag = Hup;
            Hrow[j] = h;
            Hleft = h;
            if (end_allowed(alg, i, j, m, n) && !(alg == 0 && h <= 0) && (!found || h > best)) {
                best = h; bi = i; bj = j; found = 1;
            }
        }
    }
    free(Hrow); free(Frow);
    *score = found ? best : 0;
    *a_end = found ? bi : 0;
    *b_end = found ? bj : 0;
    return 0;
}

/*
 * Residue encoding: codes[k] = position of text[k] in the alphabet string
 * (case-insensitive for letters), or -1 in *bad_index for the first
 * character that is not in it.  Returns 0, or 1 when a character was not
 * found.
 */
int oracle_encode(const char *alphabet, const char *text, int64_t len,
                  uint8_t *codes, int64_t *bad_index)
{
    if (!alphabet || (len > 0 && (!text || !codes)) || !bad_index || len < 0) return -1;
    size_t K = strlen(alphabet);
    *bad_index = -1;
    for (int64_t k = 0; k < len; k++) {
        char c = text[k];
        if (c >= 'a' && c <= 'z') c = (char)(c - 'a' + 'A');
        size_t x = 0;
        while (x < K && alphabet[x] != c) x++;
        if (x == K) { *bad_index = k; return 1; }
        codes[k] = (uint8_t)x;
    }
    return 0;
}
