// sw_device.cuh -- device-side building blocks shared by the kernels of
// libswgb: constants, the scoring table, packed-byte helpers and the
// inter-block progress flags.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace swgb {

constexpr int kNeg = -(1 << 30);      // stands for -infinity in int32 lanes
// Scores of the int32 fill stay below this bound (min(m, n) * max S < it):
// the fill keys rows as U * 16 + tag, which must not overflow int32.
constexpr long long kMaxScoreBound = 1LL << 26;
constexpr int kPadScore = -128;       // profile value of padding rows / columns
constexpr int kMaxAlphabet = 32;
constexpr unsigned kFull = 0xffffffffu;

// Error codes written by kernels into the context's error word.
constexpr int kErrTimeout = 1;        // a bounded inter-block wait gave up
constexpr int kErrBadCode = 2;        // a residue code >= alphabet
constexpr int kErrOverflow = 3;       // a score would leave the int32 range

struct DevScoring {
    int8_t mat[kMaxAlphabet * kMaxAlphabet];   // mat[x*K + y]: a-residue x vs b-residue y
    int32_t K;
    int32_t go;     // gap open (positive, subtracted)
    int32_t ge;     // gap extend (positive, subtracted)
    int32_t alg;    // kAlgLocal, kAlgGlobal, kAlgSemiGlobal or kAlgOverlap
};

// The algorithms of paper Section 2.1.  Local: Smith-Waterman (zero floor,
// best cell anywhere).  Global (NW): all of a against all of b, gaps at the
// borders charged, end cell (m, n).  Semi-global (HW): all of a against a
// substring of b, so row 0 is free and the end cell is the best of the last
// row.  Overlap (OV): rows 0 and column 0 free, end cell the best of the
// last row and the last column.  No zero floor except for the local one.
enum Alg { kAlgLocal = 0, kAlgGlobal = 1, kAlgSemiGlobal = 2, kAlgOverlap = 3 };

// Cost of a gap of k letters, o + (k - 1) e, negated; 0 for k = 0.
__host__ __device__ __forceinline__ long long neg_gap(long long k, int go, int ge) {
    return k == 0 ? 0 : -((long long)go + (k - 1) * (long long)ge);
}
// H of the matrix's left border, H(i, 0), and of its top border, H(0, j).
__host__ __device__ __forceinline__ long long left_border_h(int alg, long long i, int go, int ge) {
    return (alg == kAlgGlobal || alg == kAlgSemiGlobal) ? neg_gap(i, go, ge) : 0;
}
__host__ __device__ __forceinline__ long long top_border_h(int alg, long long j, int go, int ge) {
    return alg == kAlgGlobal ? neg_gap(j, go, ge) : 0;
}
constexpr int kNoScore = -0x7fffffff - 1;   // no end-cell candidate (the other algorithms' scores may be <= 0)

// Order of end-cell candidates: larger score, then smaller row i, then
// smaller column j (the first maximum in row-major order).
__host__ __device__ __forceinline__ bool cand_better(int s1, int j1, int i1, int s2, int j2, int i2) {
    if (s1 != s2) return s1 > s2;
    if (i1 != i2) return i1 < i2;
    return j1 < j2;
}

// The end cells of the global, semi-global and overlap algorithms that lie
// on the matrix border (the fill computes rows and columns from 1 on):
// folded into the candidate (cs, ci, cj) by the same order.  Global: (m, n)
// when m or n is 0; semi-global: (m, 0); overlap: (0, n), (m, 0), and
// (0, 0) when m or n is 0 (row 0 or column 0 is then an end line).
__host__ __device__ inline void border_end_candidates(int alg, long long m, long long n, int go, int ge, int *cs,
                                                      int *ci, int *cj) {
    auto take = [&](long long sc, long long i, long long j) {
        if (cand_better((int)sc, (int)j, (int)i, *cs, *cj, *ci)) { *cs = (int)sc; *ci = (int)i; *cj = (int)j; }
    };
    if (alg == kAlgGlobal) {
        if (m == 0) take(top_border_h(alg, n, go, ge), 0, n);
        else if (n == 0) take(left_border_h(alg, m, go, ge), m, 0);
    } else if (alg == kAlgSemiGlobal) {
        take(left_border_h(alg, m, go, ge), m, 0);
    } else if (alg == kAlgOverlap) {
        take(0, 0, n);
        take(0, m, 0);
        if (m == 0 || n == 0) take(0, 0, 0);
    }
}

// Sign-extend byte k of w to int32 with one byte permute (prmt with the
// sign-replicate selector bit).
template <int k>
__device__ __forceinline__ int sext8(uint32_t w) {
    constexpr uint32_t sel = k | ((8 | k) << 4) | ((8 | k) << 8) | ((8 | k) << 12);
    uint32_t d;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(w), "n"(sel));
    return static_cast<int>(d);
}

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Four (a, b) pairs stored to p[0..3] (32 bytes, 16-byte aligned) only when
// pred != 0, as predicated instructions (no branch in the caller's stream).
__device__ __forceinline__ void st_global_4x2_if(unsigned pred, int2 *p, int a0, int b0, int a1, int b1,
                                                 int a2, int b2, int a3, int b3) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t"
                 "@q st.global.v4.s32 [%1], {%2, %3, %4, %5};\n\t"
                 "@q st.global.v4.s32 [%1+16], {%6, %7, %8, %9};\n\t}"
                 :: "r"(pred), "l"(p), "r"(a0), "r"(b0), "r"(a1), "r"(b1), "r"(a2), "r"(b2), "r"(a3), "r"(b3));
}

__device__ __forceinline__ int ld_volatile(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}

}  // namespace swgb
