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
    int32_t pad_;
};

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

// Order of end-cell candidates: larger score, then smaller row i, then
// smaller column j (the first maximum in row-major order).
__device__ __forceinline__ bool cand_better(int s1, int j1, int i1, int s2, int j2, int i2) {
    if (s1 != s2) return s1 > s2;
    if (i1 != i2) return i1 < i2;
    return j1 < j2;
}

}  // namespace swgb
