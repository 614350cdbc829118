// fill16.cu -- launches of the packed 16-bit pair fill (wavefront16.cuh) and
// the test of whether a scoring scheme and tile shape keep it exact.
#include "sw.h"
#include "sw_ctx.h"
#include "wavefront16.cuh"

#include <algorithm>

using namespace swgb;

#define CU(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; } } while (0)

namespace {

// largest pair profile (small alphabets); larger alphabets take the int16 profile
constexpr size_t kPairProfileMax = 110 * 1024;

template <int R, int W, int MODE, int PK, bool LEFT>
int launch16(sw_ctx *c, const FillLaunch &L, int K, long long tickets, int max_blocks) {
    auto kern = wavefront16_kernel<R, W, MODE, PK, LEFT>;
    const size_t smem = p16_profile_bytes(R, W, K, PK);
    static int attr_set[64] = {0};
    if (c->device >= 64 || !attr_set[c->device]) {
        const size_t cap = PK == kP16Pair ? kPairProfileMax : p16_profile_bytes(R, W, kMaxAlphabet, PK);
        CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
        if (c->device < 64) attr_set[c->device] = 1;
    }
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (W + 2) * 32, smem));
    if (occ < 1) return SW_ECUDA;
    if (max_blocks > 0) occ = std::min(occ, max_blocks);
    const long long grid = std::min<long long>(tickets, (long long)occ * c->nsm);
    const int kp = kt_begin(c, SW_KT_FILL);
    kern<<<(unsigned)grid, (W + 2) * 32, smem, c->stream>>>(L);
    kt_end(c, kp);
    CU(cudaGetLastError());
    ++c->launches;
    return SW_OK;
}

template <int R, int MODE, bool LEFT = false, int W = 4>
int launch16_pk(sw_ctx *c, const FillLaunch &L, int K, long long tickets, int B) {
    if (p16_profile_bytes(R, W, K, kP16Pair) <= kPairProfileMax)
        return launch16<R, W, MODE, kP16Pair, LEFT>(c, L, K, tickets, B);
    return launch16<R, W, MODE, kP16Int16, LEFT>(c, L, K, tickets, B);
}

// left: the coarse-tile refills (checkpoint mode only), whose tasks enter the
// fill at a checkpoint column.  W = 2 (score mode only): blocks of two compute
// warps for batches, whose pairs' last strips are partly empty (a strip of
// four warps runs its pair's width with one to four of them busy).
template <int R>
int launch16_mode(sw_ctx *c, int mode, bool left, int W, const FillLaunch &L, int K, long long tickets, int B) {
    if (W == 2) return mode == kModeScore && !left ? launch16_pk<R, kModeScore, false, 2>(c, L, K, tickets, B) : SW_EINVAL;
    if (W != 4) return SW_EINVAL;
    if (left) return mode == kModeScoreCk ? launch16_pk<R, kModeScoreCk, true>(c, L, K, tickets, B) : SW_EINVAL;
    switch (mode) {
        case kModeScore: return launch16_pk<R, kModeScore>(c, L, K, tickets, B);
        case kModeScoreCk: return launch16_pk<R, kModeScoreCk>(c, L, K, tickets, B);
        default: return SW_EINVAL;
    }
}

}  // namespace

bool swgb::p16_fits(const DevScoring &s, int R) {
    if (R != 8 && R != 12 && R != 16) return false;
    if (s.alg != kAlgLocal) return false;            // the packed fill keeps the zero floor
    int lo = 127, hi = -128;
    for (int k = 0; k < s.K * s.K; ++k) { lo = std::min(lo, (int)s.mat[k]); hi = std::max(hi, (int)s.mat[k]); }
    return p16_spread(R, s.go, s.ge, hi, lo) < kP16Span;
}

int swgb::launch_fill16(sw_ctx *c, const FillConfig &cfg, int mode, const FillLaunch &L, int K,
                        long long tickets) {
    if (tickets <= 0) return SW_OK;
    switch (cfg.R) {
        case 8: return launch16_mode<8>(c, mode, cfg.left != 0, cfg.W, L, K, tickets, cfg.B);
        case 12: return launch16_mode<12>(c, mode, cfg.left != 0, cfg.W, L, K, tickets, cfg.B);
        case 16: return launch16_mode<16>(c, mode, cfg.left != 0, cfg.W, L, K, tickets, cfg.B);
        default: return SW_EINVAL;
    }
}
