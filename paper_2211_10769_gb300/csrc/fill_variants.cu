// fill_variants.cu -- launches of the int32 wavefront fill for the global,
// semi-global and overlap algorithms of paper Section 2.1 (no zero floor,
// algorithm-specific borders and end cells; wavefront.cuh with LOCAL =
// false), in their own translation unit so that they compile in parallel
// with the local fill.
#include "sw.h"
#include "sw_ctx.h"
#include "wavefront.cuh"

#include <algorithm>

using namespace swgb;

#define CU(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; } } while (0)

namespace {

constexpr size_t kProf32MaxBytes = 64 * 1024;    // as the local fill: an int32 profile up to this size

template <int R, int MODE, int PK>
int launch_v(sw_ctx *c, const FillLaunch &L, int K, long long tickets, int max_blocks) {
    constexpr int W = 4;
    auto kern = wavefront_kernel<R, W, MODE, PK, false>;
    constexpr int HC = W * 32 * R;
    constexpr size_t PB = PK == kProf32 ? 4 : 1;
    const size_t smem = (size_t)(K + 1) * HC * PB;
    static int attr_set[64] = {0};
    if (c->device >= 64 || !attr_set[c->device]) {
        const size_t cap = PK == kProf32 ? kProf32MaxBytes : (size_t)(kMaxAlphabet + 1) * HC;
        CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
        if (c->device < 64) attr_set[c->device] = 1;
    }
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (W + 2) * 32, smem));
    if (occ < 1) return SW_ECUDA;
    if (max_blocks > 0) occ = std::min(occ, max_blocks);
    const long long grid = std::min<long long>(tickets, (long long)occ * c->nsm);
    const int kp = kt_begin(c, MODE == kModeTb ? SW_KT_FILL_TB : SW_KT_FILL);
    kern<<<(unsigned)grid, (W + 2) * 32, smem, c->stream>>>(L);
    kt_end(c, kp);
    CU(cudaGetLastError());
    ++c->launches;
    return SW_OK;
}

template <int R, int MODE>
int launch_v_pk(sw_ctx *c, bool fold, const FillLaunch &L, int K, long long tickets, int B) {
    const bool p32 = c->prof32 && (size_t)(K + 1) * (size_t)(4 * 32 * R) * 4 <= kProf32MaxBytes;
    if (p32) return launch_v<R, MODE, kProf32>(c, L, K, tickets, B);
    if (fold) return launch_v<R, MODE, kProf8Fold>(c, L, K, tickets, B);
    return launch_v<R, MODE, kProf8>(c, L, K, tickets, B);
}

template <int R>
int launch_v_mode(sw_ctx *c, int mode, bool fold, const FillLaunch &L, int K, long long tickets, int B) {
    switch (mode) {
        case kModeScore: return launch_v_pk<R, kModeScore>(c, fold, L, K, tickets, B);
        case kModeScoreCk: return launch_v_pk<R, kModeScoreCk>(c, fold, L, K, tickets, B);
        case kModeTb: return launch_v_pk<R, kModeTb>(c, fold, L, K, tickets, B);
        default: return SW_EINVAL;
    }
}

}  // namespace

// The fewest rows a lane (8, 12 or 16) that give at most one strip per SM,
// as for the local fill: the strips of a pair form one chain.
FillConfig swgb::variant_fill_config(const sw_ctx *c, int64_t rows) {
    int R = 16;
    for (int r : {8, 12}) {
        const int64_t sh = 4LL * 32 * r;
        if ((rows + sh - 1) / sh <= (int64_t)c->nsm) { R = r; break; }
    }
    FillConfig f{R, 4, 0, 2};
    f.alg = 1;
    return f;
}

int swgb::launch_fill_variant(sw_ctx *c, const FillConfig &cfg, int mode, bool fold, const FillLaunch &L, int K,
                              long long tickets) {
    if (tickets <= 0) return SW_OK;
    if (cfg.W != 4) return SW_EINVAL;
    switch (cfg.R) {
        case 8: return launch_v_mode<8>(c, mode, fold, L, K, tickets, cfg.B);
        case 12: return launch_v_mode<12>(c, mode, fold, L, K, tickets, cfg.B);
        case 16: return launch_v_mode<16>(c, mode, fold, L, K, tickets, cfg.B);
        default: return SW_EINVAL;
    }
}

// Scores of the int32 fill are keyed as U * 16 + row tag: |U| must stay below
// kMaxScoreBound.  The largest score is at most min(m, n) * max S.  Without
// the zero floor H(i, j) is still at least the score of the all-gap path to
// (i, j), -(2 open + (i + j) extend), so U = H - open and the values one step
// off it (E, F, H + S with a padding score of -128) stay above
// -(3 open + (m + n) extend + 256).
bool swgb::score_range_ok(const sw_scoring *sc, int64_t m, int64_t n) {
    if ((double)std::min(m, n) * (double)max_pos_score(sc) >= (double)kMaxScoreBound) return false;
    if (sc->algorithm == SW_ALG_LOCAL) return true;
    const double low = 3.0 * sc->gap_open + (double)(m + n) * sc->gap_extend + 256.0;
    return low < (double)kMaxScoreBound;
}
