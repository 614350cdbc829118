// noalloc.cu -- sw_score_noalloc: the pairwise score / end-cell fill for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a serving process whose own caching
// allocator owns the whole device memory budget, a latency-critical
// pipeline that must not hit the implicit device synchronisation of
// cudaMalloc / cudaFree, or a plug-in that is given a stream and buffers but
// no allocation rights.  This entry point allocates nothing: every scratch
// byte the fill needs (boundary-row ring, per-strip progress counters and
// end-cell candidates, ticket counter, error word, task and scoring records)
// lives in one file-scope __device__ array, g_noalloc_scratch, of
// kNoAllocScratchBytes.  Each GPU that loads the library holds that array
// until the process exits.
//
// The array's name is only a host-side stand-in in host code, so every call
// looks up its device address with cudaGetSymbolAddress in the current
// context (and sets the fill's shared-memory limit there).  Nothing is
// cached across calls: a device reset (cudaDeviceReset) or a new primary
// context reloads the module, possibly at another address, and a cached
// address would then point at freed memory.  The first call in a context
// loads the module and should come before any stream capture; later
// lookups are host-side table reads.  Every call shares the array and it keeps
// the previous call's contents, so each call clears the counters that must
// start at zero; calls whose work overlaps on the GPU (different streams,
// or host threads racing) would race on the array and must be serialised
// by the caller.
#include "sw.h"
#include "sw_ctx.h"
#include "wavefront.cuh"
#include "aux_kernels.cuh"

#include <algorithm>
#include <cstring>

using namespace swgb;

namespace {

constexpr int kR = 8, kW = 4;                         // tile shape of the fill
constexpr int kHC = kW * 32 * kR;                     // rows per strip
constexpr long long kMaxCols = 262144;                // longest b
constexpr long long kMaxStrips = 16384;               // longest a = kMaxStrips * kHC rows
constexpr int kSlots = 2;                             // boundary-row ring (safe for >= 2)

// layout of the scratch array (byte offsets, each 256-byte aligned)
constexpr size_t kOffRing = 0;
constexpr size_t kOffProg = kOffRing + (size_t)kSlots * kMaxCols * sizeof(int2);
constexpr size_t kOffCand = kOffProg + (size_t)kMaxStrips * sizeof(int);
constexpr size_t kOffTask = kOffCand + (size_t)kMaxStrips * sizeof(int4);
constexpr size_t kOffScoring = kOffTask + 256;
constexpr size_t kOffMisc = kOffScoring + ((sizeof(DevScoring) + 255) / 256) * 256;  // ticket, err, result
constexpr size_t kNoAllocScratchBytes = kOffMisc + 256;
static_assert(sizeof(FillTask) <= 256, "task record must fit its slot");

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array in the current context, and the
// fill's shared-memory limit there.
int setup_device(unsigned char **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return SW_ECUDA;
    }
    if (cudaFuncSetAttribute(wavefront_kernel<kR, kW, kModeScore, kProf8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (kMaxAlphabet + 1) * kHC) != cudaSuccess) {
        cudaGetLastError();
        return SW_ECUDA;
    }
    *out = static_cast<unsigned char *>(p);
    return SW_OK;
}

}  // namespace

#define CU(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; } } while (0)

extern "C" int sw_score_noalloc(void *cuda_stream, const uint8_t *a, int64_t m, const uint8_t *b,
                                int64_t n, const sw_scoring *sc, sw_hit *out) {
    if (!out) return SW_EINVAL;
    DevScoring ds;
    int rc = check_scoring(sc, &ds);
    if (rc) return rc;
    if (ds.alg != kAlgLocal) return SW_EINVAL;          // the local algorithm only
    if (m < 0 || n < 0 || (m > 0 && !a) || (n > 0 && !b)) return SW_EINVAL;
    const long long nstrips = (m + kHC - 1) / kHC;
    if (n > kMaxCols || nstrips > kMaxStrips) return SW_ERANGE;
    if ((double)std::min(m, n) * (double)max_pos_score(sc) >= (double)kMaxScoreBound) return SW_ERANGE;
    if (m == 0 || n == 0) { *out = sw_hit{0, 0, 0, 0}; return SW_OK; }
    if (!is_device_ptr(a) || !is_device_ptr(b)) return SW_EINVAL;   // inputs must already be on the device
    int dev = 0;
    CU(cudaGetDevice(&dev));
    unsigned char *base = nullptr;
    rc = setup_device(&base);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    int2 *ring = reinterpret_cast<int2 *>(base + kOffRing);
    int *prog = reinterpret_cast<int *>(base + kOffProg);
    int4 *cand = reinterpret_cast<int4 *>(base + kOffCand);
    FillTask *task = reinterpret_cast<FillTask *>(base + kOffTask);
    DevScoring *scoring = reinterpret_cast<DevScoring *>(base + kOffScoring);
    unsigned long long *ticket = reinterpret_cast<unsigned long long *>(base + kOffMisc);
    int *err = reinterpret_cast<int *>(base + kOffMisc + 8);
    int4 *result = reinterpret_cast<int4 *>(base + kOffMisc + 16);

    FillTask t{};
    t.a = a; t.b = b;
    t.rows = (int32_t)m; t.ncols = (int32_t)n;
    t.nstrips = (int32_t)nstrips;
    t.scoring = 0; t.ticket0 = 0; t.top = nullptr;
    t.bnd = ring; t.nslot = kSlots;
    t.ckpt_every = 0; t.ckpt = nullptr; t.row0 = 0; t.tb = nullptr; t.tb_ld = 0;

    // the array keeps the last call's contents: clear what must start at zero
    CU(cudaMemsetAsync(prog, 0, (size_t)nstrips * sizeof(int), st));
    CU(cudaMemsetAsync(base + kOffMisc, 0, 256, st));
    CU(cudaMemcpyAsync(task, &t, sizeof(t), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(scoring, &ds, sizeof(ds), cudaMemcpyHostToDevice, st));

    int nsm = 0;
    CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256;
    validate_codes_kernel<<<(unsigned)std::min<long long>((m + threads - 1) / threads, 4LL * nsm), threads, 0, st>>>(a, m, ds.K, err);
    validate_codes_kernel<<<(unsigned)std::min<long long>((n + threads - 1) / threads, 4LL * nsm), threads, 0, st>>>(b, n, ds.K, err);
    CU(cudaGetLastError());

    FillLaunch L{};
    L.tasks = task; L.scorings = scoring; L.ticket = ticket; L.prog = prog; L.cand = cand;
    L.err = err; L.total = nstrips; L.spin_limit = 1LL << 26; L.ntasks = 1;
    const size_t smem = (size_t)(ds.K + 1) * kHC;
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, wavefront_kernel<kR, kW, kModeScore, kProf8>, (kW + 2) * 32, smem));
    if (occ < 1) return SW_ECUDA;
    const long long grid = std::min<long long>(nstrips, (long long)occ * nsm);
    wavefront_kernel<kR, kW, kModeScore, kProf8><<<(unsigned)grid, (kW + 2) * 32, smem, st>>>(L);
    CU(cudaGetLastError());
    reduce_candidates_kernel<<<1, 32, 0, st>>>(task, 1, cand, scoring, result);
    CU(cudaGetLastError());

    int4 res[2];
    CU(cudaMemcpyAsync(res, result, sizeof(int4), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&res[1], err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    rc = map_kernel_error(res[1].x);
    if (rc) return rc;
    *out = sw_hit{res[0].x, 0, (int64_t)res[0].y, (int64_t)res[0].z};
    return SW_OK;
}
