// aux_kernels.cuh -- small kernels around the fill: residue encoding, code
// validation and the traceback walk over recomputed decision bits.
#pragma once
#include "sw_device.cuh"

namespace swgb {

// codes[k] = table[text[k]]; table maps a byte to its code or 255.  The
// first position holding an unknown letter is recorded in *bad (atomicMin).
static __global__ void encode_kernel(const uint8_t *__restrict__ text, long long len,
                              const uint8_t *__restrict__ table, uint8_t *__restrict__ codes,
                              unsigned long long *bad)
{
    __shared__ uint8_t t[256];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) t[k] = table[k];
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += stride) {
        const uint8_t c = t[text[k]];
        codes[k] = c;
        if (c == 255) atomicMin(bad, (unsigned long long)k);
    }
}

// Sets *err = kErrBadCode if any code is >= K.
static __global__ void validate_codes_kernel(const uint8_t *__restrict__ s, long long len, int K, int *err)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += stride)
        bad |= s[k] >= K;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(err, 0, kErrBadCode);
}

// State of the traceback walk, kept on the device between row groups.
struct WalkState {
    int32_t i, j;          // current cell (1-based rows/cols; 0 = border)
    int32_t state;         // 0 = H, 1 = E, 2 = F
    int32_t done;          // 1 once the walk reached a zero cell or the border, 2 on inconsistent bits
    int64_t nruns;         // run records written so far
    int32_t cur_op;        // op of the open run (0 = M, 1 = I, 2 = D, -1 = none)
    int32_t cur_len;
};

// Walk the canonical path through one group of rows (G0, G1] using the
// decision bits of that group: word ((i-1-G0)/R)*ld + (j-1), nibble
// (i-1-G0) % R.  Runs of equal operations are appended to `runs` as
// (op, length) from the end of the alignment towards its start.  The walk
// follows these rules (one per decision bit):
//   state H: stop if the H source is zero; diagonal -> emit M, go up-left;
//            source E -> state E; source F -> state F;
//   state E: emit I, go left; back to H if the E-opened bit is set;
//   state F: emit D, go up; back to H if the F-opened bit is set.
// Runs until the walk stops or leaves the group at its top (i <= G0).
template <typename Word, int R>
__global__ void walk_kernel(const Word *__restrict__ tb, long long ld, int G0,
                            WalkState *st, int2 *runs)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    WalkState w = *st;
    auto emit = [&](int op) {
        if (op == w.cur_op) { ++w.cur_len; return; }
        if (w.cur_len > 0) runs[w.nruns++] = make_int2(w.cur_op, w.cur_len);
        w.cur_op = op;
        w.cur_len = 1;
    };
    auto nib = [&](int i, int j) -> unsigned {
        const int r = i - 1 - G0;
        const Word x = tb[(size_t)(r / R) * (size_t)ld + (size_t)(j - 1)];
        return (unsigned)(x >> (4 * (r % R))) & 15u;
    };
    while (!w.done) {
        if (w.state == 0) {
            if (w.i == 0 || w.j == 0) { w.done = 1; break; }
            if (w.i <= G0) break;
            const unsigned src = nib(w.i, w.j) & 3u;
            if (src == 0) { w.done = 1; break; }
            if (src == 1) { emit(0); --w.i; --w.j; }
            else w.state = (src == 2) ? 1 : 2;
        } else if (w.state == 1) {
            if (w.i <= G0) break;
            if (w.j <= 0) { w.done = 2; break; }       // inconsistent bits: report, never read column 0
            const unsigned x = nib(w.i, w.j);
            emit(1);
            if (x & 4u) w.state = 0;
            --w.j;
        } else {
            if (w.i <= G0) break;
            const unsigned x = nib(w.i, w.j);
            emit(2);
            if (x & 8u) w.state = 0;
            --w.i;
        }
    }
    if (w.done == 1 && w.cur_len > 0) {
        runs[w.nruns++] = make_int2(w.cur_op, w.cur_len);
        w.cur_len = 0;
        w.cur_op = -1;
    }
    *st = w;
}

}  // namespace swgb
