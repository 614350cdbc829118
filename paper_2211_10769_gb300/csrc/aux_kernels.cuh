// aux_kernels.cuh -- small kernels around the fill: residue encoding and
// code validation.
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

}  // namespace swgb
