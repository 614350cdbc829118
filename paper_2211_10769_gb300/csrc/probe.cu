// probe.cu -- measured integer instruction rates of the GPU (the denominator
// of the integer-ALU roofline): each probe kernel runs eight independent
// dependency chains of one instruction form per thread on every SM and
// reports warp-lane results per SM per clock, using the SM clock counter
// and the global nanosecond timer read inside the kernel.  A second probe
// runs one dependent chain in one warp and reports the latency of a form
// (SM clocks from one instruction to the next that needs its result), which
// bounds a wavefront step whose rows form such a chain.
#include "sw_probe.h"
#include "sw_ctx.h"

#include <algorithm>
#include <cstring>

namespace {

constexpr int kChains = 8;

template <int OP>
__device__ __forceinline__ unsigned step(unsigned x, unsigned y, unsigned z, unsigned c) {
    if constexpr (OP == SW_PROBE_IADD) return x + y;
    else if constexpr (OP == SW_PROBE_IMAX) return (unsigned)max((int)x, (int)y);
    else if constexpr (OP == SW_PROBE_VIADDMAX_S32) return (unsigned)__viaddmax_s32((int)x, (int)c, (int)y);
    else if constexpr (OP == SW_PROBE_VIMAX3_S32_RELU) return (unsigned)__vimax3_s32_relu((int)x, (int)y, (int)z);
    else if constexpr (OP == SW_PROBE_VIADDMAX_S16X2) return __viaddmax_s16x2(x, c, y);
    else if constexpr (OP == SW_PROBE_VIMAX3_S16X2_RELU) return __vimax3_s16x2_relu(x, y, z);
    else if constexpr (OP == SW_PROBE_PRMT) return __byte_perm(x, y, c);
    else if constexpr (OP == SW_PROBE_VADDUS4) return __vaddus4(x, y);
    else if constexpr (OP == SW_PROBE_VSUBUS4) return __vsubus4(x, y);
    else if constexpr (OP == SW_PROBE_VMAXU4) return __vmaxu4(x, y);
    else return x ^ __shfl_xor_sync(0xffffffffu, y, 1);
}

template <int OP>
__global__ void __launch_bounds__(256) probe_kernel(unsigned seed, int iters, unsigned *sink,
                                                    unsigned long long *clk)
{
    unsigned x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = seed * (threadIdx.x + 1) + k * 0x9e3779b9u;
    const unsigned c = seed | 1u;
    __syncthreads();
    unsigned long long c0 = clock64();
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                x[k] = step<OP>(x[k], x[(k + 1) % kChains], x[(k + 2) % kChains], c + u);
        }
    }
    __syncthreads();
    unsigned long long c1 = clock64();
    unsigned long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    unsigned acc = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc ^= x[k];
    if (acc == 0x12345678u) sink[threadIdx.x] = acc;     // keeps the chains live
    if (threadIdx.x == 0) {
        atomicMax(&clk[0], c1 - c0);
        atomicMax(&clk[1], t1 - t0);
    }
}

template <int OP>
int run(sw_ctx *c, int iters, double *per_sm_clk, double *mhz) {
    swgb::DevBuf buf;
    if (buf.ensure(4096)) return SW_ENOMEM;
    if (cudaMemsetAsync(buf.p, 0, 4096, c->stream) != cudaSuccess) return SW_ECUDA;
    const int blocks_per_sm = 8, threads = 256;
    const int grid = c->nsm * blocks_per_sm;
    unsigned long long *clk = reinterpret_cast<unsigned long long *>(static_cast<char *>(buf.p) + 2048);
    probe_kernel<OP><<<grid, threads, 0, c->stream>>>(0x1234567u, iters, static_cast<unsigned *>(buf.p), clk);
    if (cudaGetLastError() != cudaSuccess) return SW_ECUDA;
    ++c->launches;
    unsigned long long h[2];
    if (cudaMemcpyAsync(h, clk, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) return SW_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SW_ECUDA;
    const double ops_per_sm = (double)blocks_per_sm * threads * iters * 16.0 * kChains;
    *per_sm_clk = ops_per_sm / (double)h[0];          // lane results per SM per clock
    *mhz = (double)h[0] / (double)h[1] * 1000.0;      // clock ticks per ns -> MHz
    return SW_OK;
}

// One warp, one dependency chain: every instruction needs the previous
// one's result, so the SM clock ticks per instruction are its latency.
template <int OP>
__global__ void __launch_bounds__(32) latency_kernel(unsigned seed, int iters, unsigned *sink,
                                                      unsigned long long *clk)
{
    unsigned x = seed * (threadIdx.x + 1);
    const unsigned y = seed ^ 0x5bd1e995u, z = seed + 0x3c6ef372u, c = seed | 1u;
    __syncwarp();
    const unsigned long long c0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            if constexpr (OP == SW_PROBE_SHFL) x = __shfl_xor_sync(0xffffffffu, x, 1) + 1u;
            else x = step<OP>(x, y, z, c);
        }
    }
    __syncwarp();
    const unsigned long long c1 = clock64();
    if (x == 0x12345678u) sink[threadIdx.x] = x;          // keeps the chain live
    if (threadIdx.x == 0) clk[0] = c1 - c0;
}

template <int OP>
int run_latency(sw_ctx *c, int iters, double *cycles) {
    swgb::DevBuf buf;
    if (buf.ensure(4096)) return SW_ENOMEM;
    if (cudaMemsetAsync(buf.p, 0, 4096, c->stream) != cudaSuccess) return SW_ECUDA;
    unsigned long long *clk = reinterpret_cast<unsigned long long *>(static_cast<char *>(buf.p) + 2048);
    latency_kernel<OP><<<1, 32, 0, c->stream>>>(0x1234567u, iters, static_cast<unsigned *>(buf.p), clk);
    if (cudaGetLastError() != cudaSuccess) return SW_ECUDA;
    ++c->launches;
    unsigned long long h = 0;
    if (cudaMemcpyAsync(&h, clk, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) return SW_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SW_ECUDA;
    *cycles = (double)h / ((double)iters * 32.0);
    return SW_OK;
}

}  // namespace

extern "C" int sw_probe_latency(sw_ctx *c, int op, int iters, double *cycles) {
    if (!c || !cycles || iters < 1) return SW_EINVAL;
    swgb::DeviceGuard g(c->device);
    switch (op) {
        case SW_PROBE_IADD: return run_latency<SW_PROBE_IADD>(c, iters, cycles);
        case SW_PROBE_IMAX: return run_latency<SW_PROBE_IMAX>(c, iters, cycles);
        case SW_PROBE_VIADDMAX_S32: return run_latency<SW_PROBE_VIADDMAX_S32>(c, iters, cycles);
        case SW_PROBE_VIMAX3_S32_RELU: return run_latency<SW_PROBE_VIMAX3_S32_RELU>(c, iters, cycles);
        case SW_PROBE_VIADDMAX_S16X2: return run_latency<SW_PROBE_VIADDMAX_S16X2>(c, iters, cycles);
        case SW_PROBE_VIMAX3_S16X2_RELU: return run_latency<SW_PROBE_VIMAX3_S16X2_RELU>(c, iters, cycles);
        case SW_PROBE_PRMT: return run_latency<SW_PROBE_PRMT>(c, iters, cycles);
        case SW_PROBE_SHFL: return run_latency<SW_PROBE_SHFL>(c, iters, cycles);
        case SW_PROBE_VADDUS4: return run_latency<SW_PROBE_VADDUS4>(c, iters, cycles);
        case SW_PROBE_VSUBUS4: return run_latency<SW_PROBE_VSUBUS4>(c, iters, cycles);
        case SW_PROBE_VMAXU4: return run_latency<SW_PROBE_VMAXU4>(c, iters, cycles);
        default: return SW_EINVAL;
    }
}

extern "C" int sw_probe_int_rate(sw_ctx *c, int op, int iters, double *per_sm_per_clk, double *sm_mhz) {
    if (!c || !per_sm_per_clk || !sm_mhz || iters < 1) return SW_EINVAL;
    swgb::DeviceGuard g(c->device);
    switch (op) {
        case SW_PROBE_IADD: return run<SW_PROBE_IADD>(c, iters, per_sm_per_clk, sm_mhz);
        case SW_PROBE_IMAX: return run<SW_PROBE_IMAX>(c, iters, per_sm_per_clk, sm_mhz);
        case SW_PROBE_VIADDMAX_S32: return run<SW_PROBE_VIADDMAX_S32>(c, iters, per_sm_per_clk, sm_mhz);
        case SW_PROBE_VIMAX3_S32_RELU: return run<SW_PROBE_VIMAX3_S32_RELU>(c, iters, per_sm_per_clk, sm_mhz);
        case SW_PROBE_VIADDMAX_S16X2: return run<SW_PROBE_VIADDMAX_S16X2>(c, iters, per_sm_per_clk, sm_mhz);
        case SW_PROBE_VIMAX3_S16X2_RELU: return run<SW_PROBE_VIMAX3_S16X2_RELU>(c, iters, per_sm_per_clk, sm_mhz);
        case SW_PROBE_PRMT: return run<SW_PROBE_PRMT>(c, iters, per_sm_per_clk, sm_mhz);
        case SW_PROBE_SHFL: return run<SW_PROBE_SHFL>(c, iters, per_sm_per_clk, sm_mhz);
        case SW_PROBE_VADDUS4: return run<SW_PROBE_VADDUS4>(c, iters, per_sm_per_clk, sm_mhz);
        case SW_PROBE_VSUBUS4: return run<SW_PROBE_VSUBUS4>(c, iters, per_sm_per_clk, sm_mhz);
        case SW_PROBE_VMAXU4: return run<SW_PROBE_VMAXU4>(c, iters, per_sm_per_clk, sm_mhz);
        default: return SW_EINVAL;
    }
}
