// calibrate.cu -- measured peak of the bound the T-table kernels run into:
// independent, bank-conflict-free 4-byte shared-memory lookups.
//
// Each warp reads a 256-entry table replicated per bank (entry x for lane l
// at word 32x + l, the layout the AES kernels use) at indices drawn from a
// linear congruential stream that does not depend on the loaded values, and
// XORs the results -- the lookup pattern of a T-table round without the rest
// of the cipher.  The rate it sustains (lookups per clock per SM) is the
// roofline peak the AES kernels can at best reach; the unit-count figure is
// 32 (one 128-byte wavefront per clock per SM).
//
// logic_rate_kernel measures the other pipe: three-input logic instructions
// (LOP3), the only kind of instruction in the bitsliced kernel's circuits.
// Every thread runs eight independent chains, so the rate is the pipe's and
// not a chain's latency; the unit-count figure is 64 lanes per clock per SM.
#include <cuda_runtime.h>

#include <cstdint>

#include "capi_internal.h"

namespace aesgb {

constexpr int kCalLookups = 16;  // per thread per iteration, like one AES round

__global__ void __launch_bounds__(1024, 1) lookup_rate_kernel(uint32_t *sink, int iters) {
    __shared__ uint32_t tab[256 * 32];
    for (int i = threadIdx.x; i < 256 * 32; i += blockDim.x) tab[i] = static_cast<uint32_t>(i) * 0x9e3779b9u;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t a = threadIdx.x * 2654435761u + blockIdx.x, acc = 0;
    for (int it = 0; it < iters; ++it) {
        a = a * 1664525u + 1013904223u;
#pragma unroll
        for (int j = 0; j < kCalLookups; ++j) {
            const uint32_t x = ((a >> ((j & 3) * 8)) ^ static_cast<uint32_t>(j) * 37u) & 255u;
            acc ^= tab[x * 32u + lane];
        }
    }
    if (acc == 0x2545f491u) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;  // keeps the loads alive
}

constexpr int kCalChains = 8;     // independent LOP3 chains per thread
constexpr int kCalUnroll = 32;    // chain steps per loop trip (8 x 32 LOP3 per trip)

template <uint8_t LUT>
__device__ __forceinline__ uint32_t lop3_cal(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}

__global__ void __launch_bounds__(1024, 1) logic_rate_kernel(uint32_t *sink, int iters) {
    uint32_t x[kCalChains];
#pragma unroll
    for (int c = 0; c < kCalChains; ++c) x[c] = (threadIdx.x + 1u) * (2654435761u + 2u * c) ^ blockIdx.x;
    const uint32_t k0 = x[0] * 3u + 1u, k1 = x[1] * 5u + 7u;  // loop-invariant operands
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kCalUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kCalChains; ++c) x[c] = lop3_cal<0x96>(x[c], k0 + c, (u & 1) ? k1 : k0);
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kCalChains; ++c) acc ^= x[c];
    if (acc == 0x2545f491u) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;  // keeps the chains alive
}

}  // namespace aesgb

using namespace aesgb;

extern "C" int aes_calibrate_lookup_rate(void *sink_dev, size_t sink_bytes, void *stream, double *lookups,
                                         double *seconds) {
    if (!sink_dev || !lookups || !seconds) return AES_E_ARG;
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    const int sms = sm_count(dev);
    if (sms < 0) return sms;
    if (sink_bytes < static_cast<size_t>(sms) * 1024 * 4) return AES_E_RANGE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int iters = 4096;
    uint32_t *sink = static_cast<uint32_t *>(sink_dev);
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return AES_E_CUDA;
    lookup_rate_kernel<<<sms, 1024, 0, s>>>(sink, 64);  // warm-up
    cudaEventRecord(a, s);
    lookup_rate_kernel<<<sms, 1024, 0, s>>>(sink, iters);
    cudaEventRecord(b, s);
    float ms = 0.f;
    const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!ok) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    *lookups = static_cast<double>(sms) * 1024.0 * iters * kCalLookups;
    *seconds = ms * 1e-3;
    return AES_OK;
}

extern "C" int aes_calibrate_logic_rate(void *sink_dev, size_t sink_bytes, void *stream, double *ops,
                                        double *seconds) {
    if (!sink_dev || !ops || !seconds) return AES_E_ARG;
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    const int sms = sm_count(dev);
    if (sms < 0) return sms;
    if (sink_bytes < static_cast<size_t>(sms) * 1024 * 4) return AES_E_RANGE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int iters = 2048;
    uint32_t *sink = static_cast<uint32_t *>(sink_dev);
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return AES_E_CUDA;
    logic_rate_kernel<<<sms, 1024, 0, s>>>(sink, 32);  // warm-up
    cudaEventRecord(a, s);
    logic_rate_kernel<<<sms, 1024, 0, s>>>(sink, iters);
    cudaEventRecord(b, s);
    float ms = 0.f;
    const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!ok) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    *ops = static_cast<double>(sms) * 1024.0 * iters * kCalUnroll * kCalChains;
    *seconds = ms * 1e-3;
    return AES_OK;
}
