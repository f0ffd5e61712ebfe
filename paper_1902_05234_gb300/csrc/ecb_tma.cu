// ecb_tma.cu -- ECB kernel with TMA-staged input (layout AES_LAYOUT_R4_TMA).
//
// Same rounds and R4 tables as ecb_kernel (aes_kernels.cuh); only the way the
// plaintext reaches the threads differs.  Each warp owns two shared-memory
// tiles of 32 x NB blocks (the warp's share of one pass, 512 NB contiguous
// bytes).  Lane 0 fills them with 1-D bulk copies (cp.async.bulk, the TMA
// engine) two passes ahead, each tracked by an mbarrier with a transaction
// count; the lanes wait on the barrier, read their blocks from the tile with
// 128-bit shared loads, cipher them and store with 128-bit global stores.
//
// Every wait is bounded (about one second of global time): a wait that runs
// out counts itself in a device counter read by aes_wait_timeouts, waits (again
// bounded) for its warp's copies still in flight, and the warp stops.
#include <cuda_runtime.h>

#include <cstdint>

#include "aes_kernels.cuh"
#include "capi_internal.h"
#include "registry.h"

namespace aesgb {

__device__ unsigned long long g_wait_timeouts = 0;

constexpr unsigned long long kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Bounded wait for the phase of the given parity; false if it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitLimitNs) return false;
    return true;
}
// Global -> shared bulk copy of `bytes` (a multiple of 16, both addresses
// 16-byte aligned), completing as transactions on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// extra_tx is 0 except in the failure-detection self-test
// (aes_tma_selftest_timeout), where every barrier expects that many bytes more
// than its copy delivers, so that no wait can finish and each must run out.
template <int DIR, int NR, int NB>
__global__ void __launch_bounds__(max_threads_for_nb(NB), 1)
    ecb_tma_kernel(const __grid_constant__ EcbArgs a, const uint32_t extra_tx) {
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr uint32_t kTile = 512u * NB;  // one warp's blocks of one pass
    constexpr unsigned long long kTileBlocks = 32ull * NB;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint8_t *stage = smem + table_smem_bytes(DIR, kLayoutR4) + warp * 2u * kTile;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + table_smem_bytes(DIR, kLayoutR4) + nwarps * 2u * kTile) +
                    2u * warp;
    const unsigned long long n = a.nblocks;
    const unsigned long long step = static_cast<unsigned long long>(gridDim.x) * nwarps * kTileBlocks;
    unsigned long long base = (blockIdx.x * static_cast<unsigned long long>(nwarps) + warp) * kTileBlocks;

    // lane 0: the tile of pass `b` into buffer `buf`, if there is one
    auto issue = [&](unsigned long long b, int buf) {
        if (b >= n) return;
        const unsigned long long cnt = n - b < kTileBlocks ? n - b : kTileBlocks;
        const uint32_t bytes = static_cast<uint32_t>(cnt * 16ull);
        // the copy stays inside the input and inside this warp's tile
        if (!AESGB_CHECK(b + cnt <= n && cnt >= 1 && cnt <= kTileBlocks &&
                         static_cast<uint32_t>(stage - smem) + (buf + 1) * kTile <= dyn_smem_bytes()))
            return;
        mbar_arrive_expect_tx(&bar[buf], bytes + extra_tx);
        bulk_load(stage + buf * kTile, a.in + b, bytes, &bar[buf]);
    };
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    Tab<kLayoutR4, DIR>::fill(smem, threadIdx.x, blockDim.x);
    __syncthreads();
    griddep_release();
    griddep_wait();  // global memory (the bulk copies included) only after this
    if (lane == 0) {
        issue(base, 0);
        issue(base + step, 1);
    }
    __syncwarp();

    const Tab<kLayoutR4, DIR> tab(smem, lane);
    const ParamKey key{a.rk.w};
    bool failed = false;
    unsigned int it = 0;
    for (; base < n; base += step, ++it) {
        const int buf = static_cast<int>(it & 1u);
        // every lane waits (each acquires the copy's writes); the outcome is
        // made warp-uniform so that the lanes never part at a timeout
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar[buf], (it >> 1) & 1u))) {
            failed = true;
            break;
        }
        uint32_t s[NB][4];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const uint32_t at = buf * kTile + (lane + 32u * i) * 16u;
            (void)AESGB_CHECK(at + 16u <= kTile * 2u);
            const uint4 v = *reinterpret_cast<const uint4 *>(stage + at);
            s[i][0] = v.x; s[i][1] = v.y; s[i][2] = v.z; s[i][3] = v.w;
        }
        __syncwarp();  // every lane has read the tile before it is refilled
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(base + 2 * step, buf);
        }
        cipher_states<DIR, NR, NB>(tab, key, s);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const unsigned long long b = base + lane + 32ull * i;
            if (b < n) st_block(a.out + b, make_uint4(s[i][0], s[i][1], s[i][2], s[i][3]));
        }
    }
    if (failed) {
        // count the timeout once per warp, then wait (bounded) for the copies
        // this warp still has in flight: the current pass's and the next one's
        if (lane == 0) atomicAdd(&g_wait_timeouts, 1ull);
        for (unsigned int k = 0; k < 2; ++k)
            if (base + k * step < n) (void)mbar_wait_bounded(&bar[(it + k) & 1u], ((it + k) >> 1) & 1u);
    }
}

AESGB_BOUNDS_READER(ecb_tma)

#define AESGB_TMA(D, NR, NB)                                                     \
    if (dir == D && nr == NR && nb == NB)                                        \
        return reinterpret_cast<const void *>(&ecb_tma_kernel<D, NR, NB>);
#define AESGB_TMA_NR(D, NR) AESGB_TMA(D, NR, 1) AESGB_TMA(D, NR, 2) AESGB_TMA(D, NR, 4)

const void *ecb_kernel_tma(int dir, int nr, int nb) {
    AESGB_TMA_NR(kEncrypt, 10)
    AESGB_TMA_NR(kEncrypt, 12)
    AESGB_TMA_NR(kEncrypt, 14)
    AESGB_TMA_NR(kDecrypt, 10)
    AESGB_TMA_NR(kDecrypt, 12)
    AESGB_TMA_NR(kDecrypt, 14)
    return nullptr;
}

uint32_t ecb_tma_smem_bytes(int dir, int threads, int nb) {
    const uint32_t warps = static_cast<uint32_t>(threads / 32);
    return table_smem_bytes(dir, kLayoutR4) + warps * 2u * 512u * static_cast<uint32_t>(nb) + warps * 16u;
}

int launch_tma_selftest_timeout(const uint8_t *in, uint8_t *out, size_t nblocks, void *stream) {
    const void *fn = reinterpret_cast<const void *>(&ecb_tma_kernel<kEncrypt, 10, 1>);
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    const uint32_t smem = ecb_tma_smem_bytes(kEncrypt, 32, 1);
    int st = ensure_smem_attr(fn, dev, smem);
    if (st != AES_OK) return st;
    EcbArgs args{};
    args.in = reinterpret_cast<const uint4 *>(in);
    args.out = reinterpret_cast<uint4 *>(out);
    args.nblocks = nblocks;
    uint32_t extra = 16;
    void *params[] = {&args, &extra};
    if (cudaLaunchKernel(fn, dim3(1), dim3(32), params, smem, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    return AES_OK;
}

int read_wait_timeouts(unsigned long long *count) {
    unsigned long long v = 0;
    const unsigned long long zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_wait_timeouts, sizeof v) != cudaSuccess ||
        cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof zero) != cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    *count = v;
    return AES_OK;
}

}  // namespace aesgb
