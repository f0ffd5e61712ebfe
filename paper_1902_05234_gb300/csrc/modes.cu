// modes.cu -- the other block-parallel uses of the T-table cipher:
//
//  CTR (Wang & Chu section 3.1.5, eq (5); Table 1 marks it, with ECB, as
//  suitable for parallel execution): C_i = P_i xor E(counter block of block i),
//  the counter block of block i being the caller's first counter block plus i
//  as a 128-bit big-endian integer (mod 2^128).  Encryption and decryption are
//  the same operation.
//
//  CBC decryption (section 3.1.2; eq (2) as printed omits the cipher, the
//  reading is P_i = D(C_i) xor C_{i-1}, C_{-1} = IV).  Encryption chains and
//  stays sequential (Table 1), but every decryption step needs only two
//  ciphertext blocks, so it parallelises like ECB: lane l of a warp takes the
//  previous ciphertext block from lane l-1 by a shuffle, lane 0 from lane 31
//  of the previous slice or from memory / the IV.
//
// Both reuse the bank-replicated tables and the round code of ECB; round keys
// and the counter / IV travel in the kernel parameters (constant bank).
#include <cstring>

#include "aes_kernels.cuh"
#include "capi_internal.h"
#include "registry.h"

namespace aesgb {

struct CtrArgs {
    const uint4 *in;
    uint4 *out;
    unsigned long long nblocks;
    RoundKeys rk;
    unsigned long long ctr_hi, ctr_lo;  // first counter block as a 128-bit integer
};

struct CbcArgs {
    const uint4 *in;
    uint4 *out;
    unsigned long long nblocks;
    RoundKeys rk;
    uint4 iv;
};

__device__ __forceinline__ uint32_t bswap32(uint32_t v) { return __byte_perm(v, 0u, 0x0123u); }

// Counter block ctr + i as four state words (byte 0 of the block = most
// significant byte of the integer).
__device__ __forceinline__ void counter_state(unsigned long long hi, unsigned long long lo, unsigned long long i,
                                              uint32_t (&s)[4]) {
    const unsigned long long l = lo + i;
    const unsigned long long h = hi + (l < lo ? 1ull : 0ull);
    s[0] = bswap32(static_cast<uint32_t>(h >> 32));
    s[1] = bswap32(static_cast<uint32_t>(h));
    s[2] = bswap32(static_cast<uint32_t>(l >> 32));
    s[3] = bswap32(static_cast<uint32_t>(l));
}

template <int NR, int NB, int LAYOUT>
__global__ void __launch_bounds__(max_threads_for_nb(NB), 1) ctr_kernel(const __grid_constant__ CtrArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t lane = threadIdx.x & 31u;
    const unsigned long long n = a.nblocks;
    const unsigned long long wpc = blockDim.x >> 5;
    const unsigned long long step = static_cast<unsigned long long>(gridDim.x) * wpc * 32ull * NB;
    unsigned long long base = (blockIdx.x * wpc + (threadIdx.x >> 5)) * 32ull * NB;
    Tab<LAYOUT, kEncrypt>::fill(smem, threadIdx.x, blockDim.x);
    __syncthreads();
    griddep_release();
    griddep_wait();  // global memory only after this (see aes_kernels.cuh)
    uint4 cur[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const unsigned long long b = base + lane + 32ull * i;
        cur[i] = b < n ? ld_block(a.in + b) : make_uint4(0, 0, 0, 0);
    }
    const Tab<LAYOUT, kEncrypt> tab(smem, lane);
    const ParamKey key{a.rk.w};
    for (; base < n; base += step) {
        uint4 nxt[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const unsigned long long b = base + step + lane + 32ull * i;
            nxt[i] = b < n ? ld_block(a.in + b) : make_uint4(0, 0, 0, 0);
        }
        uint32_t s[NB][4];
#pragma unroll
        for (int i = 0; i < NB; ++i) counter_state(a.ctr_hi, a.ctr_lo, base + lane + 32ull * i, s[i]);
        cipher_states<kEncrypt, NR, NB>(tab, key, s);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const unsigned long long b = base + lane + 32ull * i;
            if (b < n)
                st_block(a.out + b, make_uint4(cur[i].x ^ s[i][0], cur[i].y ^ s[i][1], cur[i].z ^ s[i][2],
                                               cur[i].w ^ s[i][3]));
            cur[i] = nxt[i];
        }
    }
}

__device__ __forceinline__ uint4 shfl_up1(uint4 v) {
    return make_uint4(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1),
                      __shfl_up_sync(0xffffffffu, v.z, 1), __shfl_up_sync(0xffffffffu, v.w, 1));
}
__device__ __forceinline__ uint4 shfl_from31(uint4 v) {
    return make_uint4(__shfl_sync(0xffffffffu, v.x, 31), __shfl_sync(0xffffffffu, v.y, 31),
                      __shfl_sync(0xffffffffu, v.z, 31), __shfl_sync(0xffffffffu, v.w, 31));
}

// Decryption of the two chained modes whose decryption is parallel (section
// 3.1.2-3.1.3, Table 1 marks their encryption unsuitable): each plaintext
// block needs its ciphertext block C_i and the one before, C_{i-1} (the IV
// before block 0).
//   CBC  P_i = D(C_i) xor C_{i-1}   (inverse cipher on the current block)
//   CFB  P_i = C_i xor E(C_{i-1})   (forward cipher on the previous block)
enum : int { kChainCbc = 0, kChainCfb = 1 };

template <int MODE, int NR, int NB, int LAYOUT>
__global__ void __launch_bounds__(max_threads_for_nb(NB), 1) chain_dec_kernel(const __grid_constant__ CbcArgs a) {
    constexpr int DIR = MODE == kChainCbc ? kDecrypt : kEncrypt;
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t lane = threadIdx.x & 31u;
    const unsigned long long n = a.nblocks;
    const unsigned long long wpc = blockDim.x >> 5;
    const unsigned long long step = static_cast<unsigned long long>(gridDim.x) * wpc * 32ull * NB;
    unsigned long long base = (blockIdx.x * wpc + (threadIdx.x >> 5)) * 32ull * NB;
    Tab<LAYOUT, DIR>::fill(smem, threadIdx.x, blockDim.x);
    __syncthreads();
    griddep_release();
    griddep_wait();  // global memory only after this (see aes_kernels.cuh)
    // the ciphertext block just before a slice (lane 0's chaining value; the
    // IV before block 0), loaded one pass ahead like the slice itself
    auto before = [&](unsigned long long b) {
        return b == 0 ? a.iv
                      : (lane == 0 && b < n && AESGB_CHECK(b - 1 < n) ? ld_block(a.in + (b - 1))
                                                                       : make_uint4(0, 0, 0, 0));
    };
    uint4 cur[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const unsigned long long b = base + lane + 32ull * i;
        cur[i] = b < n ? ld_block(a.in + b) : make_uint4(0, 0, 0, 0);
    }
    uint4 before_cur = before(base);
    const Tab<LAYOUT, DIR> tab(smem, lane);
    const ParamKey key{a.rk.w};
    for (; base < n; base += step) {
        uint4 nxt[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const unsigned long long b = base + step + lane + 32ull * i;
            nxt[i] = b < n ? ld_block(a.in + b) : make_uint4(0, 0, 0, 0);
        }
        const uint4 before_nxt = before(base + step);
        // chaining values: the ciphertext block just before each of ours
        uint4 prev[NB];
        const uint4 before_slice0 = before_cur;
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const uint4 up = shfl_up1(cur[i]);
            const uint4 from_prev_slice = i == 0 ? before_slice0 : shfl_from31(cur[i > 0 ? i - 1 : 0]);
            prev[i] = lane == 0 ? from_prev_slice : up;
        }
        uint32_t s[NB][4];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const uint4 x = MODE == kChainCbc ? cur[i] : prev[i];  // the block the cipher runs on
            s[i][0] = x.x; s[i][1] = x.y; s[i][2] = x.z; s[i][3] = x.w;
        }
        cipher_states<DIR, NR, NB>(tab, key, s);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const unsigned long long b = base + lane + 32ull * i;
            const uint4 y = MODE == kChainCbc ? prev[i] : cur[i];  // the block XORed onto its output
            if (b < n) st_block(a.out + b, make_uint4(y.x ^ s[i][0], y.y ^ s[i][1], y.z ^ s[i][2], y.w ^ s[i][3]));
            cur[i] = nxt[i];
        }
        before_cur = before_nxt;
    }
}

AESGB_BOUNDS_READER(modes)

#define AESGB_M(KERNEL, NR, NB)                                                \
    if (nr == NR && nb == NB) return reinterpret_cast<const void *>(&KERNEL<NR, NB, kLayoutR4>);
#define AESGB_C(MODE, NR, NB)                                                  \
    if (nr == NR && nb == NB) return reinterpret_cast<const void *>(&chain_dec_kernel<MODE, NR, NB, kLayoutR4>);

// One block per thread: ECB measures the same at 16 and 32 bytes per thread,
// and the counter / chaining state would not fit 64 registers at two.
const void *ctr_kernel_ptr(int nr, int nb) {
    AESGB_M(ctr_kernel, 10, 1) AESGB_M(ctr_kernel, 12, 1) AESGB_M(ctr_kernel, 14, 1)
    return nullptr;
}

const void *cbc_dec_kernel_ptr(int nr, int nb) {
    AESGB_C(kChainCbc, 10, 1) AESGB_C(kChainCbc, 12, 1) AESGB_C(kChainCbc, 14, 1)
    return nullptr;
}

const void *cfb_dec_kernel_ptr(int nr, int nb) {
    AESGB_C(kChainCfb, 10, 1) AESGB_C(kChainCfb, 12, 1) AESGB_C(kChainCfb, 14, 1)
    return nullptr;
}

namespace {

aes_launch_cfg mode_cfg(int dir, int nr, size_t nblocks) {
    aes_launch_cfg c = default_cfg(dir, nr, nblocks);
    c.layout = AES_LAYOUT_R4;
    c.blocks_per_thread = 1;
    return c;
}

template <class Args>
int launch_mode(const void *fn, int dir, const aes_launch_cfg &c, size_t nblocks, Args &args, void *stream) {
    if (!fn) return AES_E_CONFIG;
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    const uint32_t smem = table_smem_bytes(dir, AES_LAYOUT_R4);
    int st = ensure_smem_attr(fn, dev, smem);
    if (st != AES_OK) return st;
    int grid = 0;
    st = persistent_grid(fn, dev, c, smem, static_cast<unsigned long long>(c.threads) * c.blocks_per_thread,
                         nblocks, &grid, nullptr);
    if (st != AES_OK) return st;
    void *params[] = {&args};
    return launch_pdl(fn, grid, c.threads, smem, params, stream);
}

}  // namespace
}  // namespace aesgb

using namespace aesgb;

extern "C" {

int aes_ctr_crypt(const uint32_t *rk, int nrounds, const uint8_t *ctr0, const uint8_t *in, uint8_t *out,
                  size_t nblocks, void *stream) {
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    if (!rk || !ctr0) return AES_E_ARG;
    if (nblocks == 0) return AES_OK;
    st = check_buffers(in, out, nblocks);
    if (st != AES_OK) return st;
    const aes_launch_cfg c = mode_cfg(kEncrypt, nrounds, nblocks);
    CtrArgs args;
    args.in = reinterpret_cast<const uint4 *>(in);
    args.out = reinterpret_cast<uint4 *>(out);
    args.nblocks = nblocks;
    order_round_keys(kEncrypt, rk, nrounds, &args.rk);
    unsigned long long hi = 0, lo = 0;
    for (int b = 0; b < 8; ++b) hi = (hi << 8) | ctr0[b];
    for (int b = 8; b < 16; ++b) lo = (lo << 8) | ctr0[b];
    args.ctr_hi = hi;
    args.ctr_lo = lo;
    return launch_mode(ctr_kernel_ptr(nrounds, c.blocks_per_thread), kEncrypt, c, nblocks, args, stream);
}

int aes_cbc_decrypt(const uint32_t *rk_dec, int nrounds, const uint8_t *iv, const uint8_t *in, uint8_t *out,
                    size_t nblocks, void *stream) {
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    if (!rk_dec || !iv) return AES_E_ARG;
    if (nblocks == 0) return AES_OK;
    st = check_buffers(in, out, nblocks);
    if (st != AES_OK) return st;
    if (in == out) return AES_E_OVERLAP;  // a block's ciphertext is still needed after its plaintext is written
    const aes_launch_cfg c = mode_cfg(kDecrypt, nrounds, nblocks);
    CbcArgs args;
    args.in = reinterpret_cast<const uint4 *>(in);
    args.out = reinterpret_cast<uint4 *>(out);
    args.nblocks = nblocks;
    order_round_keys(kDecrypt, rk_dec, nrounds, &args.rk);
    std::memcpy(&args.iv, iv, 16);
    return launch_mode(cbc_dec_kernel_ptr(nrounds, c.blocks_per_thread), kDecrypt, c, nblocks, args, stream);
}

int aes_cfb_decrypt(const uint32_t *rk_enc, int nrounds, const uint8_t *iv, const uint8_t *in, uint8_t *out,
                    size_t nblocks, void *stream) {
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    if (!rk_enc || !iv) return AES_E_ARG;
    if (nblocks == 0) return AES_OK;
    st = check_buffers(in, out, nblocks);
    if (st != AES_OK) return st;
    if (in == out) return AES_E_OVERLAP;  // as CBC: C_i is read again after P_i would overwrite it
    const aes_launch_cfg c = mode_cfg(kEncrypt, nrounds, nblocks);
    CbcArgs args;
    args.in = reinterpret_cast<const uint4 *>(in);
    args.out = reinterpret_cast<uint4 *>(out);
    args.nblocks = nblocks;
    order_round_keys(kEncrypt, rk_enc, nrounds, &args.rk);
    std::memcpy(&args.iv, iv, 16);
    return launch_mode(cfb_dec_kernel_ptr(nrounds, c.blocks_per_thread), kEncrypt, c, nblocks, args, stream);
}

}  // extern "C"
