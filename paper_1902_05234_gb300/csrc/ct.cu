// ct.cu -- constant-time ECB: the bitsliced cipher of bitslice.cuh on GB300.
//
// Each thread owns 32 blocks: lane l of a warp takes blocks base + 32 j + l,
// j = 0..31, so every warp-wide 128-bit load or store still covers 512
// contiguous bytes.  The thread transposes its 32 x 128 bits into 128 bit
// planes, runs the rounds as logic operations on whole planes, transposes
// back and stores.  No address depends on key or data.  Round keys reach the
// circuits as mask planes built on the host from the schedule (one mask byte
// per byte position and key step, see build_masks) and expanded into shared
// memory at the start of the kernel.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "aes_kernels.cuh"
#include "bitslice.cuh"
#include "capi_internal.h"
#include "registry.h"

namespace aesgb {

constexpr int kCtThreads = 256;  // 128 plane registers + the circuits' temporaries per thread

struct CtArgs {
    const uint4 *in;
    uint4 *out;
    unsigned long long nblocks;
    int nr;
    uint8_t masks[15][16];  // [key step][byte q = r + 4c]
};

// Key bytes of steps 0..Nr as the kernel takes them (bitslice.cuh adds step 0
// to the input and gives step i to the circuits of round i).  K_i is round
// key i of the encryption schedule w, as a state (byte q = r + 4c is row r,
// column c); a byte m wanted at an S-box output is passed as mu = OUT^-1 m
// (bsc::k_mu_enc / k_mu_dec), which the S-box's product chains add for free.
//   encryption  step 0: K_0.  Round i adds its key at the S-box outputs,
//               before ShiftRows and MixColumns, together with the S-box's
//               constant 63: m[q] = 63 + K'_i[r + 4((c - r) mod 4)], where
//               K'_i = InvMixColumns(K_i) for i < Nr and K_Nr itself (the
//               last round has no MixColumns); ShiftRows then carries byte
//               (r, (c - r) mod 4) to (r, c), and MixColumns(K'_i) = K_i.
//   decryption  (inverse cipher, FIPS-197 5.3): step 0 is K_Nr; round i adds
//               K_{Nr-i} right after InvSubBytes, m = K_{Nr-i}, and the column
//               circuit applies InvMixColumns to the sum.
void build_masks(int dir, const uint32_t *rk, int nr, uint8_t (*out)[16]) {
    uint8_t w[240];
    std::memcpy(w, rk, 16 * (nr + 1));
    if (dir == 1)  // rk is dw: its keys 1..Nr-1 are InvMixColumns(w_r); MixColumns gives w back
        for (int r = 1; r < nr; ++r)
            for (int c = 0; c < 4; ++c) {
                uint32_t col;
                std::memcpy(&col, w + 16 * r + 4 * c, 4);
                col = bsmath::mix_column_model(col);
                std::memcpy(w + 16 * r + 4 * c, &col, 4);
            }
    std::memcpy(out[0], w + (dir == 0 ? 0 : 16 * nr), 16);
    for (int i = 1; i <= nr; ++i) {
        uint8_t m[16];
        if (dir == 0) {
            uint8_t k[16];
            for (int c = 0; c < 4; ++c) {
                uint32_t col;
                std::memcpy(&col, w + 16 * i + 4 * c, 4);
                if (i < nr) col = bsmath::inv_mix_column_model(col);
                std::memcpy(k + 4 * c, &col, 4);
            }
            for (int q = 0; q < 16; ++q) {
                const int r = q & 3, c = q >> 2;
                m[q] = static_cast<uint8_t>(0x63 ^ k[r + 4 * ((c - r + 4) & 3)]);
            }
        } else {
            std::memcpy(m, w + 16 * (nr - i), 16);
        }
        for (int q = 0; q < 16; ++q) out[i][q] = bs::apply_rows(dir == 0 ? bsc::k_mu_enc : bsc::k_mu_dec, m[q]);
    }
}

// Mask byte -> 8 planes, in the state's layout (plane 8r + b of column c).
AESGB_HD void expand_mask(const uint8_t (*m)[16], int i, bs::RoundMasks *dst) {
    const int app = i >> 7, p = i & 127, c = p >> 5, rb = p & 31;
#if defined(__CUDA_ARCH__)
    if (!AESGB_CHECK(app < 15)) return;
#endif
    dst[app].m[c][rb] = ((m[app][(rb >> 3) + 4 * c] >> (rb & 7)) & 1) ? 0xffffffffu : 0u;
}

template <int DIR>
__global__ void __launch_bounds__(kCtThreads, 1) ct_kernel(const __grid_constant__ CtArgs a) {
    __shared__ bs::RoundMasks masks[15];
    for (int i = threadIdx.x; i < (a.nr + 1) * 128; i += blockDim.x) expand_mask(a.masks, i, masks);
    __syncthreads();
    griddep_release();
    griddep_wait();  // global memory only after this (see aes_kernels.cuh)
    const uint32_t lane = threadIdx.x & 31u;
    const unsigned long long wpc = blockDim.x >> 5;
    const unsigned long long step = static_cast<unsigned long long>(gridDim.x) * wpc * 1024ull;
    const unsigned long long n = a.nblocks;
    for (unsigned long long base = (blockIdx.x * wpc + (threadIdx.x >> 5)) * 1024ull; base < n; base += step) {
        bs::Planes s;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const unsigned long long blk = base + 32ull * j + lane;
            const uint4 v = blk < n ? ld_block(a.in + blk) : make_uint4(0, 0, 0, 0);
            s.w[0][j] = v.x;
            s.w[1][j] = v.y;
            s.w[2][j] = v.z;
            s.w[3][j] = v.w;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) bs::transpose32(s.w[c]);
        bs::cipher_planes<DIR>(s, masks, a.nr);
#pragma unroll
        for (int c = 0; c < 4; ++c) bs::transpose32(s.w[c]);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const unsigned long long blk = base + 32ull * j + lane;
            if (blk < n) st_block(a.out + blk, make_uint4(s.w[0][j], s.w[1][j], s.w[2][j], s.w[3][j]));
        }
    }
}

AESGB_BOUNDS_READER(ct)

}  // namespace aesgb

using namespace aesgb;

extern "C" {

int aes_ecb_crypt_ct(int dir, const uint32_t *rk, int nrounds, const uint8_t *in, uint8_t *out, size_t nblocks,
                     void *stream) {
    if (dir != 0 && dir != 1) return AES_E_ARG;
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    if (!rk) return AES_E_ARG;
    if (nblocks == 0) return AES_OK;
    st = check_buffers(in, out, nblocks);
    if (st != AES_OK) return st;
    CtArgs args;
    std::memset(&args, 0, sizeof args);
    args.in = reinterpret_cast<const uint4 *>(in);
    args.out = reinterpret_cast<uint4 *>(out);
    args.nblocks = nblocks;
    args.nr = nrounds;
    build_masks(dir, rk, nrounds, args.masks);
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    const void *fn = dir == 0 ? reinterpret_cast<const void *>(&ct_kernel<0>)
                              : reinterpret_cast<const void *>(&ct_kernel<1>);
    aes_launch_cfg c{kCtThreads, 1, 0, 0};
    int grid = 0;
    st = persistent_grid(fn, dev, c, 0, static_cast<unsigned long long>(kCtThreads) * 32ull, nblocks, &grid,
                         nullptr);
    if (st != AES_OK) return st;
    void *params[] = {&args};
    return launch_pdl(fn, grid, kCtThreads, 0, params, stream);
}

int aes_ct_ops_per_block(int dir, int nrounds, double *ops_per_block) {
    if ((dir != 0 && dir != 1) || !ops_per_block) return AES_E_ARG;
    const int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    // per thread and 32-block group: 128 planes of step-0 key, the rounds,
    // 8 transposes of 32 words (stages 16 and 8: one byte permute per word,
    // stages 4, 2 and 1: one bit-select per word)
    long long g = 128 + 8 * (2 * 32 + 3 * 32);
    if (dir == 0)
        g += 16LL * nrounds * bsc::k_sbox_enc.kGates + 4LL * (nrounds - 1) * bsc::k_mix_columns.kGates;
    else
        g += 16LL * nrounds * bsc::k_sbox_core_dec.kGates + 4LL * (nrounds - 1) * bsc::k_inv_mix_out.kGates +
             16LL * bsc::k_sbox_out_dec.kGates;
    *ops_per_block = static_cast<double>(g) / 32.0;
    return AES_OK;
}

int aes_ct_selftest_host(int dir, const uint32_t *rk, int nrounds, const uint8_t *in, uint8_t *out,
                         size_t nblocks) {
    if ((dir != 0 && dir != 1) || !rk || (nblocks && (!in || !out))) return AES_E_ARG;
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    uint8_t mb[15][16];
    build_masks(dir, rk, nrounds, mb);
    static bs::RoundMasks masks[15];  // 7.5 KB: kept off the host stack
    for (int i = 0; i < (nrounds + 1) * 128; ++i) expand_mask(mb, i, masks);
    for (size_t g = 0; g < nblocks; g += 32) {
        bs::Planes s;
        for (int j = 0; j < 32; ++j) {
            uint32_t v[4] = {0, 0, 0, 0};
            if (g + j < nblocks) std::memcpy(v, in + 16 * (g + j), 16);
            for (int c = 0; c < 4; ++c) s.w[c][j] = v[c];
        }
        for (int c = 0; c < 4; ++c) bs::transpose32(s.w[c]);
        if (dir == 0) bs::cipher_planes<0>(s, masks, nrounds);
        else bs::cipher_planes<1>(s, masks, nrounds);
        for (int c = 0; c < 4; ++c) bs::transpose32(s.w[c]);
        for (int j = 0; j < 32; ++j) {
            if (g + j >= nblocks) break;
            uint32_t v[4] = {s.w[0][j], s.w[1][j], s.w[2][j], s.w[3][j]};
            std::memcpy(out + 16 * (g + j), v, 16);
        }
    }
    return AES_OK;
}

}  // extern "C"
