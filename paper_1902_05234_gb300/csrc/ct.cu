// ct.cu -- constant-time ECB: the bitsliced cipher of bitslice.cuh on GB300.
//
// Each thread owns 32 blocks: lane l of a warp takes blocks base + 32 j + l,
// j = 0..31, so every warp-wide 128-bit load or store still covers 512
// contiguous bytes.  The thread transposes its 32 x 128 bits into 128 bit
// planes, runs the rounds as logic operations on whole planes, transposes
// back and stores.  No address depends on key or data.  Round keys reach the
// S-box circuit as mask planes built on the host from the schedule (one
// input and one output mask byte per byte position and round, see
// build_masks) and expanded into shared memory at the start of the kernel.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "aes_kernels.cuh"
#include "bitslice.cuh"
#include "capi_internal.h"

namespace aesgb {

constexpr int kCtThreads = 256;  // 128 plane registers + the S-box circuit's temporaries per thread

struct CtArgs {
    const uint4 *in;
    uint4 *out;
    unsigned long long nblocks;
    int nr;
    uint8_t masks[14][16][2];  // [application][byte q = r + 4c][0 in, 1 out]
};

// Mask bytes of every S-box application, in application order.
//  encryption, application i (round i+1): input  phi^-1(K_i[q])
//                                         output 63, and K_Nr at the byte's
//                                         place after ShiftRows in the last
//  decryption (inverse cipher, FIPS-197 5.3), application i (round Nr-1-i,
//  applied after InvShiftRows): input  D_in (63 + K_Nr at the byte's place
//                               before InvShiftRows) in the first,
//                               D_in 63 after that
//                               output K_{Nr-1-i}[q]
// K_r[q] is byte q of round key r of the encryption schedule w.
void build_masks(int dir, const uint8_t *w, int nr, uint8_t (*m)[16][2]) {
    using bsmath::apply;
    using bsmath::kMaps;
    for (int i = 0; i < nr; ++i)
        for (int q = 0; q < 16; ++q) {
            const int r = q & 3, c = q >> 2;
            if (dir == 0) {
                m[i][q][0] = apply(kMaps.enc_in, w[16 * i + q]);
                const int dest = r + 4 * ((c - r + 4) & 3);
                m[i][q][1] = static_cast<uint8_t>(0x63 ^ (i == nr - 1 ? w[16 * nr + dest] : 0));
            } else {
                const int src = r + 4 * ((c - r + 4) & 3);
                m[i][q][0] = i == 0 ? apply(kMaps.dec_in, static_cast<uint8_t>(0x63 ^ w[16 * nr + src]))
                                    : kMaps.dec_in_c;
                m[i][q][1] = w[16 * (nr - 1 - i) + q];
            }
        }
}

// The encryption schedule w as bytes from either schedule of aes_expand_key:
// rk_enc is w; rk_dec is dw, whose round keys 1..Nr-1 are InvMixColumns(w_r),
// so MixColumns gives them back.
void schedule_bytes(int dir, const uint32_t *rk, int nr, uint8_t *w) {
    std::memcpy(w, rk, 16 * (nr + 1));
    if (dir == 0) return;
    for (int r = 1; r < nr; ++r)
        for (int c = 0; c < 4; ++c) {
            uint32_t col;
            std::memcpy(&col, w + 16 * r + 4 * c, 4);
            col = bsmath::mix_column_model(col);
            std::memcpy(w + 16 * r + 4 * c, &col, 4);
        }
}

template <int DIR>
__global__ void __launch_bounds__(kCtThreads, 1) ct_kernel(const __grid_constant__ CtArgs a) {
    __shared__ bs::RoundMasks masks[14];
    for (int i = threadIdx.x; i < a.nr * 16 * 2 * 8; i += blockDim.x) {
        const int b = i & 7, io = (i >> 3) & 1, q = (i >> 4) & 15, app = i >> 8;
        masks[app].m[q][io][b] = ((a.masks[app][q][io] >> b) & 1) ? 0xffffffffu : 0u;
    }
    __syncthreads();
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
    uint8_t w[240];
    schedule_bytes(dir, rk, nrounds, w);
    build_masks(dir, w, nrounds, args.masks);
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    const void *fn = dir == 0 ? reinterpret_cast<const void *>(&ct_kernel<0>)
                              : reinterpret_cast<const void *>(&ct_kernel<1>);
    aes_launch_cfg c{kCtThreads, 1, 0, 0};
    int grid = 0;
    st = persistent_grid(fn, dev, c, 0, static_cast<unsigned long long>(kCtThreads) * 32ull, nblocks, &grid);
    if (st != AES_OK) return st;
    void *params[] = {&args};
    if (cudaLaunchKernel(fn, dim3(grid), dim3(kCtThreads), params, 0, static_cast<cudaStream_t>(stream)) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    return AES_OK;
}

int aes_ct_selftest_host(int dir, const uint32_t *rk, int nrounds, const uint8_t *in, uint8_t *out,
                         size_t nblocks) {
    if ((dir != 0 && dir != 1) || !rk || (nblocks && (!in || !out))) return AES_E_ARG;
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    uint8_t w[240];
    uint8_t mb[14][16][2];
    schedule_bytes(dir, rk, nrounds, w);
    build_masks(dir, w, nrounds, mb);
    bs::RoundMasks masks[14];
    for (int i = 0; i < nrounds; ++i)
        for (int q = 0; q < 16; ++q)
            for (int io = 0; io < 2; ++io)
                for (int b = 0; b < 8; ++b) masks[i].m[q][io][b] = ((mb[i][q][io] >> b) & 1) ? 0xffffffffu : 0u;
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
