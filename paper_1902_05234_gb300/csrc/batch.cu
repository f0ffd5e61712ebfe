// batch.cu -- many independent ECB messages, each with its own key, key size
// and direction, in ONE persistent launch driven by a device descriptor table.
//
// The paper's unit of parallelism is one AES state (section 4.1, eq (1)); a
// batch only changes which key and which buffer a state belongs to, never the
// arithmetic.  Two kernels run back to back on the caller's stream:
//
//  plan   (one CTA)  validates every descriptor (bad ones get a status and no
//                    work), orders the messages encryptions first, and writes
//                    the exclusive prefix `start[]` of their chunk counts,
//                    where a chunk is `chunk_blocks` consecutive blocks of one
//                    message -- the work of one warp.
//  batch  (persistent, one CTA per SM)  warps take chunks of the encryption
//                    range, then of the decryption range, from two atomic
//                    counters (dynamic: whichever warp is free takes the next
//                    chunk).  A chunk's message is found by a warp-wide 32-ary
//                    search in start[]; its round keys are staged through the
//                    warp's own shared-memory slot into registers.  The CTA's T tables are filled for
//                    encryption first and refilled once for decryption,
//                    between two CTA barriers that every warp reaches; each
//                    phase's table layout is part of the launch configuration
//                    (default R4 for encryption, 128 KiB, and R2 for
//                    decryption, also 128 KiB: faster to fill than R4's
//                    160 KiB and as fast to use).
//
// Workspace layout (caller- or library-owned device memory, see
// aes_batch_workspace_bytes):
//   BatchHeader | uint32 order[n] | uint64 start[n+1] | uint64 count[n]
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <utility>

#include "aesgb.h"
#include "aes_kernels.cuh"
#include "batch_internal.h"
#include "capi_internal.h"
#include "registry.h"

namespace aesgb {

static_assert(sizeof(aes_desc) == 40, "aes_desc is 40 bytes");
static_assert(offsetof(aes_desc, nblocks) == 24 && offsetof(aes_desc, nrounds) == 32 &&
                  offsetof(aes_desc, dir) == 36,
              "aes_desc field offsets");

struct BatchHeader {
    unsigned long long total_chunks;  // T
    unsigned long long enc_chunks;    // E: chunks [0, E) encrypt, [E, T) decrypt
    unsigned long long next[2];       // work counters of the two phases (zeroed by the plan)
    unsigned int n;
    unsigned int chunk_blocks;
    unsigned int n_invalid;
    unsigned int pad;
};

__host__ __device__ constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t batch_ws_bytes(int n) {
    const size_t nn = n > 0 ? static_cast<size_t>(n) : 0;
    return align_up(sizeof(BatchHeader), 256) + align_up(4 * nn, 256) + align_up(8 * (nn + 1), 256) +
           align_up(8 * nn, 256);
}

struct WsView {
    BatchHeader *hdr;
    uint32_t *order;
    unsigned long long *start;
    unsigned long long *count;
};

__host__ __device__ inline WsView ws_view(void *ws, int n) {
    const size_t nn = static_cast<size_t>(n);
    uint8_t *p = static_cast<uint8_t *>(ws);
    WsView v;
    v.hdr = reinterpret_cast<BatchHeader *>(p);
    p += align_up(sizeof(BatchHeader), 256);
    v.order = reinterpret_cast<uint32_t *>(p);
    p += align_up(4 * nn, 256);
    v.start = reinterpret_cast<unsigned long long *>(p);
    p += align_up(8 * (nn + 1), 256);
    v.count = reinterpret_cast<unsigned long long *>(p);
    return v;
}

// ---------------------------------------------------------------------------
// plan kernel
// ---------------------------------------------------------------------------
constexpr int kPlanThreads = 1024;

// Exclusive scan of one value per thread over the CTA; returns the prefix and
// writes the CTA total to *total.
template <typename T>
__device__ T cta_exclusive_scan(T v, T *warp_sums, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T s = lane < nw ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;  // inclusive warp prefix
    }
    __syncthreads();
    const T before = warp == 0 ? T(0) : warp_sums[warp - 1];
    *total = warp_sums[nw - 1];
    __syncthreads();
    return before + x - v;
}

__device__ int check_desc(const aes_desc &d) {
    if (d.nrounds != 10 && d.nrounds != 12 && d.nrounds != 14) return AES_E_NROUNDS;
    if (d.dir != 0 && d.dir != 1) return AES_E_ARG;
    if (d.nblocks == 0) return AES_OK;
    if (!d.rk || !d.in || !d.out) return AES_E_ARG;
    if (d.nblocks > (~0ull >> 5)) return AES_E_ARG;
    const unsigned long long a = reinterpret_cast<unsigned long long>(d.in),
                             b = reinterpret_cast<unsigned long long>(d.out);
    if (((a | b) & 15ull) || (reinterpret_cast<unsigned long long>(d.rk) & 3ull)) return AES_E_ALIGN;
    const unsigned long long len = d.nblocks << 4;
    if (a != b && a < b + len && b < a + len) return AES_E_OVERLAP;
    return AES_OK;
}

__global__ void __launch_bounds__(kPlanThreads, 1)
    batch_plan_kernel(const aes_desc *__restrict__ desc, int n, void *ws, int32_t *status,
                      unsigned int chunk_blocks) {
    __shared__ unsigned long long s_u64[32];
    __shared__ unsigned int s_u32[32];
    __shared__ unsigned int s_base[2];
    const WsView v = ws_view(ws, n);

    // pass 1: number of encryption messages (invalid ones count as encryption
    // with no chunks, so they sit harmlessly in the first range)
    unsigned int n_enc = 0, n_bad = 0;
    for (int t0 = 0; t0 < n; t0 += blockDim.x) {
        const int i = t0 + static_cast<int>(threadIdx.x);
        unsigned int e = 0, bad = 0;
        if (i < n) {
            const aes_desc d = desc[i];
            const int st = check_desc(d);
            bad = st != AES_OK;
            e = bad || d.dir == 0;
            if (status) status[i] = st;
        }
        unsigned int tot = 0, totb = 0;
        (void)cta_exclusive_scan<unsigned int>(e, s_u32, &tot);
        (void)cta_exclusive_scan<unsigned int>(bad, s_u32, &totb);
        n_enc += tot;
        n_bad += totb;
    }
    // pass 2: stable partition (encryptions first) and chunk counts by position
    if (threadIdx.x == 0) { s_base[0] = 0; s_base[1] = n_enc; }
    __syncthreads();
    for (int t0 = 0; t0 < n; t0 += blockDim.x) {
        const int i = t0 + static_cast<int>(threadIdx.x);
        unsigned int e = 0;
        unsigned long long cnt = 0;
        if (i < n) {
            const aes_desc d = desc[i];
            const bool ok = check_desc(d) == AES_OK;
            e = !ok || d.dir == 0;
            cnt = ok ? (d.nblocks + chunk_blocks - 1) / chunk_blocks : 0ull;
        }
        unsigned int tot_e = 0, tot_d = 0;
        const unsigned int pe = cta_exclusive_scan<unsigned int>(e, s_u32, &tot_e);
        const unsigned int pd = cta_exclusive_scan<unsigned int>(i < n ? 1u - e : 0u, s_u32, &tot_d);
        if (i < n) {
            const unsigned int pos = e ? s_base[0] + pe : s_base[1] + pd;
            v.order[pos] = static_cast<uint32_t>(i);
            v.count[pos] = cnt;
        }
        __syncthreads();
        if (threadIdx.x == 0) { s_base[0] += tot_e; s_base[1] += tot_d; }
        __syncthreads();
    }
    __threadfence_block();
    __syncthreads();
    // pass 3: exclusive prefix of the counts in partition order
    unsigned long long run = 0;
    for (int t0 = 0; t0 < n; t0 += blockDim.x) {
        const int p = t0 + static_cast<int>(threadIdx.x);
        const unsigned long long c = p < n ? v.count[p] : 0ull;
        unsigned long long tot = 0;
        const unsigned long long pre = cta_exclusive_scan<unsigned long long>(c, s_u64, &tot);
        if (p < n) v.start[p] = run + pre;
        run += tot;
    }
    if (threadIdx.x == 0) {
        v.start[n] = run;
        v.hdr->total_chunks = run;
        v.hdr->next[0] = 0;
        v.hdr->next[1] = 0;
        v.hdr->n = static_cast<unsigned int>(n);
        v.hdr->chunk_blocks = chunk_blocks;
        v.hdr->n_invalid = n_bad;
    }
    // enc_chunks: start[n_enc] (or the total when every message encrypts)
    __syncthreads();
    if (threadIdx.x == 0) v.hdr->enc_chunks = n_enc >= static_cast<unsigned int>(n) ? run : v.start[n_enc];
}

// ---------------------------------------------------------------------------
// batch kernel
// ---------------------------------------------------------------------------
struct BatchArgs {
    const aes_desc *desc;
    void *ws;
    int n;
};

constexpr uint32_t kKeySlotBytes = 256;  // 60 words rounded up

// Shared memory of the tables of a launch: the larger of its two phases'.
__host__ __device__ constexpr uint32_t batch_table_bytes(int le, int ld) {
    return table_smem_bytes(kEncrypt, le) > table_smem_bytes(kDecrypt, ld) ? table_smem_bytes(kEncrypt, le)
                                                                            : table_smem_bytes(kDecrypt, ld);
}

#if defined(AESGB_BOUNDS_CHECK)
// Debug build: every chunk a warp takes adds one to its tag, so that after one
// launch each of the T chunks must carry exactly 1 (aes_debug_batch_coverage
// reads and clears the tags).  Chunks past the array are counted in bulk.
constexpr unsigned int kTagChunks = 1u << 16;
static __device__ unsigned int g_chunk_tag[kTagChunks];
static __device__ unsigned long long g_chunk_tag_beyond;
#endif

// Round keys of the current message held in registers for a whole chunk
// (4*(NR+1) words; every index is a compile-time constant once the rounds
// are unrolled, so the array stays in registers).
template <int NR> struct RegKey {
    uint32_t w[4 * (NR + 1)];
    __device__ __forceinline__ uint32_t operator()(int i) const { return w[i]; }
};

// Blocks [first, first + count) of one message, as passes of 32*NB blocks per
// warp with the next pass prefetched.  The round keys are read once per chunk
// from the warp's shared-memory slot (16-byte broadcasts) into registers.
template <int DIR, int NR, int NB, int LAYOUT>
__device__ __forceinline__ void batch_chunk(const Tab<LAYOUT, DIR> &tab, const uint32_t *kslot,
                                            const uint4 *in, uint4 *out, unsigned long long first,
                                            unsigned long long count, uint32_t lane) {
    RegKey<NR> key;
#pragma unroll
    for (int q = 0; q < NR + 1; ++q) {
        const uint4 v = reinterpret_cast<const uint4 *>(kslot)[q];
        key.w[4 * q] = v.x; key.w[4 * q + 1] = v.y; key.w[4 * q + 2] = v.z; key.w[4 * q + 3] = v.w;
    }
    const unsigned long long end = first + count;
    uint4 cur[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const unsigned long long b = first + lane + 32ull * i;
        cur[i] = b < end ? ld_block(in + b) : make_uint4(0, 0, 0, 0);
    }
    for (unsigned long long base = first; base < end; base += 32ull * NB) {
        uint4 nxt[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const unsigned long long b = base + 32ull * NB + lane + 32ull * i;
            nxt[i] = b < end ? ld_block(in + b) : make_uint4(0, 0, 0, 0);
        }
        uint32_t s[NB][4];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            s[i][0] = cur[i].x; s[i][1] = cur[i].y; s[i][2] = cur[i].z; s[i][3] = cur[i].w;
        }
        cipher_states<DIR, NR, NB>(tab, key, s);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const unsigned long long b = base + lane + 32ull * i;
            if (b < end) st_block(out + b, make_uint4(s[i][0], s[i][1], s[i][2], s[i][3]));
            cur[i] = nxt[i];
        }
    }
}

// Partition position q of the message owning chunk c: the largest q in
// [lo, n) with start[q] <= c (start[n] = T > c).  32-ary search by the whole
// warp: each lane probes one of 31 evenly spaced positions per step.
__device__ __forceinline__ int find_message(const unsigned long long *start, int lo, int n,
                                            unsigned long long c, uint32_t lane) {
    int hi = n;
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) / 32;
        const int q = lo + static_cast<int>(lane + 1) * step;
        const bool le = q < hi && start[q] <= c;
        const int k = __popc(__ballot_sync(0xffffffffu, le));
        const int nlo = lo + k * step;
        const int nhi = lo + (k + 1) * step;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    return lo;
}

// All chunks of one direction, handed out one at a time to whichever warp
// asks next (an atomic counter in the workspace; the next chunk index is
// requested before the current chunk is processed, so the atomic's latency is
// hidden).  Chunk c of this phase is chunk c_begin + c of the partition.
template <int DIR, int NB, int LAYOUT>
__device__ void batch_phase(const BatchArgs &a, const WsView &v, uint8_t *smem, uint32_t *kslot,
                            unsigned long long c_begin, unsigned long long c_end) {
    const uint32_t lane = threadIdx.x & 31u;
    const Tab<LAYOUT, DIR> tab(smem, lane);
    unsigned long long *counter = &v.hdr->next[DIR];
    const unsigned long long nchunks = c_end - c_begin;
    const unsigned int cb = v.hdr->chunk_blocks;
    const int n = a.n;
    int p = 0;                                  // partition position of the current message
    unsigned long long p_start = 0, p_end = 0;  // its chunk range [p_start, p_end)
    const uint4 *in = nullptr;
    uint4 *out = nullptr;
    unsigned long long nb = 0;
    int nr = 10;
    bool have = false;
    unsigned long long ticket = 0;
    // the warp's key slot lies inside the launch's shared memory
    if (!AESGB_CHECK(static_cast<uint32_t>(reinterpret_cast<uint8_t *>(kslot) - smem) + kKeySlotBytes <=
                     dyn_smem_bytes()))
        return;
    if (lane == 0) ticket = atomicAdd(counter, 1ull);
    unsigned long long rel = __shfl_sync(0xffffffffu, ticket, 0);
    while (rel < nchunks) {
        if (lane == 0) ticket = atomicAdd(counter, 1ull);  // next chunk, consumed after this one
        const unsigned long long c = c_begin + rel;
        if (!have || c >= p_end) {
            p = find_message(v.start, have ? p + 1 : 0, n, c, lane);
            // p is a partition position with c in its chunk range, and names
            // a message (each value is the same in every lane: no divergence)
            if (!AESGB_CHECK(p >= 0 && p < n && v.order[p] < static_cast<uint32_t>(n) && v.start[p] <= c &&
                             c < v.start[p + 1]))
                break;
            p_start = v.start[p];
            p_end = v.start[p + 1];
            const aes_desc d = a.desc[v.order[p]];
            in = reinterpret_cast<const uint4 *>(d.in);
            out = reinterpret_cast<uint4 *>(d.out);
            nb = d.nblocks;
            nr = d.nrounds;
            __syncwarp();
            const int nw = 4 * (nr + 1);
            for (int i = static_cast<int>(lane); i < nw; i += 32) {
                const int step = i >> 2;
                const int src = DIR == kEncrypt ? step : nr - step;
                kslot[i] = d.rk[4 * src + (i & 3)];
            }
            __syncwarp();
            have = true;
        }
        const unsigned long long first = (c - p_start) * cb;
        const unsigned long long cnt = nb - first < cb ? nb - first : cb;
        if (!AESGB_CHECK(first < nb && cnt >= 1 && cnt <= cb && (nr == 10 || nr == 12 || nr == 14))) break;
#if defined(AESGB_BOUNDS_CHECK)
        if (lane == 0) {
            if (c < kTagChunks) atomicAdd(&g_chunk_tag[c], 1u);
            else atomicAdd(&g_chunk_tag_beyond, 1ull);
        }
#endif
        switch (nr) {
        case 10: batch_chunk<DIR, 10, NB, LAYOUT>(tab, kslot, in, out, first, cnt, lane); break;
        case 12: batch_chunk<DIR, 12, NB, LAYOUT>(tab, kslot, in, out, first, cnt, lane); break;
        default: batch_chunk<DIR, 14, NB, LAYOUT>(tab, kslot, in, out, first, cnt, lane); break;
        }
        rel = __shfl_sync(0xffffffffu, ticket, 0);
    }
}

constexpr int kBatchMaxThreads = 512;  // up to 128 registers: round keys live in registers

// LE, LD: table layouts of the encryption and decryption phases.
template <int NB, int LE, int LD>
__global__ void __launch_bounds__(kBatchMaxThreads, 1) batch_kernel(const __grid_constant__ BatchArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const WsView v = ws_view(a.ws, a.n);
    const unsigned long long T = v.hdr->total_chunks, E = v.hdr->enc_chunks;
    uint32_t *kslot =
        reinterpret_cast<uint32_t *>(smem + batch_table_bytes(LE, LD) + (threadIdx.x >> 5) * kKeySlotBytes);
    if (E > 0) {
        Tab<LE, kEncrypt>::fill(smem, threadIdx.x, blockDim.x);
        __syncthreads();
        batch_phase<kEncrypt, NB, LE>(a, v, smem, kslot, 0, E);
    }
    if (T > E) {
        __syncthreads();  // every warp is done with the encryption tables
        Tab<LD, kDecrypt>::fill(smem, threadIdx.x, blockDim.x);
        __syncthreads();
        batch_phase<kDecrypt, NB, LD>(a, v, smem, kslot, E, T);
    }
}

AESGB_BOUNDS_READER(batch)

uint32_t batch_smem_bytes(const aes_batch_cfg &c) {
    return batch_table_bytes(c.layout_enc, c.layout_dec) + static_cast<uint32_t>(c.threads / 32) * kKeySlotBytes;
}

// The compiled (blocks per thread, encryption layout, decryption layout)
// combinations: the default pair R4 / R2 at 1, 2 and 4 blocks per thread, and
// the pairs R4 / R4, R2 / R2 and R1 / R1 at 1 and 2 (the tuner's range).
const void *batch_kernel_ptr(int nb, int le, int ld) {
#define AESGB_BK(NB, LE, LD) \
    if (nb == NB && le == LE && ld == LD) return reinterpret_cast<const void *>(&batch_kernel<NB, LE, LD>);
    AESGB_BK(1, kLayoutR4, kLayoutR2) AESGB_BK(2, kLayoutR4, kLayoutR2) AESGB_BK(4, kLayoutR4, kLayoutR2)
    AESGB_BK(1, kLayoutR4, kLayoutR4) AESGB_BK(2, kLayoutR4, kLayoutR4)
    AESGB_BK(1, kLayoutR2, kLayoutR2) AESGB_BK(2, kLayoutR2, kLayoutR2)
    AESGB_BK(1, kLayoutR1, kLayoutR1) AESGB_BK(2, kLayoutR1, kLayoutR1)
#undef AESGB_BK
    return nullptr;
}

int validate_batch_cfg(const aes_batch_cfg &c) {
    if (c.blocks_per_thread != 1 && c.blocks_per_thread != 2 && c.blocks_per_thread != 4) return AES_E_CONFIG;
    if (c.threads < 32 || c.threads % 32 || c.threads > kBatchMaxThreads) return AES_E_CONFIG;
    if (c.chunk_passes < 1 || c.chunk_passes > 1024) return AES_E_CONFIG;
    if (c.ctas_per_sm < 0 || c.ctas_per_sm > 1) return AES_E_CONFIG;
    if (!batch_kernel_ptr(c.blocks_per_thread, c.layout_enc, c.layout_dec)) return AES_E_CONFIG;
    return AES_OK;
}

int enqueue_batch(const aes_desc *desc, int n, void *ws, size_t ws_bytes, int32_t *status,
                  const aes_batch_cfg &c, cudaStream_t s) {
    if (n == 0) return AES_OK;
    if (n > AES_BATCH_MAX_DESCS) return AES_E_RANGE;  // keeps the kernels' int indices far from overflow
    if (!desc || !ws) return AES_E_ARG;
    if (ws_bytes < batch_ws_bytes(n)) return AES_E_RANGE;
    if (reinterpret_cast<uintptr_t>(ws) & 255u) return AES_E_ALIGN;
    int st = validate_batch_cfg(c);
    if (st != AES_OK) return st;
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    const unsigned int chunk_blocks = static_cast<unsigned int>(32 * c.blocks_per_thread * c.chunk_passes);
    batch_plan_kernel<<<1, kPlanThreads, 0, s>>>(desc, n, ws, status, chunk_blocks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return AES_E_CUDA;
    const void *fn = batch_kernel_ptr(c.blocks_per_thread, c.layout_enc, c.layout_dec);
    const uint32_t smem = batch_smem_bytes(c);
    st = ensure_smem_attr(fn, dev, smem);
    if (st != AES_OK) return st;
    const int sms = sm_count(dev);
    if (sms < 0) return sms;
    BatchArgs args{desc, ws, n};
    void *params[] = {&args};
    e = cudaLaunchKernel(fn, dim3(sms), dim3(c.threads), params, smem, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    return AES_OK;
}

// ---------------------------------------------------------------------------
// host-side planning (for callers that know their batch: the server)
// ---------------------------------------------------------------------------
// Writes into a HOST buffer of batch_ws_bytes(n) bytes exactly what the plan
// kernel would write into the workspace for these descriptors, which must all
// be valid (check_desc): encryptions first in input order, then decryptions;
// start[] the exclusive prefix of ceil(nblocks / chunk_blocks); counters 0.
void plan_on_host(const aes_desc *desc, int n, unsigned int chunk_blocks, void *ws_host) {
    const WsView v = ws_view(ws_host, n);
    int pos = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < n; ++i)
            if ((desc[i].dir == 0) == (pass == 0)) {
                v.order[pos] = static_cast<uint32_t>(i);
                v.count[pos] = (desc[i].nblocks + chunk_blocks - 1) / chunk_blocks;
                ++pos;
            }
    unsigned long long run = 0, enc_chunks = 0;
    for (int p = 0; p < n; ++p) {
        v.start[p] = run;
        run += v.count[p];
        if (desc[v.order[p]].dir == 0) enc_chunks = run;
    }
    v.start[n] = run;
    v.hdr->total_chunks = run;
    v.hdr->enc_chunks = enc_chunks;
    v.hdr->next[0] = 0;
    v.hdr->next[1] = 0;
    v.hdr->n = static_cast<unsigned int>(n);
    v.hdr->chunk_blocks = chunk_blocks;
    v.hdr->n_invalid = 0;
    v.hdr->pad = 0;
}

unsigned int batch_chunk_blocks(const aes_batch_cfg &c) {
    return static_cast<unsigned int>(32 * c.blocks_per_thread * c.chunk_passes);
}

// The persistent batch kernel alone, on a workspace planned already.
int enqueue_batch_kernel(const aes_desc *desc, int n, void *ws, const aes_batch_cfg &c, cudaStream_t s) {
    if (n == 0) return AES_OK;
    if (n > AES_BATCH_MAX_DESCS) return AES_E_RANGE;
    int st = validate_batch_cfg(c);
    if (st != AES_OK) return st;
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    const void *fn = batch_kernel_ptr(c.blocks_per_thread, c.layout_enc, c.layout_dec);
    const uint32_t smem = batch_smem_bytes(c);
    st = ensure_smem_attr(fn, dev, smem);
    if (st != AES_OK) return st;
    const int sms = sm_count(dev);
    if (sms < 0) return sms;
    BatchArgs args{desc, ws, n};
    void *params[] = {&args};
    if (cudaLaunchKernel(fn, dim3(sms), dim3(c.threads), params, smem, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    return AES_OK;
}

// ---------------------------------------------------------------------------
// library-owned workspaces for aes_ecb_batch: one per (device, stream)
// ---------------------------------------------------------------------------
// A stream is named by its CUDA stream id (cudaStreamGetId), which is unique
// for the process's lifetime and tells apart the per-thread default streams
// that share one handle value.  Work on one stream runs in order, so a
// workspace reused by the next call on the same stream is never in use by
// another batch; calls on different streams never share one.  Growth is
// stream-ordered: the old buffer goes back with cudaFreeAsync behind the
// batches already enqueued on that stream, the new one comes from
// cudaMallocAsync, and neither waits for the device.  A context's mutex is
// held from the size check to the end of the enqueue, so no thread can free a
// buffer that another thread has looked up but not yet enqueued.
namespace {
struct StreamWs {
    std::mutex mu;
    void *ptr = nullptr;
    size_t bytes = 0;
    int dev = 0;
    cudaEvent_t last = nullptr;  // recorded after the newest batch that uses ptr
    std::atomic<int> users{0};   // callers that looked it up and have not finished (never evicted then)
};
using WsKey = std::pair<int, unsigned long long>;  // device, stream id
std::mutex g_ws_mu;
std::map<WsKey, std::shared_ptr<StreamWs>> g_ws;
// Above this many contexts, idle ones (last batch complete) are released
// when a new one is made: streams the caller destroyed leave contexts behind.
constexpr size_t kMaxStreamWs = 64;

// Release the device memory of contexts other than `keep` whose last batch
// has completed (g_ws_mu held).  The memory is idle, so it goes back in the
// order of stream s without waiting for anything.
void evict_idle_locked(const StreamWs *keep, cudaStream_t s) {
    for (auto it = g_ws.begin(); it != g_ws.end() && g_ws.size() > kMaxStreamWs;) {
        StreamWs &w = *it->second;
        std::unique_lock<std::mutex> lk(w.mu, std::try_to_lock);
        const bool idle = &w != keep && w.users.load() == 0 && lk.owns_lock() &&
                          (w.last == nullptr || cudaEventQuery(w.last) == cudaSuccess);
        (void)cudaGetLastError();
        if (!idle) {
            ++it;
            continue;
        }
        if (w.ptr) (void)cudaFreeAsync(w.ptr, s);
        if (w.last) (void)cudaEventDestroy(w.last);
        w.ptr = nullptr;
        w.bytes = 0;
        w.last = nullptr;
        lk.unlock();
        it = g_ws.erase(it);
    }
    (void)cudaGetLastError();
}
}  // namespace

// The context of (dev, stream s), created on first use.  Its user count is
// raised here, under the map's mutex, so eviction (also under it) never takes
// a context that a caller is about to lock; the caller lowers it when done.
int stream_workspace(int dev, cudaStream_t s, std::shared_ptr<StreamWs> *out) {
    unsigned long long id = 0;
    if (cudaStreamGetId(s, &id) != cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_ws_mu);
    std::shared_ptr<StreamWs> &slot = g_ws[WsKey{dev, id}];
    if (!slot) {
        slot = std::make_shared<StreamWs>();
        slot->dev = dev;
    }
    *out = slot;  // (evict_idle_locked keeps this entry, so the reference stays valid)
    (*out)->users.fetch_add(1);
    if (g_ws.size() > kMaxStreamWs) evict_idle_locked(out->get(), s);
    return AES_OK;
}

// Enqueue the batch on s with the context's workspace, grown first if it is
// smaller than `need` (w.mu held by the caller).
int enqueue_with_stream_ws(StreamWs &w, const aes_desc *desc, int n, size_t need, int32_t *status,
                           cudaStream_t s) {
    if (w.bytes < need) {
        const size_t sz = need < (1u << 20) ? (1u << 20) : need * 2;
        void *p = nullptr;
        const int st = lib_malloc_device_async(&p, sz, s);
        if (st != AES_OK) return st;  // the old workspace stays as it was
        if (w.ptr) (void)cudaFreeAsync(w.ptr, s);
        w.ptr = p;
        w.bytes = sz;
    }
    if (!w.last && cudaEventCreateWithFlags(&w.last, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        w.last = nullptr;
        return AES_E_CUDA;
    }
    const int st = enqueue_batch(desc, n, w.ptr, w.bytes, status, batch_cfg_for(n), s);
    if (st != AES_OK) return st;
    if (cudaEventRecord(w.last, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    return AES_OK;
}

void batch_shutdown() {
    std::map<WsKey, std::shared_ptr<StreamWs>> all;
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        all.swap(g_ws);
    }
    int cur = 0;
    const bool have_cur = cudaGetDevice(&cur) == cudaSuccess;
    for (auto &kv : all) {
        StreamWs &w = *kv.second;
        std::lock_guard<std::mutex> lk(w.mu);
        if (w.ptr || w.last) (void)cudaSetDevice(w.dev);
        if (w.ptr) (void)cudaFree(w.ptr);  // no library work is in flight (aes_shutdown's contract)
        if (w.last) (void)cudaEventDestroy(w.last);
        w.ptr = nullptr;
        w.bytes = 0;
        w.last = nullptr;
    }
    if (have_cur) (void)cudaSetDevice(cur);
    (void)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// graph: plan + batch captured once, replayed many times
// ---------------------------------------------------------------------------
struct BatchGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// ---------------------------------------------------------------------------
// Batch scratch in a file-scope device array, for callers that cannot
// allocate device memory (see aes_ecb_batch_noalloc in aesgb.h).
// ---------------------------------------------------------------------------
constexpr size_t noalloc_scratch_bytes(size_t n) {
    return align_up(sizeof(BatchHeader), 256) + align_up(4 * n, 256) + align_up(8 * (n + 1), 256) +
           align_up(8 * n, 256);
}
constexpr size_t kNoAllocBytes = noalloc_scratch_bytes(AES_BATCH_NOALLOC_MAX_DESCS);

// One copy per device that loads this library; it lives until the process exits.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kMaxDev = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDev];  // device address of g_noalloc_scratch, per device
}  // namespace

// Device address of this device's scratch array, looked up once per device
// (the host-side name of the array is not a device address).
int noalloc_scratch_ptr(int dev, void **out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return AES_E_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return AES_OK;
}

// Debug build: counts of chunks taken exactly once and more than once since
// the last call, and of chunks past the tag array; clears the tags.
int read_chunk_coverage(unsigned long long *once, unsigned long long *repeated, unsigned long long *beyond) {
#if defined(AESGB_BOUNDS_CHECK)
    static unsigned int tags[kTagChunks];
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    const unsigned long long zero = 0;
    if (cudaMemcpyFromSymbol(tags, g_chunk_tag, sizeof tags) != cudaSuccess ||
        cudaMemcpyFromSymbol(beyond, g_chunk_tag_beyond, sizeof *beyond) != cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    *once = 0;
    *repeated = 0;
    for (unsigned int i = 0; i < kTagChunks; ++i) {
        *once += tags[i] == 1;
        *repeated += tags[i] > 1;
    }
    void *tag_addr = nullptr;
    if (cudaGetSymbolAddress(&tag_addr, g_chunk_tag) != cudaSuccess ||
        cudaMemset(tag_addr, 0, sizeof tags) != cudaSuccess ||
        cudaMemcpyToSymbol(g_chunk_tag_beyond, &zero, sizeof zero) != cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    return AES_OK;
#else
    *once = *repeated = *beyond = 0;
    return AES_E_CONFIG;
#endif
}

}  // namespace aesgb

using namespace aesgb;

extern "C" {

size_t aes_batch_workspace_bytes(int n) { return n < 0 ? 0 : batch_ws_bytes(n); }

int aes_debug_batch_coverage(unsigned long long *once, unsigned long long *repeated, unsigned long long *beyond) {
    if (!once || !repeated || !beyond) return AES_E_ARG;
    return read_chunk_coverage(once, repeated, beyond);
}

int aes_ecb_batch_ws(const aes_desc *desc_dev, int n, void *ws, size_t ws_bytes, int32_t *status_dev,
                     const aes_batch_cfg *cfg, void *stream) {
    if (n < 0) return AES_E_ARG;
    const aes_batch_cfg c = cfg ? *cfg : batch_cfg_for(n);
    return enqueue_batch(desc_dev, n, ws, ws_bytes, status_dev, c, static_cast<cudaStream_t>(stream));
}

int aes_ecb_batch(const aes_desc *desc_dev, int n, void *stream) {
    return aes_ecb_batch_ex(desc_dev, n, nullptr, stream);
}

int aes_ecb_batch_ex(const aes_desc *desc_dev, int n, int32_t *status_dev, void *stream) {
    if (n < 0) return AES_E_ARG;
    if (n == 0) return AES_OK;
    if (n > AES_BATCH_MAX_DESCS) return AES_E_RANGE;  // before the workspace is sized for it
    if (!desc_dev) return AES_E_ARG;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    // a graph captured from this call would keep the workspace's address after
    // a later call on the stream has replaced it: capture aes_ecb_batch_ws
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return AES_E_CONFIG;
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    std::shared_ptr<StreamWs> w;
    const int st = stream_workspace(dev, s, &w);
    if (st != AES_OK) return st;
    int r;
    {
        std::lock_guard<std::mutex> lk(w->mu);
        r = enqueue_with_stream_ws(*w, desc_dev, n, batch_ws_bytes(n), status_dev, s);
    }
    w->users.fetch_sub(1);
    return r;
}

int aes_ecb_batch_noalloc(const aes_desc *desc_dev, int n, int32_t *status_dev, void *stream) {
    if (n < 0) return AES_E_ARG;
    if (n > AES_BATCH_NOALLOC_MAX_DESCS) return AES_E_RANGE;
    if (n == 0) return AES_OK;
    if (batch_ws_bytes(n) > kNoAllocBytes) return AES_E_RANGE;
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    void *scratch = nullptr;
    const int st = noalloc_scratch_ptr(dev, &scratch);
    if (st != AES_OK) return st;
    // the plan kernel rewrites the header (work counters zeroed) and every
    // array the batch kernel reads, so what the previous call left behind in
    // the scratch is never used
    return enqueue_batch(desc_dev, n, scratch, kNoAllocBytes, status_dev, batch_cfg_for(n),
                         static_cast<cudaStream_t>(stream));
}

int aes_batch_graph_create(const aes_desc *desc_dev, int n, void *ws, size_t ws_bytes, int32_t *status_dev,
                           const aes_batch_cfg *cfg, aes_batch_graph **out) {
    if (!out || n <= 0) return AES_E_ARG;
    *out = nullptr;
    if (n > AES_BATCH_MAX_DESCS) return AES_E_RANGE;
    const aes_batch_cfg c = cfg ? *cfg : batch_cfg_for(n);
    int st0 = validate_batch_cfg(c);
    if (st0 != AES_OK) return st0;
    // one-time per-kernel set-up (shared-memory attribute) before capturing
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    st0 = ensure_smem_attr(batch_kernel_ptr(c.blocks_per_thread, c.layout_enc, c.layout_dec), dev,
                           batch_smem_bytes(c));
    if (st0 != AES_OK) return st0;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return AES_E_CUDA;
    BatchGraph *g = new BatchGraph();
    int st = AES_OK;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = AES_E_CUDA;
    if (st == AES_OK) {
        st = enqueue_batch(desc_dev, n, ws, ws_bytes, status_dev, c, s);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (st == AES_OK && e != cudaSuccess) st = AES_E_CUDA;
        g->graph = graph;
        if (st == AES_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) st = AES_E_CUDA;
    }
    cudaStreamDestroy(s);
    if (st != AES_OK) {
        (void)cudaGetLastError();
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return st;
    }
    *out = reinterpret_cast<aes_batch_graph *>(g);
    return AES_OK;
}

int aes_batch_graph_launch(aes_batch_graph *graph, void *stream) {
    if (!graph) return AES_E_ARG;
    BatchGraph *g = reinterpret_cast<BatchGraph *>(graph);
    if (cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    return AES_OK;
}

int aes_batch_graph_destroy(aes_batch_graph *graph) {
    if (!graph) return AES_OK;
    BatchGraph *g = reinterpret_cast<BatchGraph *>(graph);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return AES_OK;
}

}  // extern "C"
