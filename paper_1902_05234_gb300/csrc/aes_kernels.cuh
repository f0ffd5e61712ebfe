// aes_kernels.cuh -- sm_103a device code for bulk AES (T-table form).
//
// One AES block (16-byte state) is four 32-bit column words; byte r of a word
// is row r.  A full round (Wang & Chu eq (26)) computes each output column as
// four table lookups, one per row, XORed with the round-key column:
//
//   encrypt  e_j = T0[s_{0,j}] ^ T1[s_{1,j+1}] ^ T2[s_{2,j+2}] ^ T3[s_{3,j+3}] ^ k_j
//   decrypt  e_j = D0[s_{0,j}] ^ D1[s_{1,j-1}] ^ D2[s_{2,j-2}] ^ D3[s_{3,j-3}] ^ k_j
//
// (column indices mod 4; T_k of eqs (22)-(25), D_k their inverse-cipher
// analogues, FIPS-197 5.3.5).  The final round has no MixColumns: S-box bytes
// (encrypt: byte 1 of T0, which is S(x); decrypt: an InvS table) are gathered
// into the output column with byte permutes.
//
// The lookups are the bound (16 per block per round), so the tables sit in
// shared memory laid out so that lane l of a warp only ever touches bank l:
//
//   R4  "replicated, four tables": entry x of table t for lane l at byte
//       x*256 + 4*l + 128*(t&1) + 65536*(t>>1).  The address is ONE byte
//       permute of the state word with a per-lane constant (x lands in bits
//       8..15, 4*l in bits 0..7) plus an immediate.  128 KiB; decryption adds
//       InvS at 131072 + x*128 + 4*l (160 KiB).
//   R1  one table per bank-replicated at x*256 + 4*l, the other three by
//       byte rotation (one funnel shift each); decryption keeps InvS in the
//       gaps at +128.  64 KiB.
//   P4  four plain 1 KiB tables (t*1024 + 4x): the paper's "shared memory"
//       alternative of section 4.2, with bank conflicts.
//   CONST  the tables in constant memory, as the paper places them (4.2).
//   REG  the table in registers, the third placement of section 4.2: lane l
//       of every warp holds T0[l + 32j], j = 0..7, in eight registers.  A
//       lookup of x takes register j from lane x mod 32 by shuffle, for all
//       eight j (a shuffle reads the same register in every source lane), and
//       keeps j = x / 32 with three selects; T1..T3 are byte rotations of T0.
//       Decryption adds InvS, four bytes per register (two registers).  No
//       shared memory.
//
// Round keys are uniform across the grid (section 4.3 puts them in constant
// memory): the single-buffer kernels take them as kernel parameters, so each
// XOR with a key word reads the constant bank directly.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "aes_tables.h"
#include "bounds.cuh"

namespace aesgb {

enum : int { kLayoutR4 = 0, kLayoutR1 = 1, kLayoutP4 = 2, kLayoutConst = 3, kLayoutR2 = 5, kLayoutReg = 6 };
enum : int { kEncrypt = 0, kDecrypt = 1 };

constexpr int kMaxRkWords = 60;  // 4 * (14 + 1)

// Round keys in the order they are applied: words 4i..4i+3 are the key of
// step i = 0..Nr (for decryption the host reverses the dw schedule).
struct RoundKeys {
    uint32_t w[kMaxRkWords];
};

struct EcbArgs {
    const uint4 *in;
    uint4 *out;
    unsigned long long nblocks;
    RoundKeys rk;
    // At most this many units per warp take even contiguous shares (0: always
    // grid-stride passes); see ecb_kernel.
    unsigned int even_split_units;
};

__host__ __device__ constexpr uint32_t table_smem_bytes(int dir, int layout) {
    return layout == kLayoutR4   ? (dir == kDecrypt ? 160u * 1024u : 128u * 1024u)
           : layout == kLayoutR2 ? (dir == kDecrypt ? 128u * 1024u : 64u * 1024u)
           : layout == kLayoutR1 ? 64u * 1024u
           : layout == kLayoutP4 ? (dir == kDecrypt ? 5u * 1024u : 4u * 1024u)
                                 : 0u;
}

constexpr int max_threads_for_nb(int nb) { return nb >= 8 ? 256 : nb >= 4 ? 512 : 1024; }
// The register-table layout holds eight (decryption ten) table words per
// thread, and the compiler keeps the shuffled candidates of several lookups
// live at once: at most 256 threads (up to 255 registers each; at 512 threads
// it spills).
constexpr int max_threads_for(int nb, int layout) {
    return layout == kLayoutReg && max_threads_for_nb(nb) > 256 ? 256 : max_threads_for_nb(nb);
}

// Each module keeps its own copy of the compile-time tables in constant memory.
static __constant__ ConstTables c_tab = make_const_tables();

// The same T0 and D0, and InvS packed four bytes per word (byte k of word w is
// InvS[4w + k]), in global memory for the shared-memory table fills and the
// register layout: a warp reads each with coalesced loads (one 128-byte line
// per register), where constant memory would serve 32 different addresses one
// at a time.  Compile-time constants, never written, so a kernel may read them
// before it waits for the previous kernel in its stream.
struct FillTables {
    uint32_t t0[2][256];
    uint32_t is4[64];
};
constexpr FillTables make_fill_tables() {
    FillTables f{};
    for (int x = 0; x < 256; ++x) {
        f.t0[0][x] = kAes.te0[x];
        f.t0[1][x] = kAes.td0[x];
    }
    for (int w = 0; w < 64; ++w)
        f.is4[w] = static_cast<uint32_t>(kAes.isbox[4 * w]) | (static_cast<uint32_t>(kAes.isbox[4 * w + 1]) << 8) |
                   (static_cast<uint32_t>(kAes.isbox[4 * w + 2]) << 16) |
                   (static_cast<uint32_t>(kAes.isbox[4 * w + 3]) << 24);
    return f;
}
static __device__ const FillTables g_fill = make_fill_tables();

// Table reads and writes at a byte offset into the dynamic shared memory
// (checked against the launch's size in the debug build).
__device__ __forceinline__ uint32_t lds32(const uint8_t *smem, uint32_t off) {
    if (!AESGB_CHECK(off + 4u <= dyn_smem_bytes())) return 0u;
    return *reinterpret_cast<const uint32_t *>(smem + off);
}
__device__ __forceinline__ void sts32(uint8_t *smem, uint32_t off, uint32_t v) {
    if (!AESGB_CHECK(off + 4u <= dyn_smem_bytes())) return;
    *reinterpret_cast<uint32_t *>(smem + off) = v;
}
__device__ __forceinline__ uint32_t rotl32(uint32_t v, int n) {
    return n == 0 ? v : __funnelshift_l(v, v, n);
}
// Byte b of s moved to bits 8..15, byte 0 of `low` kept in bits 0..7, upper
// half from `low` too (zero): x*256 + lane*4 in one PRMT.
__device__ __forceinline__ uint32_t byte_to_bits8(uint32_t s, uint32_t low, int b) {
    return __byte_perm(s, low, 0x7604u | (static_cast<uint32_t>(b) << 4));
}
// Byte b of s as an integer 0..255.
__device__ __forceinline__ uint32_t byte_of(uint32_t s, int b) {
    return __byte_perm(s, 0u, 0x4440u | static_cast<uint32_t>(b));
}

// Fill of the bank-replicated layouts (R4, R2, R1).  Warp w loads T0 (D0)
// into eight registers per lane (entry lane + 32j in register j) and InvS into
// two; then for every entry x = 32j + c with c = w, w + nw, ... it broadcasts
// T0[x] (and InvS[x]) from lane c by shuffle, and each lane l calls
// put(x, l, T0[x], InvS[x]) to store the entry into its own replicas, which
// sit in bank l: a warp's stores never conflict, and no lane waits on a
// constant-cache load per entry.  T1..T3 are rotations of T0 (eqs
// (22)-(25)), so put() derives them.  Every thread of the CTA calls this
// (full-warp shuffles); nthr is a multiple of 32, at most 1024.
template <int DIR, class Put>
__device__ __forceinline__ void fill_replicated(int tid, int nthr, Put put) {
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    uint32_t r[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = g_fill.t0[DIR][lane + 32 * j];
    const uint32_t is0 = DIR == kDecrypt ? g_fill.is4[lane] : 0u;
    const uint32_t is1 = DIR == kDecrypt ? g_fill.is4[lane + 32] : 0u;
    for (int c = warp; c < 32; c += nw) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t x = 32u * j + static_cast<uint32_t>(c);
            const uint32_t t0 = __shfl_sync(0xffffffffu, r[j], c);
            uint32_t is = 0u;
            if (DIR == kDecrypt) {  // packed word x / 4 sits in lane (x / 4) mod 32 of is0 (x < 128) or is1
                const uint32_t wv = __shfl_sync(0xffffffffu, j < 4 ? is0 : is1, static_cast<int>((x >> 2) & 31u));
                is = (wv >> (8u * (x & 3u))) & 0xffu;
            }
            put(x, static_cast<uint32_t>(lane), t0, is);
        }
    }
}

// ---------------------------------------------------------------------------
// Table policies.  lookup(t, s, b): table t at index byte b of word s.
// final_word(s, b): a word whose byte kFinalByte is S(x) (encrypt) or IS(x)
// (decrypt) for x = byte b of s.
// ---------------------------------------------------------------------------
template <int LAYOUT, int DIR> struct Tab;

template <int DIR> struct Tab<kLayoutR4, DIR> {
    static constexpr int kFinalByte = DIR == kEncrypt ? 1 : 0;
    const uint8_t *smem;
    uint32_t lane4, lane8;
    __device__ Tab(const uint8_t *s, uint32_t lane) : smem(s), lane4(lane * 4u), lane8(lane * 8u) {}
    __device__ static void fill(uint8_t *smem, int tid, int nthr) {
        fill_replicated<DIR>(tid, nthr, [smem](uint32_t x, uint32_t l, uint32_t t0, uint32_t is) {
            const uint32_t o = x * 256u + l * 4u;
            sts32(smem, o, t0);
            sts32(smem, o + 128u, rotl32(t0, 8));
            sts32(smem, o + 65536u, rotl32(t0, 16));
            sts32(smem, o + 65536u + 128u, rotl32(t0, 24));
            if (DIR == kDecrypt) sts32(smem, 131072u + x * 128u + l * 4u, is);
        });
    }
    __device__ __forceinline__ uint32_t lookup(int t, uint32_t s, int b) const {
        return lds32(smem, byte_to_bits8(s, lane4, b) + 128u * (t & 1) + 65536u * (t >> 1));
    }
    __device__ __forceinline__ uint32_t final_word(uint32_t s, int b) const {
        if (DIR == kEncrypt) return lds32(smem, byte_to_bits8(s, lane4, b));
        return lds32(smem, 131072u + (byte_to_bits8(s, lane8, b) >> 1));
    }
};

// Two bank-replicated tables, T0 and T1, laid out as the first half of R4
// (64 KiB).  Decryption adds InvS at 65536 + 256x + 4l: the same address as
// the T0 entry plus a constant, so the final round needs no address shift of
// its own (64 KiB more, with half of each 256-byte row unused).  T2 = rotl(T0, 16)
// and T3 = rotl(T1, 16), so a column of a round is
//   T0[a] ^ T1[b] ^ rotl16(T0[c] ^ T1[d] ^ rotr16(k)):
// one 16-bit rotation per column (kPairRotate) instead of two more tables.
template <int DIR> struct Tab<kLayoutR2, DIR> {
    static constexpr int kFinalByte = DIR == kEncrypt ? 1 : 0;
    static constexpr bool kPairRotate = true;
    const uint8_t *smem;
    uint32_t lane4;
    __device__ Tab(const uint8_t *s, uint32_t lane) : smem(s), lane4(lane * 4u) {}
    __device__ static void fill(uint8_t *smem, int tid, int nthr) {
        fill_replicated<DIR>(tid, nthr, [smem](uint32_t x, uint32_t l, uint32_t t0, uint32_t is) {
            const uint32_t o = x * 256u + l * 4u;
            sts32(smem, o, t0);
            sts32(smem, o + 128u, rotl32(t0, 8));
            if (DIR == kDecrypt) sts32(smem, 65536u + o, is);
        });
    }
    // T0 for t = 0, 2 and T1 for t = 1, 3: full_round rotates the t = 2, 3 pair
    __device__ __forceinline__ uint32_t lookup(int t, uint32_t s, int b) const {
        return lds32(smem, byte_to_bits8(s, lane4, b) + 128u * (t & 1));
    }
    __device__ __forceinline__ uint32_t final_word(uint32_t s, int b) const {
        return lds32(smem, byte_to_bits8(s, lane4, b) + (DIR == kEncrypt ? 0u : 65536u));
    }
};

template <int DIR> struct Tab<kLayoutR1, DIR> {
    static constexpr int kFinalByte = DIR == kEncrypt ? 1 : 0;
    const uint8_t *smem;
    uint32_t lane4;
    __device__ Tab(const uint8_t *s, uint32_t lane) : smem(s), lane4(lane * 4u) {}
    __device__ static void fill(uint8_t *smem, int tid, int nthr) {
        fill_replicated<DIR>(tid, nthr, [smem](uint32_t x, uint32_t l, uint32_t t0, uint32_t is) {
            const uint32_t o = x * 256u + l * 4u;
            sts32(smem, o, t0);
            if (DIR == kDecrypt) sts32(smem, o + 128u, is);
        });
    }
    __device__ __forceinline__ uint32_t lookup(int t, uint32_t s, int b) const {
        return rotl32(lds32(smem, byte_to_bits8(s, lane4, b)), 8 * t);
    }
    __device__ __forceinline__ uint32_t final_word(uint32_t s, int b) const {
        return lds32(smem, byte_to_bits8(s, lane4, b) + (DIR == kEncrypt ? 0u : 128u));
    }
};

template <int DIR> struct Tab<kLayoutP4, DIR> {
    static constexpr int kFinalByte = DIR == kEncrypt ? 1 : 0;
    const uint8_t *smem;
    __device__ Tab(const uint8_t *s, uint32_t) : smem(s) {}
    __device__ static void fill(uint8_t *smem, int tid, int nthr) {
        const int n = DIR == kEncrypt ? 1024 : 1280;
        for (int i = tid; i < n; i += nthr) {
            uint32_t v;
            if (i < 1024) v = DIR == kEncrypt ? c_tab.te[i >> 8][i & 255] : c_tab.td[i >> 8][i & 255];
            else v = c_tab.is[i - 1024];
            sts32(smem, static_cast<uint32_t>(i * 4), v);
        }
    }
    __device__ __forceinline__ uint32_t lookup(int t, uint32_t s, int b) const {
        return lds32(smem, (byte_of(s, b) << 2) + 1024u * t);
    }
    __device__ __forceinline__ uint32_t final_word(uint32_t s, int b) const {
        return lds32(smem, (byte_of(s, b) << 2) + (DIR == kEncrypt ? 0u : 4096u));
    }
};

template <int DIR> struct Tab<kLayoutConst, DIR> {
    static constexpr int kFinalByte = DIR == kEncrypt ? 1 : 0;
    __device__ Tab(const uint8_t *, uint32_t) {}
    __device__ static void fill(uint8_t *, int, int) {}
    __device__ __forceinline__ uint32_t lookup(int t, uint32_t s, int b) const {
        return DIR == kEncrypt ? c_tab.te[t][byte_of(s, b)] : c_tab.td[t][byte_of(s, b)];
    }
    __device__ __forceinline__ uint32_t final_word(uint32_t s, int b) const {
        return DIR == kEncrypt ? c_tab.te[0][byte_of(s, b)] : c_tab.is[byte_of(s, b)];
    }
};

template <int DIR> struct Tab<kLayoutReg, DIR> {
    static constexpr int kFinalByte = DIR == kEncrypt ? 1 : 0;
    uint32_t t[8];   // T0[lane + 32j] (D0 for decryption)
    uint32_t is[2];  // decryption: InvS bytes 4w..4w+3, w = lane + 32j, byte k at bits 8k..8k+7
    __device__ Tab(const uint8_t *, uint32_t lane) {
#pragma unroll
        for (int j = 0; j < 8; ++j) t[j] = g_fill.t0[DIR][lane + 32 * j];
#pragma unroll
        for (int j = 0; j < 2; ++j) is[j] = DIR == kEncrypt ? 0u : g_fill.is4[lane + 32 * j];
    }
    __device__ static void fill(uint8_t *, int, int) {}
    // T0[x]: every lane of the warp calls this together (full-warp shuffles)
    __device__ __forceinline__ uint32_t get(uint32_t x) const {
        const int src = static_cast<int>(x & 31u);
        uint32_t v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __shfl_sync(0xffffffffu, t[j], src);
        const bool b5 = (x & 32u) != 0u, b6 = (x & 64u) != 0u, b7 = (x & 128u) != 0u;
        const uint32_t a0 = b5 ? v[1] : v[0], a1 = b5 ? v[3] : v[2], a2 = b5 ? v[5] : v[4], a3 = b5 ? v[7] : v[6];
        const uint32_t c0 = b6 ? a1 : a0, c1 = b6 ? a3 : a2;
        return b7 ? c1 : c0;
    }
    __device__ __forceinline__ uint32_t lookup(int t_, uint32_t s, int b) const {
        return rotl32(get(byte_of(s, b)), 8 * t_);
    }
    __device__ __forceinline__ uint32_t final_word(uint32_t s, int b) const {
        const uint32_t x = byte_of(s, b);
        if (DIR == kEncrypt) return get(x);
        const uint32_t w = x >> 2;
        const uint32_t v0 = __shfl_sync(0xffffffffu, is[0], static_cast<int>(w & 31u));
        const uint32_t v1 = __shfl_sync(0xffffffffu, is[1], static_cast<int>(w & 31u));
        return ((w & 32u) ? v1 : v0) >> (8u * (x & 3u));
    }
};

// ---------------------------------------------------------------------------
// Rounds
// ---------------------------------------------------------------------------

// Whether a layout keeps only T0 and T1 (T2, T3 are then their 16-bit rotations).
template <class TabT, class = void> struct PairRotate { static constexpr bool value = false; };
template <class TabT> struct PairRotate<TabT, decltype(void(TabT::kPairRotate))> {
    static constexpr bool value = TabT::kPairRotate;
};
template <class TabT> __device__ constexpr bool pair_rotate() { return PairRotate<TabT>::value; }

// Column of the input state whose row-r byte feeds output column j.
template <int DIR> __device__ constexpr int src_col(int j, int r) {
    return DIR == kEncrypt ? ((j + r) & 3) : ((j - r + 4) & 3);
}

// eq (26): one full round (SubBytes, ShiftRows, MixColumns, AddRoundKey or the
// inverse-cipher equivalents) on one state.
template <int DIR, class TabT, class Key>
__device__ __forceinline__ void full_round(const TabT &tab, uint32_t (&s)[4], const Key &k, int kw) {
    uint32_t t[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t l0 = tab.lookup(0, s[src_col<DIR>(j, 0)], 0), l1 = tab.lookup(1, s[src_col<DIR>(j, 1)], 1);
        const uint32_t l2 = tab.lookup(2, s[src_col<DIR>(j, 2)], 2), l3 = tab.lookup(3, s[src_col<DIR>(j, 3)], 3);
        if constexpr (pair_rotate<TabT>()) {
            const uint32_t kw16 = __byte_perm(k(kw + j), 0u, 0x1032u);  // rotr16 (= rotl16) of the key word
            t[j] = l0 ^ l1 ^ __byte_perm(l2 ^ l3 ^ kw16, 0u, 0x1032u);
        } else {
            t[j] = (l0 ^ l1) ^ (l2 ^ l3) ^ k(kw + j);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = t[j];
}

// Final round: (Inv)SubBytes + (Inv)ShiftRows + AddRoundKey, no MixColumns.
template <int DIR, class TabT, class Key>
__device__ __forceinline__ void final_round(const TabT &tab, uint32_t (&s)[4], const Key &k, int kw) {
    constexpr uint32_t fb = TabT::kFinalByte;
    constexpr uint32_t sel_lo = ((4u + fb) << 4) | fb;           // bytes 0,1 <- w0.fb, w1.fb
    constexpr uint32_t sel_hi = ((4u + fb) << 12) | (fb << 8);   // bytes 2,3 <- w2.fb, w3.fb
    uint32_t t[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t w0 = tab.final_word(s[src_col<DIR>(j, 0)], 0);
        const uint32_t w1 = tab.final_word(s[src_col<DIR>(j, 1)], 1);
        const uint32_t w2 = tab.final_word(s[src_col<DIR>(j, 2)], 2);
        const uint32_t w3 = tab.final_word(s[src_col<DIR>(j, 3)], 3);
        const uint32_t lo = __byte_perm(w0, w1, sel_lo);
        const uint32_t hi = __byte_perm(w2, w3, sel_hi);
        t[j] = __byte_perm(lo, hi, 0x7610u) ^ k(kw + j);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = t[j];
}

// Key accessor over the kernel-parameter round keys (constant bank).
struct ParamKey {
    const uint32_t *w;
    __device__ __forceinline__ uint32_t operator()(int i) const { return w[i]; }
};

// Full cipher (encrypt) or equivalent inverse cipher (decrypt) on NB states.
template <int DIR, int NR, int NB, class TabT, class Key>
__device__ __forceinline__ void cipher_states(const TabT &tab, const Key &k, uint32_t (&s)[NB][4]) {
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) s[i][j] ^= k(j);
#pragma unroll
    for (int r = 1; r < NR; ++r)
#pragma unroll
        for (int i = 0; i < NB; ++i) full_round<DIR>(tab, s[i], k, 4 * r);
#pragma unroll
    for (int i = 0; i < NB; ++i) final_round<DIR>(tab, s[i], k, 4 * NR);
}

// Programmatic dependent launch.  The host launches the single-buffer kernels
// with programmatic stream serialisation (launch_pdl), so a kernel may start
// -- fill its tables, which reads only constant memory -- while the previous
// kernel in the stream is still draining.  griddep_wait() returns once that
// kernel has completed and its writes are visible; every global load or store
// comes after it.  griddep_release() lets the next such kernel start early.
// Both are no-ops in a launch without the attribute.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint4 ld_block(const uint4 *p) { return __ldcs(p); }
__device__ __forceinline__ void st_block(uint4 *p, uint4 v) { __stcs(p, v); }

// ---------------------------------------------------------------------------
// Single-buffer ECB kernel (persistent).  A warp's unit of work is 32*NB
// consecutive blocks, lane l taking blocks base + l + 32*i, so every
// warp-wide 128-bit load/store covers 512 contiguous bytes; the next unit's
// blocks are loaded before the current ones are ciphered.  Units are assigned
// in one of two ways, decided per launch (the same in every warp):
//  * at most a.even_split_units units per warp: warp w of W takes the
//    contiguous units [w*U/W, (w+1)*U/W), so every CTA gets the same work
//    within one unit per warp and no launch ends on a partly filled pass.  The
//    host asks for it only when one CTA per SM is all that fits, so that every
//    SM holds one CTA of the launch and the shares are per SM too;
//  * otherwise grid-stride passes: warp w takes units w, w + W, w + 2W, ...,
//    so the grid sweeps the buffer front to back (at most one pass of
//    imbalance among many); with several CTAs per SM, CTAs that finish a pass
//    early free their slots for the next launch's CTAs.
// ---------------------------------------------------------------------------
template <int DIR, int NR, int NB, int LAYOUT>
__global__ void __launch_bounds__(max_threads_for(NB, LAYOUT), 1)
    ecb_kernel(const __grid_constant__ EcbArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t lane = threadIdx.x & 31u;
    const unsigned long long wpc = blockDim.x >> 5;
    const unsigned long long W = static_cast<unsigned long long>(gridDim.x) * wpc;
    const unsigned long long w = blockIdx.x * wpc + (threadIdx.x >> 5);
    const unsigned long long U = (a.nblocks + 32ull * NB - 1) / (32ull * NB);
    unsigned long long base, step, n;  // blocks base, base + step, ... below n
    if (U <= a.even_split_units * W) {
        const unsigned long long u1 = (w + 1) * U / W;
        base = w * U / W * 32ull * NB;
        step = 32ull * NB;
        n = u1 * 32ull * NB < a.nblocks ? u1 * 32ull * NB : a.nblocks;
    } else {
        base = w * 32ull * NB;
        step = W * 32ull * NB;
        n = a.nblocks;
    }

    Tab<LAYOUT, DIR>::fill(smem, threadIdx.x, blockDim.x);
    __syncthreads();
    griddep_release();
    griddep_wait();

    uint4 cur[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const unsigned long long b = base + lane + 32ull * i;
        cur[i] = b < n ? ld_block(a.in + b) : make_uint4(0, 0, 0, 0);
    }

    const Tab<LAYOUT, DIR> tab(smem, lane);
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
        for (int i = 0; i < NB; ++i) {
            s[i][0] = cur[i].x; s[i][1] = cur[i].y; s[i][2] = cur[i].z; s[i][3] = cur[i].w;
        }
        cipher_states<DIR, NR, NB>(tab, key, s);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const unsigned long long b = base + lane + 32ull * i;
            if (b < n) st_block(a.out + b, make_uint4(s[i][0], s[i][1], s[i][2], s[i][3]));
            cur[i] = nxt[i];
        }
    }
}

}  // namespace aesgb
