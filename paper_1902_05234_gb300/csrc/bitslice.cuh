// bitslice.cuh -- constant-time (table-free) AES on bit planes.
//
// 32 blocks are processed together: word W[c][p] holds, in bit j, bit p of
// column c of block j (p = 8 r + b: row r, bit b of the byte).  Every step of
// a round is then a fixed sequence of logic operations on these words, with no
// memory access that depends on data -- the side channel the paper's remark on
// xtime and power analysis (section 3.2.1, Def. 3) is about.  The logic comes
// from the generated circuits of bitslice_circuits.h (see gen_bitslice.py),
// each gate one LOP3:
//   encryption round  S-box circuit per byte (the round key enters as the
//                     circuit's output mask), ShiftRows as a permutation of
//                     registers, MixColumns circuit per column;
//   decryption round  InvShiftRows as a permutation, the inverse S-box's
//                     nonlinear core per byte, then one circuit per column for
//                     InvMixColumns of the S-box outputs plus the round key.
// Round keys reach the circuits as mask planes (all-zero or all-one words)
// that the host derives from the schedule (see ct.cu): a key byte m wanted at
// an S-box output enters the S-box's product chains as mu = OUT^-1 m, so it
// costs no gate.  The functions are
// __host__ __device__ so the same code runs in the host self-test.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

#include "bitslice_circuits.h"
#include "bitslice_math.h"

#if defined(__CUDACC__)
#define AESGB_HD __host__ __device__ __forceinline__
#else
#define AESGB_HD inline
#endif

namespace aesgb {
namespace bs {

// d = f(a, b, c) for the 3-input function whose truth table is LUT (LOP3
// convention: bit p of LUT is f at a = bit p of 0xF0, b of 0xCC, c of 0xAA).
constexpr uint32_t lop3_value(uint8_t lut, uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d = 0;
    for (int p = 0; p < 8; ++p)
        if ((lut >> p) & 1)
            d |= (((0xF0 >> p) & 1) ? a : ~a) & (((0xCC >> p) & 1) ? b : ~b) & (((0xAA >> p) & 1) ? c : ~c);
    return d;
}

template <uint8_t LUT>
AESGB_HD uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
#else
    return lop3_value(LUT, a, b, c);
#endif
}

// ------------------------------------------------------ circuit execution
// v[0..kIn) are the inputs; gate g writes v[kIn + g].  The gate list is a
// compile-time table, so each gate becomes one instruction on registers.
template <const auto &C, std::size_t G>
AESGB_HD void run_gate(uint32_t *v) {
    constexpr uint8_t lut = C.g[G].lut;
    constexpr int a = C.g[G].a, b = C.g[G].b, c = C.g[G].c, d = C.kIn + static_cast<int>(G);
    v[d] = lop3<lut>(v[a], v[b], v[c]);
}

template <const auto &C, std::size_t... G>
AESGB_HD void run_gates(uint32_t *v, std::index_sequence<G...>) {
    (run_gate<C, G>(v), ...);
}

template <const auto &C, std::size_t O>
AESGB_HD void take_out(const uint32_t *v, uint32_t *out) {
    constexpr int i = C.out[O];
    out[O] = v[i];
}

template <const auto &C, std::size_t... O>
AESGB_HD void take_outs(const uint32_t *v, uint32_t *out, std::index_sequence<O...>) {
    (take_out<C, O>(v, out), ...);
}

// out[0..kOut) = C(in[0..kIn)); out may alias in.
template <const auto &C>
AESGB_HD void run(const uint32_t *in, uint32_t *out) {
    using Circ = std::remove_cv_t<std::remove_reference_t<decltype(C)>>;
    uint32_t v[Circ::kIn + Circ::kGates];
#pragma unroll
    for (int i = 0; i < Circ::kIn; ++i) v[i] = in[i];
    run_gates<C>(v, std::make_index_sequence<Circ::kGates>{});
    take_outs<C>(v, out, std::make_index_sequence<Circ::kOut>{});
}

// ------------------------------------------ compile-time checks of the tables
// Each check evaluates a circuit on 32 cases at once (bit t of every word is
// case t) against the AES definitions in aes_tables.h / bitslice_math.h.
template <class Circ>
constexpr void eval_cx(const Circ &C, const uint32_t *in, uint32_t *out) {
    uint32_t v[Circ::kIn + Circ::kGates]{};
    for (int i = 0; i < Circ::kIn; ++i) v[i] = in[i];
    for (int g = 0; g < Circ::kGates; ++g)
        v[Circ::kIn + g] = lop3_value(C.g[g].lut, v[C.g[g].a], v[C.g[g].b], v[C.g[g].c]);
    for (int o = 0; o < Circ::kOut; ++o) out[o] = v[C.out[o]];
}

constexpr uint8_t test_mask(int t, int k) { return static_cast<uint8_t>((t * 29 + k * 113 + 7) ^ (t >> 3)); }

// mu = OUT^-1 m for the generated row masks (bit i = parity of row i & m).
constexpr uint8_t apply_rows(const uint8_t (&rows)[8], uint8_t m) {
    uint8_t r = 0;
    for (int i = 0; i < 8; ++i) {
        uint8_t v = static_cast<uint8_t>(rows[i] & m), p = 0;
        for (; v; v = static_cast<uint8_t>(v & (v - 1))) p ^= 1;
        r |= static_cast<uint8_t>(p << i);
    }
    return r;
}

template <int N>
constexpr void to_planes(const uint8_t (&val)[32], uint32_t *planes) {
    for (int b = 0; b < N; ++b) {
        uint32_t w = 0;
        for (int t = 0; t < 32; ++t) w |= static_cast<uint32_t>((val[t] >> b) & 1) << t;
        planes[b] = w;
    }
}
constexpr uint8_t byte_of_planes(const uint32_t *planes, int t) {
    uint8_t v = 0;
    for (int b = 0; b < 8; ++b) v |= static_cast<uint8_t>(((planes[b] >> t) & 1) << b);
    return v;
}

constexpr bool check_sbox_circuits() {
    for (int base = 0; base < 256; base += 32) {
        uint8_t x[32]{}, m[32]{}, mue[32]{}, mud[32]{};
        for (int t = 0; t < 32; ++t) {
            x[t] = static_cast<uint8_t>(base + t);
            m[t] = test_mask(base + t, 0);
            mue[t] = apply_rows(bsc::k_mu_enc, m[t]);
            mud[t] = apply_rows(bsc::k_mu_dec, m[t]);
        }
        uint32_t in[16]{}, y[8]{}, o[8]{};
        to_planes<8>(x, in);
        to_planes<8>(mue, in + 8);
        eval_cx(bsc::k_sbox_enc, in, y);  // S(x) + 63 + m
        for (int t = 0; t < 32; ++t)
            if (byte_of_planes(y, t) != static_cast<uint8_t>(kAes.sbox[x[t]] ^ 0x63 ^ m[t])) return false;
        to_planes<8>(mud, in + 8);
        eval_cx(bsc::k_sbox_core_dec, in, o);
        eval_cx(bsc::k_sbox_out_dec, o, y);  // S^-1(x) + m
        for (int t = 0; t < 32; ++t)
            if (byte_of_planes(y, t) != static_cast<uint8_t>(kAes.isbox[x[t]] ^ m[t])) return false;
    }
    return true;
}

// inv_mix_out is linear in the four bytes' core outputs, each the S-box core
// of its own byte plus its own key's mu: checked on the 1,024 columns with one
// varying byte (the others zero), every byte with its own key.
constexpr bool check_inv_mix_circuit() {
    for (int r0 = 0; r0 < 4; ++r0)
        for (int base = 0; base < 256; base += 32) {
            uint32_t in[32]{}, out[32]{};
            for (int r = 0; r < 4; ++r) {
                uint8_t x[32]{}, mu[32]{};
                for (int t = 0; t < 32; ++t) {
                    x[t] = r == r0 ? static_cast<uint8_t>(base + t) : 0;
                    mu[t] = apply_rows(bsc::k_mu_dec, test_mask(base + t, r0 * 4 + r));
                }
                uint32_t xp[16]{};
                to_planes<8>(x, xp);
                to_planes<8>(mu, xp + 8);
                eval_cx(bsc::k_sbox_core_dec, xp, in + 8 * r);
            }
            eval_cx(bsc::k_inv_mix_out, in, out);
            for (int t = 0; t < 32; ++t) {
                uint8_t s[4]{};
                for (int r = 0; r < 4; ++r)
                    s[r] = static_cast<uint8_t>(kAes.isbox[r == r0 ? base + t : 0] ^ test_mask(base + t, r0 * 4 + r));
                const uint32_t want = bsmath::inv_mix_column_model(pack4(s[0], s[1], s[2], s[3]));
                for (int r = 0; r < 4; ++r)
                    if (byte_of_planes(out + 8 * r, t) != static_cast<uint8_t>(want >> (8 * r))) return false;
            }
        }
    return true;
}

// mix_columns is linear: the 32 unit columns decide it (case t = unit vector t).
constexpr bool check_mix_circuit() {
    uint32_t in[32]{}, out[32]{};
    for (int j = 0; j < 32; ++j) in[j] = 1u << j;
    eval_cx(bsc::k_mix_columns, in, out);
    for (int t = 0; t < 32; ++t) {
        const uint32_t want = bsmath::mix_column_model(1u << t);
        for (int p = 0; p < 32; ++p)
            if (((out[p] >> t) & 1) != ((want >> p) & 1)) return false;
    }
    return true;
}

static_assert(check_sbox_circuits(), "S-box / inverse S-box circuits");
static_assert(check_inv_mix_circuit(), "InvMixColumns output circuit");
static_assert(check_mix_circuit(), "MixColumns circuit");

// ------------------------------------------------------- rounds on planes
// State: W[c][8 r + b] = plane (row r, column c, bit b).
struct Planes {
    uint32_t w[4][32];
};

// Key planes of one step, in the state's layout: the key itself for step 0,
// the mu planes (see ct.cu) for the rounds.
struct RoundMasks {
    uint32_t m[4][32];
};

AESGB_HD void add_masks(Planes &s, const RoundMasks &k) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int p = 0; p < 32; ++p) s.w[c][p] ^= k.m[c][p];
}

// Row r rotated left by r columns (ShiftRows, eq (19)) or right (inverse).
template <int DIR>
AESGB_HD void shift_rows(Planes &s) {
#pragma unroll
    for (int r = 1; r < 4; ++r)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            uint32_t t[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) t[c] = s.w[DIR == 0 ? (c + r) & 3 : (c - r + 4) & 3][8 * r + b];
#pragma unroll
            for (int c = 0; c < 4; ++c) s.w[c][8 * r + b] = t[c];
        }
}

// Encryption round: SubBytes with the folded key (as mu planes), ShiftRows,
// and MixColumns unless it is the last round.
template <bool MIX>
AESGB_HD void enc_round(Planes &s, const RoundMasks &k) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int r = q & 3, c = q >> 2;
        uint32_t in[16];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            in[b] = s.w[c][8 * r + b];
            in[8 + b] = k.m[c][8 * r + b];
        }
        run<bsc::k_sbox_enc>(in, &s.w[c][8 * r]);
    }
    shift_rows<0>(s);
    if (MIX)
#pragma unroll
        for (int c = 0; c < 4; ++c) run<bsc::k_mix_columns>(s.w[c], s.w[c]);
}

// Decryption round: InvShiftRows, InvSubBytes, AddRoundKey and (unless it is
// the last round) InvMixColumns, the last three per column: the S-box cores
// take the key as mu planes, one circuit maps the column's four cores through
// the S-box output map and InvMixColumns.
template <bool MIX>
AESGB_HD void dec_round(Planes &s, const RoundMasks &k) {
    shift_rows<1>(s);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t o[32];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            uint32_t in[16];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                in[b] = s.w[c][8 * r + b];
                in[8 + b] = k.m[c][8 * r + b];
            }
            run<bsc::k_sbox_core_dec>(in, &o[8 * r]);
        }
        if (MIX) {
            run<bsc::k_inv_mix_out>(o, s.w[c]);
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) run<bsc::k_sbox_out_dec>(&o[8 * r], &s.w[c][8 * r]);
        }
    }
}

// The whole cipher on one 32-block plane set.  masks[0] is added first, then
// round i = 1..nr uses masks[i] (host-built, see ct.cu).
template <int DIR>
AESGB_HD void cipher_planes(Planes &s, const RoundMasks *masks, int nr) {
    add_masks(s, masks[0]);
#pragma unroll 1
    for (int i = 1; i < nr; ++i) {
        if (DIR == 0) enc_round<true>(s, masks[i]);
        else dec_round<true>(s, masks[i]);
    }
    if (DIR == 0) enc_round<false>(s, masks[nr]);
    else dec_round<false>(s, masks[nr]);
}

// In-place transpose of a 32x32 bit matrix: afterwards bit j of a[i] is the
// old bit i of a[j].  Five stages swap blocks of 16, 8, 4, 2, 1 bits between
// words 16, 8, 4, 2, 1 apart; the 16- and 8-bit stages are byte permutes, the
// others one shift (as a multiplication) and one bit-select per word.
AESGB_HD uint32_t byte_perm(uint32_t x, uint32_t y, uint32_t sel) {
#if defined(__CUDA_ARCH__)
    return __byte_perm(x, y, sel);
#else
    const uint64_t v = (static_cast<uint64_t>(y) << 32) | x;
    uint32_t r = 0;
    for (int i = 0; i < 4; ++i) r |= static_cast<uint32_t>((v >> (8 * ((sel >> (4 * i)) & 7))) & 0xFF) << (8 * i);
    return r;
#endif
}

// x << s and x >> s (0 < s < 32) as multiplications, which the GPU runs on its
// multiply-add pipe rather than the integer-logic pipe that the circuits keep
// busy: x * 2^s keeps the low word, the high word of x * 2^(32-s) is x >> s.
AESGB_HD uint32_t shl_mul(uint32_t x, int s) {
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("mul.lo.u32 %0, %1, %2;" : "=r"(d) : "r"(x), "r"(1u << s));
    return d;
#else
    return x << s;
#endif
}
AESGB_HD uint32_t shr_mul(uint32_t x, int s) {
#if defined(__CUDA_ARCH__)
    return __umulhi(x, 1u << (32 - s));
#else
    return x >> s;
#endif
}

AESGB_HD void transpose32(uint32_t *a) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t x = a[k], y = a[k + 16];
        a[k] = byte_perm(x, y, 0x5410u);
        a[k + 16] = byte_perm(x, y, 0x7632u);
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if (k & 8) continue;
        const uint32_t x = a[k], y = a[k + 8];
        a[k] = byte_perm(x, y, 0x6240u);
        a[k + 8] = byte_perm(x, y, 0x7351u);
    }
    uint32_t m = 0x0F0F0F0Fu;
#pragma unroll
    for (int s = 4; s > 0; s >>= 1, m ^= (m << s)) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if (k & s) continue;  // k runs over the words whose partner is k + s
            const uint32_t x = a[k], y = a[k + s];
            a[k] = lop3<0xD8>(x, shl_mul(y, s), ~m);     // ~m ? (y << s) : x
            a[k + s] = lop3<0xD8>(y, shr_mul(x, s), m);  //  m ? (x >> s) : y
        }
    }
}

}  // namespace bs
}  // namespace aesgb
