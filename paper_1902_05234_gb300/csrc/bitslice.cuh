// bitslice.cuh -- constant-time (table-free) AES on bit planes.
//
// 32 blocks are processed together: word W[c][p] holds, in bit j, bit p of
// column c of block j (p = 8 r + b: row r, bit b of the byte).  Every step of
// a round is then a fixed sequence of logic operations on these words, with no
// memory access that depends on data -- the side channel the paper's remark on
// xtime and power analysis (section 3.2.1, Def. 3) is about:
//   SubBytes    the tower-field circuit of bitslice_math.h on each byte's 8
//               planes; round keys are added inside its linear input / output
//               maps as all-zero / all-one mask planes;
//   ShiftRows   a permutation of plane registers (data moves only);
//   MixColumns  eq (20) with xtime on planes (a shift of plane indices plus
//               XORs into planes 1, 3, 4); InvMixColumns = MixColumns after a
//               cheap pre-step (see bitslice_math.h).
// The functions are __host__ __device__ so the same code runs in the host
// self-test.
#pragma once

#include <cstdint>

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
template <uint8_t LUT>
AESGB_HD uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
#else
    uint32_t d = 0;
    for (int p = 0; p < 8; ++p)
        if ((LUT >> p) & 1)
            d |= (((0xF0 >> p) & 1) ? a : ~a) & (((0xCC >> p) & 1) ? b : ~b) & (((0xAA >> p) & 1) ? c : ~c);
    return d;
#endif
}

// ------------------------------------------------------------ linear maps
enum MatId : int { kEncIn = 0, kEncOut = 1, kDecIn = 2, kDecOut = 3, kLinDelta = 4 };

AESGB_CX_HD bsmath::Mat8 mat_of(int id) {
    return id == kEncIn    ? bsmath::kMaps.enc_in
           : id == kEncOut ? bsmath::kMaps.enc_out
           : id == kDecIn  ? bsmath::kMaps.dec_in
           : id == kDecOut ? bsmath::kMaps.dec_out
                           : bsmath::kMaps.lin_delta;
}

// Each map y = M x is evaluated as a straight-line XOR program with shared
// subexpressions, found at compile time by repeatedly naming the pair of
// variables that occurs together in the most rows (variable 8 + k =
// v[a[k]] ^ v[b[k]]); row i is then the XOR of the variables in rows[i].
struct XorProg {
    int nnew;
    int a[24], b[24];
    uint32_t rows[8];  // bit j: variable j (0..7 inputs, 8.. shared pairs)
};

AESGB_CX_HD XorProg make_prog(const bsmath::Mat8 &m) {
    XorProg p{};
    for (int i = 0; i < 8; ++i) p.rows[i] = m.row[i];
    int nv = 8;
    while (p.nnew < 24) {
        int bi = -1, bj = -1, best = 1;
        for (int i = 0; i < nv; ++i)
            for (int j = i + 1; j < nv; ++j) {
                int cnt = 0;
                for (int r = 0; r < 8; ++r) cnt += ((p.rows[r] >> i) & 1) && ((p.rows[r] >> j) & 1);
                if (cnt > best) { best = cnt; bi = i; bj = j; }
            }
        if (bi < 0) break;
        p.a[p.nnew] = bi;
        p.b[p.nnew] = bj;
        for (int r = 0; r < 8; ++r)
            if (((p.rows[r] >> bi) & 1) && ((p.rows[r] >> bj) & 1))
                p.rows[r] = (p.rows[r] & ~((1u << bi) | (1u << bj))) | (1u << nv);
        ++nv;
        ++p.nnew;
    }
    return p;
}

AESGB_CX_HD XorProg prog_of(int id) { return make_prog(mat_of(id)); }

template <int ID, int K = 0>
AESGB_HD void prog_vars(uint32_t (&v)[32]) {
    if constexpr (K < prog_of(ID).nnew) {
        constexpr int ia = prog_of(ID).a[K], ib = prog_of(ID).b[K];
        v[8 + K] = v[ia] ^ v[ib];
        prog_vars<ID, K + 1>(v);
    }
}

template <int ID, int I, int J = 0>
AESGB_HD uint32_t prog_row(const uint32_t (&v)[32]) {
    if constexpr (J == 32) {
        return 0u;
    } else if constexpr (((prog_of(ID).rows[I] >> J) & 1) != 0) {
        return v[J] ^ prog_row<ID, I, J + 1>(v);
    } else {
        return prog_row<ID, I, J + 1>(v);
    }
}

// y = M x + k  (k: mask planes, all-zero or all-one words)
template <int ID>
AESGB_HD void matvec(const uint32_t (&x)[8], const uint32_t (&k)[8], uint32_t (&y)[8]) {
    uint32_t v[32];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = x[i];
    prog_vars<ID>(v);
    y[0] = prog_row<ID, 0>(v) ^ k[0];
    y[1] = prog_row<ID, 1>(v) ^ k[1];
    y[2] = prog_row<ID, 2>(v) ^ k[2];
    y[3] = prog_row<ID, 3>(v) ^ k[3];
    y[4] = prog_row<ID, 4>(v) ^ k[4];
    y[5] = prog_row<ID, 5>(v) ^ k[5];
    y[6] = prog_row<ID, 6>(v) ^ k[6];
    y[7] = prog_row<ID, 7>(v) ^ k[7];
}

// ----------------------------------------------------------------- GF(16)
AESGB_HD void g16_mul(const uint32_t *a, const uint32_t *b, uint32_t *c) {
    const uint32_t p0 = a[0] & b[0];
    const uint32_t p1 = (a[0] & b[1]) ^ (a[1] & b[0]);
    const uint32_t p2 = (a[0] & b[2]) ^ (a[1] & b[1]) ^ (a[2] & b[0]);
    const uint32_t p3 = (a[0] & b[3]) ^ (a[1] & b[2]) ^ (a[2] & b[1]) ^ (a[3] & b[0]);
    const uint32_t p4 = (a[1] & b[3]) ^ (a[2] & b[2]) ^ (a[3] & b[1]);
    const uint32_t p5 = (a[2] & b[3]) ^ (a[3] & b[2]);
    const uint32_t p6 = a[3] & b[3];
    // z^4 = z + 1, z^5 = z^2 + z, z^6 = z^3 + z^2
    c[0] = p0 ^ p4;
    c[1] = p1 ^ p4 ^ p5;
    c[2] = p2 ^ p5 ^ p6;
    c[3] = p3 ^ p6;
}

AESGB_CX_HD uint8_t half_lut(uint16_t truth, int half) {  // f(x2 x1 x0) for x3 = half
    uint8_t lut = 0;
    #pragma unroll
    for (int p = 0; p < 8; ++p) {
        const int x2 = (0xF0 >> p) & 1, x1 = (0xCC >> p) & 1, x0 = (0xAA >> p) & 1;
        const int x = half * 8 + x2 * 4 + x1 * 2 + x0;
        lut |= static_cast<uint8_t>(((truth >> x) & 1) << p);
    }
    return lut;
}

template <int K>
AESGB_HD uint32_t inv16_bit(const uint32_t *x) {
    constexpr uint16_t T = bsmath::inv16_truth(K);
    const uint32_t lo = lop3<half_lut(T, 0)>(x[2], x[1], x[0]);
    const uint32_t hi = lop3<half_lut(T, 1)>(x[2], x[1], x[0]);
    return lop3<0xD8>(lo, hi, x[3]);  // x3 ? hi : lo
}

AESGB_HD void g16_inv(const uint32_t *x, uint32_t *y) {
    y[0] = inv16_bit<0>(x);
    y[1] = inv16_bit<1>(x);
    y[2] = inv16_bit<2>(x);
    y[3] = inv16_bit<3>(x);
}

// Tower-field inversion: t[0..3] = a0, t[4..7] = a1.
AESGB_HD void tower_inv(const uint32_t (&t)[8], uint32_t (&o)[8]) {
    const uint32_t zero[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t lin[8];
    matvec<kLinDelta>(t, zero, lin);  // lambda a1^2 + a0^2 in lin[0..3]
    uint32_t prod[4], delta[4], d[4], s[4];
    g16_mul(t + 4, t, prod);
    #pragma unroll
    for (int i = 0; i < 4; ++i) delta[i] = lin[i] ^ prod[i];
    g16_inv(delta, d);
    #pragma unroll
    for (int i = 0; i < 4; ++i) s[i] = t[4 + i] ^ t[i];
    g16_mul(t + 4, d, o + 4);
    g16_mul(s, d, o);
}

// One S-box (or inverse S-box) over 32 blocks' byte planes, in place:
// x <- OUT( inv_T( IN x + kin ) ) + kout.
template <int DIR>
AESGB_HD void sbox_planes(uint32_t (&x)[8], const uint32_t (&kin)[8], const uint32_t (&kout)[8]) {
    uint32_t t[8], o[8];
    matvec<DIR == 0 ? kEncIn : kDecIn>(x, kin, t);
    tower_inv(t, o);
    matvec<DIR == 0 ? kEncOut : kDecOut>(o, kout, x);
}

// ------------------------------------------------------- rounds on planes
// State: W[c][8 r + b] = plane (row r, column c, bit b).
struct Planes {
    uint32_t w[4][32];
};

AESGB_HD void xtime_planes(const uint32_t (&u)[8], uint32_t (&x)[8]) {
    x[0] = u[7];
    x[1] = u[0] ^ u[7];
    x[2] = u[1];
    x[3] = u[2] ^ u[7];
    x[4] = u[3] ^ u[7];
    x[5] = u[4];
    x[6] = u[5];
    x[7] = u[6];
}

// MixColumns (eq (20)) on one column: out_r = a_r + t + xtime(a_r + a_{r+1}),
// t = a_0 + a_1 + a_2 + a_3.
AESGB_HD void mix_column(uint32_t *col) {  // col[8 r + b]
    uint32_t t[8], keep0[8];
    #pragma unroll
    for (int b = 0; b < 8; ++b) {
        t[b] = col[b] ^ col[8 + b] ^ col[16 + b] ^ col[24 + b];
        keep0[b] = col[b];
    }
    #pragma unroll
    for (int r = 0; r < 4; ++r) {
        uint32_t u[8], x[8];
        #pragma unroll
        for (int b = 0; b < 8; ++b) u[b] = col[8 * r + b] ^ (r < 3 ? col[8 * (r + 1) + b] : keep0[b]);
        xtime_planes(u, x);
        #pragma unroll
        for (int b = 0; b < 8; ++b) col[8 * r + b] ^= t[b] ^ x[b];
    }
}

// InvMixColumns = MixColumns after a0 += 04(a0 + a2), a2 += same, a1 += 04(a1 + a3), a3 += same.
AESGB_HD void inv_mix_column(uint32_t *col) {
    uint32_t u[8], v[8], x[8], y[8];
    #pragma unroll
    for (int b = 0; b < 8; ++b) {
        u[b] = col[b] ^ col[16 + b];
        v[b] = col[8 + b] ^ col[24 + b];
    }
    xtime_planes(u, x);
    xtime_planes(x, u);
    xtime_planes(v, y);
    xtime_planes(y, v);
    #pragma unroll
    for (int b = 0; b < 8; ++b) {
        col[b] ^= u[b];
        col[16 + b] ^= u[b];
        col[8 + b] ^= v[b];
        col[24 + b] ^= v[b];
    }
    mix_column(col);
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

// Mask planes of one round: m[q][0][b] is added at the S-box input, m[q][1][b]
// at its output, for byte q = r + 4 c.
struct RoundMasks {
    uint32_t m[16][2][8];
};

template <int DIR>
AESGB_HD void sub_bytes(Planes &s, const RoundMasks &k) {
    #pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int r = q & 3, c = q >> 2;
        uint32_t x[8];
        #pragma unroll
        for (int b = 0; b < 8; ++b) x[b] = s.w[c][8 * r + b];
        sbox_planes<DIR>(x, k.m[q][0], k.m[q][1]);
        #pragma unroll
        for (int b = 0; b < 8; ++b) s.w[c][8 * r + b] = x[b];
    }
}

// The whole cipher on one 32-block plane set.  masks[i] is the i-th round's
// masks in application order (host-built, see ct.cu).
template <int DIR>
AESGB_HD void cipher_planes(Planes &s, const RoundMasks *masks, int nr) {
    #pragma unroll
    for (int i = 0; i < nr; ++i) {
        if (DIR == 0) {
            sub_bytes<0>(s, masks[i]);
            shift_rows<0>(s);
            if (i + 1 < nr)
                #pragma unroll
                for (int c = 0; c < 4; ++c) mix_column(s.w[c]);
        } else {
            shift_rows<1>(s);
            sub_bytes<1>(s, masks[i]);
            if (i + 1 < nr)
                #pragma unroll
                for (int c = 0; c < 4; ++c) inv_mix_column(s.w[c]);
        }
    }
}

// In-place transpose of a 32x32 bit matrix: afterwards bit j of a[i] is the
// old bit i of a[j].  Five stages swap blocks of 16, 8, 4, 2, 1 bits between
// words 16, 8, 4, 2, 1 apart; the 16- and 8-bit stages are byte permutes.
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
            const uint32_t t = ((a[k] >> s) ^ a[k + s]) & m;
            a[k + s] ^= t;
            a[k] ^= t << s;
        }
    }
}

}  // namespace bs
}  // namespace aesgb
