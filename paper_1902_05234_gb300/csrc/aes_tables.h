// aes_tables.h -- compile-time AES tables for the GPU library.
//
// Everything here is constexpr C++17 evaluated by the compiler, so the tables
// exist as initialised data in the host library and in each kernel module's
// __constant__ bank; nothing is computed or uploaded at run time.
//
// GF(2^8) (Wang & Chu section 3.2.1, Defs. 1-3, m(x) = x^8+x^4+x^3+x+1 of eq (8))
// is built from exponent/logarithm tables of the generator 03: 03^i is formed
// by repeated multiplication by x+1, i.e. a ^ xtime(a) (Def. 3).  The S-box
// (Def. 4; values per FIPS-197 5.1.1, which the paper cites but does not
// print) is the inverse 03^(255 - log a) followed by the affine map in its
// rotate-and-XOR form s = b ^ rotl(b,1) ^ rotl(b,2) ^ rotl(b,3) ^ rotl(b,4) ^ 0x63.
//
// Word packing used by every kernel: byte r of a 32-bit word (bits 8r..8r+7)
// is row r of a state column, so a little-endian load of in[4c..4c+3] gives
// column c (state s[r][c] = in[r + 4c]).
//
//   te0[x] = column (02 S(x), S(x), S(x), 03 S(x))            eq (22); T_k = rotl(te0, 8k), eqs (23)-(25)
//   td0[x] = column (0e IS(x), 09 IS(x), 0d IS(x), 0b IS(x))   decryption analogue (FIPS-197 5.3.3 matrix)
#pragma once
#include <cstdint>

namespace aesgb {

struct GfTables {
    uint8_t exp[256];  // exp[i] = 03^i, exp[255] = exp[0]
    uint8_t log[256];  // log[exp[i]] = i, log[0] unused
};

constexpr uint8_t xtime_c(uint8_t a) {
    return static_cast<uint8_t>((a << 1) ^ ((a & 0x80) ? 0x1b : 0x00));
}

constexpr GfTables make_gf() {
    GfTables g{};
    uint8_t a = 1;
    for (int i = 0; i < 255; ++i) {
        g.exp[i] = a;
        g.log[a] = static_cast<uint8_t>(i);
        a = static_cast<uint8_t>(a ^ xtime_c(a));  // a * 03
    }
    g.exp[255] = g.exp[0];
    return g;
}

inline constexpr GfTables kGf = make_gf();

constexpr uint8_t gmul_c(uint8_t a, uint8_t b) {
    if (a == 0 || b == 0) return 0;
    return kGf.exp[(kGf.log[a] + kGf.log[b]) % 255];
}

constexpr uint8_t ginv_c(uint8_t a) { return a == 0 ? 0 : kGf.exp[(255 - kGf.log[a]) % 255]; }

constexpr uint8_t rotl8_c(uint8_t b, int n) {
    return static_cast<uint8_t>((b << n) | (b >> (8 - n)));
}

struct AesTables {
    uint8_t sbox[256];
    uint8_t isbox[256];
    uint32_t te0[256];
    uint32_t td0[256];
};

constexpr uint32_t pack4(uint8_t r0, uint8_t r1, uint8_t r2, uint8_t r3) {
    return static_cast<uint32_t>(r0) | (static_cast<uint32_t>(r1) << 8) |
           (static_cast<uint32_t>(r2) << 16) | (static_cast<uint32_t>(r3) << 24);
}

constexpr AesTables make_aes_tables() {
    AesTables t{};
    for (int x = 0; x < 256; ++x) {
        const uint8_t b = ginv_c(static_cast<uint8_t>(x));
        const uint8_t s = static_cast<uint8_t>(b ^ rotl8_c(b, 1) ^ rotl8_c(b, 2) ^
                                               rotl8_c(b, 3) ^ rotl8_c(b, 4) ^ 0x63);
        t.sbox[x] = s;
        t.isbox[s] = static_cast<uint8_t>(x);
    }
    for (int x = 0; x < 256; ++x) {
        const uint8_t s = t.sbox[x], is = t.isbox[x];
        t.te0[x] = pack4(gmul_c(s, 2), s, s, gmul_c(s, 3));
        t.td0[x] = pack4(gmul_c(is, 0x0e), gmul_c(is, 0x09), gmul_c(is, 0x0d), gmul_c(is, 0x0b));
    }
    return t;
}

inline constexpr AesTables kAes = make_aes_tables();

// Tables as the kernels read them from constant memory: the four rotations of
// te0 and td0, and the inverse S-box in byte 0 of a word.
struct ConstTables {
    uint32_t te[4][256];
    uint32_t td[4][256];
    uint32_t is[256];
};

constexpr uint32_t rotl32_c(uint32_t v, int n) { return n == 0 ? v : (v << n) | (v >> (32 - n)); }

constexpr ConstTables make_const_tables() {
    ConstTables c{};
    for (int x = 0; x < 256; ++x) {
        for (int k = 0; k < 4; ++k) {
            c.te[k][x] = rotl32_c(kAes.te0[x], 8 * k);
            c.td[k][x] = rotl32_c(kAes.td0[x], 8 * k);
        }
        c.is[x] = kAes.isbox[x];
    }
    return c;
}

// Compile-time sanity anchors taken from the field's definition: 03 generates
// all 255 nonzero elements, and the affine map sends the inverse of 0 (0) to 0x63.
static_assert(kGf.exp[254] != 1 && kGf.exp[255] == 1, "03 must have order 255");
static_assert(kAes.sbox[0] == 0x63, "S(0) is the affine constant");

}  // namespace aesgb
