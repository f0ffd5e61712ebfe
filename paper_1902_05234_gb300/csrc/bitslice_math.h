// bitslice_math.h -- compile-time derivation of a constant-time AES S-box
// circuit (no table lookups) for the bitsliced kernels.
//
// The S-box (Wang & Chu Def. 4; FIPS-197 5.1.1) is inversion in GF(2^8)
// followed by an affine map.  Inversion is computed in an isomorphic tower
// field GF((2^4)^2) = GF(16)[y] / (y^2 + y + lambda), GF(16) = GF(2)[z] /
// (z^4 + z + 1), where
//     (a1 y + a0)^-1 = (a1 d) y + (a1 + a0) d,   d = (lambda a1^2 + a1 a0 + a0^2)^-1
// (multiplying out with y^2 = y + lambda gives 1), which needs three GF(16)
// multiplications and one GF(16) inversion instead of a GF(2^8) inversion.
// Everything the circuit needs is found here by search at compile time:
//   * lambda: the first element of GF(16) with trace 1 (y^2 + y + lambda is
//     then irreducible);
//   * an isomorphism phi: tower -> AES field, phi(g^k) = beta^k for a
//     primitive tower element g and a root beta, in the AES field, of g's
//     minimal polynomial over GF(2);
//   * the 8x8 GF(2) matrices of phi, its inverse, the affine map and their
//     products: encryption uses  S(x) = A phi(inv_T(phi^-1 x)) + 63,
//     decryption  S^-1(y) = phi(inv_T(phi^-1 A^-1 (y + 63))).
// static_asserts below check the resulting S-box and inverse S-box, byte
// by byte, against the tables derived in aes_tables.h, and the MixColumns
// factorisation used for decryption against the InvMixColumns matrix.
#pragma once
#include <cstdint>

#include "aes_tables.h"

#if defined(__CUDACC__)
#define AESGB_CX_HD __host__ __device__ constexpr  // also evaluated in device code
#else
#define AESGB_CX_HD constexpr
#endif

namespace aesgb {
namespace bsmath {

// ---------------------------------------------------------------- GF(16)
AESGB_CX_HD uint8_t g16_mul(uint8_t a, uint8_t b) {
    uint8_t p = 0;
    for (int i = 0; i < 4; ++i)
        if ((b >> i) & 1) p ^= static_cast<uint8_t>(a << i);
    for (int d = 6; d >= 4; --d)
        if ((p >> d) & 1) p ^= static_cast<uint8_t>(0x13 << (d - 4));  // z^4 = z + 1
    return static_cast<uint8_t>(p & 0xF);
}
AESGB_CX_HD uint8_t g16_pow(uint8_t a, int e) {
    uint8_t r = 1;
    for (int i = 0; i < e; ++i) r = g16_mul(r, a);
    return r;
}
AESGB_CX_HD uint8_t g16_inv(uint8_t a) { return a ? g16_pow(a, 14) : 0; }
constexpr uint8_t g16_trace(uint8_t a) {
    return static_cast<uint8_t>(a ^ g16_mul(a, a) ^ g16_pow(a, 4) ^ g16_pow(a, 8));
}
constexpr uint8_t find_lambda() {
    for (int l = 1; l < 16; ++l)
        if (g16_trace(static_cast<uint8_t>(l)) == 1) return static_cast<uint8_t>(l);
    return 0;
}
inline constexpr uint8_t kLambda = find_lambda();

// ------------------------------------------------------- tower field, bytes
// t = a1 << 4 | a0, element a1 y + a0
constexpr uint8_t tw_mul(uint8_t a, uint8_t b) {
    const uint8_t a1 = a >> 4, a0 = a & 15, b1 = b >> 4, b0 = b & 15;
    const uint8_t h = static_cast<uint8_t>(g16_mul(a1, b1) ^ g16_mul(a1, b0) ^ g16_mul(a0, b1));
    const uint8_t l = static_cast<uint8_t>(g16_mul(g16_mul(a1, b1), kLambda) ^ g16_mul(a0, b0));
    return static_cast<uint8_t>(h << 4 | l);
}
constexpr uint8_t tw_inv(uint8_t a) {
    const uint8_t a1 = a >> 4, a0 = a & 15;
    const uint8_t delta =
        static_cast<uint8_t>(g16_mul(kLambda, g16_mul(a1, a1)) ^ g16_mul(a1, a0) ^ g16_mul(a0, a0));
    const uint8_t d = g16_inv(delta);
    return static_cast<uint8_t>(g16_mul(a1, d) << 4 | g16_mul(static_cast<uint8_t>(a1 ^ a0), d));
}

// ------------------------------------------------------------- AES field
constexpr uint8_t aes_mul(uint8_t a, uint8_t b) { return gmul_c(a, b); }

// --------------------------------------------------------- GF(2) matrices
// row i of a matrix is a byte: output bit i = parity(row[i] & input)
struct Mat8 {
    uint8_t row[8];
};
constexpr uint8_t parity8(uint8_t v) {
    v ^= v >> 4;
    v ^= v >> 2;
    v ^= v >> 1;
    return v & 1;
}
constexpr uint8_t apply(const Mat8 &m, uint8_t x) {
    uint8_t y = 0;
    for (int i = 0; i < 8; ++i) y |= static_cast<uint8_t>(parity8(static_cast<uint8_t>(m.row[i] & x)) << i);
    return y;
}
constexpr Mat8 from_columns(const uint8_t (&col)[8]) {  // column j = image of bit j
    Mat8 m{};
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) m.row[i] |= static_cast<uint8_t>(((col[j] >> i) & 1) << j);
    return m;
}
constexpr Mat8 mat_mul(const Mat8 &a, const Mat8 &b) {  // a * b (b applied first)
    uint8_t col[8]{};
    for (int j = 0; j < 8; ++j) col[j] = apply(a, apply(b, static_cast<uint8_t>(1u << j)));
    return from_columns(col);
}
constexpr Mat8 mat_inv(const Mat8 &m) {  // by the images of all 256 inputs
    uint8_t col[8]{};
    for (int x = 0; x < 256; ++x)
        for (int j = 0; j < 8; ++j)
            if (apply(m, static_cast<uint8_t>(x)) == (1u << j)) col[j] = static_cast<uint8_t>(x);
    return from_columns(col);
}

// The affine map's linear part: b'_i = b_i + b_{i+4} + b_{i+5} + b_{i+6} + b_{i+7}.
constexpr Mat8 affine_matrix() {
    Mat8 m{};
    for (int i = 0; i < 8; ++i)
        for (int k = 0; k < 8; ++k)
            if (k == 0 || k >= 4) m.row[i] |= static_cast<uint8_t>(1u << ((i + k) % 8));
    return m;
}

// ------------------------------------------------------------ isomorphism
constexpr bool tw_is_primitive(uint8_t g) {
    uint8_t x = g;
    for (int k = 1; k < 255; ++k) {
        if (x == 1) return false;
        x = tw_mul(x, g);
    }
    return x == 1;
}
constexpr uint8_t tw_primitive() {
    for (int g = 2; g < 256; ++g)
        if (tw_is_primitive(static_cast<uint8_t>(g))) return static_cast<uint8_t>(g);
    return 0;
}

struct Iso {
    Mat8 t2a;  // tower -> AES
    Mat8 a2t;  // AES -> tower
};

constexpr Iso find_iso() {
    const uint8_t g = tw_primitive();
    // minimal polynomial of g over GF(2): prod over the 8 conjugates g^(2^i),
    // coefficients kept as tower elements (they come out 0 or 1)
    uint8_t poly[9]{};
    poly[0] = 1;
    uint8_t conj = g;
    for (int i = 0; i < 8; ++i) {
        uint8_t next[9]{};
        for (int k = 0; k <= 8; ++k) {
            if (k > 0) next[k] ^= poly[k - 1];         // * x
            next[k] ^= tw_mul(poly[k], conj);            // * conj (minus = plus)
        }
        for (int k = 0; k <= 8; ++k) poly[k] = next[k];
        conj = tw_mul(conj, conj);
    }
    // a root beta of the same polynomial in the AES field
    uint8_t beta = 0;
    for (int b = 2; b < 256 && !beta; ++b) {
        uint8_t acc = 0, p = 1;
        for (int k = 0; k <= 8; ++k) {
            if (poly[k] & 1) acc ^= p;
            p = aes_mul(p, static_cast<uint8_t>(b));
        }
        if (acc == 0) beta = static_cast<uint8_t>(b);
    }
    // phi(g^k) = beta^k; the matrix from the images of the tower basis
    uint8_t col[8]{};
    uint8_t gk = 1, bk = 1;
    for (int k = 0; k < 255; ++k) {
        for (int j = 0; j < 8; ++j)
            if (gk == (1u << j)) col[j] = bk;
        gk = tw_mul(gk, g);
        bk = aes_mul(bk, beta);
    }
    Iso iso{};
    iso.t2a = from_columns(col);
    iso.a2t = mat_inv(iso.t2a);
    return iso;
}
inline constexpr Iso kIso = find_iso();

// ------------------------------------------------ the S-box circuit's maps
struct SboxMaps {
    Mat8 enc_in;     // AES -> tower
    Mat8 enc_out;    // tower -> AES, then the affine map's matrix; constant 0x63
    Mat8 dec_in;     // (AES -> tower) * A^-1; constant dec_in_c
    uint8_t dec_in_c;
    Mat8 dec_out;    // tower -> AES
    Mat8 lin_delta;  // (a1, a0) -> lambda a1^2 + a0^2 (4 output bits used)
};

constexpr SboxMaps make_maps() {
    SboxMaps m{};
    const Mat8 A = affine_matrix();
    const Mat8 Ai = mat_inv(A);
    m.enc_in = kIso.a2t;
    m.enc_out = mat_mul(A, kIso.t2a);
    m.dec_in = mat_mul(kIso.a2t, Ai);
    m.dec_in_c = apply(m.dec_in, 0x63);
    m.dec_out = kIso.t2a;
    uint8_t col[8]{};
    for (int j = 0; j < 8; ++j) {
        const uint8_t t = static_cast<uint8_t>(1u << j), a1 = t >> 4, a0 = t & 15;
        col[j] = static_cast<uint8_t>(g16_mul(kLambda, g16_mul(a1, a1)) ^ g16_mul(a0, a0));
    }
    m.lin_delta = from_columns(col);
    return m;
}
inline constexpr SboxMaps kMaps = make_maps();

// scalar models of the two circuits, used only by the checks below
constexpr uint8_t sbox_model(uint8_t x) {
    return static_cast<uint8_t>(apply(kMaps.enc_out, tw_inv(apply(kMaps.enc_in, x))) ^ 0x63);
}
constexpr uint8_t inv_sbox_model(uint8_t y) {
    return apply(kMaps.dec_out, tw_inv(static_cast<uint8_t>(apply(kMaps.dec_in, y) ^ kMaps.dec_in_c)));
}
constexpr bool check_sboxes() {
    for (int x = 0; x < 256; ++x) {
        if (sbox_model(static_cast<uint8_t>(x)) != kAes.sbox[x]) return false;
        if (inv_sbox_model(static_cast<uint8_t>(x)) != kAes.isbox[x]) return false;
    }
    return true;
}
static_assert(kLambda != 0, "no trace-1 element");
static_assert(check_sboxes(), "tower-field S-box circuit disagrees with the S-box");

// ------------------------------------------------- column maps (32 bits)
constexpr uint8_t xtime8(uint8_t a) { return xtime_c(a); }
constexpr uint32_t mix_column_model(uint32_t c) {  // eq (20), rows in bytes 0..3
    uint8_t a[4]{}, o[4]{};
    for (int r = 0; r < 4; ++r) a[r] = static_cast<uint8_t>(c >> (8 * r));
    for (int r = 0; r < 4; ++r)
        o[r] = static_cast<uint8_t>(aes_mul(2, a[r]) ^ aes_mul(3, a[(r + 1) % 4]) ^ a[(r + 2) % 4] ^ a[(r + 3) % 4]);
    return pack4(o[0], o[1], o[2], o[3]);
}
constexpr uint32_t inv_mix_column_model(uint32_t c) {
    uint8_t a[4]{}, o[4]{};
    for (int r = 0; r < 4; ++r) a[r] = static_cast<uint8_t>(c >> (8 * r));
    for (int r = 0; r < 4; ++r)
        o[r] = static_cast<uint8_t>(aes_mul(0x0e, a[r]) ^ aes_mul(0x0b, a[(r + 1) % 4]) ^
                                    aes_mul(0x0d, a[(r + 2) % 4]) ^ aes_mul(0x09, a[(r + 3) % 4]));
    return pack4(o[0], o[1], o[2], o[3]);
}
// InvMixColumns = MixColumns after  a0 += u, a2 += u, a1 += v, a3 += v  with
// u = 04 (a0 + a2), v = 04 (a1 + a3): the inverse matrix factors as the
// MixColumns matrix times circ(05, 00, 04, 00).  Both sides are GF(2)-linear
// in the 32 column bits, so the 32 unit vectors decide it.
constexpr uint32_t inv_mix_factored_model(uint32_t c) {
    uint8_t a[4]{};
    for (int r = 0; r < 4; ++r) a[r] = static_cast<uint8_t>(c >> (8 * r));
    const uint8_t u = xtime8(xtime8(static_cast<uint8_t>(a[0] ^ a[2])));
    const uint8_t v = xtime8(xtime8(static_cast<uint8_t>(a[1] ^ a[3])));
    return mix_column_model(pack4(static_cast<uint8_t>(a[0] ^ u), static_cast<uint8_t>(a[1] ^ v),
                                  static_cast<uint8_t>(a[2] ^ u), static_cast<uint8_t>(a[3] ^ v)));
}
constexpr bool check_inv_mix_factoring() {
    for (int b = 0; b < 32; ++b)
        if (inv_mix_factored_model(1u << b) != inv_mix_column_model(1u << b)) return false;
    return true;
}
static_assert(check_inv_mix_factoring(), "InvMixColumns factoring");

// The GF(16) inverse as four 4-input boolean functions: truth table of
// output bit k over the 16 inputs.
AESGB_CX_HD uint16_t inv16_truth(int k) {
    uint16_t t = 0;
    for (int x = 0; x < 16; ++x) t |= static_cast<uint16_t>(((g16_inv(static_cast<uint8_t>(x)) >> k) & 1) << x);
    return t;
}

}  // namespace bsmath
}  // namespace aesgb
