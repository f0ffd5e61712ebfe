/*
 * aes_oracle.c -- plain, slow, byte-by-byte CPU AES used as TEST INFRASTRUCTURE.
 *
 * Only the tests, the package smoke check and the benchmark's CPU-baseline leg
 * load this file's shared library.  The GPU library never links it, and it
 * shares no code, header or table with the GPU library: the S-box is derived
 * here, at first use, from the GF(2^8) inverse and the affine map.
 *
 * What it computes follows "GPU Accelerated AES Algorithm" (Wang & Chu,
 * arXiv 1902.05234) in the paper's notation; where the paper is silent or its
 * text is wrong, the FIPS-197 reading is taken (each place says so):
 *
 *   orc_gf_add        Def. 1, eq (7): addition in GF(2^8) is XOR of coefficients
 *   orc_clmul         eqs (9)-(11): polynomial product before reduction
 *   orc_poly_mod      eqs (12)-(13): remainder modulo m(x), eq (8)
 *   orc_gf_mul        Def. 2: product modulo m(x) = x^8+x^4+x^3+x+1
 *   orc_xtime         Def. 3, eqs (15)-(17): multiplication by x
 *   orc_gf_inv        multiplicative inverse, by brute-force search
 *   orc_sbox          Def. 4, eq (18); values from FIPS-197 5.1.1 (inverse + affine map),
 *                     because the paper cites the table without giving it
 *   orc_round         Defs. 4-7, eqs (18)-(21): SubBytes, ShiftRows, MixColumns, AddRoundKey
 *   orc_ttable        eqs (22)-(25): the four T tables
 *   orc_tround        eq (26): one round as four T-table lookups per column
 *   orc_key_expansion key schedule of 3.2.2 (Nr+1 round keys), steps of FIPS-197 5.2
 *   orc_cipher        Algorithm 1, corrected to FIPS-197 5.1: Nr-1 full rounds, a final
 *                     round without MixColumns, round key i used in round i
 *   orc_inv_cipher    decryption (claimed by the paper, never described): FIPS-197 5.3
 *   orc_eq_inv_schedule / orc_eq_inv_cipher   FIPS-197 5.3.5 (equivalent inverse cipher)
 *   orc_ecb           ECB, eq (1): C_i = cipher(P_i), independently per 16-byte block
 *   orc_ctr           CTR, eq (5): C_i = P_i xor cipher(counter block of block i)
 *   orc_cbc_encrypt / orc_cbc_decrypt   CBC (eq (2) as intended: the printed
 *                     equation omits the cipher; NIST SP 800-38A reading)
 *   orc_cfb_encrypt / orc_cfb_decrypt   CFB (eq (3) read by the text beside
 *                     it: full-block CFB of NIST SP 800-38A)
 *
 * State layout (FIPS-197 3.4): s[r][c] = in[r + 4c], r = row, c = column.
 * Round key i is bytes w[16 i .. 16 i + 15] of the expanded key, column-major
 * like the state.
 *
 * Building with -DORC_MUTANT=n plants one deliberate mistake (see the
 * MUTANT(n) sites).  The tests build such variants on the CPU to show that
 * the oracle's pins catch each of them; a normal build has ORC_MUTANT 0.
 */
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif
#define MUTANT(n) (ORC_MUTANT == (n))

/* ------------------------------------------------------------------------ */
/* GF(2^8), 3.2.1                                                            */
/* ------------------------------------------------------------------------ */

/* eq (8): m(x) = x^8 + x^4 + x^3 + x + 1 as a 9-bit integer. */
#define ORC_M_X (MUTANT(2) ? 0x11du : 0x11bu)

/* Def. 1 / eq (7): adding two polynomials over GF(2) adds their coefficients
 * mod 2, i.e. XOR of the bit vectors. */
uint8_t orc_gf_add(uint8_t a, uint8_t b) { return (uint8_t)(a ^ b); }

/* eqs (9)-(11): schoolbook product of two degree<8 polynomials over GF(2);
 * each set bit i of b contributes a * x^i, and equal powers cancel (XOR). */
uint16_t orc_clmul(uint8_t a, uint8_t b) {
    uint16_t p = 0;
    for (int i = 0; i < 8; ++i)
        if ((b >> i) & 1) p ^= (uint16_t)((uint16_t)a << i);
    return p;
}

/* eqs (12)-(13): remainder of a degree<15 polynomial divided by m(x), by long
 * division from the highest power down. */
uint8_t orc_poly_mod(uint16_t p) {
    for (int d = 14; d >= 8; --d)
        if ((p >> d) & 1) p ^= (uint16_t)(ORC_M_X << (d - 8));
    return (uint8_t)p;
}

/* Def. 2: multiplication in GF(2^8) = polynomial product modulo m(x). */
uint8_t orc_gf_mul(uint8_t a, uint8_t b) { return orc_poly_mod(orc_clmul(a, b)); }

/* Def. 3 / eqs (15)-(17): multiply by x -- a left shift, and when a degree-8
 * term appears, subtract (XOR) m(x).  Written independently of orc_gf_mul so
 * that the two can be checked against each other. */
uint8_t orc_xtime(uint8_t a) {
    uint8_t r = (uint8_t)(a << 1);
    if (a & 0x80) r ^= (uint8_t)(MUTANT(1) ? 0x1d : 0x1b); /* low byte of m(x) */
    return r;
}

/* Multiplicative inverse by exhaustive search; 0 has none and maps to 0
 * (the FIPS-197 5.1.1 convention). */
uint8_t orc_gf_inv(uint8_t a) {
    if (a == 0) return 0;
    for (int b = 1; b < 256; ++b)
        if (orc_gf_mul(a, (uint8_t)b) == 1) return (uint8_t)b;
    return 0; /* unreachable for an irreducible m(x) */
}

/* ------------------------------------------------------------------------ */
/* S-box, Def. 4.  The paper uses a 256-byte table without printing it; the   */
/* reading is FIPS-197 5.1.1: inverse in GF(2^8), then the affine map          */
/*   b'_i = b_i + b_{i+4} + b_{i+5} + b_{i+6} + b_{i+7} + c_i  (indices mod 8) */
/* with c = 0x63.                                                              */
/* ------------------------------------------------------------------------ */

static uint8_t affine(uint8_t b) {
    const uint8_t c = MUTANT(3) ? 0x62 : 0x63;
    uint8_t out = 0;
    for (int i = 0; i < 8; ++i) {
        int bit;
        if (MUTANT(4))
            bit = ((b >> i) ^ (b >> ((i + 3) % 8)) ^ (b >> ((i + 5) % 8)) ^
                   (b >> ((i + 6) % 8)) ^ (b >> ((i + 7) % 8)) ^ (c >> i)) & 1;
        else
            bit = ((b >> i) ^ (b >> ((i + 4) % 8)) ^ (b >> ((i + 5) % 8)) ^
                   (b >> ((i + 6) % 8)) ^ (b >> ((i + 7) % 8)) ^ (c >> i)) & 1;
        out |= (uint8_t)(bit << i);
    }
    return out;
}

static uint8_t g_sbox[256], g_inv_sbox[256];
static pthread_once_t g_once = PTHREAD_ONCE_INIT;

static void derive_sbox(void) {
    for (int x = 0; x < 256; ++x) g_sbox[x] = affine(orc_gf_inv((uint8_t)x));
    /* InvSubBytes is the inverse permutation: search, not a second formula. */
    for (int y = 0; y < 256; ++y)
        for (int x = 0; x < 256; ++x)
            if (g_sbox[x] == y) { g_inv_sbox[y] = (uint8_t)x; break; }
}

uint8_t orc_sbox(uint8_t x) { pthread_once(&g_once, derive_sbox); return g_sbox[x]; }
uint8_t orc_inv_sbox(uint8_t y) { pthread_once(&g_once, derive_sbox); return g_inv_sbox[y]; }

/* ------------------------------------------------------------------------ */
/* Round transformations, 3.2.2.  st[r][c] = row r, column c.                */
/* ------------------------------------------------------------------------ */

typedef uint8_t state_t[4][4];

static void load_state(state_t s, const uint8_t in[16]) {
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r) s[r][c] = in[r + 4 * c];
}
static void store_state(uint8_t out[16], state_t s) {
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r) out[r + 4 * c] = s[r][c];
}

/* Def. 4, eq (18): every byte replaced by sbox[byte]. */
static void sub_bytes(state_t s) {
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) s[r][c] = orc_sbox(s[r][c]);
}
static void inv_sub_bytes(state_t s) {
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) s[r][c] = orc_inv_sbox(s[r][c]);
}

/* Def. 5, eq (19): state'_{i,j} = state_{i,(i+j) mod 4} (row i rotated left by i). */
static void shift_rows(state_t s) {
    state_t t;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            t[i][j] = MUTANT(5) ? s[i][(j - i + 4) % 4] : s[i][(i + j) % 4];
    memcpy(s, t, sizeof t);
}
/* Inverse of eq (19): state'_{i,(i+j) mod 4} = state_{i,j}. */
static void inv_shift_rows(state_t s) {
    state_t t;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) t[i][(i + j) % 4] = s[i][j];
    memcpy(s, t, sizeof t);
}

/* Def. 6, eq (20): each column multiplied by the fixed matrix A over GF(2^8). */
static const uint8_t A_MIX[4][4] = {
    {0x02, 0x03, 0x01, 0x01},
    {0x01, 0x02, 0x03, 0x01},
    {0x01, 0x01, 0x02, 0x03},
    {0x03, 0x01, 0x01, 0x02},
};
/* Its inverse over GF(2^8) (FIPS-197 5.3.3); the tests check A * A_INV = I. */
static const uint8_t A_INV[4][4] = {
    {0x0e, 0x0b, 0x0d, 0x09},
    {0x09, 0x0e, 0x0b, 0x0d},
    {0x0d, 0x09, 0x0e, 0x0b},
    {0x0b, 0x0d, 0x09, 0x0e},
};

static void mul_columns(state_t s, const uint8_t m[4][4], int transpose) {
    for (int c = 0; c < 4; ++c) {
        uint8_t col[4];
        for (int r = 0; r < 4; ++r) {
            uint8_t acc = 0;
            for (int i = 0; i < 4; ++i)
                acc = orc_gf_add(acc, orc_gf_mul(transpose ? m[i][r] : m[r][i], s[i][c]));
            col[r] = acc;
        }
        for (int r = 0; r < 4; ++r) s[r][c] = col[r];
    }
}
static void mix_columns(state_t s) { mul_columns(s, A_MIX, MUTANT(6)); }
static void inv_mix_columns(state_t s) {
    static const uint8_t BAD[4][4] = {
        {0x0e, 0x0d, 0x0b, 0x09}, {0x09, 0x0e, 0x0d, 0x0b},
        {0x0b, 0x09, 0x0e, 0x0d}, {0x0d, 0x0b, 0x09, 0x0e}};
    mul_columns(s, MUTANT(10) ? BAD : A_INV, 0);
}

/* Def. 7, eq (21): state' = state xor epdkey, round key taken column-major. */
static void add_round_key(state_t s, const uint8_t *rk) {
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r) s[r][c] = orc_gf_add(s[r][c], rk[r + 4 * c]);
}

/* The 4x4 matrices, exported so the tests can check A * A_INV = I. */
void orc_mix_matrix(int inverse, uint8_t out[16]) {
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) out[4 * r + c] = inverse ? A_INV[r][c] : A_MIX[r][c];
}

/* One plain full round (Defs. 4-7 in order), for checking eq (26). */
void orc_round(const uint8_t in[16], const uint8_t rk[16], uint8_t out[16]) {
    state_t s;
    load_state(s, in);
    sub_bytes(s);
    shift_rows(s);
    mix_columns(s);
    add_round_key(s, rk);
    store_state(out, s);
}

/* Single transformations on a 16-byte state, exported for the tests. */
void orc_sub_bytes(uint8_t b[16]) { state_t s; load_state(s, b); sub_bytes(s); store_state(b, s); }
void orc_shift_rows(uint8_t b[16]) { state_t s; load_state(s, b); shift_rows(s); store_state(b, s); }
void orc_mix_columns(uint8_t b[16]) { state_t s; load_state(s, b); mix_columns(s); store_state(b, s); }
void orc_inv_mix_columns(uint8_t b[16]) { state_t s; load_state(s, b); inv_mix_columns(s); store_state(b, s); }

/* ------------------------------------------------------------------------ */
/* T tables, eqs (22)-(25), and the T-table round, eq (26).                  */
/* "xtime(sbox(w), 03)" is read as the GF(2^8) product 03 * sbox(w).        */
/* ------------------------------------------------------------------------ */

/* Column coefficients of T_k: T_k(w)[row] = COEF[k][row] * sbox(w). */
static const uint8_t T_COEF[4][4] = {
    {0x02, 0x01, 0x01, 0x03}, /* eq (22) */
    {0x03, 0x02, 0x01, 0x01}, /* eq (23) */
    {0x01, 0x03, 0x02, 0x01}, /* eq (24) */
    {0x01, 0x01, 0x03, 0x02}, /* eq (25) */
};

void orc_ttable(int k, uint8_t w, uint8_t col[4]) {
    int kk = MUTANT(13) && k == 1 ? 3 : k;
    uint8_t s = orc_sbox(w);
    for (int row = 0; row < 4; ++row) col[row] = orc_gf_mul(T_COEF[kk][row], s);
}

/* eq (26): e_j = T0[p_{0,j}] + T1[p_{1,j+1}] + T2[p_{2,j+2}] + T3[p_{3,j+3}] + k_j,
 * column indices mod 4, + being XOR of 4-byte columns. */
void orc_tround(const uint8_t in[16], const uint8_t rk[16], uint8_t out[16]) {
    state_t p;
    load_state(p, in);
    for (int j = 0; j < 4; ++j) {
        uint8_t e[4];
        for (int row = 0; row < 4; ++row) e[row] = rk[row + 4 * j];
        for (int k = 0; k < 4; ++k) {
            uint8_t t[4];
            orc_ttable(k, p[k][(j + k) % 4], t);
            for (int row = 0; row < 4; ++row) e[row] ^= t[row];
        }
        for (int row = 0; row < 4; ++row) out[row + 4 * j] = e[row];
    }
}

/* ------------------------------------------------------------------------ */
/* Key schedule (3.2.2; steps per FIPS-197 5.2).  Nk = key words, Nr = Nk+6. */
/* The paper's "twelve round keys" is read as Nr+1 round keys, as its own    */
/* 128 * (10 + 1) bit count says.                                            */
/* ------------------------------------------------------------------------ */

int orc_nrounds(int keybits) {
    switch (keybits) {
    case 128: return 10;
    case 192: return 12;
    case 256: return 14;
    default: return -1;
    }
}

/* w receives 16*(Nr+1) bytes: word i is w[4i..4i+3].  Returns Nr, or -1. */
int orc_key_expansion(int keybits, const uint8_t *key, uint8_t *w) {
    int nr = orc_nrounds(keybits);
    if (nr < 0) return -1;
    int nk = keybits / 32, nwords = 4 * (nr + 1);
    memcpy(w, key, (size_t)(4 * nk));
    uint8_t rcon = 0x01; /* x^0; advanced by xtime once per use */
    if (MUTANT(8)) rcon = 0x02;
    for (int i = nk; i < nwords; ++i) {
        uint8_t t[4];
        memcpy(t, w + 4 * (i - 1), 4);
        if (i % nk == 0) {
            uint8_t t0 = t[0]; /* RotWord: (a0,a1,a2,a3) -> (a1,a2,a3,a0) */
            t[0] = t[1]; t[1] = t[2]; t[2] = t[3]; t[3] = t0;
            for (int b = 0; b < 4; ++b) t[b] = orc_sbox(t[b]); /* SubWord */
            t[0] ^= rcon; /* Rcon[i/Nk] = (x^(i/Nk - 1), 0, 0, 0) */
            rcon = orc_xtime(rcon);
        } else if (nk > 6 && i % nk == 4 && !MUTANT(9)) {
            for (int b = 0; b < 4; ++b) t[b] = orc_sbox(t[b]); /* SubWord */
        }
        for (int b = 0; b < 4; ++b) w[4 * i + b] = w[4 * (i - nk) + b] ^ t[b];
    }
    return nr;
}

/* ------------------------------------------------------------------------ */
/* Cipher.  Algorithm 1 as printed applies MixColumns in the last round and  */
/* keys its loop from expandedkey[0]; the FIPS-197 5.1 reading is used.      */
/* ------------------------------------------------------------------------ */

void orc_cipher(const uint8_t *w, int nr, const uint8_t in[16], uint8_t out[16]) {
    state_t s;
    load_state(s, in);
    add_round_key(s, w);
    for (int round = 1; round < nr; ++round) {
        sub_bytes(s);
        shift_rows(s);
        mix_columns(s);
        add_round_key(s, w + 16 * round);
    }
    sub_bytes(s);
    shift_rows(s);
    if (MUTANT(7)) mix_columns(s); /* the printed Algorithm 1's last round */
    add_round_key(s, w + 16 * nr);
    store_state(out, s);
}

/* Inverse cipher, FIPS-197 5.3 (the paper claims decryption without a
 * description).  Uses the same expanded key w, rounds in reverse order. */
void orc_inv_cipher(const uint8_t *w, int nr, const uint8_t in[16], uint8_t out[16]) {
    state_t s;
    load_state(s, in);
    add_round_key(s, w + 16 * nr);
    for (int round = nr - 1; round >= 1; --round) {
        inv_shift_rows(s);
        inv_sub_bytes(s);
        add_round_key(s, w + 16 * round);
        inv_mix_columns(s);
    }
    inv_shift_rows(s);
    inv_sub_bytes(s);
    add_round_key(s, w);
    store_state(out, s);
}

/* FIPS-197 5.3.5: dw = w with InvMixColumns applied to round keys 1..Nr-1. */
void orc_eq_inv_schedule(const uint8_t *w, int nr, uint8_t *dw) {
    memcpy(dw, w, (size_t)(16 * (nr + 1)));
    int first = MUTANT(11) ? 0 : 1;
    for (int round = first; round < nr; ++round) {
        state_t s;
        load_state(s, dw + 16 * round);
        inv_mix_columns(s);
        store_state(dw + 16 * round, s);
    }
}

/* FIPS-197 5.3.5 equivalent inverse cipher, driven by dw. */
void orc_eq_inv_cipher(const uint8_t *dw, int nr, const uint8_t in[16], uint8_t out[16]) {
    state_t s;
    load_state(s, in);
    add_round_key(s, dw + 16 * nr);
    for (int round = nr - 1; round >= 1; --round) {
        inv_sub_bytes(s);
        inv_shift_rows(s);
        inv_mix_columns(s);
        add_round_key(s, dw + 16 * round);
    }
    inv_sub_bytes(s);
    inv_shift_rows(s);
    add_round_key(s, dw);
    store_state(out, s);
}

/* ------------------------------------------------------------------------ */
/* Modes.                                                                    */
/* ------------------------------------------------------------------------ */

/* ECB, eq (1): C_i = cipher(P_i) for each whole 16-byte block, independently.
 * dir 0 = encrypt (orc_cipher), 1 = decrypt (orc_inv_cipher); both take w. */
void orc_ecb(int dir, const uint8_t *w, int nr, const uint8_t *in, uint8_t *out, size_t nblocks) {
    for (size_t i = 0; i < nblocks; ++i) {
        if (dir == 0) orc_cipher(w, nr, in + 16 * i, out + 16 * i);
        else orc_inv_cipher(w, nr, in + 16 * i, out + 16 * i);
    }
}

/* Counter block of block i: the 128-bit big-endian integer ctr0 + i, mod
 * 2^128.  eq (5) writes CTR(R + i); the reading is that the caller passes the
 * counter block of the first block (R + 1 in the paper's 1-based indexing) and
 * block i (0-based) uses ctr0 + i, as in NIST SP 800-38A with the standard
 * incrementing function over the whole block. */
void orc_ctr_block(const uint8_t ctr0[16], uint64_t i, uint8_t out[16]) {
    memcpy(out, ctr0, 16);
    uint64_t carry = i;
    if (MUTANT(12)) {
        for (int b = 0; b < 16 && carry; ++b) {
            uint64_t v = (uint64_t)out[b] + (carry & 0xff);
            out[b] = (uint8_t)v;
            carry = (carry >> 8) + (v >> 8);
        }
        return;
    }
    for (int b = 15; b >= 0 && carry; --b) {
        uint64_t v = (uint64_t)out[b] + (carry & 0xff);
        out[b] = (uint8_t)v;
        carry = (carry >> 8) + (v >> 8);
    }
}

void orc_ctr(const uint8_t *w, int nr, const uint8_t ctr0[16], const uint8_t *in, uint8_t *out,
             size_t nblocks) {
    for (size_t i = 0; i < nblocks; ++i) {
        uint8_t cb[16], ks[16];
        orc_ctr_block(ctr0, (uint64_t)i, cb);
        orc_cipher(w, nr, cb, ks);
        for (int b = 0; b < 16; ++b) out[16 * i + b] = in[16 * i + b] ^ ks[b];
    }
}

/* CBC.  eq (2) as printed (C_i = P_i xor C_{i-1}) leaves out the block
 * cipher; the reading is NIST SP 800-38A: C_i = cipher(P_i xor C_{i-1}),
 * C_0 = IV, and P_i = inv_cipher(C_i) xor C_{i-1}. */
void orc_cbc_encrypt(const uint8_t *w, int nr, const uint8_t iv[16], const uint8_t *in,
                     uint8_t *out, size_t nblocks) {
    uint8_t prev[16];
    memcpy(prev, iv, 16);
    for (size_t i = 0; i < nblocks; ++i) {
        uint8_t x[16];
        for (int b = 0; b < 16; ++b) x[b] = in[16 * i + b] ^ prev[b];
        orc_cipher(w, nr, x, out + 16 * i);
        memcpy(prev, out + 16 * i, 16);
    }
}

void orc_cbc_decrypt(const uint8_t *w, int nr, const uint8_t iv[16], const uint8_t *in,
                     uint8_t *out, size_t nblocks) {
    uint8_t prev[16];
    memcpy(prev, iv, 16);
    for (size_t i = 0; i < nblocks; ++i) {
        uint8_t c[16], x[16];
        memcpy(c, in + 16 * i, 16); /* keep C_i: out may alias in */
        orc_inv_cipher(w, nr, c, x);
        for (int b = 0; b < 16; ++b) out[16 * i + b] = x[b] ^ prev[b];
        memcpy(prev, c, 16);
    }
}

/* CFB.  eq (3) as printed feeds C_{i-1} xor P_{i-1} to the cipher, which
 * contradicts the text beside it (the mode is fed with the ciphertext, not
 * the plaintext, of the previous block); the reading is the text's, as in
 * NIST SP 800-38A with full 16-byte segments: C_i = P_i xor cipher(C_{i-1}),
 * C_0 = IV, and P_i = C_i xor cipher(C_{i-1}) -- the forward cipher in both
 * directions.  MUTANT(14) follows the printed equation instead. */
void orc_cfb_encrypt(const uint8_t *w, int nr, const uint8_t iv[16], const uint8_t *in,
                     uint8_t *out, size_t nblocks) {
    uint8_t prev_c[16], prev_p[16];
    memcpy(prev_c, iv, 16);
    memset(prev_p, 0, 16);
    for (size_t i = 0; i < nblocks; ++i) {
        uint8_t x[16], ks[16], p[16];
        memcpy(p, in + 16 * i, 16); /* keep P_i: out may alias in */
        for (int b = 0; b < 16; ++b) x[b] = (uint8_t)(prev_c[b] ^ (MUTANT(14) ? prev_p[b] : 0));
        orc_cipher(w, nr, x, ks);
        for (int b = 0; b < 16; ++b) out[16 * i + b] = p[b] ^ ks[b];
        memcpy(prev_c, out + 16 * i, 16);
        memcpy(prev_p, p, 16);
    }
}

void orc_cfb_decrypt(const uint8_t *w, int nr, const uint8_t iv[16], const uint8_t *in,
                     uint8_t *out, size_t nblocks) {
    uint8_t prev_c[16], prev_p[16];
    memcpy(prev_c, iv, 16);
    memset(prev_p, 0, 16);
    for (size_t i = 0; i < nblocks; ++i) {
        uint8_t c[16], x[16], ks[16];
        memcpy(c, in + 16 * i, 16); /* keep C_i: out may alias in */
        for (int b = 0; b < 16; ++b) x[b] = (uint8_t)(prev_c[b] ^ (MUTANT(14) ? prev_p[b] : 0));
        orc_cipher(w, nr, x, ks);
        for (int b = 0; b < 16; ++b) out[16 * i + b] = c[b] ^ ks[b];
        memcpy(prev_c, c, 16);
        memcpy(prev_p, out + 16 * i, 16);
    }
}

/* ------------------------------------------------------------------------ */
/* The same ECB loop split over threads by contiguous block ranges; used    */
/* only to time the oracle on all host cores.                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    int dir, nr;
    const uint8_t *w, *in;
    uint8_t *out;
    size_t nblocks;
} ecb_job;

static void *ecb_worker(void *arg) {
    ecb_job *j = (ecb_job *)arg;
    orc_ecb(j->dir, j->w, j->nr, j->in, j->out, j->nblocks);
    return NULL;
}

int orc_ecb_mt(int dir, const uint8_t *w, int nr, const uint8_t *in, uint8_t *out, size_t nblocks,
               int nthreads) {
    enum { MAXT = 256 };
    if (nthreads < 1) nthreads = 1;
    if (nthreads > MAXT) nthreads = MAXT;
    (void)orc_sbox(0); /* derive the S-box once before the threads start */
    pthread_t tid[MAXT];
    int threaded[MAXT];
    ecb_job job[MAXT];
    size_t per = nblocks / (size_t)nthreads, rem = nblocks % (size_t)nthreads, start = 0;
    for (int t = 0; t < nthreads; ++t) {
        size_t n = per + ((size_t)t < rem ? 1 : 0);
        job[t] = (ecb_job){dir, nr, w, in + 16 * start, out + 16 * start, n};
        threaded[t] = pthread_create(&tid[t], NULL, ecb_worker, &job[t]) == 0;
        if (!threaded[t]) ecb_worker(&job[t]); /* no thread: do the range here */
        start += n;
    }
    for (int t = 0; t < nthreads; ++t)
        if (threaded[t]) pthread_join(tid[t], NULL);
    return nthreads;
}

int orc_mutant_id(void) { return ORC_MUTANT; }
