// keysched.cpp -- host key expansion for the GPU library (aes_expand_key).
//
// Paper section 3.2.2: the key schedule expands the cipher key into Nr+1 round
// keys of four words (128 * (Nr + 1) bits) and round key i is words 4i..4i+3
// (Algorithm 1, step 1).  The expansion steps follow FIPS-197 5.2; the
// decryption schedule is the FIPS-197 5.3.5 one for the equivalent inverse
// cipher.  Words are packed little-endian (byte 0 of the key string in bits
// 0..7), the packing every kernel uses.
#include <cstdint>
#include <cstring>

#include "aes_tables.h"
#include "capi_internal.h"

namespace aesgb {
namespace {

uint32_t sub_word(uint32_t w) {
    return pack4(kAes.sbox[w & 0xff], kAes.sbox[(w >> 8) & 0xff], kAes.sbox[(w >> 16) & 0xff],
                 kAes.sbox[w >> 24]);
}

// InvMixColumns of one column word (rows in bytes 0..3).
uint32_t inv_mix_column(uint32_t w) {
    const uint8_t a0 = w & 0xff, a1 = (w >> 8) & 0xff, a2 = (w >> 16) & 0xff, a3 = w >> 24;
    auto m = gmul_c;
    return pack4(static_cast<uint8_t>(m(a0, 0x0e) ^ m(a1, 0x0b) ^ m(a2, 0x0d) ^ m(a3, 0x09)),
                 static_cast<uint8_t>(m(a0, 0x09) ^ m(a1, 0x0e) ^ m(a2, 0x0b) ^ m(a3, 0x0d)),
                 static_cast<uint8_t>(m(a0, 0x0d) ^ m(a1, 0x09) ^ m(a2, 0x0e) ^ m(a3, 0x0b)),
                 static_cast<uint8_t>(m(a0, 0x0b) ^ m(a1, 0x0d) ^ m(a2, 0x09) ^ m(a3, 0x0e)));
}

}  // namespace

int expand_key_host(int keybits, const uint8_t *key, uint32_t *rk_enc, uint32_t *rk_dec) {
    if (keybits != 128 && keybits != 192 && keybits != 256) return AES_E_KEYBITS;
    if (!key) return AES_E_ARG;
    const int nk = keybits / 32, nr = nk + 6, nwords = 4 * (nr + 1);
    uint32_t w[60];
    for (int i = 0; i < nk; ++i)
        w[i] = pack4(key[4 * i], key[4 * i + 1], key[4 * i + 2], key[4 * i + 3]);
    uint8_t rcon = 1;
    for (int i = nk; i < nwords; ++i) {
        uint32_t t = w[i - 1];
        if (i % nk == 0) {
            t = sub_word((t >> 8) | (t << 24)) ^ rcon;  // RotWord moves byte 1 to byte 0
            rcon = xtime_c(rcon);
        } else if (nk == 8 && i % nk == 4) {
            t = sub_word(t);
        }
        w[i] = w[i - nk] ^ t;
    }
    if (rk_enc) std::memcpy(rk_enc, w, sizeof(uint32_t) * nwords);
    if (rk_dec) {
        for (int i = 0; i < nwords; ++i) {
            const int round = i / 4;
            rk_dec[i] = (round == 0 || round == nr) ? w[i] : inv_mix_column(w[i]);
        }
    }
    return nr;
}

}  // namespace aesgb
