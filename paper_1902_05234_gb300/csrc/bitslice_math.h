// bitslice_math.h -- scalar models used around the constant-time kernel: the
// column maps MixColumns (eq (20)) and InvMixColumns (FIPS-197 5.3.3), on a
// column packed as a word (row r in bits 8r..8r+7).  The host uses them to
// build the round-key masks; the compile-time checks of the circuits in
// bitslice.cuh use them as the definitions the circuits must meet.
#pragma once
#include <cstdint>

#include "aes_tables.h"

#if defined(__CUDACC__)
#define AESGB_CX_HD __host__ __device__ constexpr
#else
#define AESGB_CX_HD constexpr
#endif

namespace aesgb {
namespace bsmath {

constexpr uint32_t mix_column_model(uint32_t c) {  // eq (20), rows in bytes 0..3
    uint8_t a[4]{}, o[4]{};
    for (int r = 0; r < 4; ++r) a[r] = static_cast<uint8_t>(c >> (8 * r));
    for (int r = 0; r < 4; ++r)
        o[r] = static_cast<uint8_t>(gmul_c(2, a[r]) ^ gmul_c(3, a[(r + 1) % 4]) ^ a[(r + 2) % 4] ^ a[(r + 3) % 4]);
    return pack4(o[0], o[1], o[2], o[3]);
}

constexpr uint32_t inv_mix_column_model(uint32_t c) {
    uint8_t a[4]{}, o[4]{};
    for (int r = 0; r < 4; ++r) a[r] = static_cast<uint8_t>(c >> (8 * r));
    for (int r = 0; r < 4; ++r)
        o[r] = static_cast<uint8_t>(gmul_c(0x0e, a[r]) ^ gmul_c(0x0b, a[(r + 1) % 4]) ^
                                    gmul_c(0x0d, a[(r + 2) % 4]) ^ gmul_c(0x09, a[(r + 3) % 4]));
    return pack4(o[0], o[1], o[2], o[3]);
}

constexpr bool check_column_models() {  // the two maps are inverse to each other
    uint32_t x = 0x01234567u;
    for (int i = 0; i < 64; ++i) {
        if (inv_mix_column_model(mix_column_model(x)) != x) return false;
        x = x * 1664525u + 1013904223u;
    }
    return true;
}
static_assert(check_column_models(), "MixColumns / InvMixColumns models");

}  // namespace bsmath
}  // namespace aesgb
