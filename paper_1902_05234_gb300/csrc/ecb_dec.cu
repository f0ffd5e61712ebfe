// ecb_dec.cu -- instantiations of the ECB decryption kernel (Nr = 10/12/14;
// 1, 2, 4 or 8 blocks per thread; each table placement).
#include "aes_kernels.cuh"
#include "registry.h"

namespace aesgb {

#define AESGB_K(NR, NB, L)                                                    \
    if (nr == NR && nb == NB && layout == L)                                  \
        return reinterpret_cast<const void *>(&ecb_kernel<kDecrypt, NR, NB, L>);
#define AESGB_NR(NR)                                                          \
    AESGB_K(NR, 1, kLayoutR4) AESGB_K(NR, 2, kLayoutR4) AESGB_K(NR, 4, kLayoutR4) \
    AESGB_K(NR, 1, kLayoutR1) AESGB_K(NR, 2, kLayoutR1) AESGB_K(NR, 4, kLayoutR1) \
    AESGB_K(NR, 1, kLayoutP4) AESGB_K(NR, 1, kLayoutConst) \
    AESGB_K(NR, 1, kLayoutR2) AESGB_K(NR, 2, kLayoutR2) AESGB_K(NR, 4, kLayoutR2) \
    AESGB_K(NR, 8, kLayoutR4) AESGB_K(NR, 8, kLayoutR2) \
    AESGB_K(NR, 1, kLayoutReg) AESGB_K(NR, 2, kLayoutReg)

AESGB_BOUNDS_READER(ecb_dec)

const void *ecb_kernel_dec(int nr, int nb, int layout) {
    AESGB_NR(10)
    AESGB_NR(12)
    AESGB_NR(14)
    return nullptr;
}

}  // namespace aesgb
