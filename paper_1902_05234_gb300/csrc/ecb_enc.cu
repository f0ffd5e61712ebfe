// ecb_enc.cu -- instantiations of the ECB encryption kernel (Nr = 10/12/14;
// 1, 2, 4 or 8 blocks per thread; each table placement).
#include "aes_kernels.cuh"
#include "registry.h"

namespace aesgb {

#define AESGB_K(NR, NB, L)                                                    \
    if (nr == NR && nb == NB && layout == L)                                  \
        return reinterpret_cast<const void *>(&ecb_kernel<kEncrypt, NR, NB, L>);
#define AESGB_NR(NR)                                                          \
    AESGB_K(NR, 1, kLayoutR4) AESGB_K(NR, 2, kLayoutR4) AESGB_K(NR, 4, kLayoutR4) \
    AESGB_K(NR, 1, kLayoutR1) AESGB_K(NR, 2, kLayoutR1) AESGB_K(NR, 4, kLayoutR1) \
    AESGB_K(NR, 1, kLayoutP4) AESGB_K(NR, 1, kLayoutConst) \
    AESGB_K(NR, 1, kLayoutR2) AESGB_K(NR, 2, kLayoutR2) AESGB_K(NR, 4, kLayoutR2) \
    AESGB_K(NR, 8, kLayoutR4) AESGB_K(NR, 8, kLayoutR2) \
    AESGB_K(NR, 1, kLayoutReg) AESGB_K(NR, 2, kLayoutReg)

AESGB_BOUNDS_READER(ecb_enc)

const void *ecb_kernel_enc(int nr, int nb, int layout) {
    AESGB_NR(10)
    AESGB_NR(12)
    AESGB_NR(14)
    return nullptr;
}

int ecb_module_const_table(int which, uint32_t *out) {
    ConstTables h;
    cudaError_t e = cudaMemcpyFromSymbol(&h, c_tab, sizeof(h));
    if (e != cudaSuccess) return static_cast<int>(e);
    for (int x = 0; x < 256; ++x) {
        switch (which) {
        case 0: out[x] = h.te[0][x]; break;
        case 1: out[x] = h.td[0][x]; break;
        case 2: out[x] = (h.te[0][x] >> 8) & 0xffu; break;  // S(x) is byte 1 of te0
        default: out[x] = h.is[x]; break;
        }
    }
    return 0;
}

}  // namespace aesgb
