// bounds.cuh -- index checks of the debug build (AESGB_BOUNDS_CHECK defined).
//
// AESGB_CHECK(cond) is `true` in the release build (cond is not even
// compiled).  In the debug build it evaluates cond, counts a failure in this
// translation unit's device counter and returns cond, so the caller can skip
// the access; nothing traps.  Each .cu with kernels instantiates
// AESGB_BOUNDS_READER(name) once, and aes_debug_bounds_violations (capi.cu)
// sums and resets the counters.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace aesgb {

#if defined(AESGB_BOUNDS_CHECK)

static __device__ unsigned long long g_bounds_violations = 0;

__device__ __forceinline__ bool bounds_ok(bool ok) {
    if (!ok) atomicAdd(&g_bounds_violations, 1ull);
    return ok;
}

// Bytes of dynamic shared memory this launch has.
__device__ __forceinline__ uint32_t dyn_smem_bytes() {
    uint32_t r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

#define AESGB_CHECK(cond) (::aesgb::bounds_ok(cond))

#define AESGB_BOUNDS_READER(NAME)                                                              \
    int bounds_violations_##NAME(unsigned long long *out) {                                    \
        const unsigned long long zero = 0;                                                     \
        if (cudaMemcpyFromSymbol(out, g_bounds_violations, sizeof *out) != cudaSuccess ||     \
            cudaMemcpyToSymbol(g_bounds_violations, &zero, sizeof zero) != cudaSuccess) {      \
            (void)cudaGetLastError();                                                          \
            return -6; /* AES_E_CUDA */                                                        \
        }                                                                                      \
        return 0;                                                                              \
    }

#else

#define AESGB_CHECK(cond) true
#define AESGB_BOUNDS_READER(NAME)                                                              \
    int bounds_violations_##NAME(unsigned long long *out) {                                    \
        *out = 0;                                                                              \
        return 0;                                                                              \
    }

#endif

}  // namespace aesgb
