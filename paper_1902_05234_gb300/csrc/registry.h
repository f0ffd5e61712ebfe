// registry.h -- host-side lookup of the kernel instantiations compiled in the
// per-direction translation units (ecb_enc.cu, ecb_dec.cu, ecb_tma.cu), and the
// debug build's per-unit check counters.
#pragma once
#include <cstdint>

namespace aesgb {

// Host stub of ecb_kernel<dir, nr, nb, layout>, or nullptr if that
// combination is not compiled.
const void *ecb_kernel_enc(int nr, int nb, int layout);
const void *ecb_kernel_dec(int nr, int nb, int layout);

// ecb_tma.cu: the TMA-staged variant (layout AES_LAYOUT_R4_TMA), its dynamic
// shared memory (R4 tables, two tiles of 512 nb bytes and two mbarriers per
// warp), and the count of bounded device waits that ran out (read and reset).
const void *ecb_kernel_tma(int dir, int nr, int nb);
uint32_t ecb_tma_smem_bytes(int dir, int threads, int nb);
int read_wait_timeouts(unsigned long long *count);
// One warp of the TMA-staged kernel whose barriers can never complete (see
// aes_tma_selftest_timeout in aesgb.h).
int launch_tma_selftest_timeout(const uint8_t *in, uint8_t *out, size_t nblocks, void *stream);

// Failed index checks of the debug build (AESGB_BOUNDS_CHECK), one counter
// per translation unit with kernels; each call returns the count and resets it
// (AES_OK, or AES_E_CUDA).  In the release build each reports 0.
int bounds_violations_ecb_enc(unsigned long long *out);
int bounds_violations_ecb_dec(unsigned long long *out);
int bounds_violations_ecb_tma(unsigned long long *out);
int bounds_violations_modes(unsigned long long *out);
int bounds_violations_batch(unsigned long long *out);
int bounds_violations_ct(unsigned long long *out);
// batch.cu, debug build: exactly-once tags of the batch kernel's chunks (see
// aes_debug_batch_coverage in aesgb.h); AES_E_CONFIG in the release build.
int read_chunk_coverage(unsigned long long *once, unsigned long long *repeated, unsigned long long *beyond);

// Copy table `which` (0 te0, 1 td0, 2 S-box, 3 InvS) from the constant bank of
// the encrypt module on the current device.  Returns a cudaError_t value.
int ecb_module_const_table(int which, uint32_t *out);

}  // namespace aesgb
