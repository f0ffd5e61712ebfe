// capi_internal.h -- host helpers shared by the C-ABI translation units.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "aesgb.h"

namespace aesgb {

struct RoundKeys;

int current_device(int *dev);
int sm_count(int dev);
int ensure_smem_attr(const void *fn, int dev, uint32_t bytes);
// Launch `fn` with programmatic stream serialisation (the kernel may start
// before the previous kernel in the stream completes; it must call
// griddep_wait() before touching global memory).  AES_E_CUDA on failure.
int launch_pdl(const void *fn, int grid, int threads, uint32_t smem, void **params, void *stream);
int check_nrounds(int nr);
// The library's own allocations (device memory, page-locked host memory),
// through the failure injector of aes_test_fail_allocs.  AES_OK, or
// AES_E_NOMEM with *p = nullptr.
int lib_malloc_device(void **p, size_t bytes);
int lib_malloc_host(void **p, size_t bytes);
// Stream-ordered device allocation (cudaMallocAsync on s), same injector.
int lib_malloc_device_async(void **p, size_t bytes, cudaStream_t s);
int check_buffers(const void *in, const void *out, size_t nblocks);
void order_round_keys(int dir, const uint32_t *rk, int nr, RoundKeys *out);
int validate_cfg(const aes_launch_cfg &c);
// Grid of a persistent launch: as many CTAs as fit (or c.ctas_per_sm) per SM,
// never more than the work needs; *fit_per_sm (may be NULL) receives how many
// CTAs of this kernel fit on one SM.
int persistent_grid(const void *fn, int dev, const aes_launch_cfg &c, uint32_t smem,
                    unsigned long long work_items_per_cta, unsigned long long total_items, int *grid,
                    int *fit_per_sm);
int launch_ecb(int dir, const uint32_t *rk, int nr, const uint8_t *in, uint8_t *out, size_t nblocks,
               const aes_launch_cfg &c, void *stream);

// keysched.cpp
int expand_key_host(int keybits, const uint8_t *key, uint32_t *rk_enc, uint32_t *rk_dec);

// host_io.cpp
int host_pipeline(int dir, const uint32_t *rk, int nr, const uint8_t *hin, uint8_t *hout, size_t nblocks,
                  uint8_t *dbuf, size_t dbuf_bytes, void *stream);
void host_io_shutdown();

// tune.cpp
aes_launch_cfg default_cfg(int dir, int nrounds, size_t nblocks);
aes_launch_cfg tuned_or_default_cfg(int dir, int nrounds, size_t nblocks);

}  // namespace aesgb
