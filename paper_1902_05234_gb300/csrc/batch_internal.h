// batch_internal.h -- host helpers of the batched path shared with tune.cpp / capi.cu.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

#include "aesgb.h"

namespace aesgb {

size_t batch_ws_bytes(int n);
aes_batch_cfg default_batch_cfg();
aes_batch_cfg batch_cfg_for(int n);
int validate_batch_cfg(const aes_batch_cfg &c);
void batch_shutdown();

// Host-side planning and the kernel alone (see batch.cu).
void plan_on_host(const aes_desc *desc, int n, unsigned int chunk_blocks, void *ws_host);
unsigned int batch_chunk_blocks(const aes_batch_cfg &c);
int enqueue_batch_kernel(const aes_desc *desc, int n, void *ws, const aes_batch_cfg &c, cudaStream_t s);

}  // namespace aesgb
