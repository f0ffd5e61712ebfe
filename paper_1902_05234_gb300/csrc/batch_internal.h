// batch_internal.h -- host helpers of the batched path shared with tune.cpp / capi.cu.
#pragma once
#include <cstddef>

#include "aesgb.h"

namespace aesgb {

size_t batch_ws_bytes(int n);
aes_batch_cfg default_batch_cfg();
aes_batch_cfg batch_cfg_for(int n);
int validate_batch_cfg(const aes_batch_cfg &c);
void batch_shutdown();

}  // namespace aesgb
