// tune.cpp -- launch configuration choice for the single-buffer kernels.
#include <cstddef>

#include "batch_internal.h"
#include "capi_internal.h"

namespace aesgb {

aes_launch_cfg default_cfg(int /*dir*/, int /*nrounds*/, size_t /*nblocks*/) {
    aes_launch_cfg c;
    c.threads = 1024;
    c.blocks_per_thread = 2;
    c.layout = AES_LAYOUT_R4;
    c.ctas_per_sm = 1;
    return c;
}

aes_launch_cfg tuned_or_default_cfg(int dir, int nrounds, size_t nblocks) {
    return default_cfg(dir, nrounds, nblocks);
}

aes_batch_cfg default_batch_cfg() {
    aes_batch_cfg c;
    c.threads = 512;
    c.blocks_per_thread = 1;
    c.chunk_passes = 32;
    c.ctas_per_sm = 1;
    return c;
}

aes_batch_cfg batch_cfg_for(int /*n*/) { return default_batch_cfg(); }

}  // namespace aesgb
