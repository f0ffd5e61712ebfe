// capi.cu -- the C ABI of include/aesgb.h: argument checks, key schedule,
// launch-configuration choice and kernel launch for the single-buffer paths.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <map>
#include <tuple>
#include <utility>

#include "aesgb.h"
#include "aes_kernels.cuh"
#include "batch_internal.h"
#include "capi_internal.h"
#include "registry.h"

namespace aesgb {

// ---------------------------------------------------------------------------
// Per-device facts, cached
// ---------------------------------------------------------------------------
namespace {
constexpr int kMaxDevices = 64;
std::atomic<int> g_sm_count[kMaxDevices];
std::mutex g_attr_mu;
std::map<std::pair<const void *, int>, uint32_t> g_attr_bytes;  // (kernel, device) -> bytes allowed
// resident CTAs per SM, by (kernel, device, threads, shared bytes): the
// occupancy query costs microseconds, more than a small launch
std::mutex g_occ_mu;
std::map<std::tuple<const void *, int, int, uint32_t>, int> g_occ;
}  // namespace

int current_device(int *dev) {
    return cudaGetDevice(dev) == cudaSuccess && *dev >= 0 && *dev < kMaxDevices ? AES_OK : AES_E_CUDA;
}

int sm_count(int dev) {
    int v = g_sm_count[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
        return AES_E_CUDA;
    g_sm_count[dev].store(v, std::memory_order_relaxed);
    return v;
}

int ensure_smem_attr(const void *fn, int dev, uint32_t bytes) {
    if (bytes <= 48u * 1024u) return AES_OK;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto it = g_attr_bytes.find({fn, dev});
    if (it != g_attr_bytes.end() && it->second >= bytes) return AES_OK;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(bytes)) != cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    g_attr_bytes[{fn, dev}] = bytes;
    return AES_OK;
}

int check_nrounds(int nr) { return (nr == 10 || nr == 12 || nr == 14) ? AES_OK : AES_E_NROUNDS; }

int check_buffers(const void *in, const void *out, size_t nblocks) {
    if (!in || !out) return AES_E_ARG;
    if (nblocks > (SIZE_MAX >> 4)) return AES_E_ARG;
    const uintptr_t a = reinterpret_cast<uintptr_t>(in), b = reinterpret_cast<uintptr_t>(out);
    if ((a | b) & 15u) return AES_E_ALIGN;
    const uintptr_t len = static_cast<uintptr_t>(nblocks) << 4;
    if (a != b && a < b + len && b < a + len) return AES_E_OVERLAP;
    return AES_OK;
}

// Round keys in application order (see RoundKeys).  Decryption receives the
// dw schedule in FIPS order and applies round keys Nr, Nr-1, ..., 0.
void order_round_keys(int dir, const uint32_t *rk, int nr, RoundKeys *out) {
    std::memset(out, 0, sizeof(*out));
    for (int step = 0; step <= nr; ++step) {
        const int src = dir == kEncrypt ? step : nr - step;
        std::memcpy(&out->w[4 * step], rk + 4 * src, 16);
    }
}

const void *ecb_kernel_ptr(int dir, int nr, int nb, int layout) {
    if (layout == AES_LAYOUT_R4_TMA) return ecb_kernel_tma(dir, nr, nb);
    return dir == kEncrypt ? ecb_kernel_enc(nr, nb, layout) : ecb_kernel_dec(nr, nb, layout);
}

uint32_t ecb_smem_bytes(int dir, const aes_launch_cfg &c) {
    return c.layout == AES_LAYOUT_R4_TMA ? ecb_tma_smem_bytes(dir, c.threads, c.blocks_per_thread)
                                         : table_smem_bytes(dir, c.layout);
}

int validate_cfg(const aes_launch_cfg &c) {
    if (c.blocks_per_thread != 1 && c.blocks_per_thread != 2 && c.blocks_per_thread != 4 &&
        c.blocks_per_thread != 8)
        return AES_E_CONFIG;
    if (c.layout < AES_LAYOUT_R4 || c.layout > AES_LAYOUT_REG) return AES_E_CONFIG;
    if (c.threads < 32 || c.threads % 32 || c.threads > max_threads_for(c.blocks_per_thread, c.layout))
        return AES_E_CONFIG;
    if (c.ctas_per_sm < 0 || c.ctas_per_sm > 32) return AES_E_CONFIG;
    return AES_OK;
}

// Grid of a persistent launch: as many CTAs as fit (or as requested), never
// more than the work needs.
int persistent_grid(const void *fn, int dev, const aes_launch_cfg &c, uint32_t smem,
                    unsigned long long work_items_per_cta, unsigned long long total_items,
                    int *grid, int *fit_per_sm) {
    const int sms = sm_count(dev);
    if (sms < 0) return sms;
    int fit = 0;
    {
        std::lock_guard<std::mutex> lk(g_occ_mu);
        auto it = g_occ.find(std::make_tuple(fn, dev, static_cast<int>(c.threads), smem));
        if (it != g_occ.end()) fit = it->second;
    }
    if (fit == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, c.threads, smem) != cudaSuccess) {
            (void)cudaGetLastError();
            return AES_E_CUDA;
        }
        std::lock_guard<std::mutex> lk(g_occ_mu);
        g_occ[std::make_tuple(fn, dev, static_cast<int>(c.threads), smem)] = fit;
    }
    if (fit <= 0) return AES_E_CONFIG;
    if (fit_per_sm) *fit_per_sm = fit;
    const int per_sm = c.ctas_per_sm > 0 && c.ctas_per_sm < fit ? c.ctas_per_sm : fit;
    const unsigned long long need = (total_items + work_items_per_cta - 1) / work_items_per_cta;
    unsigned long long g = static_cast<unsigned long long>(per_sm) * static_cast<unsigned long long>(sms);
    if (need < g) g = need;
    *grid = static_cast<int>(g < 1 ? 1 : g);
    return AES_OK;
}

int launch_pdl(const void *fn, int grid, int threads, uint32_t smem, void **params, void *stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = static_cast<cudaStream_t>(stream);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelExC(&cfg, fn, params) != cudaSuccess) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    return AES_OK;
}

int launch_ecb(int dir, const uint32_t *rk, int nr, const uint8_t *in, uint8_t *out, size_t nblocks,
               const aes_launch_cfg &c, void *stream) {
    const void *fn = ecb_kernel_ptr(dir, nr, c.blocks_per_thread, c.layout);
    if (!fn) return AES_E_CONFIG;
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    const uint32_t smem = ecb_smem_bytes(dir, c);
    int st = ensure_smem_attr(fn, dev, smem);
    if (st != AES_OK) return st;
    int grid = 0, fit = 0;
    st = persistent_grid(fn, dev, c, smem,
                         static_cast<unsigned long long>(c.threads) * c.blocks_per_thread, nblocks, &grid, &fit);
    if (st != AES_OK) return st;
    EcbArgs args;
    args.in = reinterpret_cast<const uint4 *>(in);
    args.out = reinterpret_cast<uint4 *>(out);
    args.nblocks = nblocks;
    order_round_keys(dir, rk, nr, &args.rk);
    // Even shares (up to 8 units per warp) only where a second CTA cannot fit
    // beside the first: with room for two, the scheduler may place two CTAs
    // of one launch on an SM, and fixed shares would then double that SM's
    // work (4 MiB launches of one such configuration measured 5.4 and
    // 3.1 Tbit/s in two runs), while grid-stride passes let CTAs that finish
    // early free their slots.
    args.even_split_units = fit == 1 ? 8u : 0u;
    uint32_t extra_tx = 0;  // the TMA-staged kernel's second parameter
    void *params[] = {&args, &extra_tx};
    return launch_pdl(fn, grid, c.threads, smem, params, stream);
}

// ---------------------------------------------------------------------------
// the library's own allocations, with a host-side failure injector
// ---------------------------------------------------------------------------
namespace {
std::mutex g_inject_mu;
int g_inject_skip = 0, g_inject_fail = 0;  // allocations to let through, then to fail

// Whether this allocation is to fail (advancing the injector).
bool take_injected_failure() {
    std::lock_guard<std::mutex> lk(g_inject_mu);
    if (g_inject_fail == 0) return false;
    if (g_inject_skip > 0) {
        --g_inject_skip;
        return false;
    }
    --g_inject_fail;
    return true;
}
}  // namespace

int lib_malloc_device(void **p, size_t bytes) {
    *p = nullptr;
    if (take_injected_failure()) return AES_E_NOMEM;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return AES_E_NOMEM;
    }
    return AES_OK;
}

int lib_malloc_device_async(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (take_injected_failure()) return AES_E_NOMEM;
    if (cudaMallocAsync(p, bytes, s) != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return AES_E_NOMEM;
    }
    return AES_OK;
}

int lib_malloc_host(void **p, size_t bytes) {
    *p = nullptr;
    if (take_injected_failure()) return AES_E_NOMEM;
    if (cudaMallocHost(p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return AES_E_NOMEM;
    }
    return AES_OK;
}

}  // namespace aesgb

using namespace aesgb;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *aes_status_str(int status) {
    switch (status) {
    case AES_OK: return "AES_OK";
    case AES_E_ARG: return "AES_E_ARG: null pointer, size overflow or bad argument";
    case AES_E_KEYBITS: return "AES_E_KEYBITS: key size must be 128, 192 or 256 bits";
    case AES_E_NROUNDS: return "AES_E_NROUNDS: nrounds must be 10, 12 or 14";
    case AES_E_ALIGN: return "AES_E_ALIGN: block pointers must be 16-byte aligned";
    case AES_E_OVERLAP: return "AES_E_OVERLAP: in and out overlap without being equal";
    case AES_E_CUDA: return "AES_E_CUDA: a CUDA runtime call failed";
    case AES_E_NOMEM: return "AES_E_NOMEM: allocation failed";
    case AES_E_TIMEOUT: return "AES_E_TIMEOUT: bounded wait ran out";
    case AES_E_BUSY: return "AES_E_BUSY: admission refused (budget or slots full)";
    case AES_E_RANGE: return "AES_E_RANGE: size above the documented maximum";
    case AES_E_NOTFOUND: return "AES_E_NOTFOUND: unknown key id or ticket";
    case AES_E_CONFIG: return "AES_E_CONFIG: unsupported launch configuration";
    case AES_E_CANCELLED: return "AES_E_CANCELLED: request cancelled before its launch";
    case AES_E_UNREGISTERED: return "AES_E_UNREGISTERED: buffer outside every registered range";
    default: return "unknown status";
    }
}

int aes_version(void) { return 10000; }

int aes_wait_timeouts(unsigned long long *count) {
    if (!count) return AES_E_ARG;
    return read_wait_timeouts(count);
}

int aes_test_fail_allocs(int skip, int count) {
    if (skip < 0 || count < 0) return AES_E_ARG;
    std::lock_guard<std::mutex> lk(g_inject_mu);
    g_inject_skip = count ? skip : 0;
    g_inject_fail = count;
    return AES_OK;
}

int aes_debug_bounds_violations(unsigned long long *count) {
    if (!count) return AES_E_ARG;
    *count = 0;
#if defined(AESGB_BOUNDS_CHECK)
    int (*const readers[])(unsigned long long *) = {bounds_violations_ecb_enc, bounds_violations_ecb_dec,
                                                     bounds_violations_ecb_tma, bounds_violations_modes,
                                                     bounds_violations_batch,   bounds_violations_ct};
    for (auto rd : readers) {
        unsigned long long v = 0;
        const int st = rd(&v);
        if (st != AES_OK) return st;
        *count += v;
    }
    return AES_OK;
#else
    return AES_E_CONFIG;
#endif
}

int aes_tma_selftest_timeout(const uint8_t *in, uint8_t *out, size_t nblocks, void *stream) {
    if (nblocks == 0 || nblocks > 64) return AES_E_RANGE;
    const int st = check_buffers(in, out, nblocks);
    if (st != AES_OK) return st;
    return launch_tma_selftest_timeout(in, out, nblocks, stream);
}

int aes_expand_key(int keybits, const uint8_t *key, uint32_t *rk_enc, uint32_t *rk_dec) {
    return expand_key_host(keybits, key, rk_enc, rk_dec);
}

int aes_ecb_get_cfg(int dir, int nrounds, size_t nblocks, aes_launch_cfg *cfg) {
    if (!cfg || (dir != 0 && dir != 1)) return AES_E_ARG;
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    *cfg = tuned_or_default_cfg(dir, nrounds, nblocks);
    return AES_OK;
}

int aes_ecb_crypt_cfg(int dir, const uint32_t *rk, int nrounds, const uint8_t *in, uint8_t *out,
                      size_t nblocks, const aes_launch_cfg *cfg, void *stream) {
    if (dir != 0 && dir != 1) return AES_E_ARG;
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    if (!rk || !cfg) return AES_E_ARG;
    if (nblocks == 0) return AES_OK;
    st = check_buffers(in, out, nblocks);
    if (st != AES_OK) return st;
    st = validate_cfg(*cfg);
    if (st != AES_OK) return st;
    return launch_ecb(dir, rk, nrounds, in, out, nblocks, *cfg, stream);
}

int aes_ecb_encrypt(const uint32_t *rk, int nrounds, const uint8_t *in, uint8_t *out, size_t nblocks,
                    void *stream) {
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    const aes_launch_cfg c = tuned_or_default_cfg(0, nrounds, nblocks);
    return aes_ecb_crypt_cfg(0, rk, nrounds, in, out, nblocks, &c, stream);
}

int aes_ecb_decrypt(const uint32_t *rk_dec, int nrounds, const uint8_t *in, uint8_t *out, size_t nblocks,
                    void *stream) {
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    const aes_launch_cfg c = tuned_or_default_cfg(1, nrounds, nblocks);
    return aes_ecb_crypt_cfg(1, rk_dec, nrounds, in, out, nblocks, &c, stream);
}

int aes_device_sm_count(int device) {
    if (device < 0 || device >= 64) return AES_E_ARG;
    return sm_count(device);
}

int aes_host_table(int which, uint32_t *out) {
    if (!out || which < 0 || which > 3) return AES_E_ARG;
    for (int x = 0; x < 256; ++x) {
        switch (which) {
        case 0: out[x] = kAes.te0[x]; break;
        case 1: out[x] = kAes.td0[x]; break;
        case 2: out[x] = kAes.sbox[x]; break;
        default: out[x] = kAes.isbox[x]; break;
        }
    }
    return AES_OK;
}

int aes_shutdown(void) {
    host_io_shutdown();
    batch_shutdown();
    return AES_OK;
}

int aes_device_table(int which, uint32_t *out) {
    if (!out || which < 0 || which > 3) return AES_E_ARG;
    return ecb_module_const_table(which, out) == 0 ? AES_OK : AES_E_CUDA;
}

}  // extern "C"
