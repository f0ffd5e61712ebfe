// tune.cpp -- launch-configuration choice: size-adaptive defaults and an
// autotuner that times candidate configurations on the caller's buffers.
//
// The single-buffer kernels are tuned per (device, direction, Nr, size
// class), size class = floor(log4(nblocks)); the batch kernel per device.  A
// device is its model tag (32-bit FNV-1a hash of the device name and compute
// capability) and its SM count, so a cache written on one GPU model is not
// applied to another.  Tuned entries live in memory and, when
// AESGB_TUNE_CACHE names a file, are loaded from it on first use and written
// back after every tuning run.  The file is plain text, one entry per line
// (lines of another format are ignored):
//   ecb   <tag hex> <sms> <dir> <nr> <class> <threads> <blocks_per_thread> <layout> <ctas_per_sm>
//   batch <tag hex> <sms> <threads> <blocks_per_thread> <chunk_passes> <ctas_per_sm> <layout_enc> <layout_dec>
// (a batch line without the two layouts, as older files have, means R4 / R2)
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "batch_internal.h"
#include "capi_internal.h"

namespace aesgb {
namespace {

using DevKey = std::pair<uint32_t, int>;                   // model tag, sms
using EcbKey = std::tuple<uint32_t, int, int, int, int>;  // tag, sms, dir, nr, class
std::mutex g_mu;
std::map<EcbKey, aes_launch_cfg> g_ecb;
std::map<DevKey, aes_batch_cfg> g_batch;
bool g_env_loaded = false;

int size_class(size_t nblocks) {
    int c = 0;
    while (nblocks >= 4 && c < 24) {
        nblocks >>= 2;
        ++c;
    }
    return c;
}

int current_sms() {
    int dev = 0;
    if (current_device(&dev) != AES_OK) return 0;
    const int s = sm_count(dev);
    return s > 0 ? s : 0;
}

// FNV-1a over the device name and compute capability; 0 without a device.
uint32_t model_tag(int dev) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    uint32_t h = 2166136261u;
    auto mix = [&h](unsigned char c) { h = (h ^ c) * 16777619u; };
    for (const char *c = p.name; *c; ++c) mix(static_cast<unsigned char>(*c));
    mix(static_cast<unsigned char>(p.major));
    mix(static_cast<unsigned char>(p.minor));
    return h;
}

// (model tag, SM count) of the current device, the tag looked up once per device.
DevKey current_devkey() {
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static uint32_t tags[kMaxDev];
    static bool known[kMaxDev];
    int dev = 0;
    if (current_device(&dev) != AES_OK || dev < 0 || dev >= kMaxDev) return DevKey{0u, 0};
    uint32_t tag;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!known[dev]) {
            tags[dev] = model_tag(dev);
            known[dev] = true;
        }
        tag = tags[dev];
    }
    return DevKey{tag, current_sms()};
}

EcbKey ecb_key(int dir, int nrounds, size_t nblocks) {
    const DevKey d = current_devkey();
    return EcbKey{d.first, d.second, dir, nrounds, size_class(nblocks)};
}

int load_file_locked(const char *path) {
    FILE *f = std::fopen(path, "r");
    if (!f) return AES_E_ARG;
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
        unsigned int tag = 0;
        int a[8];
        if (std::sscanf(line, "ecb %x %d %d %d %d %d %d %d %d", &tag, &a[0], &a[1], &a[2], &a[3], &a[4], &a[5],
                        &a[6], &a[7]) == 9) {
            aes_launch_cfg c{a[4], a[5], a[6], a[7]};
            if (validate_cfg(c) == AES_OK) g_ecb[EcbKey{tag, a[0], a[1], a[2], a[3]}] = c;
        } else {
            const int got = std::sscanf(line, "batch %x %d %d %d %d %d %d %d", &tag, &a[0], &a[1], &a[2], &a[3], &a[4],
                                        &a[5], &a[6]);
            if (got != 6 && got != 8) continue;
            if (got == 6) {
                a[5] = AES_LAYOUT_R4;
                a[6] = AES_LAYOUT_R2;
            }
            aes_batch_cfg c{a[1], a[2], a[3], a[4], a[5], a[6]};
            if (validate_batch_cfg(c) == AES_OK) g_batch[DevKey{tag, a[0]}] = c;
        }
    }
    std::fclose(f);
    return AES_OK;
}

int save_file_locked(const char *path) {
    FILE *f = std::fopen(path, "w");
    if (!f) return AES_E_ARG;
    std::fprintf(f, "# aesgb tune cache v3\n");
    for (const auto &kv : g_ecb) {
        const auto &k = kv.first;
        const auto &c = kv.second;
        std::fprintf(f, "ecb %08x %d %d %d %d %d %d %d %d\n", static_cast<unsigned int>(std::get<0>(k)),
                     std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), c.threads, c.blocks_per_thread,
                     c.layout, c.ctas_per_sm);
    }
    for (const auto &kv : g_batch)
        std::fprintf(f, "batch %08x %d %d %d %d %d %d %d\n", static_cast<unsigned int>(kv.first.first),
                     kv.first.second, kv.second.threads, kv.second.blocks_per_thread, kv.second.chunk_passes,
                     kv.second.ctas_per_sm, kv.second.layout_enc, kv.second.layout_dec);
    const bool ok = std::fclose(f) == 0;
    return ok ? AES_OK : AES_E_ARG;
}

void load_env_locked() {
    if (g_env_loaded) return;
    g_env_loaded = true;
    const char *p = std::getenv("AESGB_TUNE_CACHE");
    if (p && *p) (void)load_file_locked(p);
}

void save_env_locked() {
    const char *p = std::getenv("AESGB_TUNE_CACHE");
    if (p && *p) (void)save_file_locked(p);
}

// Device time of one launch of `launch(stream)` (already validated): one
// warm-up launch (it sets the kernel's attributes), then `reps` launches
// captured in a CUDA graph on a private stream and the replay timed, so that
// microsecond launches are timed back to back on the device as an
// application's stream of launches runs them, not at the rate the host can
// issue them.  The private stream first waits for the caller's stream `s`,
// and `s` waits for it at the end.
template <class F>
float time_launches(F launch, cudaStream_t s, int reps, int *status) {
    cudaStream_t ts = nullptr;
    cudaEvent_t a = nullptr, b = nullptr, join = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    int st = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) == cudaSuccess &&
                     cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess &&
                     cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess
                 ? AES_OK
                 : AES_E_CUDA;
    if (st == AES_OK)
        st = cudaEventRecord(join, s) == cudaSuccess && cudaStreamWaitEvent(ts, join, 0) == cudaSuccess ? AES_OK
                                                                                                     : AES_E_CUDA;
    if (st == AES_OK) st = launch(ts);
    if (st == AES_OK) st = cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal) == cudaSuccess ? AES_OK
                                                                                                       : AES_E_CUDA;
    if (st == AES_OK) {
        for (int r = 0; r < reps && st == AES_OK; ++r) st = launch(ts);
        const bool ended = cudaStreamEndCapture(ts, &g) == cudaSuccess;
        if (st == AES_OK && !ended) st = AES_E_CUDA;
    }
    if (st == AES_OK) st = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess ? AES_OK : AES_E_CUDA;
    if (st == AES_OK) st = cudaGraphLaunch(ge, ts) == cudaSuccess ? AES_OK : AES_E_CUDA;  // warm replay
    if (st == AES_OK)
        st = cudaEventRecord(a, ts) == cudaSuccess && cudaGraphLaunch(ge, ts) == cudaSuccess &&
                     cudaEventRecord(b, ts) == cudaSuccess
                 ? AES_OK
                 : AES_E_CUDA;
    float ms = 0.f;
    if (st == AES_OK) st = cudaEventSynchronize(b) == cudaSuccess ? AES_OK : AES_E_CUDA;
    if (st == AES_OK) st = cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? AES_OK : AES_E_CUDA;
    if (st != AES_OK) (void)cudaGetLastError();
    if (ts && join && cudaEventRecord(join, ts) == cudaSuccess) (void)cudaStreamWaitEvent(s, join, 0);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (ts) cudaStreamDestroy(ts);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (join) cudaEventDestroy(join);
    (void)cudaGetLastError();
    *status = st;
    return ms / static_cast<float>(reps);
}

}  // namespace

// Untuned choice: R4 tables, 2 blocks per thread and 1,024 threads when the
// buffer fills every SM several times over; smaller buffers get R2 tables,
// 2 blocks per thread and 256 threads with as many CTAs per SM as fit (three):
// small CTAs spread a small buffer over every SM, and CTAs that finish early
// make room for the next launch's CTAs to fill their tables.
aes_launch_cfg default_cfg(int /*dir*/, int /*nrounds*/, size_t nblocks) {
    aes_launch_cfg c;
    c.ctas_per_sm = 1;
    const size_t sms = static_cast<size_t>(current_sms() > 0 ? current_sms() : 152);
    if (nblocks >= sms * 16384) {
        c.layout = AES_LAYOUT_R4;
        c.threads = 1024;
        c.blocks_per_thread = 2;
        return c;
    }
    c.layout = AES_LAYOUT_R2;
    c.threads = 256;
    c.blocks_per_thread = 2;
    c.ctas_per_sm = 0;
    return c;
}

aes_launch_cfg tuned_or_default_cfg(int dir, int nrounds, size_t nblocks) {
    const EcbKey key = ecb_key(dir, nrounds, nblocks);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_env_locked();
        if (!g_ecb.empty()) {
            auto it = g_ecb.find(key);
            if (it != g_ecb.end()) return it->second;
        }
    }
    return default_cfg(dir, nrounds, nblocks);
}

aes_batch_cfg default_batch_cfg() {
    aes_batch_cfg c;
    c.threads = 512;
    c.blocks_per_thread = 1;
    c.chunk_passes = 32;
    c.ctas_per_sm = 1;
    c.layout_enc = AES_LAYOUT_R4;
    c.layout_dec = AES_LAYOUT_R2;
    return c;
}

aes_batch_cfg batch_cfg_for(int /*n*/) {
    const DevKey key = current_devkey();
    std::lock_guard<std::mutex> lk(g_mu);
    load_env_locked();
    auto it = g_batch.find(key);
    return it != g_batch.end() ? it->second : default_batch_cfg();
}

}  // namespace aesgb

using namespace aesgb;

extern "C" {

int aes_tune_ecb(int dir, int nrounds, const uint32_t *rk, const uint8_t *in, uint8_t *out, size_t nblocks,
                 void *stream, aes_launch_cfg *best) {
    if (dir != 0 && dir != 1) return AES_E_ARG;
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    if (!rk || nblocks == 0) return AES_E_ARG;
    st = check_buffers(in, out, nblocks);
    if (st != AES_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<aes_launch_cfg> cands;
    for (int layout : {AES_LAYOUT_R4, AES_LAYOUT_R2, AES_LAYOUT_R1})
        for (int nb : {1, 2, 4, 8})
            for (int th : {128, 256, 512, 768, 1024}) {
                if (th > (nb >= 8 ? 256 : nb >= 4 ? 512 : 1024)) continue;
                if (nb == 8 && layout == AES_LAYOUT_R1) continue;  // not compiled
                cands.push_back(aes_launch_cfg{th, nb, layout, 0});
            }
    cands.push_back(default_cfg(dir, nrounds, nblocks));
    // enough launches that small sizes are timed over a few hundred
    // microseconds, and the better of two timings, so that replay-to-replay
    // noise does not pick a configuration at microsecond sizes
    const int reps = nblocks >= (size_t(1) << 24) ? 2 : (nblocks >= (size_t(1) << 18) ? 8 : 64);
    const int trials = nblocks >= (size_t(1) << 24) ? 1 : 2;
    float best_ms = 1e30f;
    aes_launch_cfg best_cfg = cands.back();
    for (const auto &c : cands) {
        int tst = AES_OK;
        float ms = 1e30f;
        for (int t = 0; t < trials && tst == AES_OK; ++t) {
            const float m = time_launches(
                [&](cudaStream_t ts) { return launch_ecb(dir, rk, nrounds, in, out, nblocks, c, ts); }, s, reps,
                &tst);
            if (m < ms) ms = m;
        }
        if (tst != AES_OK) continue;  // e.g. a configuration that does not fit
        if (ms < best_ms) {
            best_ms = ms;
            best_cfg = c;
        }
    }
    if (best_ms >= 1e29f) return AES_E_CUDA;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_env_locked();
        g_ecb[ecb_key(dir, nrounds, nblocks)] = best_cfg;
        save_env_locked();
    }
    if (best) *best = best_cfg;
    return AES_OK;
}

int aes_tune_batch(const aes_desc *desc_dev, int n, void *ws, size_t ws_bytes, void *stream, aes_batch_cfg *best) {
    if (!desc_dev || n <= 0 || !ws) return AES_E_ARG;
    if (ws_bytes < batch_ws_bytes(n)) return AES_E_RANGE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float best_ms = 1e30f;
    aes_batch_cfg best_cfg = default_batch_cfg();
    auto consider = [&](const aes_batch_cfg &c) {
        int tst = AES_OK;
        const float ms = time_launches(
            [&](cudaStream_t ts) { return aes_ecb_batch_ws(desc_dev, n, ws, ws_bytes, nullptr, &c, ts); }, s, 2,
            &tst);
        if (tst == AES_OK && ms < best_ms) {
            best_ms = ms;
            best_cfg = c;
        }
    };
    // granularity and chunk size with the default table layouts, then the
    // layout pairs (section 4.2's axis) at the best of those
    for (int nb : {1, 2})
        for (int th : {256, 384, 512})
            for (int passes : {8, 16, 32, 64})
                consider(aes_batch_cfg{th, nb, passes, 1, AES_LAYOUT_R4, AES_LAYOUT_R2});
    if (best_ms >= 1e29f) return AES_E_CUDA;
    const aes_batch_cfg g = best_cfg;
    const int pairs[][2] = {{AES_LAYOUT_R4, AES_LAYOUT_R4}, {AES_LAYOUT_R2, AES_LAYOUT_R2}, {AES_LAYOUT_R1, AES_LAYOUT_R1}};
    for (const auto &p : pairs)
        consider(aes_batch_cfg{g.threads, g.blocks_per_thread, g.chunk_passes, g.ctas_per_sm, p[0], p[1]});
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_env_locked();
        g_batch[current_devkey()] = best_cfg;
        save_env_locked();
    }
    if (best) *best = best_cfg;
    return AES_OK;
}

int aes_tune(int dir, int nrounds, size_t bytes_hint, void *stream) {
    if (dir != 0 && dir != 1) return AES_E_ARG;
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    const size_t nblocks = bytes_hint / 16;
    if (nblocks == 0 || nblocks > (SIZE_MAX >> 5)) return AES_E_ARG;
    // scratch input and output of the hinted size (stream-ordered); the
    // kernels' time does not depend on the bytes, so neither is filled
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *in = nullptr, *out = nullptr;
    st = lib_malloc_device_async(&in, nblocks * 16, s);
    if (st == AES_OK) st = lib_malloc_device_async(&out, nblocks * 16, s);
    if (st == AES_OK) {
        uint32_t enc[60] = {0}, dec[60] = {0};
        const uint8_t key[32] = {0};
        const int keybits = nrounds == 10 ? 128 : nrounds == 12 ? 192 : 256;
        (void)expand_key_host(keybits, key, enc, dec);
        st = aes_tune_ecb(dir, nrounds, dir == 0 ? enc : dec, static_cast<const uint8_t *>(in),
                          static_cast<uint8_t *>(out), nblocks, stream, nullptr);
    }
    if (out) (void)cudaFreeAsync(out, s);
    if (in) (void)cudaFreeAsync(in, s);
    (void)cudaGetLastError();
    return st;
}

int aes_tune_save(const char *path) {
    if (!path) return AES_E_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    return save_file_locked(path);
}

int aes_tune_load(const char *path) {
    if (!path) return AES_E_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    g_env_loaded = true;
    return load_file_locked(path);
}

int aes_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_ecb.clear();
    g_batch.clear();
    g_env_loaded = true;  // do not reload the environment file behind the caller's back
    return AES_OK;
}

int aes_tune_set_ecb(int dir, int nrounds, size_t nblocks, const aes_launch_cfg *cfg) {
    if ((dir != 0 && dir != 1) || !cfg) return AES_E_ARG;
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    st = validate_cfg(*cfg);
    if (st != AES_OK) return st;
    std::lock_guard<std::mutex> lk(g_mu);
    load_env_locked();
    g_ecb[ecb_key(dir, nrounds, nblocks)] = *cfg;
    return AES_OK;
}

int aes_batch_get_cfg(int n, aes_batch_cfg *cfg) {
    if (!cfg) return AES_E_ARG;
    *cfg = batch_cfg_for(n);
    return AES_OK;
}

}  // extern "C"
