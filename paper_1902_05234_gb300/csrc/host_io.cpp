// host_io.cpp -- ECB over host buffers (aes_ecb_host) and library shutdown.
//
// The plaintext of a host buffer moves through a caller-provided device
// staging buffer in chunks: copy in, cipher in place, copy out.  Successive
// chunks use S = 3 slots of the staging buffer on three internal streams
// (copy-in, compute, copy-out), so the host-to-device copy of chunk i+1, the
// kernel of chunk i and the device-to-host copy of chunk i-1 overlap.
// Ordering is carried by events recorded per slot; the caller's stream is
// joined at the start (earlier work on it finishes first) and at the end (it
// waits for the last copy-out).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "capi_internal.h"

namespace aesgb {
namespace {

constexpr int kSlots = 3;
constexpr int kMaxDev = 64;

struct HostIoRes {
    std::mutex mu;
    bool ready = false;
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    cudaEvent_t ev_begin = nullptr;
    cudaEvent_t ev_in[kSlots] = {}, ev_run[kSlots] = {}, ev_out[kSlots] = {};
};

HostIoRes g_res[kMaxDev];

int init_res(HostIoRes &r) {
    if (r.ready) return AES_OK;
    const unsigned fl = cudaEventDisableTiming;
    bool ok = cudaStreamCreateWithFlags(&r.s_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&r.s_run, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&r.s_out, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&r.ev_begin, fl) == cudaSuccess;
    for (int i = 0; ok && i < kSlots; ++i)
        ok = cudaEventCreateWithFlags(&r.ev_in[i], fl) == cudaSuccess &&
             cudaEventCreateWithFlags(&r.ev_run[i], fl) == cudaSuccess &&
             cudaEventCreateWithFlags(&r.ev_out[i], fl) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    r.ready = true;
    return AES_OK;
}

void destroy_res(HostIoRes &r) {
    if (!r.ready) return;
    cudaStreamDestroy(r.s_in);
    cudaStreamDestroy(r.s_run);
    cudaStreamDestroy(r.s_out);
    cudaEventDestroy(r.ev_begin);
    for (int i = 0; i < kSlots; ++i) {
        cudaEventDestroy(r.ev_in[i]);
        cudaEventDestroy(r.ev_run[i]);
        cudaEventDestroy(r.ev_out[i]);
    }
    r.s_in = r.s_run = r.s_out = nullptr;
    r.ev_begin = nullptr;
    r.ready = false;
}

}  // namespace

int host_pipeline(int dir, const uint32_t *rk, int nr, const uint8_t *hin, uint8_t *hout, size_t nblocks,
                  uint8_t *dbuf, size_t dbuf_bytes, void *stream) {
    int dev = 0;
    if (current_device(&dev) != AES_OK) return AES_E_CUDA;
    const size_t slot_blocks = (dbuf_bytes / kSlots) >> 4;
    if (slot_blocks == 0) return AES_E_ARG;
    const aes_launch_cfg cfg = tuned_or_default_cfg(dir, nr, slot_blocks);
    HostIoRes &r = g_res[dev];
    std::lock_guard<std::mutex> lk(r.mu);
    int st = init_res(r);
    if (st != AES_OK) return st;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    bool ok = cudaEventRecord(r.ev_begin, user) == cudaSuccess &&
              cudaStreamWaitEvent(r.s_in, r.ev_begin, 0) == cudaSuccess &&
              cudaStreamWaitEvent(r.s_run, r.ev_begin, 0) == cudaSuccess &&
              cudaStreamWaitEvent(r.s_out, r.ev_begin, 0) == cudaSuccess;
    size_t done = 0;
    for (int i = 0; ok && done < nblocks; ++i) {
        const int slot = i % kSlots;
        const size_t nb = nblocks - done < slot_blocks ? nblocks - done : slot_blocks;
        uint8_t *d = dbuf + static_cast<size_t>(slot) * (slot_blocks << 4);
        if (i >= kSlots) ok = cudaStreamWaitEvent(r.s_in, r.ev_out[slot], 0) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(d, hin + (done << 4), nb << 4, cudaMemcpyHostToDevice, r.s_in) == cudaSuccess;
        ok = ok && cudaEventRecord(r.ev_in[slot], r.s_in) == cudaSuccess;
        ok = ok && cudaStreamWaitEvent(r.s_run, r.ev_in[slot], 0) == cudaSuccess;
        if (ok) {
            st = launch_ecb(dir, rk, nr, d, d, nb, cfg, r.s_run);
            if (st != AES_OK) return st;
        }
        ok = ok && cudaEventRecord(r.ev_run[slot], r.s_run) == cudaSuccess;
        ok = ok && cudaStreamWaitEvent(r.s_out, r.ev_run[slot], 0) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(hout + (done << 4), d, nb << 4, cudaMemcpyDeviceToHost, r.s_out) == cudaSuccess;
        ok = ok && cudaEventRecord(r.ev_out[slot], r.s_out) == cudaSuccess;
        done += nb;
    }
    // the caller's stream continues only after the last copy-out
    ok = ok && cudaEventRecord(r.ev_begin, r.s_out) == cudaSuccess &&
         cudaStreamWaitEvent(user, r.ev_begin, 0) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        return AES_E_CUDA;
    }
    return AES_OK;
}

void host_io_shutdown() {
    for (int d = 0; d < kMaxDev; ++d) {
        std::lock_guard<std::mutex> lk(g_res[d].mu);
        destroy_res(g_res[d]);
    }
}

}  // namespace aesgb

using namespace aesgb;

extern "C" int aes_ecb_host(int dir, const uint32_t *rk, int nrounds, const uint8_t *host_in,
                            uint8_t *host_out, size_t nblocks, uint8_t *dev_buf, size_t dev_buf_bytes,
                            void *stream) {
    if (dir != 0 && dir != 1) return AES_E_ARG;
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    if (!rk) return AES_E_ARG;
    if (nblocks == 0) return AES_OK;
    if (!host_in || !host_out || !dev_buf) return AES_E_ARG;
    if (nblocks > (SIZE_MAX >> 4)) return AES_E_ARG;
    if (reinterpret_cast<uintptr_t>(dev_buf) & 15u) return AES_E_ALIGN;
    const uintptr_t a = reinterpret_cast<uintptr_t>(host_in), b = reinterpret_cast<uintptr_t>(host_out);
    const uintptr_t len = static_cast<uintptr_t>(nblocks) << 4;
    if (a != b && a < b + len && b < a + len) return AES_E_OVERLAP;
    return host_pipeline(dir, rk, nrounds, host_in, host_out, nblocks, dev_buf, dev_buf_bytes, stream);
}

extern "C" int aes_ecb_host_direct(int dir, const uint32_t *rk, int nrounds, const uint8_t *host_in,
                                   uint8_t *host_out, size_t nblocks, void *stream) {
    if (dir != 0 && dir != 1) return AES_E_ARG;
    int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    if (!rk) return AES_E_ARG;
    if (nblocks == 0) return AES_OK;
    st = check_buffers(host_in, host_out, nblocks);
    if (st != AES_OK) return st;
    // both buffers must be page-locked host memory mapped for the device
    void *dev_ptr[2] = {nullptr, nullptr};
    const void *host_ptr[2] = {host_in, host_out};
    for (int i = 0; i < 2; ++i) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, host_ptr[i]) != cudaSuccess) {
            (void)cudaGetLastError();
            return AES_E_ARG;
        }
        if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return AES_E_ARG;
        dev_ptr[i] = a.devicePointer;
    }
    const aes_launch_cfg cfg = tuned_or_default_cfg(dir, nrounds, nblocks);
    return launch_ecb(dir, rk, nrounds, static_cast<const uint8_t *>(dev_ptr[0]), static_cast<uint8_t *>(dev_ptr[1]),
                      nblocks, cfg, stream);
}
