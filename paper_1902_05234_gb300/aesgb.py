"""Thin ctypes binding of ``include/aesgb.h`` (same names, argument marshalling only).

Every computation runs in ``libaesgb.so``'s CUDA kernels; this module only
turns Python ints / numpy arrays / torch tensors into pointers and sizes and
raises ``AesError`` on a negative status.  If the library has not been built,
the first call raises: there is no CPU fallback.

Pointer arguments accept an int (a raw address) or a torch tensor (its
``data_ptr()``).  ``stream`` accepts None (torch's current CUDA stream), a
``torch.cuda.Stream`` or a raw ``cudaStream_t`` int.
"""
from __future__ import annotations

import ctypes
import os
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# AESGB_LIBRARY=debug loads the bounds-checking build (libaesgb_debug.so, made
# by ``build(debug=True)``) instead of the release library.
LIB_PATH = os.path.join(_HERE, "libaesgb_debug.so" if os.environ.get("AESGB_LIBRARY") == "debug"
                        else "libaesgb.so")

_lib = None
_lock = threading.Lock()

LAYOUT_R4, LAYOUT_R1, LAYOUT_P4, LAYOUT_CONST, LAYOUT_R4_TMA, LAYOUT_R2, LAYOUT_REG = 0, 1, 2, 3, 4, 5, 6
LAYOUT_NAMES = {0: "R4", 1: "R1", 2: "P4", 3: "CONST", 4: "R4_TMA", 5: "R2", 6: "REG"}
ENCRYPT, DECRYPT = 0, 1


class AesError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"{where}: {aes_status_str(status)} ({status})" if where else
                         f"{aes_status_str(status)} ({status})")


class aes_launch_cfg(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("blocks_per_thread", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}

    def __repr__(self):
        d = self.as_dict()
        return (f"aes_launch_cfg(threads={d['threads']}, bpt={16 * d['blocks_per_thread']}B, "
                f"layout={LAYOUT_NAMES.get(d['layout'], d['layout'])}, ctas_per_sm={d['ctas_per_sm']})")


class aes_desc(ctypes.Structure):
    _fields_ = [("rk", ctypes.c_uint64), ("in_", ctypes.c_uint64), ("out", ctypes.c_uint64),
                ("nblocks", ctypes.c_uint64), ("nrounds", ctypes.c_int32), ("dir", ctypes.c_int32)]


class aes_batch_cfg(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("blocks_per_thread", ctypes.c_int32),
                ("chunk_passes", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("layout_enc", ctypes.c_int32), ("layout_dec", ctypes.c_int32)]

    def __repr__(self):
        return (f"aes_batch_cfg(threads={self.threads}, bpt={16 * self.blocks_per_thread}B, "
                f"chunk_passes={self.chunk_passes}, ctas_per_sm={self.ctas_per_sm}, "
                f"layouts={LAYOUT_NAMES.get(self.layout_enc, self.layout_enc)}/"
                f"{LAYOUT_NAMES.get(self.layout_dec, self.layout_dec)})")


class aes_srv_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("bytes_completed", ctypes.c_uint64), ("inflight_bytes", ctypes.c_uint64),
                ("peak_inflight_bytes", ctypes.c_uint64), ("pending", ctypes.c_uint64),
                ("busy_s", ctypes.c_double), ("worker_status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("cancelled", ctypes.c_uint64), ("peak_busy_slots", ctypes.c_uint64),
                ("timed_batches", ctypes.c_uint64), ("peak_device_batches", ctypes.c_uint64),
                ("device_overlap_s", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


# numpy view of aes_desc (40 bytes) for building descriptor tables in bulk
DESC_DTYPE = np.dtype([("rk", "<u8"), ("in", "<u8"), ("out", "<u8"), ("nblocks", "<u8"),
                       ("nrounds", "<i4"), ("dir", "<i4")])
assert DESC_DTYPE.itemsize == ctypes.sizeof(aes_desc) == 40


_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i = ctypes.c_int

_SIGNATURES = {
    "aes_status_str": (ctypes.c_char_p, [_i]),
    "aes_version": (_i, []),
    "aes_expand_key": (_i, [_i, _u8p, _u32p, _u32p]),
    "aes_ecb_encrypt": (_i, [_u32p, _i, _vp, _vp, _sz, _vp]),
    "aes_ecb_decrypt": (_i, [_u32p, _i, _vp, _vp, _sz, _vp]),
    "aes_ecb_crypt_cfg": (_i, [_i, _u32p, _i, _vp, _vp, _sz, ctypes.POINTER(aes_launch_cfg), _vp]),
    "aes_ecb_get_cfg": (_i, [_i, _i, _sz, ctypes.POINTER(aes_launch_cfg)]),
    "aes_device_sm_count": (_i, [_i]),
    "aes_host_table": (_i, [_i, _u32p]),
    "aes_ecb_host": (_i, [_i, _u32p, _i, _vp, _vp, _sz, _vp, _sz, _vp]),
    "aes_batch_workspace_bytes": (_sz, [_i]),
    "aes_ecb_batch_ws": (_i, [_vp, _i, _vp, _sz, _vp, _vp, _vp]),
    "aes_ecb_batch": (_i, [_vp, _i, _vp]),
    "aes_ecb_batch_ex": (_i, [_vp, _i, _vp, _vp]),
    "aes_ecb_batch_noalloc": (_i, [_vp, _i, _vp, _vp]),
    "aes_batch_graph_create": (_i, [_vp, _i, _vp, _sz, _vp, _vp, ctypes.POINTER(_vp)]),
    "aes_batch_graph_launch": (_i, [_vp, _vp]),
    "aes_batch_graph_destroy": (_i, [_vp]),
    "aes_shutdown": (_i, []),
    "aes_calibrate_lookup_rate": (_i, [_vp, _sz, _vp, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
    "aes_calibrate_logic_rate": (_i, [_vp, _sz, _vp, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]),
    "aes_ecb_host_direct": (_i, [_i, _u32p, _i, _vp, _vp, _sz, _vp]),
    "aes_ecb_crypt_ct": (_i, [_i, _u32p, _i, _vp, _vp, _sz, _vp]),
    "aes_ct_selftest_host": (_i, [_i, _u32p, _i, _vp, _vp, _sz]),
    "aes_ct_ops_per_block": (_i, [_i, _i, ctypes.POINTER(ctypes.c_double)]),
    "aes_wait_timeouts": (_i, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "aes_tma_selftest_timeout": (_i, [_vp, _vp, _sz, _vp]),
    "aes_debug_bounds_violations": (_i, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "aes_debug_batch_coverage": (_i, [ctypes.POINTER(ctypes.c_ulonglong)] * 3),
    "aes_ctr_crypt": (_i, [_u32p, _i, _u8p, _vp, _vp, _sz, _vp]),
    "aes_cbc_decrypt": (_i, [_u32p, _i, _u8p, _vp, _vp, _sz, _vp]),
    "aes_cfb_decrypt": (_i, [_u32p, _i, _u8p, _vp, _vp, _sz, _vp]),
    "aes_tune_ecb": (_i, [_i, _i, _u32p, _vp, _vp, _sz, _vp, ctypes.POINTER(aes_launch_cfg)]),
    "aes_tune": (_i, [_i, _i, _sz, _vp]),
    "aes_tune_batch": (_i, [_vp, _i, _vp, _sz, _vp, ctypes.POINTER(aes_batch_cfg)]),
    "aes_tune_set_ecb": (_i, [_i, _i, _sz, ctypes.POINTER(aes_launch_cfg)]),
    "aes_batch_get_cfg": (_i, [_i, ctypes.POINTER(aes_batch_cfg)]),
    "aes_tune_save": (_i, [ctypes.c_char_p]),
    "aes_tune_load": (_i, [ctypes.c_char_p]),
    "aes_tune_clear": (_i, []),
    "aes_srv_create": (_i, [_sz, _i, _i, _i, ctypes.POINTER(_vp)]),
    "aes_srv_put_key": (_i, [_vp, _i, _i, _u8p]),
    "aes_srv_put_schedule": (_i, [_vp, _i, _u32p, _u32p, _i]),
    "aes_srv_set_device_timing": (_i, [_vp, _i]),
    "aes_srv_submit": (_i, [_vp, _i, _i, _vp, _vp, _sz, ctypes.POINTER(ctypes.c_uint64)]),
    "aes_srv_submit_many": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "aes_srv_poll": (_i, [_vp, ctypes.c_uint64, ctypes.POINTER(_i), ctypes.POINTER(_i),
                          ctypes.POINTER(ctypes.c_double)]),
    "aes_srv_wait": (_i, [_vp, ctypes.c_uint64, _i, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_double)]),
    "aes_srv_drain": (_i, [_vp, _i]),
    "aes_srv_results": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _i]),
    "aes_srv_stats": (_i, [_vp, ctypes.POINTER(aes_srv_stats_t)]),
    "aes_srv_destroy": (_i, [_vp]),
    "aes_srv_cancel": (_i, [_vp, ctypes.c_uint64]),
    "aes_srv_register": (_i, [_vp, _vp, _sz]),
    "aes_srv_unregister": (_i, [_vp, _vp]),
    "aes_test_fail_allocs": (_i, [_i, _i]),
    "aes_device_table": (_i, [_i, _u32p]),
}


def lib() -> ctypes.CDLL:
    """The loaded native library (loaded once; raises if it was not built)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise RuntimeError(
                        f"{LIB_PATH} is missing: build it with `python -m paper_1902_05234_gb300.build` "
                        "(there is no CPU fallback)")
                h = ctypes.CDLL(LIB_PATH)
                for name, (res, args) in _SIGNATURES.items():
                    fn = getattr(h, name, None)
                    if fn is None:
                        continue
                    fn.restype = res
                    fn.argtypes = args
                _lib = h
    return _lib


def declared_symbols() -> list[str]:
    """Function names declared in include/aesgb.h (parsed from the header)."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "aesgb.h")
    text = open(hdr).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(aes_[a-z0-9_]+)\s*\(", text)))


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take a pointer of {type(x)!r}")


def _stream(s) -> int:
    if s is None:
        torch = sys.modules.get("torch")
        if torch is not None and torch.cuda.is_initialized():
            # the raw handle of torch's current stream, without building a
            # Stream object (that costs several microseconds per call)
            return int(torch._C._cuda_getCurrentRawStream(torch._C._cuda_getDevice()))
        return 0
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _rk_arg(rk) -> ctypes.Array:
    a = np.ascontiguousarray(np.asarray(rk, dtype=np.uint32))
    return a.ctypes.data_as(_u32p), a


def _check(st: int, where: str) -> int:
    if st < 0:
        raise AesError(st, where)
    return st


# ---------------------------------------------------------------------------
# C ABI, same names
# ---------------------------------------------------------------------------

def aes_status_str(status: int) -> str:
    return lib().aes_status_str(int(status)).decode()


def aes_version() -> int:
    return int(lib().aes_version())


def aes_expand_key(keybits: int, key) -> tuple[np.ndarray, np.ndarray, int]:
    """Returns (rk_enc, rk_dec, nrounds); rk_* are uint32[60] host arrays."""
    k = np.ascontiguousarray(np.frombuffer(bytes(key), np.uint8) if isinstance(key, (bytes, bytearray))
                             else np.asarray(key, np.uint8))
    if k.size * 8 != keybits:
        raise AesError(-1, f"aes_expand_key: key has {k.size} bytes for {keybits} bits")
    enc = np.zeros(60, np.uint32)
    dec = np.zeros(60, np.uint32)
    nr = _check(lib().aes_expand_key(int(keybits), k.ctypes.data_as(_u8p),
                                     enc.ctypes.data_as(_u32p), dec.ctypes.data_as(_u32p)),
                "aes_expand_key")
    return enc, dec, nr


def aes_ecb_encrypt(rk, nrounds: int, in_, out, nblocks: int, stream=None) -> None:
    p, _keep = _rk_arg(rk)
    _check(lib().aes_ecb_encrypt(p, int(nrounds), _ptr(in_), _ptr(out), int(nblocks), _stream(stream)),
           "aes_ecb_encrypt")


def aes_ecb_decrypt(rk_dec, nrounds: int, in_, out, nblocks: int, stream=None) -> None:
    p, _keep = _rk_arg(rk_dec)
    _check(lib().aes_ecb_decrypt(p, int(nrounds), _ptr(in_), _ptr(out), int(nblocks), _stream(stream)),
           "aes_ecb_decrypt")


def make_cfg(threads=1024, blocks_per_thread=2, layout=LAYOUT_R4, ctas_per_sm=1) -> aes_launch_cfg:
    return aes_launch_cfg(int(threads), int(blocks_per_thread), int(layout), int(ctas_per_sm))


def aes_ecb_crypt_cfg(direction: int, rk, nrounds: int, in_, out, nblocks: int, cfg: aes_launch_cfg,
                      stream=None) -> None:
    p, _keep = _rk_arg(rk)
    _check(lib().aes_ecb_crypt_cfg(int(direction), p, int(nrounds), _ptr(in_), _ptr(out), int(nblocks),
                                   ctypes.byref(cfg), _stream(stream)), "aes_ecb_crypt_cfg")


def aes_ecb_get_cfg(direction: int, nrounds: int, nblocks: int) -> aes_launch_cfg:
    c = aes_launch_cfg()
    _check(lib().aes_ecb_get_cfg(int(direction), int(nrounds), int(nblocks), ctypes.byref(c)),
           "aes_ecb_get_cfg")
    return c


def aes_device_sm_count(device: int = 0) -> int:
    return _check(lib().aes_device_sm_count(int(device)), "aes_device_sm_count")


def aes_host_table(which: int) -> np.ndarray:
    out = np.zeros(256, np.uint32)
    _check(lib().aes_host_table(int(which), out.ctypes.data_as(_u32p)), "aes_host_table")
    return out


def aes_device_table(which: int) -> np.ndarray:
    out = np.zeros(256, np.uint32)
    _check(lib().aes_device_table(int(which), out.ctypes.data_as(_u32p)), "aes_device_table")
    return out


def aes_ecb_host(direction: int, rk, nrounds: int, host_in, host_out, nblocks: int, dev_buf,
                 dev_buf_bytes: int, stream=None) -> None:
    p, _keep = _rk_arg(rk)
    _check(lib().aes_ecb_host(int(direction), p, int(nrounds), _ptr(host_in), _ptr(host_out), int(nblocks),
                              _ptr(dev_buf), int(dev_buf_bytes), _stream(stream)), "aes_ecb_host")


def aes_tune_ecb(direction: int, nrounds: int, rk, in_, out, nblocks: int, stream=None) -> aes_launch_cfg:
    p, _keep = _rk_arg(rk)
    c = aes_launch_cfg()
    _check(lib().aes_tune_ecb(int(direction), int(nrounds), p, _ptr(in_), _ptr(out), int(nblocks),
                              _stream(stream), ctypes.byref(c)), "aes_tune_ecb")
    return c


def aes_tune(direction: int, nrounds: int, bytes_hint: int, stream=None) -> None:
    _check(lib().aes_tune(int(direction), int(nrounds), int(bytes_hint), _stream(stream)), "aes_tune")


def aes_tune_batch(desc_dev, n: int, ws, ws_bytes: int, stream=None) -> aes_batch_cfg:
    c = aes_batch_cfg()
    _check(lib().aes_tune_batch(_ptr(desc_dev), int(n), _ptr(ws), int(ws_bytes), _stream(stream),
                                ctypes.byref(c)), "aes_tune_batch")
    return c


def aes_tune_set_ecb(direction: int, nrounds: int, nblocks: int, cfg: aes_launch_cfg) -> None:
    _check(lib().aes_tune_set_ecb(int(direction), int(nrounds), int(nblocks), ctypes.byref(cfg)),
           "aes_tune_set_ecb")


def aes_batch_get_cfg(n: int) -> aes_batch_cfg:
    c = aes_batch_cfg()
    _check(lib().aes_batch_get_cfg(int(n), ctypes.byref(c)), "aes_batch_get_cfg")
    return c


def aes_tune_save(path: str) -> None:
    _check(lib().aes_tune_save(os.fsencode(path)), "aes_tune_save")


def aes_tune_load(path: str) -> None:
    _check(lib().aes_tune_load(os.fsencode(path)), "aes_tune_load")


def aes_tune_clear() -> None:
    _check(lib().aes_tune_clear(), "aes_tune_clear")


# --- serving ----------------------------------------------------------------

def aes_srv_create(mem_budget_bytes: int, max_keys: int, max_batch: int = 4096, slots: int = 3) -> int:
    h = _vp()
    _check(lib().aes_srv_create(int(mem_budget_bytes), int(max_keys), int(max_batch), int(slots),
                                ctypes.byref(h)), "aes_srv_create")
    return int(h.value)


def aes_srv_put_key(srv: int, key_id: int, keybits: int, key) -> None:
    k = np.ascontiguousarray(np.frombuffer(bytes(key), np.uint8))
    _check(lib().aes_srv_put_key(_vp(srv), int(key_id), int(keybits), k.ctypes.data_as(_u8p)),
           "aes_srv_put_key")


def aes_srv_put_schedule(srv: int, key_id: int, rk_enc, rk_dec, nrounds: int) -> None:
    pe, _ke = _rk_arg(rk_enc)
    pd, _kd = _rk_arg(rk_dec)
    _check(lib().aes_srv_put_schedule(_vp(srv), int(key_id), pe, pd, int(nrounds)), "aes_srv_put_schedule")


def aes_srv_set_device_timing(srv: int, on: bool) -> None:
    _check(lib().aes_srv_set_device_timing(_vp(srv), 1 if on else 0), "aes_srv_set_device_timing")


def aes_srv_submit(srv: int, key_id: int, direction: int, in_dev, out_dev, nbytes: int) -> int:
    t = ctypes.c_uint64()
    _check(lib().aes_srv_submit(_vp(srv), int(key_id), int(direction), _ptr(in_dev), _ptr(out_dev),
                                int(nbytes), ctypes.byref(t)), "aes_srv_submit")
    return int(t.value)


def aes_srv_submit_many(srv: int, key_ids, dirs, in_devs, out_devs, nbytes, arrival_offsets_s=None):
    """Returns (status, tickets uint64[n])."""
    n = len(nbytes)
    k = np.ascontiguousarray(key_ids, np.int32)
    d = np.ascontiguousarray(dirs, np.int32)
    i = np.ascontiguousarray(in_devs, np.uint64)
    o = np.ascontiguousarray(out_devs, np.uint64)
    b = np.ascontiguousarray(nbytes, np.uint64)
    a = None if arrival_offsets_s is None else np.ascontiguousarray(arrival_offsets_s, np.float64)
    t = np.zeros(n, np.uint64)
    st = lib().aes_srv_submit_many(_vp(srv), n, k.ctypes.data, d.ctypes.data, i.ctypes.data, o.ctypes.data,
                                   b.ctypes.data, None if a is None else a.ctypes.data, t.ctypes.data)
    return int(st), t


def aes_srv_poll(srv: int, ticket: int):
    done, st, lat = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().aes_srv_poll(_vp(srv), int(ticket), ctypes.byref(done), ctypes.byref(st), ctypes.byref(lat)),
           "aes_srv_poll")
    return bool(done.value), int(st.value), float(lat.value)


def aes_srv_wait(srv: int, ticket: int, timeout_ms: int = 10000):
    st, lat = ctypes.c_int(), ctypes.c_double()
    _check(lib().aes_srv_wait(_vp(srv), int(ticket), int(timeout_ms), ctypes.byref(st), ctypes.byref(lat)),
           "aes_srv_wait")
    return int(st.value), float(lat.value)


def aes_srv_drain(srv: int, timeout_ms: int = 60000) -> None:
    _check(lib().aes_srv_drain(_vp(srv), int(timeout_ms)), "aes_srv_drain")


def aes_srv_results(srv: int, tickets, release: bool = False):
    """Returns (status int32[n], latency_s float64[n], queue_s float64[n])."""
    t = np.ascontiguousarray(tickets, np.uint64)
    n = t.size
    st = np.zeros(n, np.int32)
    lat = np.zeros(n, np.float64)
    q = np.zeros(n, np.float64)
    _check(lib().aes_srv_results(_vp(srv), n, t.ctypes.data, st.ctypes.data, lat.ctypes.data, q.ctypes.data,
                                 int(bool(release))), "aes_srv_results")
    return st, lat, q


def aes_srv_stats(srv: int) -> dict:
    s = aes_srv_stats_t()
    _check(lib().aes_srv_stats(_vp(srv), ctypes.byref(s)), "aes_srv_stats")
    return s.as_dict()


def aes_srv_cancel(srv: int, ticket: int) -> None:
    """Cancel a queued (not yet launched) request; raises AesError (AES_E_BUSY) once it is launched."""
    _check(lib().aes_srv_cancel(_vp(srv), int(ticket)), "aes_srv_cancel")


def aes_srv_register(srv: int, base_dev, nbytes: int) -> None:
    """Add a device range to the server's registry of allowed request buffers."""
    _check(lib().aes_srv_register(_vp(srv), _ptr(base_dev), int(nbytes)), "aes_srv_register")


def aes_srv_unregister(srv: int, base_dev) -> None:
    _check(lib().aes_srv_unregister(_vp(srv), _ptr(base_dev)), "aes_srv_unregister")


def aes_test_fail_allocs(skip: int, count: int) -> None:
    """Failure injection: of the library's own allocations from now on, the first
    `skip` succeed and the next `count` fail as out of memory (count 0 disarms)."""
    _check(lib().aes_test_fail_allocs(int(skip), int(count)), "aes_test_fail_allocs")


def aes_srv_destroy(srv: int) -> None:
    _check(lib().aes_srv_destroy(_vp(srv)), "aes_srv_destroy")


def aes_ecb_host_direct(direction: int, rk, nrounds: int, host_in, host_out, nblocks: int, stream=None) -> None:
    p, _keep = _rk_arg(rk)
    _check(lib().aes_ecb_host_direct(int(direction), p, int(nrounds), _ptr(host_in), _ptr(host_out), int(nblocks),
                                     _stream(stream)), "aes_ecb_host_direct")


def aes_ecb_crypt_ct(direction: int, rk, nrounds: int, in_, out, nblocks: int, stream=None) -> None:
    p, _keep = _rk_arg(rk)
    _check(lib().aes_ecb_crypt_ct(int(direction), p, int(nrounds), _ptr(in_), _ptr(out), int(nblocks),
                                  _stream(stream)), "aes_ecb_crypt_ct")


def aes_wait_timeouts() -> int:
    """Bounded device waits that ran out since the last call (reading resets it)."""
    v = ctypes.c_ulonglong()
    _check(lib().aes_wait_timeouts(ctypes.byref(v)), "aes_wait_timeouts")
    return v.value


def aes_debug_bounds_violations() -> int:
    """Failed index checks since the last call (debug library only; reading resets it).

    Raises AesError (AES_E_CONFIG) when the loaded library is the release build.
    """
    v = ctypes.c_ulonglong()
    _check(lib().aes_debug_bounds_violations(ctypes.byref(v)), "aes_debug_bounds_violations")
    return v.value


def aes_debug_batch_coverage() -> tuple[int, int, int]:
    """(chunks taken once, more than once, past the tags) since the last call (debug library only)."""
    v = [ctypes.c_ulonglong() for _ in range(3)]
    _check(lib().aes_debug_batch_coverage(*[ctypes.byref(x) for x in v]), "aes_debug_batch_coverage")
    return v[0].value, v[1].value, v[2].value


def aes_tma_selftest_timeout(in_, out, nblocks: int, stream=None) -> None:
    """Failure-detection test hook: a TMA-staged launch whose waits must run out."""
    _check(lib().aes_tma_selftest_timeout(_ptr(in_), _ptr(out), int(nblocks), _stream(stream)),
           "aes_tma_selftest_timeout")


def aes_ct_ops_per_block(direction: int, nrounds: int) -> float:
    """Logic operations per 16-byte block of the constant-time kernel."""
    v = ctypes.c_double()
    _check(lib().aes_ct_ops_per_block(int(direction), int(nrounds), ctypes.byref(v)), "aes_ct_ops_per_block")
    return v.value


def aes_ct_selftest_host(direction: int, rk, nrounds: int, data: np.ndarray) -> np.ndarray:
    """Run the bitsliced cipher's code on the host (test hook) over host bytes."""
    p, _keep = _rk_arg(rk)
    src = np.ascontiguousarray(data, np.uint8)
    out = np.zeros_like(src)
    _check(lib().aes_ct_selftest_host(int(direction), p, int(nrounds), src.ctypes.data, out.ctypes.data,
                                      src.size // 16), "aes_ct_selftest_host")
    return out


def aes_cfb_decrypt(rk_enc, nrounds: int, iv, in_, out, nblocks: int, stream=None) -> None:
    p, _keep = _rk_arg(rk_enc)
    v = _block16(iv)
    _check(lib().aes_cfb_decrypt(p, int(nrounds), v.ctypes.data_as(_u8p), _ptr(in_), _ptr(out), int(nblocks),
                                 _stream(stream)), "aes_cfb_decrypt")


def _block16(b):
    a = np.ascontiguousarray(np.frombuffer(bytes(b), np.uint8) if isinstance(b, (bytes, bytearray))
                             else np.asarray(b, np.uint8))
    if a.size != 16:
        raise AesError(-1, "a counter block / IV is 16 bytes")
    return a


def aes_ctr_crypt(rk, nrounds: int, ctr0, in_, out, nblocks: int, stream=None) -> None:
    p, _keep = _rk_arg(rk)
    c = _block16(ctr0)
    _check(lib().aes_ctr_crypt(p, int(nrounds), c.ctypes.data_as(_u8p), _ptr(in_), _ptr(out), int(nblocks),
                               _stream(stream)), "aes_ctr_crypt")


def aes_cbc_decrypt(rk_dec, nrounds: int, iv, in_, out, nblocks: int, stream=None) -> None:
    p, _keep = _rk_arg(rk_dec)
    v = _block16(iv)
    _check(lib().aes_cbc_decrypt(p, int(nrounds), v.ctypes.data_as(_u8p), _ptr(in_), _ptr(out), int(nblocks),
                                 _stream(stream)), "aes_cbc_decrypt")


def aes_calibrate_logic_rate(sink_dev, sink_bytes: int, stream=None) -> tuple[float, float]:
    """(operations, seconds) of the three-input logic (LOP3) calibration kernel."""
    n, t = ctypes.c_double(), ctypes.c_double()
    _check(lib().aes_calibrate_logic_rate(_ptr(sink_dev), int(sink_bytes), _stream(stream), ctypes.byref(n),
                                          ctypes.byref(t)), "aes_calibrate_logic_rate")
    return float(n.value), float(t.value)


def aes_calibrate_lookup_rate(sink_dev, sink_bytes: int, stream=None) -> tuple[float, float]:
    """(lookups, seconds) of the shared-memory lookup calibration kernel."""
    n, t = ctypes.c_double(), ctypes.c_double()
    _check(lib().aes_calibrate_lookup_rate(_ptr(sink_dev), int(sink_bytes), _stream(stream), ctypes.byref(n),
                                           ctypes.byref(t)), "aes_calibrate_lookup_rate")
    return float(n.value), float(t.value)


def aes_shutdown() -> None:
    _check(lib().aes_shutdown(), "aes_shutdown")


def aes_batch_workspace_bytes(n: int) -> int:
    return int(lib().aes_batch_workspace_bytes(int(n)))


def aes_ecb_batch_ws(desc_dev, n: int, ws, ws_bytes: int, status_dev=None, cfg: aes_batch_cfg | None = None,
                     stream=None) -> None:
    _check(lib().aes_ecb_batch_ws(_ptr(desc_dev), int(n), _ptr(ws), int(ws_bytes), _ptr(status_dev),
                                  ctypes.addressof(cfg) if cfg is not None else None, _stream(stream)),
           "aes_ecb_batch_ws")


def aes_ecb_batch(desc_dev, n: int, stream=None) -> None:
    _check(lib().aes_ecb_batch(_ptr(desc_dev), int(n), _stream(stream)), "aes_ecb_batch")


def aes_ecb_batch_ex(desc_dev, n: int, status_dev=None, stream=None) -> None:
    _check(lib().aes_ecb_batch_ex(_ptr(desc_dev), int(n), _ptr(status_dev), _stream(stream)), "aes_ecb_batch_ex")


def aes_ecb_batch_noalloc(desc_dev, n: int, status_dev=None, stream=None) -> None:
    """Batched ECB with the library's fixed device scratch (no allocation at
    all); at most AES_BATCH_NOALLOC_MAX_DESCS descriptors, calls must not
    overlap on the GPU."""
    _check(lib().aes_ecb_batch_noalloc(_ptr(desc_dev), int(n), _ptr(status_dev), _stream(stream)),
           "aes_ecb_batch_noalloc")


AES_BATCH_NOALLOC_MAX_DESCS = 16384


def aes_batch_graph_create(desc_dev, n: int, ws, ws_bytes: int, status_dev=None,
                           cfg: aes_batch_cfg | None = None) -> int:
    h = _vp()
    _check(lib().aes_batch_graph_create(_ptr(desc_dev), int(n), _ptr(ws), int(ws_bytes), _ptr(status_dev),
                                        ctypes.addressof(cfg) if cfg is not None else None, ctypes.byref(h)),
           "aes_batch_graph_create")
    return int(h.value)


def aes_batch_graph_launch(graph: int, stream=None) -> None:
    _check(lib().aes_batch_graph_launch(_vp(graph), _stream(stream)), "aes_batch_graph_launch")


def aes_batch_graph_destroy(graph: int) -> None:
    _check(lib().aes_batch_graph_destroy(_vp(graph)), "aes_batch_graph_destroy")


def make_batch_cfg(threads=512, blocks_per_thread=1, chunk_passes=32, ctas_per_sm=1, layout_enc=LAYOUT_R4,
                   layout_dec=LAYOUT_R2) -> aes_batch_cfg:
    return aes_batch_cfg(int(threads), int(blocks_per_thread), int(chunk_passes), int(ctas_per_sm),
                         int(layout_enc), int(layout_dec))


def pack_descs(rk, in_, out, nblocks, nrounds, direction) -> np.ndarray:
    """Pack parallel sequences (device addresses as ints) into an aes_desc table."""
    t = np.zeros(len(nblocks), DESC_DTYPE)
    t["rk"], t["in"], t["out"] = rk, in_, out
    t["nblocks"], t["nrounds"], t["dir"] = nblocks, nrounds, direction
    return t


# ---------------------------------------------------------------------------
# tensor conveniences (still one C call each)
# ---------------------------------------------------------------------------

def ecb_encrypt(key, data, out=None, stream=None):
    """Encrypt a CUDA uint8 tensor (length a multiple of 16) with a raw key."""
    return _ecb_tensor(ENCRYPT, key, data, out, stream)


def ecb_decrypt(key, data, out=None, stream=None):
    return _ecb_tensor(DECRYPT, key, data, out, stream)


def _ecb_tensor(direction, key, data, out, stream):
    import torch
    kb = 8 * len(bytes(key)) if isinstance(key, (bytes, bytearray)) else 8 * int(np.asarray(key).size)
    enc, dec, nr = aes_expand_key(kb, key)
    if data.dtype != torch.uint8 or not data.is_cuda or data.numel() % 16:
        raise AesError(-1, "ecb: need a CUDA uint8 tensor with a multiple of 16 bytes")
    if out is None:
        out = torch.empty_like(data)
    n = data.numel() // 16
    if direction == ENCRYPT:
        aes_ecb_encrypt(enc, nr, data, out, n, stream)
    else:
        aes_ecb_decrypt(dec, nr, data, out, n, stream)
    return out
