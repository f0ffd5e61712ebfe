"""CPU oracle for AES (FIPS-197 reading of Wang & Chu, arXiv 1902.05234).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only code allowed to import this package.
The GPU library neither imports nor links it, and the two share no code.

Every function here is a thin ctypes wrapper over ``aes_oracle.c``; the C file
carries the citations of the paper's definitions and equations.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_u8 = ctypes.c_uint8
_u8p = ctypes.POINTER(ctypes.c_uint8)
_lock = threading.Lock()
_libs: dict[str, ctypes.CDLL] = {}


def _declare(lib: ctypes.CDLL) -> ctypes.CDLL:
    sig = {
        "orc_gf_add": (_u8, [_u8, _u8]),
        "orc_clmul": (ctypes.c_uint16, [_u8, _u8]),
        "orc_poly_mod": (_u8, [ctypes.c_uint16]),
        "orc_gf_mul": (_u8, [_u8, _u8]),
        "orc_xtime": (_u8, [_u8]),
        "orc_gf_inv": (_u8, [_u8]),
        "orc_sbox": (_u8, [_u8]),
        "orc_inv_sbox": (_u8, [_u8]),
        "orc_mix_matrix": (None, [ctypes.c_int, _u8p]),
        "orc_round": (None, [_u8p, _u8p, _u8p]),
        "orc_tround": (None, [_u8p, _u8p, _u8p]),
        "orc_ttable": (None, [ctypes.c_int, _u8, _u8p]),
        "orc_sub_bytes": (None, [_u8p]),
        "orc_shift_rows": (None, [_u8p]),
        "orc_mix_columns": (None, [_u8p]),
        "orc_inv_mix_columns": (None, [_u8p]),
        "orc_nrounds": (ctypes.c_int, [ctypes.c_int]),
        "orc_key_expansion": (ctypes.c_int, [ctypes.c_int, _u8p, _u8p]),
        "orc_cipher": (None, [_u8p, ctypes.c_int, _u8p, _u8p]),
        "orc_inv_cipher": (None, [_u8p, ctypes.c_int, _u8p, _u8p]),
        "orc_eq_inv_schedule": (None, [_u8p, ctypes.c_int, _u8p]),
        "orc_eq_inv_cipher": (None, [_u8p, ctypes.c_int, _u8p, _u8p]),
        "orc_ecb": (None, [ctypes.c_int, _u8p, ctypes.c_int, _u8p, _u8p, ctypes.c_size_t]),
        "orc_ecb_mt": (ctypes.c_int, [ctypes.c_int, _u8p, ctypes.c_int, _u8p, _u8p,
                                      ctypes.c_size_t, ctypes.c_int]),
        "orc_ctr_block": (None, [_u8p, ctypes.c_uint64, _u8p]),
        "orc_ctr": (None, [_u8p, ctypes.c_int, _u8p, _u8p, _u8p, ctypes.c_size_t]),
        "orc_cbc_encrypt": (None, [_u8p, ctypes.c_int, _u8p, _u8p, _u8p, ctypes.c_size_t]),
        "orc_cbc_decrypt": (None, [_u8p, ctypes.c_int, _u8p, _u8p, _u8p, ctypes.c_size_t]),
        "orc_cfb_encrypt": (None, [_u8p, ctypes.c_int, _u8p, _u8p, _u8p, ctypes.c_size_t]),
        "orc_cfb_decrypt": (None, [_u8p, ctypes.c_int, _u8p, _u8p, _u8p, ctypes.c_size_t]),
        "orc_mutant_id": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (building first if needed) the oracle library at ``path``."""
    with _lock:
        key = path or _build.LIB
        if key not in _libs:
            if path is None:
                _build.build()
            _libs[key] = _declare(ctypes.CDLL(key))
        return _libs[key]


def _p(a: np.ndarray):
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(_u8p)


def _bytes(x) -> np.ndarray:
    return np.ascontiguousarray(np.frombuffer(bytes(x), dtype=np.uint8)
                                if isinstance(x, (bytes, bytearray)) else np.asarray(x, np.uint8))


class Oracle:
    """numpy-facing wrapper over one loaded oracle library (normal or mutant)."""

    def __init__(self, lib: ctypes.CDLL | None = None):
        self.lib = lib or load()

    # GF(2^8) and S-box -------------------------------------------------------
    def gf_add(self, a, b): return int(self.lib.orc_gf_add(a, b))
    def clmul(self, a, b): return int(self.lib.orc_clmul(a, b))
    def poly_mod(self, p): return int(self.lib.orc_poly_mod(p))
    def gf_mul(self, a, b): return int(self.lib.orc_gf_mul(a, b))
    def xtime(self, a): return int(self.lib.orc_xtime(a))
    def gf_inv(self, a): return int(self.lib.orc_gf_inv(a))
    def sbox(self, x): return int(self.lib.orc_sbox(x))
    def inv_sbox(self, y): return int(self.lib.orc_inv_sbox(y))

    def sbox_table(self) -> np.ndarray:
        return np.array([self.sbox(x) for x in range(256)], np.uint8)

    def inv_sbox_table(self) -> np.ndarray:
        return np.array([self.inv_sbox(x) for x in range(256)], np.uint8)

    def mix_matrix(self, inverse: bool = False) -> np.ndarray:
        out = np.zeros(16, np.uint8)
        self.lib.orc_mix_matrix(int(inverse), _p(out))
        return out.reshape(4, 4)

    def ttable(self, k: int, w: int) -> np.ndarray:
        out = np.zeros(4, np.uint8)
        self.lib.orc_ttable(k, w, _p(out))
        return out

    # single-state transformations ----------------------------------------
    def _state_op(self, fn, block):
        b = _bytes(block).copy()
        fn(_p(b))
        return b

    def sub_bytes(self, block): return self._state_op(self.lib.orc_sub_bytes, block)
    def shift_rows(self, block): return self._state_op(self.lib.orc_shift_rows, block)
    def mix_columns(self, block): return self._state_op(self.lib.orc_mix_columns, block)
    def inv_mix_columns(self, block): return self._state_op(self.lib.orc_inv_mix_columns, block)

    def round(self, block, rk):
        i, k, o = _bytes(block), _bytes(rk), np.zeros(16, np.uint8)
        self.lib.orc_round(_p(i), _p(k), _p(o))
        return o

    def tround(self, block, rk):
        i, k, o = _bytes(block), _bytes(rk), np.zeros(16, np.uint8)
        self.lib.orc_tround(_p(i), _p(k), _p(o))
        return o

    # key schedule and ciphers ---------------------------------------------
    def nrounds(self, keybits: int) -> int:
        return int(self.lib.orc_nrounds(keybits))

    def key_expansion(self, key) -> tuple[np.ndarray, int]:
        k = _bytes(key)
        nr = self.nrounds(8 * k.size)
        if nr < 0:
            raise ValueError(f"key of {k.size} bytes")
        w = np.zeros(16 * (nr + 1), np.uint8)
        got = self.lib.orc_key_expansion(8 * k.size, _p(k), _p(w))
        assert got == nr
        return w, nr

    def eq_inv_schedule(self, w: np.ndarray, nr: int) -> np.ndarray:
        dw = np.zeros_like(w)
        self.lib.orc_eq_inv_schedule(_p(np.ascontiguousarray(w)), nr, _p(dw))
        return dw

    def cipher(self, w, nr, block):
        i, o = _bytes(block), np.zeros(16, np.uint8)
        self.lib.orc_cipher(_p(np.ascontiguousarray(w)), nr, _p(i), _p(o))
        return o

    def inv_cipher(self, w, nr, block):
        i, o = _bytes(block), np.zeros(16, np.uint8)
        self.lib.orc_inv_cipher(_p(np.ascontiguousarray(w)), nr, _p(i), _p(o))
        return o

    def eq_inv_cipher(self, dw, nr, block):
        i, o = _bytes(block), np.zeros(16, np.uint8)
        self.lib.orc_eq_inv_cipher(_p(np.ascontiguousarray(dw)), nr, _p(i), _p(o))
        return o

    # modes -------------------------------------------------------------------
    def ecb(self, direction: int, key, data, nthreads: int = 1) -> np.ndarray:
        """ECB over whole 16-byte blocks; direction 0 = encrypt, 1 = decrypt."""
        w, nr = self.key_expansion(key)
        src = _bytes(data)
        if src.size % 16:
            raise ValueError("ECB takes whole 16-byte blocks")
        out = np.empty_like(src)
        if nthreads > 1:
            self.lib.orc_ecb_mt(direction, _p(w), nr, _p(src), _p(out), src.size // 16, nthreads)
        else:
            self.lib.orc_ecb(direction, _p(w), nr, _p(src), _p(out), src.size // 16)
        return out

    def ecb_encrypt(self, key, data, nthreads: int = 1):
        return self.ecb(0, key, data, nthreads)

    def ecb_decrypt(self, key, data, nthreads: int = 1):
        return self.ecb(1, key, data, nthreads)

    def ctr_block(self, ctr0, i: int) -> np.ndarray:
        c, o = _bytes(ctr0), np.zeros(16, np.uint8)
        self.lib.orc_ctr_block(_p(c), i, _p(o))
        return o

    def ctr(self, key, ctr0, data) -> np.ndarray:
        w, nr = self.key_expansion(key)
        src, c = _bytes(data), _bytes(ctr0)
        out = np.empty_like(src)
        self.lib.orc_ctr(_p(w), nr, _p(c), _p(src), _p(out), src.size // 16)
        return out

    def cbc_encrypt(self, key, iv, data) -> np.ndarray:
        w, nr = self.key_expansion(key)
        src, v = _bytes(data), _bytes(iv)
        out = np.empty_like(src)
        self.lib.orc_cbc_encrypt(_p(w), nr, _p(v), _p(src), _p(out), src.size // 16)
        return out

    def cbc_decrypt(self, key, iv, data) -> np.ndarray:
        w, nr = self.key_expansion(key)
        src, v = _bytes(data), _bytes(iv)
        out = np.empty_like(src)
        self.lib.orc_cbc_decrypt(_p(w), nr, _p(v), _p(src), _p(out), src.size // 16)
        return out

    def cfb_encrypt(self, key, iv, data) -> np.ndarray:
        w, nr = self.key_expansion(key)
        src, v = _bytes(data), _bytes(iv)
        out = np.empty_like(src)
        self.lib.orc_cfb_encrypt(_p(w), nr, _p(v), _p(src), _p(out), src.size // 16)
        return out

    def cfb_decrypt(self, key, iv, data) -> np.ndarray:
        w, nr = self.key_expansion(key)
        src, v = _bytes(data), _bytes(iv)
        out = np.empty_like(src)
        self.lib.orc_cfb_decrypt(_p(w), nr, _p(v), _p(src), _p(out), src.size // 16)
        return out
