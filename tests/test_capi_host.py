"""Host-side tests of the C-ABI library (no GPU): it loads, exports every
symbol include/aesgb.h declares, and its host logic (key schedule, tables,
argument checks that run before any CUDA call) agrees with the oracle."""
import ctypes

import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl


@pytest.fixture(scope="module")
def lib():
    return aesgb.lib()


def test_exports_every_declared_symbol(lib):
    names = aesgb.declared_symbols()
    assert "aes_ecb_encrypt" in names and "aes_expand_key" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for st in range(0, -15, -1):
        s = aesgb.aes_status_str(st)
        assert s and s != "unknown status"
    assert aesgb.aes_status_str(5) == "unknown status"


@pytest.mark.parametrize("keybits", [128, 192, 256])
def test_expand_key_matches_oracle(orc, keybits):
    for seed in range(25):
        key = wl.random_key(keybits, seed)
        enc, dec, nr = aesgb.aes_expand_key(keybits, key)
        w, onr = orc.key_expansion(key)
        assert nr == onr
        nw = 4 * (nr + 1)
        assert enc[:nw].view(np.uint8).tobytes() == w.tobytes()
        dw = orc.eq_inv_schedule(w, nr)
        assert dec[:nw].view(np.uint8).tobytes() == dw.tobytes()


def test_expand_key_errors(lib):
    key = (ctypes.c_uint8 * 32)()
    for bits in (0, 64, 127, 129, 512, -128):
        assert lib.aes_expand_key(bits, key, None, None) == -2
    assert lib.aes_expand_key(128, None, None, None) == -1


def test_host_tables_match_oracle(orc):
    te0, td0 = aesgb.aes_host_table(0), aesgb.aes_host_table(1)
    sb, isb = aesgb.aes_host_table(2), aesgb.aes_host_table(3)
    assert np.array_equal(sb, orc.sbox_table().astype(np.uint32))
    assert np.array_equal(isb, orc.inv_sbox_table().astype(np.uint32))
    for x in range(256):
        # eq (22): T0 column, row r in byte r
        col = orc.ttable(0, x)
        assert int(te0[x]) == int.from_bytes(bytes(col.tolist()), "little")
        # inverse-cipher column: (0e, 09, 0d, 0b) * InvS(x)
        i = orc.inv_sbox(x)
        exp = bytes([orc.gf_mul(0x0E, i), orc.gf_mul(0x09, i), orc.gf_mul(0x0D, i), orc.gf_mul(0x0B, i)])
        assert int(td0[x]) == int.from_bytes(exp, "little")


def test_argument_checks_before_cuda(lib):
    rk = (ctypes.c_uint32 * 60)()
    A = 1 << 20  # fake, never dereferenced: every call below fails validation first
    assert lib.aes_ecb_encrypt(rk, 11, A, A + 4096, 4, None) == -3      # nrounds
    assert lib.aes_ecb_decrypt(rk, 9, A, A + 4096, 4, None) == -3
    assert lib.aes_ecb_encrypt(None, 10, A, A + 4096, 4, None) == -1    # null rk
    assert lib.aes_ecb_encrypt(rk, 10, A, A + 4096, 0, None) == 0       # empty: no-op
    assert lib.aes_ecb_encrypt(rk, 10, 0, A, 4, None) == -1             # null in
    assert lib.aes_ecb_encrypt(rk, 10, A + 8, A + 4096, 4, None) == -4  # misaligned
    assert lib.aes_ecb_encrypt(rk, 10, A, A + 4104, 4, None) == -4
    assert lib.aes_ecb_encrypt(rk, 10, A, A + 16, 4, None) == -5        # partial overlap
    assert lib.aes_ecb_encrypt(rk, 10, A + 48, A, 4, None) == -5
    assert lib.aes_ecb_encrypt(rk, 10, A, A + 4096, 1 << 61, None) == -1  # nblocks*16 overflows
    bad = aesgb.make_cfg(threads=1000)
    assert lib.aes_ecb_crypt_cfg(0, rk, 10, A, A + 4096, 4, ctypes.byref(bad), None) == -12
    bad = aesgb.make_cfg(threads=1024, blocks_per_thread=4)
    assert lib.aes_ecb_crypt_cfg(0, rk, 10, A, A + 4096, 4, ctypes.byref(bad), None) == -12
    bad = aesgb.make_cfg(blocks_per_thread=3)
    assert lib.aes_ecb_crypt_cfg(1, rk, 10, A, A + 4096, 4, ctypes.byref(bad), None) == -12
    assert lib.aes_ecb_crypt_cfg(2, rk, 10, A, A + 4096, 4, ctypes.byref(aesgb.make_cfg()), None) == -1


def test_tune_without_buffers_checks_arguments_first(lib):
    """aes_tune refuses a bad direction, round count or size before it
    allocates or touches a device."""
    assert lib.aes_tune(2, 10, 1 << 20, None) == -1
    assert lib.aes_tune(0, 11, 1 << 20, None) == -3
    assert lib.aes_tune(0, 10, 8, None) == -1


def test_debug_counter_is_debug_build_only(lib):
    """The release library has no index checks: its counter entry point
    answers AES_E_CONFIG (with a zero count) without touching the device."""
    v = ctypes.c_ulonglong(7)
    assert lib.aes_debug_bounds_violations(ctypes.byref(v)) == -12
    assert v.value == 0
    assert lib.aes_debug_bounds_violations(None) == -1
    c = [ctypes.c_ulonglong(7) for _ in range(3)]
    assert lib.aes_debug_batch_coverage(*[ctypes.byref(x) for x in c]) == -12
    assert [x.value for x in c] == [0, 0, 0]


def test_fail_allocs_hook_arguments(lib):
    """The allocation-failure injector is host state only: setting and
    clearing it needs no device; a negative count is an argument error."""
    assert lib.aes_test_fail_allocs(-1, 1) == -1
    assert lib.aes_test_fail_allocs(0, -1) == -1
    assert lib.aes_test_fail_allocs(2, 3) == 0
    assert lib.aes_test_fail_allocs(0, 0) == 0


def test_batch_size_above_the_maximum_is_refused_before_any_work(lib):
    """More than AES_BATCH_MAX_DESCS (2^28) descriptors: AES_E_RANGE from every
    batch entry point, before any allocation or launch (fake, never used
    addresses; no device is needed)."""
    A = 1 << 20
    n = (1 << 28) + 1
    assert lib.aes_ecb_batch_ws(A, n, A, 1 << 40, None, None, None) == -10
    assert lib.aes_ecb_batch(A, n, None) == -10
    assert lib.aes_ecb_batch_ex(A, n, None, None) == -10
    g = ctypes.c_void_p()
    assert lib.aes_batch_graph_create(A, n, A, 1 << 40, None, None, ctypes.byref(g)) == -10
    srv = ctypes.c_void_p()
    assert lib.aes_srv_create(1 << 30, 4, n, 2, ctypes.byref(srv)) == -10


def test_server_calls_reject_null_handle(lib):
    rk = (ctypes.c_uint32 * 60)()
    assert lib.aes_srv_put_schedule(None, 0, rk, rk, 10) == -1
    assert lib.aes_srv_set_device_timing(None, 1) == -1
    assert lib.aes_srv_cancel(None, 1) == -1
    assert lib.aes_srv_register(None, 1 << 20, 4096) == -1
    assert lib.aes_srv_unregister(None, 1 << 20) == -1


def test_tune_cache_entries_of_another_device_model_are_not_applied(tmp_path):
    """Cache lines carry the device's model tag: an entry written for another
    model (tag deadbeef) or in the untagged older format is not used."""
    aesgb.aes_tune_clear()
    try:
        c = aesgb.make_cfg(threads=256, blocks_per_thread=4, layout=aesgb.LAYOUT_R1, ctas_per_sm=0)
        aesgb.aes_tune_set_ecb(1, 12, 1 << 22, c)
        path = tmp_path / "tune.txt"
        aesgb.aes_tune_save(str(path))
        mine = [ln for ln in path.read_text().splitlines() if ln.startswith("ecb ")]
        assert len(mine) == 1
        fields = mine[0].split()
        other = " ".join(["ecb", "deadbeef"] + fields[2:])
        untagged = " ".join(["ecb"] + fields[2:])
        path.write_text("# aesgb tune cache v2\n" + other + "\n" + untagged + "\n")
        aesgb.aes_tune_clear()
        aesgb.aes_tune_load(str(path))
        assert aesgb.aes_ecb_get_cfg(1, 12, 1 << 22).layout == aesgb.LAYOUT_R4   # the default
        path.write_text("# aesgb tune cache v2\n" + mine[0] + "\n")
        aesgb.aes_tune_load(str(path))
        assert aesgb.aes_ecb_get_cfg(1, 12, 1 << 22).as_dict() == c.as_dict()
    finally:
        aesgb.aes_tune_clear()


def test_default_cfg_is_valid():
    for d in (0, 1):
        for nr in (10, 12, 14):
            c = aesgb.aes_ecb_get_cfg(d, nr, 1 << 20)
            assert c.threads % 32 == 0 and c.blocks_per_thread in (1, 2, 4, 8)


def test_tune_cache_file_roundtrip(tmp_path):
    """Tuned entries set by hand survive save / clear / load (host logic)."""
    aesgb.aes_tune_clear()
    try:
        c = aesgb.make_cfg(threads=256, blocks_per_thread=4, layout=aesgb.LAYOUT_R1, ctas_per_sm=0)
        aesgb.aes_tune_set_ecb(1, 12, 1 << 22, c)
        got = aesgb.aes_ecb_get_cfg(1, 12, 1 << 22)
        assert got.as_dict() == c.as_dict()
        other = aesgb.aes_ecb_get_cfg(0, 12, 1 << 22)          # other direction: default
        assert other.layout == aesgb.LAYOUT_R4
        path = str(tmp_path / "tune.txt")
        aesgb.aes_tune_save(path)
        text = open(path).read()
        assert "ecb" in text and " 256 4 1 0" in text
        aesgb.aes_tune_clear()
        assert aesgb.aes_ecb_get_cfg(1, 12, 1 << 22).layout == aesgb.LAYOUT_R4
        aesgb.aes_tune_load(path)
        assert aesgb.aes_ecb_get_cfg(1, 12, 1 << 22).as_dict() == c.as_dict()
        # a different size class is not affected: its default (small buffers: R2
        # tables, 256 threads x 2 blocks, as many CTAs per SM as fit)
        small = aesgb.aes_ecb_get_cfg(1, 12, 1 << 10)
        assert (small.layout, small.threads, small.blocks_per_thread, small.ctas_per_sm) == \
            (aesgb.LAYOUT_R2, 256, 2, 0)
        with pytest.raises(aesgb.AesError):
            aesgb.aes_tune_set_ecb(0, 10, 100, aesgb.make_cfg(threads=2048))
    finally:
        aesgb.aes_tune_clear()


def test_batch_default_cfg_valid():
    c = aesgb.aes_batch_get_cfg(4096)
    assert c.threads <= 512 and c.blocks_per_thread in (1, 2, 4) and c.chunk_passes >= 1


def test_server_create_fails_cleanly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(aesgb.AesError):
        aesgb.aes_srv_create(1 << 20, 4, 8, 1)
    aesgb.aes_srv_destroy(0)          # a null handle is a no-op
