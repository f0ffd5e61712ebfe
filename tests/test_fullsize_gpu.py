"""Parity at the full workload sizes, in the launch configurations the
benchmark times: the library's default for the size and every candidate the
autotuner can pick (the benchmark tunes before timing).  Sampled windows are
checked against the oracle, properties over the whole buffer on the device.

* single buffers of 4 GiB, AES-128/192/256: 18 windows of 1 MiB (first, last,
  16 seeded random) against the oracle; decrypt(encrypt(x)) == x over all
  4 GiB on the device.
* the 4,096-message batch (5.2 GB): every message equal to the single-buffer
  path; every message up to 64 KiB, and the first and last 2 KiB of every
  larger one, against the oracle.
* the stress case: AES-256 decryption in place over 16 GiB of 64 MiB regions
  cycling uniform random / all-zero / one block repeated; 32 windows of 1 MiB
  (region boundaries included) against the oracle, and every all-zero or
  periodic region decrypted to one repeated block equal to the oracle's
  decryption of that block (ECB's identical-block invariant).
* 1 GiB, AES-128 (the benchmark's workload): every tuner candidate gives the
  same ciphertext (checked against the oracle on windows) and decrypts it back;
  every batch-tuner candidate gives the same 5.2 GB batch output.
* the single-buffer sweep, 1 MiB .. 1 GiB, every key size, both directions:
  whole outputs against the oracle up to 64 MiB, 1 MiB windows above.
* the largest single call: 2^32 + 1 blocks (64 GiB + 16 B) in place, windows
  around block 2^32 against the oracle and back.
* 1 GiB through the other kernels the benchmark times: the constant-time
  kernel (every key size), the TMA-staged layout, the R2 layout, the table in
  registers and 128 B per thread, CTR, CBC and CFB decryption -- oracle
  windows, and round trips over the whole buffer.
"""
import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

GIB = 1 << 30
MIB = 1 << 20


def _fill_random(torch, t, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(wl.BASE_SEED + seed)
    t.random_(0, 256, generator=g)


@pytest.mark.parametrize("keybits", [128, 192, 256])
def test_4gib_single_buffer_windows_and_roundtrip(orc, keybits):
    torch = torch_cuda()
    nbytes = 4 * GIB
    n = nbytes // 16
    x = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    _fill_random(torch, x, 50 + keybits)
    y = torch.empty_like(x)
    key = wl.random_key(keybits, 50).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(keybits, key)
    aesgb.aes_ecb_encrypt(enc, nr, x, y, n)
    torch.cuda.synchronize()
    win = MIB
    g = wl.rng(51)
    starts = [0, nbytes - win] + [int(v) // 16 * 16 for v in g.integers(0, nbytes - win, 16)]
    for s in starts:
        got = y[s:s + win].cpu().numpy()
        exp = orc.ecb(0, key, x[s:s + win].cpu().numpy(), nthreads=16)
        assert np.array_equal(got, exp), f"window at {s}"
    aesgb.aes_ecb_decrypt(dec, nr, y, y, n)       # in place
    torch.cuda.synchronize()
    assert torch.equal(x, y)


def test_batch_4096_messages_fullsize(orc):
    torch = torch_cuda()
    n = 4096
    lengths, keybits, dirs = wl.batch_workload(n)
    offs = np.zeros(n + 1, np.int64)
    np.cumsum(lengths, out=offs[1:])
    total = int(offs[-1])
    src = torch.empty(total, dtype=torch.uint8, device="cuda")
    _fill_random(torch, src, 52)
    dst = torch.full_like(src, 0x5A)
    ref = torch.empty_like(src)
    g = wl.rng(52)
    keys = [g.integers(0, 256, int(kb) // 8, dtype=np.uint8).tobytes() for kb in keybits]
    rks = np.zeros((n, 64), np.uint32)
    nrs = np.zeros(n, np.int64)
    for i in range(n):
        enc, dec, nr = aesgb.aes_expand_key(int(keybits[i]), keys[i])
        rks[i, :60] = enc if dirs[i] == 0 else dec
        nrs[i] = nr
        a, b = src.data_ptr() + int(offs[i]), ref.data_ptr() + int(offs[i])
        (aesgb.aes_ecb_encrypt if dirs[i] == 0 else aesgb.aes_ecb_decrypt)(rks[i, :60], nr, a, b,
                                                                         int(lengths[i]) // 16)
    rk_dev = torch.from_numpy(rks.view(np.uint8).reshape(-1)).cuda()
    table = aesgb.pack_descs(rk_dev.data_ptr() + 256 * np.arange(n, dtype=np.uint64),
                             src.data_ptr() + offs[:-1].astype(np.uint64),
                             dst.data_ptr() + offs[:-1].astype(np.uint64), lengths // 16, nrs, dirs)
    desc = torch.from_numpy(table.view(np.uint8).copy()).cuda()
    ws_bytes = aesgb.aes_batch_workspace_bytes(n)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    status = torch.full((n,), 9, dtype=torch.int32, device="cuda")
    aesgb.aes_ecb_batch_ws(desc, n, ws, ws_bytes, status)
    torch.cuda.synchronize()
    assert bool((status == 0).all())
    assert torch.equal(dst, ref)
    src_h = src.cpu().numpy()
    dst_h = dst.cpu().numpy()
    for i in range(n):
        ln = int(lengths[i])
        o = int(offs[i])
        if ln <= 64 * 1024:
            exp = orc.ecb(int(dirs[i]), keys[i], src_h[o:o + ln], nthreads=1)
            assert np.array_equal(dst_h[o:o + ln], exp), i
        else:
            w = 2048
            for s in (o, o + ln - w):  # the first and the last 2 KiB of the message
                exp = orc.ecb(int(dirs[i]), keys[i], src_h[s:s + w], nthreads=1)
                assert np.array_equal(dst_h[s:s + w], exp), (i, s)


def test_stress_16gib_aes256_decrypt_in_place(orc):
    torch = torch_cuda()
    total = 16 * GIB
    region = 64 * MIB
    kinds = wl.stress_region_kinds(total, region)
    buf = torch.empty(total, dtype=torch.uint8, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(wl.BASE_SEED + 53)
    hg = wl.rng(53)
    period_blocks = {}
    for r, kind in enumerate(kinds.tolist()):
        sl = buf[r * region:(r + 1) * region]
        if kind == 0:
            sl.random_(0, 256, generator=g)
        elif kind == 1:
            sl.zero_()
        else:
            blk = hg.integers(0, 256, 16, dtype=np.uint8)
            period_blocks[r] = blk
            sl.view(-1, 16).copy_(torch.from_numpy(blk).cuda().expand(region // 16, 16))
    key = wl.random_key(256, 53).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(256, key)
    # 32 windows of 1 MiB saved before: region boundaries and seeded random spots
    w = MIB
    starts = [region - w // 2, 2 * region - w // 2, 3 * region - w // 2, 0, total - w]
    starts += [int(v) // 16 * 16 for v in hg.integers(0, total - w, 32 - len(starts))]
    saved = [(s, buf[s:s + w].cpu().numpy()) for s in starts]
    aesgb.aes_ecb_decrypt(dec, nr, buf, buf, total // 16)
    torch.cuda.synchronize()
    for s, before in saved:
        exp = orc.ecb(1, key, before, nthreads=16)
        assert np.array_equal(buf[s:s + w].cpu().numpy(), exp), f"window at {s}"
    zero_pt = orc.ecb(1, key, np.zeros(16, np.uint8))
    for r, kind in enumerate(kinds.tolist()):
        if kind == 0:
            continue
        blocks = buf[r * region:(r + 1) * region].view(-1, 16)
        first = blocks[0].cpu().numpy()
        exp = zero_pt if kind == 1 else orc.ecb(1, key, period_blocks[r])
        assert np.array_equal(first, exp), f"region {r}"
        assert bool((blocks == blocks[0]).all()), f"region {r} not a single repeated block"


def _tuner_candidates():
    """The configurations aes_tune_ecb chooses among (tune.cpp)."""
    out = []
    for layout in (aesgb.LAYOUT_R4, aesgb.LAYOUT_R2, aesgb.LAYOUT_R1):
        for nb in (1, 2, 4, 8):
            for th in (128, 256, 512, 768, 1024):
                if th > (256 if nb >= 8 else 512 if nb >= 4 else 1024):
                    continue
                if nb == 8 and layout == aesgb.LAYOUT_R1:
                    continue
                out.append(aesgb.make_cfg(th, nb, layout, 0))
    out.append(aesgb.aes_ecb_get_cfg(0, 10, (1 << 30) // 16))
    return out


def test_1gib_every_tuner_candidate(orc):
    """The benchmark tunes before it times, so whichever candidate wins is the
    timed configuration: all of them give the same 1 GiB ciphertext, which is
    checked against the oracle on windows, and all decrypt it back."""
    torch = torch_cuda()
    nbytes = 1 << 30
    n = nbytes // 16
    x = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    _fill_random(torch, x, 60)
    key = wl.random_key(128, 60).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(128, key)
    ref = torch.empty_like(x)
    aesgb.aes_ecb_encrypt(enc, nr, x, ref, n)
    torch.cuda.synchronize()
    win = 128 * 1024
    for s in (0, nbytes // 3 // 16 * 16, nbytes - win):
        assert np.array_equal(ref[s:s + win].cpu().numpy(), orc.ecb(0, key, x[s:s + win].cpu().numpy(),
                                                                   nthreads=16)), s
    y = torch.empty_like(x)
    for cfg in _tuner_candidates():
        aesgb.aes_ecb_crypt_cfg(0, enc, nr, x, y, n, cfg)
        torch.cuda.synchronize()
        assert torch.equal(y, ref), repr(cfg)
        aesgb.aes_ecb_crypt_cfg(1, dec, nr, y, y, n, cfg)
        torch.cuda.synchronize()
        assert torch.equal(y, x), repr(cfg)


def test_batch_every_tuner_candidate_fullsize():
    """Every batch configuration aes_tune_batch can choose gives the same
    output on the 4,096-message workload (5.2 GB)."""
    torch = torch_cuda()
    n = 4096
    lengths, keybits, dirs = wl.batch_workload(n)
    offs = np.zeros(n + 1, np.int64)
    np.cumsum(lengths, out=offs[1:])
    total = int(offs[-1])
    src = torch.empty(total, dtype=torch.uint8, device="cuda")
    _fill_random(torch, src, 61)
    dst = torch.empty_like(src)
    ref = torch.empty_like(src)
    g = wl.rng(61)
    rks = np.zeros((n, 64), np.uint32)
    nrs = np.zeros(n, np.int64)
    for i in range(n):
        key = g.integers(0, 256, int(keybits[i]) // 8, dtype=np.uint8).tobytes()
        enc, dec, nr = aesgb.aes_expand_key(int(keybits[i]), key)
        rks[i, :60] = enc if dirs[i] == 0 else dec
        nrs[i] = nr
        a, b = src.data_ptr() + int(offs[i]), ref.data_ptr() + int(offs[i])
        (aesgb.aes_ecb_encrypt if dirs[i] == 0 else aesgb.aes_ecb_decrypt)(rks[i, :60], nr, a, b,
                                                                         int(lengths[i]) // 16)
    rk_dev = torch.from_numpy(rks.view(np.uint8).reshape(-1)).cuda()
    table = aesgb.pack_descs(rk_dev.data_ptr() + 256 * np.arange(n, dtype=np.uint64),
                             src.data_ptr() + offs[:-1].astype(np.uint64),
                             dst.data_ptr() + offs[:-1].astype(np.uint64), lengths // 16, nrs, dirs)
    desc = torch.from_numpy(table.view(np.uint8).copy()).cuda()
    ws_bytes = aesgb.aes_batch_workspace_bytes(n)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    pairs = [(aesgb.LAYOUT_R4, aesgb.LAYOUT_R2), (aesgb.LAYOUT_R4, aesgb.LAYOUT_R4),
             (aesgb.LAYOUT_R2, aesgb.LAYOUT_R2), (aesgb.LAYOUT_R1, aesgb.LAYOUT_R1)]
    for le, ld in pairs:                      # the tuner pairs each layout with the best of the rest
        for nb in (1, 2):
            for th in (256, 384, 512):
                for passes in (8, 16, 32, 64):
                    dst.fill_(0x5A)
                    aesgb.aes_ecb_batch_ws(desc, n, ws, ws_bytes,
                                           cfg=aesgb.make_batch_cfg(th, nb, passes, 1, le, ld))
                    torch.cuda.synchronize()
                    assert torch.equal(dst, ref), (le, ld, nb, th, passes)


def _windows(nbytes, win, seed):
    g = wl.rng(seed)
    return [0, nbytes - win] + [int(v) // 16 * 16 for v in g.integers(0, nbytes - win, 3)]


@pytest.mark.parametrize("keybits", [128, 192, 256])
def test_1gib_constant_time_windows_and_roundtrip(orc, keybits):
    """The bitsliced kernel at the size the benchmark times it (1 GiB, every
    key size): windows against the oracle, decryption in place back to the
    plaintext over the whole buffer."""
    torch = torch_cuda()
    nbytes = GIB
    n = nbytes // 16
    x = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    _fill_random(torch, x, 70 + keybits)
    key = wl.random_key(keybits, 70).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(keybits, key)
    y = torch.empty_like(x)
    aesgb.aes_ecb_crypt_ct(0, enc, nr, x, y, n)
    torch.cuda.synchronize()
    win = 64 * 1024
    for s in _windows(nbytes, win, 71):
        assert np.array_equal(y[s:s + win].cpu().numpy(), orc.ecb(0, key, x[s:s + win].cpu().numpy(), nthreads=16)), s
    aesgb.aes_ecb_crypt_ct(1, dec, nr, y, y, n)
    torch.cuda.synchronize()
    assert torch.equal(x, y)


@pytest.mark.parametrize("cfg", [(1024, 2), (512, 4)])
def test_1gib_tma_staged_windows_and_roundtrip(orc, cfg):
    """The TMA-staged layout at 1 GiB (the study's configurations): windows
    against the oracle, in-place decryption back, no bounded wait run out."""
    torch = torch_cuda()
    nbytes = GIB
    n = nbytes // 16
    x = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    _fill_random(torch, x, 72)
    key = wl.random_key(128, 72).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(128, key)
    c = aesgb.make_cfg(cfg[0], cfg[1], aesgb.LAYOUT_R4_TMA, 0)
    y = torch.empty_like(x)
    aesgb.aes_ecb_crypt_cfg(0, enc, nr, x, y, n, c)
    torch.cuda.synchronize()
    win = 64 * 1024
    for s in _windows(nbytes, win, 73):
        assert np.array_equal(y[s:s + win].cpu().numpy(), orc.ecb(0, key, x[s:s + win].cpu().numpy(), nthreads=16)), s
    aesgb.aes_ecb_crypt_cfg(1, dec, nr, y, y, n, c)
    torch.cuda.synchronize()
    assert torch.equal(x, y)
    assert aesgb.aes_wait_timeouts() == 0


@pytest.mark.parametrize("keybits", [128, 256])
@pytest.mark.parametrize("cfg", [(1024, 1), (512, 4)])
def test_1gib_r2_layout_windows_and_roundtrip(orc, keybits, cfg):
    """The two-table layout at 1 GiB, both directions: encryption windows
    against the oracle, decryption in place back to the input."""
    torch = torch_cuda()
    nbytes = GIB
    n = nbytes // 16
    x = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    _fill_random(torch, x, 74 + keybits)
    key = wl.random_key(keybits, 74).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(keybits, key)
    c = aesgb.make_cfg(cfg[0], cfg[1], aesgb.LAYOUT_R2, 0)
    y = torch.empty_like(x)
    aesgb.aes_ecb_crypt_cfg(0, enc, nr, x, y, n, c)
    torch.cuda.synchronize()
    win = 64 * 1024
    for s in _windows(nbytes, win, 75):
        assert np.array_equal(y[s:s + win].cpu().numpy(), orc.ecb(0, key, x[s:s + win].cpu().numpy(), nthreads=16)), s
    aesgb.aes_ecb_crypt_cfg(1, dec, nr, y, y, n, c)
    torch.cuda.synchronize()
    assert torch.equal(x, y)


@pytest.mark.parametrize("keybits", [128, 192, 256])
@pytest.mark.parametrize("cfg", [(256, 8, 0), (256, 8, 5), (256, 1, 6), (256, 2, 6)])
def test_1gib_register_and_128B_layouts_windows_and_roundtrip(orc, keybits, cfg):
    """The placement study's additions at the size it times them (1 GiB): 128 B
    per thread on the R4 and R2 tables, and the table in registers at 16 and
    32 B per thread.  Encryption windows against the oracle; decryption in
    place back to the input; encryption equal to the default configuration's
    over the whole buffer."""
    torch = torch_cuda()
    nbytes = GIB
    n = nbytes // 16
    x = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    _fill_random(torch, x, 76 + keybits)
    key = wl.random_key(keybits, 76).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(keybits, key)
    c = aesgb.make_cfg(cfg[0], cfg[1], cfg[2], 0)
    ref = torch.empty_like(x)
    aesgb.aes_ecb_encrypt(enc, nr, x, ref, n)
    y = torch.empty_like(x)
    aesgb.aes_ecb_crypt_cfg(0, enc, nr, x, y, n, c)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    win = 64 * 1024
    for s in _windows(nbytes, win, 77):
        assert np.array_equal(y[s:s + win].cpu().numpy(), orc.ecb(0, key, x[s:s + win].cpu().numpy(), nthreads=16)), s
    aesgb.aes_ecb_crypt_cfg(1, dec, nr, y, y, n, c)
    torch.cuda.synchronize()
    assert torch.equal(x, y)


@pytest.mark.parametrize("keybits", [128, 256])
def test_1gib_ctr_cbc_cfb_windows(orc, keybits):
    """CTR, CBC and CFB decryption at the size the benchmark times them (1 GiB):
    windows against the oracle, each started from its own counter block or
    chaining block; CTR applied twice gives the input back."""
    torch = torch_cuda()
    nbytes = GIB
    n = nbytes // 16
    x = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    _fill_random(torch, x, 74 + keybits)
    key = wl.random_key(keybits, 74).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(keybits, key)
    ctr0 = np.frombuffer(bytes(range(240, 256)), np.uint8)  # low bytes near a carry
    iv = np.frombuffer(bytes(range(16)), np.uint8)
    y = torch.empty_like(x)
    win = 64 * 1024
    aesgb.aes_ctr_crypt(enc, nr, ctr0, x, y, n)
    torch.cuda.synchronize()
    for s in _windows(nbytes, win, 75):
        exp = orc.ctr(key, orc.ctr_block(ctr0, s // 16), x[s:s + win].cpu().numpy())
        assert np.array_equal(y[s:s + win].cpu().numpy(), exp), ("ctr", s)
    aesgb.aes_ctr_crypt(enc, nr, ctr0, y, y, n)
    torch.cuda.synchronize()
    assert torch.equal(x, y)
    aesgb.aes_cbc_decrypt(dec, nr, iv, x, y, n)
    torch.cuda.synchronize()
    for s in _windows(nbytes, win, 76):
        chain = iv if s == 0 else x[s - 16:s].cpu().numpy()
        exp = orc.cbc_decrypt(key, chain, x[s:s + win].cpu().numpy())
        assert np.array_equal(y[s:s + win].cpu().numpy(), exp), ("cbc", s)
    aesgb.aes_cfb_decrypt(enc, nr, iv, x, y, n)
    torch.cuda.synchronize()
    for s in _windows(nbytes, win, 77):
        chain = iv if s == 0 else x[s - 16:s].cpu().numpy()
        exp = orc.cfb_decrypt(key, chain, x[s:s + win].cpu().numpy())
        assert np.array_equal(y[s:s + win].cpu().numpy(), exp), ("cfb", s)


def test_over_2_32_blocks_in_place(orc):
    """One call over more than 2^32 blocks (2^32 + 1 blocks = 64 GiB + 16 B),
    in place: the block index is 64-bit end to end.  Windows around block 2^32
    (byte 2^36), the start and the end against the oracle; decryption in place
    restores them."""
    torch = torch_cuda()
    n = (1 << 32) + 1
    nbytes = 16 * n
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    _fill_random(torch, buf, 80)
    key = wl.random_key(128, 80).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(128, key)
    w = 32 * 1024
    starts = [0, (1 << 36) - w // 2, nbytes - w]
    saved = [(s, buf[s:s + w].cpu().numpy()) for s in starts]
    aesgb.aes_ecb_encrypt(enc, nr, buf, buf, n)
    torch.cuda.synchronize()
    for s, before in saved:
        assert np.array_equal(buf[s:s + w].cpu().numpy(), orc.ecb(0, key, before, nthreads=16)), s
    aesgb.aes_ecb_decrypt(dec, nr, buf, buf, n)
    torch.cuda.synchronize()
    for s, before in saved:
        assert np.array_equal(buf[s:s + w].cpu().numpy(), before), s


@pytest.mark.parametrize("keybits", [128, 192, 256])
def test_single_buffer_sweep_parity(orc, keybits):
    """The single-buffer sweep's sizes (1 MiB .. 1 GiB in powers of 4; 4 GiB is
    the test above) in both directions, default launch configuration: the
    whole output against the oracle up to 64 MiB; above that 16 random 1 MiB
    windows plus the first and the last, and decryption back over the whole
    buffer."""
    torch = torch_cuda()
    key = wl.random_key(keybits, 90).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(keybits, key)
    g = wl.rng(90 + keybits)
    for mib in (1, 4, 16, 64, 256, 1024):
        nbytes = mib * MIB
        n = nbytes // 16
        x = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        _fill_random(torch, x, 91 + mib)
        y = torch.empty_like(x)
        z = torch.empty_like(x)
        aesgb.aes_ecb_encrypt(enc, nr, x, y, n)
        aesgb.aes_ecb_decrypt(dec, nr, x, z, n)
        torch.cuda.synchronize()
        if mib <= 64:
            xh = x.cpu().numpy()
            assert np.array_equal(y.cpu().numpy(), orc.ecb(0, key, xh, nthreads=16)), (mib, "enc")
            assert np.array_equal(z.cpu().numpy(), orc.ecb(1, key, xh, nthreads=16)), (mib, "dec")
        else:
            starts = [0, nbytes - MIB] + [int(v) // 16 * 16 for v in g.integers(0, nbytes - MIB, 16)]
            for s in starts:
                xw = x[s:s + MIB].cpu().numpy()
                assert np.array_equal(y[s:s + MIB].cpu().numpy(), orc.ecb(0, key, xw, nthreads=16)), (mib, s)
                assert np.array_equal(z[s:s + MIB].cpu().numpy(), orc.ecb(1, key, xw, nthreads=16)), (mib, s)
            aesgb.aes_ecb_decrypt(dec, nr, y, y, n)
            torch.cuda.synchronize()
            assert torch.equal(x, y), mib
        del x, y, z
