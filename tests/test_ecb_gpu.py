"""ECB parity on the GPU: every key size, both directions, every launch
configuration the tuner can pick, edge sizes, in place, guard bytes.
Bit-exact against the CPU oracle (integer work: tolerance 0)."""
import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl
from gpu_util import gpu_ecb, torch_cuda

pytestmark = pytest.mark.gpu

KEYBITS = [128, 192, 256]


def oracle_ecb(orc, direction, key, data):
    return orc.ecb(direction, key, data, nthreads=8)


def test_c1_1mib_encrypt_then_decrypt(orc):
    """1 MiB (65,536 blocks) of seeded random bytes, one 128-bit key: encrypt,
    then decrypt the ciphertext; both compared in full with the oracle."""
    data = wl.random_bytes(1 << 20, 1)
    key = wl.random_key(128, 1).tobytes()
    ct, ok = gpu_ecb(0, key, data, guard=4096)
    assert ok
    assert np.array_equal(ct, oracle_ecb(orc, 0, key, data))
    pt, ok = gpu_ecb(1, key, ct, guard=4096)
    assert ok
    assert np.array_equal(pt, data)
    assert np.array_equal(pt, oracle_ecb(orc, 1, key, ct))


SIZES = [1, 2, 3, 31, 32, 33, 63, 64, 65, 1023, 1024, 1025, 2047, 2048, 2049, 4097, 65537, 311297]


@pytest.mark.parametrize("keybits", KEYBITS)
@pytest.mark.parametrize("direction", [0, 1])
def test_edge_sizes_default_cfg(orc, keybits, direction):
    key = wl.random_key(keybits, 2).tobytes()
    for n in SIZES:
        data = wl.random_bytes(16 * n, 100 + n)
        got, ok = gpu_ecb(direction, key, data, guard=256)
        assert ok, f"guard bytes touched at n={n}"
        assert np.array_equal(got, oracle_ecb(orc, direction, key, data)), f"n={n}"


def test_default_cfg_both_sides_of_the_size_switch(orc):
    """The untuned configuration switches from the small-buffer choice (R2
    tables, 256 threads x 2 blocks, three CTAs per SM) to the large-buffer one
    (R4, 1,024 threads x 2 blocks, one CTA per SM) at 16,384 blocks per SM.
    Buffers just below and above the switch, both directions, against the
    oracle."""
    torch = torch_cuda()
    sms = aesgb.aes_device_sm_count(torch.cuda.current_device())
    key = wl.random_key(128, 12).tobytes()
    for n in (sms * 16384 - 1, sms * 16384 + 33):
        data = wl.random_bytes(16 * n, 13)
        for direction in (0, 1):
            cfg = aesgb.aes_ecb_get_cfg(direction, 10, n)
            got, ok = gpu_ecb(direction, key, data, guard=64)
            assert ok and np.array_equal(got, orc.ecb(direction, key, data, nthreads=16)), (n, direction, cfg)


def all_cfgs():
    out = []
    for layout in (aesgb.LAYOUT_R4, aesgb.LAYOUT_R1, aesgb.LAYOUT_P4, aesgb.LAYOUT_CONST, aesgb.LAYOUT_R4_TMA,
                   aesgb.LAYOUT_R2, aesgb.LAYOUT_REG):
        nbs = {aesgb.LAYOUT_R4: (1, 2, 4, 8), aesgb.LAYOUT_R2: (1, 2, 4, 8), aesgb.LAYOUT_R1: (1, 2, 4),
               aesgb.LAYOUT_R4_TMA: (1, 2, 4), aesgb.LAYOUT_REG: (1, 2)}.get(layout, (1,))
        for nb in nbs:
            for threads in (64, 256, 512, 1024):
                limit = 256 if (nb == 8 or layout == aesgb.LAYOUT_REG) else 512 if nb == 4 else 1024
                if threads > limit:
                    continue
                for cps in (0, 1):
                    out.append(aesgb.make_cfg(threads, nb, layout, cps))
    return out


def test_config_limits_refused():
    """Configurations beyond a layout's compiled limits answer AES_E_CONFIG
    before any launch: 128 B per thread above 256 threads or on the R1
    layout, the register layout above 256 threads or at 64 B per thread."""
    torch = torch_cuda()
    enc, _, nr = aesgb.aes_expand_key(128, bytes(16))
    x = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    for threads, nb, layout in ((512, 8, aesgb.LAYOUT_R4), (256, 8, aesgb.LAYOUT_R1), (512, 1, aesgb.LAYOUT_REG),
                                (128, 4, aesgb.LAYOUT_REG), (256, 3, aesgb.LAYOUT_R4), (256, 1, 7)):
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_ecb_crypt_cfg(0, enc, nr, x, x, 256, aesgb.make_cfg(threads, nb, layout, 0))
        assert e.value.status == -12, (threads, nb, layout)


@pytest.mark.parametrize("keybits", KEYBITS)
@pytest.mark.parametrize("direction", [0, 1])
def test_every_cfg(orc, keybits, direction):
    """Each configuration at a ragged size that spans several grid passes for
    the small configurations and a partial pass for the large ones."""
    n = 400_003
    key = wl.random_key(keybits, 3).tobytes()
    data = wl.random_bytes(16 * n, 7)
    exp = oracle_ecb(orc, direction, key, data)
    for cfg in all_cfgs():
        got, ok = gpu_ecb(direction, key, data, cfg=cfg, guard=64)
        assert ok, repr(cfg)
        assert np.array_equal(got, exp), repr(cfg)
    assert aesgb.aes_wait_timeouts() == 0


@pytest.mark.parametrize("keybits", KEYBITS)
@pytest.mark.parametrize("direction", [0, 1])
def test_tma_staged_edge_sizes(orc, keybits, direction):
    """The TMA-staged kernel at sizes around its tile (32 x blocks_per_thread
    blocks per warp and pass): partial first tiles, warps without work, and a
    partial last tile, in place and out of place; no bounded wait runs out."""
    key = wl.random_key(keybits, 11).tobytes()
    for cfg in (aesgb.make_cfg(1024, 2, aesgb.LAYOUT_R4_TMA, 1), aesgb.make_cfg(64, 4, aesgb.LAYOUT_R4_TMA, 0)):
        for n in (1, 2, 31, 32, 33, 63, 64, 65, 127, 129, 1023, 1025, 4097, 65_537):
            data = wl.random_bytes(16 * n, 100 + n)
            exp = oracle_ecb(orc, direction, key, data)
            got, ok = gpu_ecb(direction, key, data, cfg=cfg, guard=64)
            assert ok and np.array_equal(got, exp), (repr(cfg), n)
            got, ok = gpu_ecb(direction, key, data, cfg=cfg, inplace=True, guard=64)
            assert ok and np.array_equal(got, exp), (repr(cfg), n, "in place")
    assert aesgb.aes_wait_timeouts() == 0


@pytest.mark.parametrize("keybits", KEYBITS)
@pytest.mark.parametrize("direction", [0, 1])
def test_r2_layout_edge_sizes(orc, keybits, direction):
    """The two-table layout (T2, T3 as 16-bit rotations of T0, T1) at sizes
    around a warp's pass of 32 x blocks_per_thread blocks and a CTA's pass,
    in place and out of place, with guard bytes."""
    key = wl.random_key(keybits, 12).tobytes()
    cfgs = (aesgb.make_cfg(1024, 1, aesgb.LAYOUT_R2, 1), aesgb.make_cfg(256, 2, aesgb.LAYOUT_R2, 0),
            aesgb.make_cfg(512, 4, aesgb.LAYOUT_R2, 1))
    for cfg in cfgs:
        for n in (1, 31, 32, 33, 127, 129, 1023, 1025, 4097, 65_537, 300_007):
            data = wl.random_bytes(16 * n, 200 + n)
            exp = oracle_ecb(orc, direction, key, data)
            got, ok = gpu_ecb(direction, key, data, cfg=cfg, guard=64)
            assert ok and np.array_equal(got, exp), (repr(cfg), n)
            got, ok = gpu_ecb(direction, key, data, cfg=cfg, inplace=True, guard=64)
            assert ok and np.array_equal(got, exp), (repr(cfg), n, "in place")


@pytest.mark.parametrize("keybits", KEYBITS)
def test_in_place(orc, keybits):
    key = wl.random_key(keybits, 4).tobytes()
    data = wl.random_bytes(16 * 100_001, 8)
    ct, ok = gpu_ecb(0, key, data, inplace=True, guard=512)
    assert ok and np.array_equal(ct, oracle_ecb(orc, 0, key, data))
    pt, ok = gpu_ecb(1, key, ct, inplace=True, guard=512)
    assert ok and np.array_equal(pt, data)


def test_16_byte_offsets_and_zero_blocks(orc):
    torch = torch_cuda()
    key = wl.random_key(128, 5).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(128, key)
    data = wl.random_bytes(16 * 1000, 9)
    src = torch.from_numpy(data).cuda()
    dst = torch.zeros(16 * 1002, dtype=torch.uint8, device="cuda")
    # in at +16 bytes, out at +32 bytes: both only 16-byte aligned
    aesgb.aes_ecb_encrypt(enc, nr, src.data_ptr() + 16, dst.data_ptr() + 32, 999)
    torch.cuda.synchronize()
    got = dst.cpu().numpy()
    assert np.array_equal(got[32:32 + 16 * 999], oracle_ecb(orc, 0, key, data[16:]))
    assert not got[:32].any() and not got[32 + 16 * 999:].any()
    before = dst.clone()
    aesgb.aes_ecb_encrypt(enc, nr, src.data_ptr(), dst.data_ptr(), 0)   # no-op
    torch.cuda.synchronize()
    assert torch.equal(before, dst)
    with pytest.raises(aesgb.AesError) as e:
        aesgb.aes_ecb_encrypt(enc, nr, src.data_ptr() + 8, dst.data_ptr(), 10)
    assert e.value.status == -4


def test_ecb_invariants_on_device():
    """Equal blocks -> equal ciphertext; permuted input -> permuted output."""
    torch = torch_cuda()
    key = wl.random_key(256, 6).tobytes()
    g = np.random.default_rng(11)
    blocks = g.integers(0, 256, (50_000, 16), dtype=np.uint8)
    blocks[1000:2000] = blocks[5]
    ct, _ = gpu_ecb(0, key, blocks.reshape(-1))
    ct = ct.reshape(-1, 16)
    assert (ct[1000:2000] == ct[5]).all()
    perm = g.permutation(blocks.shape[0])
    ctp, _ = gpu_ecb(0, key, blocks[perm].reshape(-1))
    assert np.array_equal(ctp.reshape(-1, 16), ct[perm])


def test_device_tables_match_host_tables():
    torch_cuda()
    for which in range(4):
        assert np.array_equal(aesgb.aes_device_table(which), aesgb.aes_host_table(which))


def test_tensor_convenience_roundtrip(orc):
    torch = torch_cuda()
    key = wl.random_key(192, 7).tobytes()
    data = wl.random_bytes(16 * 4096, 12)
    x = torch.from_numpy(data).cuda()
    c = aesgb.ecb_encrypt(key, x)
    p = aesgb.ecb_decrypt(key, c)
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy(), oracle_ecb(orc, 0, key, data))
    assert torch.equal(p, x)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_pipeline(orc, pinned):
    """aes_ecb_host: host in -> staging chunks -> host out, several chunks and
    a ragged last chunk; both directions; in place on the host buffer."""
    torch = torch_cuda()
    key = wl.random_key(256, 8).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(256, key)
    n = 100_003
    data = wl.random_bytes(16 * n, 13)
    h_in = torch.from_numpy(data.copy())
    h_out = torch.zeros_like(h_in)
    if pinned:
        h_in, h_out = h_in.pin_memory(), h_out.pin_memory()
    stage_bytes = 3 * 16 * 4099            # 4,099-block slots: 25 chunks, the last one partial
    stage = torch.empty(stage_bytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    aesgb.aes_ecb_host(0, enc, nr, h_in, h_out, n, stage, stage_bytes, s)
    s.synchronize()
    exp = oracle_ecb(orc, 0, key, data)
    assert np.array_equal(h_out.numpy(), exp)
    aesgb.aes_ecb_host(1, dec, nr, h_out, h_out, n, stage, stage_bytes, s)   # in place
    s.synchronize()
    assert np.array_equal(h_out.numpy(), data)
    with pytest.raises(aesgb.AesError):
        aesgb.aes_ecb_host(0, enc, nr, h_in, h_out, n, stage, 32, s)          # staging too small


def test_lookup_rate_calibration():
    torch = torch_cuda()
    sms = aesgb.aes_device_sm_count(0)
    sink = torch.zeros(sms * 4096, dtype=torch.uint8, device="cuda")
    n, t = aesgb.aes_calibrate_lookup_rate(sink, sink.numel())
    rate = n / t / sms                       # lookups per second per SM
    assert 1e9 < rate < 32 * 3.0e9           # below 32 per clock at any plausible clock
    with pytest.raises(aesgb.AesError):
        aesgb.aes_calibrate_lookup_rate(sink, 16)


@pytest.mark.parametrize("keybits", [128, 256])
def test_back_to_back_dependent_launches(orc, keybits):
    """Kernels launched back to back on one stream, each reading what the one
    before wrote.  The single-buffer kernels are launched with programmatic
    stream serialisation (they may start while the previous kernel drains and
    wait for it before touching global memory), so a missing wait would show
    here: 12 in-place encryptions through the register-path, R1, TMA-staged
    and constant-time kernels in turn, then 12 decryptions, no synchronisation
    in between, against the oracle applied as many times."""
    torch = torch_cuda()
    key = wl.random_key(keybits, 21).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(keybits, key)
    cfgs = [None, aesgb.make_cfg(1024, 2, aesgb.LAYOUT_R1, 0), aesgb.make_cfg(1024, 2, aesgb.LAYOUT_R4_TMA, 0),
            aesgb.make_cfg(1024, 2, aesgb.LAYOUT_R2, 0), "ct"]
    k = 12
    for n in (1, 33, 4097, 300_001):
        data = wl.random_bytes(16 * n, 200 + n)
        x = torch.from_numpy(data.copy()).cuda()
        for direction, rk in ((0, enc), (1, dec)):
            for i in range(k):
                cfg = cfgs[i % len(cfgs)]
                if cfg is None:
                    (aesgb.aes_ecb_encrypt if direction == 0 else aesgb.aes_ecb_decrypt)(rk, nr, x, x, n)
                elif cfg == "ct":
                    aesgb.aes_ecb_crypt_ct(direction, rk, nr, x, x, n)
                else:
                    aesgb.aes_ecb_crypt_cfg(direction, rk, nr, x, x, n, cfg)
            if direction == 0:
                torch.cuda.synchronize()
                exp = data
                for _ in range(k):
                    exp = orc.ecb(0, key, exp, nthreads=16)
                assert np.array_equal(x.cpu().numpy(), exp), n
        torch.cuda.synchronize()
        assert np.array_equal(x.cpu().numpy(), data), n
    assert aesgb.aes_wait_timeouts() == 0


def test_tma_wait_timeout_is_reported_and_context_survives(orc):
    """Failure detection on the device without a fault: the TMA-staged kernel
    run with barriers that can never complete (aes_tma_selftest_timeout).  Its
    bounded waits run out, the warp reports one timeout and stops without
    writing its output, and the context then runs ordinary launches."""
    torch = torch_cuda()
    n = 64
    data = wl.random_bytes(16 * n, 31)
    x = torch.from_numpy(data.copy()).cuda()
    y = torch.full_like(x, 0x5A)
    aesgb.aes_wait_timeouts()  # reset
    aesgb.aes_tma_selftest_timeout(x, y, n)
    torch.cuda.synchronize()
    assert aesgb.aes_wait_timeouts() == 1
    assert bool((y == 0x5A).all())
    key = wl.random_key(128, 31).tobytes()
    got, ok = gpu_ecb(0, key, data, cfg=aesgb.make_cfg(1024, 2, aesgb.LAYOUT_R4_TMA, 0), guard=64)
    assert ok and np.array_equal(got, orc.ecb(0, key, data))
    assert aesgb.aes_wait_timeouts() == 0
    with pytest.raises(aesgb.AesError):
        aesgb.aes_tma_selftest_timeout(x, y, 65)


@pytest.mark.parametrize("direction", [0, 1])
def test_even_shares_at_one_cta_per_sm(orc, direction):
    """With one CTA per SM (R4, 1,024 threads), up to 8 units (32 x blocks per
    thread) per warp are split into even contiguous shares; above that the
    kernel takes grid-stride passes.  Sizes around both ends of the even
    range and ragged tails, against the oracle, in place and out of place."""
    torch = torch_cuda()
    sms = aesgb.aes_device_sm_count(torch.cuda.current_device())
    key = wl.random_key(128, 14).tobytes()
    warps = sms * 32
    for nb in (1, 2):
        cfg = aesgb.make_cfg(1024, nb, aesgb.LAYOUT_R4, 1)
        unit = 32 * nb
        for n in (1, unit * warps - 1, unit * warps + 17, 8 * unit * warps, 8 * unit * warps + 1,
                  3 * unit * warps + 5):
            data = wl.random_bytes(16 * n, 15 + n % 97)
            exp = orc.ecb(direction, key, data, nthreads=16)
            got, ok = gpu_ecb(direction, key, data, cfg=cfg, guard=64)
            assert ok and np.array_equal(got, exp), (nb, n)
            got, ok = gpu_ecb(direction, key, data, cfg=cfg, inplace=True, guard=64)
            assert ok and np.array_equal(got, exp), (nb, n, "in place")
