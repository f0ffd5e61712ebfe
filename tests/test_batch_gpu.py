"""Batched ECB (one persistent launch over a device descriptor table): every
message bit-exact against the oracle and against the single-buffer path;
invalid descriptors skipped with a status; graph replay; every batch
configuration."""
import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl
from batch_util import DeviceBatch
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def small_mix(n, lo=16, hi=256 * 1024, seed=5):
    g = wl.rng(seed)
    lengths = wl.log_uniform_lengths(n, lo, hi, g)
    keybits = g.choice(np.array([128, 192, 256]), size=n)
    dirs = g.integers(0, 2, size=n)
    return lengths, keybits, dirs


def check_against_oracle(orc, b: DeviceBatch, out, skip=()):
    for i in range(b.n):
        got = b.message(out, i)
        if i in skip:
            assert np.all(got == 0x5A), f"invalid message {i} was written"
            continue
        exp = orc.ecb(int(b.dirs[i]), b.keys[i], b.message(b.data, i), nthreads=8)
        assert np.array_equal(got, exp), f"message {i} (len {b.lengths[i]}, AES-{b.keybits[i]}, dir {b.dirs[i]})"


def test_batch_mixed_with_invalid_descriptors(orc):
    torch = torch_cuda()
    lengths, keybits, dirs = small_mix(300)
    lengths[7] = 0                      # empty message: fine, nothing written
    lengths[15] = 4096                  # longer than the 16-byte shift below
    b = DeviceBatch(torch, lengths, keybits, dirs, seed=1)
    bad = {11: ("nrounds", 11, -3), 12: ("dir", 2, -1), 13: ("rk", 0, -1), 14: ("in", 8, -4)}
    for i, (field, val, _) in bad.items():
        if field == "in":
            b.table[i]["in"] += val
        else:
            b.table[i][field] = val
    # partial overlap of in and out: message 15 writes over its own input shifted by 16 bytes
    b.table[15]["out"] = b.table[15]["in"] + 16
    b.upload()
    ws, nbytes = b.workspace()
    status = torch.full((b.n,), 99, dtype=torch.int32, device="cuda")
    aesgb.aes_ecb_batch_ws(b.desc_dev, b.n, ws, nbytes, status)
    out = b.output()
    st = status.cpu().numpy()
    for i, (_, _, code) in bad.items():
        assert st[i] == code, (i, st[i])
    assert st[15] == -5
    ok = [i for i in range(b.n) if i not in bad and i != 15]
    assert np.all(st[ok] == 0)
    check_against_oracle(orc, b, out, skip=set(bad) | {15})


@pytest.mark.parametrize("only_dir", [0, 1])
def test_batch_single_direction(orc, only_dir):
    torch = torch_cuda()
    lengths, keybits, _ = small_mix(64, seed=6)
    b = DeviceBatch(torch, lengths, keybits, np.full(64, only_dir), seed=2)
    ws, nbytes = b.workspace()
    aesgb.aes_ecb_batch_ws(b.desc_dev, b.n, ws, nbytes)
    check_against_oracle(orc, b, b.output())


def test_batch_edge_counts(orc):
    torch = torch_cuda()
    # n = 1, a single block
    b = DeviceBatch(torch, [16], [256], [1], seed=3)
    ws, nbytes = b.workspace()
    aesgb.aes_ecb_batch_ws(b.desc_dev, 1, ws, nbytes)
    check_against_oracle(orc, b, b.output())
    # n = 0 is a no-op
    aesgb.aes_ecb_batch_ws(b.desc_dev, 0, ws, nbytes)
    # every descriptor invalid: nothing written, all statuses set
    b = DeviceBatch(torch, [32, 48, 64], [128, 128, 128], [0, 1, 0], seed=4)
    b.table["nrounds"] = 9
    b.upload()
    ws, nbytes = b.workspace()
    status = torch.zeros(3, dtype=torch.int32, device="cuda")
    aesgb.aes_ecb_batch_ws(b.desc_dev, 3, ws, nbytes, status)
    assert np.all(b.output() == 0x5A)
    assert np.all(status.cpu().numpy() == -3)
    with pytest.raises(aesgb.AesError) as e:
        aesgb.aes_ecb_batch_ws(b.desc_dev, 3, ws, 64)
    assert e.value.status == -10


def test_batch_equals_single_buffer_path():
    """Each message through the batch equals the same message through
    aes_ecb_encrypt/decrypt (itself checked against the oracle)."""
    torch = torch_cuda()
    lengths, keybits, dirs = small_mix(120, lo=16, hi=4 * 1024 * 1024, seed=7)
    b = DeviceBatch(torch, lengths, keybits, dirs, seed=5)
    ws, nbytes = b.workspace()
    aesgb.aes_ecb_batch_ws(b.desc_dev, b.n, ws, nbytes)
    torch.cuda.synchronize()
    ref = torch.empty_like(b.in_dev)
    for i in range(b.n):
        nb = int(b.lengths[i]) // 16
        if nb == 0:
            continue
        enc, dec, nr = aesgb.aes_expand_key(int(b.keybits[i]), b.keys[i])
        off = int(b.offsets[i])
        src = b.in_dev.data_ptr() + off
        dst = ref.data_ptr() + off
        if b.dirs[i] == 0:
            aesgb.aes_ecb_encrypt(enc, nr, src, dst, nb)
        else:
            aesgb.aes_ecb_decrypt(dec, nr, src, dst, nb)
    torch.cuda.synchronize()
    total = int(b.offsets[-1])
    assert torch.equal(ref[:total], b.out_dev[:total])


def test_batch_in_place(orc):
    torch = torch_cuda()
    lengths, keybits, dirs = small_mix(80, seed=8)
    b = DeviceBatch(torch, lengths, keybits, dirs, seed=6, inplace=True)
    ws, nbytes = b.workspace()
    aesgb.aes_ecb_batch_ws(b.desc_dev, b.n, ws, nbytes)
    check_against_oracle(orc, b, b.output())


LAYOUT_PAIRS = [(aesgb.LAYOUT_R4, aesgb.LAYOUT_R2), (aesgb.LAYOUT_R4, aesgb.LAYOUT_R4),
                (aesgb.LAYOUT_R2, aesgb.LAYOUT_R2), (aesgb.LAYOUT_R1, aesgb.LAYOUT_R1)]


def batch_cfgs():
    out = []
    for nb in (1, 2, 4):
        for threads in (64, 256, 512):
            for passes in (1, 3, 8):
                out.append(aesgb.make_batch_cfg(threads, nb, passes, 1))
    for le, ld in LAYOUT_PAIRS[1:]:                  # the other table layouts of the two phases
        for nb in (1, 2):
            for threads in (64, 512):
                for passes in (1, 8):
                    out.append(aesgb.make_batch_cfg(threads, nb, passes, 1, le, ld))
    return out


def test_batch_cfg_layout_pairs_refused_outside_the_compiled_set():
    """A layout pair or granularity the batch kernel is not compiled for is
    refused before any launch (AES_E_CONFIG)."""
    torch = torch_cuda()
    b = DeviceBatch(torch, [64, 4096], [128, 256], [0, 1], seed=10)
    ws, nbytes = b.workspace()
    for cfg in (aesgb.make_batch_cfg(512, 1, 8, 1, aesgb.LAYOUT_R2, aesgb.LAYOUT_R4),
                aesgb.make_batch_cfg(512, 4, 8, 1, aesgb.LAYOUT_R2, aesgb.LAYOUT_R2),
                aesgb.make_batch_cfg(512, 1, 8, 1, aesgb.LAYOUT_P4, aesgb.LAYOUT_P4),
                aesgb.make_batch_cfg(512, 1, 8, 1, aesgb.LAYOUT_REG, aesgb.LAYOUT_REG)):
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_ecb_batch_ws(b.desc_dev, b.n, ws, nbytes, cfg=cfg)
        assert e.value.status == -12, repr(cfg)


def test_batch_every_cfg(orc):
    torch = torch_cuda()
    lengths, keybits, dirs = small_mix(150, hi=128 * 1024, seed=9)
    b = DeviceBatch(torch, lengths, keybits, dirs, seed=7)
    total = int(b.offsets[-1])
    exp = np.concatenate([orc.ecb(int(b.dirs[i]), b.keys[i], b.message(b.data, i), nthreads=8)
                          for i in range(b.n)])
    ws, nbytes = b.workspace()
    for cfg in batch_cfgs():
        b.out_dev.fill_(0x5A)
        aesgb.aes_ecb_batch_ws(b.desc_dev, b.n, ws, nbytes, cfg=cfg)
        assert np.array_equal(b.output(), exp), repr(cfg)
    assert total > 0


def test_batch_graph_replay_and_library_workspace(orc):
    torch = torch_cuda()
    lengths, keybits, dirs = small_mix(100, seed=10)
    b = DeviceBatch(torch, lengths, keybits, dirs, seed=8)
    ws, nbytes = b.workspace()
    g = aesgb.aes_batch_graph_create(b.desc_dev, b.n, ws, nbytes)
    try:
        aesgb.aes_batch_graph_launch(g)
        out1 = b.output()
        check_against_oracle(orc, b, out1)
        # new contents of the same descriptor table: flip every direction (and
        # its schedule), replay the same graph
        b2 = DeviceBatch(torch, lengths, keybits, 1 - dirs, seed=8)
        b.desc_dev.copy_(b2.desc_dev)
        b.out_dev.fill_(0x5A)
        keep = b2  # the arenas b2's descriptors point at
        aesgb.aes_batch_graph_launch(g)
        torch.cuda.synchronize()
        check_against_oracle(orc, keep, keep.output())
        assert np.all(b.output() == 0x5A)   # the replay wrote through b2's pointers only
    finally:
        aesgb.aes_batch_graph_destroy(g)
    # the library-owned workspace variant
    b.out_dev.fill_(0x5A)
    b.upload()
    aesgb.aes_ecb_batch(b.desc_dev, b.n)
    check_against_oracle(orc, b, b.output())


def test_batch_many_tiny_messages(orc):
    """20,000 messages of 16..256 bytes: the plan kernel scans 20 tiles of
    1,024 descriptors and the 32-ary search runs over 20,000 positions."""
    torch = torch_cuda()
    g = wl.rng(12)
    n = 20_000
    lengths = 16 * g.integers(1, 17, size=n)
    keybits = g.choice(np.array([128, 192, 256]), size=n)
    dirs = g.integers(0, 2, size=n)
    b = DeviceBatch(torch, lengths, keybits, dirs, seed=13)
    ws, nbytes = b.workspace()
    status = torch.full((n,), 5, dtype=torch.int32, device="cuda")
    aesgb.aes_ecb_batch_ws(b.desc_dev, n, ws, nbytes, status)
    out = b.output()
    assert bool((status == 0).all())
    for i in range(0, n, 97):
        exp = orc.ecb(int(b.dirs[i]), b.keys[i], b.message(b.data, i))
        assert np.array_equal(b.message(out, i), exp), i
    # every message against the single-buffer path on the device
    ref = torch.full_like(b.out_dev, 0x5A)
    for i in range(0, n, 7):
        enc, dec, nr = aesgb.aes_expand_key(int(b.keybits[i]), b.keys[i])
        off = int(b.offsets[i])
        (aesgb.aes_ecb_encrypt if b.dirs[i] == 0 else aesgb.aes_ecb_decrypt)(
            enc if b.dirs[i] == 0 else dec, nr, b.in_dev.data_ptr() + off, ref.data_ptr() + off,
            int(b.lengths[i]) // 16)
    torch.cuda.synchronize()
    got = b.out_dev.cpu().numpy()
    refh = ref.cpu().numpy()
    for i in range(0, n, 7):
        assert np.array_equal(b.message(got, i), b.message(refh, i)), i


def test_library_workspace_batch_with_status(orc):
    """aes_ecb_batch_ex: the library-owned workspace with the per-message
    status array -- invalid descriptors are skipped with their status, every
    other message equals the oracle."""
    torch = torch_cuda()
    lengths, keybits, dirs = small_mix(60, hi=32 * 1024, seed=12)
    b = DeviceBatch(torch, lengths, keybits, dirs, seed=12)
    b.table[5]["nrounds"] = 11
    b.table[9]["dir"] = 3
    b.upload()
    status = torch.full((b.n,), 77, dtype=torch.int32, device="cuda")
    aesgb.aes_ecb_batch_ex(b.desc_dev, b.n, status)
    out = b.output()
    st = status.cpu().numpy()
    assert st[5] == -3 and st[9] == -1 and np.all(np.delete(st, [5, 9]) == 0)
    for i in range(b.n):
        if i in (5, 9):
            assert np.all(b.message(out, i) == 0x5A), i
        else:
            assert np.array_equal(b.message(out, i), orc.ecb(int(b.dirs[i]), b.keys[i], b.message(b.data, i))), i
