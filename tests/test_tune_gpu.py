"""The autotuner picks a configuration by timing, the plain entry points use
it afterwards, and results stay bit-exact."""
import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl
from batch_util import DeviceBatch
from gpu_util import gpu_ecb, torch_cuda

pytestmark = pytest.mark.gpu


def test_tune_ecb_then_use(orc, tmp_path):
    torch = torch_cuda()
    aesgb.aes_tune_clear()
    try:
        n = 1 << 20                                  # 16 MiB
        x = torch.from_numpy(wl.random_bytes(16 * n, 80)).cuda()
        y = torch.empty_like(x)
        key = wl.random_key(192, 80).tobytes()
        enc, dec, nr = aesgb.aes_expand_key(192, key)
        best = aesgb.aes_tune_ecb(1, nr, dec, x, y, n)
        assert best.layout in (aesgb.LAYOUT_R4, aesgb.LAYOUT_R1, aesgb.LAYOUT_R2) and best.blocks_per_thread in (1, 2, 4)
        assert aesgb.aes_ecb_get_cfg(1, nr, n).as_dict() == best.as_dict()
        aesgb.aes_ecb_decrypt(dec, nr, x, y, n)
        torch.cuda.synchronize()
        w = 65536
        assert np.array_equal(y[:w].cpu().numpy(), orc.ecb(1, key, x[:w].cpu().numpy(), nthreads=8))
        assert np.array_equal(y[-w:].cpu().numpy(), orc.ecb(1, key, x[-w:].cpu().numpy(), nthreads=8))
        path = str(tmp_path / "t.txt")
        aesgb.aes_tune_save(path)
        assert "ecb" in open(path).read()
    finally:
        aesgb.aes_tune_clear()


def test_tune_batch_then_use(orc):
    torch = torch_cuda()
    aesgb.aes_tune_clear()
    try:
        g = wl.rng(81)
        lengths = wl.log_uniform_lengths(200, 16, 1 << 20, g)
        b = DeviceBatch(torch, lengths, g.choice(np.array([128, 192, 256]), size=200),
                        g.integers(0, 2, size=200), seed=81)
        ws, nbytes = b.workspace()
        best = aesgb.aes_tune_batch(b.desc_dev, b.n, ws, nbytes)
        got = aesgb.aes_batch_get_cfg(b.n)
        assert (got.threads, got.blocks_per_thread, got.chunk_passes, got.layout_enc, got.layout_dec) == \
               (best.threads, best.blocks_per_thread, best.chunk_passes, best.layout_enc, best.layout_dec)
        b.out_dev.fill_(0x5A)
        aesgb.aes_ecb_batch_ws(b.desc_dev, b.n, ws, nbytes)
        out = b.output()
        for i in range(0, b.n, 7):
            exp = orc.ecb(int(b.dirs[i]), b.keys[i], b.message(b.data, i), nthreads=4)
            assert np.array_equal(b.message(out, i), exp)
    finally:
        aesgb.aes_tune_clear()


def test_tune_from_a_size_hint(orc, tmp_path):
    """aes_tune(dir, nrounds, bytes_hint): the library allocates its own
    scratch, records a configuration for that size class, frees the scratch,
    and later calls of that class use it with exact output."""
    torch = torch_cuda()
    aesgb.aes_tune_clear()
    try:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        aesgb.aes_tune(1, 12, 3 << 20)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] > free0 - (64 << 20)      # the scratch went back
        n = (3 << 20) // 16 + 5                                        # same size class
        key = wl.random_key(192, 85).tobytes()
        data = wl.random_bytes(16 * n, 85)
        got, ok = gpu_ecb(1, key, data, guard=64)
        assert ok and np.array_equal(got, orc.ecb(1, key, data, nthreads=8))
        tuned = aesgb.aes_ecb_get_cfg(1, 12, n)
        assert tuned.threads % 32 == 0 and tuned.layout in (aesgb.LAYOUT_R4, aesgb.LAYOUT_R2, aesgb.LAYOUT_R1)
        path = str(tmp_path / "tune.txt")
        aesgb.aes_tune_save(path)
        assert sum(1 for line in open(path) if line.startswith("ecb ")) == 1   # one entry: this size class
    finally:
        aesgb.aes_tune_clear()
