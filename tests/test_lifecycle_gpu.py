"""aes_shutdown releases what the library created lazily (the host pipeline's
streams and events, the library-owned batch workspace); every entry point
works again afterwards, creating them anew, with results exact against the
oracle -- twice over, so a second shutdown after re-creation is covered too."""
import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def use_everything(torch, orc, seed):
    key = wl.random_key(192, seed).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(192, key)
    n = 40_003
    data = wl.random_bytes(16 * n, seed)
    exp = orc.ecb(0, key, data, nthreads=8)
    # device buffers, tuned and default configurations
    x = torch.from_numpy(data).cuda()
    y = torch.empty_like(x)
    aesgb.aes_tune_ecb(0, nr, enc, x, y, n)
    aesgb.aes_ecb_encrypt(enc, nr, x, y, n)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), exp)
    # host pipeline through the library's internal streams
    h_in = torch.from_numpy(data.copy()).pin_memory()
    h_out = torch.zeros_like(h_in).pin_memory()
    stage = torch.empty(3 << 16, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    aesgb.aes_ecb_host(0, enc, nr, h_in, h_out, n, stage, stage.numel(), s)
    s.synchronize()
    assert np.array_equal(h_out.numpy(), exp)
    # batch with the library-owned workspace
    rk_dev = torch.from_numpy(enc.view(np.uint8).copy()).cuda()
    table = aesgb.pack_descs([rk_dev.data_ptr()], [x.data_ptr()], [y.data_ptr()], [n], [nr], [0])
    desc = torch.from_numpy(table.view(np.uint8).copy()).cuda()
    y.fill_(0x5A)
    aesgb.aes_ecb_batch(desc, 1)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), exp)
    # constant-time kernel
    aesgb.aes_ecb_crypt_ct(1, dec, nr, y, y, n)
    torch.cuda.synchronize()
    assert torch.equal(y, x)


def test_shutdown_then_use_again(orc):
    torch = torch_cuda()
    for round_ in range(3):
        use_everything(torch, orc, 600 + round_)
        torch.cuda.synchronize()
        aesgb.aes_shutdown()
