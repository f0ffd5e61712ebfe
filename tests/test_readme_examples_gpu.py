"""The usage examples of README.md, run as written (with concrete buffers and
keys) and checked against the oracle."""
import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def test_readme_single_buffer_batch_and_server(orc):
    torch = torch_cuda()
    key16 = wl.random_key(128, 240).tobytes()
    key32 = wl.random_key(256, 241).tobytes()

    # single buffer
    enc, dec, nr = aesgb.aes_expand_key(128, key16)
    x = torch.from_numpy(wl.random_bytes(1 << 20, 240)).cuda()
    y = torch.empty_like(x)
    aesgb.aes_ecb_encrypt(enc, nr, x, y, x.numel() // 16)
    aesgb.aes_ecb_decrypt(dec, nr, y, y, y.numel() // 16)
    torch.cuda.synchronize()
    assert torch.equal(x, y)

    # batch
    x1 = torch.from_numpy(wl.random_bytes(16 * 1000, 242)).cuda()
    x2 = torch.from_numpy(wl.random_bytes(16 * 3001, 243)).cuda()
    y1, y2 = torch.empty_like(x1), torch.empty_like(x2)
    msgs = [(128, key16, 0, x1, y1), (256, key32, 1, x2, y2)]
    rks = np.zeros((len(msgs), 64), np.uint32)
    nrs = np.zeros(len(msgs), np.int64)
    for i, (kb, key, d, _, _) in enumerate(msgs):
        enc_i, dec_i, nrs[i] = aesgb.aes_expand_key(kb, key)
        rks[i, :60] = enc_i if d == 0 else dec_i
    rk_dev = torch.from_numpy(rks.view(np.uint8).reshape(-1)).cuda()
    table = aesgb.pack_descs(rk_dev.data_ptr() + 256 * np.arange(len(msgs), dtype=np.uint64),
                             [m[3].data_ptr() for m in msgs], [m[4].data_ptr() for m in msgs],
                             [m[3].numel() // 16 for m in msgs], nrs, [m[2] for m in msgs])
    desc = torch.from_numpy(table.view(np.uint8).copy()).cuda()
    aesgb.aes_ecb_batch(desc, len(msgs))
    torch.cuda.synchronize()
    assert np.array_equal(y1.cpu().numpy(), orc.ecb(0, key16, x1.cpu().numpy()))
    assert np.array_equal(y2.cpu().numpy(), orc.ecb(1, key32, x2.cpu().numpy()))

    # server
    srv = aesgb.aes_srv_create(4 << 30, max_keys=1024, slots=4)
    try:
        aesgb.aes_srv_put_key(srv, 7, 128, key16)
        z = torch.empty_like(x)
        t = aesgb.aes_srv_submit(srv, 7, 0, x, z, x.numel())
        status, latency_s = aesgb.aes_srv_wait(srv, t)
        assert status == 0 and latency_s > 0
    finally:
        aesgb.aes_srv_destroy(srv)
    assert np.array_equal(z.cpu().numpy(), orc.ecb(0, key16, x.cpu().numpy(), nthreads=8))
