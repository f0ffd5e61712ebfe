"""Build a batch of ECB messages on the device for the batch tests: random
messages packed back to back in an input arena, one random key per message,
round keys uploaded to a key arena, and the aes_desc table."""
import numpy as np

from paper_1902_05234_gb300 import aesgb


class DeviceBatch:
    def __init__(self, torch, lengths, keybits, dirs, seed=0, inplace=False, fill=0x5A):
        self.torch = torch
        self.lengths = np.asarray(lengths, np.int64)
        self.keybits = np.asarray(keybits, np.int64)
        self.dirs = np.asarray(dirs, np.int64)
        n = self.n = len(self.lengths)
        assert np.all(self.lengths % 16 == 0)
        self.offsets = np.zeros(n + 1, np.int64)
        np.cumsum(self.lengths, out=self.offsets[1:])
        total = int(self.offsets[-1])
        g = np.random.default_rng(190205230 + seed)
        self.data = g.integers(0, 256, total, dtype=np.uint8) if total else np.zeros(0, np.uint8)
        self.keys = [g.integers(0, 256, int(kb) // 8, dtype=np.uint8).tobytes() for kb in self.keybits]
        rks = np.zeros((max(n, 1), 64), np.uint32)       # 256-byte stride per message
        self.nrounds = np.zeros(n, np.int64)
        for i in range(n):
            enc, dec, nr = aesgb.aes_expand_key(int(self.keybits[i]), self.keys[i])
            rks[i, :60] = enc if self.dirs[i] == 0 else dec
            self.nrounds[i] = nr
        self.in_dev = torch.from_numpy(self.data).cuda() if total else torch.zeros(16, dtype=torch.uint8,
                                                                                  device="cuda")
        self.out_dev = self.in_dev if inplace else torch.full((max(total, 16),), fill, dtype=torch.uint8,
                                                              device="cuda")
        self.rk_dev = torch.from_numpy(rks.view(np.uint8).reshape(-1)).cuda()
        base_in, base_out, base_rk = self.in_dev.data_ptr(), self.out_dev.data_ptr(), self.rk_dev.data_ptr()
        self.table = aesgb.pack_descs(base_rk + 256 * np.arange(n, dtype=np.uint64),
                                      base_in + self.offsets[:-1].astype(np.uint64),
                                      base_out + self.offsets[:-1].astype(np.uint64),
                                      self.lengths // 16, self.nrounds, self.dirs)
        self.upload()

    def upload(self):
        t = self.torch
        self.desc_dev = t.from_numpy(self.table.view(np.uint8).copy()).cuda()

    def workspace(self):
        t = self.torch
        nbytes = aesgb.aes_batch_workspace_bytes(self.n)
        return t.empty(max(nbytes, 256), dtype=t.uint8, device="cuda"), nbytes

    def output(self) -> np.ndarray:
        self.torch.cuda.synchronize()
        return self.out_dev.cpu().numpy()[: int(self.offsets[-1])]

    def message(self, arr, i):
        return arr[self.offsets[i]: self.offsets[i + 1]]
