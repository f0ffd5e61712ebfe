"""The C ABI from plain C: tests/c_client/aes_client.c is compiled as strict
C99 against include/aesgb.h (-Wall -Wextra -Werror -pedantic), linked to
libaesgb.so and the CUDA runtime, and run.  Key expansion and error codes are
checked on the CPU; ECB on the device against the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "c_client", "aes_client.c")


def cuda_lib_dir():
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
              "/usr/local/cuda/targets/x86_64-linux/lib"):
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return d
    return None


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda_lib = cuda_lib_dir()
    if cuda_lib is None:
        pytest.skip("no CUDA runtime library to link")
    lib = aesgb.LIB_PATH
    assert os.path.exists(lib), "build the library first"
    exe = str(tmp_path_factory.mktemp("c_client") / "aes_client")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-O1",
           "-I", os.path.join(ROOT, "include"), "-isystem", "/usr/local/cuda/include", SRC, "-o", exe,
           lib, f"-Wl,-rpath,{os.path.dirname(lib)}", f"-L{cuda_lib}", "-lcudart", f"-Wl,-rpath,{cuda_lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def run(exe, *args):
    r = subprocess.run([exe, *args], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    return r.stdout.split("\n")


@pytest.mark.parametrize("keybits", [128, 192, 256])
def test_c_key_expansion_matches_oracle(orc, client, keybits):
    key = wl.random_key(keybits, 500 + keybits).tobytes()
    out = run(client, "keys", key.hex())
    nr = int(out[0])
    w, onr = orc.key_expansion(key)
    assert nr == onr
    assert bytes.fromhex(out[1]) == w.tobytes()[:16 * (nr + 1)]
    dw = orc.eq_inv_schedule(w, nr)
    assert bytes.fromhex(out[2]) == dw.tobytes()[:16 * (nr + 1)]


def test_c_error_codes(client):
    out = run(client, "errors")
    assert out[:3] == ["-2", "-1", "-3"]
    assert out[3].startswith("AES_E_OVERLAP")


@pytest.mark.gpu
@pytest.mark.parametrize("keybits", [128, 256])
def test_c_ecb_on_device_matches_oracle(orc, client, tmp_path, keybits):
    key = wl.random_key(keybits, 510 + keybits).tobytes()
    data = wl.random_bytes(16 * 70_001, 511)
    src, enc, dec = (str(tmp_path / n) for n in ("in.bin", "enc.bin", "dec.bin"))
    data.tofile(src)
    run(client, "ecb", key.hex(), src, enc, dec)
    assert np.array_equal(np.fromfile(enc, np.uint8), orc.ecb(0, key, data, nthreads=8))
    assert np.array_equal(np.fromfile(dec, np.uint8), data)
