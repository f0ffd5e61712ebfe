"""The CPU oracle against its pins (no GPU): paper values, closed forms,
invariants and an independent library.  See ``oracle_pins.py``."""
import pytest

import oracle_pins as pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    if pin.__name__.startswith("pin_library"):
        pytest.importorskip("cryptography")
    pin(orc)


def test_gf_inverse_brute_force_small(orc):
    # brute force on every pair: exactly one b with a*b = 1 for each a != 0
    for a in range(1, 256):
        hits = [b for b in range(256) if orc.gf_mul(a, b) == 1]
        assert hits == [orc.gf_inv(a)]


def test_ctr_counter_arithmetic(orc):
    import numpy as np
    c0 = np.zeros(16, np.uint8)
    c0[15] = 0xFF
    assert orc.ctr_block(c0, 1).tolist() == [0] * 14 + [1, 0]
    full = np.full(16, 0xFF, np.uint8)
    assert orc.ctr_block(full, 1).tolist() == [0] * 16     # wraps mod 2^128
    assert orc.ctr_block(c0, 0).tolist() == c0.tolist()


def test_multithreaded_ecb_matches_single(orc):
    import numpy as np
    rng = np.random.default_rng(7)
    key = rng.integers(0, 256, 32, dtype=np.uint8)
    data = rng.integers(0, 256, 16 * 1001, dtype=np.uint8)
    for d in (0, 1):
        assert np.array_equal(orc.ecb(d, key, data, nthreads=1), orc.ecb(d, key, data, nthreads=5))
