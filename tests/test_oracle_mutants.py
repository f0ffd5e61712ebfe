"""Plant one mistake at a time in the oracle (on the CPU, in a separately
built copy) and check that at least one pin catches it.  This is the evidence
that the pins constrain every part of the oracle: a dropped term, a wrong
constant, index or direction each make some pin fail."""
import os

import pytest

import oracle
from oracle import build as obuild
import oracle_pins as pins

# mutant id -> what it plants (the MUTANT(n) sites of aes_oracle.c)
MUTANTS = {
    1: "xtime reduces with 0x1d instead of 0x1b",
    2: "polynomial reduction by x^8+x^4+x^3+x^2+1 instead of m(x)",
    3: "affine constant 0x62 instead of 0x63",
    4: "affine map uses b_{i+3} instead of b_{i+4}",
    5: "ShiftRows rotates rows right instead of left",
    6: "MixColumns uses the transpose of A",
    7: "final round applies MixColumns (Algorithm 1 as printed)",
    8: "Rcon starts at x instead of 1",
    9: "AES-256 key schedule drops the extra SubWord",
    10: "InvMixColumns with 0b and 0d swapped",
    11: "equivalent-inverse schedule also transforms round key 0",
    12: "CTR counter incremented little-endian",
    13: "T1 built with the coefficients of T3",
    14: "CFB feeds C_{i-1} xor P_{i-1} to the cipher (eq (3) as printed)",
}


@pytest.mark.parametrize("mid", sorted(MUTANTS), ids=lambda m: f"m{m}")
def test_mutant_is_caught(mid, tmp_path):
    pytest.importorskip("cryptography")
    path = os.path.join(str(tmp_path), f"liboracle_m{mid}.so")
    obuild.build(out_path=path, mutant=mid, force=True)
    o = oracle.Oracle(oracle.load(path))
    assert o.lib.orc_mutant_id() == mid
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(o)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"mutant {mid} ({MUTANTS[mid]}) passed every pin"
