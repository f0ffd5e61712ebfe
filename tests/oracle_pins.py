"""Pins for the CPU oracle: checks against what the paper and the mathematics fix.

Each ``pin_*`` function takes an ``oracle.Oracle`` and raises AssertionError if
the oracle disagrees with:

* values the paper prints (``tests/golden/*.txt``, each line cited),
* the field axioms and closed forms of GF(2^8) (brute force over all elements),
* invariants of the S-box, of MixColumns and of ECB,
* an independent library (OpenSSL through the ``cryptography`` package) on
  random keys and blocks, for every key size and mode the oracle offers.

``test_oracle.py`` runs every pin on the real oracle; ``test_oracle_mutants.py``
builds oracle variants with one planted mistake each and checks that at least
one pin fails for every variant.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def paper_gf_examples():
    return [tuple(t[:4]) for t in _golden_lines("paper_gf_examples.txt")]


def paper_matrices():
    mats: dict[str, list[list[int]]] = {}
    for t in _golden_lines("paper_matrices.txt"):
        mats.setdefault(t[0], []).append([int(v, 16) for v in t[1:]])
    return {k: np.array(v, dtype=np.int64) for k, v in mats.items()}


# ---------------------------------------------------------------------------
# GF(2^8)
# ---------------------------------------------------------------------------

def pin_paper_gf_examples(o):
    """Def. 1-3 worked examples, eqs (7)-(17)."""
    for op, a, b, exp in paper_gf_examples():
        if op == "add":
            assert o.gf_add(int(a, 16), int(b, 16)) == int(exp, 16), (op, a, b)
        elif op == "clmul":
            assert o.clmul(int(a, 16), int(b, 16)) == int(exp, 16), (op, a, b)
        elif op == "polymod":
            assert o.poly_mod(int(a, 16)) == int(exp, 16), (op, a)
        elif op == "mul":
            assert o.gf_mul(int(a, 16), int(b, 16)) == int(exp, 16), (op, a, b)
        elif op == "xtime":
            assert o.xtime(int(a, 16)) == int(exp, 16), (op, a)
        elif op == "modulus":
            m = int(a, 16)
            # x^8 reduces to m(x) - x^8: the remainder of x^8 = clmul(0x80, 2).
            assert o.poly_mod(o.clmul(0x80, 0x02)) == (m & 0xFF), "m(x) of eq (8)"
        else:
            raise AssertionError(f"unknown fixture op {op}")


def _poly_divmod(num: int, den: int) -> int:
    """Remainder of GF(2)[x] division, written here from the definition."""
    dd = den.bit_length() - 1
    while num and num.bit_length() - 1 >= dd:
        num ^= den << (num.bit_length() - 1 - dd)
    return num


def pin_modulus_irreducible(o):
    """m(x) of eq (8) has no factor of degree 1..4 (brute force), so GF(2^8) is a field;
    and the oracle's reduction of x^8 equals m(x) - x^8."""
    m = 0x100 | o.poly_mod(o.clmul(0x80, 0x02))
    assert m == 0x11B
    for d in range(2, 32):  # every polynomial of degree 1..4
        assert _poly_divmod(m, d) != 0, f"m(x) divisible by {d:#x}"


def pin_gf_field_axioms(o):
    """xtime == multiplication by x; commutativity and identity for all pairs
    involving 0..255 x {0,1,2,3,0x53}; distributivity and associativity on a
    seeded sample; every nonzero element has exactly one inverse."""
    for a in range(256):
        assert o.xtime(a) == o.gf_mul(a, 2), f"xtime({a:#x}) != {a:#x}*02"
        assert o.gf_mul(a, 1) == a and o.gf_mul(a, 0) == 0
        assert o.gf_add(a, a) == 0
    rng = np.random.default_rng(1902052301)
    trip = rng.integers(0, 256, size=(600, 3))
    for a, b, c in trip.tolist():
        assert o.gf_mul(a, b) == o.gf_mul(b, a)
        assert o.gf_mul(a, o.gf_add(b, c)) == o.gf_add(o.gf_mul(a, b), o.gf_mul(a, c))
        assert o.gf_mul(o.gf_mul(a, b), c) == o.gf_mul(a, o.gf_mul(b, c))
    assert o.gf_inv(0) == 0
    for a in range(1, 256):
        inv = o.gf_inv(a)
        assert o.gf_mul(a, inv) == 1, f"inv({a:#x})"
        others = [b for b in (1, 2, 3, 0x8D, 0xF6) if b != inv]
        assert all(o.gf_mul(a, b) != 1 for b in others)


# ---------------------------------------------------------------------------
# S-box
# ---------------------------------------------------------------------------

def pin_sbox_invariants(o):
    """Bijective; S(0) = 0x63 (the affine constant, inverse of 0 being 0);
    no fixed and no complement-fixed points; InvS is its inverse; maximum
    differential count 4 (true of any affine map of field inversion)."""
    s = o.sbox_table().astype(np.int64)
    inv = o.inv_sbox_table().astype(np.int64)
    assert sorted(s.tolist()) == list(range(256))
    assert s[0] == 0x63
    x = np.arange(256)
    assert np.all(s != x) and np.all(s != (x ^ 0xFF))
    assert np.all(inv[s] == x) and np.all(s[inv] == x)
    worst = 0
    for dx in range(1, 256):
        counts = np.bincount(s ^ s[x ^ dx], minlength=256)
        worst = max(worst, int(counts.max()))
    assert worst == 4, worst


# ---------------------------------------------------------------------------
# Round transformations
# ---------------------------------------------------------------------------

def pin_paper_matrices(o):
    """A of eq (20) matches the paper; A * A_INV = I over GF(2^8);
    MixColumns then InvMixColumns is the identity on random states."""
    mats = paper_matrices()
    a = o.mix_matrix(False).astype(np.int64)
    assert np.array_equal(a, mats["A_MIX"])
    ai = o.mix_matrix(True).astype(np.int64)
    for r in range(4):
        for c in range(4):
            acc = 0
            for k in range(4):
                acc ^= o.gf_mul(int(a[r, k]), int(ai[k, c]))
            assert acc == (1 if r == c else 0), (r, c)
    rng = np.random.default_rng(1902052302)
    for _ in range(50):
        st = rng.integers(0, 256, 16, dtype=np.uint8)
        assert np.array_equal(o.inv_mix_columns(o.mix_columns(st)), st)


def pin_ttables(o):
    """eqs (22)-(25): T_k(w)[row] = coefficient(k,row) * sbox(w) with the
    coefficients printed in the paper; and eq (26): one T-table round equals
    SubBytes, ShiftRows, MixColumns, AddRoundKey (Defs. 4-7) on random states."""
    mats = paper_matrices()
    for k in range(4):
        coef = mats[f"T{k}"][0]
        for w in range(256):
            s = o.sbox(w)
            exp = [o.gf_mul(int(c), s) for c in coef]
            assert o.ttable(k, w).tolist() == exp, (k, w)
    rng = np.random.default_rng(1902052303)
    for _ in range(300):
        st = rng.integers(0, 256, 16, dtype=np.uint8)
        rk = rng.integers(0, 256, 16, dtype=np.uint8)
        assert np.array_equal(o.tround(st, rk), o.round(st, rk))


def pin_roundtrip(o):
    """InvCipher(Cipher(x)) = x, and the equivalent inverse cipher driven by
    the InvMixColumns'd schedule equals the straightforward inverse cipher
    (FIPS-197 5.3.5), for every key size."""
    rng = np.random.default_rng(1902052304)
    for nbytes in (16, 24, 32):
        for _ in range(40):
            key = rng.integers(0, 256, nbytes, dtype=np.uint8)
            w, nr = o.key_expansion(key)
            assert nr == {16: 10, 24: 12, 32: 14}[nbytes]
            assert w.size == 16 * (nr + 1)
            assert np.array_equal(w[: nbytes], key)
            dw = o.eq_inv_schedule(w, nr)
            blk = rng.integers(0, 256, 16, dtype=np.uint8)
            ct = o.cipher(w, nr, blk)
            assert np.array_equal(o.inv_cipher(w, nr, ct), blk)
            assert np.array_equal(o.eq_inv_cipher(dw, nr, ct), blk)


def pin_ecb_invariants(o):
    """ECB (eq (1)): equal plaintext blocks give equal ciphertext blocks, and
    permuting the input blocks permutes the output blocks the same way."""
    rng = np.random.default_rng(1902052305)
    key = rng.integers(0, 256, 16, dtype=np.uint8)
    blocks = rng.integers(0, 256, (64, 16), dtype=np.uint8)
    blocks[10] = blocks[3]
    blocks[40] = blocks[3]
    ct = o.ecb_encrypt(key, blocks.reshape(-1)).reshape(64, 16)
    assert np.array_equal(ct[10], ct[3]) and np.array_equal(ct[40], ct[3])
    perm = rng.permutation(64)
    ct_p = o.ecb_encrypt(key, blocks[perm].reshape(-1)).reshape(64, 16)
    assert np.array_equal(ct_p, ct[perm])
    assert np.array_equal(o.ecb_decrypt(key, ct.reshape(-1)).reshape(64, 16), blocks)


# ---------------------------------------------------------------------------
# Independent library (OpenSSL through the `cryptography` package)
# ---------------------------------------------------------------------------

def _lib_cipher(mode_name, key, arg=None):
    from cryptography.hazmat.primitives.ciphers import Cipher, algorithms, modes
    try:  # newer releases keep CFB among the "decrepit" modes
        from cryptography.hazmat.decrepit.ciphers.modes import CFB
    except ImportError:
        CFB = modes.CFB
    mode = {"ecb": lambda: modes.ECB(), "ctr": lambda: modes.CTR(bytes(arg)),
            "cbc": lambda: modes.CBC(bytes(arg)), "cfb": lambda: CFB(bytes(arg))}[mode_name]()
    return Cipher(algorithms.AES(bytes(key)), mode)


def pin_library_ecb(o):
    """ECB encrypt and decrypt agree with OpenSSL for 128/192/256-bit keys."""
    rng = np.random.default_rng(1902052306)
    for nbytes in (16, 24, 32):
        for _ in range(12):
            key = rng.integers(0, 256, nbytes, dtype=np.uint8)
            data = rng.integers(0, 256, 16 * 37, dtype=np.uint8)
            c = _lib_cipher("ecb", key)
            enc = c.encryptor()
            exp_ct = enc.update(data.tobytes()) + enc.finalize()
            assert o.ecb_encrypt(key, data).tobytes() == exp_ct, nbytes
            dec = c.decryptor()
            exp_pt = dec.update(data.tobytes()) + dec.finalize()
            assert o.ecb_decrypt(key, data).tobytes() == exp_pt, nbytes


def pin_library_ctr(o):
    """CTR (eq (5)) agrees with OpenSSL, including a counter that wraps 2^64
    and 2^128."""
    rng = np.random.default_rng(1902052307)
    starts = [rng.integers(0, 256, 16, dtype=np.uint8) for _ in range(4)]
    wrap64 = np.zeros(16, np.uint8); wrap64[8:] = 0xFF; wrap64[15] = 0xF0
    wrap128 = np.full(16, 0xFF, np.uint8); wrap128[15] = 0xF8
    for i, ctr0 in enumerate(starts + [wrap64, wrap128]):
        key = rng.integers(0, 256, (16, 24, 32)[i % 3], dtype=np.uint8)
        data = rng.integers(0, 256, 16 * 40, dtype=np.uint8)
        enc = _lib_cipher("ctr", key, ctr0).encryptor()
        exp = enc.update(data.tobytes()) + enc.finalize()
        assert o.ctr(key, ctr0, data).tobytes() == exp, i


def pin_library_cbc(o):
    """CBC encrypt and decrypt agree with OpenSSL."""
    rng = np.random.default_rng(1902052308)
    for nbytes in (16, 24, 32):
        key = rng.integers(0, 256, nbytes, dtype=np.uint8)
        iv = rng.integers(0, 256, 16, dtype=np.uint8)
        data = rng.integers(0, 256, 16 * 33, dtype=np.uint8)
        c = _lib_cipher("cbc", key, iv)
        enc = c.encryptor()
        exp_ct = enc.update(data.tobytes()) + enc.finalize()
        assert o.cbc_encrypt(key, iv, data).tobytes() == exp_ct
        dec = c.decryptor()
        exp_pt = dec.update(exp_ct) + dec.finalize()
        assert o.cbc_decrypt(key, iv, np.frombuffer(exp_ct, np.uint8)).tobytes() == exp_pt
        assert exp_pt == data.tobytes()


def pin_library_cfb(o):
    """CFB (eq (3) read by its text: full-block CFB) agrees with OpenSSL's
    CFB-128, both directions; decrypt(encrypt(x)) = x."""
    rng = np.random.default_rng(1902052309)
    for nbytes in (16, 24, 32):
        key = rng.integers(0, 256, nbytes, dtype=np.uint8)
        iv = rng.integers(0, 256, 16, dtype=np.uint8)
        data = rng.integers(0, 256, 16 * 29, dtype=np.uint8)
        c = _lib_cipher("cfb", key, iv)
        enc = c.encryptor()
        exp_ct = enc.update(data.tobytes()) + enc.finalize()
        assert o.cfb_encrypt(key, iv, data).tobytes() == exp_ct
        dec = c.decryptor()
        exp_pt = dec.update(exp_ct) + dec.finalize()
        assert o.cfb_decrypt(key, iv, np.frombuffer(exp_ct, np.uint8)).tobytes() == exp_pt
        assert exp_pt == data.tobytes()


ALL_PINS = [
    pin_paper_gf_examples,
    pin_modulus_irreducible,
    pin_gf_field_axioms,
    pin_sbox_invariants,
    pin_paper_matrices,
    pin_ttables,
    pin_roundtrip,
    pin_ecb_invariants,
    pin_library_ecb,
    pin_library_ctr,
    pin_library_cbc,
    pin_library_cfb,
]
