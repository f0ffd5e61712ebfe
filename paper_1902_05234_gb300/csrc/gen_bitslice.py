#!/usr/bin/env python3
"""gen_bitslice.py -- writes bitslice_circuits.h, the straight-line LOP3
circuits of the constant-time (bitsliced) AES kernel.

Every gate is one 3-input logic instruction (LOP3: any boolean function of
three 32-bit words, bit by bit), so the cost of a circuit is its gate count.
The circuits:

  sbox_enc      x (8 planes), m (8 mask planes)  ->  S(x) + m + 63
                (the constant 63 is left to the mask, which the host builds)
  sbox_core_dec x (8 planes)                     ->  o (8 planes), the tower-
                field inverse of the inverse S-box's input, with the affine
                map's constant folded into the gates
  sbox_out_dec  o, m                             ->  S^-1(x) + m
  inv_mix_out   o of a column's 4 bytes, m (32) ->  InvMixColumns(S^-1(x)) + m
  mix_columns   a column (32 planes)             ->  MixColumns(a)

S-box construction (FIPS-197 5.1.1: inversion in GF(2^8) then an affine
map), computed in the tower field GF((2^4)^2) = GF(16)[y]/(y^2 + y + lambda):
  (a1 y + a0)^-1 = (a1 d) y + (a1 + a0) d,  d = (lambda a1^2 + a1 a0 + a0^2)^-1.
  * top layer: the linear forms of x the rest needs (a1, a0, a1 + a0,
    lambda a1^2 + a0^2 and the Mastrovito forms below), as an XOR program;
  * delta: the GF(16) product a1 a0 written as sum_i a1_i (F_ki . a0), each
    term one AND-XOR gate accumulating onto lambda a1^2 + a0^2;
  * d: the four bits of the GF(16) inverse, each one gate over delta's bits
    and first-level gates (gates over three of delta's bits), chosen by
    exhaustive search to share first-level gates;
  * the products a1 d and (a1 + a0) d in the same Mastrovito form, sharing
    the forms F_ki . d;
  * bottom layer: phi (tower -> AES field) and, for encryption, the affine
    matrix, with the masks, as an XOR program.
XOR programs come from a closure construction that builds every target as
the XOR of at most three signals already available -- one gate per target,
the lower bound, when it reaches all of them -- or else from a randomised
greedy search that repeatedly names the pair or triple of variables whose
sharing saves the most gates.

The tower (GF(16) modulus, lambda) and the isomorphism are parameters; the
defaults were chosen by `--search`, which tries every irreducible quartic,
every lambda of trace 1 and every isomorphism and keeps the cheapest.

Usage:  python gen_bitslice.py            # writes bitslice_circuits.h
        python gen_bitslice.py --check    # exit 1 if the header is stale
        python gen_bitslice.py --search   # print the cost of every tower (minutes, on all cores)
"""
import argparse
import itertools
import os
import random
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_PATH = os.path.join(HERE, "bitslice_circuits.h")

# ------------------------------------------------------------ AES field
def aes_mul(a, b):
    """GF(2^8) product modulo x^8 + x^4 + x^3 + x + 1 (FIPS-197 4.2)."""
    p = 0
    for i in range(8):
        if (b >> i) & 1:
            p ^= a << i
    for d in range(14, 7, -1):
        if (p >> d) & 1:
            p ^= 0x11B << (d - 8)
    return p


def aes_inv(a):
    return 0 if a == 0 else next(b for b in range(1, 256) if aes_mul(a, b) == 1)


def affine(b):
    """FIPS-197 5.1.1 affine map, constant 63 included."""
    r = 0
    for i in range(8):
        r |= (((b >> i) ^ (b >> ((i + 4) % 8)) ^ (b >> ((i + 5) % 8)) ^ (b >> ((i + 6) % 8))
               ^ (b >> ((i + 7) % 8))) & 1) << i
    return r ^ 0x63


SBOX = [affine(aes_inv(x)) for x in range(256)]
ISBOX = [0] * 256
for _x in range(256):
    ISBOX[SBOX[_x]] = _x


# ------------------------------------------------ GF(2) matrices, rows as masks
def parity(v):
    return bin(v).count("1") & 1


def apply(m, x):
    return sum(parity(m[i] & x) << i for i in range(len(m)))


def from_cols(cols, nout=8):
    return [sum(((cols[j] >> i) & 1) << j for j in range(len(cols))) for i in range(nout)]


def mat_mul(a, b):  # a after b
    return from_cols([apply(a, apply(b, 1 << j)) for j in range(8)])


def mat_inv(m):
    cols = [0] * 8
    for x in range(256):
        y = apply(m, x)
        for j in range(8):
            if y == 1 << j:
                cols[j] = x
    return from_cols(cols)


AFF = from_cols([affine(1 << j) ^ 0x63 for j in range(8)])  # linear part


# ---------------------------------------------------------------- GF(16)
QUARTICS = (0x13, 0x19, 0x1F)  # the irreducible polynomials of degree 4


def g16_mul(a, b, mod):
    p = 0
    for i in range(4):
        if (b >> i) & 1:
            p ^= a << i
    for d in range(6, 3, -1):
        if (p >> d) & 1:
            p ^= mod << (d - 4)
    return p & 15


def g16_inv(a, mod):
    return 0 if a == 0 else next(b for b in range(1, 16) if g16_mul(a, b, mod) == 1)


def g16_trace(a, mod):
    t, x = a, a
    for _ in range(3):
        x = g16_mul(x, x, mod)
        t ^= x
    return t


class Tower:
    """GF((2^4)^2) with GF(16) = GF(2)[z]/(mod), y^2 + y + lam, and the
    isomorphism to the AES field that sends the first primitive tower
    element g to the beta_index-th root (in increasing order) of its
    minimal polynomial."""

    def __init__(self, mod, lam, beta_index):
        assert g16_trace(lam, mod) == 1, "y^2 + y + lambda must be irreducible"
        self.mod, self.lam = mod, lam
        g = next(c for c in range(2, 256) if self.order(c) == 255)
        gp = [1]
        for _ in range(254):
            gp.append(self.mul(gp[-1], g))
        roots = []
        for beta in range(2, 256):
            bp = [1]
            for _ in range(254):
                bp.append(aes_mul(bp[-1], beta))
            phi = {0: 0}
            for k in range(255):
                phi[gp[k]] = bp[k]
            if len(set(bp)) == 255:
                m = from_cols([phi[1 << j] for j in range(8)])
                if all(apply(m, t) == phi[t] for t in range(256)):
                    roots.append((beta, m))
        self.nroots = len(roots)
        self.beta, self.t2a = roots[beta_index]
        self.a2t = mat_inv(self.t2a)

    def mul(self, a, b):
        a1, a0, b1, b0 = a >> 4, a & 15, b >> 4, b & 15
        m = self.mod
        h = g16_mul(a1, b1, m) ^ g16_mul(a1, b0, m) ^ g16_mul(a0, b1, m)
        lo = g16_mul(g16_mul(a1, b1, m), self.lam, m) ^ g16_mul(a0, b0, m)
        return h << 4 | lo

    def order(self, c):
        x = c
        for k in range(1, 256):
            if x == 1:
                return k
            x = self.mul(x, c)
        return 0

    def mastrovito(self):
        """F[k][i]: 4-bit mask over v with (u v)_k = sum_i u_i (F[k][i] . v)."""
        F = [[0] * 4 for _ in range(4)]
        for i in range(4):
            for j in range(4):
                p = g16_mul(1 << i, 1 << j, self.mod)
                for k in range(4):
                    if (p >> k) & 1:
                        F[k][i] |= 1 << j
        return F

    def lin_delta(self):
        """rows (over the 8 tower bits) of lambda a1^2 + a0^2."""
        cols = []
        for j in range(8):
            h, lo = (1 << j) >> 4, (1 << j) & 15
            cols.append(g16_mul(self.lam, g16_mul(h, h, self.mod), self.mod) ^ g16_mul(lo, lo, self.mod))
        return from_cols(cols, 4)


# ---------------------------------------------------------- circuit builder
class Circuit:
    """Variables 0..nin-1 are inputs, nin+g the output of gate g.  A signal is
    (variable, negated); consumers fold a negation into their truth table."""

    def __init__(self, name, nin):
        self.name, self.nin = name, nin
        self.gates = []  # (lut, a, b, c)
        self.outs = []

    def gate(self, f, sigs):
        lut = 0
        for p in range(8):
            bits = ((p >> 2) & 1, (p >> 1) & 1, p & 1)
            if f(*[bits[i] ^ sigs[i][1] for i in range(len(sigs))]):
                lut |= 1 << p
        v = [s[0] for s in sigs] + [sigs[0][0]] * (3 - len(sigs))
        self.gates.append((lut, v[0], v[1], v[2]))
        return (self.nin + len(self.gates) - 1, 0)

    def raw(self, lut, a, b, c):
        self.gates.append((lut, a, b, c))
        return (self.nin + len(self.gates) - 1, 0)

    def xor(self, sigs, const=0):
        return self.gate(lambda *b: (sum(b) + const) & 1, sigs)

    def eval(self, inputs):
        """inputs: list of python ints (bit vectors); returns output ints."""
        full = (1 << 512) - 1
        v = list(inputs)
        for lut, a, b, c in self.gates:
            x, y, z = v[a], v[b], v[c]
            r = 0
            for p in range(8):
                if (lut >> p) & 1:
                    r |= (x if p & 4 else full ^ x) & (y if p & 2 else full ^ y) & (z if p & 1 else full ^ z)
            v.append(r)
        out = []
        for var, neg in self.outs:
            out.append(v[var] ^ (full if neg else 0))
        return out


def _row_cost(n):
    return max(0, (n - 1 + 1) // 2)  # ceil((n - 1) / 2) XOR3 gates for n leaves


def greedy_plan(nin, rows, rng, noise):
    rows = [set(r) for r in rows]
    nv = nin
    defs = []
    while True:
        cnt = {}
        for r in rows:
            lst = sorted(r)
            for c in itertools.combinations(lst, 2):
                cnt[c] = cnt.get(c, 0) + 1
            if len(lst) >= 3:
                for c in itertools.combinations(lst, 3):
                    cnt[c] = cnt.get(c, 0) + 1
        best, best_s = None, 0.0
        for c, k in cnt.items():
            if k < 2:
                continue
            cs = set(c)
            sav = -1
            for r in rows:
                if cs <= r:
                    sav += _row_cost(len(r)) - _row_cost(len(r) - len(c) + 1)
            if sav <= 0:
                continue
            s = sav + (rng.random() * 0.9 if noise else 0.0)
            if s > best_s:
                best, best_s = c, s
        if best is None:
            break
        cs = set(best)
        for r in rows:
            if cs <= r:
                r -= cs
                r.add(nv)
        defs.append(best)
        nv += 1
    return defs, rows


def closure_plan(nin, masks):
    """One gate per distinct target: repeatedly build a target that is the
    XOR of at most three signals already available (inputs and targets built
    before).  That meets the lower bound of one gate per target that is not an
    input.  Of the targets reachable at each step, the one whose shallowest
    decomposition is shallowest is built first, so the circuit stays shallow.
    Returns [(mask, (vars...))] in build order, or None if some target never
    becomes reachable this way."""
    avail = {1 << j: j for j in range(nin)}
    depth = {j: 0 for j in range(nin)}
    pending = sorted({m for m in masks if m not in avail})
    plan = []
    nv = nin
    while pending:
        items = sorted(avail.items())
        pairs = {}  # xor of two available signals -> the shallowest such pair
        for (ma, va), (mb, vb) in itertools.combinations(items, 2):
            x = ma ^ mb
            d = max(depth[va], depth[vb])
            if x not in pairs or d < pairs[x][0]:
                pairs[x] = (d, (va, vb))
        hit = None  # (depth, target, vars)
        for t in pending:
            best = None
            if t in pairs:
                best = (pairs[t][0] + 1, pairs[t][1])
            for ma, va in items:
                r = pairs.get(t ^ ma)
                if r is not None and va not in r[1]:
                    d = max(depth[va], r[0]) + 1
                    if best is None or d < best[0]:
                        best = (d, (va,) + r[1])
            if best is not None and (hit is None or best[0] < hit[0]):
                hit = (best[0], t, best[1])
        if hit is None:
            return None
        d, t, vs = hit
        plan.append((t, vs))
        avail[t] = nv
        depth[nv] = d
        nv += 1
        pending.remove(t)
    return plan


def xor_program(C, ins, targets, restarts, seed):
    """ins: signals; targets: list of (mask over ins, const).  Adds the gates of
    the cheapest plan found (the closure construction when it reaches its
    lower bound, else the greedy search) and returns one signal per target."""
    nin = len(ins)
    plan = closure_plan(nin, [m for m, _ in targets])
    rows = [[i for i in range(nin) if (m >> i) & 1] for m, _ in targets]
    rng = random.Random(seed)
    best = None
    for r in range(restarts):
        defs, fin = greedy_plan(nin, rows, rng, noise=r > 0)
        cost = len(defs) + sum(_row_cost(len(f)) for f in fin)
        if best is None or cost < best[0]:
            best = (cost, defs, fin)
    if plan is not None and len(plan) < best[0]:
        sig_of = list(ins)  # plan variable -> signal: the inputs, then the targets in build order
        by_mask = {1 << j: ins[j] for j in range(nin)}
        for t, vs in plan:
            g = C.xor([sig_of[v] for v in vs])
            sig_of.append(g)
            by_mask[t] = g
        return [(by_mask[m][0], by_mask[m][1] ^ const) for m, const in targets]
    _, defs, fin = best
    sig = list(ins)
    for d in defs:
        sig.append(C.xor([sig[i] for i in d]))
    outs = []
    for (m, const), leaves in zip(targets, fin):
        leaves = sorted(leaves)
        if not leaves:
            raise ValueError("zero target")
        cur = [sig[i] for i in leaves]
        while len(cur) > 3:
            cur = [C.xor(cur[:3])] + cur[3:]
        if len(cur) == 1:
            outs.append((cur[0][0], cur[0][1] ^ const))
        else:
            outs.append(C.xor(cur, const))
    return outs


def _lop(lut, a, b, c, full=0xFFFF):
    r = 0
    for p in range(8):
        if (lut >> p) & 1:
            r |= (a if p & 4 else full ^ a) & (b if p & 2 else full ^ b) & (c if p & 1 else full ^ c)
    return r


def _lut_for(T, a, b, c, full=0xFFFF):
    """LUT with _lop(LUT, a, b, c) == T, or None if T is not a function of (a, b, c)."""
    lut = 0
    for p in range(8):
        m = (a if p & 4 else full ^ a) & (b if p & 2 else full ^ b) & (c if p & 1 else full ^ c)
        t = T & m
        if t and t != m:
            return None
        if t:
            lut |= 1 << p
    return lut


_INV_PLANS = {}
_INV_MAX_COMBOS = 4_000_000


def _prod(xs):
    r = 1
    for x in xs:
        r *= x
    return r


def inverse_plan(mod):
    """A LOP3 program for the 4 bits of the GF(16) inverse over inputs x0..x3.
    Every output is one gate over inputs and first-level gates (gates over three
    inputs); the search picks, per output, a realisation over one first-level
    gate and two inputs or over two first-level gates and one input, so that
    the outputs together use the fewest distinct first-level gates.  Returns
    (firsts, finals): firsts = [(lut, i, j, k)], finals = [(lut, s1, s2, s3)]
    with s = ('x', i) or ('g', index into firsts)."""
    if mod in _INV_PLANS:
        return _INV_PLANS[mod]
    X = [sum(((v >> i) & 1) << v for v in range(16)) for i in range(4)]
    outs = [sum(((g16_inv(x, mod) >> k) & 1) << x for x in range(16)) for k in range(4)]
    firsts = {}
    for t in itertools.combinations(range(4), 3):
        for lut in range(256):
            f = _lop(lut, X[t[0]], X[t[1]], X[t[2]])
            if f not in firsts and f not in (0, 0xFFFF) and f not in X:
                firsts[f] = (lut, t)
    fl = sorted(firsts)
    single = [[] for _ in range(4)]  # (g, i, j, lut)
    pair = [[] for _ in range(4)]    # (g1, g2, i, lut)
    for k in range(4):
        for g in fl:
            for i, j in itertools.combinations(range(4), 2):
                lut = _lut_for(outs[k], g, X[i], X[j])
                if lut is not None:
                    single[k].append((g, i, j, lut))
                    break
    for k in range(4):
        if single[k]:
            continue
        for a, g1 in enumerate(fl):
            for g2 in fl[a + 1:]:
                for i in range(4):
                    lut = _lut_for(outs[k], g1, g2, X[i])
                    if lut is not None:
                        pair[k].append((g1, g2, i, lut))
                        break
    options = [[("s",) + o for o in single[k]] if single[k] else [("p",) + o for o in pair[k]] for k in range(4)]
    # The choice below is exhaustive up to _INV_MAX_COMBOS combinations (the
    # default tower's modulus needs about 3.2 million).  Beyond that the
    # longest option lists keep only their first halves, repeatedly, and the
    # plan is the best of what is left: an upper bound, not the optimum.
    while _prod(len(o) for o in options) > _INV_MAX_COMBOS:
        k = max(range(4), key=lambda i: len(options[i]))
        options[k] = options[k][:max(1, len(options[k]) // 2)]
    best = None
    for combo in itertools.product(*options):
        used = set()
        for o in combo:
            used |= {o[1]} if o[0] == "s" else {o[1], o[2]}
        if best is None or len(used) < best[0]:
            best = (len(used), combo, sorted(used))
    _, combo, used = best
    gidx = {g: n for n, g in enumerate(used)}
    fr = [(firsts[g][0],) + firsts[g][1] for g in used]
    finals = []
    for o in combo:
        if o[0] == "s":
            _, g, i, j, lut = o
            finals.append((lut, ("g", gidx[g]), ("x", i), ("x", j)))
        else:
            _, g1, g2, i, lut = o
            finals.append((lut, ("g", gidx[g1]), ("g", gidx[g2]), ("x", i)))
    _INV_PLANS[mod] = (fr, finals)
    return fr, finals


def build_inverse(C, delta, mod):
    """d = delta^-1 in GF(16) (delta's signals are not negated)."""
    assert all(not neg for _, neg in delta)
    x = [v for v, _ in delta]
    firsts, finals = inverse_plan(mod)
    g = [C.raw(lut, x[i], x[j], x[k])[0] for lut, i, j, k in firsts]
    var = lambda s: x[s[1]] if s[0] == "x" else g[s[1]]  # noqa: E731
    return [C.raw(lut, var(a), var(b), var(c)) for lut, a, b, c in finals]


def and_xor_chain(C, terms, acc):
    """acc + sum of u & f over terms [(u, f)]; acc may be None."""
    for u, f in terms:
        if acc is None:
            acc = C.gate(lambda a, b: a & b, [u, f])
        else:
            acc = C.gate(lambda a, b, c: (a & b) ^ c, [u, f, acc])
    return acc


def sbox_core(C, x, mu, tw, IN, const, side, restarts, seed):
    """Tower-field inverse of IN x + const, plus mu; returns signals
    o = (a1 + a0) d + mu_lo (bits 0..3), a1 d + mu_hi (bits 4..7).  Each
    product chain starts from its mu plane, so the masks cost no gate."""
    F = tw.mastrovito()
    a1 = [IN[4 + i] for i in range(4)]
    a0 = [IN[i] for i in range(4)]
    c1 = [(const >> (4 + i)) & 1 for i in range(4)]
    c0 = [(const >> i) & 1 for i in range(4)]
    LIN = tw.lin_delta()
    lin, linc = [], []
    for k in range(4):
        m, c = 0, 0
        for j in range(8):
            if (LIN[k] >> j) & 1:
                m ^= IN[j]
                c ^= (const >> j) & 1
        lin.append(m)
        linc.append(c)
    U, Uc, V, Vc = (a1, c1, a0, c0) if side == 0 else (a0, c0, a1, c1)

    def form(mask4, rows, cs):
        m, c = 0, 0
        for j in range(4):
            if (mask4 >> j) & 1:
                m ^= rows[j]
                c ^= cs[j]
        return (m, c)

    targets = {}
    order = []

    def want(t):
        if t not in targets:
            targets[t] = len(order)
            order.append(t)
        return targets[t]

    iu = [want((U[i], Uc[i])) for i in range(4)]
    ia1 = [want((a1[i], c1[i])) for i in range(4)]
    ias = [want((a1[i] ^ a0[i], c1[i] ^ c0[i])) for i in range(4)]
    il = [want((lin[k], linc[k])) for k in range(4)]
    iF = {(k, i): want(form(F[k][i], V, Vc)) for k in range(4) for i in range(4) if F[k][i]}
    sig = xor_program(C, [(j, 0) for j in range(8)], order, restarts, seed)
    # delta_k = lin_k + sum_i U_i (F_ki . V)
    delta = []
    for k in range(4):
        terms = [(sig[iu[i]], sig[iF[(k, i)]]) for i in range(4) if F[k][i]]
        acc = and_xor_chain(C, terms, sig[il[k]])
        if acc[1]:
            acc = C.xor([acc])
        delta.append(acc)
    d = build_inverse(C, delta, tw.mod)
    dforms = sorted({F[k][i] for k in range(4) for i in range(4) if F[k][i]})
    fsig = xor_program(C, d, [(m, 0) for m in dforms], restarts, seed + 1)
    fmap = dict(zip(dforms, fsig))
    o = [None] * 8
    for k in range(4):
        o[4 + k] = and_xor_chain(C, [(sig[ia1[i]], fmap[F[k][i]]) for i in range(4) if F[k][i]], mu[4 + k])
        o[k] = and_xor_chain(C, [(sig[ias[i]], fmap[F[k][i]]) for i in range(4) if F[k][i]], mu[k])
    return o


def mix_matrix(coef):
    """32x32 rows: output bit 8r+b of a column over input bits 8r'+b'."""
    rows = [0] * 32
    for j in range(32):
        col = [0, 0, 0, 0]
        col[j // 8] = 1 << (j % 8)
        for r in range(4):
            o = 0
            for k in range(4):
                o ^= aes_mul(coef[k], col[(r + k) % 4])
            for b in range(8):
                if (o >> b) & 1:
                    rows[8 * r + b] |= 1 << j
    return rows


MIX = (2, 3, 1, 1)
INV_MIX = (0x0E, 0x0B, 0x0D, 0x09)


def build_all(params, restarts=24, seed=1902):
    """Returns the circuits and the two output maps OUT (o -> S-box output):
    a mask m wanted at an S-box output is supplied as mu = OUT^-1 m."""
    (emod, elam, ebeta, eside), (dmod, dlam, dbeta, dside) = params
    circuits = {}
    x = [(j, 0) for j in range(8)]
    mu = [(8 + j, 0) for j in range(8)]
    # encryption S-box: y = A phi(inv_T(phi^-1 x)) + m   (63 left to the mask)
    tw = Tower(emod, elam, ebeta)
    C = Circuit("sbox_enc", 16)
    o = sbox_core(C, x, mu, tw, tw.a2t, 0, eside, restarts, seed)
    out_enc = mat_mul(AFF, tw.t2a)
    C.outs = xor_program(C, o, [(out_enc[m], 0) for m in range(8)], restarts, seed + 2)
    circuits["sbox_enc"] = C
    # decryption: S^-1(y) = phi(inv_T(phi^-1 A^-1 y + phi^-1 A^-1 63))
    tw = Tower(dmod, dlam, dbeta)
    IN = mat_mul(tw.a2t, mat_inv(AFF))
    const = apply(IN, 0x63)
    C = Circuit("sbox_core_dec", 16)
    C.outs = sbox_core(C, x, mu, tw, IN, const, dside, restarts, seed + 3)
    circuits["sbox_core_dec"] = C
    out_dec = tw.t2a
    C = Circuit("sbox_out_dec", 8)
    C.outs = xor_program(C, x, [(out_dec[m], 0) for m in range(8)], restarts, seed + 4)
    circuits["sbox_out_dec"] = C
    # InvMixColumns of the column's four bytes OUT o_r
    M = mix_matrix(INV_MIX)
    rows = []
    for i in range(32):
        r = 0
        for j in range(32):
            if (M[i] >> j) & 1:
                rr, bb = j // 8, j % 8
                for t in range(8):
                    if (out_dec[bb] >> t) & 1:
                        r ^= 1 << (8 * rr + t)
        rows.append((r, 0))
    C = Circuit("inv_mix_out", 32)
    C.outs = xor_program(C, [(j, 0) for j in range(32)], rows, max(4, restarts // 3), seed + 5)
    circuits["inv_mix_out"] = C
    C = Circuit("mix_columns", 32)
    C.outs = xor_program(C, [(j, 0) for j in range(32)], [(r, 0) for r in mix_matrix(MIX)],
                         max(4, restarts // 2), seed + 6)
    circuits["mix_columns"] = C
    return circuits, (Tower(emod, elam, ebeta), Tower(dmod, dlam, dbeta)), (out_enc, out_dec)


# ------------------------------------------------------------ verification
def planes_of(values, nbits):
    """bit-plane ints: plane j has bit t = bit j of values[t]."""
    return [sum(((v >> j) & 1) << t for t, v in enumerate(values)) for j in range(nbits)]


def unplanes(planes, n):
    return [sum(((planes[j] >> t) & 1) << j for j in range(len(planes))) for t in range(n)]


def verify(circuits, outs):
    """Every circuit against the definitions, masks supplied as mu = OUT^-1 m."""
    mu_enc, mu_dec = mat_inv(outs[0]), mat_inv(outs[1])
    rng = random.Random(5234)
    xs = list(range(256))
    ms = [rng.randrange(256) for _ in range(256)]
    y = unplanes(circuits["sbox_enc"].eval(planes_of(xs, 8) + planes_of([apply(mu_enc, m) for m in ms], 8)), 256)
    assert all(y[t] == SBOX[xs[t]] ^ 0x63 ^ ms[t] for t in range(256)), "sbox_enc"
    o = circuits["sbox_core_dec"].eval(planes_of(xs, 8) + planes_of([apply(mu_dec, m) for m in ms], 8))
    y = unplanes(circuits["sbox_out_dec"].eval(o), 256)
    assert all(y[t] == ISBOX[xs[t]] ^ ms[t] for t in range(256)), "sbox_out_dec"
    # columns: 511 random columns and the all-zero one, each with a random key
    cols = [[rng.randrange(256) for _ in range(4)] for _ in range(511)] + [[0, 0, 0, 0]]
    cm = [[rng.randrange(256) for _ in range(4)] for _ in range(512)]
    ins = []
    for r in range(4):
        ins += circuits["sbox_core_dec"].eval(planes_of([c[r] for c in cols], 8) +
                                              planes_of([apply(mu_dec, m[r]) for m in cm], 8))
    out = circuits["inv_mix_out"].eval(ins)
    for r in range(4):
        got = unplanes(out[8 * r:8 * r + 8], 512)
        for t in range(512):
            s = [ISBOX[v] ^ k for v, k in zip(cols[t], cm[t])]
            want = aes_mul(14, s[r]) ^ aes_mul(11, s[(r + 1) % 4]) ^ aes_mul(13, s[(r + 2) % 4]) \
                ^ aes_mul(9, s[(r + 3) % 4])
            assert got[t] == want, "inv_mix_out"
    ins = []
    for r in range(4):
        ins += planes_of([c[r] for c in cols], 8)
    out = circuits["mix_columns"].eval(ins)
    for r in range(4):
        got = unplanes(out[8 * r:8 * r + 8], 512)
        for t in range(512):
            a = cols[t]
            want = aes_mul(2, a[r]) ^ aes_mul(3, a[(r + 1) % 4]) ^ a[(r + 2) % 4] ^ a[(r + 3) % 4]
            assert got[t] == want, "mix_columns"
    for C in circuits.values():
        assert all(not neg for _, neg in C.outs), C.name + ": negated output"


# ----------------------------------------------------------------- output
DEFAULT = ((0x13, 10, 2, 0), (0x13, 8, 3, 0))  # chosen by --search


def emit(circuits, towers, params, outs):
    lines = [
        "// bitslice_circuits.h -- GENERATED by gen_bitslice.py; do not edit.",
        "//",
        "// Straight-line LOP3 circuits of the constant-time AES kernel.  Gate g of",
        "// a circuit computes variable nin + g = lop3<lut>(v[a], v[b], v[c]); the",
        "// first nin variables are the inputs, out[] names the outputs.  What each",
        "// circuit computes, and how the S-box circuits are built, is described in",
        "// gen_bitslice.py; static_asserts in bitslice.cuh check every table",
        "// against the AES definitions.",
        "//",
    ]
    for name, tw, p in (("encryption", towers[0], params[0]), ("decryption", towers[1], params[1])):
        lines.append(f"// {name} tower: GF(16) modulus 0x{tw.mod:02x}, lambda {tw.lam}, isomorphism "
                     f"g -> {tw.beta} (root {p[2]}), Mastrovito forms on {'a0' if p[3] == 0 else 'a1'}")
    lines += ["#pragma once", "", "#include <cstdint>", "", "namespace aesgb {", "namespace bsc {", "",
              "struct Gate {", "    uint8_t lut;", "    uint16_t a, b, c;", "};", "",
              "template <int NIN, int NG, int NOUT>", "struct Circuit {",
              "    static constexpr int kIn = NIN, kGates = NG, kOut = NOUT;",
              "    Gate g[NG];", "    uint16_t out[NOUT];", "};", ""]
    for name, C in circuits.items():
        lines.append(f"// {name}: {C.nin} inputs, {len(C.gates)} gates, {len(C.outs)} outputs")
        lines.append(f"inline constexpr Circuit<{C.nin}, {len(C.gates)}, {len(C.outs)}> k_{name} = {{")
        lines.append("    {")
        row = []
        for lut, a, b, c in C.gates:
            row.append(f"{{0x{lut:02x}, {a}, {b}, {c}}}")
        for i in range(0, len(row), 6):
            lines.append("        " + ", ".join(row[i:i + 6]) + ",")
        lines.append("    },")
        lines.append("    {" + ", ".join(str(v) for v, _ in C.outs) + "},")
        lines.append("};")
        lines.append("")
    for name, m in (("enc", outs[0]), ("dec", outs[1])):
        inv = mat_inv(m)
        lines.append(f"// mu = OUT_{name}^-1 m: bit i of mu is the parity of (row i & m); a mask m wanted")
        lines.append(f"// at an S-box output enters the {name}ryption circuits as mu.")
        lines.append(f"inline constexpr uint8_t k_mu_{name}[8] = {{" + ", ".join(f"0x{r:02x}" for r in inv) + "};")
        lines.append("")
    lines += ["}  // namespace bsc", "}  // namespace aesgb", ""]
    return "\n".join(lines)


def _search_one(p):
    circ, _, _ = build_all((p, p), restarts=4)
    e = len(circ["sbox_enc"].gates)
    dcost = len(circ["sbox_core_dec"].gates) * 4 + len(circ["inv_mix_out"].gates)
    return p, e, dcost


def search():
    """Cost of every tower, on all host cores: the encryption S-box's gates,
    and a decryption column's (four inverse S-box cores and the InvMixColumns
    output circuit)."""
    import multiprocessing
    params = [(mod, lam, bi, side)
              for mod in QUARTICS for lam in range(1, 16) if g16_trace(lam, mod) == 1
              for bi in range(Tower(mod, lam, 0).nroots) for side in (0, 1)]
    results = {"enc": [], "dec": []}
    with multiprocessing.Pool() as pool:
        for n, (p, e, dcost) in enumerate(pool.imap_unordered(_search_one, params), 1):
            print(f"[{n}/{len(params)}] tower {p}: encryption S-box {e}, decryption column {dcost}", flush=True)
            results["enc"].append((e, p))
            results["dec"].append((dcost, p))
    for k in results:
        results[k].sort()
        print(k, results[k][:8])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--check", action="store_true")
    ap.add_argument("--search", action="store_true")
    args = ap.parse_args()
    if args.search:
        search()
        return 0
    circuits, towers, outs = build_all(DEFAULT)
    verify(circuits, outs)
    text = emit(circuits, towers, DEFAULT, outs)
    if args.check:
        with open(OUT_PATH) as f:
            if f.read() != text:
                print("bitslice_circuits.h is stale", file=sys.stderr)
                return 1
        return 0
    with open(OUT_PATH, "w") as f:
        f.write(text)
    for name, C in circuits.items():
        print(f"{name}: {len(C.gates)} gates")
    return 0


if __name__ == "__main__":
    sys.exit(main())
