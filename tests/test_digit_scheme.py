"""The arithmetic of the tensor-core reduction (FP64 mode 2), checked with exact integers.

The kernel (paper_2104_01253_gb300/csrc/kc_reduce_tc.cuh) computes each dot product of a
512-row chunk as an exact integer from fixed-point digit expansions.  This test replays
those steps in Python integers with the kernel's own constants (read from the header) and
checks the claims the kernel's exactness rests on, at the range limits:
  * the offset forms of X (basis entries, |q| < 2) and Y (w, v scaled by the chunk's
    largest exponent) fit their digit counts (below 2^60);
  * every accumulator sum D_st = sum_i (A value) d_t,i stays within 2^24, where FP32
    holds integers exactly;
  * bias removal and the 1024^s 32^t combination give exactly X^T Y, which fits the
    128-bit accumulation (|X^T Y| < 2^127);
  * the FP64 result is within the error of one final rounding of the exact dot product.
It checks the scheme, not the GPU: the GPU results are compared with the oracle in
tests/test_gpu_dcgs2.py (mode 2).
"""
import math
import re
import struct
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

HDR = (Path(__file__).resolve().parents[1] / "paper_2104_01253_gb300" / "csrc" /
       "kc_reduce_tc.cuh").read_text()


def _const(name):
    m = re.search(r"constexpr int (?:\w+ = \d+, )*%s = (\d+)" % name, HDR)
    assert m, name
    return int(m.group(1))


NA, BA, NB, BB = _const("TX_NA"), _const("TX_BA"), _const("TX_NB"), _const("TX_BB")
R, QP, PB, WSHIFT = _const("TX_R"), _const("TX_QP"), _const("TX_PB"), _const("TX_WSHIFT")
OFFA = sum((1 << (BA - 1)) << (BA * s) for s in range(NA))
OFFB = sum((1 << (BB - 1)) << (BB * t) for t in range(NB))
ABIAS = (1 << BA) + (1 << (BA - 1))        # A value 2^BA + u_s = ABIAS + d_s


def _bits(v):
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def _expo(v):
    return (_bits(v) >> 52) & 0x7FF


def _fixed(v, P):
    """round(v 2^P), half away from zero (the kernel's branch-free conversion)."""
    b = _bits(v)
    e = (b >> 52) & 0x7FF
    mm = ((b << 11) & (2 ** 64 - 1)) | ((1 << 63) if e else 0)
    n = 1086 - P - (e if e else 1)
    a = ((mm >> (n - 1)) if n - 1 < 64 else 0)
    a = (a + 1) >> 1
    return -a if b >> 63 else a


def _chunk_dot(xcol, px, vals, py):
    X = [_fixed(t, px) for t in xcol]
    Y = [_fixed(t, py) for t in vals]
    assert all(0 <= x + OFFA < 2 ** 60 for x in X) and all(0 <= y + OFFB < 2 ** 60 for y in Y)
    ua = [[((x + OFFA) >> (BA * s)) & ((1 << BA) - 1) for s in range(NA)] for x in X]
    bd = [[(((y + OFFB) >> (BB * t)) & ((1 << BB) - 1)) - (1 << (BB - 1)) for t in range(NB)]
          for y in Y]
    bsum = [sum(row[t] for row in bd) for t in range(NB)]
    V = 0
    for s in range(NA):
        for t in range(NB):
            D = sum(((1 << BA) + ua[i][s]) * bd[i][t] for i in range(len(X)))
            assert abs(D) <= 2 ** 24                      # exact in the FP32 accumulator
            V += (D - ABIAS * bsum[t]) << (BA * s + BB * t)
    exact = sum(x * y for x, y in zip(X, Y))
    assert V == exact and abs(exact) < 2 ** 127
    return math.ldexp(float(V), -(px + py)), X, Y


def test_constants_describe_a_consistent_scheme():
    assert NA * BA >= 58 and NB * BB >= 59          # |X| < 2^57, |Y| < 2^58 plus the offset
    assert OFFA < 2 ** 60 and OFFB + 2 ** 58 <= 2 ** 60
    assert R * (2 ** (BA + 1) - 1) * (1 << (BB - 1)) <= 2 ** 24
    # a 32-row quarter of an A tile holds TX_CPQ columns of NA digit rows, below the row
    # of ones (row TX_ONES of the first quarter)
    assert _const("TX_CPQ") * NA <= _const("TX_ONES") < 32


@pytest.mark.parametrize("case", ["random", "wide_range", "q_near_2", "max_equal", "max_neg"])
def test_chunk_dot_products_are_exact(case):
    rng = np.random.default_rng(11)
    q = rng.standard_normal(R)
    q /= np.linalg.norm(q)
    w = rng.standard_normal(R) * 1e37
    v = rng.standard_normal(R) * 1e-41
    if case == "wide_range":
        w[::2] *= 1e-12
    elif case == "q_near_2":
        q[:] = np.where(q >= 0, 1.999, -1.999)
    elif case == "max_equal":
        q[:], w[:], v[:] = 1.999, 2.0 - 2 ** -52, 2.0 - 2 ** -52
    elif case == "max_neg":
        q[:], w[:], v[:] = -1.999, -(2.0 - 2 ** -52), -(2.0 - 2 ** -52)
    pw, pv = PB - max(map(_expo, w)), PB - max(map(_expo, v))
    ex = lambda a, b: sum(Fraction(x) * Fraction(y) for x, y in zip(a, b))
    for name, (xc, px, vals, py) in {"C": (q, QP, w, pw), "S": (q, QP, v, pv),
                                     "beta": (w, pw - WSHIFT, w, pw),
                                     "s": (w, pw - WSHIFT, v, pv)}.items():
        got, X, Y = _chunk_dot(xc, px, vals, py)
        ref = ex(xc, vals)
        # conversion error (half a unit of each fixed-point form) plus one final rounding
        two = Fraction(2)
        bound = (sum(abs(Fraction(a)) for a in xc) * two ** -(py + 1) +
                 sum(abs(Fraction(b)) for b in vals) * two ** -(px + 1) +
                 two ** -(px + py + 2) * len(xc) + abs(ref) * two ** -52)
        assert abs(Fraction(got) - ref) <= bound, name
