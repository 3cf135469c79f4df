"""Test helpers: golden-file parsing and exact fp32 arithmetic on rationals.

The exact-rational helpers are an independent restatement used to pin the
oracle's fp32 warp coordinate sequence; they share nothing with the oracle's C.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_hand_cases(name: str = "hand_cases.txt") -> list:
    """Parse the hand-worked case file into dicts."""
    cases = []
    cur = None
    lines = [ln.strip() for ln in open(os.path.join(GOLDEN, name))]
    i = 0

    def read_block(i, h, w, c):
        rows = []
        for _ in range(h):
            vals = [int(v) for v in lines[i].split()]
            assert len(vals) == w * c, (lines[i], w, c)
            rows.append(vals)
            i += 1
        return np.array(rows, dtype=np.uint8).reshape(h, w, c), i

    while i < len(lines):
        ln = lines[i]
        i += 1
        if not ln or ln.startswith("#"):
            continue
        key, _, rest = ln.partition(" ")
        if key == "case":
            cur = {"name": rest}
        elif key == "cite":
            cur["cite"] = rest
        elif key == "op":
            cur["op"] = rest
        elif key == "in":
            h, w, c = (int(v) for v in rest.split())
            cur["in"], i = read_block(i, h, w, c)
        elif key == "out":
            h, w, c = (int(v) for v in rest.split())
            cur["out"], i = read_block(i, h, w, c)
        elif key == "M":
            cur["M"] = np.array([float(v) for v in rest.split()], dtype=np.float32).reshape(2, 3)
        elif key == "end":
            assert "cite" in cur, cur["name"]
            cases.append(cur)
            cur = None
    return cases


# ---------------------------------------------------------------------------
# Exact binary32 rounding of a rational (round to nearest, ties to even).
# ---------------------------------------------------------------------------
def round_f32(q) -> Fraction:
    q = Fraction(q)
    if q == 0:
        return Fraction(0)
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    # normalise e so that 2^e <= a < 2^(e+1)
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)                       # subnormals share the minimum exponent
    ulp = Fraction(2) ** (e - 23)
    m = a / ulp
    n = math.floor(m)
    r = m - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    out = sign * n * ulp
    if abs(out) > Fraction(2) ** 127 * (2 - Fraction(2) ** -23):
        raise OverflowError("binary32 overflow")
    return out


def fmaf_exact(a, b, c) -> Fraction:
    """fmaf(a, b, c) for binary32 a, b, c: one rounding of the exact a*b + c."""
    return round_f32(Fraction(a) * Fraction(b) + Fraction(c))


def sub_f32(a, b) -> Fraction:
    return round_f32(Fraction(a) - Fraction(b))


def f32(x) -> Fraction:
    """The exact value of a binary32 number given as a Python/numpy float."""
    v = np.float32(x)
    return Fraction(float(v))
