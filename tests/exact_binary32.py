"""Binary32 arithmetic emulated with exact rationals (test helper, CPU only).

Each binary32 operation is its exact rational result rounded once to the
nearest binary32, ties to even (IEEE 754 round-to-nearest), so a sequence of
operations written here with ``rn32`` is what a correctly rounded binary32
machine computes, independently of any compiler or library.
"""
import math
from fractions import Fraction

import numpy as np


def rn32(x: Fraction) -> np.float32:
    """Round an exact rational to the nearest binary32, ties to even (normal range)."""
    if x == 0:
        return np.float32(0.0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    assert e >= -126, "outside the normal binary32 range"
    q = Fraction(2) ** (e - 23)          # ulp for a 24-bit significand
    m = a / q
    fl = math.floor(m)
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return np.float32(s * float(fl * q))


def F(x) -> Fraction:
    return Fraction(float(x))


def op(x: Fraction) -> Fraction:
    """One binary32 operation: the exact result rounded once."""
    return F(rn32(x))


def compensated_exact(u, rf, nt: int, T: int) -> list:
    """The binary32 compensated form of Eq. 2, every operation rounded once.

    Time is cut into blocks of T steps (the last may be shorter).  At a block's
    start each point carries h = stored value, l = 0; a step computes
      dh = (hl - 2h) + hr,  dl = (ll - 2l) + lr,  d = dh + dl,  inc = rf*d,
      (s, e) = TwoSum(h, inc) in Knuth's six operations
               s = h + inc, bb = s - h, e = (h - (s - bb)) + (inc - bb),
      h' = s,  l' = l + e;
    at the block's end the stored value is h + l.  Returns binary32 values."""
    n = len(u)
    r = F(rf)
    stored = [F(x) for x in u]
    done = 0
    while done < nt:
        steps = min(T, nt - done)
        h, l = list(stored), [Fraction(0)] * n
        for _ in range(steps):
            h2, l2 = [None] * n, [None] * n
            for i in range(n):
                im, ip = (i - 1) % n, (i + 1) % n
                dh = op(op(h[im] - op(2 * h[i])) + h[ip])
                dl = op(op(l[im] - op(2 * l[i])) + l[ip])
                inc = op(r * op(dh + dl))
                s = op(h[i] + inc)
                bb = op(s - h[i])
                e = op(op(h[i] - op(s - bb)) + op(inc - bb))
                h2[i], l2[i] = s, op(l[i] + e)
            h, l = h2, l2
        stored = [op(h[i] + l[i]) for i in range(n)]
        done += steps
    return [np.float32(float(x)) for x in stored]
