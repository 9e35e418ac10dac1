"""The FP32 form of the K-nearest distance rounding, restated step by step in
numpy float32 (round-to-nearest per operation, the fused multiply-add by
exact rational arithmetic), against the FP32 rounding of the canonical FP64
value: the two agree on every pair, including pairs whose squared distance
falls exactly on an FP32 rounding midpoint (where the FP32 form defers to
FP64).  This checks the error-free-transform argument of canon_d2_f32 on the
CPU; the GPU tests compare the kernel's output with the oracle."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def rn32(x: Fraction) -> np.float32:
    """Round a rational to the nearest float32 (ties to even), normal range."""
    if x == 0:
        return f32(0.0)
    sign = -1 if x < 0 else 1
    x = abs(x)
    e = x.numerator.bit_length() - x.denominator.bit_length()
    while Fraction(2) ** e > x:
        e -= 1
    while Fraction(2) ** (e + 1) <= x:
        e += 1
    e = max(e, -126)
    q = x / Fraction(2) ** (e - 23)
    n = q.numerator // q.denominator
    r = q - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return f32(sign * float(Fraction(n) * Fraction(2) ** (e - 23)))


def fma(a, b, c):
    return rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def gap_sq(a, b, L, cyclic):
    s, t = two_sum(b, f32(-a))
    h, l = abs(s), (f32(-t) if s < 0 else t)
    if cyclic:
        if not h <= L:
            return False, f32(0), f32(0)
        u, v = two_sum(L, f32(-h))
        wh, wl = fast_two_sum(u, f32(v - l))
        if wh < h or (wh == h and wl < l):
            h, l = wh, wl
    sh = f32(h * h)
    e = fma(h, h, f32(-sh))
    e = fma(f32(2) * h, l, e)
    return True, sh, fma(l, l, e)


def fp32_form(q, p, L, cyc):
    """None where the FP32 form hands over to FP64."""
    if all(q[i] == p[i] for i in range(3)):
        return f32(0)
    ok, parts = True, []
    for i in range(3):
        o, sh, sl = gap_sq(q[i], p[i], L[i], cyc[i])
        ok &= o
        parts.append((sh, sl))
    (xh, xl), (yh, yl), (zh, zl) = parts
    s, e = two_sum(xh, yh)
    H, lo = fast_two_sum(s, f32(e + f32(xl + yl)))
    s, e = two_sum(H, zh)
    H, lo = fast_two_sum(s, f32(e + f32(lo + zl)))
    if ok and f32(2.0 ** -70) <= H <= f32(2.0 ** 120):
        hb = np.array([H], f32).view(np.uint32)[0]
        nb = np.array([hb + 1 if lo >= 0 else hb - 1], np.uint32).view(f32)[0]
        m = f32(0.5) * abs(f32(nb - H))
        if f32(m - abs(lo)) > H * f32(2.0 ** -40):
            return H
    return None


def canonical(q, p, L, cyc):
    """The canonical FP64 predicate value: per-axis gap, cyclic min, RN, no FMA."""
    acc = np.float64(0)
    for a, b, LL, c in zip(q, p, L, cyc):
        d = abs(np.float64(b) - np.float64(a))
        if c:
            w = np.float64(LL) - d
            d = w if w < d else d
        acc = acc + d * d
    return acc


def pairs(rng, kind, n):
    L = np.array([1.0, 0.5, 0.25], f32)
    for _ in range(n):
        cyc = [bool(x) for x in rng.integers(0, 2, 3)]
        q = (rng.random(3) * L).astype(f32)
        if kind == "near":
            p = (q + (rng.standard_normal(3) * 1e-3).astype(f32)).astype(f32)
        elif kind == "half_box":   # cyclic gaps next to L / 2
            p = np.mod(q + L * f32(0.5) + (rng.standard_normal(3) * 1e-6).astype(f32), L).astype(f32)
        elif kind == "coarse":     # coordinates on a 2^-16 grid: many exact midpoints
            q = (rng.integers(0, 1 << 16, 3) / float(1 << 16) * L).astype(f32)
            p = np.mod(q + rng.integers(-4000, 4000, 3) / float(1 << 16) * L, L).astype(f32)
        else:                      # one tiny coordinate next to ordinary ones
            p = (rng.random(3) * L).astype(f32)
            q[0] = f32(1e-20 * rng.random())
        yield [f32(x) for x in q], [f32(x) for x in p], [f32(x) for x in L], cyc


@pytest.mark.parametrize("kind", ["near", "half_box", "coarse", "mixed_scale"])
def test_fp32_form_equals_rounded_canonical(kind):
    rng = np.random.default_rng({"near": 1, "half_box": 2, "coarse": 3, "mixed_scale": 4}[kind])
    handed_over = 0
    for q, p, L, cyc in pairs(rng, kind, 1500):
        want = f32(canonical(q, p, L, cyc))
        got = fp32_form(q, p, L, cyc)
        if got is None:
            handed_over += 1
            continue
        assert got == want, (q, p, cyc, got, want)
    if kind == "coarse":
        assert handed_over > 20   # exact midpoints do occur and are handed over
    else:
        assert handed_over < 30
