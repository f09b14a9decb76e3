"""Pins of the oracle's FP32-only ranking (oracle_fp32_rows, fp32_mismatch).

The join filters candidates with a single-precision squared distance and
ranks them in canonical FP64 (Sec. 4 kernel; Sec. 2.1 defines the result).
The diagnostic asks what ranking by the FP32 value alone would return.  Its
oracle is pinned here against:

* an exact-rational emulation of single-precision arithmetic (fractions;
  round to nearest, ties to even, subnormals included), written apart from
  the oracle's C, on tiny random and near-tie inputs;
* a hand-worked case where two exact distances round to the same FP32 value
  and the index tie-break then reverses their exact order;
* integer inputs, where every FP32 step is exact and the FP32-only rows are
  the exact rows (no mismatch).
"""
from fractions import Fraction

import numpy as np
import pytest

import knn_inputs as gen
import oracle


def round_f32(x: Fraction) -> Fraction:
    """Nearest single-precision value to x (ties to even), as a fraction."""
    if x == 0:
        return Fraction(0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)                       # below 2^-126: subnormal spacing
    ulp = Fraction(2) ** (e - 23)
    q = a / ulp
    lo = q.numerator // q.denominator
    rem = q - lo
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and lo % 2 == 1):
        lo += 1
    return sign * lo * ulp


def filter_d2_emulated(a, b):
    """The filter's FP32 squared distance, step by step in exact rationals:
    one rounding per subtraction, per fused multiply-add and per final
    addition of the two accumulators (d >= 4)."""
    d = len(a)
    t = [round_f32(Fraction(float(a[k])) - Fraction(float(b[k]))) for k in range(d)]
    if d < 4:
        s = Fraction(0)
        for k in range(d):
            s = round_f32(t[k] * t[k] + s)
        return s
    e = o = Fraction(0)
    for k in range(d):
        if k & 1:
            o = round_f32(t[k] * t[k] + o)
        else:
            e = round_f32(t[k] * t[k] + e)
    return round_f32(e + o)


def fp32_rows_emulated(points, K):
    n = len(points)
    out = np.empty((n, K), np.int32)
    for i in range(n):
        keys = sorted((filter_d2_emulated(points[i], points[j]), j) for j in range(n) if j != i)
        out[i] = [j for _, j in keys[:K]]
    return out


def test_round_f32_matches_numpy_on_doubles():
    # the emulation's rounding agrees with the platform's double -> float cast
    u = gen.uniform_f64(gen.stream_key(0, "round_f32"), 800).reshape(2, 400)
    mags = u[0] * 10.0 ** (-44.0 + 80.0 * u[1])      # 1e-44 .. 1e36, subnormals included
    vals = np.concatenate([mags, -mags, [1 + 2 ** -24, 1 + 3 * 2 ** -24, 2 ** -149 * 1.5,
                                         2 ** -140 + 2 ** -170]])
    for v in vals:
        assert float(round_f32(Fraction(float(v)))) == float(np.float32(v))


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6])
def test_fp32_rows_match_exact_rational_emulation(d):
    n, K = 28, 9
    p = gen.make_points("uniform", n, d, seed=70 + d)
    # near ties: copies of a few points moved by one FP32 ulp in one coordinate
    q = p.copy()
    q[: n // 2] = p[: n // 2][::-1]
    q[n // 2:, 0] = np.nextafter(q[n // 2:, 0], np.float32(2.0))
    pts = np.concatenate([p, q[: n // 2]]).astype(np.float32)
    want = fp32_rows_emulated(pts, K)
    got = oracle.fp32_rows(pts, K, np.arange(len(pts)))
    np.testing.assert_array_equal(got, want)


def test_fp32_rows_on_colliding_distances():
    # distances across columns differ only below single precision
    pts = gen.points_columns(6, 6, gen.stream_key(0, "columns_tiny"))
    want = fp32_rows_emulated(pts, 12)
    got = oracle.fp32_rows(pts, 12, np.arange(len(pts)))
    np.testing.assert_array_equal(got, want)
    ids, _ = oracle.bf(pts, 12)
    assert (got != ids).any()  # the case does reorder


def test_hand_worked_reversal():
    # query (0,0); B = (1, 2^-6 + 2^-29) has id 1, A = (1, 2^-6) has id 2.
    # Exact: D_A = 1 + 2^-12 < D_B = 1 + 2^-12 + 2^-34 (+ 2^-58 lost in FP64),
    # so the exact row is [A, B].  FP32: fma(h, h, 1) rounds 1 + 2^-12 + 2^-34
    # to 1 + 2^-12 (ulp 2^-23), both keys equal, the index puts B first.
    pts = np.array([[0.0, 0.0], [1.0, 2.0 ** -6 + 2.0 ** -29], [1.0, 2.0 ** -6], [5.0, 5.0]], np.float32)
    ids, dist = oracle.bf(pts, 2)
    assert list(ids[0]) == [2, 1] and dist[0, 0] < dist[0, 1]
    assert list(oracle.fp32_rows(pts, 2, [0])[0]) == [1, 2]
    assert oracle.fp32_mismatch(pts, ids, [0]) == (1, 2, 0)
    ids1, _ = oracle.bf(pts, 1)
    assert oracle.fp32_mismatch(pts, ids1, [0]) == (1, 1, 1)


@pytest.mark.parametrize("d", [2, 3, 6])
def test_integer_inputs_have_no_mismatch(d):
    # coordinates below 30: differences, squares and sums are exact in FP32
    m = {2: 30, 3: 10, 6: 3}[d]
    pts = gen.points_lattice(m, d)
    pts = pts[gen.permutation(len(pts), gen.stream_key(0, "lattice_fp32", d))]
    ids, _ = oracle.bf(pts, 12)
    np.testing.assert_array_equal(oracle.fp32_rows(pts, 12, np.arange(len(pts))), ids)
    assert oracle.fp32_mismatch(pts, ids, np.arange(len(pts))) == (0, 0, 0)


def fp32_pins_fail(mutant):
    """True when a pin of this file detects the planted mistake."""
    for d in (2, 4, 6):
        n, K = 28, 9
        p = gen.make_points("uniform", n, d, seed=70 + d)
        q = p.copy()
        q[:, 0] = np.nextafter(q[:, 0], np.float32(2.0))
        pts = np.concatenate([p, q[: n // 2]]).astype(np.float32)
        if not np.array_equal(oracle.fp32_rows(pts, K, np.arange(len(pts)), mutant=mutant),
                              fp32_rows_emulated(pts, K)):
            return True
    return False


@pytest.mark.parametrize("mutant", oracle.FP32_MUTANTS)
def test_fp32_pins_catch_planted_mistakes(mutant):
    assert fp32_pins_fail(mutant)
