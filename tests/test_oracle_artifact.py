"""Pins of the oracle's artifact stages (the c_i, m_i, p_i of Sec. 2.3 and
Sec. 8.5): the compute stage against exact rational arithmetic rounded to
binary32 once per fused step, and against its closed form x (1 - (127/128)^n);
the stream stage against a plain float32 loop, with the window start worked
out by integer arithmetic from the definition."""
from fractions import Fraction

import numpy as np
import pytest


def _rne_f32(q: Fraction) -> float:
    """Round a rational to the nearest binary32 (ties to even), exactly."""
    if q == 0:
        return 0.0
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)                      # subnormals share the lowest exponent
    ulp = Fraction(2) ** (e - 23)
    m = a / ulp
    f = m.numerator // m.denominator
    r = m - f
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return sign * float(f * ulp)


def _fma_chain(x: float, steps: int) -> float:
    a, b = Fraction(0), Fraction(_rne_f32(Fraction(x) / 128))
    for _ in range(steps):
        a = Fraction(_rne_f32(a * Fraction(127, 128) + b))
    return float(a)


def test_compute_synth_matches_exact_fused_steps(orc):
    g = np.random.default_rng(0)
    x = np.concatenate([g.standard_normal(6), [1.0, -3.5, 1e-30, 7e20]]).astype(np.float32)
    for steps in (0, 1, 2, 7, 40):
        got = orc.compute_synth(x[None, :], steps)[0]
        want = np.array([_fma_chain(float(v), steps) for v in x], np.float32)
        assert np.array_equal(got, want), steps


def test_compute_synth_closed_form(orc):
    g = np.random.default_rng(1)
    x = g.standard_normal((3, 64)).astype(np.float32)
    for steps in (1, 100, 1000):
        y = orc.compute_synth(x, steps).astype(np.float64)
        exact = x.astype(np.float64) * (1.0 - (127.0 / 128.0) ** steps)
        # one rounding per step, each at most 2^-24 of a value below |x|; the
        # errors decay by 127/128 per later step
        assert np.all(np.abs(y - exact) <= 2.0 ** -24 * np.abs(x) * min(steps, 128) + 1e-45)
    assert np.array_equal(orc.compute_synth(x, 1), x * np.float32(1 / 128))


def _window(x0: np.float32, W: int, R: int, L: int) -> int:
    bits = int(np.array([x0], np.float32).view(np.uint32)[0])
    h = ((bits * 0x9E3779B97F4A7C15) % (1 << 64)) >> 32
    return W * (h % (L // W - R // W + 1))


@pytest.mark.parametrize("W,R,L", [(4, 4, 64), (8, 24, 64), (16, 64, 64), (12, 36, 1200)])
def test_stream_synth_matches_float32_loop(orc, W, R, L):
    g = np.random.default_rng(W + R)
    x = g.standard_normal((5, W)).astype(np.float32)
    T = g.standard_normal(L).astype(np.float32)
    got = orc.stream_synth(x, T, R)
    for q in range(5):
        b = _window(x[q, 0], W, R, L)
        assert 0 <= b and b + R <= L
        for j in range(W):
            a = np.float32(x[q, j])
            for r in range(R // W):
                a = np.float32(a + T[b + r * W + j])
            assert got[q, j] == a


def test_stream_window_of_a_known_value(orc):
    # bits(1.0f) = 0x3F800000; 0x3F800000 * 0x9E3779B97F4A7C15 mod 2^64 =
    # 0x8312F9C735800000, whose high half 0x8312F9C7 = 2199058887 is 887 mod
    # 1000: with W = 4, R = 4, L = 4000 a row starting with 1.0 reads window 887.
    assert _window(np.float32(1.0), 4, 4, 4000) == 4 * 887
    x = np.zeros((1, 4), np.float32)
    x[0, 0] = 1.0
    T = np.zeros(4000, np.float32)
    T[4 * 887: 4 * 887 + 4] = [10.0, 20.0, 30.0, 40.0]
    assert np.array_equal(orc.stream_synth(x, T, 4)[0], np.array([11.0, 20.0, 30.0, 40.0], np.float32))


def test_artifact_pipeline_topk(orc):
    g = np.random.default_rng(3)
    x = g.standard_normal((4, 32)).astype(np.float32)
    T = g.standard_normal(32 * 10).astype(np.float32)
    z, idx, val = orc.pipeline_artifact(x, [("c", 5), ("m", T, 64)], top_k=3)
    ref = orc.stream_synth(orc.compute_synth(x, 5), T, 64)
    assert np.array_equal(z, ref)
    order = np.argsort(-ref.astype(np.float64), axis=1, kind="stable")[:, :3]
    assert np.array_equal(idx, order)
