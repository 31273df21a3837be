"""Pins of the oracle's stage math against facts outside the oracle itself:
closed forms and special values, the number-format definitions (golden
fixtures), library routines (numpy / scipy / torch) and brute force."""
import os

import numpy as np
import pytest
import torch
from scipy.special import erf

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            out.append(line.split()[:2])
    return out


# --- normalisation ---------------------------------------------------------
def test_normalize_special_values(orc):
    x = np.array([0, 127, 128, 255], np.uint8)
    y = orc.normalize_u8(x)
    assert y.tolist() == [-1.9921875, -0.0078125, 0.0078125, 1.9921875]


def test_normalize_all_bytes_exact_grid(orc):
    x = np.arange(256, dtype=np.uint8)
    y = orc.normalize_u8(x)
    # y * 128 is the odd integer 2x - 255: every value is exact in float32
    assert np.array_equal(y * 128.0, 2.0 * np.arange(256) - 255.0)
    assert np.array_equal(y.astype(np.float32).astype(np.float64), y)
    assert np.array_equal(y[::-1], -y)            # symmetric about 127.5
    assert np.all(np.diff(y) == 1.0 / 64.0)       # uniform step


def test_norm_pool2_matches_reshape_mean(orc):
    x = synth.images_u8(3, 2, 6, 8, 3)
    y = orc.norm_pool2(x)
    ref = x.astype(np.float64).reshape(2, 3, 2, 4, 2, 3).mean(axis=(2, 4))
    ref = (ref - 127.5) / 64.0
    assert np.array_equal(y, ref.reshape(2, -1))


def test_norm_pool2_constant_and_single_pixel(orc):
    x = np.full((1, 4, 4, 3), 200, np.uint8)
    assert np.all(orc.norm_pool2(x) == (200 - 127.5) / 64)
    x = np.zeros((1, 2, 2, 3), np.uint8)
    x[0, 1, 1, 2] = 4                            # block mean 1 in channel 2 only
    assert orc.norm_pool2(x).tolist() == [[-127.5 / 64, -127.5 / 64, -126.5 / 64]]


def test_norm_pool2_exact_in_float32(orc):
    x = synth.images_u8(1, 3, 8, 8, 3)
    y = orc.norm_pool2(x)
    assert np.array_equal(y.astype(np.float32).astype(np.float64), y)


# --- dense layers ------------------------------------------------------------
@pytest.mark.parametrize("act", [0, 1, 2])
def test_linear_matches_numpy(orc, act):
    g = np.random.default_rng(1)
    x = g.standard_normal((5, 37))
    w = g.standard_normal((11, 37))
    y, a = orc.linear(x, w, act, want_absdot=True)
    pre = x @ w.T
    ref = {0: pre, 1: np.maximum(pre, 0), 2: 0.5 * pre * (1 + erf(pre / np.sqrt(2)))}[act]
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a, np.abs(x) @ np.abs(w).T, rtol=1e-12)
    assert np.all(a + 1e-12 >= np.abs(pre))


def test_linear_identity_relu(orc):
    x = np.array([[-2.0, 0.0, 3.5]])
    assert orc.linear(x, np.eye(3), orc.ACT_RELU).tolist() == [[0.0, 0.0, 3.5]]


def test_gelu_values_and_odd_identity(orc):
    assert orc.gelu(0.0) == 0.0
    assert abs(orc.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(orc.gelu(-1.0) + 0.15865525393145707) < 1e-15
    for v in np.linspace(-6, 6, 25):
        assert abs((orc.gelu(v) - orc.gelu(-v)) - v) < 1e-14   # gelu(x) - gelu(-x) = x
    assert abs(orc.gelu(10.0) - 10.0) < 1e-12 and abs(orc.gelu(-10.0)) < 1e-12


# --- argmax / top-k ----------------------------------------------------------
def test_argmax_lowest_index_on_ties(orc):
    z = np.array([[1, 3, 3, 0], [5, 5, 5, 5], [-1, -2, -0.5, -0.5]], np.float64)
    assert orc.argmax(z).tolist() == [1, 0, 2]
    g = np.random.default_rng(2)
    z = g.integers(0, 4, size=(200, 10)).astype(np.float64)   # many ties
    assert np.array_equal(orc.argmax(z), np.argmax(z, axis=1))  # numpy: first maximum


def test_topk_brute_force(orc):
    g = np.random.default_rng(3)
    z = g.integers(0, 6, size=(50, 30)).astype(np.float64)
    idx, val = orc.topk(z, 5)
    for q in range(z.shape[0]):
        order = sorted(range(30), key=lambda j: (-z[q, j], j))[:5]
        assert idx[q].tolist() == order
        assert val[q].tolist() == [z[q, j] for j in order]


# --- number formats -------------------------------------------------------------
def test_bf16_golden(orc):
    for f32hex, bhex in _rows("bf16_rne.txt"):
        v = np.frombuffer(bytes.fromhex(f32hex)[::-1], np.float32).astype(np.float64)
        assert orc.bf16_bits(v)[0] == int(bhex, 16), f32hex


def test_bf16_matches_torch(orc):
    g = np.random.default_rng(4)
    v = np.concatenate([g.standard_normal(20000) * 10 ** g.uniform(-30, 30, 20000),
                        g.standard_normal(1000)]).astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(v).to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(orc.round_bf16(v), ref)


def test_e4m3_golden(orc):
    for a, b in _rows("e4m3_rne.txt"):
        r = orc.round_e4m3(np.array([float(a)]))[0]
        assert r == float(b) and np.signbit(r) == np.signbit(float(b)), (a, b, r)


def test_e4m3_matches_torch_in_range(orc):
    g = np.random.default_rng(5)
    v = (g.standard_normal(50000) * 10 ** g.uniform(-4, 2.3, 50000))
    v = v[np.abs(v) < 440].astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(v).to(torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(orc.round_e4m3(v), ref)


def test_round_f32_is_nearest(orc):
    v = np.array([1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, 0.1])
    assert orc.round_f32(v).tolist() == [1.0, 1 + 2.0 ** -22, float(np.float32(0.1))]


# --- whole pipelines vs a numpy composition ------------------------------------------
def test_pipeline_mlp_matches_numpy(orc):
    g = np.random.default_rng(6)
    x = g.integers(0, 256, size=(7, 4, 4, 3), dtype=np.uint8)
    ws = [g.standard_normal((16, 48)), g.standard_normal((8, 16)), g.standard_normal((5, 8))]
    logits, idx = orc.pipeline_mlp(x, ws)
    y = (x.reshape(7, -1).astype(np.float64) - 127.5) / 64
    h = np.maximum(y @ ws[0].T, 0)
    h = np.maximum(h @ ws[1].T, 0)
    z = h @ ws[2].T
    np.testing.assert_allclose(logits, z, rtol=1e-12, atol=1e-12)
    assert np.array_equal(idx, np.argmax(z, axis=1))


@pytest.mark.parametrize("emulate", [False, True])
def test_pipeline_gemm3_matches_composition(orc, emulate):
    g = np.random.default_rng(7)
    x = g.integers(0, 256, size=(4, 8, 8, 3), dtype=np.uint8)
    ws = [g.standard_normal((32, 48)) / 7, g.standard_normal((24, 32)) / 6,
          g.standard_normal((20, 24)) / 5]
    logits, idx = orc.pipeline_gemm3(x, ws, top_k=5, emulate_bf16=emulate)

    def rb(a):  # bfloat16 rounding through torch (library route)
        return torch.from_numpy(np.asarray(a, np.float64)).float().bfloat16().double().numpy()

    def gl(a):
        return 0.5 * a * (1 + erf(a / np.sqrt(2)))

    y = x.astype(np.float64).reshape(4, 4, 2, 4, 2, 3).mean(axis=(2, 4)).reshape(4, -1)
    y = (y - 127.5) / 64
    wa, wb, wc = ws
    if emulate:
        y, wa, wb, wc = rb(y), rb(wa), rb(wb), rb(wc)
    h = gl(y @ wa.T)
    if emulate:
        h = rb(h)
    h = gl(h @ wb.T)
    if emulate:
        h = rb(h)
    z = h @ wc.T
    np.testing.assert_allclose(logits, z, rtol=1e-10, atol=1e-12)
    ref = np.array([sorted(range(20), key=lambda j: (-z[q, j], j))[:5] for q in range(4)])
    assert np.array_equal(idx, ref)
