"""Pins of the oracle's FP8 arm (OCP FP8 E4M3 codes, per-tensor scaling, scaled
dense layers, the emulated FP8 pipeline): the format's defining constants, an
independent library decoder (torch.float8_e4m3fn), exact small cases against
numpy, and closeness of the emulated FP8 pipeline to the FP64 pipeline."""
import numpy as np
import pytest
import torch

import synth


def test_e4m3_decode_constants(orc):
    c = np.array([0x00, 0x01, 0x07, 0x08, 0x38, 0x3C, 0x40, 0x7E, 0x7F, 0x80, 0xFE], np.uint8)
    v = orc.e4m3_decode(c)
    want = [0.0, 2.0 ** -9, 7 * 2.0 ** -9, 2.0 ** -6, 1.0, 1.5, 2.0, 448.0, np.nan, -0.0, -448.0]
    for a, b in zip(v, want):
        assert (np.isnan(a) and np.isnan(b)) or a == b


def test_e4m3_decode_matches_torch_and_rounding(orc):
    codes = np.arange(256, dtype=np.uint8)
    v = orc.e4m3_decode(codes)
    t = torch.from_numpy(codes).view(torch.float8_e4m3fn).float().double().numpy()
    fin = ~np.isnan(v)
    assert np.array_equal(np.isnan(t), ~fin)
    assert np.array_equal(v[fin], t[fin])
    # every finite code value is a fixed point of the oracle's rounding, and the
    # positive codes are strictly increasing
    assert np.array_equal(orc.round_e4m3(v[fin]), v[fin])
    assert np.all(np.diff(v[1:127]) > 0)


def test_quantize_scale_and_extremes(orc):
    g = np.random.default_rng(0)
    w = g.standard_normal(5000).astype(np.float32).astype(np.float64)
    s, q = orc.quantize_e4m3(w)
    assert s == float(np.float32(np.abs(w).max() / 448.0))
    i = np.argmax(np.abs(w))
    assert abs(q[i]) == 448.0
    assert np.all(np.abs(q) <= 448.0)
    # agrees with torch's cast of the same binary32 quotient (all within range)
    t = torch.from_numpy((w / s).astype(np.float32)).to(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(q, t)


def test_quantize_exact_on_grid(orc):
    # a tensor already on the e4m3 grid, scaled by 2^-5, whose largest value is
    # 448: scale 2^-5 exactly and every code reproduces the tensor
    codes = np.arange(1, 127, dtype=np.uint8)
    grid = orc.e4m3_decode(codes)
    w = np.concatenate([grid, -grid]) * 2.0 ** -5
    s, q = orc.quantize_e4m3(w)
    assert s == 2.0 ** -5
    assert np.array_equal(q * s, w)


def test_linear_fp8_exact_small_case(orc):
    g = np.random.default_rng(1)
    xq = g.integers(-8, 9, (3, 16)).astype(np.float64)
    wq = g.integers(-8, 9, (5, 16)).astype(np.float64)
    y, yq, a = orc.linear_fp8(xq, wq, 0.25, orc.ACT_RELU, s_out=0.5)
    ref = np.maximum(xq @ wq.T * 0.25, 0.0)
    assert np.array_equal(y, ref)
    assert np.array_equal(a, np.abs(xq) @ np.abs(wq).T * 0.25)
    assert np.array_equal(yq, orc.round_e4m3(ref / 0.5))


def calib_scales(orc, ws, x_calib):
    """Static activation scales: max |input of layer l| / 448 over the FP64
    activations of calibration queries (layers 1 and 2)."""
    y = orc.normalize_u8(x_calib.reshape(x_calib.shape[0], -1))
    h1 = orc.linear(y, ws[0], orc.ACT_RELU)
    h2 = orc.linear(h1, ws[1], orc.ACT_RELU)
    return [float(np.abs(h1).max() / 448.0), float(np.abs(h2).max() / 448.0)]


@pytest.mark.slow
def test_fp8_pipeline_close_to_fp64(orc):
    x, ws = synth.cfg1_inputs(0, n_queries=48)
    xc = synth.images_u8(0, 64, 64, 64, 3, tag="cfg5.calibration")
    sc = calib_scales(orc, ws, xc)
    z8, i8, hidden, sws = orc.pipeline_fp8(x, ws, sc)
    z, i = orc.pipeline_mlp(x, ws)
    assert len(hidden) == 2 and len(sws) == 3
    rel = np.abs(z8 - z).max() / np.abs(z).max()
    assert rel < 0.15, rel
    assert np.mean(i8 == i) >= 0.75
