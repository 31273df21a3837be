"""Pins of the oracle's text-tagging pipeline (embedding gather, GEMMs
512 -> 2048 (GELU) -> 512 -> 64, per-token argmax): numpy indexing for the
gather, a closed-form case with one-hot embeddings and selector weights, token
independence, and closeness of the bf16-emulated arm to FP64."""
import numpy as np

import synth


def test_embed_gather_matches_numpy(orc):
    g = np.random.default_rng(0)
    E = g.standard_normal((50, 24))
    tok = g.integers(-3, 60, (7, 9)).astype(np.int32)     # includes padding and out-of-range IDs
    got = orc.embed_gather(tok, E)
    valid = (tok >= 0) & (tok < 50)
    ref = np.where(valid[..., None], E[np.clip(tok, 0, 49)], 0.0)
    assert np.array_equal(got, ref)


def test_text_pipeline_closed_form(orc):
    V, D, F, T = 1000, 512, 2048, 64
    E = np.zeros((V, D))
    E[np.arange(V), np.arange(V) % D] = 4.0
    w1 = np.zeros((F, D))
    w1[np.arange(D), np.arange(D)] = 2.0
    w2 = np.zeros((D, F))
    w2[np.arange(D), np.arange(D)] = 1.0
    w3 = np.zeros((T, D))
    w3[np.arange(T), np.arange(T)] = 1.0
    tok = np.random.default_rng(1).integers(-1, V, (5, 40)).astype(np.int32)
    z, tags = orc.pipeline_text(tok, E, [w1, w2, w3])
    feat = np.where(tok >= 0, tok % D, -1)
    want = np.where((feat >= 0) & (feat < T), feat, 0)
    assert np.array_equal(tags, want)
    # the winning logit is gelu(8) = 8 Phi(8)
    hit = (feat >= 0) & (feat < T)
    assert np.allclose(z.max(axis=2)[hit], orc.gelu(8.0), rtol=1e-15)


def test_tokens_are_independent(orc):
    tok, _, E, ws = synth.cfg4_inputs(0, n_queries=2)
    z, tags = orc.pipeline_text(tok[:, :32], E, ws)
    tok2 = tok[:, :32].copy()
    tok2[:, 16:] = np.random.default_rng(2).integers(-1, 32000, (2, 16))
    z2, tags2 = orc.pipeline_text(tok2, E, ws)
    assert np.array_equal(z[:, :16], z2[:, :16]) and np.array_equal(tags[:, :16], tags2[:, :16])


def test_bf16_emulation_close_to_fp64(orc):
    tok, lens, E, ws = synth.cfg4_inputs(0, n_queries=3)
    z, tags = orc.pipeline_text(tok, E, ws)
    zb, tb = orc.pipeline_text(tok, E, ws, emulate_bf16=True)
    real = np.arange(tok.shape[1])[None, :] < lens[:, None]
    assert np.abs(zb - z)[real].max() <= 3e-2 * np.abs(z)[real].max()
    assert np.mean(tb[real] == tags[real]) >= 0.9
