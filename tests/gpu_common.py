"""Shared inputs and tolerance helpers of the GPU parity tests."""
import functools

import numpy as np

import synth

FP32_REL = 1e-5   # |y_gpu - y_fp64| <= FP32_REL * sum_k |w_jk x_k| per element


@functools.lru_cache(maxsize=None)
def cfg1_data(n: int = 256, seed: int = 0):
    x, ws = synth.cfg1_inputs(seed, n_queries=n)
    return x, ws


@functools.lru_cache(maxsize=None)
def cfg1_oracle(n: int = 256, seed: int = 0):
    import oracle
    x, ws = cfg1_data(n, seed)
    logits, idx = oracle.pipeline_mlp(x, ws)
    return logits, idx


def chain_bound(orc, x_u8, ws, acts):
    """Per-element bound on |gpu - fp64| for a dense chain run in FP32: each
    layer adds FP32_REL * sum|w x| and passes on |W| times the incoming bound
    (ReLU is 1-Lipschitz).  Also returns the FP64 logits."""
    y = orc.normalize_u8(x_u8.reshape(x_u8.shape[0], -1))
    e = np.zeros_like(y)
    for w, act in zip(ws, acts):
        w = np.asarray(w, np.float64)
        y, a = orc.linear(y, w, act, want_absdot=True)
        e = FP32_REL * a + e @ np.abs(w).T
    return y, e


def argmax_margin_ok(z64, err):
    """Queries whose FP64 top-1 beats the runner-up by more than twice `err`
    (the per-query logit error actually observed): there the GPU's argmax must
    equal the FP64 one."""
    s = np.sort(z64, axis=1)
    return (s[:, -1] - s[:, -2]) > 2 * np.max(err, axis=1)


def first_argmax(z):
    """Index of the largest value per row, lowest index on ties."""
    return np.argmax(z, axis=1)
