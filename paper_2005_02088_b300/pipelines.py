"""Construction helpers for the synthetic query pipelines.

They only fill the C structures of ``include/camelot.h`` and move buffers;
all computation happens in libcamelot.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import camelot as cm


def stage_normalize(H: int, W: int, Cc: int, max_batch: int) -> int:
    d = cm.StageDesc()
    d.kind = cm.STAGE_NORMALIZE_U8
    d.dims[0], d.dims[1], d.dims[2] = H, W, Cc
    d.max_batch = max_batch
    return cm.camelot_stage_prepare(d)


def stage_norm_pool2(H: int, W: int, Cc: int, max_batch: int) -> int:
    d = cm.StageDesc()
    d.kind = cm.STAGE_NORM_POOL2_BF16
    d.dims[0], d.dims[1], d.dims[2] = H, W, Cc
    d.max_batch = max_batch
    return cm.camelot_stage_prepare(d)


def stage_dense(kind: int, weights, acts, top_k: int, max_batch: int) -> int:
    """Dense chain stage from device tensors ``weights[l]`` of shape [out, in]
    (float32 for MLP_FP32, bfloat16 for GEMM_BF16)."""
    d = cm.StageDesc()
    d.kind = kind
    d.n_layers = len(weights)
    d.dims[0] = weights[0].shape[1]
    for i, w in enumerate(weights):
        assert w.is_cuda and w.is_contiguous()
        d.dims[i + 1] = w.shape[0]
        d.act[i] = acts[i]
        d.weights[i] = w.data_ptr()
    d.top_k = top_k
    d.max_batch = max_batch
    torch.cuda.synchronize()
    return cm.camelot_stage_prepare(d)


def alloc(instances, quotas, batch: int) -> cm.Alloc:
    a = cm.Alloc()
    a.n_stages = len(instances)
    for i, (n, p) in enumerate(zip(instances, quotas)):
        a.instances[i] = n
        a.sm_quota[i] = p
    a.batch = batch
    return a


def options(**kw) -> cm.Options:
    o = cm.camelot_options_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def run_all(p: int, queries: np.ndarray, stream_id: int = 0, chunk: int = 64,
            timeout_s: float = 60.0) -> list:
    """Submit every row of ``queries`` (host uint8, [n, ...]) with back-pressure
    and poll until all complete; returns the completions in query order."""
    import time
    q = np.ascontiguousarray(queries.reshape(queries.shape[0], -1))
    n = q.shape[0]
    buf = (cm.Completion * 4096)()
    out = []
    i = 0
    t_end = time.time() + timeout_s
    while len(out) < n:
        if i < n:
            m = min(chunk, n - i)
            if cm.camelot_submit(p, stream_id, q[i:i + m], m, allow_eagain=True) is not None:
                i += m
        k = cm.camelot_poll(p, buf, timeout_us=0)
        for j in range(k):
            out.append(_copy(buf[j]))
        if time.time() > t_end:
            raise TimeoutError(f"{len(out)} of {n} completions after {timeout_s}s")
    return out


def _copy(c: cm.Completion) -> cm.Completion:
    d = cm.Completion()
    C.pointer(d)[0] = c
    return d
