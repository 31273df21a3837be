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


def stage_compute_synth(W: int, steps: int, top_k: int, max_batch: int) -> int:
    """Artifact compute-intensive stage (c_i): `steps` FMA steps per value."""
    d = cm.StageDesc()
    d.kind = cm.STAGE_COMPUTE_SYNTH
    d.dims[0], d.dims[1] = W, steps
    d.top_k = top_k
    d.max_batch = max_batch
    return cm.camelot_stage_prepare(d)


def stage_stream_synth(W: int, R: int, table, top_k: int, max_batch: int) -> int:
    """Artifact memory- or host-link-intensive stage (m_i / p_i): R table
    floats per query from `table` (a device tensor, or pinned host memory
    mapped into the device: pass its data pointer)."""
    d = cm.StageDesc()
    d.kind = cm.STAGE_STREAM_SYNTH
    L = table.numel() if hasattr(table, "numel") else int(table[1])
    ptr = table.data_ptr() if hasattr(table, "data_ptr") else int(table[0])
    d.dims[0], d.dims[1], d.dims[2] = W, R, L
    d.weights[0] = ptr
    d.top_k = top_k
    d.max_batch = max_batch
    return cm.camelot_stage_prepare(d)


def stage_norm_pool2(H: int, W: int, Cc: int, max_batch: int) -> int:
    d = cm.StageDesc()
    d.kind = cm.STAGE_NORM_POOL2_BF16
    d.dims[0], d.dims[1], d.dims[2] = H, W, Cc
    d.max_batch = max_batch
    return cm.camelot_stage_prepare(d)


def stage_dense(kind: int, weights, acts, top_k: int, max_batch: int, ring_slots: int = 0) -> int:
    """Dense chain stage from device tensors ``weights[l]`` of shape [out, in]
    (float32 for MLP_FP32, bfloat16 for GEMM_BF16); ``ring_slots`` caps the
    bulk-copy ring of a tensor-core stage (0 = all that fit)."""
    d = cm.StageDesc()
    d.kind = kind
    d.ring_slots = ring_slots
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


def stage_normalize_e4m3(H: int, W: int, Cc: int, max_batch: int) -> int:
    d = cm.StageDesc()
    d.kind = cm.STAGE_NORMALIZE_U8_E4M3
    d.dims[0], d.dims[1], d.dims[2] = H, W, Cc
    d.max_batch = max_batch
    return cm.camelot_stage_prepare(d)


def stage_fp8(weights, acts, scales, top_k: int, max_batch: int) -> int:
    """GEMM_FP8 chain from f32 device tensors ``weights[l]`` [out, in] (quantised
    to e4m3 by the library); ``scales[l]`` is layer l's input scale and, for an
    intermediate stage, ``scales[n_layers]`` its output scale."""
    d = cm.StageDesc()
    d.kind = cm.STAGE_GEMM_FP8
    d.n_layers = len(weights)
    d.dims[0] = weights[0].shape[1]
    for i, w in enumerate(weights):
        assert w.is_cuda and w.is_contiguous() and w.dtype == torch.float32
        d.dims[i + 1] = w.shape[0]
        d.act[i] = acts[i]
        d.weights[i] = w.data_ptr()
    for i, sc in enumerate(scales):
        d.scales[i] = float(sc)
    d.top_k = top_k
    d.max_batch = max_batch
    torch.cuda.synchronize()
    return cm.camelot_stage_prepare(d)


def calibrate_fp8_scales(weights, images_u8: np.ndarray, n_ctas: int = 16) -> list:
    """Static activation scales of the FP8 arm for a ReLU MLP behind the u8
    normalisation: max |input of layer l| / 448 (l >= 1) over calibration images,
    with the activations computed by the library's FP32 stages, one layer at a
    time, and each scale by camelot_fp8_scale.  Returns [s_1, ..., s_{L-1}]."""
    n = images_u8.shape[0]
    H, W, Cc = images_u8.shape[1:4]
    x = torch.from_numpy(np.ascontiguousarray(images_u8.reshape(n, -1))).cuda()
    s0 = stage_normalize(H, W, Cc, n)
    stages = [s0]
    try:
        y = torch.empty((n, H * W * Cc), dtype=torch.float32, device="cuda")
        _run_stage(s0, x, n, y, n_ctas)
        scales = []
        for w in weights[:-1]:
            st = stage_dense(cm.STAGE_MLP_FP32, [w], [cm.ACT_RELU], top_k=0, max_batch=n)
            stages.append(st)
            h = torch.empty((n, w.shape[0]), dtype=torch.float32, device="cuda")
            _run_stage(st, y, n, h, n_ctas)
            scales.append(cm.camelot_fp8_scale(h, h.numel()))
            y = h
        return scales
    finally:
        for st in stages:
            cm.camelot_stage_release(st)


def _run_stage(st: int, inp, n: int, out, n_ctas: int) -> None:
    _, _, sb = cm.camelot_stage_info(st, n)
    scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
    cm.camelot_stage_launch(st, n_ctas, inp, n, out, None, None, None, scr, sb, None)
    torch.cuda.synchronize()


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
