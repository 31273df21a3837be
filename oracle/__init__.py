"""CPU oracle of the Camelot query pipeline -- TEST INFRASTRUCTURE ONLY.

A plain FP64 C++ restatement of what the pipeline computes (``camelot_oracle.cpp``)
wrapped with ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product library
(``paper_2005_02088_b300``) never does, and the two share no code.

Every function carries the paper passage it restates in the C++ source.  The
pins that tie it to something other than itself live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "camelot_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ACT_NONE, ACT_RELU, ACT_GELU = 0, 1, 2
POLICY_MAX_PEAK, POLICY_MIN_SM = 0, 1


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with g++ (OpenMP) if it is missing or stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC",
                    "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
        return _lib


P = C.c_void_p
I64 = C.c_int64


def _declare(L):
    sig = {
        "orc_normalize_u8": (None, [P, I64, P]),
        "orc_norm_pool2": (None, [P, I64, C.c_int, C.c_int, C.c_int, P]),
        "orc_gelu": (C.c_double, [C.c_double]),
        "orc_compute_synth": (None, [P, I64, C.c_int, P]),
        "orc_stream_synth": (None, [P, I64, C.c_int, P, I64, C.c_int, P]),
        "orc_linear": (None, [P, I64, C.c_int, P, C.c_int, C.c_int, P, P]),
        "orc_argmax": (None, [P, I64, C.c_int, P]),
        "orc_topk": (None, [P, I64, C.c_int, C.c_int, P, P]),
        "orc_round_f32": (None, [P, I64, P]),
        "orc_round_bf16": (None, [P, I64, P]),
        "orc_bf16_bits": (None, [P, I64, P]),
        "orc_round_e4m3": (None, [P, I64, P]),
        "orc_e4m3_decode": (None, [P, I64, P]),
        "orc_embed_gather": (None, [P, I64, P, C.c_int, C.c_int, P]),
        "orc_quantize_e4m3": (C.c_double, [P, I64, P]),
        "orc_linear_fp8": (None, [P, I64, C.c_int, P, C.c_int, C.c_double, C.c_int, C.c_double, P, P, P]),
        "orc_pipeline_mlp": (None, [P, I64, P, P, P, P, P, P, C.c_int]),
        "orc_pipeline_gemm3": (None, [P, I64, C.c_int, C.c_int, P, P, P, P, C.c_int, C.c_int,
                                      P, P, C.c_int]),
        "orc_simulate": (I64, [P, I64, C.c_int, C.c_double, C.c_int, P, P, P, P, I64, P, P]),
        "orc_simulate_qos": (I64, [P, I64, C.c_int, C.c_double, C.c_double, P, C.c_int, P, P, P, P, I64,
                                   P, P, P]),
        "orc_allocate_exhaustive": (C.c_int, [C.c_int] * 6 + [P] * 4 + [C.c_double] * 4
                                    + [C.c_int] + [P] * 5),
        "orc_allocate_exhaustive_hl": (C.c_int, [C.c_int] * 6 + [P] * 4 + [C.c_double] * 4
                                       + [C.c_int, P, C.c_double] + [P] * 5),
        "orc_allocate_anneal": (C.c_int, [C.c_int] * 6 + [P] * 4 + [C.c_double] * 4
                                + [C.c_int, C.c_int, C.c_double, C.c_double, C.c_uint64]
                                + [P] * 5),
        "orc_min_gpus": (C.c_double, [P, P, C.c_int, C.c_double, C.c_double]),
        "orc_pred_nparams": (I64, []),
        "orc_pred_forward": (None, [P, P, I64, P]),
        "orc_pred_grad": (C.c_double, [P, P, P, I64, P]),
        "orc_adam_step": (None, [P, P, P, P, I64, C.c_int, C.c_double, C.c_double,
                                 C.c_double, C.c_double]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# stage math
# ---------------------------------------------------------------------------
def normalize_u8(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint8)
    y = np.empty(x.shape, np.float64)
    lib().orc_normalize_u8(_p(x), x.size, _p(y))
    return y.reshape(x.shape[0], -1) if x.ndim > 1 else y


def norm_pool2(x: np.ndarray) -> np.ndarray:
    """x [n, H, W, C] u8 -> [n, H/2 * W/2 * C] float64."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    n, H, W, Cc = x.shape
    y = np.empty((n, (H // 2) * (W // 2) * Cc), np.float64)
    lib().orc_norm_pool2(_p(x), n, H, W, Cc, _p(y))
    return y


def gelu(v: float) -> float:
    return lib().orc_gelu(float(v))


def linear(x: np.ndarray, w: np.ndarray, act: int = ACT_NONE, want_absdot: bool = False):
    """y = act(x @ w.T) with x [n, K], w [N, K]; optionally sum |w x| per output."""
    x = _f64(x)
    w = _f64(w)
    n, K = x.shape
    N = w.shape[0]
    y = np.empty((n, N), np.float64)
    a = np.empty((n, N), np.float64) if want_absdot else None
    lib().orc_linear(_p(x), n, K, _p(w), N, act, _p(y), _p(a) if a is not None else None)
    return (y, a) if want_absdot else y


def argmax(z: np.ndarray) -> np.ndarray:
    z = _f64(z)
    idx = np.empty(z.shape[0], np.int32)
    lib().orc_argmax(_p(z), z.shape[0], z.shape[1], _p(idx))
    return idx


def topk(z: np.ndarray, k: int):
    z = _f64(z)
    idx = np.empty((z.shape[0], k), np.int32)
    val = np.empty((z.shape[0], k), np.float64)
    lib().orc_topk(_p(z), z.shape[0], z.shape[1], k, _p(idx), _p(val))
    return idx, val


def round_f32(v) -> np.ndarray:
    v = _f64(v)
    out = np.empty_like(v)
    lib().orc_round_f32(_p(v), v.size, _p(out))
    return out


def round_bf16(v) -> np.ndarray:
    v = _f64(v)
    out = np.empty_like(v)
    lib().orc_round_bf16(_p(v), v.size, _p(out))
    return out


def bf16_bits(v) -> np.ndarray:
    v = _f64(v)
    out = np.empty(v.shape, np.uint16)
    lib().orc_bf16_bits(_p(v), v.size, _p(out))
    return out


def round_e4m3(v) -> np.ndarray:
    v = _f64(v)
    out = np.empty_like(v)
    lib().orc_round_e4m3(_p(v), v.size, _p(out))
    return out


# ---------------------------------------------------------------------------
# whole pipelines
# ---------------------------------------------------------------------------
def e4m3_decode(codes) -> np.ndarray:
    """Values of OCP FP8 E4M3 codes (uint8 array)."""
    c = np.ascontiguousarray(codes, dtype=np.uint8)
    out = np.empty(c.shape, np.float64)
    lib().orc_e4m3_decode(_p(c), c.size, _p(out))
    return out


def quantize_e4m3(w):
    """Per-tensor FP8 quantisation: (scale s, code values of w / s)."""
    w = _f64(w)
    q = np.empty_like(w)
    s = lib().orc_quantize_e4m3(_p(w), w.size, _p(q))
    return s, q


def linear_fp8(xq, wq, vscale: float, act: int = ACT_NONE, s_out: float = 0.0):
    """FP8-arm dense layer on code values: (y, output code values or None,
    sum |wq xq| * vscale)."""
    xq, wq = _f64(xq), _f64(wq)
    nq, K = xq.shape
    N = wq.shape[0]
    y = np.empty((nq, N), np.float64)
    a = np.empty((nq, N), np.float64)
    yq = np.empty((nq, N), np.float64) if s_out > 0 else None
    lib().orc_linear_fp8(_p(xq), nq, K, _p(wq), N, float(vscale), act, float(s_out), _p(y),
                         _p(yq) if yq is not None else None, _p(a))
    return y, yq, a


def f32(v) -> float:
    return float(np.float32(v))


def pipeline_fp8(x_u8: np.ndarray, ws, act_scales):
    """The FP8 arm of the plain 2-stage pipeline, emulated on code values:
    stage 1 = e4m3(2 x - 255) (scale 1/128); each layer l of the ReLU MLP uses
    e4m3 weights with scale s_w = max|W| / 448 and input scale s_l (s_0 = 1/128,
    s_1, s_2 = act_scales); hidden outputs are re-quantised with the next
    layer's scale; the logits stay unquantised.  Returns (logits, argmax,
    [hidden code values], [s_w])."""
    x = np.ascontiguousarray(x_u8, dtype=np.uint8).reshape(x_u8.shape[0], -1).astype(np.float64)
    xq = round_e4m3((x - 127.5) * 2.0)
    scales = [f32(1.0 / 128.0)] + [f32(s) for s in act_scales]
    hidden, sws = [], []
    for l, w in enumerate(ws):
        sw, wq = quantize_e4m3(w)
        sws.append(sw)
        vscale = f32(sw * scales[l])
        last = l == len(ws) - 1
        y, yq, _ = linear_fp8(xq, wq, vscale, ACT_NONE if last else ACT_RELU,
                              0.0 if last else scales[l + 1])
        if last:
            return y, argmax(y), hidden, sws
        hidden.append(yq)
        xq = yq


def compute_synth(x, steps: int) -> np.ndarray:
    """Artifact compute stage c_i (binary32, as the stage is defined)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().orc_compute_synth(_p(x), x.size, int(steps), _p(y))
    return y


def stream_synth(x, table, R: int) -> np.ndarray:
    """Artifact memory / host-link stage m_i / p_i over `table` (binary32)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    T = np.ascontiguousarray(table, dtype=np.float32).reshape(-1)
    nq, W = x.shape
    y = np.empty_like(x)
    lib().orc_stream_synth(_p(x), nq, W, _p(T), T.size, int(R), _p(y))
    return y


def pipeline_artifact(x, stages, top_k: int):
    """A chain of artifact stages, each ("c", steps) or ("m", table, R), then
    the top-k of the last stage's rows: returns (rows, idx, val)."""
    z = np.ascontiguousarray(x, dtype=np.float32)
    for st in stages:
        z = compute_synth(z, st[1]) if st[0] == "c" else stream_synth(z, st[1], st[2])
    idx, val = topk(z.astype(np.float64), top_k)
    return z, idx, val


def embed_gather(tokens, E) -> np.ndarray:
    """Rows E[token] (zero rows for padding / out-of-range IDs); tokens [..., T]."""
    t = np.ascontiguousarray(tokens, dtype=np.int32)
    E = _f64(E)
    out = np.empty(t.shape + (E.shape[1],), np.float64)
    lib().orc_embed_gather(_p(t), t.size, _p(E), E.shape[0], E.shape[1], _p(out))
    return out


def pipeline_text(tokens, E, ws, emulate_bf16: bool = False):
    """Text-tagging pipeline on padded token queries [n, T]: e = E[tok],
    h = gelu(W1 e), g = W2 h, z = W3 g, tag = argmax of z per token.  With
    emulate_bf16 the embedding table and weights are rounded to bfloat16 and so
    are h and g (the logits stay unrounded), as the BF16 GEMM stages round.
    Returns (logits [n, T, 64], tags [n, T])."""
    t = np.ascontiguousarray(tokens, dtype=np.int32)
    n, T = t.shape
    r = (lambda a: round_bf16(a)) if emulate_bf16 else (lambda a: _f64(a))
    e = embed_gather(t, r(E)).reshape(n * T, -1)
    w1, w2, w3 = (r(w) for w in ws)
    h = linear(e, w1, ACT_GELU)
    h = r(h) if emulate_bf16 else h
    g = linear(h, w2, ACT_NONE)
    g = r(g) if emulate_bf16 else g
    z = linear(g, w3, ACT_NONE)
    return z.reshape(n, T, -1), argmax(z).reshape(n, T)


def pipeline_mlp(x_u8: np.ndarray, ws, nthreads: int = 0):
    """Plain 2-stage pipeline: normalise, 3-layer ReLU MLP, argmax.
    Returns (logits [n, N3] float64, idx [n] int32)."""
    x = np.ascontiguousarray(x_u8, dtype=np.uint8).reshape(x_u8.shape[0], -1)
    w1, w2, w3 = (_f64(w) for w in ws)
    dims = np.array([w1.shape[1], w1.shape[0], w2.shape[0], w3.shape[0]], np.int32)
    n = x.shape[0]
    logits = np.empty((n, dims[3]), np.float64)
    idx = np.empty(n, np.int32)
    lib().orc_pipeline_mlp(_p(x), n, _p(dims), _p(w1), _p(w2), _p(w3), _p(logits), _p(idx),
                           int(nthreads))
    return logits, idx


def pipeline_gemm3(x_u8: np.ndarray, ws, top_k: int = 5, emulate_bf16: bool = False,
                   nthreads: int = 0):
    """3-stage pipeline: pool+normalise, gelu(Wb gelu(Wa y)), logits Wc h, top-k.
    Returns (logits [n, N3], idx [n, k])."""
    x = np.ascontiguousarray(x_u8, dtype=np.uint8)
    n, H, W, _ = x.shape
    wa, wb, wc = (_f64(w) for w in ws)
    dims = np.array([wa.shape[1], wa.shape[0], wb.shape[0], wc.shape[0]], np.int32)
    logits = np.empty((n, dims[3]), np.float64)
    idx = np.empty((n, top_k), np.int32)
    lib().orc_pipeline_gemm3(_p(x), n, H, W, _p(dims), _p(wa), _p(wb), _p(wc), top_k,
                             int(bool(emulate_bf16)), _p(logits), _p(idx), int(nthreads))
    return logits, idx


# ---------------------------------------------------------------------------
# event-driven simulator
# ---------------------------------------------------------------------------
def simulate(arrivals_s, B: int, t_wait: float, instances, tau, caps=None, mult=None):
    """Completion time of every query (seconds) and the issued batch sizes.

    ``tau[s][b-1]`` = service time of a b-query batch at stage s; ``mult`` an
    optional ``[stages, m]`` array of per-batch service-time multipliers."""
    arr = _f64(arrivals_s)
    ns = len(instances)
    inst = np.ascontiguousarray(instances, dtype=np.int32)
    tau = _f64(tau).reshape(ns, B)
    caps = np.ascontiguousarray(caps if caps is not None else [1 << 30] * ns, dtype=np.int32)
    if mult is not None:
        mult = _f64(mult).reshape(ns, -1)
        mlen = mult.shape[1]
    else:
        mlen = 0
    done = np.empty(arr.size, np.float64)
    bs = np.empty(arr.size, np.int32)
    nb = lib().orc_simulate(_p(arr), arr.size, int(B), float(t_wait), ns, _p(inst), _p(tau),
                            _p(caps), _p(mult) if mult is not None else None, mlen, _p(done),
                            _p(bs))
    return done, bs[:nb]


def simulate_qos(arrivals_s, B: int, t_wait: float, qos_budget: float, lat, instances, tau, caps=None):
    """simulate() with the QoS form of the batch trigger (Sec. 5.2 step 2): a
    partial batch of k queries also leaves once its oldest query has waited
    qos_budget - lat[k - 1] (lat[k - 1] = predicted latency of a k-query batch,
    qos_budget = QoS less its margin).  Returns (done, batch sizes, issue times)."""
    arr = _f64(arrivals_s)
    ns = len(instances)
    inst = np.ascontiguousarray(instances, dtype=np.int32)
    tau = _f64(tau).reshape(ns, B)
    lat = _f64(lat).reshape(B)
    caps = np.ascontiguousarray(caps if caps is not None else [1 << 30] * ns, dtype=np.int32)
    done = np.empty(arr.size, np.float64)
    bs = np.empty(arr.size, np.int32)
    iss = np.empty(arr.size, np.float64)
    nb = lib().orc_simulate_qos(_p(arr), arr.size, int(B), float(t_wait), float(qos_budget), _p(lat), ns,
                                _p(inst), _p(tau), _p(caps), None, 0, _p(done), _p(bs), _p(iss))
    return done, bs[:nb], iss[:nb]


# ---------------------------------------------------------------------------
# allocator
# ---------------------------------------------------------------------------
def _alloc_args(prob):
    f = _f64(prob["f"])      # [nb, n, L]
    bw = _f64(prob["bw"])
    d = _f64(prob["d"])
    mem = _f64(prob["mem"])  # [nb, n]
    nb, n, L = f.shape
    return f, bw, d, mem, nb, n, L


def allocate(prob: dict, policy: int, solver: str = "exhaustive", iters: int = 5000,
             T0: float = 1.0, alpha: float = 0.995, seed: int = 0):
    """Solve Eq. 1 (policy 0) or Eq. 3 (policy 1) on a profile table.

    ``prob`` keys: f, bw, d ([nb, n, L]), mem ([nb, n]), unit, S, I, BW, F, qos,
    load, and optionally hb ([nb, n, L] host-link demand) with HB (its budget;
    exhaustive solver only).  Returns None if infeasible, else dict(bi, N, l, p,
    thr, sms)."""
    f, bw, d, mem, nb, n, L = _alloc_args(prob)
    bi = C.c_int(0)
    N = np.zeros(n, np.int32)
    lv = np.zeros(n, np.int32)
    thr = C.c_double(0)
    sms = C.c_int(0)
    common = (n, L, nb, int(prob["unit"]), int(prob["S"]), int(prob["I"]), _p(f), _p(bw),
              _p(d), _p(mem), float(prob["BW"]), float(prob["F"]), float(prob["qos"]),
              float(prob.get("load", 0.0)), int(policy))
    outs = (C.byref(bi), _p(N), _p(lv), C.byref(thr), C.byref(sms))
    if solver == "exhaustive" and prob.get("hb") is not None:
        hb = _f64(prob["hb"])
        ok = lib().orc_allocate_exhaustive_hl(*common, _p(hb), float(prob["HB"]), *outs)
    elif solver == "exhaustive":
        ok = lib().orc_allocate_exhaustive(*common, *outs)
    else:
        ok = lib().orc_allocate_anneal(*common, int(iters), float(T0), float(alpha),
                                       int(seed), *outs)
    if not ok:
        return None
    return dict(bi=bi.value, N=N.tolist(), l=lv.tolist(),
                p=[(x + 1) * int(prob["unit"]) for x in lv.tolist()], thr=thr.value,
                sms=sms.value)


def min_gpus(Cs, Ms, G: float, F: float) -> float:
    Cs, Ms = _f64(Cs), _f64(Ms)
    return lib().orc_min_gpus(_p(Cs), _p(Ms), Cs.size, float(G), float(F))


# ---------------------------------------------------------------------------
# predictor MLP
# ---------------------------------------------------------------------------
def pred_nparams() -> int:
    return int(lib().orc_pred_nparams())


def pred_forward(theta, X) -> np.ndarray:
    theta, X = _f64(theta), _f64(X)
    y = np.empty(X.shape[0], np.float64)
    lib().orc_pred_forward(_p(theta), _p(X), X.shape[0], _p(y))
    return y


def pred_grad(theta, X, t):
    theta, X, t = _f64(theta), _f64(X), _f64(t)
    g = np.empty_like(theta)
    loss = lib().orc_pred_grad(_p(theta), _p(X), _p(t), X.shape[0], _p(g))
    return loss, g


def adam_step(theta, g, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays theta, m, v."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(g)
    lib().orc_adam_step(_p(theta), _p(g), _p(m), _p(v), theta.size, int(t), lr, b1, b2, eps)
