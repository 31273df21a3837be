"""ctypes binding of ``libcamelot.so`` (declared in ``include/camelot.h``).

Argument marshalling only: every step of the query path runs in the library's
CUDA kernels and C++ runtime.  Functions keep the C names; errors raise
``CamelotError`` carrying the status code and ``camelot_last_error()``.
There is no fallback: if the library cannot be loaded, importing fails.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

MAX_LAYERS, MAX_STAGES, MAX_TOPK = 4, 8, 5
PRED_FEATURES, PRED_PARAMS = 12, 5057

OK, EINVAL, ENOMEM, EAGAIN, ETIMEDOUT, ECUDA, ESTATE, EINFEASIBLE = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "EAGAIN", "ETIMEDOUT", "ECUDA", "ESTATE", "EINFEASIBLE"]

STAGE_NORMALIZE_U8, STAGE_NORM_POOL2_BF16, STAGE_MLP_FP32, STAGE_GEMM_BF16 = 1, 2, 3, 4
STAGE_GEMM_FP8, STAGE_NORMALIZE_U8_E4M3, STAGE_EMBED_GATHER = 5, 6, 7
STAGE_COMPUTE_SYNTH, STAGE_STREAM_SYNTH = 8, 9
ACT_NONE, ACT_RELU, ACT_GELU = 0, 1, 2
HANDOFF_GLOBAL, HANDOFF_HOST_STAGED = 0, 1
POLICY_MAX_PEAK, POLICY_MIN_SM = 0, 1
SOLVER_EXHAUSTIVE, SOLVER_ANNEAL = 0, 1


class CamelotError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class StageDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_layers", C.c_int32), ("dims", C.c_int32 * (MAX_LAYERS + 1)),
                ("act", C.c_int32 * MAX_LAYERS), ("top_k", C.c_int32), ("max_batch", C.c_int32),
                ("weights", C.c_void_p * MAX_LAYERS), ("scales", C.c_float * (MAX_LAYERS + 1)),
                ("rows_per_query", C.c_int32), ("ring_slots", C.c_int32)]


class Alloc(C.Structure):
    _fields_ = [("n_stages", C.c_int32), ("instances", C.c_int32 * MAX_STAGES),
                ("sm_quota", C.c_int32 * MAX_STAGES), ("batch", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("query_slots", C.c_uint32), ("batch_slots", C.c_uint32), ("max_wait_ns", C.c_int64),
                ("idle_exit_ns", C.c_int64), ("wait_limit_ns", C.c_int64),
                ("logits_sink", C.c_void_p), ("exit_after_trace", C.c_int32),
                ("data_slots", C.c_uint32), ("device_data", C.c_int32), ("qos_ns", C.c_int64),
                ("qos_margin_ns", C.c_int64), ("batch_latency_ns", C.c_int64 * 32)]


class StageCost(C.Structure):
    _fields_ = [("stage_id", C.c_int32), ("pad_", C.c_int32), ("flop_per_query", C.c_double), ("bytes_per_batch", C.c_double),
                ("bytes_per_query", C.c_double), ("mem_bytes", C.c_double)]


class Completion(C.Structure):
    _fields_ = [("query_id", C.c_uint64), ("stream_id", C.c_uint32), ("status", C.c_int32),
                ("idx", C.c_int32 * MAX_TOPK), ("val", C.c_float * MAX_TOPK),
                ("batch_size", C.c_int32), ("pad_", C.c_int32), ("t_arrival_ns", C.c_int64),
                ("t_batch_ns", C.c_int64), ("t_done_ns", C.c_int64), ("t_poll_ns", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64),
                ("batches", C.c_uint64 * MAX_STAGES), ("kernel_launches", C.c_uint64),
                ("relayed_bytes", C.c_uint64), ("device_bytes_per_batch_slot", C.c_uint64),
                ("device_ring_bytes", C.c_uint64), ("device_status", C.c_int32),
                ("device_where", C.c_int32), ("last_launch_ms", C.c_double),
                ("total_launch_ms", C.c_double), ("busy_ns", C.c_uint64 * MAX_STAGES),
                ("body_ns", C.c_uint64 * MAX_STAGES), ("acquire_ns", C.c_uint64 * MAX_STAGES)]


class ServerOptions(C.Structure):
    _fields_ = [("device_bytes_budget", C.c_uint64), ("host_queue_queries", C.c_uint32),
                ("max_admit", C.c_uint32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("waiting", C.c_uint64), ("deferred", C.c_uint64), ("inflight_bytes", C.c_uint64),
                ("peak_inflight_bytes", C.c_uint64), ("total_inflight_bytes", C.c_uint64),
                ("status", C.c_int32), ("pad_", C.c_int32)]


XRING_MAX_SLOTS = 64


class XringHandle(C.Structure):
    """camelot_xring_handle: plain bytes, safe to send to another process."""
    _fields_ = [("slot_bytes", C.c_uint64), ("slots", C.c_uint32), ("device", C.c_int32),
                ("mem", C.c_ubyte * 64), ("ready", (C.c_ubyte * 64) * XRING_MAX_SLOTS),
                ("free_", (C.c_ubyte * 64) * XRING_MAX_SLOTS)]


class Profile(C.Structure):
    _fields_ = [("n_stages", C.c_int32), ("n_levels", C.c_int32), ("n_batches", C.c_int32),
                ("unit", C.c_int32), ("batch_sizes", C.c_void_p), ("thr_qps", C.c_void_p),
                ("bw_gbs", C.c_void_p), ("dur_s", C.c_void_p), ("mem_bytes", C.c_void_p),
                ("host_gbs", C.c_void_p)]


class Constraints(C.Structure):
    _fields_ = [("total_sms", C.c_int32), ("max_instances", C.c_int32), ("bw_gbs", C.c_double),
                ("mem_bytes", C.c_double), ("qos_s", C.c_double), ("load_qps", C.c_double),
                ("solver", C.c_int32), ("anneal_iters", C.c_int32), ("anneal_t0", C.c_double),
                ("anneal_alpha", C.c_double), ("seed", C.c_uint64), ("host_gbs", C.c_double)]


# Every symbol include/camelot.h declares, with its ctypes signature.
P = C.c_void_p
_SIGS = {
    "camelot_last_error": (C.c_char_p, []),
    "camelot_version": (C.c_int, []),
    "camelot_stage_prepare": (C.c_int, [P, P]),
    "camelot_stage_release": (C.c_int, [P]),
    "camelot_stage_info": (C.c_int, [P, P, P, C.c_uint32, P]),
    "camelot_stage_export_weights": (C.c_int, [P, C.c_int, P, C.c_size_t, P]),
    "camelot_stage_launch": (C.c_int, [P, C.c_int, P, C.c_uint32, P, P, P, P, P, C.c_size_t, P]),
    "camelot_stage_launch_noalloc": (C.c_int, [P, C.c_int, P, C.c_uint32, P, P, P, P, P]),
    "camelot_stage_time": (C.c_int, [P, C.c_int, P, C.c_uint32, P, P, P, P, P, C.c_size_t, P,
                                     C.c_uint32, P]),
    "camelot_corunner_start": (C.c_int, [P, P, C.c_size_t, C.c_int, C.c_int64, P]),
    "camelot_corunner_stop": (C.c_int, [P, P]),
    "camelot_predictor_create": (C.c_int, [P, P]),
    "camelot_predictor_set_params": (C.c_int, [P, P]),
    "camelot_predictor_get_params": (C.c_int, [P, P]),
    "camelot_predictor_set_norm": (C.c_int, [P, P, P]),
    "camelot_predictor_forward": (C.c_int, [P, P, C.c_uint32, P, P]),
    "camelot_predictor_grad": (C.c_int, [P, P, P, P, C.c_uint32, P, P, P]),
    "camelot_predictor_train_step": (C.c_int, [P, P, P, P, C.c_uint32, C.c_float, P, P]),
    "camelot_predictor_destroy": (C.c_int, [P]),
    "camelot_predictor_features": (C.c_int, [P, C.c_int, C.c_uint32, P, P, P, P, P, P]),
    "camelot_profile_from_latency": (C.c_int, [P, C.c_int, P, C.c_int, C.c_int, P, P, P, P, P]),
    "camelot_profile_predict": (C.c_int, [P, P, C.c_int, P, C.c_int, C.c_int, C.c_int, C.c_int32, C.c_double,
                                          P, P, P, P]),
    "camelot_fp8_scale": (C.c_int, [P, C.c_size_t, P, P]),
    "camelot_options_default": (None, [P]),
    "camelot_pipeline_create": (C.c_int, [P, C.c_int, P, C.c_int, P, P]),
    "camelot_submit": (C.c_int, [P, C.c_uint32, P, C.c_uint32, P, P]),
    "camelot_submit_trace": (C.c_int, [P, C.c_uint32, P, C.c_uint32, P, P]),
    "camelot_poll": (C.c_int, [P, P, C.c_uint32, P, C.c_int64]),
    "camelot_pipeline_stats": (C.c_int, [P, P]),
    "camelot_pipeline_destroy": (C.c_int, [P]),
    "camelot_pipeline_stall_relay": (C.c_int, [P, C.c_int]),
    "camelot_allocate": (C.c_int, [P, C.c_int, P, P, P]),
    "camelot_trigger_latency": (C.c_int, [P, P, P]),
    "camelot_profile_add_handover": (C.c_int, [P, P, P, P, P]),
    "camelot_simulate_profile": (C.c_int, [P, P, P, C.c_double, C.c_double, C.c_uint32, C.c_uint64, P, P, P]),
    "camelot_server_options_default": (None, [P]),
    "camelot_server_create": (C.c_int, [P, C.c_int, P, P]),
    "camelot_server_submit": (C.c_int, [P, C.c_int, C.c_uint32, P, C.c_uint32, P]),
    "camelot_server_poll": (C.c_int, [P, C.c_int, P, C.c_uint32, P, C.c_int64]),
    "camelot_server_stats": (C.c_int, [P, C.c_int, P]),
    "camelot_server_destroy": (C.c_int, [P]),
    "camelot_xring_create": (C.c_int, [C.c_uint64, C.c_uint32, P, P]),
    "camelot_xring_open": (C.c_int, [P, P]),
    "camelot_xring_slot": (P, [P, C.c_uint32]),
    "camelot_xring_produce_begin": (C.c_int, [P, C.c_uint32, P]),
    "camelot_xring_produce_end": (C.c_int, [P, C.c_uint32, P]),
    "camelot_xring_consume_begin": (C.c_int, [P, C.c_uint32, P]),
    "camelot_xring_consume_end": (C.c_int, [P, C.c_uint32, P]),
    "camelot_xring_destroy": (C.c_int, [P]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcamelot.so (building it first when the sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise OSError(f"libcamelot.so not found at {path}")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st: int, allow=()):
    if st != OK and st not in allow:
        raise CamelotError(st, load().camelot_last_error().decode())
    return st


def _ptr(x) -> int | None:
    """Device/host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(type(x))


# ---------------------------------------------------------------------------
# same-named wrappers
# ---------------------------------------------------------------------------
def camelot_version() -> int:
    return load().camelot_version()


def camelot_last_error() -> str:
    return load().camelot_last_error().decode()


def camelot_stage_prepare(desc: StageDesc) -> int:
    h = C.c_void_p()
    _check(load().camelot_stage_prepare(C.byref(desc), C.byref(h)))
    return h.value


def camelot_stage_release(st: int) -> None:
    _check(load().camelot_stage_release(st))


def camelot_stage_info(st: int, n: int = 1):
    a, b, s = C.c_size_t(), C.c_size_t(), C.c_size_t()
    _check(load().camelot_stage_info(st, C.byref(a), C.byref(b), n, C.byref(s)))
    return a.value, b.value, s.value


def camelot_stage_export_weights(st: int, layer: int, rows: int, cols: int, esz: int):
    """Layer weights as the kernels use them: numpy uint16 (bf16 bits) or
    uint8 (e4m3 codes) [rows, cols], and the weight scale."""
    import numpy as np
    out = np.empty((rows, cols), np.uint16 if esz == 2 else np.uint8)
    sc = C.c_float()
    _check(load().camelot_stage_export_weights(st, layer, out.ctypes.data, out.nbytes, C.byref(sc)))
    return out, sc.value


def camelot_stage_launch(st: int, n_ctas: int, inp, n: int, out=None, out_idx=None, out_val=None,
                         out_logits=None, scratch=None, scratch_bytes: int = 0, stream=None) -> None:
    _check(load().camelot_stage_launch(st, n_ctas, _ptr(inp), n, _ptr(out), _ptr(out_idx),
                                       _ptr(out_val), _ptr(out_logits), _ptr(scratch),
                                       scratch_bytes, _ptr(stream)))


def camelot_stage_launch_noalloc(st: int, n_ctas: int, inp, n: int, out=None, out_idx=None,
                                 out_val=None, out_logits=None, stream=None) -> None:
    """Stage launch whose scratch is the library's static device buffer."""
    _check(load().camelot_stage_launch_noalloc(st, n_ctas, _ptr(inp), n, _ptr(out), _ptr(out_idx),
                                               _ptr(out_val), _ptr(out_logits), _ptr(stream)))


def camelot_stage_time(st: int, n_ctas: int, inp, n: int, out=None, out_idx=None, out_val=None,
                       out_logits=None, scratch=None, scratch_bytes: int = 0, stream=None,
                       runs: int = 1):
    """Per-launch durations (ms, numpy float32 [runs]) of ``runs`` back-to-back launches."""
    import numpy as np
    ms = np.zeros(runs, np.float32)
    _check(load().camelot_stage_time(st, n_ctas, _ptr(inp), n, _ptr(out), _ptr(out_idx),
                                     _ptr(out_val), _ptr(out_logits), _ptr(scratch), scratch_bytes,
                                     _ptr(stream), runs, ms.ctypes.data))
    return ms


def camelot_corunner_start(src, dst, nbytes: int, n_ctas: int, max_ns: int = 120_000_000_000) -> int:
    h = C.c_void_p()
    _check(load().camelot_corunner_start(_ptr(src), _ptr(dst), nbytes, n_ctas, max_ns, C.byref(h)))
    return h.value


def camelot_corunner_stop(c: int) -> float:
    """Stops the co-runner; returns the GB/s it streamed (read + write)."""
    g = C.c_double()
    _check(load().camelot_corunner_stop(c, C.byref(g)))
    return g.value


def _f32_host(a, n):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def camelot_predictor_create(init_params) -> int:
    a = _f32_host(init_params, PRED_PARAMS)
    h = C.c_void_p()
    _check(load().camelot_predictor_create(a.ctypes.data, C.byref(h)))
    return h.value


def camelot_predictor_set_params(p: int, params) -> None:
    a = _f32_host(params, PRED_PARAMS)
    _check(load().camelot_predictor_set_params(p, a.ctypes.data))


def camelot_predictor_get_params(p: int):
    import numpy as np
    out = np.empty(PRED_PARAMS, np.float32)
    _check(load().camelot_predictor_get_params(p, out.ctypes.data))
    return out


def camelot_predictor_set_norm(p: int, mean, inv_std) -> None:
    m, s = _f32_host(mean, PRED_FEATURES), _f32_host(inv_std, PRED_FEATURES)
    _check(load().camelot_predictor_set_norm(p, m.ctypes.data, s.ctypes.data))


def camelot_predictor_forward(p: int, X, n: int, y, stream=None) -> None:
    _check(load().camelot_predictor_forward(p, _ptr(X), n, _ptr(y), _ptr(stream)))


def camelot_predictor_grad(p: int, X, t, idx, n: int, grad, loss=None, stream=None) -> None:
    _check(load().camelot_predictor_grad(p, _ptr(X), _ptr(t), _ptr(idx), n, _ptr(grad), _ptr(loss),
                                         _ptr(stream)))


def camelot_predictor_train_step(p: int, X, t, idx, n: int, lr: float, loss=None, stream=None) -> None:
    _check(load().camelot_predictor_train_step(p, _ptr(X), _ptr(t), _ptr(idx), n, lr, _ptr(loss),
                                               _ptr(stream)))


def camelot_predictor_destroy(p: int) -> None:
    _check(load().camelot_predictor_destroy(p))


def _costs(costs):
    arr = (StageCost * len(costs))()
    for i, c in enumerate(costs):
        arr[i] = StageCost(int(c[0]), 0, float(c[1]), float(c[2]), float(c[3]), float(c[4]))
    return arr


def camelot_predictor_features(costs, stage, batch, sms, co_sms, co_gbs):
    """costs: sequence of (stage_id, flop_per_query, bytes_per_batch,
    bytes_per_query, mem_bytes); `stage` indexes it; the other arguments are
    arrays of the same length (or scalars).  Returns float32 [n, 12]."""
    import numpy as np
    stage = np.ascontiguousarray(stage, np.int32)
    n = stage.size
    batch = np.ascontiguousarray(np.broadcast_to(batch, (n,)), np.int32)
    sms = np.ascontiguousarray(np.broadcast_to(sms, (n,)), np.int32)
    co_sms = np.ascontiguousarray(np.broadcast_to(co_sms, (n,)), np.int32)
    co_gbs = np.ascontiguousarray(np.broadcast_to(co_gbs, (n,)), np.float64)
    X = np.empty((n, PRED_FEATURES), np.float32)
    _check(load().camelot_predictor_features(_costs(costs), len(costs), n, stage.ctypes.data, batch.ctypes.data,
                                             sms.ctypes.data, co_sms.ctypes.data, co_gbs.ctypes.data,
                                             X.ctypes.data))
    return X


def camelot_profile_from_latency(costs, batch_sizes, lat_s):
    """lat_s [n_batches, n_stages, n_levels] seconds -> (thr, bw, dur, mem) arrays."""
    import numpy as np
    lat = np.ascontiguousarray(lat_s, np.float64)
    nb, n, L = lat.shape
    bs = np.ascontiguousarray(batch_sizes, np.int32)
    thr, bw, dur = (np.empty_like(lat) for _ in range(3))
    mem = np.empty((nb, n), np.float64)
    _check(load().camelot_profile_from_latency(_costs(costs), n, bs.ctypes.data, nb, L, lat.ctypes.data,
                                               thr.ctypes.data, bw.ctypes.data, dur.ctypes.data, mem.ctypes.data))
    return thr, bw, dur, mem


def camelot_profile_predict(pred: int, costs, batch_sizes, unit: int, n_levels: int, co_sms: int = 0,
                            co_gbs: float = 0.0):
    """Predicted (thr, bw, dur, mem) arrays for every batch size, stage and level."""
    import numpy as np
    bs = np.ascontiguousarray(batch_sizes, np.int32)
    nb, n = bs.size, len(costs)
    thr, bw, dur = (np.empty((nb, n, n_levels), np.float64) for _ in range(3))
    mem = np.empty((nb, n), np.float64)
    _check(load().camelot_profile_predict(pred, _costs(costs), n, bs.ctypes.data, nb, unit, n_levels, co_sms,
                                          float(co_gbs), thr.ctypes.data, bw.ctypes.data, dur.ctypes.data,
                                          mem.ctypes.data))
    return thr, bw, dur, mem


def camelot_fp8_scale(x, n: int, stream=None) -> float:
    s = C.c_float()
    _check(load().camelot_fp8_scale(_ptr(x), n, _ptr(stream), C.byref(s)))
    return s.value


def camelot_options_default() -> Options:
    o = Options()
    load().camelot_options_default(C.byref(o))
    return o


def camelot_pipeline_create(stages, alloc: Alloc, mode: int, opts: Options | None = None) -> int:
    arr = (C.c_void_p * len(stages))(*stages)
    h = C.c_void_p()
    _check(load().camelot_pipeline_create(arr, len(stages), C.byref(alloc), mode,
                                          C.byref(opts) if opts is not None else None, C.byref(h)))
    return h.value


def camelot_submit(p: int, stream_id: int, queries, n: int, arrival_ns=None, allow_eagain=False):
    """Returns the first query ID, or None on EAGAIN when ``allow_eagain``."""
    first = C.c_uint64()
    st = _check(load().camelot_submit(p, stream_id, _ptr(queries), n, _ptr(arrival_ns),
                                      C.byref(first)), allow=(EAGAIN,) if allow_eagain else ())
    return None if st == EAGAIN else first.value


def camelot_submit_trace(p: int, stream_id: int, queries, n: int, arrival_off_ns) -> int:
    first = C.c_uint64()
    _check(load().camelot_submit_trace(p, stream_id, _ptr(queries), n, _ptr(arrival_off_ns),
                                       C.byref(first)))
    return first.value


def camelot_poll(p: int, buf, timeout_us: int = 0, allow_timeout: bool = True) -> int:
    """Fill ``buf`` (a ctypes array of Completion) and return the count."""
    n = C.c_uint32()
    _check(load().camelot_poll(p, buf, len(buf), C.byref(n), timeout_us),
           allow=(ETIMEDOUT,) if allow_timeout else ())
    return n.value


def camelot_pipeline_stats(p: int) -> Stats:
    s = Stats()
    _check(load().camelot_pipeline_stats(p, C.byref(s)))
    return s


def camelot_pipeline_destroy(p: int) -> None:
    _check(load().camelot_pipeline_destroy(p))


def camelot_pipeline_stall_relay(p: int, stall: bool) -> None:
    _check(load().camelot_pipeline_stall_relay(p, 1 if stall else 0))


def camelot_allocate(prof: Profile, policy: int, cons: Constraints):
    a = Alloc()
    obj = C.c_double()
    _check(load().camelot_allocate(C.byref(prof), policy, C.byref(cons), C.byref(a), C.byref(obj)))
    return a, obj.value


def camelot_trigger_latency(prof: Profile, alloc: Alloc):
    """Predicted batch latency in ns for b = 1..32 (a list of 32 ints)."""
    out = (C.c_int64 * 32)()
    _check(load().camelot_trigger_latency(C.byref(prof), C.byref(alloc), out))
    return list(out)


def camelot_profile_add_handover(prof: Profile, handover_s, thr, bw, dur) -> None:
    """In place on the float64 arrays thr, bw, dur (which may be the profile's own)."""
    import numpy as np
    h = np.ascontiguousarray(handover_s, np.float64)
    _check(load().camelot_profile_add_handover(C.byref(prof), h.ctypes.data, _ptr(thr), _ptr(bw), _ptr(dur)))


def camelot_simulate_profile(prof: Profile, alloc: Alloc, handover_s, max_wait_s: float, rate_qps: float,
                             n_queries: int = 20000, seed: int = 1):
    """(p50 s, p99 s, throughput q/s) of the simulated pipeline."""
    import numpy as np
    h = None if handover_s is None else np.ascontiguousarray(handover_s, np.float64)
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(load().camelot_simulate_profile(C.byref(prof), C.byref(alloc), None if h is None else h.ctypes.data,
                                           max_wait_s, rate_qps, n_queries, seed, C.byref(a), C.byref(b),
                                           C.byref(c)))
    return a.value, b.value, c.value


def camelot_server_options_default() -> ServerOptions:
    o = ServerOptions()
    load().camelot_server_options_default(C.byref(o))
    return o


def camelot_server_create(pipelines, opts: ServerOptions | None = None) -> int:
    arr = (C.c_void_p * len(pipelines))(*pipelines)
    h = C.c_void_p()
    _check(load().camelot_server_create(arr, len(pipelines), C.byref(opts) if opts is not None else None,
                                        C.byref(h)))
    return h.value


def camelot_server_submit(s: int, pipeline: int, stream_id: int, queries, n: int, arrival_ns=None,
                          allow_eagain: bool = False) -> bool:
    """True if queued, False on EAGAIN when ``allow_eagain``."""
    st = _check(load().camelot_server_submit(s, pipeline, stream_id, _ptr(queries), n, _ptr(arrival_ns)),
                allow=(EAGAIN,) if allow_eagain else ())
    return st == OK


def camelot_server_poll(s: int, pipeline: int, buf, timeout_us: int = 0) -> int:
    n = C.c_uint32()
    _check(load().camelot_server_poll(s, pipeline, buf, len(buf), C.byref(n), timeout_us), allow=(ETIMEDOUT,))
    return n.value


def camelot_server_stats(s: int, pipeline: int) -> ServerStats:
    st = ServerStats()
    _check(load().camelot_server_stats(s, pipeline, C.byref(st)))
    return st


def camelot_server_destroy(s: int) -> None:
    _check(load().camelot_server_destroy(s))


def camelot_xring_create(slot_bytes: int, slots: int):
    """Producer side: returns (ring, handle bytes for the consumer process)."""
    x, h = C.c_void_p(), XringHandle()
    _check(load().camelot_xring_create(slot_bytes, slots, C.byref(x), C.byref(h)))
    return x.value, bytes(h)


def camelot_xring_open(handle: bytes) -> int:
    h = XringHandle.from_buffer_copy(handle)
    x = C.c_void_p()
    _check(load().camelot_xring_open(C.byref(h), C.byref(x)))
    return x.value


def camelot_xring_slot(x: int, k: int) -> int:
    return load().camelot_xring_slot(x, k) or 0


def camelot_xring_produce_begin(x: int, k: int, stream=None) -> None:
    _check(load().camelot_xring_produce_begin(x, k, _ptr(stream)))


def camelot_xring_produce_end(x: int, k: int, stream=None) -> None:
    _check(load().camelot_xring_produce_end(x, k, _ptr(stream)))


def camelot_xring_consume_begin(x: int, k: int, stream=None) -> None:
    _check(load().camelot_xring_consume_begin(x, k, _ptr(stream)))


def camelot_xring_consume_end(x: int, k: int, stream=None) -> None:
    _check(load().camelot_xring_consume_end(x, k, _ptr(stream)))


def camelot_xring_destroy(x: int) -> None:
    _check(load().camelot_xring_destroy(x))
