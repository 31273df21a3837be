"""Learned latency predictor of the allocator (Sec. 7.1) and its profiling
harness.

The paper predicts each microservice's duration, bandwidth and throughput
under a given SM share and batch size from solo-run profiling with decision
trees, and feeds the predictions to the allocator (Sec. 7.2-7.3).  Here one
MLP (12 -> 64 -> 64 -> 1, FP32) predicts log p99 latency of a stage batch
from features that also describe a memory-bandwidth co-runner, so contention
(Sec. 4.2) enters the prediction.  Training and inference run in the
library's kernels (``camelot_predictor_*``), and the library also builds the
feature rows (``camelot_predictor_features``) and the allocator's table
(``camelot_profile_from_latency``, ``camelot_profile_predict``); this module
drives the profiling runs (``camelot_stage_time`` with and without
``camelot_corunner_*``) and marshals arrays.
"""
from __future__ import annotations

import json
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import camelot as cm

FEATURES = ("stage", "batch", "sms", "flop_per_batch", "bytes_per_batch", "flop_per_byte",
            "corunner_sms", "corunner_gbs", "corunner_active", "sms_in_use", "log2_batch", "inv_sms")
assert len(FEATURES) == cm.PRED_FEATURES


@dataclass(frozen=True)
class StageCost:
    """Algorithmic work of one stage: FLOPs per query, bytes read or written
    once per batch (weights) and per query (inputs + outputs)."""
    stage_id: int
    flop_per_query: float
    bytes_per_batch: float
    bytes_per_query: float

    def flop(self, B):
        return self.flop_per_query * np.asarray(B, np.float64)

    def bytes(self, B):
        return self.bytes_per_batch + self.bytes_per_query * np.asarray(B, np.float64)


def dense_cost(stage_id: int, dims, in_bytes: int, out_bytes: int, weight_bytes: int = 4) -> StageCost:
    macs = sum(a * b for a, b in zip(dims[:-1], dims[1:]))
    return StageCost(stage_id, 2.0 * macs, float(weight_bytes * macs), float(in_bytes + out_bytes))


def c_costs(costs: dict, mem_bytes: float = 64e6) -> tuple:
    """The stages' costs in stage-id order, as camelot_stage_cost tuples."""
    return tuple((int(k), c.flop_per_query, c.bytes_per_batch, c.bytes_per_query, mem_bytes)
                 for k, c in sorted(costs.items()))


def feature_rows(costs: dict, stage, B, p, co_sms, co_gbs) -> np.ndarray:
    """Raw feature matrix [n, 12] (float32) for arrays of stage ids, batch
    sizes, SM quotas, co-runner SMs (0 = none) and co-runner solo GB/s, built
    by camelot_predictor_features."""
    ids = sorted(costs)
    stage = np.atleast_1d(np.asarray(stage, np.int64))
    index = np.searchsorted(np.asarray(ids), stage)
    assert np.all(np.asarray(ids)[index] == stage), "unknown stage id"
    return cm.camelot_predictor_features(c_costs(costs), index, np.asarray(B, np.int64),
                                         np.asarray(p, np.int64), np.asarray(co_sms, np.int64),
                                         np.asarray(co_gbs, np.float64))


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases, in the flat layout of the C ABI."""
    g = np.random.default_rng(seed)
    H, I = 64, cm.PRED_FEATURES
    parts = [g.uniform(-1, 1, H * I) * np.sqrt(6.0 / I), np.zeros(H),
             g.uniform(-1, 1, H * H) * np.sqrt(6.0 / H), np.zeros(H),
             g.uniform(-1, 1, H) * np.sqrt(3.0 / H), np.zeros(1)]
    th = np.concatenate(parts).astype(np.float32)
    assert th.size == cm.PRED_PARAMS
    return th


class LatencyPredictor:
    """Owns a ``camelot_predictor``; targets are log(p99 latency in us)."""

    def __init__(self, params=None, seed: int = 0):
        self.h = cm.camelot_predictor_create(init_params(seed) if params is None else params)
        self.mean = np.zeros(cm.PRED_FEATURES, np.float32)
        self.inv_std = np.ones(cm.PRED_FEATURES, np.float32)

    def close(self):
        if self.h:
            cm.camelot_predictor_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_norm(self, mean, inv_std):
        self.mean = np.asarray(mean, np.float32)
        self.inv_std = np.asarray(inv_std, np.float32)
        cm.camelot_predictor_set_norm(self.h, self.mean, self.inv_std)

    def fit(self, X: np.ndarray, y: np.ndarray, epochs: int = 300, lr: float = 1e-3, batch: int = 256,
            seed: int = 0, lr_final: float | None = None) -> list:
        """Minibatch Adam on the GPU.  Feature scaling is fitted on X.  The
        minibatch order is a seeded permutation per epoch, passed to the kernels
        as an index array.  Returns the mean minibatch loss of each epoch."""
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        n = X.shape[0]
        mu = X.mean(axis=0)
        sd = X.std(axis=0)
        self.set_norm(mu, np.where(sd > 0, 1.0 / np.maximum(sd, 1e-30), 1.0))
        dev = torch.device("cuda")
        Xd = torch.from_numpy(X).to(dev)
        yd = torch.from_numpy(y).to(dev)
        steps = (n + batch - 1) // batch
        loss = torch.zeros(steps, dtype=torch.float32, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        rng = np.random.default_rng(seed)
        hist = []
        for ep in range(epochs):
            lr_ep = lr if lr_final is None else lr * (lr_final / lr) ** (ep / max(1, epochs - 1))
            perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).to(dev)
            base = perm.data_ptr()
            for s in range(steps):
                m = min(batch, n - s * batch)
                cm.camelot_predictor_train_step(self.h, Xd, yd, base + 4 * s * batch, m, lr_ep,
                                                loss.data_ptr() + 4 * s, stream)
            hist.append(float(loss.mean()))
        torch.cuda.synchronize()
        return hist

    def predict(self, X: np.ndarray) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float32)
        Xd = torch.from_numpy(X).cuda()
        yd = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        cm.camelot_predictor_forward(self.h, Xd, X.shape[0], yd, torch.cuda.current_stream().cuda_stream)
        return yd.cpu().numpy()

    def params(self) -> np.ndarray:
        torch.cuda.synchronize()
        return cm.camelot_predictor_get_params(self.h)

    def save(self, path: str):
        """Parameters and feature scaling, as a .npz with a JSON header."""
        meta = {"features": FEATURES, "hidden": [64, 64], "target": "log(p99 latency / 1 us)"}
        np.savez(path, params=self.params(), mean=self.mean, inv_std=self.inv_std,
                 meta=np.frombuffer(json.dumps(meta).encode(), np.uint8))

    @classmethod
    def load(cls, path: str) -> "LatencyPredictor":
        z = np.load(path)
        meta = json.loads(bytes(z["meta"]).decode())
        if tuple(meta["features"]) != FEATURES:
            raise ValueError("feature set of the saved predictor differs")
        p = cls(params=z["params"])
        p.set_norm(z["mean"], z["inv_std"])
        return p


def mape(pred, true) -> float:
    pred, true = np.asarray(pred, np.float64), np.asarray(true, np.float64)
    return float(np.mean(np.abs(pred - true) / true))


# ---------------------------------------------------------------------------
# profiling harness
# ---------------------------------------------------------------------------
class StageRunner:
    """A prepared stage with device input/output buffers of max_batch rows and
    its scratch, timed by ``camelot_stage_time``."""

    def __init__(self, stage: int, inp: torch.Tensor, max_batch: int, top_k: int = 0):
        self.st, self.inp, self.max_batch = stage, inp, max_batch
        _, out_row, sb = cm.camelot_stage_info(stage, max_batch)
        self.sb = sb
        self.scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
        self.out = None if top_k else torch.zeros(max_batch * out_row, dtype=torch.uint8, device="cuda")
        k = max(top_k, 1)
        self.idx = torch.empty((max_batch, k), dtype=torch.int32, device="cuda") if top_k else None
        self.val = torch.empty((max_batch, k), dtype=torch.float32, device="cuda") if top_k else None
        self.stream = torch.cuda.current_stream().cuda_stream

    def time_ms(self, B: int, p: int, runs: int) -> np.ndarray:
        return cm.camelot_stage_time(self.st, p, self.inp, B, self.out, self.idx, self.val, None,
                                     self.scr, self.sb, self.stream, runs)


class CoRunner:
    """The bandwidth hog: an FP32 copy of ``nbytes`` on ``n`` SMs."""

    def __init__(self, nbytes: int = 1 << 30):
        self.nbytes = nbytes
        self.src = torch.ones(nbytes // 4, dtype=torch.float32, device="cuda")
        self.dst = torch.empty_like(self.src)
        self._solo = {}

    def start(self, n: int) -> int:
        return cm.camelot_corunner_start(self.src, self.dst, self.nbytes, n)

    @staticmethod
    def stop(h: int) -> float:
        return cm.camelot_corunner_stop(h)

    def solo_gbs(self, n: int, seconds: float = 0.05) -> float:
        """GB/s the co-runner streams alone on n SMs (measured once per n)."""
        if n not in self._solo:
            torch.cuda.synchronize()
            h = self.start(n)
            time.sleep(seconds)
            self._solo[n] = self.stop(h)
        return self._solo[n]


def sample_configs(n: int, seed: int, stages, batches, levels, total_sms: int, unit: int = 8,
                   p_absent: float = 0.25) -> dict:
    """Random profiling configurations: stage, batch, SM quota, and a
    co-runner on a random disjoint quota (absent with probability p_absent)."""
    g = np.random.default_rng(seed)
    st = g.choice(np.asarray(stages), n)
    B = g.choice(np.asarray(batches), n)
    p = g.choice(np.asarray(levels), n)
    c = np.zeros(n, np.int64)
    for i in range(n):
        room = (total_sms - p[i]) // unit
        if room >= 1 and g.random() >= p_absent:
            c[i] = unit * g.integers(1, room + 1)
    return {"stage": st, "batch": B, "sms": p, "corunner_sms": c}


def collect(runners: dict, cfg: dict, runs: int, co: CoRunner, log=None) -> dict:
    """Measure every configuration: p99 of ``runs`` back-to-back launches.
    Configurations sharing a co-runner quota run under one co-runner launch."""
    n = len(cfg["stage"])
    p99 = np.zeros(n)
    gbs = np.zeros(n)
    order = np.argsort(cfg["corunner_sms"], kind="stable")
    t0 = time.time()
    for c in np.unique(cfg["corunner_sms"]):
        ids = order[cfg["corunner_sms"][order] == c]
        h = None
        if c > 0:
            g = co.solo_gbs(int(c))
            gbs[ids] = g
            h = co.start(int(c))
        try:
            for i in ids:
                r = runners[int(cfg["stage"][i])]
                r.time_ms(int(cfg["batch"][i]), int(cfg["sms"][i]), 1)   # warm
                ms = r.time_ms(int(cfg["batch"][i]), int(cfg["sms"][i]), runs)
                p99[i] = np.percentile(ms, 99) * 1e3
        finally:
            if h is not None:
                co.stop(h)
        if log:
            log(f"co-runner {int(c)} SMs: {len(ids)} configs, {time.time() - t0:.1f}s")
    out = dict(cfg)
    out["corunner_gbs"] = gbs
    out["p99_us"] = p99
    return out


def solo_table(runners: dict, stages, batches, levels, runs: int) -> np.ndarray:
    """Measured p99 (us) of every (stage, batch, quota) alone: the exhaustive
    profiling that the predictor stands in for.  Shape [stages][batches][levels]."""
    t = np.zeros((len(stages), len(batches), len(levels)))
    for si, s in enumerate(stages):
        for bi, B in enumerate(batches):
            for li, p in enumerate(levels):
                r = runners[int(s)]
                r.time_ms(int(B), int(p), 1)
                t[si, bi, li] = np.percentile(r.time_ms(int(B), int(p), runs), 99) * 1e3
    return t


def predicted_table(pred: LatencyPredictor, costs: dict, stages, batches, levels,
                    co_sms: int = 0, co_gbs: float = 0.0) -> np.ndarray:
    """Predicted p99 (us), same shape as ``solo_table`` ([stage][batch][level]),
    from camelot_profile_predict (one forward launch inside the library).
    ``levels`` must be unit, 2 unit, ... ."""
    unit = levels[0]
    assert list(levels) == [unit * (i + 1) for i in range(len(levels))]
    ids = sorted(costs)
    _, _, dur, _ = cm.camelot_profile_predict(pred.h, c_costs(costs), list(batches), unit, len(levels),
                                              co_sms, co_gbs)
    # [batch][stage][level] seconds -> [stage][batch][level] us, stages in the order asked
    d = np.transpose(dur, (1, 0, 2)) * 1e6
    return d[[ids.index(int(s)) for s in stages]]


class AllocTable:
    """The allocator's per-instance table (Table 2 quantities) from p99 batch
    latencies, converted by camelot_profile_from_latency: f = B / d,
    bandwidth = bytes(B) / d, duration d."""

    def __init__(self, costs: dict, stages, batches, levels, lat_us: np.ndarray, unit: int = 8,
                 mem_bytes: float = 64e6):
        n, nb, L = len(stages), len(batches), len(levels)
        sub = {int(s): costs[int(s)] for s in stages}
        assert sorted(sub) == [int(s) for s in stages], "stages in ascending id order"
        lat_s = np.transpose(np.asarray(lat_us, np.float64), (1, 0, 2)) * 1e-6      # [nb][n][L]
        self.batches = np.ascontiguousarray(batches, np.int32)
        self.thr, self.bw, self.dur, self.mem = cm.camelot_profile_from_latency(
            c_costs(sub, mem_bytes), self.batches, lat_s)
        self.levels = list(levels)
        self.prof = cm.Profile(n, L, nb, unit, self.batches.ctypes.data, self.thr.ctypes.data,
                               self.bw.ctypes.data, self.dur.ctypes.data, self.mem.ctypes.data)

    def objective(self, alloc: cm.Alloc) -> float:
        """min_i N_i f_i(p_i) of an allocation under this table (Eq. 1)."""
        bi = int(np.where(self.batches == alloc.batch)[0][0])
        return float(min(alloc.instances[i] * self.thr[bi, i, self.levels.index(alloc.sm_quota[i])]
                         for i in range(self.thr.shape[1])))


def allocate(table: AllocTable, total_sms: int, bw_gbs: float, qos_s: float,
             policy: int = cm.POLICY_MAX_PEAK, load_qps: float = 0.0, unit: int = 8):
    cons = cm.Constraints(total_sms, total_sms // unit, bw_gbs, 1e12, qos_s, load_qps,
                          cm.SOLVER_EXHAUSTIVE, 0, 0.0, 0.0, 0)
    return cm.camelot_allocate(table.prof, policy, cons)


def study(runners: dict, costs: dict, *, n_samples: int = 20000, runs: int = 100, seed: int = 0,
          total_sms: int = 148, unit: int = 8, batches=tuple(range(1, 65)), alloc_batches=(8, 16, 32, 64),
          epochs: int = 600, lr: float = 3e-3, lr_final: float = 3e-4, co_bytes: int = 1 << 30,
          bw_gbs: float = 6500.0, qos_s: float = 20e-3, train_frac: float = 0.7, log=None) -> dict:
    """Profile, train and evaluate the predictor end to end.

    1. ``n_samples`` random (stage, batch, SM quota, co-runner quota)
       configurations, each labelled with the p99 of ``runs`` launches.
    2. The exhaustive solo table (every stage x batch x quota, no co-runner):
       the measured profiling the predictor stands in for.
    3. GPU training on ``train_frac`` of the samples; MAPE on the rest, beside
       the MAPE of looking the held-out samples up in the solo table (the
       contention-unaware method without a predictor).
    4. Eq. 1 and Eq. 3 solved on the measured table (brute force) and on the
       predicted table; the predicted choice is scored on the measured table.
    """
    stages = sorted(runners)
    levels = list(range(unit, (total_sms // unit) * unit + 1, unit))
    alloc_sms = max(levels)
    say = log or (lambda m: None)
    co = CoRunner(co_bytes)
    cfg = sample_configs(n_samples, seed, stages, list(batches), levels, total_sms, unit)
    t0 = time.time()
    data = collect(runners, cfg, runs, co, log=say)
    t_collect = time.time() - t0
    say(f"profiled {n_samples} configurations in {t_collect:.1f}s")
    t0 = time.time()
    solo = solo_table(runners, stages, list(batches), levels, runs)
    t_solo = time.time() - t0
    say(f"solo table ({solo.size} entries) in {t_solo:.1f}s")

    X = feature_rows(costs, data["stage"], data["batch"], data["sms"], data["corunner_sms"],
                     data["corunner_gbs"])
    y = np.log(data["p99_us"]).astype(np.float32)
    perm = np.random.default_rng(seed + 1).permutation(n_samples)
    ntr = int(train_frac * n_samples)
    tr, te = perm[:ntr], perm[ntr:]
    pred = LatencyPredictor(seed=seed)
    torch.cuda.synchronize()
    t0 = time.time()
    hist = pred.fit(X[tr], y[tr], epochs=epochs, lr=lr, lr_final=lr_final, seed=seed)
    t_train = time.time() - t0
    steps = epochs * ((ntr + 255) // 256)
    say(f"trained {steps} steps in {t_train:.1f}s; loss {hist[0]:.4f} -> {hist[-1]:.5f}")

    est = np.exp(pred.predict(X[te]).astype(np.float64))
    true = data["p99_us"][te]
    con = data["corunner_sms"][te] > 0
    bi = {int(b): i for i, b in enumerate(batches)}
    li = {int(q): i for i, q in enumerate(levels)}
    look = np.array([solo[stages.index(int(s)), bi[int(b)], li[int(q)]]
                     for s, b, q in zip(data["stage"][te], data["batch"][te], data["sms"][te])])
    mape_d = {"all": mape(est, true), "no_corunner": mape(est[~con], true[~con]),
              "corunner": mape(est[con], true[con])}
    for s in stages:
        m = data["stage"][te] == s
        mape_d[f"stage{s}"] = mape(est[m], true[m])
        mape_d[f"stage{s}_corunner"] = mape(est[m & con], true[m & con])

    sel = [list(batches).index(b) for b in alloc_batches]
    meas = AllocTable(costs, stages, alloc_batches, levels, solo[:, sel, :], unit)
    t0 = time.time()
    ptab = predicted_table(pred, costs, stages, alloc_batches, levels)
    t_inf = time.time() - t0
    ptable = AllocTable(costs, stages, alloc_batches, levels, ptab, unit)

    def desc(a):
        n = len(stages)
        return {"instances": list(a.instances[:n]), "sm_quota": list(a.sm_quota[:n]), "batch": a.batch}

    a_bf, o_bf = allocate(meas, alloc_sms, bw_gbs, qos_s, unit=unit)
    a_pr, o_pr = allocate(ptable, alloc_sms, bw_gbs, qos_s, unit=unit)
    max_peak = {"brute_force": desc(a_bf), "brute_force_min_thr_qps": o_bf,
                "predicted": desc(a_pr), "predicted_claim_qps": o_pr,
                "predicted_measured_qps": meas.objective(a_pr),
                "ratio_to_brute_force": meas.objective(a_pr) / o_bf}
    min_sm = []
    for frac in (0.25, 0.5, 0.75):
        load = frac * o_bf
        a_b, s_b = allocate(meas, alloc_sms, bw_gbs, qos_s, cm.POLICY_MIN_SM, load, unit)
        try:
            a_p, s_p = allocate(ptable, alloc_sms, bw_gbs, qos_s, cm.POLICY_MIN_SM, load, unit)
            got = meas.objective(a_p)
            min_sm.append({"load_qps": load, "brute_force_sms": s_b, "predicted_sms": s_p,
                           "predicted": desc(a_p), "predicted_measured_qps": got,
                           "meets_load": bool(got >= load)})
        except cm.CamelotError as e:
            min_sm.append({"load_qps": load, "brute_force_sms": s_b, "predicted_error": str(e)})
    res = {
        "samples": n_samples, "runs_per_label": runs, "train_samples": int(ntr),
        "test_samples": int(n_samples - ntr), "profiling_s": t_collect,
        "corunner_solo_gbs": {int(k): v for k, v in sorted(co._solo.items())},
        "train": {"epochs": epochs, "steps": steps, "seconds": t_train, "steps_per_s": steps / t_train,
                  "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1]},
        "mape": mape_d,
        "without_predictor": {
            "method": "solo-run profiling table (every stage x batch x quota measured alone; "
                      "contention-unaware), looked up for the held-out samples",
            "mape_corunner": mape(look[con], true[con]), "mape_no_corunner": mape(look[~con], true[~con]),
            "table_entries": int(solo.size), "profiling_s": t_solo},
        "inference": {"table_rows": int(ptab.size), "seconds": t_inf},
        "table_mape_no_corunner": mape(ptab, solo[:, sel, :]),
        "allocation": {"total_sms": alloc_sms, "levels": levels, "batches": list(alloc_batches),
                       "max_peak": max_peak, "min_sm": min_sm},
    }
    res["_predictor"] = pred
    res["_data"] = data
    res["_solo"] = solo
    return res
