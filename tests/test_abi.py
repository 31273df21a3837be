"""CPU checks of the C-ABI library: it loads without a GPU, exports every
function include/camelot.h declares, and its host-only allocator (Eq. 1 /
Eq. 3) chooses what the oracle's exhaustive search chooses."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2005_02088_b300 import camelot as cm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "camelot.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(camelot_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = C.CDLL(cm.lib_path())
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(cm._SIGS), "binding and header disagree"


def test_version_and_defaults():
    assert cm.camelot_version() >= 100
    o = cm.camelot_options_default()
    assert o.query_slots == 65536 and o.batch_slots >= 2 and o.idle_exit_ns > 0


def _profile(prob, batch_sizes=None):
    f = np.ascontiguousarray(prob["f"], np.float64)
    nb, n, L = f.shape
    keep = [np.ascontiguousarray(prob[k], np.float64) for k in ("bw", "d", "mem")]
    bs = np.ascontiguousarray(batch_sizes or list(range(1, nb + 1)), np.int32)
    pr = cm.Profile(n, L, nb, prob["unit"], bs.ctypes.data, f.ctypes.data, keep[0].ctypes.data,
                    keep[1].ctypes.data, keep[2].ctypes.data)
    return pr, (f, bs, *keep)


def _cons(prob, solver=cm.SOLVER_EXHAUSTIVE, seed=0):
    return cm.Constraints(prob["S"], prob["I"], prob["BW"], prob["F"], prob["qos"],
                          prob.get("load", 0.0), solver, 0, 0.0, 0.0, seed)


def _random_problem(g, S, n, nb):
    unit = 8
    L = S // unit
    f = np.sort(g.integers(1, 40, size=(nb, n, L)).astype(np.float64), axis=2)
    bw = g.integers(0, 10, size=(nb, n, L)).astype(np.float64)
    d = -np.sort(-g.integers(1, 10, size=(nb, n, L)).astype(np.float64), axis=2)
    mem = g.integers(1, 5, size=(nb, n)).astype(np.float64)
    return dict(f=f, bw=bw, d=d, mem=mem, unit=unit, S=S, I=int(g.integers(2, 9)),
                BW=float(g.integers(10, 60)), F=float(g.integers(4, 30)),
                qos=float(g.integers(8, 30)), load=float(g.integers(5, 60)))


@pytest.mark.parametrize("seed", range(20))
@pytest.mark.parametrize("policy", [0, 1])
def test_allocate_matches_oracle_exhaustive(orc, seed, policy):
    g = np.random.default_rng(1000 + seed)
    S = [16, 32, 64, 96, 148][seed % 5]
    prob = _random_problem(g, S, n=2 + seed % 3, nb=1 + seed % 2)
    ref = orc.allocate(prob, policy)
    pr, keep = _profile(prob)
    if ref is None:
        with pytest.raises(cm.CamelotError) as e:
            cm.camelot_allocate(pr, policy, _cons(prob))
        assert e.value.status == cm.EINFEASIBLE
        return
    a, obj = cm.camelot_allocate(pr, policy, _cons(prob))
    n = prob["f"].shape[1]
    assert [a.instances[i] for i in range(n)] == ref["N"]
    assert [a.sm_quota[i] for i in range(n)] == ref["p"]
    assert a.batch == ref["bi"] + 1
    assert obj == (ref["thr"] if policy == 0 else ref["sms"])


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("policy", [0, 1])
def test_allocate_host_link_matches_oracle(orc, seed, policy):
    # the host-link budget (profile host_gbs, constraints host_gbs) against the
    # oracle's exhaustive search with the same constraint
    g = np.random.default_rng(4000 + seed)
    prob = _random_problem(g, [16, 32, 64, 96][seed % 4], n=2 + seed % 2, nb=1 + seed % 2)
    prob["hb"] = g.integers(0, 8, size=prob["f"].shape).astype(np.float64)
    prob["HB"] = float(g.integers(4, 24))
    ref = orc.allocate(prob, policy)
    pr, keep = _profile(prob)
    hb = np.ascontiguousarray(prob["hb"], np.float64)
    pr.host_gbs = hb.ctypes.data
    cons = _cons(prob)
    cons.host_gbs = prob["HB"]
    if ref is None:
        with pytest.raises(cm.CamelotError) as e:
            cm.camelot_allocate(pr, policy, cons)
        assert e.value.status == cm.EINFEASIBLE
        return
    a, obj = cm.camelot_allocate(pr, policy, cons)
    n = prob["f"].shape[1]
    assert [a.instances[i] for i in range(n)] == ref["N"]
    assert [a.sm_quota[i] for i in range(n)] == ref["p"]
    assert obj == (ref["thr"] if policy == 0 else ref["sms"])
    # without the budget the host demand is ignored
    a0, obj0 = (None, None)
    cons.host_gbs = 0.0
    ref0 = orc.allocate({k: v for k, v in prob.items() if k not in ("hb", "HB")}, policy)
    if ref0 is not None:
        a0, obj0 = cm.camelot_allocate(pr, policy, cons)
        assert obj0 == (ref0["thr"] if policy == 0 else ref0["sms"])


@pytest.mark.parametrize("seed", range(10))
def test_allocate_anneal_reaches_optimum_without_tight_budgets(orc, seed):
    # bandwidth and memory budgets loose: the one-step moves of the annealer
    # connect the whole feasible region, and it finds the exhaustive optimum
    g = np.random.default_rng(2000 + seed)
    prob = _random_problem(g, [16, 32, 64][seed % 3], n=2, nb=1)
    prob.update(BW=1e9, F=1e9, qos=1e9)
    ref = orc.allocate(prob, 0)
    pr, keep = _profile(prob)
    a, obj = cm.camelot_allocate(pr, 0, _cons(prob, cm.SOLVER_ANNEAL, seed))
    assert obj == ref["thr"]


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("policy", [0, 1])
def test_allocate_anneal_feasible_and_never_beats_optimum(orc, seed, policy):
    # with tight budgets the feasible region can be cut into pieces that
    # single-step moves cannot cross, so the heuristic may stop short
    g = np.random.default_rng(3000 + seed)
    prob = _random_problem(g, [16, 32, 64][seed % 3], n=2 + seed % 2, nb=1)
    ref = orc.allocate(prob, policy)
    pr, keep = _profile(prob)
    try:
        a, obj = cm.camelot_allocate(pr, policy, _cons(prob, cm.SOLVER_ANNEAL, seed))
    except cm.CamelotError as e:
        assert e.status == cm.EINFEASIBLE
        return
    assert ref is not None
    n = prob["f"].shape[1]
    N = [a.instances[i] for i in range(n)]
    lv = [a.sm_quota[i] // 8 - 1 for i in range(n)]
    assert sum(N[i] * a.sm_quota[i] for i in range(n)) <= prob["S"] and sum(N) <= prob["I"]
    assert sum(N[i] * prob["bw"][0, i, lv[i]] for i in range(n)) <= prob["BW"]
    assert sum(prob["d"][0, i, lv[i]] for i in range(n)) <= prob["qos"]
    if policy == 0:
        assert obj <= ref["thr"]
    else:
        assert obj >= ref["sms"]


def test_allocate_golden_cases(orc):
    import json
    cases = json.load(open(os.path.join(ROOT, "tests", "golden", "alloc_cases.json")))["cases"]
    for c in cases:
        prob = {k: (np.array(v, np.float64) if isinstance(v, list) else v)
                for k, v in c["problem"].items()}
        pr, keep = _profile(prob)
        a, obj = cm.camelot_allocate(pr, c["policy"], _cons(prob))
        n = prob["f"].shape[1]
        assert [a.instances[i] for i in range(n)] == c["expect"]["N"], c["name"]
        assert [a.sm_quota[i] // 8 - 1 for i in range(n)] == c["expect"]["l"], c["name"]


def test_allocate_full_gpu_size_is_fast():
    # 3 stages on 148 SMs in 8-SM steps: exhaustive search stays well under the
    # paper's 5 ms annealing budget per decision (Sec. 8.7) times a few.
    import time
    g = np.random.default_rng(7)
    L = 18
    f = np.sort(g.uniform(100, 5000, size=(1, 3, L)), axis=2)
    prob = dict(f=f, bw=np.zeros_like(f), d=np.full_like(f, 1e-3), mem=np.ones((1, 3)),
                unit=8, S=148, I=18, BW=1e9, F=1e18, qos=0.02)
    pr, keep = _profile(prob)
    t = time.perf_counter()
    a, obj = cm.camelot_allocate(pr, 0, _cons(prob))
    dt = time.perf_counter() - t
    assert obj > 0 and dt < 0.5
    assert sum(a.instances[i] * a.sm_quota[i] for i in range(3)) <= 148


def test_allocate_rejects_bad_input():
    prob = dict(f=-np.ones((1, 2, 2)), bw=np.zeros((1, 2, 2)), d=np.zeros((1, 2, 2)),
                mem=np.zeros((1, 2)), unit=8, S=16, I=2, BW=1, F=1, qos=1)
    pr, keep = _profile(prob)
    with pytest.raises(cm.CamelotError) as e:
        cm.camelot_allocate(pr, 0, _cons(prob))
    assert e.value.status == cm.EINVAL


def test_stage_prepare_rejects_bad_ring_slots():
    """ring_slots is checked before any device work: 1, 6 and any value on a
    kind without a bulk-copy ring are EINVAL (no GPU needed)."""
    import ctypes
    for kind, slots in ((cm.STAGE_GEMM_BF16, 1), (cm.STAGE_GEMM_BF16, 6), (cm.STAGE_GEMM_FP8, -1),
                        (cm.STAGE_MLP_FP32, 3), (cm.STAGE_NORMALIZE_U8, 2)):
        d = cm.StageDesc()
        d.kind, d.max_batch, d.ring_slots = kind, 16, slots
        st = ctypes.c_void_p()
        assert cm.load().camelot_stage_prepare(ctypes.byref(d), ctypes.byref(st)) == cm.EINVAL
        assert b"ring_slots" in cm.load().camelot_last_error()
        assert st.value is None
