"""Pins of the oracle's allocation policies (Eq. 1, Eq. 3): hand-solved cases,
an independent itertools brute force, the annealing solver agreeing with
exhaustive search on tiny instances, and Eq. 2's closed form."""
import itertools
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _linear_problem(S=32, unit=8, rates=(1.0, 0.5), nb=1, BW=1e9, F=1e18, qos=1e9, load=0.0,
                    I=None):
    """Per-instance throughput proportional to its SMs: f_i(p) = rate_i * p."""
    n, L = len(rates), S // unit
    p = np.arange(1, L + 1) * unit
    f = np.array([[r * p for r in rates]] * nb, np.float64)
    return dict(f=f, bw=np.zeros_like(f), d=np.zeros_like(f), mem=np.zeros((nb, n)),
                unit=unit, S=S, I=I if I is not None else S // unit, BW=BW, F=F, qos=qos,
                load=load)


def _brute(prob, policy):
    """Independent enumeration written with itertools (tie-break: objective,
    then SMs, then lexicographic (bi, N, l))."""
    f, bw, d, mem = (np.asarray(prob[k]) for k in ("f", "bw", "d", "mem"))
    nb, n, L = f.shape
    unit, S, I = prob["unit"], prob["S"], prob["I"]
    maxN = max(1, min(I, S // unit))
    best, key = None, None
    for bi in range(nb):
        for N in itertools.product(range(1, maxN + 1), repeat=n):
            for lv in itertools.product(range(L), repeat=n):
                sm = sum(N[i] * (lv[i] + 1) * unit for i in range(n))
                if sm > S or sum(N) > I:
                    continue
                if sum(N[i] * bw[bi, i, lv[i]] for i in range(n)) > prob["BW"]:
                    continue
                if sum(N[i] * mem[bi, i] for i in range(n)) > prob["F"]:
                    continue
                if sum(d[bi, i, lv[i]] for i in range(n)) > prob["qos"]:
                    continue
                if prob.get("hb") is not None and \
                        sum(N[i] * np.asarray(prob["hb"])[bi, i, lv[i]] for i in range(n)) > prob["HB"]:
                    continue
                thr = min(N[i] * f[bi, i, lv[i]] for i in range(n))
                if policy == 1 and thr < prob["load"]:
                    continue
                k = ((-thr, sm) if policy == 0 else (sm, -thr)) + (bi,) + N + lv
                if key is None or k < key:
                    key, best = k, dict(bi=bi, N=list(N), l=list(lv), thr=thr, sms=sm)
    return best


def test_hand_solved_max_peak(orc):
    # f1(p) = p, f2(p) = p/2 on 32 SMs: the best min-throughput is 8 qps, reached
    # with 24 SMs as (1 x 8 SMs, 1 x 16 SMs); the tie (1 x 8, 2 x 8) loses on the
    # lexicographic rule (N2 = 1 < 2).
    r = orc.allocate(_linear_problem(), 0)
    assert r == dict(bi=0, N=[1, 1], l=[0, 1], p=[8, 16], thr=8.0, sms=24)


def test_hand_solved_min_sm(orc):
    # load 12 qps: stage 1 needs 16 SMs, stage 2 needs 24 SMs.
    r = orc.allocate(_linear_problem(S=64, load=12.0), 1)
    assert r["sms"] == 40 and r["thr"] >= 12.0
    assert r == _brute(_linear_problem(S=64, load=12.0), 1) | {"p": r["p"]}


def test_bandwidth_constraint_binds(orc):
    # Without the bandwidth constraint (Constraint-3) both stages take 32 SMs;
    # a demand of 10 GB/s per quota level caps the total at 40 GB/s.
    prob = _linear_problem(S=64, rates=(1.0, 1.0))
    L = prob["f"].shape[2]
    prob["bw"] = np.array([[[10.0 * (l + 1) for l in range(L)]] * 2])
    free = orc.allocate(dict(prob, BW=1e9), 0)
    capped = orc.allocate(dict(prob, BW=40.0), 0)
    assert free["thr"] == 32.0
    assert capped["thr"] < free["thr"]
    assert capped == _brute(dict(prob, BW=40.0), 0) | {"p": capped["p"]}


def test_host_link_constraint_binds(orc):
    # Stage 1 reads host memory: 2 GB/s of host-link demand per quota level.
    # A 6 GB/s link caps it at 24 SMs in total, which caps the min-throughput
    # at 24 (it was 32 with the link unconstrained); stage 2 is unaffected.
    prob = _linear_problem(S=64, rates=(1.0, 1.0))
    L = prob["f"].shape[2]
    hb = np.zeros_like(prob["f"])
    hb[0, 0, :] = [2.0 * (l + 1) for l in range(L)]
    free = orc.allocate(prob, 0)
    capped = orc.allocate(dict(prob, hb=hb, HB=6.0), 0)
    assert free["thr"] == 32.0 and capped["thr"] == 24.0
    assert capped["N"][0] * hb[0, 0, capped["l"][0]] <= 6.0
    assert capped == _brute(dict(prob, hb=hb, HB=6.0), 0) | {"p": capped["p"]}
    # a budget that covers every allocation changes nothing
    assert orc.allocate(dict(prob, hb=hb, HB=1e9), 0) == free


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("policy", [0, 1])
def test_host_link_exhaustive_equals_brute_force(orc, seed, policy):
    g = np.random.default_rng(300 + seed)
    S = [16, 32, 64][seed % 3]
    prob = _random_problem(g, S, n=2 + seed % 2, nb=1 + seed % 2)
    prob["hb"] = g.integers(0, 6, size=prob["f"].shape).astype(np.float64)
    prob["HB"] = float(g.integers(4, 20))
    r = orc.allocate(prob, policy)
    b = _brute(prob, policy)
    if b is None:
        assert r is None
    else:
        r.pop("p")
        assert r == b


def test_infeasible_returns_none(orc):
    assert orc.allocate(_linear_problem(qos=-1.0), 0) is None
    assert orc.allocate(_linear_problem(load=1e9), 1) is None


def _random_problem(g, S, n, nb):
    unit = 8
    L = S // unit
    f = g.integers(1, 20, size=(nb, n, L)).astype(np.float64)
    f = np.sort(f, axis=2)                       # more SMs never slower
    bw = g.integers(0, 10, size=(nb, n, L)).astype(np.float64)
    d = g.integers(1, 10, size=(nb, n, L)).astype(np.float64)
    d = -np.sort(-d, axis=2)
    mem = g.integers(1, 5, size=(nb, n)).astype(np.float64)
    return dict(f=f, bw=bw, d=d, mem=mem, unit=unit, S=S, I=int(g.integers(2, 6)),
                BW=float(g.integers(10, 40)), F=float(g.integers(4, 20)),
                qos=float(g.integers(8, 25)), load=float(g.integers(5, 30)))


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("policy", [0, 1])
def test_exhaustive_equals_independent_brute_force(orc, seed, policy):
    g = np.random.default_rng(100 + seed)
    S = [16, 32, 64][seed % 3]
    prob = _random_problem(g, S, n=2 + seed % 2, nb=1 + seed % 2)
    r = orc.allocate(prob, policy)
    b = _brute(prob, policy)
    if b is None:
        assert r is None
    else:
        r.pop("p")
        assert r == b


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("policy", [0, 1])
def test_anneal_equals_exhaustive_on_tiny(orc, seed, policy):
    g = np.random.default_rng(200 + seed)
    S = [16, 32, 64][seed % 3]
    prob = _random_problem(g, S, n=2 + seed % 2, nb=1)
    ex = orc.allocate(prob, policy)
    sa = orc.allocate(prob, policy, solver="anneal", iters=5000, seed=seed)
    if ex is None:
        assert sa is None
    else:
        assert sa is not None
        assert (sa["thr"], sa["sms"]) == (ex["thr"], ex["sms"])


def test_eq2_min_gpus_closed_form(orc):
    # y = max(sum C / G, sum M / F), whole GPUs
    assert orc.min_gpus([100, 200], [10, 20], 150, 100) == 2
    assert orc.min_gpus([10, 20], [60, 70], 1000, 100) == 2
    assert orc.min_gpus([1], [1], 10, 10) == 1


def test_golden_alloc_cases(orc):
    cases = json.load(open(os.path.join(GOLD, "alloc_cases.json")))["cases"]
    for c in cases:
        prob = {k: (np.array(v, np.float64) if isinstance(v, list) else v)
                for k, v in c["problem"].items()}
        r = orc.allocate(prob, c["policy"])
        assert r is not None, c["name"]
        for k, v in c["expect"].items():
            assert r[k] == v, (c["name"], k, r[k], v)
