"""Pins of the oracle's event-driven pipeline simulator: queueing closed forms
(M/M/1, M/D/1, M/M/2), hand-derived timelines of the batch trigger and of the
bounded inter-stage buffers, and the min-over-stages throughput of a saturated
deterministic pipeline (Sec. 4.1: the slowest stage sets the peak)."""
import math

import numpy as np
import pytest


def _poisson(rate, n, seed):
    g = np.random.default_rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, n))
    return t


def test_mm1_sojourn(orc):
    lam, mu, n = 0.5, 1.0, 200_000
    arr = _poisson(lam, n, 11)
    mult = np.random.default_rng(12).exponential(1.0, size=(1, n))
    done, bs = orc.simulate(arr, 1, 0.0, [1], [[1.0 / mu]], mult=mult)
    soj = (done - arr)[n // 10:]
    assert np.all(bs == 1)
    assert abs(soj.mean() - 1 / (mu - lam)) / (1 / (mu - lam)) < 0.04
    p99 = math.log(100) / (mu - lam)                  # sojourn ~ Exp(mu - lam)
    assert abs(np.quantile(soj, 0.99) - p99) / p99 < 0.06


def test_md1_mean_wait(orc):
    lam, mu, n = 0.7, 1.0, 200_000
    arr = _poisson(lam, n, 13)
    done, _ = orc.simulate(arr, 1, 0.0, [1], [[1.0 / mu]])
    soj = (done - arr)[n // 10:]
    rho = lam / mu
    ref = rho / (2 * mu * (1 - rho)) + 1 / mu         # Pollaczek-Khinchine + service
    assert abs(soj.mean() - ref) / ref < 0.04


def test_mm2_erlang_c(orc):
    lam, mu, c, n = 1.5, 1.0, 2, 200_000
    arr = _poisson(lam, n, 14)
    mult = np.random.default_rng(15).exponential(1.0, size=(1, n))
    done, _ = orc.simulate(arr, 1, 0.0, [c], [[1.0 / mu]], mult=mult)
    soj = (done - arr)[n // 10:]
    a = lam / mu
    rho = a / c
    s = sum(a ** k / math.factorial(k) for k in range(c))
    pc = (a ** c / math.factorial(c)) / (1 - rho)
    erlang_c = pc / (s + pc)
    ref = erlang_c / (c * mu - lam) + 1 / mu
    assert abs(soj.mean() - ref) / ref < 0.05


def test_batch_trigger_timeline(orc):
    # B = 4, wait bound 1.0: three queries at 0, 0.1, 0.2 form a partial batch at
    # t = 1.0 (oldest + wait); the next four arrive together and go at once.
    arr = np.array([0.0, 0.1, 0.2, 5.0, 5.0, 5.0, 5.0])
    tau = [[0.5, 0.6, 0.7, 0.8]]
    done, bs = orc.simulate(arr, 4, 1.0, [1], tau)
    assert bs.tolist() == [3, 4]
    assert done.tolist() == [1.7, 1.7, 1.7, 5.8, 5.8, 5.8, 5.8]


def test_full_batch_issued_immediately(orc):
    arr = np.array([0.0, 0.0, 0.3, 0.4, 0.4])
    done, bs = orc.simulate(arr, 2, 10.0, [1], [[1.0, 2.0]])
    # batch {0,1} at 0 (done 2); {2,3} is full at 0.4 but the instance is busy
    # until 2 -> done 4; query 4 waits for its wait bound (10.4) -> done 11.4.
    assert bs.tolist() == [2, 2, 1]
    assert done.tolist() == [2.0, 2.0, 4.0, 4.0, 11.4]


@pytest.mark.parametrize("cap,period", [(1, 4.0), (2, 3.0)])
def test_bounded_buffer_backpressure(orc, cap, period):
    # stage 0 takes 1, stage 1 takes 3; a slot is held from the producer's start
    # to the consumer's finish.  cap=1 serialises the stages (period 1+3); cap=2
    # lets them overlap (period = slowest stage = 3).
    arr = np.zeros(6)
    done, _ = orc.simulate(arr, 1, 0.0, [1, 1], [[1.0], [3.0]], caps=[cap, 1])
    gaps = np.diff(done)
    assert done[0] == 4.0
    assert np.all(gaps == period)


@pytest.mark.parametrize("inst,tau,B", [([1, 2], [2.0, 3.0], 4), ([3, 1, 2], [1.0, 0.2, 0.9], 2),
                                        ([2, 2], [0.25, 0.25], 8)])
def test_saturated_throughput_is_min_over_stages(orc, inst, tau, B):
    n = 4000
    arr = np.zeros(n)
    tt = [[t * (b + 1) / B for b in range(B)] for t in tau]   # full batch costs tau
    done, _ = orc.simulate(arr, B, 0.0, inst, tt)
    thr = (n // 2) / (done[-1] - done[n // 2 - 1])
    ref = min(i * B / t for i, t in zip(inst, tau))
    assert abs(thr - ref) / ref < 1e-3


def test_exactly_once_in_order_single_instance(orc):
    arr = np.sort(np.random.default_rng(5).uniform(0, 50, 500))
    done, bs = orc.simulate(arr, 8, 0.3, [1, 1], [[0.1] * 8, [0.2] * 8], caps=[2, 1])
    assert bs.sum() == arr.size
    assert np.all(np.isfinite(done)) and np.all(done >= arr)
    assert np.all(np.diff(done) >= 0)


ARR_QOS = np.array([0.0, 0.75, 1.25, 100.0, 100.125, 100.25, 100.375, 200.0, 300.0, 302.25])
LAT = [0.5, 1.0, 1.5, 2.0]          # predicted latency of a batch of 1..4


def test_qos_trigger_timeline(orc):
    # Sec. 5.2 step 2 with a latency prediction: budget 3 (QoS less margin), so
    # k waiting queries may wait 3 - LAT[k-1] = 2.5, 2.0, 1.5, 1.0.  Queries at
    # 0, 0.75, 1.25: three wait at 1.25 and their bound 1.5 is not yet reached,
    # so they leave at 1.5.  Four at 100..100.375 fill the batch.  A lone query
    # at 200 leaves at 202.5.  At 302.25 a second query joins one that has
    # waited 2.25 > 2.0: the pair leaves at once.
    done, bs, iss = orc.simulate_qos(ARR_QOS, 4, 10.0, 3.0, LAT, [1], [[0.0625] * 4])
    assert bs.tolist() == [3, 4, 1, 2]
    assert iss.tolist() == [1.5, 100.375, 202.5, 302.25]
    assert done.tolist() == [1.5625] * 3 + [100.4375] * 4 + [202.5625] + [302.3125] * 2


def test_qos_trigger_capped_by_wait_bound(orc):
    # the same arrivals with a fixed wait bound of 1.125 below every QoS bound but
    # the last: the pair at 0 / 0.75 leaves at 1.125, the query at 1.25 at 2.375
    done, bs, iss = orc.simulate_qos(ARR_QOS, 4, 1.125, 3.0, LAT, [1], [[0.0625] * 4])
    assert bs.tolist() == [2, 1, 4, 1, 1, 1]
    assert iss.tolist() == [1.125, 2.375, 100.375, 201.125, 301.125, 303.375]


def test_qos_trigger_budget_spent_issues_on_arrival(orc):
    # predicted latency above the budget: no query may wait, each leaves on arrival
    arr = np.array([0.0, 0.5, 0.75])
    done, bs, iss = orc.simulate_qos(arr, 4, 10.0, 1.0, [2.0, 2.0, 2.0, 2.0], [1], [[0.125] * 4])
    assert bs.tolist() == [1, 1, 1]
    assert iss.tolist() == [0.0, 0.5, 0.75]


def test_qos_trigger_reduces_to_plain_rule(orc):
    # zero predicted latency and a budget above the wait bound: the plain trigger
    arr = np.sort(np.random.default_rng(9).uniform(0, 20, 300))
    d1, b1 = orc.simulate(arr, 8, 0.3, [1, 2], [[0.05] * 8, [0.2] * 8], caps=[4, 1])
    d2, b2, _ = orc.simulate_qos(arr, 8, 0.3, 5.0, [0.0] * 8, [1, 2], [[0.05] * 8, [0.2] * 8], caps=[4, 1])
    assert np.array_equal(b1, b2) and np.array_equal(d1, d2)
