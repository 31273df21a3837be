"""Host-side logic of the latency predictor (no GPU): feature rows, random
profiling configurations, the allocator table built from latencies, and the
initial parameters.  The allocator comparison is checked against a brute-force
enumeration written here."""
import itertools

import numpy as np
import pytest

from paper_2005_02088_b300 import camelot as cm, predictor as pr

COSTS = {1: pr.StageCost(1, 2 * 12288, 0.0, 12288 + 49152),
         2: pr.dense_cost(2, [12288, 512, 256, 10], 49152, 8)}


def test_dense_cost_counts_the_cfg1_mlp():
    c = COSTS[2]
    macs = 12288 * 512 + 512 * 256 + 256 * 10
    assert c.flop_per_query == 2 * macs == 12_850_176
    assert c.bytes_per_batch == 4 * macs == 25_700_352
    assert c.bytes(16) == 4 * macs + 16 * (49152 + 8)


def test_feature_rows_values():
    X = pr.feature_rows(COSTS, [2, 1], [16, 1], [32, 8], [0, 40], [999.0, 3000.0])
    assert X.shape == (2, 12) and X.dtype == np.float32
    f = dict(zip(pr.FEATURES, X[0].astype(np.float64)))
    assert f["stage"] == 2 and f["batch"] == 16 and f["sms"] == 32
    assert f["flop_per_batch"] == np.float32(16 * 12_850_176)
    assert f["bytes_per_batch"] == np.float32(25_700_352 + 16 * 49160)
    assert f["corunner_sms"] == 0 and f["corunner_gbs"] == 0 and f["corunner_active"] == 0
    assert f["sms_in_use"] == 32 and f["log2_batch"] == 4 and f["inv_sms"] == np.float32(1 / 32)
    g = dict(zip(pr.FEATURES, X[1].astype(np.float64)))
    assert g["corunner_sms"] == 40 and g["corunner_gbs"] == 3000 and g["corunner_active"] == 1
    assert g["sms_in_use"] == 48 and g["log2_batch"] == 0
    assert g["flop_per_byte"] == np.float32(2 * 12288 / (12288 + 49152))


def test_sample_configs_are_disjoint_and_seeded():
    levels = list(range(8, 145, 8))
    a = pr.sample_configs(5000, 3, [1, 2], list(range(1, 65)), levels, 148)
    b = pr.sample_configs(5000, 3, [1, 2], list(range(1, 65)), levels, 148)
    for k in a:
        assert np.array_equal(a[k], b[k])
    assert np.all(a["sms"] + a["corunner_sms"] <= 148)
    assert np.all(a["corunner_sms"] % 8 == 0)
    assert set(np.unique(a["stage"])) == {1, 2}
    assert a["batch"].min() >= 1 and a["batch"].max() <= 64
    absent = np.mean(a["corunner_sms"][a["sms"] <= 140] == 0)
    assert 0.2 < absent < 0.3
    # the largest quota leaves no room for a co-runner
    assert np.all(a["corunner_sms"][a["sms"] == 144] == 0)


def test_init_params_layout():
    th = pr.init_params(5)
    assert th.shape == (cm.PRED_PARAMS,) and th.dtype == np.float32
    b1 = th[768:832]
    b2 = th[832 + 4096:832 + 4096 + 64]
    assert not b1.any() and not b2.any() and th[-1] == 0
    assert np.abs(th[:768]).max() <= np.sqrt(6 / 12)
    assert np.array_equal(th, pr.init_params(5)) and not np.array_equal(th, pr.init_params(6))


def test_mape():
    assert pr.mape([110, 90], [100, 100]) == pytest.approx(0.1)


def _brute(thr, levels, batches, S):
    """max over (batch, N_i, p_i) of min_i N_i thr[b, i, p] s.t. sum N_i p_i <= S."""
    best = None
    for bi, _ in enumerate(batches):
        for n1, n2 in itertools.product(range(1, S // 8 + 1), repeat=2):
            for l1, l2 in itertools.product(range(len(levels)), repeat=2):
                if n1 * levels[l1] + n2 * levels[l2] > S:
                    continue
                o = min(n1 * thr[bi, 0, l1], n2 * thr[bi, 1, l2])
                if best is None or o > best + 1e-9:
                    best = o
    return best


def test_alloc_table_and_allocation_match_brute_force():
    g = np.random.default_rng(0)
    levels = [8, 16, 24, 32]
    batches = [8, 16]
    # latency falls with the quota, rises with the batch
    lat = np.empty((2, 2, 4))
    for s in range(2):
        for bi, B in enumerate(batches):
            lat[s, bi] = (50 + 30 * s) * B / 8 * (8 / np.array(levels)) ** 0.8 * g.uniform(0.9, 1.1, 4)
    t = pr.AllocTable(COSTS, [1, 2], batches, levels, lat)
    assert np.allclose(t.thr[1, 0, 2], 16 / (lat[0, 1, 2] * 1e-6))
    a, obj = pr.allocate(t, 32, 1e9, 1.0)
    assert obj == pytest.approx(t.objective(a))
    assert obj == pytest.approx(_brute(t.thr, levels, batches, 32), rel=1e-12)
    assert sum(a.instances[i] * a.sm_quota[i] for i in range(2)) <= 32
