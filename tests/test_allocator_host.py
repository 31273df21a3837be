"""Host-only helpers of the batch trigger and the predictor-backed allocator
table (no GPU): the latency table the QoS trigger reads, built from a
camelot_profile, and the Table 2 conversion of predicted or measured
latencies."""
import numpy as np
import pytest

from paper_2005_02088_b300 import camelot as cm, pipelines as pl


def test_trigger_latency_from_profile():
    # host-only helper: the latency table the QoS rule reads, from a profile
    bsz = np.array([8, 16, 32], np.int32)
    n, L = 2, 4
    dur = np.zeros((3, n, L))
    for j, b in enumerate(bsz):
        for i in range(n):
            for l in range(L):
                dur[j, i, l] = (i + 1) * 1e-4 * b / (l + 1)
    z = np.zeros((3, n, L))
    mem = np.zeros((3, n))
    prof = cm.Profile(n, L, 3, 8, bsz.ctypes.data, z.ctypes.data, z.ctypes.data, dur.ctypes.data,
                      mem.ctypes.data)
    a = pl.alloc([2, 1], [16, 32], 16)
    lat = cm.camelot_trigger_latency(prof, a)
    # stage 0 at level 1 (16 SMs), stage 1 at level 3 (32 SMs): b 1e-4 / 2 + 2 b 1e-4 / 4 = b 1e-4 s
    for b in range(1, 33):
        ref = (8 if b < 8 else b) * 1e-4
        assert lat[b - 1] == round(ref * 1e9), (b, lat[b - 1], ref)
    with pytest.raises(cm.CamelotError):
        cm.camelot_trigger_latency(prof, pl.alloc([1, 1], [12, 8], 16))   # 12 SMs: not a level



def test_profile_from_latency_table2():
    costs = [(1, 24576.0, 0.0, 61440.0, 1e6), (2, 2.0e7, 2.5e7, 49160.0, 3e6)]
    bs = [8, 16]
    lat = np.array([[[1e-4, 5e-5, 4e-5], [2e-3, 1e-3, 7e-4]],
                    [[1.5e-4, 8e-5, 6e-5], [3e-3, 1.6e-3, 1.1e-3]]])
    thr, bw, dur, mem = cm.camelot_profile_from_latency(costs, bs, lat)
    for b, B in enumerate(bs):
        for i, c in enumerate(costs):
            assert mem[b, i] == c[4]
            for l in range(3):
                d = lat[b, i, l]
                assert dur[b, i, l] == d
                assert thr[b, i, l] == B / d
                assert bw[b, i, l] == (c[2] + B * c[3]) / d / 1e9
    with pytest.raises(cm.CamelotError):
        cm.camelot_profile_from_latency(costs, bs, -lat)


def test_predictor_features_rows():
    costs = [(7, 100.0, 1000.0, 10.0, 0.0)]
    X = cm.camelot_predictor_features(costs, [0, 0], [4, 1], [16, 8], [0, 24], [500.0, 700.0])
    F, Y = 400.0, 1040.0
    assert X[0].tolist() == [7, 4, 16, F, Y, np.float32(F / Y), 0, 0, 0, 16, 2, np.float32(1 / 16)]
    assert X[1].tolist() == [7, 1, 8, 100, 1010, np.float32(100 / 1010), 24, 700, 1, 32, 0, np.float32(1 / 8)]
    with pytest.raises(cm.CamelotError):
        cm.camelot_predictor_features(costs, [1], [4], [16], [0], [0.0])   # no stage index 1


def test_c_only_caller_compiles_and_links(tmp_path):
    # the C program of the predictor-backed allocation test builds against the
    # header and the library alone (it runs in the GPU tests)
    import os
    import subprocess
    from paper_2005_02088_b300 import build
    src = os.path.join(os.path.dirname(__file__), "c", "alloc_from_predictor.c")
    libdir = os.path.dirname(build.LIB)
    subprocess.run(["gcc", "-O2", "-Wall", "-Werror", "-I", os.path.join(os.path.dirname(libdir), "include"), src,
                    "-o", str(tmp_path / "a"), "-L", libdir, "-lcamelot", f"-Wl,-rpath,{libdir}"], check=True)


def _prof(dur, batches=(8, 16, 32), unit=8, bw=None):
    """A camelot_profile over dur [n_batches][n_stages][n_levels] (kept alive by the returned tuple)."""
    dur = np.ascontiguousarray(dur, np.float64)
    nb, n, L = dur.shape
    bs = np.ascontiguousarray(batches, np.int32)
    thr = np.ascontiguousarray(bs[:, None, None] / dur, np.float64)
    bw = np.ascontiguousarray(bw if bw is not None else np.full_like(dur, 100.0), np.float64)
    mem = np.zeros((nb, n), np.float64)
    prof = cm.Profile(n, L, nb, unit, bs.ctypes.data, thr.ctypes.data, bw.ctypes.data, dur.ctypes.data,
                      mem.ctypes.data)
    return prof, (bs, thr, bw, dur, mem)


def test_profile_add_handover_closed_form():
    dur = np.array([[[1e-4, 6e-5], [2e-4, 1e-4]], [[1.8e-4, 1e-4], [3.5e-4, 1.9e-4]]])
    bw0 = np.array([[[50.0, 80.0], [20.0, 40.0]], [[60.0, 90.0], [25.0, 45.0]]])
    prof, keep = _prof(dur, batches=(8, 16), bw=bw0)
    thr, bw, d = (np.empty_like(dur) for _ in range(3))
    cm.camelot_profile_add_handover(prof, [1e-5, 2e-5], thr, bw, d)
    h = np.array([1e-5, 2e-5])[None, :, None]
    assert np.array_equal(d, dur + h)
    assert np.array_equal(thr, np.array([8.0, 16.0])[:, None, None] / (dur + h))
    assert np.allclose(bw, bw0 * dur / (dur + h), rtol=1e-15)
    # a negative correction (launch overhead in the solo times) is fine while d' > 0
    cm.camelot_profile_add_handover(prof, [-5e-5, 0.0], thr, bw, d)
    assert np.array_equal(d[:, 0], dur[:, 0] - 5e-5)
    with pytest.raises(cm.CamelotError):
        cm.camelot_profile_add_handover(prof, [-1e-4, 0.0], thr, bw, d)


def test_simulate_profile_special_cases(orc):
    # two stages, 8-SM levels; stage 0: 20 us per batch of 8, stage 1: 100 us
    dur = np.zeros((3, 2, 2))
    for bi, B in enumerate((8, 16, 32)):
        dur[bi, 0] = [20e-6 * B / 8, 12e-6 * B / 8]
        dur[bi, 1] = [100e-6 * B / 8, 60e-6 * B / 8]
    prof, keep = _prof(dur)
    a = pl.alloc([1, 3], [8, 8], 8)
    # far below capacity, B = 1 would not form: a lone query waits the whole bound
    p50, p99, _ = cm.camelot_simulate_profile(prof, a, None, 1e-3, 0.5, n_queries=400, seed=3)
    lone = 1e-3 + 20e-6 + 100e-6            # durations below the smallest profiled batch: that batch's
    assert p50 == pytest.approx(lone, rel=1e-9)
    # hand-over time adds to every stage's service
    p50h, _, _ = cm.camelot_simulate_profile(prof, a, [5e-6, 7e-6], 1e-3, 0.5, n_queries=400, seed=3)
    assert p50h == pytest.approx(lone + 12e-6, rel=1e-9)
    # overload: throughput = min over stages of N_i B / d_i (Sec. 4.1)
    _, _, thr = cm.camelot_simulate_profile(prof, a, None, 1e-4, 5e7, n_queries=200000, seed=4)
    assert thr == pytest.approx(min(1 * 8 / 20e-6, 3 * 8 / 100e-6), rel=2e-3)
    # moderate load: the library's simulator agrees with the oracle's (both event-driven,
    # independent code) on p99 within sampling noise
    lam = 0.6 * min(8 / 20e-6, 3 * 8 / 100e-6)
    _, p99, _ = cm.camelot_simulate_profile(prof, a, None, 50e-6, lam, n_queries=200000, seed=5)
    arr = np.cumsum(np.random.default_rng(6).exponential(1 / lam, 200000))
    tau = [[20e-6 * b / 8 if b >= 8 else 20e-6 for b in range(1, 9)],
           [100e-6 * b / 8 if b >= 8 else 100e-6 for b in range(1, 9)]]
    done, _ = orc.simulate(arr, 8, 50e-6, [1, 3], tau)
    ref = np.quantile((done - arr)[20000:], 0.99)
    assert p99 == pytest.approx(ref, rel=0.05)
