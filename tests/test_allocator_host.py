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
