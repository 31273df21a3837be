"""The allocation-free stage launch (camelot_stage_launch_noalloc).

For callers that cannot allocate device memory when they run a stage (an
application whose memory manager owns the device pool, a serving loop that
cannot pay cudaMalloc's latency and synchronisation mid-request, a plug-in
handed only its buffers), the library keeps the stage's scratch in a static
16 MiB device array.  This test runs the FP32 MLP stage of the plain 2-stage
pipeline through that entry point twice in a row, with different inputs so
stale scratch contents would show, and checks both results against the
ordinary entry point (caller-provided scratch) and the FP64 oracle bound.
It lives in a file of its own that pytest collects last.
"""
import numpy as np
import pytest
import torch

from gpu_common import cfg1_data, chain_bound

pytestmark = pytest.mark.gpu


def _run_ref(cm, st, y, n, n_ctas):
    _, _, sb = cm.camelot_stage_info(st, n)
    scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
    out = [torch.empty((n, 1), dtype=torch.int32, device="cuda"),
           torch.empty((n, 1), dtype=torch.float32, device="cuda"),
           torch.empty((n, 10), dtype=torch.float32, device="cuda")]
    cm.camelot_stage_launch(st, n_ctas, y, n, None, out[0], out[1], out[2], scr, sb, None)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


def _run_noalloc(cm, st, y, n, n_ctas):
    out = [torch.full((n, 1), -7, dtype=torch.int32, device="cuda"),
           torch.full((n, 1), np.nan, dtype=torch.float32, device="cuda"),
           torch.full((n, 10), np.nan, dtype=torch.float32, device="cuda")]
    cm.camelot_stage_launch_noalloc(st, n_ctas, y, n, None, out[0], out[1], out[2], None)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


def test_noalloc_matches_caller_scratch_twice(orc):
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    x, ws = cfg1_data(256)
    wd = [torch.from_numpy(w).cuda() for w in ws]
    st = pl.stage_dense(cm.STAGE_MLP_FP32, wd, [1, 1, 0], top_k=1, max_batch=64)
    try:
        calls = [(0, 16, 24), (100, 11, 37)]          # (first query, batch, SMs)
        for q0, n, n_ctas in calls:
            xs = x[q0:q0 + n]
            y = torch.from_numpy(((xs.reshape(n, -1).astype(np.float32) - 127.5) / 64)).cuda()
            got = _run_noalloc(cm, st, y, n, n_ctas)
            ref = _run_ref(cm, st, y, n, n_ctas)
            for a, b in zip(got, ref):
                assert np.array_equal(a, b)
            z64, bound = chain_bound(orc, xs, ws, [1, 1, 0])
            assert np.all(np.abs(got[2] - z64) <= bound + 1e-30)
    finally:
        cm.camelot_stage_release(st)


def test_noalloc_refuses_batches_beyond_the_static_buffer():
    # a 256 -> 65536 layer needs about 0.5 MiB of scratch per query: 64 queries
    # exceed the 16 MiB buffer and are refused before anything runs
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    w = torch.zeros((65536, 256), dtype=torch.float32, device="cuda")
    st = pl.stage_dense(cm.STAGE_MLP_FP32, [w], [0], top_k=0, max_batch=64)
    try:
        y = torch.zeros((64, 256), dtype=torch.float32, device="cuda")
        out = torch.zeros((64, 65536), dtype=torch.float32, device="cuda")
        with pytest.raises(cm.CamelotError) as e:
            cm.camelot_stage_launch_noalloc(st, 8, y, 64, out, None, None, None, None)
        assert e.value.status == cm.EINVAL
        cm.camelot_stage_launch_noalloc(st, 8, y, 4, out, None, None, None, None)   # small: runs
        torch.cuda.synchronize()
        assert float(out[:4].abs().sum()) == 0.0
    finally:
        cm.camelot_stage_release(st)
