"""The allocation-free stage launch (camelot_stage_launch_noalloc).

For callers that cannot allocate device memory when they run a stage (an
application whose memory manager owns the device pool, a serving loop that
cannot pay cudaMalloc's latency and synchronisation mid-request, a plug-in
handed only its buffers), the library keeps the stage's scratch in a static
16 MiB device array.  These tests run stages through that entry point several
times in a row, with different inputs so that stale scratch contents would
show, and check the results against the ordinary entry point (caller-provided
scratch): bit for bit, and for the FP32 MLP also against the FP64 oracle
bound.  Outputs start as NaN or -7 so that a call that did not run cannot
pass.  The file is collected last.
"""
import numpy as np
import pytest
import torch

from gpu_common import cfg1_data, chain_bound

pytestmark = pytest.mark.gpu


def _outs(n, k, width):
    return [torch.full((n, k), -7, dtype=torch.int32, device="cuda"),
            torch.full((n, k), np.nan, dtype=torch.float32, device="cuda"),
            torch.full((n, width), np.nan, dtype=torch.float32, device="cuda")]


def _run_ref(cm, st, y, n, n_ctas):
    _, _, sb = cm.camelot_stage_info(st, n)
    scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
    out = _outs(n, 1, 10)
    cm.camelot_stage_launch(st, n_ctas, y, n, None, out[0], out[1], out[2], scr, sb, None)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


def _run_noalloc(cm, st, y, n, n_ctas):
    out = _outs(n, 1, 10)
    cm.camelot_stage_launch_noalloc(st, n_ctas, y, n, None, out[0], out[1], out[2], None)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


def test_noalloc_matches_caller_scratch_twice(orc):
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    x, ws = cfg1_data(256)
    wd = [torch.from_numpy(w).cuda() for w in ws]
    st = pl.stage_dense(cm.STAGE_MLP_FP32, wd, [1, 1, 0], top_k=1, max_batch=64)
    try:
        # (first query, batch, SMs): two calls in a row, then the largest batch on one SM
        calls = [(0, 16, 24), (100, 11, 37), (150, 64, 1)]
        for q0, n, n_ctas in calls:
            xs = x[q0:q0 + n]
            y = torch.from_numpy(((xs.reshape(n, -1).astype(np.float32) - 127.5) / 64)).cuda()
            got = _run_noalloc(cm, st, y, n, n_ctas)
            ref = _run_ref(cm, st, y, n, n_ctas)
            assert np.all(got[0] >= 0) and np.all(np.isfinite(got[2]))
            for a, b in zip(got, ref):
                assert np.array_equal(a, b)
            z64, bound = chain_bound(orc, xs, ws, [1, 1, 0])
            assert np.all(np.abs(got[2] - z64) <= bound + 1e-30)
    finally:
        cm.camelot_stage_release(st)


def test_noalloc_normalize_stage_bit_exact():
    # a stage whose scratch layout is fixed by its max_batch, not by n
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    x, _ = cfg1_data(256)
    st = pl.stage_normalize(64, 64, 3, max_batch=32)
    try:
        for q0, n, n_ctas in ((0, 32, 8), (40, 7, 3)):
            xin = torch.from_numpy(np.ascontiguousarray(x[q0:q0 + n].reshape(n, -1))).cuda()
            got = torch.full((n, 12288), np.nan, dtype=torch.float32, device="cuda")
            cm.camelot_stage_launch_noalloc(st, n_ctas, xin, n, got, None, None, None, None)
            _, _, sb = cm.camelot_stage_info(st, n)
            scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
            ref = torch.full((n, 12288), np.nan, dtype=torch.float32, device="cuda")
            cm.camelot_stage_launch(st, n_ctas, xin, n, ref, None, None, None, scr, sb, None)
            torch.cuda.synchronize()
            g = got.cpu().numpy()
            assert np.array_equal(g.view(np.uint32), ref.cpu().numpy().view(np.uint32))
            assert np.array_equal(g, (x[q0:q0 + n].reshape(n, -1).astype(np.float32) - 127.5) / 64)
    finally:
        cm.camelot_stage_release(st)


def test_noalloc_refuses_batches_beyond_the_static_buffer():
    # a 256 -> 65536 layer needs about 0.5 MiB of scratch per query: 64 queries
    # exceed the 16 MiB buffer and are refused before anything runs; 4 fit and
    # give what the ordinary launch gives
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    g = np.random.default_rng(11)
    w = torch.from_numpy((g.standard_normal((65536, 256)) / 16).astype(np.float32)).cuda()
    st = pl.stage_dense(cm.STAGE_MLP_FP32, [w], [0], top_k=0, max_batch=64)
    try:
        y = torch.from_numpy(g.standard_normal((64, 256)).astype(np.float32)).cuda()
        out = torch.full((64, 65536), np.nan, dtype=torch.float32, device="cuda")
        with pytest.raises(cm.CamelotError) as e:
            cm.camelot_stage_launch_noalloc(st, 8, y, 64, out, None, None, None, None)
        assert e.value.status == cm.EINVAL
        cm.camelot_stage_launch_noalloc(st, 8, y, 4, out, None, None, None, None)
        _, _, sb = cm.camelot_stage_info(st, 4)
        scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
        ref = torch.full((4, 65536), np.nan, dtype=torch.float32, device="cuda")
        cm.camelot_stage_launch(st, 8, y, 4, ref, None, None, None, scr, sb, None)
        torch.cuda.synchronize()
        got = out[:4].cpu().numpy()
        assert np.all(np.isfinite(got)) and float(np.abs(got).sum()) > 0
        assert np.array_equal(got.view(np.uint32), ref.cpu().numpy().view(np.uint32))
        assert bool(torch.isnan(out[4:]).all())          # rows past the batch untouched
    finally:
        cm.camelot_stage_release(st)


def test_noalloc_refuses_tensor_core_stages():
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    w = torch.zeros((128, 128), dtype=torch.bfloat16, device="cuda")
    st = pl.stage_dense(cm.STAGE_GEMM_BF16, [w], [0], top_k=0, max_batch=32)
    try:
        y = torch.zeros((4, 128), dtype=torch.bfloat16, device="cuda")
        out = torch.zeros((4, 128), dtype=torch.bfloat16, device="cuda")
        with pytest.raises(cm.CamelotError) as e:
            cm.camelot_stage_launch_noalloc(st, 2, y, 4, out, None, None, None, None)
        assert e.value.status == cm.EINVAL
    finally:
        cm.camelot_stage_release(st)
