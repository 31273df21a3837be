"""GPU parity of the artifact stages (the c_i, m_i, p_i of Sec. 2.3 and Sec.
8.5): the compute stage and the stream stage over a device table and over a
pinned host table, as direct launches at several CTA counts and as a 3-stage
pipeline through both handoffs.  Both stages are defined in binary32, so every
value must equal the oracle's bit for bit."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _launch(cm, st, ctas, x, out_w, top_k=0):
    n = x.shape[0]
    _, _, sb = cm.camelot_stage_info(st, n)
    scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
    if top_k:
        idx = torch.empty((n, top_k), dtype=torch.int32, device="cuda")
        val = torch.empty((n, top_k), dtype=torch.float32, device="cuda")
        lg = torch.empty((n, out_w), dtype=torch.float32, device="cuda")
        cm.camelot_stage_launch(st, ctas, x, n, None, idx, val, lg, scr, sb, None)
        torch.cuda.synchronize()
        return lg.cpu().numpy(), idx.cpu().numpy(), val.cpu().numpy()
    out = torch.empty((n, out_w), dtype=torch.float32, device="cuda")
    cm.camelot_stage_launch(st, ctas, x, n, out, None, None, None, scr, sb, None)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("steps", [0, 1, 37, 300])
def test_compute_synth_bit_exact(orc, steps):
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    g = np.random.default_rng(steps)
    x = g.standard_normal((7, 1028)).astype(np.float32)
    st = pl.stage_compute_synth(1028, steps, 0, 16)
    try:
        xd = torch.from_numpy(x).cuda()
        ref = orc.compute_synth(x, steps)
        for ctas in (1, 5, 16):
            assert np.array_equal(_launch(cm, st, ctas, xd, 1028), ref), ctas
    finally:
        cm.camelot_stage_release(st)


@pytest.mark.parametrize("where", ["device", "host"])
def test_stream_synth_bit_exact(orc, where):
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    W, R, L = 256, 256 * 9, 256 * 1000
    g = np.random.default_rng(5)
    x = g.standard_normal((11, W)).astype(np.float32)
    T = g.standard_normal(L).astype(np.float32)
    table = torch.from_numpy(T).cuda() if where == "device" else torch.from_numpy(T).pin_memory()
    st = pl.stage_stream_synth(W, R, table, 0, 16)
    stf = pl.stage_stream_synth(W, R, table, 5, 16)
    try:
        xd = torch.from_numpy(x).cuda()
        ref = orc.stream_synth(x, T, R)
        for ctas in (1, 3, 8):
            assert np.array_equal(_launch(cm, st, ctas, xd, W), ref), ctas
        lg, idx, val = _launch(cm, stf, 4, xd, W, top_k=5)
        assert np.array_equal(lg, ref)
        ridx, rval = orc.topk(ref, 5)
        assert np.array_equal(idx, ridx) and np.array_equal(val, rval.astype(np.float32))
    finally:
        cm.camelot_stage_release(st)
        cm.camelot_stage_release(stf)


def test_stream_synth_rejects_bad_dims():
    from paper_2005_02088_b300 import camelot as cm
    T = torch.zeros(4096, device="cuda")
    for dims in [(6, 12, 4096), (8, 12, 4096), (8, 16, 4092), (8, 8192, 4096)]:
        d = cm.StageDesc()
        d.kind = cm.STAGE_STREAM_SYNTH
        d.dims[0], d.dims[1], d.dims[2] = dims
        d.weights[0] = T.data_ptr()
        d.max_batch = 8
        with pytest.raises(cm.CamelotError):
            cm.camelot_stage_prepare(d)


def test_artifact_pipeline_both_handoffs(orc):
    """p (host table) -> c -> m (device table) + top-5: completions and logits
    rows identical to the oracle in both handoff modes."""
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    W, n = 512, 40
    g = np.random.default_rng(9)
    x = g.standard_normal((n, W)).astype(np.float32)
    Th = g.standard_normal(W * 64).astype(np.float32)
    Td = g.standard_normal(W * 512).astype(np.float32)
    th = torch.from_numpy(Th).pin_memory()
    td = torch.from_numpy(Td).cuda()
    stages = [pl.stage_stream_synth(W, W * 4, th, 0, 16), pl.stage_compute_synth(W, 50, 0, 16),
              pl.stage_stream_synth(W, W * 16, td, 5, 16)]
    z, ridx, _ = orc.pipeline_artifact(x, [("m", Th, W * 4), ("c", 50), ("m", Td, W * 16)], top_k=5)
    try:
        for mode in (0, 1):
            sink = torch.zeros((4096, W), dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            p = cm.camelot_pipeline_create(stages, pl.alloc([1, 2, 2], [8, 8, 8], 16), mode,
                                           pl.options(logits_sink=sink.data_ptr()))
            try:
                comps = pl.run_all(p, x.view(np.uint8).reshape(n, -1), stream_id=2, chunk=8, timeout_s=60)
            finally:
                cm.camelot_pipeline_destroy(p)
            idx = np.array([[c.idx[r] for r in range(5)] for c in comps])
            assert np.array_equal(idx, ridx), mode
            assert np.array_equal(sink[:n].cpu().numpy(), z), mode
    finally:
        for st in stages:
            cm.camelot_stage_release(st)
