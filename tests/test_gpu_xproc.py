"""Cross-process handoff (Sec. 6.2): the plain 2-stage pipeline split over two
processes (normalise in the producer, the FP32 MLP + argmax in the consumer),
batches handed over in place through the IPC ring.  Results identical to the
same two stages launched in one process; the paced run reports a latency per
batch."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _in_process(x, ws, B):
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    s0 = pl.stage_normalize(64, 64, 3, B)
    wd = [torch.from_numpy(w).cuda() for w in ws]
    s1 = pl.stage_dense(cm.STAGE_MLP_FP32, wd, [1, 1, 0], 1, B)
    try:
        out = []
        q = torch.from_numpy(x).cuda()
        mid = torch.empty((B, 12288), dtype=torch.float32, device="cuda")
        idx = torch.empty((B, 1), dtype=torch.int32, device="cuda")
        val = torch.empty((B, 1), dtype=torch.float32, device="cuda")
        _, _, sb0 = cm.camelot_stage_info(s0, B)
        _, _, sb1 = cm.camelot_stage_info(s1, B)
        scr0 = torch.empty(sb0 + 256, dtype=torch.uint8, device="cuda")
        scr1 = torch.empty(sb1 + 256, dtype=torch.uint8, device="cuda")
        for b in range(0, x.shape[0], B):
            nb = min(B, x.shape[0] - b)
            cm.camelot_stage_launch(s0, 16, q[b:b + nb], nb, mid, None, None, None, scr0, sb0, None)
            cm.camelot_stage_launch(s1, 64, mid, nb, None, idx, val, None, scr1, sb1, None)
            torch.cuda.synchronize()
            out.append(idx[:nb].cpu().numpy().copy())
        return np.concatenate(out)
    finally:
        cm.camelot_stage_release(s0)
        cm.camelot_stage_release(s1)


@pytest.mark.parametrize("paced", [False, True])
def test_two_process_split_matches_one_process(paced):
    from paper_2005_02088_b300 import xproc
    n, B = 100, 16
    x, ws = synth.cfg1_inputs(0, n_queries=n)
    xr = np.ascontiguousarray(x.reshape(n, -1))
    res = xproc.run_split({"kind": "normalize", "dims": (64, 64, 3)},
                          {"kind": "mlp_fp32", "weights": ws, "acts": [1, 1, 0], "top_k": 1},
                          xr, batch=B, top_k=1, slots=4, paced=paced, timeout_s=180)
    assert np.array_equal(res["idx"], _in_process(xr, ws, B))
    assert 0 < res["ring_create_s"] < 5 and 0 < res["ring_open_s"] < 5
    if paced:
        assert len(res["latency_s"]) == (n + B - 1) // B and min(res["latency_s"]) > 0


def test_ring_handle_rejects_malformed():
    from paper_2005_02088_b300 import camelot as cm
    h = cm.XringHandle()
    h.slots, h.slot_bytes = 0, 1024
    with pytest.raises(cm.CamelotError):
        cm.camelot_xring_open(bytes(h))
    h.slots, h.device = 4, 77
    with pytest.raises(cm.CamelotError):
        cm.camelot_xring_open(bytes(h))


def test_ring_cannot_be_opened_by_its_creator():
    """cudaIpcOpenMemHandle refuses the creating process: the library reports
    ECUDA and leaves the ring usable; the wrong side's calls are EINVAL."""
    from paper_2005_02088_b300 import camelot as cm
    x, h = cm.camelot_xring_create(4096, 2)
    try:
        with pytest.raises(cm.CamelotError):
            cm.camelot_xring_open(h)
        with pytest.raises(cm.CamelotError):
            cm.camelot_xring_consume_begin(x, 0, None)
        with pytest.raises(cm.CamelotError):
            cm.camelot_xring_produce_begin(x, 2, None)
        assert cm.camelot_xring_slot(x, 1) - cm.camelot_xring_slot(x, 0) == 4096
        cm.camelot_xring_produce_begin(x, 0, None)
        cm.camelot_xring_produce_end(x, 0, None)
        torch.cuda.synchronize()
    finally:
        cm.camelot_xring_destroy(x)
