"""The serving loop: four pipelines of uneven size share the GPU (the plain
FP32 2-stage pipeline, the text-tagging pipeline, the 3-stage BF16 pipeline and
the FP8 2-stage pipeline), each a persistent kernel on its own SMs, fed through
camelot_server with a device-memory budget small enough that admission must
wait.  Every query completes once, in order per pipeline, with results
identical to running its pipeline alone."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _build(cm, pl):
    x1, w1 = synth.cfg1_inputs(0, n_queries=64)
    tok, lens, E, wt = synth.cfg4_inputs(3, n_queries=24)
    x3, w3 = synth.cfg2_inputs(0, n_queries=24)
    bf = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).cuda()
    keep = []
    # P1: FP32 2-stage
    wd1 = [torch.from_numpy(w).cuda() for w in w1]
    p1 = [pl.stage_normalize(64, 64, 3, 32), pl.stage_dense(cm.STAGE_MLP_FP32, wd1, [1, 1, 0], 1, 32)]
    # P2: text tagging
    Eb = bf(E)
    wtb = [bf(w) for w in wt]
    d = cm.StageDesc()
    d.kind = cm.STAGE_EMBED_GATHER
    d.dims[0], d.dims[1], d.dims[2] = 32000, 512, 128
    d.weights[0] = Eb.data_ptr()
    d.max_batch = 8
    torch.cuda.synchronize()
    s20 = cm.camelot_stage_prepare(d)
    d = cm.StageDesc()
    d.kind = cm.STAGE_GEMM_BF16
    d.n_layers = 3
    d.dims[0], d.dims[1], d.dims[2], d.dims[3] = 512, 2048, 512, 64
    for i, w in enumerate(wtb):
        d.weights[i] = w.data_ptr()
    d.act[0] = 2
    d.top_k, d.max_batch, d.rows_per_query = 1, 8, 128
    s21 = cm.camelot_stage_prepare(d)
    p2 = [s20, s21]
    # P3: BF16 3-stage
    wb3 = [bf(w) for w in w3]
    p3 = [pl.stage_norm_pool2(224, 224, 3, 32),
          pl.stage_dense(cm.STAGE_GEMM_BF16, [wb3[0], wb3[1]], [2, 2], 0, 32),
          pl.stage_dense(cm.STAGE_GEMM_BF16, [wb3[2]], [0], 5, 32)]
    # P4: FP8 2-stage (calibrated on the library's FP32 stages)
    sc = pl.calibrate_fp8_scales(wd1, synth.images_u8(0, 64, 64, 64, 3, tag="cfg5.calibration"))
    p4 = [pl.stage_normalize_e4m3(64, 64, 3, 32), pl.stage_fp8(wd1, [1, 1, 0], [1.0 / 128] + sc, 1, 32)]
    keep += [wd1, Eb, wtb, wb3]
    specs = [(p1, [1, 2], [8, 8], 16, x1.reshape(64, -1), 10),
             (p2, [1, 2], [8, 16], 8, tok, 128),
             (p3, [1, 2, 1], [8, 16, 8], 16, x3.reshape(24, -1), 1000),
             (p4, [1, 2], [8, 8], 16, x1.reshape(64, -1), 10)]
    return specs, keep


def _pipeline(cm, pl, spec):
    stages, inst, quota, B, q, width = spec
    sink = torch.zeros((4096, width), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    p = cm.camelot_pipeline_create(stages, pl.alloc(inst, quota, B), 0,
                                   pl.options(query_slots=4096, data_slots=256, device_data=1,
                                              logits_sink=sink.data_ptr()))
    return p, sink


def test_four_pipelines_mix_equals_alone():
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    specs, keep = _build(cm, pl)
    try:
        alone = []
        for spec in specs:
            p, sink = _pipeline(cm, pl, spec)
            try:
                comps = pl.run_all(p, spec[4], stream_id=1, chunk=8, timeout_s=120)
            finally:
                cm.camelot_pipeline_destroy(p)
            n = spec[4].shape[0]
            alone.append((np.array([[c.idx[r] for r in range(5)] for c in comps]), sink[:n].cpu().numpy().copy()))
        pipes = [_pipeline(cm, pl, spec) for spec in specs]
        o = cm.camelot_server_options_default()
        o.device_bytes_budget = 1 << 20            # ~7 of the 150 KB images: admission must wait
        o.max_admit = 16
        srv = cm.camelot_server_create([p for p, _ in pipes], o)
        try:
            ns = [spec[4].shape[0] for spec in specs]
            sent = [0] * 4
            got = [[] for _ in range(4)]
            buf = (cm.Completion * 512)()
            import time
            t_end = time.time() + 120
            while any(len(g) < n for g, n in zip(got, ns)):
                for i, spec in enumerate(specs):
                    if sent[i] < ns[i]:
                        k = min(32, ns[i] - sent[i])
                        rows = np.ascontiguousarray(spec[4][sent[i]:sent[i] + k])
                        if cm.camelot_server_submit(srv, i, 7, rows, k, allow_eagain=True):
                            sent[i] += k
                    m = cm.camelot_server_poll(srv, i, buf, 0)
                    for j in range(m):
                        got[i].append(pl._copy(buf[j]))
                assert time.time() < t_end, [len(g) for g in got]
            stats = [cm.camelot_server_stats(srv, i) for i in range(4)]
        finally:
            cm.camelot_server_destroy(srv)
            for p, _ in pipes:
                cm.camelot_pipeline_destroy(p)
        for i, (g, (idx_a, sink_a)) in enumerate(zip(got, alone)):
            assert [c.query_id for c in g] == list(range(ns[i]))
            idx = np.array([[c.idx[r] for r in range(5)] for c in g])
            assert np.array_equal(idx, idx_a), i
            assert np.array_equal(pipes[i][1][:ns[i]].cpu().numpy(), sink_a), i
            assert stats[i].completed == ns[i] and stats[i].waiting == 0
        assert max(s.peak_inflight_bytes for s in stats) <= 1 << 20
        assert sum(s.deferred for s in stats) > 0        # admission did wait for memory
    finally:
        for spec in specs:
            for st in spec[0]:
                cm.camelot_stage_release(st)
        del keep
