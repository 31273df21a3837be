"""GPU parity of the tensor-core GEMM_BF16 stages (tcgen05 MMA, TMA weight
stream, TMEM accumulator) against the FP64 oracle on bf16-rounded operands,
and of the whole 3-stage pipeline (2x2 pool + normalise to bf16 -> 37632 ->
1024 -> 1024 GELU -> 1024 -> 1000 logits + top-5).

Tolerance: the accumulation is FP32 in an order the tensor core fixes.  A
pre-activation may differ from the exact sum by at most the instruction-model
bound of tests/tc_bound.py (per MMA instruction, (t + 2) 2^-23 times the
accumulator plus the instruction's |products|, summed over the chunk, then
the chunk-order f32 sum); the GELU passes at most 1.13 times that on, and the
bf16 output must lie between the roundings of the interval's ends.  The
serial-sum worst case 4 K 2^-24 sum|w x| is checked as well."""
import time

import numpy as np
import pytest
import torch

import synth
import tc_bound
from gpu_common import bf16_chain_check

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def _bf(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)


def _f64(t):
    return t.float().cpu().numpy().astype(np.float64)


def _scratch(cm, st, n):
    _, _, sb = cm.camelot_stage_info(st, n)
    return torch.empty(sb + 256, dtype=torch.uint8, device="cuda"), sb


def _layer_bound(orc, x64, w64, act):
    ref, a = orc.linear(x64, w64, act, want_absdot=True)
    K = x64.shape[1]
    return ref, (1.13 if act == 2 else 1.0) * 4 * K * U * a


# 4096 -> 1024 and 37632 -> 1024 are two K-chunks: on 37 or 74 CTAs reduced by
# the reduce pass, on 8 or 4 CTAs added in pairs by each CTA's epilogue
@pytest.mark.parametrize("K,N,n,act,ctas", [(1024, 256, 16, 2, 8), (4096, 1024, 32, 2, 37),
                                             (4096, 1024, 31, 2, 8), (1024, 1000, 5, 0, 3),
                                             (512, 128, 1, 1, 1), (37632, 1024, 9, 2, 74),
                                             (37632, 1024, 9, 2, 4)])
def test_gemm_layer_matches_oracle(orc, K, N, n, act, ctas):
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    g = np.random.default_rng(K + N + n)
    x = _bf(g.standard_normal((n, K)))
    w = _bf(g.standard_normal((N, K)) / np.sqrt(K))
    xd, wd = x.cuda(), w.cuda()
    st = pl.stage_dense(cm.STAGE_GEMM_BF16, [wd], [act], top_k=0, max_batch=32)
    try:
        out = torch.full((n, N), float("nan"), dtype=torch.bfloat16, device="cuda")
        scr, sb = _scratch(cm, st, n)
        cm.camelot_stage_launch(st, ctas, xd, n, out, None, None, None, scr, sb, None)
        torch.cuda.synchronize()
        got = _f64(out)
        assert np.all(np.isfinite(got))
        # inside the bf16 bracket of the accumulation bound (instruction model)
        ref, lo, hi = tc_bound.bf16_layer_bracket(orc, _f64(x), _f64(w), act)
        assert np.all((got >= lo) & (got <= hi))
        # and inside the serial-sum worst case (4 K u sum|w x|) plus one bf16 unit
        _, bound = _layer_bound(orc, _f64(x), _f64(w), act)
        assert np.all(np.abs(got - ref) <= bound + 2.0 ** -8 * np.abs(ref) + 1e-30)
        # the typical error is far below the bound: nearly every value is the oracle's own rounding
        assert np.mean(got == orc.round_bf16(ref)) > 0.97, np.mean(got == orc.round_bf16(ref))
    finally:
        cm.camelot_stage_release(st)


def test_gemm_chain_topk_and_partition_independence(orc):
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    g = np.random.default_rng(5)
    n = 12
    dims = [2048, 1024, 1000]
    x = _bf(g.standard_normal((n, dims[0])))
    ws = [_bf(g.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i])) for i in range(2)]
    st = pl.stage_dense(cm.STAGE_GEMM_BF16, [w.cuda() for w in ws], [2, 0], top_k=5, max_batch=32)
    try:
        res = []
        # 1, 4 and 8 CTAs add the first layer's two K-chunks in each CTA's
        # epilogue, 9, 64 and 148 in the reduce pass: the same bits either way
        for ctas in (1, 4, 8, 9, 64, 148):
            idx = torch.empty((n, 5), dtype=torch.int32, device="cuda")
            val = torch.empty((n, 5), dtype=torch.float32, device="cuda")
            lg = torch.empty((n, 1000), dtype=torch.float32, device="cuda")
            scr, sb = _scratch(cm, st, n)
            cm.camelot_stage_launch(st, ctas, x.cuda(), n, None, idx, val, lg, scr, sb, None)
            torch.cuda.synchronize()
            res.append((idx.cpu().numpy(), val.cpu().numpy(), lg.cpu().numpy()))
        for r in res[1:]:
            for a, b in zip(res[0], r):
                assert np.array_equal(a, b)
        idx, val, lg = res[0]
        # top-5 is exact on the GPU's own logits
        ref_idx, ref_val = orc.topk(lg.astype(np.float64), 5)
        assert np.array_equal(idx, ref_idx) and np.array_equal(val, ref_val.astype(np.float32))
        # logits within the bound of the bf16-emulated FP64 chain
        h, b1 = _layer_bound(orc, _f64(x), _f64(ws[0]), 2)
        h_r = orc.round_bf16(h)
        z, b2 = _layer_bound(orc, h_r, _f64(ws[1]), 0)
        # the hidden layer's bf16 rounding may differ by one unit: propagate it
        e_h = b1 + 2.0 ** -8 * np.abs(h) + 1e-30
        bound = b2 + e_h @ np.abs(_f64(ws[1])).T
        assert np.all(np.abs(lg - z) <= bound)
    finally:
        cm.camelot_stage_release(st)


def test_three_stage_pipeline_bf16(orc):
    """cfg2 end to end through the persistent pipeline, both handoffs.  The
    final stage on 8 SMs takes its top-5 from per-CTA candidates merged by the
    instance's leader, on 16 SMs (its two K-chunks then unpaired) from the
    row-wise pass after the reduce: the results must be the same bits."""
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    n = 48
    x, ws32 = synth.cfg2_inputs(0, n_queries=n)
    wb = [_bf(w) for w in ws32]
    s0 = pl.stage_norm_pool2(224, 224, 3, max_batch=32)
    s1 = pl.stage_dense(cm.STAGE_GEMM_BF16, [wb[0].cuda(), wb[1].cuda()], [2, 2], top_k=0, max_batch=32)
    s2 = pl.stage_dense(cm.STAGE_GEMM_BF16, [wb[2].cuda()], [0], top_k=5, max_batch=32)
    try:
        outs = {}
        for mode, fq in ((0, 8), (1, 8), (0, 16)):
            sink = torch.zeros((65536, 1000), dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            p = cm.camelot_pipeline_create([s0, s1, s2], pl.alloc([1, 2, 1], [8, 24, fq], 16), mode,
                                           pl.options(logits_sink=sink.data_ptr()))
            try:
                comps = pl.run_all(p, x, stream_id=3, chunk=16, timeout_s=120)
            finally:
                cm.camelot_pipeline_destroy(p)
            outs[(mode, fq)] = (comps, sink[:n].cpu().numpy())
        comps, lg = outs[(0, 8)]
        assert [c.query_id for c in comps] == list(range(n))
        for key in ((1, 8), (0, 16)):                             # handoff- and quota-independent
            c2, lg2 = outs[key]
            assert np.array_equal(lg.view(np.uint32), lg2.view(np.uint32)), key
            assert [list(c.idx) for c in comps] == [list(c.idx) for c in c2], key
            assert np.array_equal(np.array([list(c.val) for c in comps], np.float32).view(np.uint32),
                                  np.array([list(c.val) for c in c2], np.float32).view(np.uint32)), key
        idx = np.array([[c.idx[r] for r in range(5)] for c in comps])
        ref_idx, _ = orc.topk(lg.astype(np.float64), 5)
        assert np.array_equal(idx, ref_idx)                        # exact on its own logits
        # element-wise, link by link, against the oracle; top-5 exact where fixed
        res = bf16_chain_check(orc, x, wb, lg, idx)
        assert res["top5_fixed_on_gpu_input"] >= 0.9 * n, res
        # accuracy of the bf16 arm against the unquantised FP64 pipeline (reported)
        z64, i64 = orc.pipeline_gemm3(x, [np.asarray(w, np.float64) for w in ws32], top_k=5)
        res["top1_agree_fp64"] = float(np.mean(idx[:, 0] == i64[:, 0]))
        res["top5_set_agree_fp64"] = float(np.mean([set(a) == set(b) for a, b in zip(idx, i64)]))
        res["max_abs_err_fp64"] = float(np.abs(lg - z64).max())
        print("bf16 3-stage parity:", res)
    finally:
        for s in (s0, s1, s2):
            cm.camelot_stage_release(s)


@pytest.mark.parametrize("slots", [2, 3, 4])
def test_ring_slots_do_not_change_results(slots):
    """The 3-stage pipeline with the GEMM stages' bulk-copy rings capped at 2, 3
    or 4 slots gives bit-identical results to the full ring, over a saturated
    trace long enough for many ring wraps per CTA.  With an odd slot count a
    slot's successive fills alternate between the two MMA issuers: the case in
    which a parity wait on a barrier shared by both issuers can pass a phase
    early and stall the ring."""
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    n = 2048
    x, ws32 = synth.cfg2_inputs(0, n_queries=64)
    xd = torch.from_numpy(np.ascontiguousarray(x.reshape(64, -1))).cuda()[torch.arange(n).cuda() % 64]
    wd = [_bf(w).cuda() for w in ws32]
    off = torch.zeros(n, dtype=torch.int64, device="cuda")
    res = {}
    for r in (0, slots):
        st = [pl.stage_norm_pool2(224, 224, 3, max_batch=32),
              pl.stage_dense(cm.STAGE_GEMM_BF16, [wd[0], wd[1]], [2, 2], top_k=0, max_batch=32, ring_slots=r),
              pl.stage_dense(cm.STAGE_GEMM_BF16, [wd[2]], [0], top_k=5, max_batch=32, ring_slots=r)]
        try:
            torch.cuda.synchronize()
            p = cm.camelot_pipeline_create(st, pl.alloc([2, 6, 2], [8, 8, 8], 32),
                                           0, pl.options(exit_after_trace=1))
            try:
                assert cm.camelot_submit_trace(p, 0, xd, n, off) == 0
                buf = (cm.Completion * 4096)()
                comps, t_end = [], time.time() + 60
                while len(comps) < n and time.time() < t_end:
                    k = cm.camelot_poll(p, buf, timeout_us=2000)
                    comps += [pl._copy(buf[i]) for i in range(k)]
                assert cm.camelot_pipeline_stats(p).device_status == 0
            finally:
                cm.camelot_pipeline_destroy(p)
        finally:
            for s in st:
                cm.camelot_stage_release(s)
        assert [c.query_id for c in comps] == list(range(n)) and all(c.status == 0 for c in comps)
        res[r] = (np.array([list(c.idx) for c in comps]), np.array([list(c.val) for c in comps], np.float32))
    assert np.array_equal(res[0][0], res[slots][0])
    assert np.array_equal(res[0][1].view(np.uint32), res[slots][1].view(np.uint32))
