"""GPU parity of the FP8 arm (OCP FP8 E4M3 operands, per-tensor scales, f32
accumulation on tcgen05 kind::f8f6f4) against the oracle's emulation.

Integer decisions are checked exactly where both sides take them in the same
binary32 precision (stage-1 codes, weight codes and scale).  A layer's output
code comes from an f32 accumulation whose order the tensor core fixes: with
y64 the FP64 value on the same codes and e = (4 K + 2) 2^-24 sum |wq xq| vscale,
the GPU's code must lie between the codes of act(y64 - e) / s and act(y64 + e) / s
(rounding is monotone); and since the typical error is far below that worst
case, over 95 % of the codes must equal the oracle's own."""
import numpy as np
import pytest
import torch

import synth
import tc_bound
from gpu_common import fp8_chain_check

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _stage_fp8(cm, pl, ws, acts, scales, top_k, max_batch=32):
    d = cm.StageDesc()
    d.kind = cm.STAGE_GEMM_FP8
    d.n_layers = len(ws)
    d.dims[0] = ws[0].shape[1]
    for i, w in enumerate(ws):
        d.dims[i + 1] = w.shape[0]
        d.act[i] = acts[i]
        d.weights[i] = w.data_ptr()
    for i, s in enumerate(scales):
        d.scales[i] = s
    d.top_k = top_k
    d.max_batch = max_batch
    torch.cuda.synchronize()
    return cm.camelot_stage_prepare(d)


def _calib(orc, ws):
    from test_oracle_fp8 import calib_scales
    xc = synth.images_u8(0, 64, 64, 64, 3, tag="cfg5.calibration")
    return [float(np.float32(s)) for s in calib_scales(orc, ws, xc)]


def _code_bounds(orc, y64, absdot, K, act, s_out):
    e = (4 * K + 2) * U * absdot
    lo, hi = y64 - e, y64 + e
    if act == 1:
        lo, hi = np.maximum(lo, 0), np.maximum(hi, 0)
    f = lambda v: orc.round_e4m3(v.astype(np.float32).astype(np.float64) / s_out)
    return f(lo), f(hi)


def test_normalize_e4m3_bit_exact(orc):
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    x, _ = synth.cfg1_inputs(0, n_queries=40)
    d = cm.StageDesc()
    d.kind = cm.STAGE_NORMALIZE_U8_E4M3
    d.dims[0], d.dims[1], d.dims[2] = 64, 64, 3
    d.max_batch = 64
    st = cm.camelot_stage_prepare(d)
    try:
        _, orow, sb = cm.camelot_stage_info(st, 40)
        assert orow == 12288
        out = torch.zeros((40, 12288), dtype=torch.uint8, device="cuda")
        scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
        cm.camelot_stage_launch(st, 5, torch.from_numpy(x.reshape(40, -1)).cuda(), 40, out, None, None, None,
                                scr, sb, None)
        got = orc.e4m3_decode(out.cpu().numpy())
    finally:
        cm.camelot_stage_release(st)
    ref = orc.round_e4m3((x.reshape(40, -1).astype(np.float64) - 127.5) * 2.0)
    assert np.array_equal(got, ref)


def test_weight_codes_and_scale_exact(orc):
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    g = np.random.default_rng(3)
    w = (g.standard_normal((296, 384)) * 0.05).astype(np.float32)
    st = _stage_fp8(cm, pl, [torch.from_numpy(w).cuda()], [0], [0.01, 0.02], top_k=0)
    try:
        codes, sw = cm.camelot_stage_export_weights(st, 0, 296, 384, 1)
    finally:
        cm.camelot_stage_release(st)
    s_ref, q_ref = orc.quantize_e4m3(w)
    assert sw == s_ref
    assert np.array_equal(orc.e4m3_decode(codes), q_ref)
    # the BF16 stage's tiled weights read back as the bf16 bit patterns
    wb = torch.from_numpy(w).to(torch.bfloat16)
    st2 = pl.stage_dense(cm.STAGE_GEMM_BF16, [wb.cuda()], [0], top_k=0, max_batch=32)
    try:
        bits, s2 = cm.camelot_stage_export_weights(st2, 0, 296, 384, 2)
    finally:
        cm.camelot_stage_release(st2)
    assert s2 == 1.0
    assert np.array_equal(bits, wb.view(torch.int16).numpy().view(np.uint16))


@pytest.mark.parametrize("K,N,n,act,ctas", [(12288, 512, 16, 1, 8), (512, 256, 32, 1, 3), (256, 128, 5, 0, 1)])
def test_fp8_layer_codes_within_bound(orc, K, N, n, act, ctas):
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    g = np.random.default_rng(K + N)
    w = (g.standard_normal((N, K)) / np.sqrt(K)).astype(np.float32)
    xq_codes = g.integers(0, 256, (n, K)).astype(np.uint8)
    xq_codes[(xq_codes & 0x7F) == 0x7F] = 0x38          # no NaN codes
    s_in = 1.0 / 128
    sw, wq = orc.quantize_e4m3(w)
    vscale = orc.f32(sw * orc.f32(s_in))
    y64, _, a = orc.linear_fp8(orc.e4m3_decode(xq_codes), wq, vscale, act)
    s_out = orc.f32(np.abs(y64).max() / 448.0)       # outputs span the code range
    st = _stage_fp8(cm, pl, [torch.from_numpy(w).cuda()], [act], [s_in, s_out], top_k=0)
    try:
        out = torch.zeros((n, N), dtype=torch.uint8, device="cuda")
        _, _, sb = cm.camelot_stage_info(st, n)
        scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
        cm.camelot_stage_launch(st, ctas, torch.from_numpy(xq_codes).cuda(), n, out, None, None, None, scr, sb,
                                None)
        got = orc.e4m3_decode(out.cpu().numpy())
    finally:
        cm.camelot_stage_release(st)
    lo, hi = _code_bounds(orc, y64, a, K, act, s_out)
    assert np.all((got >= lo) & (got <= hi))
    # and inside the much narrower bracket of the instruction model
    own_t, lo_t, hi_t = tc_bound.e4m3_layer_bracket(orc, orc.e4m3_decode(xq_codes), wq, vscale, act, s_out)
    assert np.all((got >= lo_t) & (got <= hi_t))
    # the worst-case bracket is wide at large K; the typical accumulation error
    # is far smaller, so nearly every code equals the oracle's own rounding
    own = orc.round_e4m3((np.maximum(y64, 0) if act == 1 else y64).astype(np.float32).astype(np.float64) / s_out)
    assert np.mean(got == own) > 0.95, np.mean(got == own)


def test_fp8_mlp_fused_equals_chained_and_oracle(orc):
    """The 3-layer FP8 stage gives the same logits, bit for bit, as three
    single-layer stages chained through their e4m3 outputs; each link is within
    its bound of the oracle on the GPU's own inputs; the result does not depend
    on the number of CTAs."""
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    x, ws = synth.cfg1_inputs(0, n_queries=32)
    sc = _calib(orc, ws)
    scales = [orc.f32(1.0 / 128)] + sc
    wd = [torch.from_numpy(w).cuda() for w in ws]
    xq = orc.round_e4m3((x.reshape(32, -1).astype(np.float64) - 127.5) * 2.0)
    xq_codes = torch.from_numpy(xq.astype(np.float32)).to(torch.float8_e4m3fn).view(torch.uint8).cuda()
    fused = _stage_fp8(cm, pl, wd, [1, 1, 0], scales, top_k=1)
    links = [_stage_fp8(cm, pl, [wd[0]], [1], scales[0:2], 0), _stage_fp8(cm, pl, [wd[1]], [1], scales[1:3], 0),
             _stage_fp8(cm, pl, [wd[2]], [0], scales[2:3], 1)]
    try:
        res = []
        for ctas in (1, 7, 64, 148):
            _, _, sb = cm.camelot_stage_info(fused, 32)
            scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
            idx = torch.empty((32, 1), dtype=torch.int32, device="cuda")
            val = torch.empty((32, 1), dtype=torch.float32, device="cuda")
            lg = torch.empty((32, 10), dtype=torch.float32, device="cuda")
            cm.camelot_stage_launch(fused, ctas, xq_codes, 32, None, idx, val, lg, scr, sb, None)
            torch.cuda.synchronize()
            res.append((idx.cpu().numpy(), lg.cpu().numpy()))
        for r in res[1:]:
            assert np.array_equal(r[0], res[0][0]) and np.array_equal(r[1], res[0][1])
        h = xq_codes
        hid = []
        for i, st in enumerate(links):
            _, _, sb = cm.camelot_stage_info(st, 32)
            scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
            if i < 2:
                o = torch.zeros((32, ws[i].shape[0]), dtype=torch.uint8, device="cuda")
                cm.camelot_stage_launch(st, 9, h, 32, o, None, None, None, scr, sb, None)
                hid.append(o)
                h = o
            else:
                idx = torch.empty((32, 1), dtype=torch.int32, device="cuda")
                val = torch.empty((32, 1), dtype=torch.float32, device="cuda")
                lg = torch.empty((32, 10), dtype=torch.float32, device="cuda")
                cm.camelot_stage_launch(st, 9, h, 32, None, idx, val, lg, scr, sb, None)
        torch.cuda.synchronize()
        assert np.array_equal(lg.cpu().numpy(), res[0][1])
        assert np.array_equal(idx.cpu().numpy(), res[0][0])
        # each link against the oracle on the GPU's own input codes
        ins = [xq] + [orc.e4m3_decode(t.cpu().numpy()) for t in hid]
        for l in range(3):
            sw, wq = orc.quantize_e4m3(ws[l])
            vscale = orc.f32(sw * scales[l])
            K = ws[l].shape[1]
            y64, _, a = orc.linear_fp8(ins[l], wq, vscale, 1 if l < 2 else 0)
            if l < 2:
                lo, hi = _code_bounds(orc, y64, a, K, 1, scales[l + 1])
                assert np.all((ins[l + 1] >= lo) & (ins[l + 1] <= hi)), l
            else:
                assert np.all(np.abs(res[0][1] - y64) <= (4 * K + 2) * U * a + 1e-30)
        # the argmax is exact on the GPU's own logits
        assert np.array_equal(res[0][0][:, 0], np.argmax(res[0][1], axis=1))
    finally:
        for st in [fused] + links:
            cm.camelot_stage_release(st)


def test_fp8_pipeline_both_handoffs(orc):
    """cfg1 with e4m3 stages end to end: normalise -> e4m3 handoff (12 KB per
    query) -> FP8 MLP + argmax; identical through both handoffs; top-1
    agreement with the FP64 pipeline reported and bounded."""
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    n = 96
    x, ws = synth.cfg1_inputs(0, n_queries=n)
    sc = _calib(orc, ws)
    scales = [orc.f32(1.0 / 128)] + sc
    d = cm.StageDesc()
    d.kind = cm.STAGE_NORMALIZE_U8_E4M3
    d.dims[0], d.dims[1], d.dims[2] = 64, 64, 3
    d.max_batch = 32
    s0 = cm.camelot_stage_prepare(d)
    s1 = _stage_fp8(cm, pl, [torch.from_numpy(w).cuda() for w in ws], [1, 1, 0], scales, top_k=1)
    try:
        outs = {}
        for mode in (0, 1):
            sink = torch.zeros((65536, 10), dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            p = cm.camelot_pipeline_create([s0, s1], pl.alloc([1, 2], [8, 16], 16), mode,
                                           pl.options(logits_sink=sink.data_ptr()))
            try:
                comps = pl.run_all(p, x, stream_id=2, chunk=32, timeout_s=60)
            finally:
                cm.camelot_pipeline_destroy(p)
            outs[mode] = ([c.idx[0] for c in comps], sink[:n].cpu().numpy(), [c.query_id for c in comps])
        assert outs[0][2] == list(range(n))
        assert np.array_equal(outs[0][1], outs[1][1]) and outs[0][0] == outs[1][0]
        lg = outs[0][1]
        assert outs[0][0] == list(np.argmax(lg, axis=1))
        # element-wise, link by link, against the oracle; argmax exact where fixed
        res = fp8_chain_check(orc, x, ws, scales, lg, np.array(outs[0][0]))
        assert res["argmax_fixed_on_gpu_input"] >= 0.9 * n, res
        # accuracy of the FP8 arm against the FP64 pipeline (reported; top-1 >= 90 %)
        z8, i8, _, _ = orc.pipeline_fp8(x, ws, sc)
        z64, i64 = orc.pipeline_mlp(x, ws)
        res["top1_agree_fp64"] = float(np.mean(np.array(outs[0][0]) == i64))
        res["max_abs_err_fp64"] = float(np.abs(lg - z64).max())
        res["max_abs_logit_fp64"] = float(np.abs(z64).max())
        print("fp8 2-stage parity:", res)
        assert res["top1_agree_fp64"] >= 0.9
    finally:
        cm.camelot_stage_release(s0)
        cm.camelot_stage_release(s1)
