"""Shared inputs and tolerance helpers of the GPU parity tests."""
import functools

import numpy as np

import synth

FP32_REL = 1e-5   # |y_gpu - y_fp64| <= FP32_REL * sum_k |w_jk x_k| per element


@functools.lru_cache(maxsize=None)
def cfg1_data(n: int = 256, seed: int = 0):
    x, ws = synth.cfg1_inputs(seed, n_queries=n)
    return x, ws


@functools.lru_cache(maxsize=None)
def cfg1_oracle(n: int = 256, seed: int = 0):
    import oracle
    x, ws = cfg1_data(n, seed)
    logits, idx = oracle.pipeline_mlp(x, ws)
    return logits, idx


def chain_bound(orc, x_u8, ws, acts):
    """Per-element bound on |gpu - fp64| for a dense chain run in FP32: each
    layer adds FP32_REL * sum|w x| and passes on |W| times the incoming bound
    (ReLU is 1-Lipschitz).  Also returns the FP64 logits."""
    y = orc.normalize_u8(x_u8.reshape(x_u8.shape[0], -1))
    e = np.zeros_like(y)
    for w, act in zip(ws, acts):
        w = np.asarray(w, np.float64)
        y, a = orc.linear(y, w, act, want_absdot=True)
        e = FP32_REL * a + e @ np.abs(w).T
    return y, e


def argmax_margin_ok(z64, err):
    """Queries whose FP64 top-1 beats the runner-up by more than twice `err`
    (the per-query logit error actually observed): there the GPU's argmax must
    equal the FP64 one."""
    s = np.sort(z64, axis=1)
    return (s[:, -1] - s[:, -2]) > 2 * np.max(err, axis=1)


def first_argmax(z):
    """Index of the largest value per row, lowest index on ties."""
    return np.argmax(z, axis=1)


def direct(st, inp, n, out_cols=0, out_dtype=None, top_k=0, logits_cols=0, ctas=37, max_batch=32):
    """Run a prepared stage by direct launches over n rows of `inp` (a device
    tensor, one row per query), max_batch rows at a time.  Returns the output
    rows (intermediate stage) or (idx, val, logits) as host arrays."""
    import torch
    from paper_2005_02088_b300 import camelot as cm
    out = torch.empty((n, out_cols), dtype=out_dtype, device="cuda") if out_cols else None
    idx = torch.empty((n, top_k), dtype=torch.int32, device="cuda") if top_k else None
    val = torch.empty((n, top_k), dtype=torch.float32, device="cuda") if top_k else None
    lg = torch.full((n, logits_cols), float("nan"), dtype=torch.float32, device="cuda") if logits_cols else None
    _, _, sb = cm.camelot_stage_info(st, max_batch)
    scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
    for q0 in range(0, n, max_batch):
        m = min(max_batch, n - q0)
        cm.camelot_stage_launch(st, ctas, inp[q0:q0 + m], m, out[q0:q0 + m] if out is not None else None,
                                idx[q0:q0 + m] if idx is not None else None,
                                val[q0:q0 + m] if val is not None else None,
                                lg[q0:q0 + m] if lg is not None else None, scr, sb, None)
    torch.cuda.synchronize()
    if top_k:
        return idx.cpu().numpy(), val.cpu().numpy(), lg.cpu().numpy() if lg is not None else None
    return out


def f64(t):
    return t.float().cpu().numpy().astype(np.float64)


def bf16_chain_check(orc, x_u8, wb, lg, idx, ctas=37):
    """Link-by-link parity of the 3-stage BF16 pipeline for the images x_u8,
    given the pipeline's f32 logits `lg` and top-5 `idx` for them.

    The same stages run as direct launches of single layers (pool; 37632 ->
    1024 GELU; 1024 -> 1024 GELU; 1024 -> 1000 + top-5) whose final logits must
    equal the pipeline's bit for bit, which makes every hidden row of the
    chain a row of the pipeline.  Then, per element and against the oracle:
    the pooled bf16 rows exactly; each hidden layer on the GPU's own input
    inside the bf16 bracket of the tensor-core accumulation bound; the logits
    within their bound, and the top-5 exact wherever the bound fixes it.  The
    whole chain is also held against the oracle's bf16-emulated pipeline (its
    own hidden roundings): the logits there differ by the hidden rows' bf16
    disagreements carried through |W3|, which is the bound used for its top-5.
    Returns a dict of counts and agreement rates."""
    import torch
    import tc_bound as tb
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    n = x_u8.shape[0]
    wd = [w.cuda() for w in wb]
    w64 = [w.float().numpy().astype(np.float64) for w in wb]
    st = [pl.stage_norm_pool2(224, 224, 3, max_batch=32),
          pl.stage_dense(cm.STAGE_GEMM_BF16, [wd[0]], [2], top_k=0, max_batch=32),
          pl.stage_dense(cm.STAGE_GEMM_BF16, [wd[1]], [2], top_k=0, max_batch=32),
          pl.stage_dense(cm.STAGE_GEMM_BF16, [wd[2]], [0], top_k=5, max_batch=32)]
    try:
        xin = torch.from_numpy(np.ascontiguousarray(x_u8.reshape(n, -1))).cuda()
        y0 = direct(st[0], xin, n, w64[0].shape[1], torch.bfloat16, ctas=ctas)
        h1 = direct(st[1], y0, n, 1024, torch.bfloat16, ctas=ctas)
        h2 = direct(st[2], h1, n, 1024, torch.bfloat16, ctas=ctas)
        i3, v3, z3 = direct(st[3], h2, n, top_k=5, logits_cols=w64[2].shape[0], ctas=ctas)
    finally:
        for s in st:
            cm.camelot_stage_release(s)
    assert np.array_equal(z3.view(np.uint32), np.ascontiguousarray(lg, np.float32).view(np.uint32))
    assert np.array_equal(i3, np.asarray(idx)[:, :5])
    res = {"queries": n}
    y0_64 = f64(y0)
    assert np.array_equal(y0_64, orc.round_bf16(orc.norm_pool2(x_u8)))
    for l, (xi, w, o) in enumerate(((y0_64, w64[0], h1), (f64(h1), w64[1], h2))):
        G, lo, hi = tb.bf16_layer_bracket(orc, xi, w, 2)
        ov = f64(o)
        assert np.all((ov >= lo) & (ov <= hi)), l
        res[f"layer{l + 1}_equal_to_oracle_rounding"] = float(np.mean(ov == orc.round_bf16(G)))
    h2_64 = f64(h2)
    z, e = tb.logits_bound(orc, h2_64, w64[2])
    err = np.abs(z3 - z)
    assert np.all(err <= e), float((err / e).max())
    res["logits_max_err_over_bound"] = float((err / e).max())
    res["top5_fixed_on_gpu_input"] = tb.check_topk(i3, z, e, 5)
    # against the oracle's own bf16-emulated pipeline
    H1 = orc.round_bf16(orc.linear(y0_64, w64[0], 2))
    H2 = orc.round_bf16(orc.linear(H1, w64[1], 2))
    z_emul = orc.linear(H2, w64[2], 0)
    e_all = e + np.abs(h2_64 - H2) @ np.abs(w64[2]).T
    assert np.all(np.abs(z3 - z_emul) <= e_all)
    res["top5_fixed_vs_emulated"] = tb.check_topk(i3, z_emul, e_all, 5)
    res["hidden2_rows_equal_emulated"] = float(np.mean(np.all(h2_64 == H2, axis=1)))
    res["top5_set_agree_emulated"] = float(np.mean([set(a) == set(b) for a, b in
                                                    zip(i3, orc.topk(z_emul, 5)[0])]))
    return res


def fp8_chain_check(orc, x_u8, ws, scales, lg, idx, ctas=37):
    """Link-by-link parity of the FP8 2-stage pipeline (e4m3 normalise; FP8 MLP
    12288 -> 512 -> 256 -> 10 with ReLU, static scales; argmax) for the images
    x_u8, given the pipeline's logits and argmax.  Direct launches of the
    normalise stage and of three single-layer FP8 stages must reproduce the
    pipeline's logits bit for bit; each hidden layer's codes, on the GPU's own
    input codes, lie inside the code bracket of the accumulation bound; the
    logits lie within their bound and the argmax is exact wherever the bound
    fixes it; against the oracle's own emulated chain, the logits differ by the
    hidden code disagreements carried through |W3| (scaled), which is the bound
    for the argmax there.  `scales` = [1/128, s_1, s_2] (f32)."""
    import torch
    import tc_bound as tb
    from paper_2005_02088_b300 import camelot as cm
    n = x_u8.shape[0]
    st = []

    def fp8_stage(w, act, sc, top_k):
        d = cm.StageDesc()
        d.kind = cm.STAGE_GEMM_FP8
        d.n_layers = 1
        d.dims[0], d.dims[1] = w.shape[1], w.shape[0]
        d.act[0] = act
        d.weights[0] = w.data_ptr()
        for i, s in enumerate(sc):
            d.scales[i] = s
        d.top_k = top_k
        d.max_batch = 32
        torch.cuda.synchronize()
        st.append(cm.camelot_stage_prepare(d))
        return st[-1]

    wd = [torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda() for w in ws]
    try:
        d = cm.StageDesc()
        d.kind = cm.STAGE_NORMALIZE_U8_E4M3
        d.dims[0], d.dims[1], d.dims[2] = 64, 64, 3
        d.max_batch = 32
        st.append(cm.camelot_stage_prepare(d))
        xin = torch.from_numpy(np.ascontiguousarray(x_u8.reshape(n, -1))).cuda()
        c0 = direct(st[0], xin, n, 12288, torch.uint8, ctas=ctas)
        l1 = fp8_stage(wd[0], 1, scales[0:2], 0)
        c1 = direct(l1, c0, n, ws[0].shape[0], torch.uint8, ctas=ctas)
        l2 = fp8_stage(wd[1], 1, scales[1:3], 0)
        c2 = direct(l2, c1, n, ws[1].shape[0], torch.uint8, ctas=ctas)
        l3 = fp8_stage(wd[2], 0, scales[2:3], 1)
        i3, _, z3 = direct(l3, c2, n, top_k=1, logits_cols=ws[2].shape[0], ctas=ctas)
    finally:
        for s in st:
            cm.camelot_stage_release(s)
    assert np.array_equal(z3.view(np.uint32), np.ascontiguousarray(lg, np.float32).view(np.uint32))
    assert np.array_equal(i3[:, 0], np.asarray(idx).reshape(n, -1)[:, 0])
    res = {"queries": n}
    codes = [orc.e4m3_decode(c.cpu().numpy()) for c in (c0, c1, c2)]
    x = np.ascontiguousarray(x_u8, np.uint8).reshape(n, -1).astype(np.float64)
    assert np.array_equal(codes[0], orc.round_e4m3((x - 127.5) * 2.0))
    emul = [codes[0]]
    for l in range(2):
        sw, wq = orc.quantize_e4m3(ws[l])
        vs = orc.f32(sw * scales[l])
        own, lo, hi = tb.e4m3_layer_bracket(orc, codes[l], wq, vs, 1, scales[l + 1])
        assert np.all((codes[l + 1] >= lo) & (codes[l + 1] <= hi)), l
        res[f"layer{l + 1}_codes_equal_to_oracle"] = float(np.mean(codes[l + 1] == own))
        _, yq, _ = orc.linear_fp8(emul[l], wq, vs, 1, scales[l + 1])
        emul.append(yq)
    sw, wq = orc.quantize_e4m3(ws[2])
    vs = orc.f32(sw * scales[2])
    z, e = tb.logits_bound(orc, codes[2], wq, kstep=32, vscale=vs)
    err = np.abs(z3 - z)
    assert np.all(err <= e), float((err / e).max())
    res["logits_max_err_over_bound"] = float((err / e).max())
    res["argmax_fixed_on_gpu_input"] = tb.check_topk(i3, z, e, 1)
    z_emul, _, _ = orc.linear_fp8(emul[2], wq, vs, 0)
    e_all = e + vs * (np.abs(codes[2] - emul[2]) @ np.abs(wq).T)
    assert np.all(np.abs(z3 - z_emul) <= e_all)
    res["argmax_fixed_vs_emulated"] = tb.check_topk(i3, z_emul, e_all, 1)
    res["hidden2_rows_equal_emulated"] = float(np.mean(np.all(codes[2] == emul[2], axis=1)))
    return res
