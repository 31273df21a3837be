"""GPU parity of single stages, launched directly through the C-ABI
(camelot_stage_launch), against the FP64 oracle: bit-exact normalisation and
2x2 pooling, FP32 dense layers within the stated tolerance, and results that
do not depend on the SM quota or on the batch a query travels in."""
import numpy as np
import pytest
import torch

from gpu_common import FP32_REL, argmax_margin_ok, cfg1_data, chain_bound, first_argmax

pytestmark = pytest.mark.gpu

cm = None
pl = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global cm, pl
    from paper_2005_02088_b300 import camelot as _cm, pipelines as _pl
    cm, pl = _cm, _pl
    assert torch.cuda.is_available()
    cm.load()
    yield


def _scratch(st, n):
    _, _, sb = cm.camelot_stage_info(st, n)
    return torch.empty(sb + 256, dtype=torch.uint8, device="cuda"), sb


def _launch(st, n_ctas, inp, n, out=None, idx=None, val=None, logits=None):
    scr, sb = _scratch(st, n)
    cm.camelot_stage_launch(st, n_ctas, inp, n, out, idx, val, logits, scr, sb, None)
    torch.cuda.synchronize()


@pytest.mark.parametrize("n", [1, 7, 16, 33])
def test_normalize_bit_exact(orc, n):
    x = np.random.default_rng(n).integers(0, 256, size=(n, 64, 64, 3), dtype=np.uint8)
    st = pl.stage_normalize(64, 64, 3, max_batch=64)
    try:
        xd = torch.from_numpy(x).cuda()
        out = torch.empty((n, 12288), dtype=torch.float32, device="cuda")
        _launch(st, 5, xd, n, out=out)
        ref = orc.normalize_u8(x.reshape(n, -1))
        assert np.array_equal(out.cpu().numpy().astype(np.float64), ref)
    finally:
        cm.camelot_stage_release(st)


@pytest.mark.parametrize("n,H,W", [(1, 224, 224), (5, 224, 224), (3, 8, 16)])
def test_norm_pool2_bit_exact(orc, n, H, W):
    x = np.random.default_rng(H + n).integers(0, 256, size=(n, H, W, 3), dtype=np.uint8)
    st = pl.stage_norm_pool2(H, W, 3, max_batch=32)
    try:
        out = torch.empty((n, (H // 2) * (W // 2) * 3), dtype=torch.bfloat16, device="cuda")
        _launch(st, 7, torch.from_numpy(x).cuda(), n, out=out)
        ref = orc.bf16_bits(orc.norm_pool2(x))
        got = out.view(torch.int16).cpu().numpy().view(np.uint16)
        assert np.array_equal(got, ref)
    finally:
        cm.camelot_stage_release(st)


def _layer_check(orc, xin, w, act, out):
    ref, absdot = orc.linear(xin.astype(np.float64), w.astype(np.float64), act, want_absdot=True)
    err = np.abs(out.astype(np.float64) - ref)
    assert np.all(err <= FP32_REL * absdot + 1e-30), float((err / (absdot + 1e-30)).max())


@pytest.mark.parametrize("K,N,act,n", [(12288, 512, 1, 16), (512, 256, 1, 16), (512, 256, 1, 5),
                                       (12288, 512, 0, 1), (100, 200, 2, 3), (48, 1000, 0, 17)])
def test_dense_layer_tolerance(orc, K, N, act, n):
    g = np.random.default_rng(K + N + n)
    x = g.standard_normal((n, K)).astype(np.float32)
    w = (g.standard_normal((N, K)) / np.sqrt(K)).astype(np.float32)
    wd = torch.from_numpy(w).cuda()
    st = pl.stage_dense(cm.STAGE_MLP_FP32, [wd], [act], top_k=0, max_batch=64)
    try:
        out = torch.empty((n, N), dtype=torch.float32, device="cuda")
        _launch(st, 11, torch.from_numpy(x).cuda(), n, out=out)
        _layer_check(orc, x, w, act, out.cpu().numpy())
    finally:
        cm.camelot_stage_release(st)


def _mlp_stage(ws, top_k=1):
    wd = [torch.from_numpy(w).cuda() for w in ws]
    return pl.stage_dense(cm.STAGE_MLP_FP32, wd, [cm.ACT_RELU, cm.ACT_RELU, cm.ACT_NONE],
                          top_k=top_k, max_batch=64)


def _run_mlp(st, y, n, n_ctas, k=1):
    idx = torch.empty((n, k), dtype=torch.int32, device="cuda")
    val = torch.empty((n, k), dtype=torch.float32, device="cuda")
    logits = torch.empty((n, 10), dtype=torch.float32, device="cuda")
    _launch(st, n_ctas, y, n, idx=idx, val=val, logits=logits)
    return idx.cpu().numpy(), val.cpu().numpy(), logits.cpu().numpy()


def test_mlp_stage_vs_fp64_chain(orc):
    x, ws = cfg1_data(256)
    n = 16
    y = torch.from_numpy(((x[:n].reshape(n, -1).astype(np.float32) - 127.5) / 64)).cuda()
    st = _mlp_stage(ws)
    try:
        idx, val, logits = _run_mlp(st, y, n, 24)
        z64, bound = chain_bound(orc, x[:n], ws, [1, 1, 0])
        assert np.all(np.abs(logits - z64) <= bound + 1e-30)
        assert np.array_equal(idx[:, 0], first_argmax(logits))
        ok = argmax_margin_ok(z64, np.abs(logits - z64))
        assert np.array_equal(idx[ok, 0], np.argmax(z64, axis=1)[ok])
        assert np.mean(idx[:, 0] == np.argmax(z64, axis=1)) >= 15 / 16
        assert np.array_equal(val[:, 0], logits[np.arange(n), idx[:, 0]])
    finally:
        cm.camelot_stage_release(st)


def test_mlp_stage_independent_of_sm_quota_and_batch(orc):
    x, ws = cfg1_data(256)
    n = 16
    y = torch.from_numpy(((x[:n].reshape(n, -1).astype(np.float32) - 127.5) / 64)).cuda()
    st = _mlp_stage(ws, top_k=3)
    try:
        base = _run_mlp(st, y, n, 1, k=3)
        for n_ctas in (8, 37, 64, 72, 144, 148):   # 128- and 64-neuron task blocks
            got = _run_mlp(st, y, n, n_ctas, k=3)
            for a, b in zip(base, got):
                assert np.array_equal(a, b), n_ctas
        for q in (0, 5, 15):   # alone vs in the batch
            alone = _run_mlp(st, y[q:q + 1].contiguous(), 1, 8, k=3)
            for a, b in zip(alone, base):
                assert np.array_equal(a[0], b[q])
    finally:
        cm.camelot_stage_release(st)


def test_topk_large_width_matches_sort(orc):
    # final task layer (N > 32) followed by the warp top-k over 1000 logits
    g = np.random.default_rng(9)
    n, K, N = 9, 64, 1000
    x = g.standard_normal((n, K)).astype(np.float32)
    w = (g.standard_normal((N, K)) / 8).astype(np.float32)
    w[7] = w[3]   # an exact tie: lower index first
    st = pl.stage_dense(cm.STAGE_MLP_FP32, [torch.from_numpy(w).cuda()], [0], top_k=5, max_batch=16)
    try:
        idx = torch.empty((n, 5), dtype=torch.int32, device="cuda")
        val = torch.empty((n, 5), dtype=torch.float32, device="cuda")
        logits = torch.empty((n, N), dtype=torch.float32, device="cuda")
        _launch(st, 3, torch.from_numpy(x).cuda(), n, idx=idx, val=val, logits=logits)
        lg = logits.cpu().numpy()
        ref_idx, ref_val = orc.topk(lg.astype(np.float64), 5)
        assert np.array_equal(idx.cpu().numpy(), ref_idx)
        assert np.array_equal(val.cpu().numpy(), ref_val.astype(np.float32))
        _layer_check(orc, x, w, 0, lg)
    finally:
        cm.camelot_stage_release(st)


def test_launch_rejects_bad_arguments():
    st = pl.stage_normalize(64, 64, 3, max_batch=4)
    try:
        buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
        with pytest.raises(cm.CamelotError) as e:
            cm.camelot_stage_launch(st, 1, buf, 5, buf, None, None, None, buf, 1 << 20, None)
        assert e.value.status == cm.EINVAL        # n > max_batch
        with pytest.raises(cm.CamelotError) as e:
            cm.camelot_stage_launch(st, 1, buf, 0, buf, None, None, None, buf, 1 << 20, None)
        assert e.value.status == cm.EINVAL        # empty batch
        with pytest.raises(cm.CamelotError) as e:
            cm.camelot_stage_launch(st, 10000, buf, 1, buf, None, None, None, buf, 1 << 20, None)
        assert e.value.status == cm.EINVAL        # more CTAs than SMs
    finally:
        cm.camelot_stage_release(st)
