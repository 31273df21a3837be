"""GPU parity and invariants of the persistent SM-partitioned pipeline
(camelot_pipeline_create / submit / submit_trace / poll) on the plain 2-stage
workload (normalise -> 12288-512-256-10 ReLU MLP -> argmax):

* results match the FP64 oracle (argmax exact where the margin is clear,
  logits within the FP32 bound);
* every query ID comes back exactly once and in order (Sec. 5.2);
* results do not depend on the handoff mechanism (global memory, Sec. 6.2, or
  host-staged, Sec. 4.2), on the SM partition (Eq. 1's N_i, p_i) or on the
  batches queries travel in;
* back-pressure, trace replay, idle exit and relaunch behave as documented."""
import time

import numpy as np
import pytest
import torch

from gpu_common import argmax_margin_ok, cfg1_data, chain_bound, first_argmax

pytestmark = pytest.mark.gpu

cm = pl = None
N_Q = 256


@pytest.fixture(scope="module")
def stages():
    global cm, pl
    from paper_2005_02088_b300 import camelot as _cm, pipelines as _pl
    cm, pl = _cm, _pl
    x, ws = cfg1_data(N_Q)
    s0 = pl.stage_normalize(64, 64, 3, max_batch=32)
    wd = [torch.from_numpy(w).cuda() for w in ws]
    s1 = pl.stage_dense(cm.STAGE_MLP_FP32, wd, [cm.ACT_RELU, cm.ACT_RELU, cm.ACT_NONE], top_k=1,
                        max_batch=32)
    yield s0, s1
    cm.camelot_stage_release(s0)
    cm.camelot_stage_release(s1)


def _run(stages, mode, inst=(1, 1), quota=(8, 16), batch=16, opts=None, n=N_Q, chunk=64):
    x, _ = cfg1_data(N_Q)
    sink = torch.zeros((65536, 10), dtype=torch.float32, device="cuda")
    o = opts or pl.options()
    o.logits_sink = sink.data_ptr()
    torch.cuda.synchronize()
    p = cm.camelot_pipeline_create(list(stages), pl.alloc(list(inst), list(quota), batch), mode, o)
    try:
        comps = pl.run_all(p, x[:n], stream_id=7, chunk=chunk)
        stats = cm.camelot_pipeline_stats(p)
    finally:
        cm.camelot_pipeline_destroy(p)
    logits = sink[:n].cpu().numpy()
    return comps, logits, stats


def _check_against_oracle(orc, comps, logits, n=N_Q):
    x, ws = cfg1_data(N_Q)
    assert [c.query_id for c in comps] == list(range(n))
    assert all(c.stream_id == 7 and c.status == 0 for c in comps)
    z64, bound = chain_bound(orc, x[:n], ws, [1, 1, 0])
    assert np.all(np.abs(logits - z64) <= bound + 1e-30)
    idx = np.array([c.idx[0] for c in comps])
    assert np.array_equal(idx, first_argmax(logits))          # integer result: exact
    assert np.array_equal(np.array([c.val[0] for c in comps], np.float32),
                          logits[np.arange(n), idx])
    ok = argmax_margin_ok(z64, np.abs(logits - z64))
    assert np.array_equal(idx[ok], np.argmax(z64, axis=1)[ok])
    assert np.mean(idx == np.argmax(z64, axis=1)) >= 0.99
    assert all(c.idx[1] == -1 for c in comps)
    for c in comps:
        assert c.t_batch_ns <= c.t_done_ns and 1 <= c.batch_size <= 16


def test_global_handoff_matches_oracle(orc, stages):
    comps, logits, stats = _run(stages, 0)
    _check_against_oracle(orc, comps, logits)
    assert stats.completed == N_Q and stats.relayed_bytes == 0


def test_host_staged_identical_to_global(orc, stages):
    c0, l0, _ = _run(stages, 0)
    c1, l1, st1 = _run(stages, 1)
    _check_against_oracle(orc, c1, l1)
    assert np.array_equal(l0, l1)
    assert [c.idx[0] for c in c0] == [c.idx[0] for c in c1]
    assert st1.relayed_bytes > 0
    # one device copy per in-flight batch with the global handoff, two when staged
    # through the host (Sec. 6.2's memory saving)
    _, _, st0 = _run(stages, 0, n=32)
    assert st1.device_ring_bytes == 2 * st0.device_ring_bytes


@pytest.mark.parametrize("inst,quota,batch", [((1, 1), (1, 1), 16), ((2, 3), (4, 8), 16),
                                              ((1, 4), (8, 8), 5), ((3, 2), (2, 24), 32)])
def test_result_independent_of_partition_and_batch(stages, inst, quota, batch):
    _, ref, _ = _run(stages, 0)
    comps, logits, _ = _run(stages, 0, inst, quota, batch)
    assert [c.query_id for c in comps] == list(range(N_Q))
    assert np.array_equal(logits, ref)


def test_trace_replay_device_resident(orc, stages):
    x, _ = cfg1_data(N_Q)
    xd = torch.from_numpy(x).cuda()
    off = torch.from_numpy(np.arange(N_Q, dtype=np.int64) * 20000).cuda()   # 50k qps
    sink = torch.zeros((65536, 10), dtype=torch.float32, device="cuda")
    o = pl.options(logits_sink=sink.data_ptr())
    torch.cuda.synchronize()
    p = cm.camelot_pipeline_create(list(stages), pl.alloc([1, 2], [8, 16], 16), 0, o)
    try:
        first = cm.camelot_submit_trace(p, 7, xd, N_Q, off)
        assert first == 0
        buf = (cm.Completion * 1024)()
        comps = []
        t_end = time.time() + 30
        while len(comps) < N_Q and time.time() < t_end:
            k = cm.camelot_poll(p, buf, timeout_us=1000)
            comps += [pl._copy(buf[i]) for i in range(k)]
        # host submissions continue after the trace with the next IDs
        more = cm.camelot_submit(p, 7, x[:3], 3)
        assert more == N_Q
        while len(comps) < N_Q + 3 and time.time() < t_end:
            k = cm.camelot_poll(p, buf, timeout_us=1000)
            comps += [pl._copy(buf[i]) for i in range(k)]
    finally:
        cm.camelot_pipeline_destroy(p)
    logits = sink[:N_Q + 3].cpu().numpy()
    _check_against_oracle(orc, comps[:N_Q], logits[:N_Q])
    assert np.array_equal(logits[N_Q:], logits[:3])
    arr = np.array([c.t_arrival_ns for c in comps[:N_Q]])
    assert np.all(np.diff(arr) == 20000)                     # device-clock arrivals
    assert all(c.t_batch_ns >= c.t_arrival_ns for c in comps[:N_Q])


def test_backpressure_eagain_then_drain(stages):
    x, _ = cfg1_data(N_Q)
    o = pl.options(query_slots=64)
    p = cm.camelot_pipeline_create(list(stages), pl.alloc([1, 1], [8, 8], 16), 0, o)
    try:
        assert cm.camelot_submit(p, 0, x[:64], 64) == 0
        assert cm.camelot_submit(p, 0, x[:1], 1, allow_eagain=True) is None   # ring full
        buf = (cm.Completion * 64)()
        got = 0
        t_end = time.time() + 20
        while got < 64 and time.time() < t_end:
            got += cm.camelot_poll(p, buf, timeout_us=1000)
        assert got == 64
        assert cm.camelot_submit(p, 0, x[:1], 1) == 64
    finally:
        cm.camelot_pipeline_destroy(p)


def test_empty_inputs(stages):
    """n = 0: a submit queues nothing, launches nothing and returns the next ID;
    an empty or over-long trace is EINVAL; a poll with nothing outstanding times
    out empty.  The pipeline then runs normally."""
    x, _ = cfg1_data(N_Q)
    p = cm.camelot_pipeline_create(list(stages), pl.alloc([1, 1], [8, 8], 16), 0,
                                   pl.options(query_slots=64))
    try:
        assert cm.camelot_submit(p, 0, None, 0) == 0
        buf = (cm.Completion * 8)()
        assert cm.camelot_poll(p, buf, timeout_us=2000) == 0
        st = cm.camelot_pipeline_stats(p)
        assert st.submitted == 0 and st.completed == 0 and st.kernel_launches == 0
        xd = torch.from_numpy(x[:1]).cuda()
        off = torch.zeros(65, dtype=torch.int64, device="cuda")
        for n in (0, 65):                     # empty; longer than query_slots
            with pytest.raises(cm.CamelotError) as e:
                cm.camelot_submit_trace(p, 0, xd, n, off)
            assert e.value.status == cm.EINVAL
        assert cm.camelot_submit(p, 0, x[:3], 3) == 0
        comps, t_end = [], time.time() + 20
        while len(comps) < 3 and time.time() < t_end:
            k = cm.camelot_poll(p, buf, timeout_us=1000)
            comps += [pl._copy(buf[i]) for i in range(k)]
        assert [c.query_id for c in comps] == [0, 1, 2] and all(c.status == 0 for c in comps)
        assert cm.camelot_submit(p, 0, None, 0) == 3
    finally:
        cm.camelot_pipeline_destroy(p)


def test_trace_fills_every_query_slot(stages):
    """The longest trace allowed (n = query_slots): every slot of the completion
    ring in use at once; results equal the host-submitted run."""
    _, ref, _ = _run(stages, 0)
    x, _ = cfg1_data(N_Q)
    xd = torch.from_numpy(x).cuda()
    off = torch.zeros(N_Q, dtype=torch.int64, device="cuda")
    sink = torch.zeros((65536, 10), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    p = cm.camelot_pipeline_create(list(stages), pl.alloc([1, 2], [8, 16], 16), 0,
                                   pl.options(query_slots=N_Q, logits_sink=sink.data_ptr()))
    try:
        assert cm.camelot_submit_trace(p, 7, xd, N_Q, off) == 0
        buf = (cm.Completion * N_Q)()
        comps, t_end = [], time.time() + 30
        while len(comps) < N_Q and time.time() < t_end:
            k = cm.camelot_poll(p, buf, timeout_us=1000)
            comps += [pl._copy(buf[i]) for i in range(k)]
    finally:
        cm.camelot_pipeline_destroy(p)
    assert [c.query_id for c in comps] == list(range(N_Q))
    assert np.array_equal(sink[:N_Q].cpu().numpy(), ref)


def test_small_data_ring_wraps(stages):
    # 64 pinned query rows behind 256 descriptors: submissions wait for stage 0
    # to free data rows, results are unchanged
    _, ref, _ = _run(stages, 0)
    comps, logits, _ = _run(stages, 0, opts=pl.options(query_slots=256, data_slots=64), chunk=32)
    assert [c.query_id for c in comps] == list(range(N_Q))
    assert np.array_equal(logits, ref)


@pytest.mark.parametrize("data_slots,chunk", [(0, 64), (64, 48)])
def test_device_data_ring_identical(stages, data_slots, chunk):
    # query bytes DMA-copied into a device ring at submit (wrapping when the
    # ring is small): the same results as the mapped host ring
    _, ref, _ = _run(stages, 0)
    o = pl.options(query_slots=256, data_slots=data_slots, device_data=1)
    comps, logits, _ = _run(stages, 0, opts=o, chunk=chunk)
    assert [c.query_id for c in comps] == list(range(N_Q))
    assert np.array_equal(logits, ref)


def test_idle_exit_and_relaunch(stages):
    x, _ = cfg1_data(N_Q)
    o = pl.options(idle_exit_ns=20_000_000)
    p = cm.camelot_pipeline_create(list(stages), pl.alloc([1, 1], [8, 8], 16), 0, o)
    try:
        buf = (cm.Completion * 16)()
        for rnd in range(3):
            cm.camelot_submit(p, 0, x[:4], 4)
            got = 0
            t_end = time.time() + 10
            while got < 4 and time.time() < t_end:
                got += cm.camelot_poll(p, buf, timeout_us=1000)
            assert got == 4
            time.sleep(0.1)      # longer than the idle bound: the kernel exits
        st = cm.camelot_pipeline_stats(p)
        assert st.kernel_launches >= 3 and st.completed == 12 and st.device_status == 0
    finally:
        cm.camelot_pipeline_destroy(p)


def test_create_rejects_bad_allocations(stages):
    with pytest.raises(cm.CamelotError) as e:
        cm.camelot_pipeline_create(list(stages), pl.alloc([1, 1], [100, 100], 16), 0)
    assert e.value.status == cm.EINVAL              # more SMs than the GPU has
    with pytest.raises(cm.CamelotError) as e:
        cm.camelot_pipeline_create(list(stages)[::-1], pl.alloc([1, 1], [8, 8], 16), 0)
    assert e.value.status == cm.EINVAL              # rows do not chain
    with pytest.raises(cm.CamelotError) as e:
        cm.camelot_pipeline_create(list(stages), pl.alloc([1, 1], [8, 8], 64), 0)
    assert e.value.status == cm.EINVAL              # batch above the stage maximum
