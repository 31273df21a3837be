"""The batch trigger on the GPU against the oracle's simulator (Sec. 5.2 steps
1-2), and the device-side timeout path.

Trigger: a device-resident trace replayed on the device clock, with gaps far
longer than the pipeline's service time, so that every stage-0 instance is free
whenever a batch could leave.  The pipeline's QoS rule (QoS 5 ms less a 0.5 ms
margin, predicted batch latency 1 ms + 0.25 ms per query, wait cap 10 ms) lets
the oldest of k waiting queries wait 3.5 - 0.25 k ms.  The arrivals are placed
so that no decision falls within 0.1 ms of an arrival.  The issued batch sizes
must equal the oracle's (orc_simulate_qos) exactly, and each batch must leave
no earlier than the oracle says and at most SLACK later (the trigger polls).

Timeout: a host-staged pipeline whose relay thread is stalled on the host
(camelot_pipeline_stall_relay): the producer's bounded wait for a free slot
gives up after wait_limit_ns, the device records the error and every CTA
unwinds; the host reports ESTATE, destroy is clean, and a new pipeline on the
same GPU runs and matches the oracle.  Nothing is faulted on the GPU."""
import time

import numpy as np
import pytest
import torch

from gpu_common import cfg1_data, chain_bound

pytestmark = pytest.mark.gpu

MS = 1_000_000
SLACK_NS = 200_000
B = 8


def _burst_trace():
    """Arrival offsets (ns): bursts 20 ms apart, each ending in a decision of
    the QoS rule or a full batch."""
    bursts = [
        [0.0, 0.5, 1.0, 1.5, 2.0],          # k = 5 at 2.0 ms: bound 2.25 -> leaves at 2.25 with 5
        [0.05 * i for i in range(8)],       # full batch of 8 at 0.35 ms
        [0.0],                              # alone: bound 3.25 -> leaves at 3.25
        [0.0, 2.0, 2.9],                    # k = 3 at 2.9 ms: bound 2.75 passed -> leaves at once
        [0.0, 0.7, 1.4, 2.1],               # k = 4 at 2.1: bound 2.5 -> leaves at 2.5 with 4
        [0.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9],   # 8 full at 0.7, then 2 more: bound 3.0
    ]
    t, out = 0.0, []
    for b in bursts * 3:
        out += [t + a for a in b]
        t += 20.0
    return np.round(np.array(out) * MS).astype(np.int64)


def _lat_ns():
    return [1 * MS + (b + 1) * MS // 4 for b in range(32)]


def test_qos_trigger_matches_simulator(orc):
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    x, ws = cfg1_data(256)
    off = _burst_trace()
    n = off.size
    xq = torch.from_numpy(np.ascontiguousarray(x.reshape(256, -1))).cuda()[torch.arange(n).cuda() % 256]
    s0 = pl.stage_normalize(64, 64, 3, max_batch=B)
    s1 = pl.stage_dense(cm.STAGE_MLP_FP32, [torch.from_numpy(w).cuda() for w in ws], [1, 1, 0], top_k=1,
                        max_batch=B)
    try:
        o = pl.options(max_wait_ns=10 * MS, qos_ns=5 * MS, qos_margin_ns=MS // 2, exit_after_trace=1)
        for b, v in enumerate(_lat_ns()):
            o.batch_latency_ns[b] = v
        torch.cuda.synchronize()
        p = cm.camelot_pipeline_create([s0, s1], pl.alloc([1, 1], [8, 16], B), cm.HANDOFF_GLOBAL, o)
        try:
            cm.camelot_submit_trace(p, 4, xq, n, torch.from_numpy(off).cuda())
            buf = (cm.Completion * 4096)()
            comps, t_end = [], time.time() + 60
            while len(comps) < n and time.time() < t_end:
                k = cm.camelot_poll(p, buf, timeout_us=2000)
                comps += [pl._copy(buf[i]) for i in range(k)]
            assert cm.camelot_pipeline_stats(p).device_status == 0
        finally:
            cm.camelot_pipeline_destroy(p)
    finally:
        cm.camelot_stage_release(s0)
        cm.camelot_stage_release(s1)
    assert [c.query_id for c in comps] == list(range(n)) and all(c.status == 0 for c in comps)
    # batches as the device formed them: runs of queries with one t_batch
    firsts = [0] + [i for i in range(1, n) if comps[i].t_batch_ns != comps[i - 1].t_batch_ns]
    sizes = np.diff(firsts + [n])
    assert all(comps[i].batch_size == sizes[j] for j, f in enumerate(firsts) for i in range(f, f + sizes[j]))
    lag_dev = np.array([comps[f].t_batch_ns - comps[f].t_arrival_ns for f in firsts], np.float64)
    # the oracle: one stage-0 instance, service far below the gaps
    lat_s = np.array(_lat_ns()[:B]) * 1e-9
    _, bs, iss = orc.simulate_qos(off * 1e-9, B, 10e-3, 4.5e-3, lat_s, [1, 1],
                                  [[20e-6] * B, [50e-6] * B])
    assert sizes.tolist() == bs.tolist()
    starts = np.concatenate([[0], np.cumsum(bs)[:-1]])
    lag_sim = (iss - off[starts] * 1e-9) * 1e9
    d = lag_dev - lag_sim
    assert np.all(d >= -2_000) and np.all(d <= SLACK_NS), (d.min(), d.max())
    # the rule made a difference: partial batches left well before the 10 ms cap
    assert np.sum(bs < B) >= 9 and lag_sim.max() < 3.5 * MS


def test_device_wait_times_out_on_stalled_relay(orc):
    from paper_2005_02088_b300 import camelot as cm, pipelines as pl
    x, ws = cfg1_data(256)
    s0 = pl.stage_normalize(64, 64, 3, max_batch=16)
    s1 = pl.stage_dense(cm.STAGE_MLP_FP32, [torch.from_numpy(w).cuda() for w in ws], [1, 1, 0], top_k=1,
                        max_batch=16)
    try:
        torch.cuda.synchronize()
        o = pl.options(wait_limit_ns=50 * MS, batch_slots=4)
        p = cm.camelot_pipeline_create([s0, s1], pl.alloc([1, 1], [8, 8], 16), cm.HANDOFF_HOST_STAGED, o)
        try:
            cm.camelot_pipeline_stall_relay(p, True)
            q = np.ascontiguousarray(x.reshape(256, -1))
            cm.camelot_submit(p, 0, q, 256)          # 16 batches; the stage-0 ring holds 4
            buf = (cm.Completion * 256)()
            t0, err = time.time(), None
            while time.time() - t0 < 20:
                try:
                    got = cm.camelot_poll(p, buf, timeout_us=10_000)
                except cm.CamelotError as e:
                    err = e
                    break
                assert got == 0                       # nothing can complete while the relay stalls
            assert err is not None and err.status == cm.ESTATE, err
            waited = time.time() - t0
            st = cm.camelot_pipeline_stats(p)
            assert st.device_status == 2             # no free output slot in time
            assert waited < 10, waited
            with pytest.raises(cm.CamelotError) as e2:
                cm.camelot_submit(p, 0, q, 1)
            assert e2.value.status == cm.ESTATE
        finally:
            cm.camelot_pipeline_destroy(p)
        # the GPU is fine: a new pipeline runs and matches the oracle
        sink = torch.zeros((65536, 10), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        p = cm.camelot_pipeline_create([s0, s1], pl.alloc([1, 1], [8, 8], 16), cm.HANDOFF_HOST_STAGED,
                                       pl.options(logits_sink=sink.data_ptr()))
        try:
            comps = pl.run_all(p, x[:64], stream_id=1)
        finally:
            cm.camelot_pipeline_destroy(p)
        assert [c.query_id for c in comps] == list(range(64)) and all(c.status == 0 for c in comps)
        z64, bound = chain_bound(orc, x[:64], ws, [1, 1, 0])
        assert np.all(np.abs(sink[:64].cpu().numpy() - z64) <= bound + 1e-30)
    finally:
        cm.camelot_stage_release(s0)
        cm.camelot_stage_release(s1)
