"""Two stages in two processes, handing batches over through the library's
cross-process ring (Sec. 6.2: in the paper every microservice is a process,
and the next stage maps the previous one's global-memory output through a CUDA
IPC handle instead of receiving a host copy).

The producer process runs the first stage with direct launches, writing each
batch into a ring slot; the consumer process maps the ring (camelot_xring_open)
and runs the second stage on the slot in place.  The GPU orders the two sides
by stream waits on the ring's inter-process events; the host sides tell each
other which slot they recorded over a pipe.  Processes are started with the
spawn method (CUDA cannot be forked).

Stage specifications are plain data, so that they travel to the child
processes:  {"kind": "normalize", "dims": (H, W, C)} or
{"kind": "mlp_fp32", "weights": [float32 arrays [out, in]], "acts": [...],
"top_k": k}.
"""
from __future__ import annotations

import multiprocessing as mp
import time

import numpy as np


def _build(spec: dict, max_batch: int):
    import torch

    from . import camelot as cm, pipelines as pl
    if spec["kind"] == "normalize":
        return pl.stage_normalize(*spec["dims"], max_batch), []
    if spec["kind"] == "mlp_fp32":
        ws = [torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda() for w in spec["weights"]]
        return pl.stage_dense(cm.STAGE_MLP_FP32, ws, spec["acts"], spec["top_k"], max_batch), ws
    raise ValueError(f"unknown stage kind {spec['kind']!r}")


def _producer(ctrl, conn, spec, queries, B, slots, ctas, paced):
    import torch

    from . import camelot as cm
    torch.cuda.set_device(0)
    st, keep = _build(spec, B)
    x = None
    try:
        _, out_row, sb = cm.camelot_stage_info(st, B)
        t0 = time.perf_counter()
        x, handle = cm.camelot_xring_create(B * out_row, slots)
        t_create = time.perf_counter() - t0
        ctrl.send(("handle", handle, t_create))
        q = torch.from_numpy(np.ascontiguousarray(queries)).cuda()
        scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        assert ctrl.recv()[0] == "go"
        n = q.shape[0]
        nb = (n + B - 1) // B
        free_seen = set(range(slots))
        for b in range(nb):
            k = b % slots
            while k not in free_seen:
                msg = conn.recv()
                if msg[0] == "free":
                    free_seen.add(msg[1])
            free_seen.discard(k)
            nbq = min(B, n - b * B)
            cm.camelot_xring_produce_begin(x, k, stream.cuda_stream)
            cm.camelot_stage_launch(st, ctas, q[b * B:b * B + nbq], nbq, cm.camelot_xring_slot(x, k), None, None,
                                    None, scr, sb, stream.cuda_stream)
            cm.camelot_xring_produce_end(x, k, stream.cuda_stream)
            conn.send(("ready", k, nbq, b, time.perf_counter_ns()))
            if paced:
                while True:
                    msg = conn.recv()
                    if msg[0] == "free":
                        free_seen.add(msg[1])
                    elif msg[0] == "done" and msg[1] == b:
                        break
        conn.send(("end",))
        stream.synchronize()
        while ctrl.recv()[0] != "closed":
            pass
    finally:
        if x is not None:
            cm.camelot_xring_destroy(x)
        cm.camelot_stage_release(st)
        del keep


def _consumer(ctrl, conn, spec, B, ctas, top_k, paced):
    import torch

    from . import camelot as cm
    torch.cuda.set_device(0)
    msg = ctrl.recv()
    assert msg[0] == "handle"
    t0 = time.perf_counter()
    x = cm.camelot_xring_open(msg[1])
    t_open = time.perf_counter() - t0
    st, keep = _build(spec, B)
    try:
        _, _, sb = cm.camelot_stage_info(st, B)
        scr = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
        slots = 64
        idx = torch.empty((slots, B, top_k), dtype=torch.int32, device="cuda")
        val = torch.empty((slots, B, top_k), dtype=torch.float32, device="cuda")
        host = []
        stream = torch.cuda.Stream()
        lat = []
        ctrl.send(("opened", t_open))
        t_first = None
        while True:
            msg = conn.recv()
            if msg[0] == "end":
                break
            _, k, nbq, b, t_sent = msg
            if t_first is None:
                t_first = time.perf_counter()
            cm.camelot_xring_consume_begin(x, k, stream.cuda_stream)
            cm.camelot_stage_launch(st, ctas, cm.camelot_xring_slot(x, k), nbq, None, idx[k], val[k], None, scr, sb,
                                    stream.cuda_stream)
            cm.camelot_xring_consume_end(x, k, stream.cuda_stream)
            with torch.cuda.stream(stream):
                h = torch.empty((nbq, top_k), dtype=torch.int32, pin_memory=True)
                h.copy_(idx[k, :nbq], non_blocking=True)
            host.append(h)
            conn.send(("free", k))
            if paced:
                stream.synchronize()
                lat.append((time.perf_counter_ns() - t_sent) * 1e-9)
                conn.send(("done", b))
        stream.synchronize()
        t_all = time.perf_counter() - (t_first or time.perf_counter())
        ctrl.send(("result", np.concatenate([h.numpy() for h in host]), t_all, lat))
        ctrl.recv()   # the parent's acknowledgement
    finally:
        cm.camelot_xring_destroy(x)
        cm.camelot_stage_release(st)
        del keep


def run_split(producer_spec: dict, consumer_spec: dict, queries: np.ndarray, batch: int, top_k: int,
              slots: int = 8, ctas=(16, 64), paced: bool = False, timeout_s: float = 120.0) -> dict:
    """Run `queries` (rows of the producer stage's input) through the two
    stages in two processes.  Returns the consumer's top-k indices [n, top_k],
    the ring setup times (create in the producer, open in the consumer, s), the
    consumer's wall time from its first batch to its last result (s), and, when
    `paced` (one batch in flight), the per-batch latency from the producer's
    launch to the consumer's result (s)."""
    ctx = mp.get_context("spawn")
    ctl_p, ctl_p_child = ctx.Pipe()        # parent <-> producer
    ctl_c, ctl_c_child = ctx.Pipe()        # parent <-> consumer
    link_p, link_c = ctx.Pipe()            # producer <-> consumer (slot messages)
    pp = ctx.Process(target=_producer, args=(ctl_p_child, link_p, producer_spec, queries, batch, slots, ctas[0],
                                             paced))
    pc = ctx.Process(target=_consumer, args=(ctl_c_child, link_c, consumer_spec, batch, ctas[1], top_k, paced))
    pp.start()
    pc.start()
    out = {}
    try:
        deadline = time.time() + timeout_s

        def recv(c):
            while not c.poll(0.05):
                if time.time() > deadline or not (pp.is_alive() and pc.is_alive()):
                    raise RuntimeError("cross-process run failed or timed out")
            return c.recv()

        msg = recv(ctl_p)
        out["ring_create_s"] = msg[2]
        ctl_c.send(msg)
        out["ring_open_s"] = recv(ctl_c)[1]
        ctl_p.send(("go",))
        m = recv(ctl_c)
        out["idx"], out["consumer_s"], out["latency_s"] = m[1], m[2], m[3]
        ctl_c.send(("ack",))
        pc.join(timeout_s)
        ctl_p.send(("closed",))
        pp.join(timeout_s)
    finally:
        for p in (pp, pc):
            if p.is_alive():
                p.terminate()
                p.join(5)
    return out
