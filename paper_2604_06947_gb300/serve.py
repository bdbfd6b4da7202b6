"""Serving driver: a stream of independent problems through the batched path.

Marshalling and scheduling only: requests are handed to the library's batch
(fqnm_batch_*) when their scheduled arrival time passes, the library admits
and steps them, and finished states are collected.  The same stream can be run
one problem at a time through the single-problem path (fqnm_create / load /
step), the baseline the batched path is compared with.
"""
from __future__ import annotations

import time
from typing import Dict, List, Optional

import numpy as np

from . import fqnm as F
from . import inputs as I


def prepare(requests: List[I.ServeRequest]) -> List[np.ndarray]:
    """Quantise every request's initial field on the GPU (eq. quantisation,
    once per problem), before the clock starts."""
    out = []
    for rq in requests:
        p = I.materialise(rq)
        out.append(F.fqnm_quantise(p.u0, p.delta))
        p.u0 = None
    return out


class DeviceStream:
    """Initial states of a whole request stream resident on the GPU (one int32
    buffer, problem i at offs[i]), and a buffer for the final states."""

    def __init__(self, requests: List[I.ServeRequest]):
        import torch
        self.ns = np.array([rq.problem.n for rq in requests], dtype=np.int64)
        self.offs = np.concatenate([[0], np.cumsum(self.ns)[:-1]])
        total = int(self.ns.sum())
        self.q = torch.empty(total, dtype=torch.int32, device="cuda")
        self.out = torch.empty(total, dtype=torch.int32, device="cuda")
        for i, rq in enumerate(requests):
            p = I.materialise(rq)
            u = torch.from_numpy(p.u0).cuda()
            F.fqnm_quantise_device(u, p.n, p.delta, self.q_ptr(i))
            p.u0 = None
        torch.cuda.synchronize()

    def q_ptr(self, i: int) -> int:
        return self.q.data_ptr() + 4 * int(self.offs[i])

    def out_ptr(self, i: int) -> int:
        return self.out.data_ptr() + 4 * int(self.offs[i])

    def q0(self, i: int):
        return self.q[int(self.offs[i]):int(self.offs[i] + self.ns[i])]

    def result(self, i: int):
        return self.out[int(self.offs[i]):int(self.offs[i] + self.ns[i])]


def _percentiles(lat_ns: np.ndarray) -> Dict[str, float]:
    return {"p50_ms": float(np.percentile(lat_ns, 50) / 1e6),
            "p99_ms": float(np.percentile(lat_ns, 99) / 1e6),
            "max_ms": float(lat_ns.max() / 1e6)}


def serve_batched(requests: List[I.ServeRequest], q0s=None,
                  budget_bytes: int = 16 << 30, max_slots: int = 1024,
                  plan: Optional[dict] = None, keep: Optional[set] = None,
                  lead_s: float = 0.02, dev: Optional[DeviceStream] = None,
                  deadline_s: float = 600.0, margin: Optional[int] = None) -> dict:
    """Run the stream through one batch in real time.

    q0s: host initial states (host submission), or dev: a DeviceStream whose
    initial and final states stay on the GPU (device submission).
    keep: request indices whose host final states are returned (all if None).
    """
    b = F.fqnm_batch_create(budget_bytes, max_slots)
    try:
        if margin is not None:
            F.fqnm_batch_set_margin(b, margin)
        if plan == "autotune":
            F.fqnm_batch_autotune(b, 3)
        elif plan:
            F.fqnm_batch_set_plan(b, **plan)
        specs = [F.make_spec(rq.problem) for rq in requests]
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival_s)
        lat = np.zeros(len(requests), dtype=np.int64)
        results: Dict[int, np.ndarray] = {}
        id2req: Dict[int, int] = {}
        t0 = F.fqnm_clock_ns() + int(lead_s * 1e9)
        nxt, done, t_last = 0, 0, t0
        t_stop = t0 + int(deadline_s * 1e9)
        while done < len(requests):
            now = F.fqnm_clock_ns()
            if now > t_stop:
                raise TimeoutError("serving did not finish within %.0f s (%d of %d done)"
                                   % (deadline_s, done, len(requests)))
            while nxt < len(order):
                i = order[nxt]
                t_arr = t0 + int(requests[i].arrival_s * 1e9)
                if t_arr > now:
                    break
                if dev is None:
                    rid = F.fqnm_batch_submit(b, specs[i], q0s[i], requests[i].problem.steps,
                                              t_arr)
                else:
                    rid = F.fqnm_batch_submit_device(b, specs[i], dev.q_ptr(i),
                                                     requests[i].problem.n,
                                                     requests[i].problem.steps, t_arr,
                                                     dev.out_ptr(i))
                id2req[rid] = i
                nxt += 1
            active, queued = F.fqnm_batch_progress(b, 1)
            for rid in F.fqnm_batch_completed(b):
                i = id2req[rid]
                q, l = F.fqnm_batch_poll(b, rid, requests[i].problem.n)
                lat[i] = l
                if dev is None and (keep is None or i in keep):
                    results[i] = q
                done += 1
                t_last = F.fqnm_clock_ns()
            if active == 0 and queued == 0 and nxt < len(order):
                wait = (t0 + int(requests[order[nxt]].arrival_s * 1e9) - F.fqnm_clock_ns()) / 1e9
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        stats = F.fqnm_batch_stats(b)
        final_plan = F.fqnm_batch_get_plan(b)
    finally:
        F.fqnm_batch_destroy(b)
    work = sum(rq.problem.n * rq.problem.steps for rq in requests)
    makespan = (t_last - t0) / 1e9
    out = {"requests": len(requests), "cell_updates": work,
           "makespan_s": makespan, "value": work / makespan,
           "gpu_s": stats["gpu_ms"] / 1e3, "value_gpu": work / (stats["gpu_ms"] / 1e3),
           "launches": stats["launches"], "epochs": stats["epochs"],
           "plan": final_plan, "latency_ns": lat, "results": results}
    out.update(_percentiles(lat))
    return out


def serve_one_by_one(requests: List[I.ServeRequest], q0s=None,
                     keep: Optional[set] = None, dev: Optional[DeviceStream] = None,
                     out=None) -> dict:
    """Each problem alone through the single-problem path, in arrival order;
    latencies from a FIFO queue over the measured service times.  With dev,
    states are loaded from and returned to device memory (out: a device
    int32 buffer laid out like dev.out)."""
    order = sorted(range(len(requests)), key=lambda i: requests[i].arrival_s)
    service = np.zeros(len(requests))
    results: Dict[int, np.ndarray] = {}
    for i in order:
        p = requests[i].problem
        t = time.perf_counter()
        s = F.Solver.for_problem(p)
        if dev is None:
            s.load(q0s[i]).step(p.steps)
            q = s.state()
        else:
            s.load_device(dev.q_ptr(i), p.n).step(p.steps)
            F.fqnm_checkpoint_device(s.h, out.data_ptr() + 4 * int(dev.offs[i]))
            F.fqnm_sync(s.h)
            q = None
        s.close()
        service[i] = time.perf_counter() - t
        if q is not None and (keep is None or i in keep):
            results[i] = q
    finish, lat = 0.0, np.zeros(len(requests), dtype=np.int64)
    for i in order:
        start = max(finish, requests[i].arrival_s)
        finish = start + service[i]
        lat[i] = int((finish - requests[i].arrival_s) * 1e9)
    work = sum(rq.problem.n * rq.problem.steps for rq in requests)
    out = {"requests": len(requests), "cell_updates": work,
           "busy_s": float(service.sum()), "value": work / float(service.sum()),
           "latency_ns": lat, "results": results}
    out.update(_percentiles(lat))
    return out
