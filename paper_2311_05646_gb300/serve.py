"""Continuous-batching service for eps-build and gradient requests.

Clients (designs under optimisation) keep their design, their forward and
adjoint fields and their output buffers resident on the device for their
whole optimisation run.  Each client issues requests one at a time (an eps
build, then a gradient, then the next parameter update -- steps 2 and 5 of
the protocol of Sec. 2, repeated as in step 7).  The service loop:

* admits a new client only when its resident footprint -- the bytes libadg
  reports for its compiled design (adg_design_bytes) plus its fields, eps
  and gradient buffers -- fits under the memory budget and in the device's
  free memory (memory-gated admission); others wait in arrival order;
* forms a batch from all pending requests -- one per client, whatever their
  grid sizes -- and submits it as one job table (adg_batch_submit), while up
  to `max_inflight` earlier batches are still running: requests that arrive
  while others are on the GPU join the next batch (continuous batching);
* completes each request when its batch's ticket is done, and records its
  latency (submit -> completion seen on the host).

Nothing here computes the method: all device work goes through libadg.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import adg


@dataclass
class Request:
    client: "Client"
    op: str                     # "build" or "grad"
    params: np.ndarray
    t_submit: float = 0.0
    t_done: float = 0.0
    result: object = None


@dataclass
class Client:
    """One design under optimisation with its resident device buffers.  The
    fields are given (efwd, eadj) or made at admission by make_fields()."""
    cid: int
    desc: dict
    efwd: object = None         # torch complex64 [C][nz][ny][nx]
    eadj: object = None
    make_fields: object = None  # () -> (efwd, eadj), called once admitted
    w: object = None
    iterations: int = 50
    step_nm: float = 1.0
    design: object = None
    eps: object = None
    grad: object = None
    grad_host: object = None    # pinned copy of the last gradient
    params: np.ndarray = None
    done_iters: int = 0
    t_arrive: float = 0.0
    need: int = 0               # bytes counted against the budget while admitted
    history: list = field(default_factory=list)

    def buffer_bytes(self) -> int:
        """The client's own device buffers: forward and adjoint fields
        (complex64), eps (fp32) and the gradient (fp32)."""
        nx, ny, nz = self.desc["grid"]["n"]
        samples = nx * ny * nz * self.desc["grid"]["ncomp"]
        return samples * (8 + 8 + 4) + 4 * len(self.desc["params"])


def footprint(ctx: adg.Context, client: Client, tile=None) -> int:
    """Resident bytes of a client: its compiled design as libadg reports it,
    plus its buffers (the design is compiled and released again)."""
    d = adg.Design(ctx, client.desc, tile=tile)
    try:
        return adg.adg_design_bytes(d) + client.buffer_bytes()
    finally:
        d.close()


class Server:
    def __init__(self, ctx: adg.Context, mem_budget_bytes: int, max_inflight: int = 2,
                 graph: bool = False, on_result=None, tuner=None, reserve_bytes: int = 1 << 30):
        self.ctx = ctx
        self.reserve = int(reserve_bytes)  # device memory left free at admission
        self.tuner = tuner  # tuning.Autotuner: the tile shape per design size class
        self.budget = int(mem_budget_bytes)
        self.used = 0
        self.max_inflight = max_inflight
        self.graph = graph
        self.waiting = collections.deque()   # clients not yet admitted
        self.active = []
        self.pending = collections.deque()   # requests ready to batch
        self.inflight = collections.deque()  # (ticket, [requests])
        self.completed = []
        self.finished_clients = []
        self.on_result = on_result
        self.batches = 0

    # ---- admission --------------------------------------------------------
    def arrive(self, client: Client, now: float):
        client.t_arrive = now
        self.waiting.append(client)
        self._admit(now)

    def _admit(self, now: float):
        import torch
        while self.waiting:
            c = self.waiting[0]
            tile = self.tuner.best(c.desc) if self.tuner is not None else None
            design = adg.Design(self.ctx, c.desc, tile=tile)
            need = adg.adg_design_bytes(design) + c.buffer_bytes()
            # buffers still to allocate must also fit in what the device has free
            to_alloc = c.buffer_bytes()
            if c.efwd is not None:
                to_alloc -= 2 * int(c.efwd.numel()) * 8
            # free on the device, plus what torch's allocator holds cached
            free = torch.cuda.mem_get_info()[0] + torch.cuda.memory_reserved() - torch.cuda.memory_allocated()
            if self.active and (self.used + need > self.budget or to_alloc + self.reserve > free):
                design.close()
                return  # wait for memory; an empty server always admits one
            self.waiting.popleft()
            c.need = need
            self.used += need
            c.design = design
            if c.efwd is None and c.make_fields is not None:
                c.efwd, c.eadj = c.make_fields()
            c.eps = torch.empty(c.design.shape, dtype=torch.float32, device="cuda")
            c.grad = torch.zeros(c.design.n_params, dtype=torch.float32, device="cuda")
            c.grad_host = torch.zeros(c.design.n_params, dtype=torch.float32).pin_memory()
            c.params = np.array(c.desc["params"], dtype=np.float64)
            self.active.append(c)
            self._issue(c, "build", now)

    def _release(self, c: Client):
        self.active.remove(c)
        self.used -= c.need
        c.design.close()
        c.eps = c.grad = c.efwd = c.eadj = None
        self.finished_clients.append(c)

    # ---- requests ---------------------------------------------------------
    def _issue(self, c: Client, op: str, now: float):
        self.pending.append(Request(c, op, c.params.copy(), t_submit=now))

    def _complete(self, r: Request, now: float):
        r.t_done = now
        c = r.client
        self.completed.append(r)
        if self.on_result is not None:
            self.on_result(r)
        if r.op == "build":
            self._issue(c, "grad", now)
            return
        g = c.grad_host.numpy().astype(np.float64)
        r.result = g
        c.done_iters += 1
        gi = float(np.abs(g).max()) if g.size else 0.0
        if gi > 0:  # p <- p - alpha g / ||g||_inf (alpha in nm)
            c.params = c.params - c.step_nm * g / gi
        if c.done_iters >= c.iterations:
            self._release(c)
            self._admit(now)
        else:
            self._issue(c, "build", now)

    # ---- the loop ---------------------------------------------------------
    def _submit_batch(self):
        reqs, seen = [], set()
        keep = collections.deque()
        while self.pending:
            r = self.pending.popleft()
            if id(r.client) in seen:
                keep.append(r)
                continue
            seen.add(id(r.client))
            reqs.append(r)
        self.pending = keep
        if not reqs:
            return
        items = []
        for r in reqs:
            c = r.client
            if r.op == "build":
                items.append(adg.BatchItem(c.design, r.params, eps=c.eps))
            else:
                items.append(adg.BatchItem(c.design, r.params, efwd=c.efwd, eadj=c.eadj, w=c.w,
                                           grad=c.grad))
        import torch
        t = adg.adg_batch_submit(self.ctx, items, graph=self.graph)
        # gradients back to pinned host buffers on the same stream; the event
        # after them marks the batch's results as readable
        for r in reqs:
            if r.op == "grad":
                r.client.grad_host.copy_(r.client.grad, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record()
        self.inflight.append((t, reqs, ev))
        self.batches += 1

    def poll(self, now_fn=time.perf_counter):
        """Complete finished batches; submit pending requests while slots free."""
        progressed = False
        while self.inflight and self.inflight[0][2].query():
            t, reqs, _ = self.inflight.popleft()
            adg.adg_batch_poll(self.ctx, t)  # releases the ticket
            now = now_fn()
            for r in reqs:
                self._complete(r, now)
            progressed = True
        while self.pending and len(self.inflight) < self.max_inflight:
            self._submit_batch()
            progressed = True
        return progressed

    def idle(self) -> bool:
        return not (self.waiting or self.active or self.pending or self.inflight)

    def drain(self, timeout_s: float = 600.0):
        t0 = time.perf_counter()
        while not self.idle():
            if not self.poll():
                time.sleep(20e-6)
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server did not drain")


def latency_stats(reqs) -> dict:
    lat = np.array([r.t_done - r.t_submit for r in reqs], dtype=np.float64)
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "n": 0}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "n": int(lat.size)}
