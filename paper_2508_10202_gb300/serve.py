"""Continuous-batching server for F / F* matvecs on resident operators.

The paper's motivation for many matvecs is the outer loop of Bayesian
inverse problems (Remark 1: N_d N_t actions of F and F* to assemble a
data-space Hessian, repeated per sensor configuration).  This module serves
such requests for several operators kept resident on one GPU:

* admission by an HBM budget: operator storage is charged once; every batch
  charges its scratch, gathered inputs and outputs while it is in flight, and
  waits in the queue until the budget has room.  A request that could never
  fit is rejected;
* continuous batching: whenever a stream and memory free up, the oldest
  waiting request opens a batch and later requests for the same operator and
  direction join it (up to ``max_batch_rhs`` right-hand sides); batches of
  different operators run concurrently on separate CUDA streams;
* one launch per batch: each (operator, direction, size bucket) is captured
  once as a CUDA graph over static buffers (scratch supplied to the library,
  so the graph holds kernel and memset nodes, no allocation) and replayed;
  batches that do not fit a graph run the direct call;
* results are independent of the mix: every right-hand side is computed by
  the same per-column arithmetic whatever else is in its batch, and the tests
  check that a request gives the same numbers alone and in the mix.

Latency is wall-clock from a request's arrival to the host observing its
batch's completion event.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import torch

from .operator import Operator

__all__ = ["Request", "Server", "ServerError", "latency_stats"]

BUCKETS = (1, 2, 4, 8, 16, 32, 64)
# bf16 hi/lo on the tensor cores both ways; f16x2 lowers the error further but
# adds a pass over each input, which costs the mix about 18 % of its capacity
DEFAULT_PRECISION = {"F": ("sssss", "bf16x2"), "F*": ("sssss", "bf16x2")}


class ServerError(RuntimeError):
    pass


@dataclass(eq=False)   # requests compare by identity
class Request:
    """One F (``which="F"``) or F* request of K right-hand sides.

    ``x`` is a CUDA float32 tensor (K, Nt, N) with N = Nm for F, Nd for F*.
    """
    op: str
    which: str
    x: torch.Tensor
    rid: int = -1
    arrival: float = 0.0
    out: torch.Tensor | None = None
    t_launch: float | None = None
    t_done: float | None = None
    status: str = "new"
    error: str | None = None
    batch_size: int = 0

    @property
    def K(self) -> int:
        return self.x.shape[0] if self.x.dim() == 3 else 1

    @property
    def latency_ms(self) -> float | None:
        return None if self.t_done is None else 1e3 * (self.t_done - self.arrival)


@dataclass
class _Slot:
    """A captured graph over static buffers for one (operator, direction, bucket)."""
    graph: torch.cuda.CUDAGraph
    x: torch.Tensor
    y: torch.Tensor
    ws: torch.Tensor
    nbytes: int
    busy: bool = False


@dataclass
class _Batch:
    reqs: list
    op: str
    which: str
    K: int
    stream: int
    event: torch.cuda.Event
    nbytes: int
    slot: tuple | None = None
    keep: list = field(default_factory=list)


class Server:
    def __init__(self, operators: dict[str, Operator], budget_bytes: int, n_streams: int = 4,
                 max_batch_rhs: int = 64, precision: dict | None = None, graphs: bool = True,
                 keep_outputs: bool = True, policy: str = "fifo", starve_ms: float = 20.0):
        if not operators:
            raise ServerError("no operators")
        self.ops = dict(operators)
        self.precision = dict(DEFAULT_PRECISION if precision is None else precision)
        for op in self.ops.values():
            for which, p in self.precision.items():
                op.set_precision(which, *p)
        self.device = torch.device("cuda", next(iter(self.ops.values())).device)
        self.budget = int(budget_bytes)
        self.resident = sum(op.info().fhat_bytes for op in self.ops.values())
        if self.resident > self.budget:
            raise ServerError(f"resident operators need {self.resident} bytes, budget is {self.budget}")
        self.in_use = 0
        self.max_batch_rhs = int(max_batch_rhs)
        self.graphs_enabled = graphs
        # False: a finished request drops its output (load generators that
        # only measure latency would otherwise hold every result in HBM)
        self.keep_outputs = keep_outputs
        # "fifo": the oldest request that fits opens the next batch.  "fullest":
        # the (operator, direction) with the most queued right-hand sides opens
        # it (one pass over F-hat serves up to max_batch_rhs of them, so fuller
        # batches raise throughput), unless the oldest request has waited
        # starve_ms, which then goes first.
        if policy not in ("fifo", "fullest"):
            raise ServerError(f"unknown policy {policy!r}")
        self.policy = policy
        self.starve_s = starve_ms * 1e-3
        self.streams = [torch.cuda.Stream(self.device) for _ in range(n_streams)]
        self.free_streams = collections.deque(range(n_streams))
        self.queue: collections.deque[Request] = collections.deque()
        self.inflight: list[_Batch] = []
        self.slots: dict[tuple, _Slot] = {}
        self.removed: set[str] = set()
        self.completed: list[Request] = []
        self.n_batches = 0
        self.n_graph_batches = 0
        self._next_rid = 0

    # -- sizes and memory ---------------------------------------------------
    def _dims(self, op: Operator, which: str) -> tuple[int, int]:
        return (op.Nm, op.Nd) if which == "F" else (op.Nd, op.Nm)

    def _bytes(self, name: str, which: str, K: int) -> int:
        op = self.ops[name]
        n_in, n_out = self._dims(op, which)
        return op.workspace_bytes(which, K) + 4 * K * op.Nt * (n_in + n_out) + 4096

    def free_bytes(self) -> int:
        return self.budget - self.resident - self.in_use

    # -- client side ----------------------------------------------------------
    def submit(self, req: Request, arrival: float | None = None) -> Request:
        req.rid = self._next_rid
        self._next_rid += 1
        req.arrival = time.perf_counter() if arrival is None else arrival
        err = self._validate(req)
        if err:
            req.status, req.error = "failed", err
            req.t_done = req.arrival
            self.completed.append(req)
            return req
        req.status = "queued"
        self.queue.append(req)
        return req

    def _validate(self, req: Request) -> str | None:
        if req.op not in self.ops or req.op in self.removed:
            return f"unknown operator {req.op!r}"
        if req.which not in ("F", "F*"):
            return f"direction {req.which!r} is not F or F*"
        op = self.ops[req.op]
        n_in, _ = self._dims(op, req.which)
        x = req.x
        if not (x.is_cuda and x.dtype == torch.float32 and x.dim() in (2, 3) and x.is_contiguous()):
            return "input must be a contiguous CUDA float32 tensor (K, Nt, N)"
        if tuple(x.shape[-2:]) != (op.Nt, n_in):
            return f"input shape {tuple(x.shape)} does not match (Nt={op.Nt}, N={n_in})"
        if req.K > self.max_batch_rhs:
            return f"{req.K} right-hand sides exceed the batch limit {self.max_batch_rhs}"
        if self._bytes(req.op, req.which, req.K) > self.budget - self.resident:
            return "request can never fit the HBM budget"
        return None

    def cancel(self, rid: int) -> bool:
        """Cancel a request that is still queued (running ones complete)."""
        for r in list(self.queue):
            if r.rid == rid:
                self.queue.remove(r)
                r.status, r.t_done = "cancelled", time.perf_counter()
                self.completed.append(r)
                return True
        return False

    def remove_operator(self, name: str) -> None:
        """Stop serving an operator: its queued requests fail; running batches finish."""
        self.removed.add(name)
        for r in list(self.queue):
            if r.op == name:
                self.queue.remove(r)
                r.status, r.error, r.t_done = "failed", f"operator {name!r} removed", time.perf_counter()
                self.completed.append(r)

    # -- scheduling -----------------------------------------------------------
    def poll(self) -> int:
        """Retire finished batches; returns how many finished."""
        done = 0
        now = None
        for b in list(self.inflight):
            if not b.event.query():
                continue
            now = time.perf_counter() if now is None else now
            for r in b.reqs:
                r.status, r.t_done = "done", now
                if not self.keep_outputs:
                    r.out = None
                self.completed.append(r)
            self.inflight.remove(b)
            self.in_use -= b.nbytes
            self.free_streams.append(b.stream)
            if b.slot is not None:
                self.slots[b.slot].busy = False
            done += 1
        return done

    def _bucket(self, K: int) -> int:
        for b in BUCKETS:
            if b >= K:
                return b
        return K

    def _slot(self, name: str, which: str, bucket: int) -> tuple | None:
        key = (name, which, bucket)
        if key in self.slots:
            return key
        if not self.graphs_enabled:
            return None
        op = self.ops[name]
        n_in, n_out = self._dims(op, which)
        wsb = op.workspace_bytes(which, bucket)
        nbytes = wsb + 4 * bucket * op.Nt * (n_in + n_out) + 256
        if nbytes > self.free_bytes():
            return None
        x = torch.zeros((bucket, op.Nt, n_in), dtype=torch.float32, device=self.device)
        y = torch.zeros((bucket, op.Nt, n_out), dtype=torch.float32, device=self.device)
        ws = torch.empty(wsb + 256, dtype=torch.uint8, device=self.device)
        off = (-ws.data_ptr()) % 256
        ws = ws[off:off + wsb]
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            op.apply_ws(which, x, y, ws, stream=side)     # warm-up outside the capture
        torch.cuda.current_stream(self.device).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(g, capture_error_mode="thread_local"):
                op.apply_ws(which, x, y, ws, stream=torch.cuda.current_stream(self.device))
        except Exception:
            self.graphs_enabled = False
            return None
        self.slots[key] = _Slot(g, x, y, ws, nbytes)
        self.in_use += nbytes
        return key

    def _order(self) -> list[Request]:
        """Queued requests in the order they may open a batch."""
        q = list(self.queue)
        if self.policy == "fifo" or not q:
            return q
        if time.perf_counter() - q[0].arrival >= self.starve_s:
            return q
        load: dict[tuple, int] = collections.defaultdict(int)
        for r in q:
            load[(r.op, r.which)] += r.K
        return sorted(q, key=lambda r: -min(load[(r.op, r.which)], self.max_batch_rhs))   # stable: oldest first

    def _take_batch(self) -> list[Request] | None:
        """The first request (in policy order) that fits opens a batch; later
        ones for the same operator and direction join while the budget and
        batch limit allow."""
        order = self._order()
        for i, r in enumerate(order):
            need = self._bytes(r.op, r.which, r.K)
            if need > self.free_bytes():
                continue
            batch, K = [r], r.K
            for q in self.queue:
                if q is r:
                    continue
                if q.op == r.op and q.which == r.which and K + q.K <= self.max_batch_rhs:
                    if self._bytes(r.op, r.which, K + q.K) <= self.free_bytes():
                        batch.append(q)
                        K += q.K
            for q in batch:
                self.queue.remove(q)
            return batch
        return None

    def schedule(self) -> int:
        """Launch batches while streams and memory allow; returns how many launched."""
        launched = 0
        while self.queue and self.free_streams:
            batch = self._take_batch()
            if batch is None:
                break
            self._launch(batch)
            launched += 1
        return launched

    def _launch(self, reqs: list[Request]) -> None:
        name, which = reqs[0].op, reqs[0].which
        op = self.ops[name]
        K = sum(r.K for r in reqs)
        sidx = self.free_streams.popleft()
        s = self.streams[sidx]
        s.wait_stream(torch.cuda.current_stream(self.device))
        _, n_out = self._dims(op, which)
        t = time.perf_counter()
        slot_key = self._slot(name, which, self._bucket(K))
        if slot_key is not None and self.slots[slot_key].busy:
            slot_key = None
        nbytes = 4 * K * op.Nt * n_out + 256
        keep = []
        with torch.cuda.stream(s):
            if slot_key is not None:
                sl = self.slots[slot_key]
                sl.busy = True
                k0 = 0
                for r in reqs:
                    sl.x[k0:k0 + r.K].copy_(r.x.view(r.K, *r.x.shape[-2:]))
                    k0 += r.K
                sl.graph.replay()
                out = sl.y[:K].clone()
                self.n_graph_batches += 1
            else:
                nbytes = self._bytes(name, which, K)
                xin = torch.cat([r.x.view(r.K, *r.x.shape[-2:]) for r in reqs]) if len(reqs) > 1 else \
                    reqs[0].x.view(reqs[0].K, *reqs[0].x.shape[-2:])
                out = op.matvec(xin, stream=s) if which == "F" else op.rmatvec(xin, stream=s)
                keep.append(xin)
            k0 = 0
            for r in reqs:
                r.out = out[k0:k0 + r.K] if r.x.dim() == 3 else out[k0]
                r.x.record_stream(s)
                r.status, r.t_launch, r.batch_size = "running", t, K
                k0 += r.K
            ev = torch.cuda.Event()
            ev.record(s)
        self.in_use += nbytes
        self.n_batches += 1
        self.inflight.append(_Batch(reqs, name, which, K, sidx, ev, nbytes, slot_key, keep))

    # -- driving loops --------------------------------------------------------
    def run_until_idle(self, timeout_s: float = 600.0) -> None:
        t_end = time.perf_counter() + timeout_s
        while self.queue or self.inflight:
            self.poll()
            self.schedule()
            if time.perf_counter() > t_end:
                raise ServerError("server did not drain within the timeout")

    def run_schedule(self, schedule: list[tuple[float, Request]], timeout_s: float = 600.0) -> list[Request]:
        """Open-loop arrivals: request i becomes visible at t0 + schedule[i][0]."""
        schedule = sorted(schedule, key=lambda p: p[0])
        t0 = time.perf_counter()
        i = 0
        out = []
        while i < len(schedule) or self.queue or self.inflight:
            now = time.perf_counter()
            while i < len(schedule) and t0 + schedule[i][0] <= now:
                out.append(self.submit(schedule[i][1], arrival=t0 + schedule[i][0]))
                i += 1
            self.poll()
            self.schedule()
            if now - t0 > timeout_s:
                raise ServerError("schedule did not finish within the timeout")
        return out

    def close(self) -> None:
        torch.cuda.synchronize(self.device)
        self.slots.clear()
        self.in_use = 0


def latency_stats(reqs: list[Request]) -> dict:
    """p50 / p99 latency (ms), throughput in right-hand-side matvecs per second."""
    import numpy as np
    done = [r for r in reqs if r.status == "done"]
    if not done:
        return {"n": 0}
    lat = np.array([r.latency_ms for r in done])
    t0 = min(r.arrival for r in done)
    t1 = max(r.t_done for r in done)
    rhs = sum(r.K for r in done)
    return {"n": len(done), "rhs": rhs, "seconds": t1 - t0, "matvec_s": rhs / (t1 - t0),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}
