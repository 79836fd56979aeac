"""CPU tests of the continuous-batching server's host-side scheduling, with
fake operators and no GPU: size buckets, admission by the HBM budget,
coalescing per (operator, direction) under the batch limit, the "fullest"
order and its starvation guard, request validation, cancellation and operator
removal.  The GPU tests (test_serving.py) run the same server on real
operators; these pin the decisions alone."""
import collections
import time

import pytest

torch = pytest.importorskip("torch")

from paper_2508_10202_gb300.serve import BUCKETS, Request, Server  # noqa: E402


class FakeOp:
    """The attributes and the one method the scheduler reads."""

    def __init__(self, Nt, Nd, Nm, ws_per_rhs=1000):
        self.Nt, self.Nd, self.Nm = Nt, Nd, Nm
        self.ws_per_rhs = ws_per_rhs

    def workspace_bytes(self, which, K):
        return self.ws_per_rhs * K


def make_server(ops, budget, max_batch_rhs=64, policy="fifo", starve_ms=20.0, streams=4):
    # the scheduler's state without the CUDA streams and graphs __init__ makes
    s = Server.__new__(Server)
    s.ops = dict(ops)
    s.budget = budget
    s.resident = 0
    s.in_use = 0
    s.max_batch_rhs = max_batch_rhs
    s.graphs_enabled = False
    s.keep_outputs = True
    s.policy = policy
    s.starve_s = starve_ms * 1e-3
    s.free_streams = collections.deque(range(streams))
    s.queue = collections.deque()
    s.inflight = []
    s.slots = {}
    s.removed = set()
    s.completed = []
    s.n_batches = 0
    s.n_graph_batches = 0
    s._next_rid = 0
    return s


def req(s, op, which, K, age_s=0.0):
    o = s.ops[op]
    n_in = o.Nm if which == "F" else o.Nd
    r = Request(op=op, which=which, x=torch.zeros((K, o.Nt, n_in), dtype=torch.float32))
    r.rid = s._next_rid
    s._next_rid += 1
    r.arrival = time.perf_counter() - age_s
    r.status = "queued"
    s.queue.append(r)
    return r


OPS = {"a": FakeOp(10, 3, 5), "b": FakeOp(20, 2, 7)}


def bytes_of(op, which, K):
    # scratch + FP32 inputs and outputs + a fixed margin (Server._bytes)
    n_in, n_out = (op.Nm, op.Nd) if which == "F" else (op.Nd, op.Nm)
    return op.ws_per_rhs * K + 4 * K * op.Nt * (n_in + n_out) + 4096


def test_bytes_and_buckets():
    s = make_server(OPS, budget=1 << 30)
    for which in ("F", "F*"):
        for K in (1, 3, 64):
            assert s._bytes("a", which, K) == bytes_of(OPS["a"], which, K)
    assert BUCKETS == tuple(sorted(BUCKETS)) and BUCKETS[0] == 1
    assert [s._bucket(K) for K in (1, 2, 3, 5, 8, 9, 33, 64)] == [1, 2, 4, 8, 8, 16, 64, 64]
    assert s._bucket(65) == 65   # beyond the largest bucket: no graph, its own size


def test_coalesces_same_operator_and_direction_up_to_the_batch_limit():
    s = make_server(OPS, budget=1 << 30, max_batch_rhs=8)
    r0 = req(s, "a", "F", 2)
    rb = req(s, "b", "F", 1)
    r1 = req(s, "a", "F", 3)
    ra = req(s, "a", "F*", 1)
    r2 = req(s, "a", "F", 4)       # 2 + 3 + 4 = 9 > 8: stays queued
    r3 = req(s, "a", "F", 3)       # 2 + 3 + 3 = 8: joins
    batch = s._take_batch()
    assert batch == [r0, r1, r3]
    assert list(s.queue) == [rb, ra, r2]
    assert s._take_batch() == [rb]
    assert s._take_batch() == [ra]
    assert s._take_batch() == [r2]
    assert s._take_batch() is None


def test_admission_by_the_budget():
    a = OPS["a"]
    # room for 3 right-hand sides of a/F at once, not 4
    budget = bytes_of(a, "F", 3) + 10
    s = make_server(OPS, budget=budget)
    r0 = req(s, "a", "F", 2)
    r1 = req(s, "a", "F", 2)       # 2 + 2 = 4 does not fit: a batch of its own later
    r2 = req(s, "a", "F", 1)       # 2 + 1 = 3 fits: joins the first
    assert s._take_batch() == [r0, r2]
    # with that batch's bytes in use, nothing else fits until it retires
    s.in_use = bytes_of(a, "F", 3)
    assert s._take_batch() is None and list(s.queue) == [r1]
    s.in_use = 0
    assert s._take_batch() == [r1]


def test_a_request_that_does_not_fit_now_lets_a_smaller_one_pass():
    a = OPS["a"]
    s = make_server(OPS, budget=bytes_of(a, "F", 4) + 10)
    s.in_use = 3000                            # bytes of batches still running
    big = req(s, "a", "F", 4)                  # cannot fit until they finish
    small = req(s, "a", "F*", 1)
    assert bytes_of(a, "F", 4) > s.free_bytes() >= bytes_of(a, "F*", 1)
    assert s._take_batch() == [small]
    assert list(s.queue) == [big]


def test_fullest_order_and_its_starvation_guard():
    s = make_server(OPS, budget=1 << 30, policy="fullest", starve_ms=50.0)
    old = req(s, "a", "F", 1)
    bs = [req(s, "b", "F", 1) for _ in range(3)]
    # nobody has waited 50 ms: the operator and direction with the most
    # queued right-hand sides opens the batch, and all of them join
    assert s._take_batch() == bs
    assert list(s.queue) == [old]
    s.queue.clear()
    starved = req(s, "a", "F", 1, age_s=1.0)
    bs = [req(s, "b", "F", 1) for _ in range(3)]
    assert s._take_batch() == [starved]        # the oldest waited past the guard
    assert s._take_batch() == bs


def test_fifo_order_ignores_queue_depth():
    s = make_server(OPS, budget=1 << 30, policy="fifo")
    first = req(s, "a", "F", 1)
    for _ in range(3):
        req(s, "b", "F", 1)
    assert s._take_batch() == [first]


def test_schedule_stops_when_streams_run_out():
    s = make_server(OPS, budget=1 << 30, streams=0)
    req(s, "a", "F", 1)
    assert s.schedule() == 0 and len(s.queue) == 1


def test_validation_cancel_and_removal():
    s = make_server(OPS, budget=1 << 30)
    for bad, why in ((Request(op="z", which="F", x=torch.zeros((1, 10, 5))), "unknown operator"),
                     (Request(op="a", which="G", x=torch.zeros((1, 10, 5))), "is not F or F*"),
                     (Request(op="a", which="F", x=torch.zeros((1, 10, 5))), "CUDA float32")):
        r = s.submit(bad)
        assert r.status == "failed" and why in r.error and r.t_done is not None
    assert len(s.queue) == 0 and len(s.completed) == 3

    keep = req(s, "b", "F", 1)
    gone = req(s, "a", "F", 1)
    also = req(s, "a", "F*", 2)
    assert s.cancel(gone.rid) and gone.status == "cancelled"
    assert not s.cancel(gone.rid) and not s.cancel(10 ** 6)
    s.remove_operator("a")
    assert also.status == "failed" and "removed" in also.error
    assert list(s.queue) == [keep]
    r = s.submit(Request(op="a", which="F", x=torch.zeros((1, 10, 5))))
    assert r.status == "failed" and "unknown operator" in r.error


def test_a_server_needs_operators():
    from paper_2508_10202_gb300.serve import ServerError
    with pytest.raises(ServerError, match="no operators"):
        Server({}, budget_bytes=1)
