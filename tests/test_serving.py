"""The continuous-batching server: results in the mix equal results alone,
budget admission, cancellation, removal and bad requests (faults injected on
the host; nothing here faults the GPU)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

OPS = {"a": (16, 4, 100), "b": (40, 9, 250), "c": (64, 20, 130)}


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2508_10202_gb300 import Operator, build
    build.build()
    cols = {k: synth.block_column(*v, seed=i, dtype=np.float32).astype(np.float64) for i, (k, v) in enumerate(OPS.items())}
    ops = {k: Operator(torch.from_numpy(c).cuda()) for k, c in cols.items()}
    yield torch, ops, cols
    for op in ops.values():
        op.free()


def make_requests(torch, ops, n, seed, kmax=12):
    from paper_2508_10202_gb300.serve import Request
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        name = list(ops)[rng.integers(len(ops))]
        which = "F" if rng.random() < 0.5 else "F*"
        op = ops[name]
        K = int(rng.integers(1, kmax + 1))
        N = op.Nm if which == "F" else op.Nd
        x = torch.from_numpy(synth.vectors(synth.TAG_M if which == "F" else synth.TAG_D, op.Nt, N, k=K,
                                           seed=1000 * seed + i, dtype=np.float32)).cuda()
        reqs.append(Request(name, which, x))
    return reqs


def alone(ops, r):
    op = ops[r.op]
    return (op.matvec(r.x) if r.which == "F" else op.rmatvec(r.x)).cpu().numpy()


@pytest.mark.parametrize("graphs,policy", [(True, "fifo"), (False, "fifo"), (True, "fullest")])
def test_mix_equals_alone_and_oracle(env, graphs, policy):
    torch, ops, cols = env
    from paper_2508_10202_gb300.serve import Server
    srv = Server(ops, budget_bytes=8 << 30, n_streams=3, graphs=graphs, policy=policy)
    reqs = make_requests(torch, ops, 40, seed=1)
    for r in reqs:
        srv.submit(r)
    srv.run_until_idle()
    assert all(r.status == "done" for r in reqs)
    assert srv.n_batches < len(reqs)                 # requests were coalesced
    if graphs:
        assert srv.n_graph_batches > 0
    for r in reqs:
        got = r.out.cpu().numpy()
        np.testing.assert_allclose(got, alone(ops, r), rtol=0, atol=1e-6 * np.abs(got).max())
    for r in reqs[:6]:                               # and against the FP64 oracle
        fn = oracle.matvec_direct if r.which == "F" else oracle.rmatvec_direct
        assert oracle.rel_l2(r.out.cpu().numpy(), fn(cols[r.op], r.x.double().cpu().numpy())) <= 1e-5
    srv.close()


def test_open_loop_schedule_reports_latency(env):
    torch, ops, _ = env
    from paper_2508_10202_gb300.serve import Server, latency_stats
    srv = Server(ops, budget_bytes=8 << 30, n_streams=2)
    reqs = make_requests(torch, ops, 30, seed=2)
    rng = np.random.default_rng(3)
    t = np.cumsum(rng.exponential(0.002, size=len(reqs)))
    out = srv.run_schedule(list(zip(t, reqs)))
    st = latency_stats(out)
    assert st["n"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_budget_admission_and_rejection(env):
    torch, ops, _ = env
    from paper_2508_10202_gb300.serve import Request, Server
    probe = Server(ops, budget_bytes=8 << 30)
    resident = probe.resident
    one = max(probe._bytes("b", w, 12) for w in ("F", "F*"))
    probe.close()
    # room for one 12-RHS batch of operator b at a time (graphs off: no static buffers)
    srv = Server(ops, budget_bytes=resident + one + 1024, n_streams=4, graphs=False)
    reqs = [r for r in make_requests(torch, ops, 30, seed=4) if r.op == "b"]
    for r in reqs:
        srv.submit(r)
    peak = 0
    while srv.queue or srv.inflight:
        srv.poll()
        srv.schedule()
        peak = max(peak, srv.in_use)
        assert srv.in_use <= srv.budget - srv.resident
    assert all(r.status == "done" for r in reqs) and peak > 0
    big = Request("b", "F", torch.zeros((60, ops["b"].Nt, ops["b"].Nm), device="cuda"))
    srv.submit(big)
    assert big.status == "failed" and "never fit" in big.error
    srv.close()


def test_cancel_remove_and_bad_requests(env):
    torch, ops, _ = env
    from paper_2508_10202_gb300.serve import Request, Server
    srv = Server(ops, budget_bytes=8 << 30, n_streams=1, graphs=False)
    reqs = make_requests(torch, ops, 12, seed=5)
    for r in reqs:
        srv.submit(r)
    bad = srv.submit(Request("a", "F", torch.zeros((3, 5, 7), device="cuda")))        # wrong shape
    wrong = srv.submit(Request("zz", "F", reqs[0].x))                                  # unknown operator
    assert bad.status == "failed" and "does not match" in bad.error
    assert wrong.status == "failed"
    queued = [r for r in reqs if r.status == "queued"]
    assert srv.cancel(queued[-1].rid) and queued[-1].status == "cancelled"
    srv.remove_operator("c")
    srv.run_until_idle()
    for r in reqs:
        if r is queued[-1]:
            continue
        if r.op == "c":
            assert r.status == "failed" and "removed" in r.error
        else:
            assert r.status == "done"
            np.testing.assert_allclose(r.out.cpu().numpy(), alone(ops, r), rtol=0,
                                       atol=1e-6 * float(r.out.abs().max()))
    srv.close()


def test_fullest_policy_order_and_starvation_guard(env):
    # host logic only: which queued request opens the next batch
    import time
    torch, ops, _ = env
    from paper_2508_10202_gb300.serve import Request, Server, ServerError
    with pytest.raises(ServerError):
        Server(ops, budget_bytes=8 << 30, policy="lifo")
    srv = Server(ops, budget_bytes=8 << 30, policy="fullest", starve_ms=1e6)
    x = {n: torch.zeros((1, op.Nt, op.Nm), device="cuda") for n, op in ops.items()}
    first = srv.submit(Request("a", "F", x["a"]))
    srv.submit(Request("b", "F", x["b"]))
    srv.submit(Request("b", "F", x["b"]))
    order = srv._order()
    assert order[0].op == "b" and order[-1] is first      # the fuller group goes first
    srv.starve_s = 0.0                                     # ... unless the oldest has waited too long
    time.sleep(0.001)
    assert srv._order()[0] is first
    srv.run_until_idle()
    srv.close()
