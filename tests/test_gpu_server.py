"""Continuous-batching server (qaoa_server_*): every result equals the same request run alone
and matches the FP64 oracle (<C> by the gate-level circuit, gradients by the oracle's adjoint),
admission by HBM footprint, queue limits, graphs on and off, shutdown with work in flight."""
import time

import numpy as np
import pytest

from paper_2312_03019_b300 import inputs as I
from tests.tolerances import c64_grad_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_03019_b300 import build
    build.build()
    from paper_2312_03019_b300 import binding
    return binding


def alone(B, g, gamma, beta, grad, prec="c64"):
    import torch
    s = B.QAOAState(g, prec)
    if grad:
        work = torch.empty(s.nbytes, dtype=torch.uint8, device="cuda")
        c, dg, db = B.qaoa_gradient(s.handle, gamma, beta, work.data_ptr(), s.nbytes)
        s.close()
        return c, dg, db
    s.apply_layers(gamma, beta)
    c, _ = s.expectation()
    s.close()
    return c, None, None


def wait_all(B, sv, tickets, timeout=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets):
        for t in tickets:
            if t not in res:
                r = B.qaoa_poll(sv, t)
                if r is not None:
                    res[t] = r
        if time.time() - t0 > timeout:
            raise TimeoutError("server did not finish")
        time.sleep(0.001)
    return res


def mixed_requests(count, seed=3):
    out = []
    rng = np.random.default_rng(seed)
    for i in range(count):
        n = int(rng.integers(8, 22))
        g = I.regular3(n, i) if (n % 2 == 0 and i % 2) else I.gnp(n, 0.3, i)
        p = int(rng.integers(1, 5))
        ga, be = I.angles(p, seed=100 + i)
        out.append((g, ga, be, bool(i % 4 == 0)))
    return out


_ORACLE = {}


def oracle_result(g, gamma, beta, grad):
    """(<C>, d gamma, d beta) of a request from the oracle, cached across the tests of this file."""
    import oracle
    key = (g.name, g.n, g.m, tuple(np.round(gamma, 15)), tuple(np.round(beta, 15)), grad)
    if key not in _ORACLE:
        if grad:
            _ORACLE[key] = oracle.adjoint_gradient(g, gamma, beta)
        else:
            _ORACLE[key] = (oracle.expectation(g, oracle.qaoa_state(g, gamma, beta))[0], None, None)
    return _ORACLE[key]


def check_against_oracle(r, g, gamma, beta, grad, prec):
    """A served result against the oracle: complex128 <C> within 1e-12 relative and derivatives
    within 1e-10 of the largest; complex64 <C> within 1e-5 |E| and derivatives within the
    rounding bound of tests/tolerances.py."""
    c, dg, db = oracle_result(g, gamma, beta, grad)
    if prec == "c128":
        assert abs(r["expectation"] - c) <= 1e-12 * max(1.0, abs(c)), (g.name, r["expectation"], c)
    else:
        assert abs(r["expectation"] - c) <= 1e-5 * max(1, g.m), (g.name, r["expectation"], c)
    if grad:
        ref = np.concatenate([dg, db])
        got = np.concatenate([r["d_gamma"], r["d_beta"]])
        scale = float(np.max(np.abs(ref)))
        tol = 1e-10 * max(1.0, scale) if prec == "c128" else c64_grad_tol(g.n, len(gamma), g.m, scale)
        assert np.max(np.abs(got - ref)) <= tol, (g.name, np.max(np.abs(got - ref)), tol)


@pytest.mark.parametrize("graphs", [True, False])
def test_results_identical_alone_and_in_the_mix(B, graphs):
    reqs = mixed_requests(48)
    sv = B.qaoa_server_create(4 << 30, "c64", max_inflight=32, max_batch=16, streams=4, use_graphs=graphs)
    tickets = [B.qaoa_submit(sv, g, ga, be, grad) for g, ga, be, grad in reqs]
    res = wait_all(B, sv, tickets)
    stats = B.qaoa_server_stats_read(sv)
    B.qaoa_server_destroy(sv)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["batches"] >= 1 and stats["batched_requests"] >= 1
    assert stats["tiled_batches"] >= 1 and stats["tiled_batched_requests"] >= 2
    if graphs:
        assert stats["graph_launches"] >= 1
    packed = streamed = 0
    for (g, ga, be, grad), t in zip(reqs, tickets):
        r = res[t]
        assert r["status"] == 0
        c, dg, db = alone(B, g, ga, be, grad)
        assert r["expectation"] == c, (g.name, r["expectation"], c)  # bit-identical
        if grad:
            assert np.array_equal(r["d_gamma"], dg) and np.array_equal(r["d_beta"], db)
        check_against_oracle(r, g, ga, be, grad, "c64")
        packed += r["batched"]
        streamed += g.n >= 15
    assert packed >= 1 and streamed >= 10


@pytest.mark.parametrize("graphs", [True, False])
def test_packed_mid_size_requests(B, graphs):
    """Mid-size complex64 forward requests (tiled states, 15 <= n <= 22, p <= 8) of one (n, p)
    run in packed launches, one launch per pass over the tiles of every request: 40 requests of
    four shapes, different graphs; each result equals the request run alone bit for bit and the
    oracle's <C> within 1e-5 |E|.  A request with p = 9 and a gradient request of the same size
    run alone."""
    reqs = []
    for i in range(40):
        n, p = ((15, 3), (18, 2), (20, 4), (22, 1))[i % 4]
        g = I.regular3(n, 500 + i) if (n % 2 == 0 and i % 3) else I.gnp(n, 0.3, 500 + i)
        ga, be = I.angles(p, seed=700 + i, beta_hi=np.pi)
        reqs.append((g, ga, be, False))
    g9 = I.gnp(18, 0.3, 9)
    reqs.append((g9, *I.angles(9, seed=9), False))
    reqs.append((I.regular3(18, 10), *I.angles(2, seed=10), True))
    sv = B.qaoa_server_create(8 << 30, "c64", max_inflight=64, max_batch=64, streams=4, use_graphs=graphs)
    try:
        tickets = [B.qaoa_submit(sv, g, ga, be, grad) for g, ga, be, grad in reqs]
        res = wait_all(B, sv, tickets)
        stats = B.qaoa_server_stats_read(sv)
    finally:
        B.qaoa_server_destroy(sv)
    assert stats["failed"] == 0 and stats["completed"] == len(reqs)
    packed = 0
    for (g, ga, be, grad), t in zip(reqs, tickets):
        r = res[t]
        assert r["status"] == 0
        c, dg, db = alone(B, g, ga, be, grad)
        assert r["expectation"] == c, (g.name, r["expectation"], c)
        check_against_oracle(r, g, ga, be, grad, "c64")
        packed += r["batched"]
    assert not res[tickets[-2]]["batched"] and not res[tickets[-1]]["batched"]
    # the scheduler starts while requests are still being submitted, so not all of them find a
    # partner of the same shape in the same turn
    assert packed == stats["tiled_batched_requests"] >= 8, stats


def test_c128_mix_against_the_oracle(B):
    """complex128 server: packed small requests (n <= 13), streamed ones (n = 15..19), with and
    without gradients, all against the oracle to 1e-12."""
    reqs = []
    for i, n in enumerate((8, 11, 13, 9, 15, 17, 19, 16, 12, 18)):
        g = I.regular3(n, 30 + i) if n % 2 == 0 else I.gnp(n, 0.35, 30 + i)
        ga, be = I.angles(1 + i % 4, seed=300 + i)
        reqs.append((g, ga, be, i % 3 == 1))
    sv = B.qaoa_server_create(2 << 30, "c128", max_inflight=8, max_batch=8, streams=4)
    try:
        tickets = [B.qaoa_submit(sv, g, ga, be, grad) for g, ga, be, grad in reqs]
        res = wait_all(B, sv, tickets)
    finally:
        B.qaoa_server_destroy(sv)
    for (g, ga, be, grad), t in zip(reqs, tickets):
        assert res[t]["status"] == 0
        check_against_oracle(res[t], g, ga, be, grad, "c128")


def test_admission_under_a_small_arena(B):
    # the arena holds about one n = 22 state at a time: requests must queue and still complete
    g = I.regular3(22, 1)
    ga, be = I.angles(2, 1)
    ref, _, _ = alone(B, g, ga, be, False)
    sv = B.qaoa_server_create(48 << 20, "c64", max_inflight=16, max_batch=8, streams=4)
    tickets = [B.qaoa_submit(sv, g, ga, be) for _ in range(6)]
    res = wait_all(B, sv, tickets)
    stats = B.qaoa_server_stats_read(sv)
    B.qaoa_server_destroy(sv)
    assert all(res[t]["expectation"] == ref for t in tickets)
    assert stats["arena_peak_bytes"] <= 48 << 20


def test_rejections_and_unknown_tickets(B):
    sv = B.qaoa_server_create(16 << 20, "c64", max_inflight=1, queue_capacity=2, max_batch=1, streams=1)
    big = I.regular3(24, 0)  # 128 MiB state: larger than the whole arena
    with pytest.raises(B.QAOAError) as ei:
        B.qaoa_submit(sv, big, [0.1], [0.2])
    assert ei.value.status == B.QAOA_ERR_OOM
    with pytest.raises(B.QAOAError) as ei:
        B.qaoa_submit(sv, I.Graph(4, np.array([[0, 0]], dtype=np.int32)), [0.1], [0.2])
    assert ei.value.status == B.QAOA_ERR_INVALID
    with pytest.raises(B.QAOAError):
        B.qaoa_submit(sv, I.ring(6), [float("nan")], [0.2])
    with pytest.raises(B.QAOAError) as ei:
        B.qaoa_poll(sv, 987654)
    assert ei.value.status == B.QAOA_ERR_INVALID
    # flood the queue: some submissions must come back with QAOA_ERR_AGAIN
    g = I.regular3(20, 2)
    ga, be = I.angles(6, 2)
    tickets, again = [], 0
    for _ in range(64):
        try:
            tickets.append(B.qaoa_submit(sv, g, ga, be))
        except B.QAOAError as e:
            assert e.status == B.QAOA_ERR_AGAIN
            again += 1
    assert again > 0
    res = wait_all(B, sv, tickets)
    assert all(r["status"] == 0 for r in res.values())
    t = tickets[0]
    with pytest.raises(B.QAOAError):
        B.qaoa_poll(sv, t)  # released after the first successful poll
    B.qaoa_server_destroy(sv)


def test_destroy_with_work_in_flight(B):
    sv = B.qaoa_server_create(2 << 30, "c64", max_inflight=8, max_batch=8, streams=2)
    g = I.regular3(24, 3)
    ga, be = I.angles(6, 3)
    for _ in range(12):
        B.qaoa_submit(sv, g, ga, be, True)
    t0 = time.time()
    B.qaoa_server_destroy(sv)  # waits for admitted work, drops the rest
    assert time.time() - t0 < 60


def test_c128_server_gradient(B):
    g = I.gnp(15, 0.4, 5)
    ga, be = I.angles(3, 5)
    c, dg, db = alone(B, g, ga, be, True, "c128")
    sv = B.qaoa_server_create(1 << 30, "c128", max_inflight=4, max_batch=4, streams=2)
    t = B.qaoa_submit(sv, g, ga, be, True)
    r = wait_all(B, sv, [t])[t]
    B.qaoa_server_destroy(sv)
    assert r["expectation"] == c and np.array_equal(r["d_gamma"], dg) and np.array_equal(r["d_beta"], db)
    check_against_oracle(r, g, ga, be, True, "c128")


def test_deadline_expires_while_queued(B):
    """With one request in flight at a time, a gradient at n = 26 holds the GPU for several
    milliseconds: requests queued behind it with a 0.1 ms deadline complete with
    QAOA_ERR_TIMEOUT without running; one with a 60 s deadline and the gradient itself complete
    normally; bad deadlines are rejected at submit.  Every input is prepared before the first
    submit, so all requests are queued while the gradient runs."""
    g_big = I.gnp(26, 0.5, 0)
    ga, be = I.angles(6, 0)
    shorts = [(I.regular3(16, i), *I.angles(2, i)) for i in range(3)]
    g_ok = I.regular3(16, 9)
    g2, b2 = I.angles(2, 9)
    sv = B.qaoa_server_create(hbm_budget_bytes=4 << 30, prec="c64", max_inflight=1)
    try:
        big = B.qaoa_submit(sv, g_big, ga, be, want_grad=True)
        short = [B.qaoa_submit(sv, g, x, y, deadline_s=1e-4) for g, x, y in shorts]
        ok = B.qaoa_submit(sv, g_ok, g2, b2, deadline_s=60.0)
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(B.QAOAError) as ei:
                B.qaoa_submit(sv, g_ok, g2, b2, deadline_s=bad)
            assert ei.value.status == B.QAOA_ERR_INVALID
        res = wait_all(B, sv, [big] + short + [ok])
        stats = B.qaoa_server_stats_read(sv)
    finally:
        B.qaoa_server_destroy(sv)
    assert res[big]["status"] == B.QAOA_OK and res[big]["has_grad"]
    assert res[ok]["status"] == B.QAOA_OK
    c, _, _ = alone(B, g_ok, g2, b2, False)
    assert res[ok]["expectation"] == c
    for t in short:
        assert res[t]["status"] == B.QAOA_ERR_TIMEOUT
        assert res[t]["t_done"] - res[t]["t_submit"] >= 1e-4
        assert res[t]["t_submit"] < res[big]["t_done"]
    assert stats["timed_out"] == 3


def test_gpu_filling_requests_on_the_lane(B):
    """Requests whose state fills the GPU (64 MiB or more: n = 24 here) run one after another on
    the low-priority lane while small ones run beside them: the n = 24 results (a forward run
    of G(24, 0.5), p = 10 and a gradient of a 3-regular n = 24 graph, p = 3) equal the same
    requests run alone bit for bit and match the oracle's stored values (tests/golden, written
    by the oracle only); the small requests equal theirs run alone."""
    import json
    import os
    gold = os.path.join(os.path.dirname(__file__), "golden")
    fwd = json.load(open(os.path.join(gold, "gnp24_p10.json")))
    grd = json.load(open(os.path.join(gold, "grad_regular3_n24_p3.json")))
    gf = I.Graph(fwd["n"], np.array(fwd["edges"], dtype=np.int32))
    gg = I.Graph(grd["n"], np.array(grd["edges"], dtype=np.int32))
    big = [(gf, np.array(fwd["gamma"]), np.array(fwd["beta"]), False),
           (gg, np.array(grd["gamma"]), np.array(grd["beta"]), True)] * 2
    small = mixed_requests(24, seed=11)
    reqs = [x for pair in zip(big + [None] * (len(small) - len(big)), small) for x in pair if x is not None]
    sv = B.qaoa_server_create(8 << 30, "c64", max_inflight=16, max_batch=8, streams=4)
    tickets = [B.qaoa_submit(sv, g, ga, be, grad) for g, ga, be, grad in reqs]
    res = wait_all(B, sv, tickets)
    B.qaoa_server_destroy(sv)
    for (g, ga, be, grad), t in zip(reqs, tickets):
        r = res[t]
        assert r["status"] == 0
        c, dg, db = alone(B, g, ga, be, grad)
        assert r["expectation"] == c, (g.name, r["expectation"], c)
        if grad:
            assert np.array_equal(r["d_gamma"], dg) and np.array_equal(r["d_beta"], db)
        if g is gf:
            assert abs(r["expectation"] - fwd["expectation"]) <= 1e-5 * fwd["m"]
        elif g is gg:
            ref = np.concatenate([grd["d_gamma"], grd["d_beta"]])
            tol = c64_grad_tol(gg.n, len(grd["gamma"]), gg.m, np.max(np.abs(ref)))
            assert abs(r["expectation"] - grd["expectation"]) <= 1e-5 * grd["m"]
            assert np.max(np.abs(np.concatenate([r["d_gamma"], r["d_beta"]]) - ref)) <= tol
