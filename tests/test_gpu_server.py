"""The request loop (hankel_server_*): results in a mixed stream of requests equal the same
requests run alone, within 10 eps sum|c_n|; graph replay, eviction and rejection behave."""
import numpy as np
import pytest

import oracle
from hankel_inputs import coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_01652_gb300 as hk  # noqa: E402

MIX = [
    ("schlomilch", 0, 1024, 1e-15), ("schlomilch", 1, 3000, 1e-8), ("fourier_bessel", 0, 2048, 1e-15),
    ("dht", 0, 1500, 1e-8), ("dht", 0, 4096, 1e-4), ("schlomilch", 0, 1 << 14, 1e-4),
    ("fourier_bessel", 0, 5000, 1e-8), ("dht", 0, 1 << 13, 1e-15),
]


def _alone(task, nu, N, eps, c, precision="auto"):
    plan = hk.Plan(task, nu, N, eps, max_nrhs=c.shape[0], precision=precision)
    return plan.exec(torch.from_numpy(c).cuda()).cpu().numpy()


def _requests(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        task, nu, N, eps = MIX[rng.integers(len(MIX))]
        nrhs = int(rng.integers(1, 4))
        out.append((task, nu, N, eps, coefficients("uniform", N, nrhs, 900 + i)))
    return out


@pytest.mark.parametrize("graphs", [False, True])
def test_mixed_stream_matches_alone(graphs):
    reqs = _requests(3, 40)
    srv = hk.Server(streams=4, max_batch=8, use_graphs=graphs)
    tickets = [srv.submit(t, nu, N, eps, c) for (t, nu, N, eps, c) in reqs]
    lat = [srv.wait(tk) for tk, _ in tickets]
    assert all(x > 0 for x in lat)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["batches"] < len(reqs)  # requests of one plan were packed together
    for (task, nu, N, eps, c), (_, f) in zip(reqs, tickets):
        ref = _alone(task, nu, N, eps, c)
        bound = 10 * eps * np.abs(c).sum(axis=1, keepdims=True)
        assert np.all(np.abs(f - ref) <= bound), (task, N, eps)
    srv.close()


def test_repeat_submissions_with_graphs_are_stable():
    # the plan's first run and a (slot, context, batch size)'s first run go uncaptured; the key's
    # second run is captured and later ones replay: every result is the same
    c = coefficients("normal", 4096, 2, 77)
    srv = hk.Server(streams=1, max_batch=2, use_graphs=True)
    outs = []
    for _ in range(5):
        t, f = srv.submit("dht", 0, 4096, 1e-8, c)
        srv.wait(t)
        outs.append(f.copy())
    for f in outs[1:]:
        assert np.array_equal(f, outs[0])
    assert srv.stats()["graphs_captured"] == 1
    srv.close()


def test_memory_cap_evicts_idle_plans():
    srv = hk.Server(streams=1, max_batch=4, memory_cap=8 << 20)  # less than one plan: every new plan evicts
    reqs = [("schlomilch", 0, 3000 + 500 * i, 1e-8, coefficients("uniform", 3000 + 500 * i, 1, 50 + i))
            for i in range(5)]
    for task, nu, N, eps, c in reqs:
        t, f = srv.submit(task, nu, N, eps, c)
        srv.wait(t)
        ref = _alone(task, nu, N, eps, c)
        assert np.all(np.abs(f - ref) <= 10 * eps * np.abs(c).sum())
    assert srv.stats()["plans_evicted"] >= 1
    srv.close()


def test_plain_fp64_server_at_relaxed_eps():
    # precision="fp64" keeps every stage in FP64 even where FP32 would be admitted
    N, eps = 4096, 1e-4
    c = coefficients("normal", N, 1, 88)
    srv = hk.Server(streams=1, max_batch=1, precision="fp64")
    t, f = srv.submit("dht", 0, N, eps, c)
    srv.wait(t)
    ref = _alone("dht", 0, N, eps, c, precision="fp64")
    assert np.array_equal(f, ref)
    srv.close()


def test_unpacked_server_runs_one_request_per_execution():
    srv = hk.Server(streams=1, max_batch=8, pack=False)
    c = coefficients("uniform", 2048, 1, 5)
    tickets = [srv.submit("schlomilch", 0, 2048, 1e-8, c) for _ in range(6)]
    for t, f in tickets:
        srv.wait(t)
    assert srv.stats()["batches"] == 6
    srv.close()


def test_rejects_invalid_requests():
    srv = hk.Server(streams=1)
    with pytest.raises(RuntimeError, match="EINVAL"):
        srv.submit("dht", 1, 100, 1e-8, np.zeros(100))
    with pytest.raises(RuntimeError, match="EINVAL"):
        srv.submit("schlomilch", 0, 100, 1e-8, np.zeros((65, 100)))  # more vectors than max_batch
    srv.close()


def test_page_locked_requests_match_pageable():
    # page-locked request arrays bypass the staging buffers; results are the same either way
    c = coefficients("normal", 4096, 3, 91)
    ct = torch.from_numpy(c).pin_memory()
    fpin = torch.empty((3, 4096), dtype=torch.float64).pin_memory()
    srv = hk.Server(streams=2, max_batch=4, use_graphs=True)
    t1, f1 = srv.submit("dht", 0, 4096, 1e-8, c)
    t2, f2 = srv.submit("dht", 0, 4096, 1e-8, ct.numpy(), fpin.numpy())
    srv.wait(t1)
    srv.wait(t2)
    t3, f3 = srv.submit("dht", 0, 4096, 1e-8, ct.numpy(), fpin.numpy())  # replay with graphs
    srv.wait(t3)
    assert np.array_equal(f1, f2) and np.array_equal(f2, f3) and np.array_equal(f3, fpin.numpy())
    srv.close()


def test_burst_of_submissions_stays_one_batch():
    # a partial batch leaves once no request of its plan has arrived for batch_window_us: five
    # requests 1.5 ms apart under a 5 ms window form one batch (timing from their oldest request
    # would have dispatched the first four alone)
    import time

    N = 4096
    cs = [coefficients("normal", N, 1, 300 + i) for i in range(5)]
    srv = hk.Server(streams=2, max_batch=16, batch_window_us=5000)
    t, _ = srv.submit("dht", 0, N, 1e-8, cs[0])  # build the plan outside the measured burst
    srv.wait(t)
    b0 = srv.stats()["batches"]
    tickets = []
    for c in cs:
        tickets.append(srv.submit("dht", 0, N, 1e-8, c))
        time.sleep(0.0015)
    for tk, f in tickets:
        srv.wait(tk)
    assert srv.stats()["batches"] - b0 == 1
    ref = _alone("dht", 0, N, 1e-8, np.concatenate(cs))
    for i, (_, f) in enumerate(tickets):
        assert np.all(np.abs(f - ref[i]) <= 10 * 1e-8 * np.abs(cs[i]).sum())
    srv.close()


@pytest.mark.parametrize("precision", ["auto", "mixed"])
def test_served_results_against_oracle(precision):
    # every request of a mixed stream, served in packed batches on several streams with graph
    # replay, against the oracle directly
    reqs = _requests(11, 24)
    srv = hk.Server(streams=4, max_batch=8, use_graphs=True, precision=precision)
    tickets = [srv.submit(t, nu, N, eps, c) for (t, nu, N, eps, c) in reqs]
    for tk, _ in tickets:
        srv.wait(tk)
    for (task, nu, N, eps, c), (_, f) in zip(reqs, tickets):
        ref = oracle.transform(task, nu, N, c)
        bound = 10 * eps * np.abs(c).sum(axis=1, keepdims=True)
        assert np.all(np.abs(f.reshape(c.shape) - ref) <= bound), (task, N, eps)
    srv.close()


def test_plan_contexts_run_side_by_side():
    # two execution contexts of one plan on two streams at once: each result equals the one run
    # alone on context 0 (same plan, same arithmetic: bitwise)
    N = 2 ** 15
    plan = hk.Plan("dht", 0, N, 1e-15, max_nrhs=4)
    assert plan.info["contexts"] == 1
    assert plan.add_context() == 1
    info = plan.info
    assert info["contexts"] == 2 and 0 < info["context_bytes"] < info["device_bytes"]
    a = torch.from_numpy(coefficients("normal", N, 4, 950)).cuda()
    b = torch.from_numpy(coefficients("normal", N, 3, 951)).cuda()
    ra = plan.exec(a).clone()
    rb = plan.exec(b).clone()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(3):
        fa = plan.exec(a, stream=s1, context=0)
        fb = plan.exec(b, stream=s2, context=1)
        torch.cuda.synchronize()
        assert torch.equal(fa, ra) and torch.equal(fb, rb)


def test_two_batches_of_one_plan_in_flight():
    # a burst for one plan with small batches: the server adds a second context to the plan and
    # runs two of its batches at once; every result meets the bar against the oracle
    N = 2 ** 16
    srv = hk.Server(streams=4, max_batch=2, use_graphs=True, batch_window_us=0, contexts_per_plan=2)
    cs = [coefficients("normal", N, 1, 960 + i) for i in range(12)]
    tickets = [srv.submit("dht", 0, N, 1e-8, c) for c in cs]
    for tk, _ in tickets:
        srv.wait(tk)
    st = srv.stats()
    assert st["contexts_added"] >= 1 and st["failed"] == 0
    rows = np.arange(0, N, 97)
    for c, (_, f) in zip(cs, tickets):
        ref = oracle.transform("dht", 0, N, c, rows=rows)
        assert np.all(np.abs(f.reshape(1, N)[:, rows] - ref) <= 10 * 1e-8 * np.abs(c).sum())
    srv.close()


def test_injected_allocation_failure_in_admission():
    # a plan build (or slot buffer) that cannot get device memory fails that request with ENOMEM;
    # the server keeps serving the others, and the same request succeeds once memory is there
    srv = hk.Server(streams=2, max_batch=4)
    try:
        c = coefficients("uniform", 3000, 1, 970)
        t, f = srv.submit("schlomilch", 0, 3000, 1e-8, c)
        srv.wait(t)  # plan cached, slot buffers made
        hk.debug_fail_allocs(0, 1)
        c2 = coefficients("uniform", 5000, 2, 971)
        t2, _ = srv.submit("fourier_bessel", 0, 5000, 1e-8, c2)  # a new plan: its first allocation fails
        assert srv.status(t2)[0] == "HANKEL_ENOMEM"
        hk.debug_fail_allocs(0, 0)
        t3, f3 = srv.submit("schlomilch", 0, 3000, 1e-8, c)  # the cached plan still serves
        srv.wait(t3)
        assert np.array_equal(f3, f)
        t4, f4 = srv.submit("fourier_bessel", 0, 5000, 1e-8, c2)
        srv.wait(t4)
        ref = oracle.transform("fourier_bessel", 0, 5000, c2)
        assert np.all(np.abs(f4 - ref) <= 10 * 1e-8 * np.abs(c2).sum(axis=1, keepdims=True))
        st = srv.stats()
        assert st["failed"] == 1 and st["completed"] == 3
    finally:
        hk.debug_fail_allocs(0, 0)
        srv.close()


@pytest.mark.parametrize("after", [0, 5, 20])
def test_injected_allocation_failure_in_plan_creation(after):
    # plan creation that runs out of device memory part way returns ENOMEM and frees what it made
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    hk.debug_fail_allocs(after, 1)
    try:
        with pytest.raises(RuntimeError, match="ENOMEM"):
            hk.Plan("dht", 0, 20000, 1e-15, max_nrhs=8)
    finally:
        hk.debug_fail_allocs(0, 0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    p = hk.Plan("dht", 0, 20000, 1e-15, max_nrhs=8)
    assert p.info["device_bytes"] > 0


def test_cancel_queued_requests():
    # one stream, one request at a time: requests behind the first can still be cancelled
    N = 2 ** 17
    srv = hk.Server(streams=1, max_batch=1, pack=False)
    cs = [coefficients("normal", N, 1, 980 + i) for i in range(10)]
    tickets = [srv.submit("dht", 0, N, 1e-15, c)[0] for c in cs]
    cancelled = [srv.cancel(t) for t in tickets[5:]]
    assert any(cancelled)
    for t, cn in zip(tickets[5:], cancelled):
        assert srv.status(t)[0] == ("HANKEL_ECANCELED" if cn else "HANKEL_OK")
    for t in tickets[:5]:
        assert srv.status(t)[0] == "HANKEL_OK"
    st = srv.stats()
    assert st["cancelled"] == sum(cancelled) and st["completed"] == 10 - sum(cancelled)
    srv.close()


def test_small_batches_run_on_their_own_plan():
    # with small_batch = 2, a lone request runs on a plan built for 2 vectors and a burst of 8
    # on the plan built for max_batch: two plans for one (task, nu, N, eps), results within the bar
    N, eps = 6000, 1e-15
    cs = [coefficients("normal", N, 1, 4400 + i) for i in range(9)]
    srv = hk.Server(streams=2, max_batch=8, use_graphs=True, small_batch=2, batch_window_us=5000)
    t, f0 = srv.submit("dht", 0, N, eps, cs[0])
    srv.wait(t)
    burst = [srv.submit("dht", 0, N, eps, c) for c in cs[1:]]
    for tk, _ in burst:
        srv.wait(tk)
    st = srv.stats()
    assert st["plans_built"] == 2 and st["failed"] == 0
    bound = lambda c: 10 * eps * np.abs(c).sum()
    assert np.abs(f0 - _alone("dht", 0, N, eps, cs[0])).max() <= bound(cs[0])
    for c, (_, f) in zip(cs[1:], burst):
        assert np.abs(f - _alone("dht", 0, N, eps, c)).max() <= bound(c)
    srv.close()
