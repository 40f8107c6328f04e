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
    if graphs:
        assert st["graphs_captured"] > 0
    for (task, nu, N, eps, c), (_, f) in zip(reqs, tickets):
        ref = _alone(task, nu, N, eps, c)
        bound = 10 * eps * np.abs(c).sum(axis=1, keepdims=True)
        assert np.all(np.abs(f - ref) <= bound), (task, N, eps)
    srv.close()


def test_repeat_submissions_with_graphs_are_stable():
    c = coefficients("normal", 4096, 2, 77)
    srv = hk.Server(streams=2, max_batch=2, use_graphs=True)
    outs = []
    for _ in range(4):
        t, f = srv.submit("dht", 0, 4096, 1e-8, c)
        srv.wait(t)
        outs.append(f.copy())
    for f in outs[1:]:
        assert np.array_equal(f, outs[0])
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
