"""GPU parity: the CUDA path against the CPU oracle, element by element.

Bar: max_k |f_k - f_k^oracle| <= 10 eps sum_n |c_n| (the paper's O(eps ||c||_1) accuracy,
Sections 5.2 and 6.1, with the constant fixed at 10). Small sizes compare every output; the
full-size workloads compare seeded sampled rows that the oracle computes one by one.
"""
import math

import numpy as np
import pytest

import oracle
from hankel_inputs import coefficients, sample_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_01652_gb300 as hk  # noqa: E402

GRID = {"unit": 0, "paper": 1}


def _run(task, nu, N, eps, c, grid="unit", **kw):
    plan = hk.Plan(task, nu, N, eps, grid=grid, max_nrhs=c.shape[0], **kw)
    cd = torch.from_numpy(c).cuda()
    f = plan.exec(cd)
    torch.cuda.synchronize()
    return f.cpu().numpy(), plan


def _check(task, nu, N, eps, c, rows=None, grid="unit", **kw):
    f, plan = _run(task, nu, N, eps, c, grid=grid, **kw)
    ref = oracle.transform(task, nu, N, c, rows=rows, grid=GRID[grid])
    got = f if rows is None else f[:, rows]
    bound = 10.0 * eps * np.abs(c).sum(axis=1)
    err = np.abs(got - ref).max(axis=1)
    assert np.all(err <= bound), (err / (eps * np.abs(c).sum(axis=1)), plan.info)
    return err / (eps * np.abs(c).sum(axis=1))


@pytest.mark.parametrize("N", [2, 3, 17, 64, 100, 257, 1000, 1023])
@pytest.mark.parametrize("task", ["schlomilch", "fourier_bessel", "dht"])
def test_small_and_ragged_sizes(task, N):
    c = coefficients("normal", N, 2, 50 + N)
    _check(task, 0, N, 1e-15, c)


def test_schlomilch_nu0_N4096_full():
    # Schlomilch, omega_n = n pi, r_k = (k-1)/(N-1), N = 4096, eps = 1e-15, every output
    c = coefficients("uniform", 4096, 1, 1000)
    _check("schlomilch", 0, 4096, 1e-15, c)


@pytest.mark.parametrize("nu", [0, 1, 4])
@pytest.mark.parametrize("eps", [1e-15, 1e-8])
def test_schlomilch_shifted_orders(nu, eps):
    N = 6000
    c = coefficients("uniform", N, 3, 2000 + nu)
    _check("schlomilch", nu, N, eps, c)


def test_schlomilch_decaying_coefficients():
    N = 5000
    c = coefficients("decaying", N, 2, 2100)
    _check("schlomilch", 1, N, 1e-15, c)


@pytest.mark.parametrize("eps", [1e-15, 1e-8])
def test_fourier_bessel_full(eps):
    N = 5000
    c = coefficients("uniform", N, 2, 3000)
    _check("fourier_bessel", 0, N, eps, c)


@pytest.mark.parametrize("eps", [1e-15, 1e-8, 1e-4])
def test_dht_full(eps):
    N = 5000
    c = coefficients("normal", N, 2, 4000)
    _check("dht", 0, N, eps, c)


def test_paper_grid():
    N = 3000
    c = coefficients("uniform", N, 1, 4100)
    _check("schlomilch", 0, N, 1e-15, c, grid="paper")
    _check("fourier_bessel", 0, N, 1e-15, c, grid="paper")


@pytest.mark.parametrize("task,nu,N,eps,kind", [
    ("schlomilch", 0, 2 ** 16, 1e-15, "uniform"), ("schlomilch", 4, 2 ** 16, 1e-8, "decaying"),
    ("fourier_bessel", 0, 2 ** 18, 1e-15, "uniform"), ("dht", 0, 2 ** 16, 1e-15, "normal"),
    ("dht", 0, 2 ** 16, 1e-8, "normal"),
])
def test_workload_sizes_sampled_rows(task, nu, N, eps, kind):
    c = coefficients(kind, N, 1, 5000 + N % 997)
    rows = sample_rows(N, 96, 7)
    _check(task, nu, N, eps, c, rows=rows)


@pytest.mark.parametrize("segment", [True, False])
@pytest.mark.parametrize("task,nu,N,eps", [
    ("dht", 0, 2 ** 17, 1e-15), ("fourier_bessel", 0, 2 ** 17, 1e-8), ("schlomilch", 1, 2 ** 17, 1e-15),
])
def test_segmented_and_full_blocks(task, nu, N, eps, segment):
    # thin far blocks run as segmented convolutions by default; both forms must meet the bar
    c = coefficients("normal", N, 2, 5500)
    rows = sample_rows(N, 48, 13)
    _check(task, nu, N, eps, c, rows=rows, segment=segment)
    plan = hk.Plan(task, nu, N, eps, segment=segment, host_only=True)
    assert any(b["mode"] != 0 for b in plan.blocks()) == segment


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("task,nu,kind", [("dht", 0, "normal"), ("schlomilch", 1, "uniform"),
                                          ("schlomilch", 4, "decaying"), ("fourier_bessel", 0, "uniform")])
@pytest.mark.parametrize("eps", [1e-4, 1e-5])
def test_fp32_stages_at_relaxed_accuracy(task, nu, kind, eps, precision):
    # FP32 transform and near-field stages are admitted at eps >= 1e-5 and meet the same bar
    N = 7000
    c = coefficients(kind, N, 2, 7000 + nu)
    _check(task, nu, N, eps, c, precision=precision)


@pytest.mark.parametrize("task,nu,kind", [("dht", 0, "normal"), ("schlomilch", 1, "uniform"),
                                          ("fourier_bessel", 0, "uniform")])
@pytest.mark.parametrize("eps", [1e-6, 1e-8, 1e-11])
def test_df64_transforms(task, nu, kind, eps):
    # double-float transforms (MIXED picks them for 1e-11 <= eps < 1e-5) meet the bar, and stay
    # close to the FP64 plan's result
    N = 7000
    c = coefficients(kind, N, 2, 7300 + nu)
    f, plan = _run(task, nu, N, eps, c, precision="df64")
    assert plan.info["precision"] == 3
    ref = oracle.transform(task, nu, N, c)
    l1 = np.abs(c).sum(axis=1, keepdims=True)
    assert np.all(np.abs(f - ref) <= 10 * eps * l1)
    g, _ = _run(task, nu, N, eps, c, precision="fp64")
    assert np.all(np.abs(f - g) <= 1e-12 * l1)


@pytest.mark.parametrize("eps", [1e-6, 1e-11])
def test_df64_sparse_vectors(eps):
    # a few nonzero coefficients make ||c||_2 close to ||c||_1, the hardest input for
    # reduced-precision stages; 16 vectors run the near field's widest vector group
    N = 9000
    rng = np.random.default_rng(7400)
    c = np.zeros((16, N))
    for r in range(16):
        idx = rng.choice(N, size=1 + r % 4, replace=False)
        c[r, idx] = rng.standard_normal(idx.size)
    f, plan = _run("dht", 0, N, eps, c, precision="mixed")
    assert plan.info["precision"] == 3
    ref = oracle.transform("dht", 0, N, c)
    l1 = np.abs(c).sum(axis=1, keepdims=True)
    assert np.all(np.abs(f - ref) <= 10 * eps * l1)


@pytest.mark.parametrize("eps", [1e-15, 1e-12, 1e-8])
def test_mixed_term_precision(eps):
    # the small low-rank terms in double-float and FP32 (MIXED) against every term in the plan
    # precision: both meet the bar, and they differ by far less than it
    N = 2 ** 17
    c = coefficients("normal", N, 4, 7500)
    rows = sample_rows(N, 64, 29)
    f, plan = _run("dht", 0, N, eps, c, precision="mixed")
    terms = [sum(b["terms"][i] for b in plan.blocks()) for i in range(3)]
    assert terms[1] + terms[2] > 0 and terms[2] > 0
    g, _ = _run("dht", 0, N, eps, c, precision="mixed", mixed_terms=False)
    ref = oracle.transform("dht", 0, N, c, rows=rows)
    l1 = np.abs(c).sum(axis=1, keepdims=True)
    assert np.all(np.abs(f[:, rows] - ref) <= 10 * eps * l1)
    assert np.all(np.abs(g[:, rows] - ref) <= 10 * eps * l1)
    assert np.all(np.abs(f - g) <= eps * l1)


@pytest.mark.parametrize("kind,eps,precision", [("normal", 1e-15, "auto"), ("decaying", 1e-15, "auto"),
                                                ("normal", 1e-8, "auto"), ("normal", 1e-8, "mixed")])
def test_tensor_core_near_field(kind, eps, precision):
    # FP64 and DF64 plans run the near field's products as exact split-digit fp16 MMAs for 8+
    # vectors and as FMAs below; both meet the bar (rows up to 40 tiles long, ragged prefixes, a
    # coefficient scale that varies along the row)
    N = 20000
    c = coefficients(kind, N, 16, 7700)
    plan = hk.Plan("dht", 0, N, eps, max_nrhs=16, precision=precision)
    cd = torch.from_numpy(c).cuda()
    f16 = plan.exec(cd).cpu().numpy()
    f4 = plan.exec(cd[:4].contiguous()).cpu().numpy()
    ref = oracle.transform("dht", 0, N, c)
    l1 = np.abs(c).sum(axis=1, keepdims=True)
    e16 = np.abs(f16 - ref) / l1
    e4 = np.abs(f4 - ref[:4]) / l1[:4]
    assert np.all(e16 <= 10 * eps) and np.all(e4 <= 10 * eps)
    # the digit sums are exact, so the tensor-core form is at least as accurate as the FMAs
    # (measured at 1e-15: 5e-16 against 2e-15 to 4e-15 of ||c||_1 on the decaying vectors)
    assert e16[:4].max() <= e4.max() + max(1e-15, 0.1 * eps)


@pytest.mark.parametrize("eps", [1e-15, 1e-12])
def test_mixed_terms_sparse_vectors(eps):
    # spikes: every term's rounding sits on a few columns
    N = 20000
    rng = np.random.default_rng(7600)
    c = np.zeros((8, N))
    for r in range(8):
        idx = rng.choice(N, size=1 + r % 3, replace=False)
        c[r, idx] = rng.standard_normal(idx.size)
    f, plan = _run("dht", 0, N, eps, c, precision="mixed")
    assert sum(b["terms"][2] for b in plan.blocks()) > 0
    ref = oracle.transform("dht", 0, N, c)
    l1 = np.abs(c).sum(axis=1, keepdims=True)
    assert np.all(np.abs(f - ref) <= 10 * eps * l1)


@pytest.mark.parametrize("eps", [1e-4, 1e-5])
def test_fp32_workload_size_sampled_rows(eps):
    N = 2 ** 20
    c = coefficients("normal", N, 2, 4 * 1000 + 3)
    rows = sample_rows(N, 48, 17)
    _check("dht", 0, N, eps, c, rows=rows)


@pytest.mark.parametrize("task,nu,eps,kind", [
    ("schlomilch", 1, 1e-15, "uniform"), ("fourier_bessel", 0, 1e-8, "uniform"),
    ("dht", 0, 1e-15, "normal"), ("dht", 0, 1e-4, "normal"),
])
def test_largest_workload_size_sampled_rows(task, nu, eps, kind):
    # N = 2^22, the largest size of the workload table
    N = 2 ** 22
    c = coefficients(kind, N, 1, 4 * 1000 + 22)
    rows = sample_rows(N, 40, 23)
    _check(task, nu, N, eps, c, rows=rows)


@pytest.mark.parametrize("lowrank", [True, False])
def test_lowrank_forms_on_and_off(lowrank):
    # blocks run their low-rank forms or their kept stacked columns; both meet the bar
    N = 6000
    c = coefficients("normal", N, 2, 5600)
    _check("dht", 0, N, 1e-15, c, lowrank=lowrank)
    _check("fourier_bessel", 0, N, 1e-8, c, lowrank=lowrank)
    _check("dht", 0, N, 1e-4, c, lowrank=lowrank, precision="fp32")
    _check("schlomilch", 2, N, 1e-5, c, lowrank=lowrank, precision="fp32")
    plan = hk.Plan("dht", 0, N, 1e-15, lowrank=lowrank, host_only=True)
    assert any(b["lowrank"] for b in plan.blocks()) == lowrank


@pytest.mark.parametrize("eps", [1e-15, 1e-8])
def test_dht_2p20_sampled_rows(eps):
    # the benchmarked workload: DHT-0, N = 2^20, standard normal coefficients
    N = 2 ** 20
    c = coefficients("normal", N, 1, 4 * 1000)
    rows = sample_rows(N, 64, 11)
    _check("dht", 0, N, eps, c, rows=rows)


def test_batched_matches_single():
    # one plan (its blocks depend on max_nrhs): five vectors at once equal five single calls
    N = 3000
    c = coefficients("normal", N, 5, 6000)
    plan = hk.Plan("dht", 0, N, 1e-8, max_nrhs=5)
    fb = plan.exec(torch.from_numpy(c).cuda()).cpu().numpy()
    for r in range(c.shape[0]):
        fs = plan.exec(torch.from_numpy(c[r:r + 1]).cuda()).cpu().numpy()
        assert np.array_equal(fb[r], fs[0])


@pytest.mark.parametrize("task,eps", [("dht", 1e-15), ("dht", 1e-8), ("fourier_bessel", 1e-15), ("dht", 1e-4)])
def test_kept_columns_against_every_column(task, eps):
    # blocks that leave out columns (bound eps per entry) against blocks that keep all
    N = 6000
    c = coefficients("normal", N, 2, 5700)
    fp, plan = _run(task, 0, N, eps, c)
    fa, plan_all = _run(task, 0, N, eps, c, prune=False)
    assert plan.info["block_cols"] < plan_all.info["block_cols"]
    l1 = np.abs(c).sum(axis=1, keepdims=True)
    assert np.all(np.abs(fp - fa) <= 2 * eps * l1)
    ref = oracle.transform(task, 0, N, c)
    assert np.all(np.abs(fp - ref) <= 10 * eps * l1)


@pytest.mark.parametrize("eps,precision", [(1e-8, "fp64"), (1e-4, "fp32")])
def test_chunks_that_split_right_hand_sides(eps, precision):
    # a small workspace cuts the stacked columns of one right-hand side across chunks; every
    # chunk adds its share of each vector's columns, so the result equals one chunk per block
    N = 5000
    c = coefficients("normal", N, 5, 6050)
    big, _ = _run("dht", 0, N, eps, c, precision=precision)
    small, plan = _run("dht", 0, N, eps, c, precision=precision, workspace_limit=3 << 20)
    assert any(b["mode"] == 0 for b in plan.blocks())
    bound = 10.0 * eps * np.abs(c).sum(axis=1, keepdims=True)
    assert np.all(np.abs(small - big) <= bound)
    ref = oracle.transform("dht", 0, N, c)
    assert np.all(np.abs(small - ref) <= bound)


def test_deterministic_and_host_entry_point():
    N = 4097
    c = coefficients("uniform", N, 2, 6100)
    plan = hk.Plan("fourier_bessel", 0, N, 1e-15, max_nrhs=2)
    cd = torch.from_numpy(c).cuda()
    f1 = plan.exec(cd).cpu().numpy()
    f2 = plan.exec(cd).cpu().numpy()
    assert np.array_equal(f1, f2)
    fh = plan.exec_host(c)
    assert np.array_equal(f1, fh)


def test_dht_self_inverse_gpu():
    # Eq. (28): (1/j_{0,N+1}^2) J D_v J D_v c ~ c, v_n = 2/J_1(j_{0,n})^2, with both DHTs on the GPU.
    N = 400
    c = coefficients("normal", N, 1, 7)[0]
    b = oracle.j0_zero_offsets(N + 1)
    j = (np.arange(1, N + 2) - 0.25) * math.pi + b
    v = np.array([2.0 / oracle.besselj_pi(1, 4 * n - 1, 4, b[n - 1]) ** 2 for n in range(1, N + 1)])
    plan = hk.Plan("dht", 0, N, 1e-15)
    y = plan.exec(torch.from_numpy(v * c).cuda())
    ct = plan.exec(torch.from_numpy(v).cuda() * y).cpu().numpy() / j[N] ** 2
    assert np.max(np.abs(ct - c)) <= 2e-11
    # the inverse entry point: one DHT of v o f between two diagonal scalings
    f = plan.exec(torch.from_numpy(c).cuda())
    ci = plan.exec_inverse(f).cpu().numpy()
    assert np.max(np.abs(ci - c)) <= 2e-11


@pytest.mark.parametrize("N,eps,nrhs", [(3000, 1e-15, 1), (5000, 1e-8, 3), (2 ** 16, 1e-15, 2), (20000, 1e-4, 2)])
def test_dht_inverse_against_oracle(N, eps, nrhs):
    # c = j_{0,N+1}^{-2} v o J(v o f) element by element against the oracle's DHT of v o f; the bar
    # is the transform's, 10 eps ||v o f||_1, scaled by v_n / j_{0,N+1}^2
    f = coefficients("normal", N, nrhs, 7100 + N)
    b = oracle.j0_zero_offsets(N + 1)
    jN1 = (N + 0.75) * math.pi + b[N]
    v = np.array([2.0 / oracle.besselj_pi(1, 4 * n - 1, 4, b[n - 1]) ** 2 for n in range(1, N + 1)])
    plan = hk.Plan("dht", 0, N, eps, max_nrhs=nrhs)
    c = plan.exec_inverse(torch.from_numpy(f).cuda()).cpu().numpy().reshape(nrhs, N)
    rows = None if N <= 5000 else sample_rows(N, 64, 29)
    y = oracle.transform("dht", 0, N, v * f, rows=rows).reshape(nrhs, -1)
    vv = v if rows is None else v[rows]
    ref = vv * y / jN1 ** 2
    got = c if rows is None else c[:, rows]
    bound = 10 * eps * np.abs(v * f).sum(axis=1, keepdims=True) * vv / jN1 ** 2
    assert np.all(np.abs(got - ref) <= bound)
    with pytest.raises(RuntimeError, match="EINVAL"):
        hk.Plan("schlomilch", 0, 100, 1e-8).exec_inverse(torch.zeros(100, dtype=torch.float64, device="cuda"))


def test_rejects_bad_arguments():
    plan = hk.Plan("schlomilch", 0, 100, 1e-8)
    with pytest.raises(TypeError):
        plan.exec(torch.zeros(100, dtype=torch.float32, device="cuda"))
    with pytest.raises(RuntimeError, match="EINVAL"):
        plan.exec(torch.zeros((2, 100), dtype=torch.float64, device="cuda"))  # nrhs > max_nrhs


# ---------------------------------------------------------------------------------------------
# Scale: the transform is linear, so c 2^s must give f 2^s within the same relative bar in every
# precision. FP32 and double-float stages scale each vector by a power of two from its largest
# |c_n|; without that, 2^120 overflows FP32 and 2^-120 sinks into its subnormals.
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("nrhs", [1, 16])
@pytest.mark.parametrize("eps,precision", [(1e-15, "auto"), (1e-8, "auto"), (1e-4, "auto"), (1e-15, "mixed"),
                                           (1e-8, "mixed"), (1e-5, "fp32")])
def test_scaled_coefficients(eps, precision, nrhs):
    N = 9000
    c = coefficients("normal", N, nrhs, 7800)
    ref = oracle.transform("dht", 0, N, c)
    l1 = np.abs(c).sum(axis=1, keepdims=True)
    plan = hk.Plan("dht", 0, N, eps, max_nrhs=nrhs, precision=precision)
    for s in (120, 60, -60, -120):
        f = plan.exec(torch.from_numpy(np.ldexp(c, s)).cuda()).cpu().numpy()
        err = np.abs(np.ldexp(f, -s) - ref)
        assert np.all(np.isfinite(f)), s
        assert np.all(err <= 10 * eps * l1), (s, (err / (eps * l1)).max())


@pytest.mark.parametrize("eps,precision", [(1e-15, "auto"), (1e-4, "auto"), (1e-8, "mixed")])
def test_coefficients_spanning_2p200(eps, precision):
    # one vector whose entries range over 2^-100 .. 2^100 (uniform exponents)
    N = 6000
    rng = np.random.default_rng(7900)
    c = (rng.uniform(0.5, 1.0, N) * np.where(rng.random(N) < 0.5, -1.0, 1.0)
         * np.ldexp(1.0, rng.integers(-100, 101, N))).reshape(1, N)
    f, plan = _run("dht", 0, N, eps, c, precision=precision)
    ref = oracle.transform("dht", 0, N, c)
    assert np.all(np.isfinite(f))
    assert np.all(np.abs(f - ref) <= 10 * eps * np.abs(c).sum())


# ---------------------------------------------------------------------------------------------
# The workload table at its stated sizes and batches
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["auto", "mixed"])
@pytest.mark.parametrize("eps", [1e-15, 1e-8])
def test_benchmarked_configuration(eps, precision):
    # DHT-0 at N = 2^20 with 16 standard normal vectors per execution (the tensor-core near field,
    # the low-rank blocks and, for MIXED, the precision lanes), on 64 seeded rows
    N, B = 2 ** 20, 16
    c = coefficients("normal", N, B, 4 * 1000 + 100)
    rows = sample_rows(N, 64, 31)
    _check("dht", 0, N, eps, c, rows=rows, precision=precision)


@pytest.mark.parametrize("eps", [1e-15, 1e-4])
def test_dht_128_vectors(eps):
    # DHT-0, N = 2^16, 128 vectors in one execution: eight tensor-core groups of 16
    N = 2 ** 16
    c = coefficients("normal", N, 128, 4 * 1000 + 128)
    rows = sample_rows(N, 64, 37)
    _check("dht", 0, N, eps, c, rows=rows)


@pytest.mark.parametrize("nu,eps,kind", [(0, 1e-15, "uniform"), (4, 1e-15, "decaying"), (0, 1e-8, "uniform"),
                                         (4, 1e-4, "uniform")])
def test_schlomilch_2p20_32_vectors(nu, eps, kind):
    # Schlomilch omega_n = (n + nu) pi at N = 2^20 with a batch of 32 vectors
    N = 2 ** 20
    c = coefficients(kind, N, 32, 2 * 1000 + 20 + nu)
    rows = sample_rows(N, 64, 41)
    _check("schlomilch", nu, N, eps, c, rows=rows)


def test_group_remainder_below_tensor_core_minimum():
    # 21 vectors: one tensor-core group of 16 and a remainder of 5 on the FMA kernels
    N = 20000
    c = coefficients("normal", N, 21, 7950)
    _check("dht", 0, N, 1e-15, c)


@pytest.mark.parametrize("nu", [1, 2])
@pytest.mark.parametrize("eps,grid", [(1e-15, "unit"), (1e-8, "unit"), (1e-15, "paper")])
def test_fourier_bessel_higher_orders(nu, eps, grid):
    # Fourier-Bessel with nu > 0 (Section 5: J_nu at the roots of J_0), every output
    N = 5000
    c = coefficients("uniform", N, 2, 3100 + nu)
    _check("fourier_bessel", nu, N, eps, c, grid=grid)


@pytest.mark.parametrize("nu", [1, 2])
def test_fourier_bessel_higher_orders_large(nu):
    N = 2 ** 18
    c = coefficients("uniform", N, 4, 3200 + nu)
    rows = sample_rows(N, 48, 43)
    _check("fourier_bessel", nu, N, 1e-15, c, rows=rows)


# ---------------------------------------------------------------------------------------------
# The FFT autotuner: measured launch splits, used by the plan, with the same results
# ---------------------------------------------------------------------------------------------
def test_autotuned_shapes_are_recorded_and_exact():
    N = 2 ** 17
    c = coefficients("normal", N, 4, 8100)
    hk.tune_cache_clear()
    tuned = hk.Plan("dht", 0, N, 1e-15, max_nrhs=4)
    shapes = tuned.fft_shapes()
    assert shapes and tuned.info["fft_shapes"] == len(shapes)
    for s in shapes:
        assert s["one_launch"] or (2 <= len(s["radices"]) <= 4 and sum(s["radices"]) == s["log2_len"]
                                   and all(5 <= r <= 8 for r in s["radices"]))
        # measured in this process (the cache was cleared): the chosen split is no slower
        assert s["ms_chosen"] > 0 and s["ms_chosen"] <= s["ms_default"]
    # a second plan takes the cached splits without measuring
    again = hk.Plan("dht", 0, N, 1e-15, max_nrhs=4)
    assert [(s["log2_len"], s["radices"]) for s in again.fft_shapes()] == [(s["log2_len"], s["radices"])
                                                                            for s in shapes]
    fixed = hk.Plan("dht", 0, N, 1e-15, max_nrhs=4, autotune=False)
    assert all(s["ms_chosen"] == 0 for s in fixed.fft_shapes())
    cd = torch.from_numpy(c).cuda()
    ft = tuned.exec(cd).cpu().numpy()
    ff = fixed.exec(cd).cpu().numpy()
    rows = sample_rows(N, 64, 47)
    ref = oracle.transform("dht", 0, N, c, rows=rows)
    l1 = np.abs(c).sum(axis=1, keepdims=True)
    assert np.all(np.abs(ft[:, rows] - ref) <= 10 * 1e-15 * l1)
    # another split changes only the rounding of the transforms
    assert np.all(np.abs(ft - ff) <= 1e-15 * l1)


# ---------------------------------------------------------------------------------------------
# Radix-32 and radix-64 FFT passes on the tensor cores (split-digit products in FP64 accuracy)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("logF,ncols,radices,tc", [
    (12, 4, [5, 7], 0b01), (12, 4, [7, 5], 0b10), (12, 4, [6, 6], 0b11), (13, 4, [6, 7], 0b01),
    (15, 8, [5, 5, 5], 0b111), (17, 4, [5, 6, 6], 0b111), (18, 8, [6, 6, 6], 0b101),
    (20, 8, [5, 5, 5, 5], 0b1111), (21, 16, [5, 5, 5, 6], 0b1111), (21, 4, [6, 5, 5, 5], 0b1110),
    (22, 2, [5, 5, 5, 7], 0b0111), (22, 2, [5, 5, 6, 6], 0b1111),
    # a first pass on the tensor cores below 4096 points (tiles spanning columns, the last one ragged)
    (10, 3, [5, 5], 0b01), (10, 16, [5, 5], 0b01), (11, 5, [6, 5], 0b01), (11, 8, [5, 6], 0b01),
    # a pass tiled by twiddle group whose last tile is ragged (15 columns x 64 sequences)
    (16, 15, [5, 5, 6], 0b111),
])
@pytest.mark.parametrize("inverse", [False, True])
def test_tensor_core_fft_passes(logF, ncols, radices, tc, inverse):
    # the same seeded columns through the FP64 passes and through a split with tensor-core passes:
    # they agree to FP64 rounding (max |difference| / max |output|)
    err, ms = hk.debug_fft_compare(logF, ncols, radices, tc, inverse=inverse)
    assert err <= 2e-15 and ms > 0


@pytest.mark.parametrize("task,nu,N,eps,kind,nrhs", [
    ("dht", 0, 2 ** 17, 1e-15, "normal", 4), ("dht", 0, 2 ** 16, 1e-8, "normal", 16),
    ("fourier_bessel", 0, 2 ** 17, 1e-15, "uniform", 2), ("schlomilch", 1, 2 ** 17, 1e-15, "uniform", 2),
    ("dht", 0, 2 ** 20, 1e-15, "normal", 16),
])
def test_tensor_core_fft_in_the_transform(task, nu, N, eps, kind, nrhs):
    # FP64 transforms forced onto the tensor-core split (HANKEL_FLAG_TENSOR_FFT), element by element
    # against the oracle on sampled rows, and within eps ||c||_1 of the FP64-pipe plan
    c = coefficients(kind, N, nrhs, 8200 + N % 991)
    rows = sample_rows(N, 64, 53)
    f, plan = _run(task, nu, N, eps, c, tensor_fft=True)
    assert any(any(s["tensor_passes"]) for s in plan.fft_shapes())
    assert plan.device_status() == "HANKEL_OK"
    ref = oracle.transform(task, nu, N, c, rows=rows)
    l1 = np.abs(c).sum(axis=1, keepdims=True)
    assert np.all(np.abs(f[:, rows] - ref) <= 10 * eps * l1)
    g, _ = _run(task, nu, N, eps, c, autotune=False)
    assert np.all(np.abs(f - g) <= eps * l1)
