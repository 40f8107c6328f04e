"""Host-side plan tables (no GPU): nodes, partition geometry and the entry-wise
representation of J_nu(r_k omega_n) against the oracle."""
import ctypes
import math
import re
import os

import numpy as np
import pytest

import oracle
import paper_1501_01652_gb300 as hk
from paper_1501_01652_gb300 import _lib

GRID = {"unit": 0, "paper": 1}
CASES = [
    ("schlomilch", 0, 1500, 1e-15, "unit"), ("schlomilch", 1, 1200, 1e-8, "unit"),
    ("schlomilch", 4, 1500, 1e-15, "unit"), ("schlomilch", 0, 1400, 1e-4, "unit"),
    ("schlomilch", 0, 900, 1e-15, "paper"), ("fourier_bessel", 0, 1500, 1e-15, "unit"),
    ("fourier_bessel", 0, 1500, 1e-8, "unit"), ("fourier_bessel", 1, 1000, 1e-15, "paper"),
    ("dht", 0, 1500, 1e-15, "unit"), ("dht", 0, 1500, 1e-8, "unit"), ("dht", 0, 1500, 1e-4, "unit"),
]


def test_library_exports_every_declared_symbol():
    header = open(os.path.join(os.path.dirname(__file__), "..", "include", "hankel.h")).read()
    declared = set(re.findall(r"^\s*(?:int|double|const char\*)\s+(hankel_\w+)\s*\(", header, re.M))
    assert declared == set(_lib.EXPORTED)
    lib = _lib.load()
    for name in declared:
        assert hasattr(lib, name), name


def test_status_strings():
    lib = _lib.load()
    for code in range(0, 7):
        assert lib.hankel_status_string(code)


def test_precision_policy():
    # AUTO: every stage FP64 below eps = 1e-5, FP32 stages at and above it
    assert hk.params("dht", 0, 4096, 1e-4)["precision"] == 2
    assert hk.params("dht", 0, 4096, 1e-5)["precision"] == 2
    for eps in (9e-6, 1e-8, 1e-11, 9e-12, 1e-15):
        assert hk.params("dht", 0, 4096, eps)["precision"] == 1
    # MIXED (opt-in): double-float transforms for 1e-11 <= eps < 1e-5, FP64 below, FP32 above
    assert hk.params("dht", 0, 4096, 1e-4, precision="mixed")["precision"] == 2
    assert hk.params("dht", 0, 4096, 9e-6, precision="mixed")["precision"] == 3
    assert hk.params("dht", 0, 4096, 1e-8, precision="mixed")["precision"] == 3
    assert hk.params("dht", 0, 4096, 1e-11, precision="mixed")["precision"] == 3
    assert hk.params("dht", 0, 4096, 9e-12, precision="mixed")["precision"] == 1
    assert hk.params("dht", 0, 4096, 1e-4, precision="fp64")["precision"] == 1
    assert hk.params("dht", 0, 4096, 1e-8, precision="fp64")["precision"] == 1
    assert hk.params("dht", 0, 4096, 1e-4, precision="df64")["precision"] == 3
    with pytest.raises(RuntimeError, match="EUNSUPPORTED"):
        hk.params("dht", 0, 4096, 9e-6, precision="fp32")
    with pytest.raises(RuntimeError, match="EUNSUPPORTED"):
        hk.params("dht", 0, 4096, 9e-12, precision="df64")


@pytest.mark.parametrize("eps", [1e-15, 1e-8])
def test_auto_plans_keep_every_term_fp64(eps):
    # below eps = 1e-5 an AUTO plan runs every far-field transform in FP64
    bl = hk.Plan("dht", 0, 2 ** 18, eps, host_only=True).blocks()
    assert all(b["terms"][0] == b["ncols"] for b in bl)


@pytest.mark.parametrize("eps,base", [(1e-15, 0), (1e-12, 0), (1e-8, 1), (1e-4, 2)])
def test_term_precision_split(eps, base):
    # MIXED plans run the small terms of a block's low-rank form in a lower precision; the
    # largest term of every block keeps the plan precision, and no term goes above it; uniform
    # plans and forced precisions keep one precision for every transform
    N = 2 ** 18
    bl = hk.Plan("dht", 0, N, eps, host_only=True, precision="mixed").blocks()
    for b in bl:
        assert sum(b["terms"]) == b["ncols"]
        if not b["lowrank"] or base == 2:
            assert b["terms"][base] == b["ncols"]
        else:
            assert b["terms"][base] >= 1
            assert all(b["terms"][q] == 0 for q in range(base))
    if base < 2:
        assert sum(b["terms"][q] for b in bl for q in range(base + 1, 3)) > 0
    u = hk.Plan("dht", 0, N, eps, host_only=True, precision="mixed", mixed_terms=False)
    assert all(b["terms"][base] == b["ncols"] for b in u.blocks())
    if base == 0:
        f = hk.Plan("dht", 0, N, eps, host_only=True, precision="fp64")
        assert all(b["terms"][0] == b["ncols"] for b in f.blocks())


def test_thin_blocks_are_segmented_at_workload_size():
    # Eq. (19) at N = 2^20 (P = 3): one square block and three thin ones on each side
    p = hk.Plan("dht", 0, 2 ** 20, 1e-15, host_only=True, refine=False)
    modes = sorted(b["mode"] for b in p.blocks())
    assert modes == [0, 1, 1, 1, 2, 2, 2]
    q = hk.Plan("dht", 0, 2 ** 20, 1e-15, host_only=True, segment=False)
    assert all(b["mode"] == 0 and b["nseg"] == 1 for b in q.blocks())
    r = hk.Plan("dht", 0, 2 ** 20, 1e-15, host_only=True)
    assert {b["mode"] for b in r.blocks()} == {0, 1, 2}


@pytest.mark.parametrize("case", CASES + [("dht", 0, 2 ** 18, 1e-15, "unit"), ("schlomilch", 0, 2 ** 18, 1e-8, "unit")],
                         ids=lambda c: "%s-nu%d-N%d-%g-%s" % c)
def test_subdivided_blocks_tile_the_same_far_set(case):
    # cutting blocks changes neither the near prefixes nor the far entries covered, and the
    # pieces do not overlap (their areas add up to the far count)
    task, nu, N, eps, grid = case
    p = hk.Plan(task, nu, N, eps, grid=grid, host_only=True)
    q = hk.Plan(task, nu, N, eps, grid=grid, host_only=True, refine=False)
    assert p.info["far_count"] == q.info["far_count"]
    assert sum((b["k1"] - b["k0"] + 1) * (b["n1"] - b["n0"] + 1) for b in p.blocks()) == p.info["far_count"]
    for k in sorted({1, 2, N // 3, N // 2, N}):
        assert p.near_prefix(k) == q.near_prefix(k)
    for b in p.blocks():
        assert any(c["k0"] <= b["k0"] and b["k1"] <= c["k1"] and c["n0"] <= b["n0"] and b["n1"] <= c["n1"]
                   for c in q.blocks())


def test_node_offsets_against_oracle_and_lemma():
    n = 20000
    b = hk.j0_zero_offsets(n)
    ref = oracle.j0_zero_offsets(n)
    assert np.max(np.abs(b - ref) / ref) <= 4e-15
    k = np.arange(1, n + 1)
    assert np.all((b >= 0) & (b <= 1 / (8 * (k - 0.25) * math.pi)))


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-nu%d-N%d-%g-%s" % c)
def test_partition_invariants(case):
    task, nu, N, eps, grid = case
    p = hk.Plan(task, nu, N, eps, grid=grid, host_only=True)
    info = p.info
    blocks = p.blocks()
    assert len(blocks) <= 1 + 2 * info["P"]
    covered = np.zeros(N + 1, dtype=np.int64)
    for b in blocks:
        k0, k1, n0, n1, F = b["k0"], b["k1"], b["n0"], b["n1"], b["F"]
        R, C = k1 - k0 + 1, n1 - n0 + 1
        assert 1 <= k0 <= k1 <= N and 1 <= n0 <= n1 <= N
        assert F & (F - 1) == 0
        if b["mode"] == 0:
            assert b["nseg"] == 1 and F >= R + C - 1
        elif b["mode"] == 1:  # column segments: every segment's convolution fits
            assert F >= R + b["S"] - 1 and b["nseg"] * b["S"] >= C > (b["nseg"] - 1) * b["S"]
        else:
            assert F >= b["S"] + C - 1 and b["nseg"] * b["S"] >= R > (b["nseg"] - 1) * b["S"]
        assert k0 > info["direct_rows"] and n0 > info["direct_cols"]
        # every entry of the block has z~ = r~_k omega~_n >= s (corner is the minimum)
        v, far = p.entry(k0, n0)
        assert far
        covered[k0:k1 + 1] += n1 - n0 + 1
    total_near = 0
    for k in range(1, N + 1):
        ne = p.near_prefix(k)
        assert covered[k] == N - ne  # far columns of row k are exactly ne+1..N
        total_near += ne
    assert total_near == info["near_count"]
    assert info["near_count"] + info["far_count"] == N * N


def _z_tilde(task, nu, N, grid, k, n):
    # exact-grid argument r~_k omega~_n of a block corner, from the definitions of Sections 4-6
    if task == "schlomilch":
        r = (k - 1) / (N - 1) if grid == "unit" else k / N
        return r * (n + nu) * math.pi
    if task == "fourier_bessel":
        r = (k - 1) / (N - 1) if grid == "unit" else k / N
        return r * (n - 0.25) * math.pi
    return (k - 0.25) / (N + 0.75) * (n - 0.25) * math.pi


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-nu%d-N%d-%g-%s" % c)
def test_far_blocks_satisfy_criterion(case):
    task, nu, N, eps, grid = case
    p = hk.Plan(task, nu, N, eps, grid=grid, host_only=True)
    s = p.info["s"]
    for b in p.blocks():
        assert _z_tilde(task, nu, N, grid, b["k0"], b["n0"]) >= s * (1 - 1e-12)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-nu%d-N%d-%g-%s" % c)
def test_entries_against_oracle(case):
    # The plan's value for each entry (near-field evaluator or far-field expansion with every
    # stacked column) is within eps of J_nu(r_k omega_n) (Sections 3-6: each expansion is used
    # only where it is eps-accurate); with the columns each block keeps and its low-rank form
    # it is within 2.5 eps.
    task, nu, N, eps, grid = case
    p = hk.Plan(task, nu, N, eps, grid=grid, host_only=True, prune=False)
    pk = hk.Plan(task, nu, N, eps, grid=grid, host_only=True)
    info = p.info
    rows = sorted({1, 2, info["direct_rows"] + 1, N // 7, N // 2, N - 1, N})
    eye = np.eye(N)
    for k in rows:
        ref = oracle.transform(task, nu, N, eye, rows=np.array([k - 1]), grid=GRID[grid])[:, 0]
        near_tol = max(4e-15, 0.011 * eps)  # the J table's degree keeps its error below eps/100
        for n in range(1, N + 1, 3):
            v, far = p.entry(k, n)
            tol = eps if far else near_tol
            assert abs(v - ref[n - 1]) <= tol, (k, n, far, v, ref[n - 1])
            vk, fk = pk.entry(k, n)
            assert fk == far and abs(vk - ref[n - 1]) <= (2.5 * eps if far else near_tol), (k, n, vk)


@pytest.mark.parametrize("case", [c for c in CASES if c[0] != "schlomilch"] + [("dht", 0, 20000, 1e-15, "unit")],
                         ids=lambda c: "%s-nu%d-N%d-%g-%s" % c)
def test_kept_columns_change_entries_within_their_bound(case):
    # Each block leaves out stacked columns whose bound max|W_l| max|T_l| sums to at most
    # eps split over the blocks of one row; the plan's far entries move by no more than that
    # (plus rounding) against the plan that keeps every column.
    task, nu, N, eps, grid = case
    p = hk.Plan(task, nu, N, eps, grid=grid, host_only=True, lowrank=False)
    q = hk.Plan(task, nu, N, eps, grid=grid, host_only=True, prune=False)
    info, blocks = p.info, p.blocks()
    assert all(b["ncols"] == info["ncols"] for b in q.blocks())
    assert q.info["block_cols"] == info["ncols"] * len(q.blocks())
    per_row = np.zeros(N + 2, dtype=int)
    for b in blocks:
        per_row[b["k0"]:b["k1"] + 1] += 1
        assert 1 <= b["ncols"] <= info["ncols"]
    for b in blocks:
        assert b["dropped"] <= eps / per_row.max() * (1 + 1e-12)
    rng = np.random.default_rng(5)
    for b in blocks:
        ks = rng.integers(b["k0"], b["k1"] + 1, 6)
        ns = rng.integers(b["n0"], b["n1"] + 1, 6)
        for k, n in zip(ks, ns):
            vp, fp = p.entry(k, n)
            vq, fq = q.entry(k, n)
            assert fp and fq
            assert abs(vp - vq) <= b["dropped"] + 4e-16, (k, n, vp, vq, b)


def _fft_work(plan):
    return sum((b["nseg"] + 1 if b["mode"] else 2) * b["F"] * math.log2(b["F"]) * b["ncols"] for b in plan.blocks())


def test_column_selection_shrinks_the_workload_transforms():
    # DHT-0 at N = 2^20: rows and columns far from the near field barely feel the perturbations
    # e_k omega_n and r b_n, so most of the 290 (eps = 1e-15) or 90 (1e-8) stacked columns go;
    # cutting the blocks further from the near field drops more, and the blocks' low-rank forms
    # need fewer terms still
    for eps, full in [(1e-15, 290), (1e-8, 90)]:
        p = hk.Plan("dht", 0, 2 ** 20, eps, host_only=True, refine=False, lowrank=False)
        r = hk.Plan("dht", 0, 2 ** 20, eps, host_only=True, max_nrhs=16, lowrank=False)
        lr = hk.Plan("dht", 0, 2 ** 20, eps, host_only=True, max_nrhs=16)
        q = hk.Plan("dht", 0, 2 ** 20, eps, host_only=True, prune=False)
        assert p.info["ncols"] == full and all(b["ncols"] == full for b in q.blocks())
        assert _fft_work(p) < 0.2 * _fft_work(q)
        assert _fft_work(r) < 0.7 * _fft_work(p)
        assert _fft_work(lr) < 0.6 * _fft_work(r)
        assert all(b["ncols"] < b["kept"] for b in lr.blocks() if b["lowrank"])


@pytest.mark.parametrize("task,nu,N,eps", [("dht", 0, 20000, 1e-15), ("dht", 0, 2 ** 17, 1e-8),
                                           ("fourier_bessel", 0, 20000, 1e-15), ("schlomilch", 1, 20000, 1e-15),
                                           ("dht", 0, 20000, 1e-4)])
def test_lowrank_forms_match_the_kept_columns(task, nu, N, eps):
    # a block's low-rank form (Chebyshev interpolation in log k, log n of a cross approximation)
    # agrees with the expansion over every stacked column to eps/2 plus the block's drop bound
    # at entries other than the ones it was validated on
    p = hk.Plan(task, nu, N, eps, host_only=True)
    blocks = p.blocks()
    assert sum(b["lowrank"] for b in blocks) >= len(blocks) // 2
    rng = np.random.default_rng(19)
    for b in blocks:
        if not b["lowrank"]:
            continue
        assert b["ncols"] < b["kept"] and b["lowrank_err"] <= 0.5 * eps
        ks = rng.integers(b["k0"], b["k1"] + 1, 40)
        ns = rng.integers(b["n0"], b["n1"] + 1, 40)
        for k, n in zip(ks, ns):
            vp, far = p.entry(k, n)
            vq = p.expansion_entry(k, n)
            assert far and abs(vp - vq) <= 0.5 * eps + b["dropped"] + 4e-16, (k, n, vp, vq, b)


@pytest.mark.parametrize("task,nu,N,eps,grid", [("dht", 0, 300, 1e-15, "unit"), ("schlomilch", 0, 300, 1e-8, "paper"),
                                                ("fourier_bessel", 0, 300, 1e-15, "paper")])
def test_expansion_without_the_partition_fails_the_bar(task, nu, N, eps, grid):
    # Negative test: the far-field expansion used for every entry (the partition dropped) misses
    # 10 eps sum|c| by orders of magnitude, because Eq. (4) is only eps-accurate for z >= s
    # (Section 3.1); the plan's own entries (partition of Eq. 19) meet the bar.
    p = hk.Plan(task, nu, N, eps, grid=grid, host_only=True)
    c = np.random.default_rng(11).standard_normal(N)
    A_exp = np.array([[p.expansion_entry(k, n) for n in range(1, N + 1)] for k in range(1, N + 1)])
    A_plan = np.array([[p.entry(k, n)[0] for n in range(1, N + 1)] for k in range(1, N + 1)])
    ref = oracle.transform(task, nu, N, c, grid=GRID[grid])
    bound = 10 * eps * np.abs(c).sum()
    assert np.all(np.isfinite(A_exp))
    assert np.max(np.abs(A_plan @ c - ref)) <= bound
    assert np.max(np.abs(A_exp @ c - ref)) > 1e3 * bound
    # where the plan itself uses the expansion, the two agree to within the drop bound
    far = np.array([[p.entry(k, n)[1] for n in range(1, N + 1)] for k in range(1, N + 1)])
    assert far.any()
    assert np.max(np.abs(A_exp[far] - A_plan[far])) <= eps


def test_dht_inverse_weights():
    # v_n = 2/J_1(j_{0,n})^2: J_1(j_{0,1}) = 0.5191474972894669 (the first extremum value of J_1 at
    # the first zero of J_0); the rest against the oracle's exact-phase J_1 at (n-1/4)pi + b_n,
    # across the switch from the small-root recurrence to the large-root expansion
    N = 20000
    v = hk.dht_inverse_weights(N)
    assert abs(v[0] - 2.0 / 0.5191474972894669 ** 2) <= 4e-15 * v[0]
    b = oracle.j0_zero_offsets(N)
    idx = np.unique(np.concatenate([np.arange(1, 40), np.linspace(1, N, 300).astype(int)]))
    ref = np.array([2.0 / oracle.besselj_pi(1, 4 * n - 1, 4, b[n - 1]) ** 2 for n in idx])
    assert np.max(np.abs(v[idx - 1] / ref - 1)) <= 4e-15
    # large-root limit: J_1(j_{0,n})^2 ~ 2/(pi j_{0,n}), so v_n ~ pi j_{0,n}
    n = np.arange(N - 10, N + 1)
    assert np.max(np.abs(v[n - 1] / (np.pi * ((n - 0.25) * np.pi + b[n - 1])) - 1)) < 1e-9


@pytest.mark.parametrize("N,eps", [(2000, 1e-15), (3000, 1e-12)])
def test_near_entries_match_oracle_j(N, eps):
    # An FP64 plan's near-field entries are J_0(z) from the Q62 fixed-point Taylor table (the
    # host restatement of the device evaluation). Schlomilch on the paper grid has
    # z = (k/N)(n pi) exactly as the plan forms it, so each entry is checked against the oracle's
    # double-double J_0(z): within half an ulp of rounding, the truncation of the fixed-point
    # Horner rule (< 2^-61), the table's Taylor remainder (eps/100) and the oracle's own rounding.
    p = hk.Plan("schlomilch", 0, N, eps, grid="paper", host_only=True)
    assert p.info["precision"] == 1  # FP64 below eps = 1e-11
    rng = np.random.default_rng(23)
    checked = 0
    for k in rng.integers(1, N + 1, 60):
        ne = p.near_prefix(int(k))
        if ne == 0:
            continue
        for n in rng.integers(1, ne + 1, 12):
            v, far = p.entry(int(k), int(n))
            assert not far
            z = (int(k) / N) * (int(n) * math.pi)
            ref = oracle.besselj_dd(0, z)
            assert abs(v - ref) <= 2.5e-16 + eps / 100, (k, n, z, v, ref)
            checked += 1
    assert checked > 100
