"""Planner parameters against the values the paper prints (Tables 1-3, Section 5, Section 4.3)."""
import math
import os

import pytest

import paper_1501_01652_gb300 as hk
from paper_1501_01652_gb300 import _lib

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    """Rows of a fixture under tests/golden: first column an int key, the rest printed values
    (floats; tokens in e-notation stay strings, the paper's one-significant-digit entries)."""
    rows = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            rows[int(line[0])] = [t if "e" in t else float(t) for t in line[1:]]
    return rows


TABLE1 = _golden("table1_s_nu_M_1e-15.txt")  # s_{nu,M}(1e-15), M = 3..12 (Table 1)
TABLE2 = _golden("table2_t_nu_T_1e-15.txt")  # t_{nu,T}(1e-15), T = 1..9 (Table 2)
TABLE3 = [v[0] for _, v in sorted(_golden("table3_neumann_radius_1e-15.txt").items())]  # K = 3..10 (Table 3)


def _matches_printed(value, printed):
    if isinstance(printed, str):  # one significant digit, e.g. "6e-8"
        return float("%.0e" % value) == float(printed)
    return round(value, 3) == printed


@pytest.mark.parametrize("nu", sorted(TABLE1))
def test_table1_s_values(nu):
    for M, printed in zip(range(3, 13), TABLE1[nu]):
        assert round(hk.s_nu_M(nu, M, 1e-15), 1) == printed, (nu, M)


@pytest.mark.parametrize("nu", sorted(TABLE2))
def test_table2_t_values(nu):
    for T, printed in zip(range(1, 10), TABLE2[nu]):
        assert _matches_printed(hk.t_nu_T(nu, T, 1e-15), printed), (nu, T)


def test_table3_neumann_radius():
    for K, printed in zip(range(3, 11), TABLE3):
        assert _matches_printed(hk.neumann_radius(K, 1e-15), printed), K


def test_lemma31_radius_meets_bound():
    for K in range(1, 12):
        r = hk.neumann_radius(K, 1e-15)
        assert abs(5.2 * (math.e * r / 2) ** K - 1e-15) <= 1e-25


def test_section5_worked_numbers():
    # p_6(1e-15) ~ 22.7 and q_3(1e-15) ~ 3.7; K = 6, T = 3 at 1e-15; (2K-1)T = 33 vs 2T+K-2 = 10
    # (printed to one decimal: the value lies in [printed, printed + 0.1))
    w = {}
    with open(os.path.join(GOLDEN, "section5_worked_numbers_1e-15.txt")) as fh:
        for line in fh:
            t = line.split("#", 1)[0].split()
            if t:
                w[t[0]] = float(t[1])
    assert w["p_6"] <= hk.p_K(6, 1e-15) < w["p_6"] + 0.1
    assert w["q_3"] <= hk.q_T(3, 1e-15) < w["q_3"] + 0.1
    p = hk.params("fourier_bessel", 0, 4096, 1e-15)
    assert (p["K"], p["T"]) == (int(w["K"]), int(w["T"]))
    assert p["npairs"] == int(w["rearranged_count"]) and (2 * p["K"] - 1) * p["T"] == int(w["full_count"])
    assert p["direct_cols"] == 22  # the first floor(p_6) columns are summed directly
    assert hk.p_K(5, 1e-15) > 30 and hk.q_T(2, 1e-15) > 30


def test_dht_counts():
    p = hk.params("dht", 0, 2 ** 20, 1e-15)
    assert (p["K"], p["T"], p["M"]) == (6, 3, 10)
    assert p["npairs"] == 100  # (2T+K-2)^2 Schlomilch evaluations
    assert p["direct_rows"] == math.floor(1.01 * max(hk.p_K(6, 1e-15), hk.q_T(3, 1e-15)))
    assert p["mu_max"] == 10


def test_table4_M_rule():
    for eps, M in [(1e-15, 10), (1e-8, 5), (1e-4, 3), (1e-3, 3), (1e-12, 8)]:
        assert hk.params("schlomilch", 0, 1000, eps)["M"] == M


def test_partition_count_crossover_paper_grid():
    # Section 4.3: for N <= 158 the number of partitions P is 0 (nu = 0, eps = 1e-15, r_k = k/N).
    for N in (20, 100, 150, 158):
        assert hk.params("schlomilch", 0, N, 1e-15, grid="paper")["P"] == 0
    for N in (159, 160, 1000):
        assert hk.params("schlomilch", 0, N, 1e-15, grid="paper")["P"] >= 1


def test_table4_beta_P():
    for N in (4096, 2 ** 16, 2 ** 20):
        p = hk.params("schlomilch", 0, N, 1e-15)
        beta = min(3 / math.log(N), 1)
        alpha = math.sqrt(hk.s_nu_M(0, 10, 1e-15) / math.pi)
        assert p["beta"] == pytest.approx(beta, rel=1e-15)
        assert p["alpha"] == pytest.approx(alpha, rel=1e-15)
        assert p["P"] == max(0, math.ceil(math.log(30 / (alpha * math.sqrt(N))) / math.log(beta)))


@pytest.mark.parametrize("bad", [
    dict(task="dht", nu=1, N=100, eps=1e-8), dict(task="schlomilch", nu=0, N=1, eps=1e-8),
    dict(task="schlomilch", nu=-1, N=100, eps=1e-8), dict(task="schlomilch", nu=0, N=100, eps=1.5),
])
def test_invalid_requests(bad):
    with pytest.raises(RuntimeError, match="EINVAL"):
        hk.params(**bad)


def test_unsupported_requests():
    with pytest.raises(RuntimeError, match="EUNSUPPORTED"):
        hk.params("schlomilch", 0, 100, 1e-17)
    with pytest.raises(RuntimeError, match="EUNSUPPORTED"):
        hk.params("schlomilch", 0, 100, 1e-8, precision="fp32")


def test_status_strings_and_fault_injection_arguments():
    lib = _lib.load()
    assert lib.hankel_status_string(6) == b"request cancelled"
    assert lib.hankel_status_string(99) == b"unknown status"
    assert lib.hankel_debug_fail_allocs(-1, 1) == 1   # EINVAL
    assert lib.hankel_debug_fail_allocs(0, 0) == 0
