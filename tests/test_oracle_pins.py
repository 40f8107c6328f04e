"""Pins for the CPU oracle against facts fixed outside the oracle itself.

Each test ties one part of the oracle to something it cannot reproduce by
construction: a printed value, an identity of the Bessel functions, an
independent arbitrary-precision library (mpmath), or a double-double brute
force that takes a different route to the same numbers.
"""
import math

import numpy as np
import pytest

import oracle
from hankel_inputs import coefficients

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 40

REGIME_Z = [1e-6, 0.3, 1.0, 1.99, 2.01, 4.5, 9.9, 17.8, 24.99, 25.01, 31.4, 60.0, 99.5, 180.0]


def test_first_zero_of_j0():
    # j_{0,1} = 2.404825557695773 (value quoted with the oracle's tolerance rule).
    b = oracle.j0_zero_offsets(1)
    assert abs(0.75 * math.pi + b[0] - 2.404825557695773) <= 4.5e-16


@pytest.mark.parametrize("nu", [0, 1, 2, 4, 10])
def test_besselj_against_mpmath(nu):
    for z in REGIME_Z:
        ref = float(mpmath.besselj(nu, z))
        assert abs(oracle.besselj(nu, z) - ref) <= 1e-15, (nu, z)
        assert abs(oracle.besselj_dd(nu, z) - ref) <= 2e-16, (nu, z)


def test_negative_order_reflection():
    # J_{-nu} = (-1)^nu J_nu (DLMF 10.4.1), used by the Neumann sums of Section 5.
    for nu in range(1, 7):
        for z in (0.7, 8.0, 40.0):
            assert oracle.besselj(-nu, z) == (-1) ** nu * oracle.besselj(nu, z)


def test_three_term_recurrence():
    # J_{nu-1}(z) + J_{nu+1}(z) = (2 nu / z) J_nu(z)  (DLMF 10.6.1)
    for nu in range(1, 12):
        for z in REGIME_Z[1:] + [500.0, 2345.6]:
            lhs = oracle.besselj(nu - 1, z) + oracle.besselj(nu + 1, z)
            rhs = 2.0 * nu / z * oracle.besselj(nu, z)
            assert abs(lhs - rhs) <= 4e-15 * max(1.0, 2.0 * nu / z), (nu, z)


def test_sum_of_squares():
    # J_0(z)^2 + 2 sum_{s>=1} J_s(z)^2 = 1  (DLMF 10.23.3)
    for z in (0.5, 3.0, 17.0, 30.0, 80.0):
        smax = int(z) + 60
        total = oracle.besselj(0, z) ** 2 + 2.0 * sum(oracle.besselj(s, z) ** 2 for s in range(1, smax))
        assert abs(total - 1.0) <= 2e-15, z


def test_schlomilch_closed_form_loose():
    # sum_{n>=1} J_0(n x) = -1/2 + 1/x on (0, 2 pi) (Schlomilch series). The partial sums
    # oscillate and converge slowly, so compare the Cesaro mean of the partial sums.
    for x in (0.5, 1.0, 2.0):
        n = np.arange(1, 40001)
        vals = np.array([oracle.besselj(0, v) for v in n * x])
        partial = np.cumsum(vals)
        mean = partial[20000:].mean()
        assert abs(mean - (-0.5 + 1.0 / x)) < 2e-3, x


def test_zeros_against_mpmath_and_lemma_bounds():
    n_all = 100000
    b = oracle.j0_zero_offsets(n_all)
    n = np.arange(1, n_all + 1, dtype=np.float64)
    # Lemma 3.2: 0 <= b_n <= 1 / (8 (n - 1/4) pi), for every n computed.
    assert np.all(b >= 0.0)
    assert np.all(b <= 1.0 / (8.0 * (n - 0.25) * math.pi))
    for k in (1, 2, 3, 7, 30, 31, 1000, 54321, 100000):
        ref = mpmath.besseljzero(0, k) - (k - mpmath.mpf(1) / 4) * mpmath.pi
        assert abs(b[k - 1] - float(ref)) <= 2e-17 + 1e-15 * abs(float(ref)), k


def test_zero_offsets_double_double_agree():
    b = oracle.j0_zero_offsets(200)
    bdd = oracle.j0_zero_offsets_dd(200)
    assert np.max(np.abs(b - bdd) / bdd) <= 4e-15


def test_dht_row_perturbation_bound():
    # Lemma 3.2: |e_{k,N}| <= 1 / (8 (N+3/4) (k-1/4) pi^2), e_k = j_{0,k}/j_{0,N+1} - (k-1/4)/(N+3/4)
    for N in (64, 1000, 4096):
        b = oracle.j0_zero_offsets(N + 1)
        k = np.arange(1, N + 1, dtype=np.float64)
        jN1 = (N + 0.75) * math.pi + b[N]
        e = (b[:N] * (N + 0.75) - b[N] * (k - 0.25)) / (jN1 * (N + 0.75))
        assert np.all(np.abs(e) <= 1.0 / (8.0 * (N + 0.75) * (k - 0.25) * math.pi ** 2))


@pytest.mark.parametrize("P,Q,delta,nu", [
    (123456789013, 4194307 * 4, 0.0, 0),
    (4 * 1048575 * 4194303 + 3, 16 * 1048575, 3.2e-4, 0),
    (1048575 * 1048576, 1048575, 0.0, 1),
    (987654321, 1234, -2.5e-3, 4),
])
def test_exact_phase_reduction_large_argument(P, Q, delta, nu):
    z = mpmath.pi * mpmath.mpf(P) / Q + delta
    ref = float(mpmath.besselj(nu, z))
    amp = float(mpmath.sqrt(2 / (mpmath.pi * z)))
    assert abs(oracle.besselj_pi(nu, P, Q, delta) - ref) <= 4e-16 * max(amp, 1e-3) + 1e-19


def test_two_point_schlomilch_by_hand():
    # N = 2, nu = 0, r = (0, 1), omega = (pi, 2 pi): f_1 = c_1 + c_2, f_2 = c_1 J_0(pi) + c_2 J_0(2 pi).
    c = np.array([0.3, -1.7])
    f = oracle.transform("schlomilch", 0, 2, c)
    assert abs(f[0] - (c[0] + c[1])) <= 1e-16
    ref = c[0] * float(mpmath.besselj(0, mpmath.pi)) + c[1] * float(mpmath.besselj(0, 2 * mpmath.pi))
    assert abs(f[1] - ref) <= 4e-16


@pytest.mark.parametrize("task,nu,grid", [
    ("schlomilch", 0, 0), ("schlomilch", 1, 0), ("schlomilch", 4, 0), ("schlomilch", 0, 1),
    ("fourier_bessel", 0, 0), ("fourier_bessel", 1, 1), ("dht", 0, 0),
])
@pytest.mark.parametrize("N", [2, 3, 17, 64])
def test_double_double_brute_force(task, nu, grid, N):
    c = coefficients("normal", N, 2, 100 + N)
    f = oracle.transform(task, nu, N, c, grid=grid)
    fdd = oracle.transform_dd(task, nu, N, c, grid=grid)
    scale = np.abs(c).sum(axis=1, keepdims=True)
    assert np.max(np.abs(f - fdd) / scale) <= 1e-15


def test_dht_entries_against_mpmath():
    # A few rows of the DHT at N = 300 summed in 40-digit arithmetic.
    N = 300
    c = coefficients("normal", N, 1, 4)[0]
    zeros = [mpmath.besseljzero(0, n) for n in range(1, N + 2)]
    rows = np.array([0, 1, 150, 299], dtype=np.int64)
    f = oracle.transform("dht", 0, N, c, rows=rows)
    for i, k in enumerate(rows):
        acc = mpmath.mpf(0)
        for n in range(N):
            acc += c[n] * mpmath.besselj(0, zeros[k] * zeros[n] / zeros[N])
        assert abs(f[i] - float(acc)) <= 1e-15 * np.abs(c).sum()


@pytest.mark.parametrize("N,tol", [(50, 2e-8), (100, 2e-9), (200, 6e-10), (400, 2e-11)])
def test_dht_self_inverse(N, tol):
    # Eq. (27)-(28): (1/j_{0,N+1}^2) J D_v J D_v c ~ c with v_n = 2 / J_1(j_{0,n})^2. The
    # residual shrinks as N grows (Fig. 8, N < 700); a wrong node or a dropped term breaks it.
    c = coefficients("normal", N, 1, 7)[0]
    b = oracle.j0_zero_offsets(N + 1)
    j = (np.arange(1, N + 2) - 0.25) * math.pi + b
    v = np.array([2.0 / oracle.besselj_pi(1, 4 * n - 1, 4, b[n - 1]) ** 2 for n in range(1, N + 1)])
    y = oracle.transform("dht", 0, N, v * c)
    ct = oracle.transform("dht", 0, N, v * y) / j[N] ** 2
    assert np.max(np.abs(ct - c)) <= tol


def test_rows_subset_matches_full():
    N = 257
    c = coefficients("uniform", N, 3, 11)
    full = oracle.transform("fourier_bessel", 0, N, c)
    rows = np.array([0, 5, 128, 256], dtype=np.int64)
    part = oracle.transform("fourier_bessel", 0, N, c, rows=rows, nthreads=2)
    assert np.array_equal(full[:, rows], part)
