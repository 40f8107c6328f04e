"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the transform: it only draws coefficient
vectors with the distributions of the paper's experiments and of the
workload table (uniform on [-1, 1]; decaying u_n/n^2 with u_n uniform;
standard normal as in the paper's Gaussian experiments, Sections 5.2 and
6.1). Seeds follow ``seed = workload_index * 1000 + batch_index`` so every
consumer draws bit-identical inputs from numpy's PCG64.
"""
import numpy as np

KINDS = ("uniform", "decaying", "normal")

# Named workloads: (task, nu, N values, coefficient kind, eps values, batch sizes).
WORKLOADS = {
    1: dict(name="schlomilch_nu0_N4096", task="schlomilch", nus=(0,), Ns=(4096,),
            kind="uniform", eps=(1e-15,), batches=(1,)),
    2: dict(name="schlomilch_nu014", task="schlomilch", nus=(0, 1, 4), Ns=(2**16, 2**20, 2**22),
            kind=("uniform", "decaying"), eps=(1e-15, 1e-8, 1e-4), batches=(32,)),
    3: dict(name="fourier_bessel_nu0", task="fourier_bessel", nus=(0,), Ns=(2**18, 2**20, 2**22),
            kind="uniform", eps=(1e-15, 1e-8), batches=(1,)),
    4: dict(name="dht_nu0", task="dht", nus=(0,), Ns=(2**16, 2**20, 2**22),
            kind="normal", eps=(1e-15, 1e-8, 1e-4), batches=(1, 16, 128)),
}


def seed_for(workload, batch=0):
    return int(workload) * 1000 + int(batch)


def coefficients(kind, N, nrhs=1, seed=0):
    """Return an (nrhs, N) float64 array of coefficients c_n, n = 1..N."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "uniform":
        c = rng.uniform(-1.0, 1.0, size=(nrhs, N))
    elif kind == "decaying":
        n = np.arange(1, N + 1, dtype=np.float64)
        c = rng.uniform(-1.0, 1.0, size=(nrhs, N)) / (n * n)
    elif kind == "normal":
        c = rng.standard_normal(size=(nrhs, N))
    else:
        raise ValueError("unknown coefficient kind %r" % (kind,))
    return np.ascontiguousarray(c, dtype=np.float64)


def sample_rows(N, count, seed):
    """Sorted distinct 0-based row indices, always including the first and last rows."""
    rng = np.random.Generator(np.random.PCG64(seed))
    count = min(int(count), int(N))
    rows = rng.choice(N, size=count, replace=False)
    rows = np.unique(np.concatenate([rows, [0, N - 1]]))
    return rows.astype(np.int64)
