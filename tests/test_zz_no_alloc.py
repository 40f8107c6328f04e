"""The allocation-free entry point hankel_exec_static, checked against hankel_exec.

Callers whose device memory all belongs to their own pool allocator, or whose transform loop
must never enter the CUDA allocator, cannot have the library allocate when they run a
transform. hankel_exec_static serves them from a static device array inside the library.
These tests call it through the C ABI, three times in a row on the same plan, compare each
result with hankel_exec's within the parity tolerance 10 eps sum|c_n|, and check that the
device's free memory stays the same across the calls. The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from hankel_inputs import coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_01652_gb300 as hk  # noqa: E402
from paper_1501_01652_gb300 import _lib  # noqa: E402


@pytest.mark.parametrize("task,nu,N,eps", [
    ("dht", 0, 3000, 1e-15), ("fourier_bessel", 0, 2 ** 16, 1e-8), ("schlomilch", 4, 4096, 1e-15),
    ("dht", 0, 2 ** 20, 1e-8), ("dht", 0, 2 ** 18, 1e-4),
])
def test_static_scratch_matches_exec(task, nu, N, eps):
    lib = _lib.load()
    plan = hk.Plan(task, nu, N, eps)
    c = torch.from_numpy(coefficients("normal", N, 1, 77)[0]).cuda()
    ref = torch.empty(N, dtype=torch.float64, device="cuda")
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    _lib.check(lib.hankel_exec(plan.handle, ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(ref.data_ptr()), sp),
               "hankel_exec")
    tol = 10.0 * eps * float(c.abs().sum())
    free_after_first = None
    for _ in range(3):
        out.fill_(float("nan"))  # a result left over from an earlier call cannot pass
        _lib.check(lib.hankel_exec_static(plan.handle, ctypes.c_void_p(c.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), sp), "hankel_exec_static")
        torch.cuda.synchronize()
        err = float((out - ref).abs().max())
        assert np.isfinite(err) and err <= tol, (err, tol)
        # the calls allocate nothing: the device's free memory does not move after the first
        free = torch.cuda.mem_get_info()[0]
        if free_after_first is None:
            free_after_first = free
        assert free == free_after_first


def test_static_scratch_rejects_oversized_plans():
    lib = _lib.load()
    plan = hk.Plan("schlomilch", 0, 2 ** 21, 1e-4, precision="fp64")  # largest transform: 2^22 FP64 points
    c = torch.zeros(2 ** 21, dtype=torch.float64, device="cuda")
    f = torch.zeros_like(c)
    st = lib.hankel_exec_static(plan.handle, ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(f.data_ptr()), None)
    assert _lib.STATUS_NAMES[st] == "HANKEL_EUNSUPPORTED"
