"""GB300-native fast Hankel-type transforms (Townsend, arXiv:1501.01652).

Thin Python binding over the C ABI of ``include/hankel.h``: every step of the
transform runs in the CUDA library ``_build/libhankel.so``; this module only
marshals arguments (torch CUDA tensors or numpy arrays) and raises on error.
There is no CPU fallback: if the library cannot be built or a CUDA call fails,
the call raises.
"""
import ctypes

import numpy as np

from . import _lib

TASKS = {"schlomilch": 0, "fourier_bessel": 1, "dht": 2}
GRIDS = {"unit": 0, "paper": 1}
PRECISIONS = {"auto": 0, "fp64": 1, "fp32": 2, "df64": 3, "mixed": 4}


def _options(task, nu, N, eps, grid="unit", gamma=None, precision="auto", max_nrhs=1, workspace_limit=0,
             host_only=False, segment=True, prune=True, refine=True, lowrank=True, mixed_terms=True, autotune=True,
             tensor_fft=False):
    lib = _lib.load()
    o = _lib.Options()
    _lib.check(lib.hankel_options_default(ctypes.byref(o), TASKS[task], int(nu), int(N), float(eps)),
               "hankel_options_default")
    o.grid = GRIDS[grid]
    if gamma is not None:
        o.gamma = int(gamma)
    o.precision = PRECISIONS[precision]
    o.max_nrhs = int(max_nrhs)
    o.workspace_limit = int(workspace_limit)
    o.flags = ((_lib.FLAG_HOST_ONLY if host_only else 0) | (0 if segment else _lib.FLAG_NO_SEGMENT)
               | (0 if prune else _lib.FLAG_ALL_COLUMNS)
               | (0 if refine else _lib.FLAG_NO_REFINE) | (0 if lowrank else _lib.FLAG_NO_LOWRANK)
               | (0 if mixed_terms else _lib.FLAG_UNIFORM_TERMS) | (0 if autotune else _lib.FLAG_NO_AUTOTUNE)
               | (_lib.FLAG_TENSOR_FFT if tensor_fft else 0))
    return o


def params(task, nu, N, eps, **kw):
    """Parameters (Table 4, Eqs. 23-24) a plan would choose, as a dict; no GPU needed."""
    lib = _lib.load()
    o = _options(task, nu, N, eps, **kw)
    info = _lib.Info()
    _lib.check(lib.hankel_params(ctypes.byref(o), ctypes.byref(info)), "hankel_params")
    return info.as_dict()


def s_nu_M(nu, M, eps):
    return _lib.load().hankel_s_nu_M(int(nu), int(M), float(eps))


def t_nu_T(nu, T, eps):
    return _lib.load().hankel_t_nu_T(int(nu), int(T), float(eps))


def neumann_radius(K, eps):
    return _lib.load().hankel_neumann_radius(int(K), float(eps))


def p_K(K, eps):
    return _lib.load().hankel_p_K(int(K), float(eps))


def q_T(T, eps):
    return _lib.load().hankel_q_T(int(T), float(eps))


def dht_inverse_weights(N):
    """v_n = 2/J_1(j_{0,n})^2, n = 1..N (host), as a numpy array."""
    lib = _lib.load()
    v = np.empty(int(N), dtype=np.float64)
    _lib.check(lib.hankel_dht_inverse_weights(int(N), v.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "hankel_dht_inverse_weights")
    return v


def j0_zero_offsets(count):
    """b_n = j_{0,n} - (n-1/4)pi, n = 1..count, from the library's node builder."""
    b = np.empty(int(count), dtype=np.float64)
    _lib.check(_lib.load().hankel_j0_zero_offsets(int(count), b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "hankel_j0_zero_offsets")
    return b


def tune_cache_put(gpu, precision, log2_len, col_bucket, radices=None, one_launch=False, ms_default=0.0,
                   ms_chosen=0.0, tensor_passes=0):
    """Store an FFT launch split in the autotuner's cache (precision: "fp64", "df64" or "fp32")."""
    s = _lib.FftShape()
    s.precision, s.log2_len, s.col_bucket = PRECISIONS[precision], int(log2_len), int(col_bucket)
    s.one_launch = 1 if one_launch else 0
    radices = list(radices or [])
    s.npass = len(radices)
    for i, r in enumerate(radices[:4]):
        s.log2_radix[i] = int(r)
    s.ms_default, s.ms_chosen = float(ms_default), float(ms_chosen)
    s.tensor_passes = int(tensor_passes)
    _lib.check(_lib.load().hankel_tune_cache_put(gpu.encode(), ctypes.byref(s)), "hankel_tune_cache_put")


def tune_cache_get(gpu, precision, log2_len, col_bucket):
    """The cached split for the key as a dict, or None."""
    s = _lib.FftShape()
    found = ctypes.c_int(0)
    _lib.check(_lib.load().hankel_tune_cache_get(gpu.encode(), PRECISIONS[precision], int(log2_len), int(col_bucket),
                                                 ctypes.byref(s), ctypes.byref(found)), "hankel_tune_cache_get")
    return s.as_dict() if found.value else None


def tune_cache_save(path):
    _lib.check(_lib.load().hankel_tune_cache_save(str(path).encode()), "hankel_tune_cache_save")


def tune_cache_load(path):
    _lib.check(_lib.load().hankel_tune_cache_load(str(path).encode()), "hankel_tune_cache_load")


def tune_cache_clear():
    _lib.check(_lib.load().hankel_tune_cache_clear(), "hankel_tune_cache_clear")


def tune_bucket(ncols):
    return _lib.load().hankel_tune_bucket(int(ncols))


def debug_fft_compare(log2_len, ncols, radices, tensor_passes=0, inverse=False):
    """Test access: seeded FP64 data through the built-in FFT split and through the given one
    (radices, bit mask of tensor-core passes); returns (max |diff| / max |ref|, ms of the given split)."""
    arr = (ctypes.c_int * 4)(*(list(radices) + [0] * (4 - len(radices))))
    err, ms = ctypes.c_double(), ctypes.c_double()
    _lib.check(_lib.load().hankel_debug_fft_compare(int(log2_len), int(ncols), int(bool(inverse)), len(radices), arr,
                                                    int(tensor_passes), ctypes.byref(err), ctypes.byref(ms)),
               "hankel_debug_fft_compare")
    return err.value, ms.value


def debug_fail_allocs(after, count):
    """Make the library's next `count` device or page-locked allocations, after `after` successful
    ones, report failure (host-side fault injection for tests; count = 0 turns it off)."""
    _lib.check(_lib.load().hankel_debug_fail_allocs(int(after), int(count)), "hankel_debug_fail_allocs")


class Plan:
    """A transform plan: f = J_nu(r omega^T) c for one task, order, size and accuracy."""

    def __init__(self, task, nu, N, eps, grid="unit", gamma=None, precision="auto", max_nrhs=1,
                 workspace_limit=0, host_only=False, segment=True, prune=True, refine=True, lowrank=True,
                 mixed_terms=True, autotune=True, tensor_fft=False):
        self._lib = _lib.load()
        self._h = ctypes.c_void_p()
        self.task, self.nu, self.N, self.eps = task, int(nu), int(N), float(eps)
        self.max_nrhs = int(max_nrhs)
        o = _options(task, nu, N, eps, grid, gamma, precision, max_nrhs, workspace_limit, host_only, segment,
                     prune, refine, lowrank, mixed_terms, autotune, tensor_fft)
        _lib.check(self._lib.hankel_plan_ex(ctypes.byref(self._h), ctypes.byref(o)), "hankel_plan_ex")

    def __del__(self):
        self.destroy()

    def destroy(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.hankel_destroy(h)
            self._h = ctypes.c_void_p()

    @property
    def handle(self):
        return self._h

    @property
    def info(self):
        info = _lib.Info()
        _lib.check(self._lib.hankel_plan_info(self._h, ctypes.byref(info)), "hankel_plan_info")
        return info.as_dict()

    def blocks(self):
        cnt = ctypes.c_int(0)
        _lib.check(self._lib.hankel_plan_blocks(self._h, None, 0, ctypes.byref(cnt)), "hankel_plan_blocks")
        arr = (_lib.Block * max(cnt.value, 1))()
        _lib.check(self._lib.hankel_plan_blocks(self._h, arr, cnt.value, ctypes.byref(cnt)), "hankel_plan_blocks")
        return [dict(k0=b.k0, k1=b.k1, n0=b.n0, n1=b.n1, F=b.fft_len, S=b.seg_len, nseg=b.nseg, mode=b.mode,
                     ncols=b.ncols, dropped=b.dropped, kept=b.kept, lowrank=bool(b.lowrank),
                     lowrank_err=b.lowrank_err, terms=(b.terms_fp64, b.terms_df64, b.terms_fp32))
                for b in arr[:cnt.value]]

    def fft_shapes(self):
        """The transform shapes the plan runs (autotuned launch splits), as dicts."""
        cnt = ctypes.c_int(0)
        _lib.check(self._lib.hankel_plan_fft_shapes(self._h, None, 0, ctypes.byref(cnt)), "hankel_plan_fft_shapes")
        arr = (_lib.FftShape * max(cnt.value, 1))()
        _lib.check(self._lib.hankel_plan_fft_shapes(self._h, arr, cnt.value, ctypes.byref(cnt)),
                   "hankel_plan_fft_shapes")
        return [a.as_dict() for a in arr[:cnt.value]]

    def entry(self, k, n):
        """(value, is_far) of the plan's representation of matrix entry (k, n), 1-based."""
        v = ctypes.c_double()
        far = ctypes.c_int()
        _lib.check(self._lib.hankel_plan_entry(self._h, int(k), int(n), ctypes.byref(v), ctypes.byref(far)),
                   "hankel_plan_entry")
        return v.value, bool(far.value)

    def expansion_entry(self, k, n):
        """The far-field expansion at entry (k, n), 1-based, ignoring the partition."""
        v = ctypes.c_double()
        _lib.check(self._lib.hankel_plan_expansion_entry(self._h, int(k), int(n), ctypes.byref(v)),
                   "hankel_plan_expansion_entry")
        return v.value

    def near_prefix(self, k):
        ne = ctypes.c_int64()
        _lib.check(self._lib.hankel_plan_near_prefix(self._h, int(k), ctypes.byref(ne)), "hankel_plan_near_prefix")
        return ne.value

    def device_status(self):
        """Status of the plan's bounded device waits since the last call ("HANKEL_OK" or
        "HANKEL_ETIMEOUT"); blocking."""
        return _lib.STATUS_NAMES[self._lib.hankel_plan_device_status(self._h)]

    def set_timing(self, enable=True):
        """Turn per-stage CUDA-event timing on or off and reset the stage statistics."""
        _lib.check(self._lib.hankel_plan_set_timing(self._h, 1 if enable else 0), "hankel_plan_set_timing")

    def stage_stats(self):
        """Accumulated per-stage statistics: {stage: {ms, flops, entries, launches}}."""
        arr = (_lib.StageStat * len(_lib.STAGES))()
        _lib.check(self._lib.hankel_plan_stage_stats(self._h, arr), "hankel_plan_stage_stats")
        return {name: {"ms": a.ms, "flops": a.flops, "entries": a.entries, "bytes": a.bytes, "launches": a.launches}
                for name, a in zip(_lib.STAGES, arr)}

    def _run(self, fn, name, c, f, stream):
        import torch

        if not (c.is_cuda and c.dtype == torch.float64):
            raise TypeError("input must be a CUDA float64 tensor")
        single = c.dim() == 1
        c2 = c.reshape(1, -1) if single else c
        if c2.shape[-1] != self.N or c2.stride(-1) != 1:
            raise ValueError("input must have N contiguous entries per row")
        nrhs = c2.shape[0]
        if f is None:
            f2 = torch.empty((nrhs, self.N), dtype=torch.float64, device=c.device)
        else:
            f2 = f.reshape(1, -1) if f.dim() == 1 else f
            if not (f2.is_cuda and f2.dtype == torch.float64) or f2.shape != (nrhs, self.N) or f2.stride(-1) != 1:
                raise ValueError("output must be a CUDA float64 tensor shaped like the input")
        if stream is None:
            stream = torch.cuda.current_stream(c.device)
        st = fn(self._h, ctypes.c_void_p(c2.data_ptr()), c2.stride(0) if nrhs > 1 else self.N,
                ctypes.c_void_p(f2.data_ptr()), f2.stride(0) if nrhs > 1 else self.N, nrhs,
                ctypes.c_void_p(stream.cuda_stream))
        _lib.check(st, name)
        if f is not None:
            return f
        return f2[0] if single else f2

    def exec(self, c, f=None, stream=None, context=0):
        """Run on torch CUDA float64 tensors of shape (N,) or (nrhs, N); returns f. context selects the
        execution context (add_context); executions on different contexts may overlap."""
        if context == 0:
            return self._run(self._lib.hankel_exec_batched, "hankel_exec_batched", c, f, stream)
        fn = self._lib.hankel_exec_batched_ctx
        return self._run(lambda h, *a: fn(h, int(context), *a), "hankel_exec_batched_ctx", c, f, stream)

    def add_context(self):
        """Another execution context (workspace) for executions in flight at once; returns its index."""
        idx = ctypes.c_int(0)
        _lib.check(self._lib.hankel_plan_add_context(self._h, ctypes.byref(idx)), "hankel_plan_add_context")
        return idx.value

    def exec_inverse(self, f, c=None, stream=None):
        """Inverse DHT (DHT plans): c = j_{0,N+1}^-2 v o J(v o f), v_n = 2/J_1(j_{0,n})^2."""
        return self._run(self._lib.hankel_exec_inverse, "hankel_exec_inverse", f, c, stream)

    def exec_host(self, c, out=None):
        """End-to-end call on host arrays (numpy float64, (N,) or (nrhs, N)); returns f."""
        c = np.ascontiguousarray(c, dtype=np.float64)
        single = c.ndim == 1
        c2 = c.reshape(1, -1) if single else c
        nrhs = c2.shape[0]
        f = out if out is not None else np.empty((nrhs, self.N), dtype=np.float64)
        dp = ctypes.POINTER(ctypes.c_double)
        st = self._lib.hankel_exec_host(self._h, c2.ctypes.data_as(dp), self.N, f.ctypes.data_as(dp), self.N, nrhs)
        _lib.check(st, "hankel_exec_host")
        return f[0] if (single and out is None) else f


class Server:
    """Request loop over cached plans (hankel_server_* of the C ABI).

    ``submit`` queues nrhs coefficient vectors (numpy float64, host memory) and returns a
    ticket; the library's dispatcher batches waiting requests of the same plan, runs batches
    of different plans concurrently on its CUDA streams and writes each result into the array
    ``submit`` returned. ``precision="fp64"`` builds every plan in FP64 (the plain form);
    ``"auto"`` picks per plan: FP64 below eps = 1e-5 and FP32 stages at eps >= 1e-5;
    ``"mixed"`` opts into narrower arithmetic below 1e-5 (double-float transforms for
    1e-11 <= eps < 1e-5, small low-rank terms in double-float or FP32).
    """

    def __init__(self, streams=4, max_batch=64, use_graphs=False, precision="auto", memory_cap=0, pack=True,
                 batch_window_us=None, contexts_per_plan=None, small_batch=None):
        self._lib = _lib.load()
        o = _lib.ServerOptions()
        _lib.check(self._lib.hankel_server_options_default(ctypes.byref(o)), "hankel_server_options_default")
        o.streams, o.max_batch, o.use_graphs = int(streams), int(max_batch), int(bool(use_graphs))
        o.precision = PRECISIONS[precision]
        o.pack_requests = 1 if pack else 0
        if batch_window_us is not None:
            o.batch_window_us = int(batch_window_us)
        if contexts_per_plan is not None:
            o.contexts_per_plan = int(contexts_per_plan)
        if small_batch is not None:
            o.small_batch = int(small_batch)
        if memory_cap:
            o.memory_cap = int(memory_cap)
        self._h = ctypes.c_void_p()
        _lib.check(self._lib.hankel_server_create(ctypes.byref(self._h), ctypes.byref(o)), "hankel_server_create")
        self._live = {}  # ticket -> (c, f) kept alive until completion

    def submit(self, task, nu, N, eps, c, f=None):
        """Queue c ((N,) or (nrhs, N) float64); returns (ticket, f) with f filled on completion.
        f: optional output array shaped like c (page-locked arrays skip the staging copies)."""
        c = np.ascontiguousarray(c, dtype=np.float64)
        c2 = c.reshape(1, -1) if c.ndim == 1 else c
        if f is None:
            f = np.empty_like(c2)
        else:
            if f.dtype != np.float64 or not f.flags["C_CONTIGUOUS"] or f.size != c2.size:
                raise ValueError("f must be a contiguous float64 array shaped like c")
            f = f.reshape(c2.shape)
        t = ctypes.c_int64()
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.check(self._lib.hankel_server_submit(self._h, TASKS[task], int(nu), int(N), float(eps),
                                                  c2.ctypes.data_as(dp), f.ctypes.data_as(dp), c2.shape[0],
                                                  ctypes.byref(t)), "hankel_server_submit")
        self._live[t.value] = (c2, f)
        return t.value, (f[0] if c.ndim == 1 else f)

    def wait(self, ticket):
        """Block until `ticket` completes; returns its latency in ms. Raises if the request failed."""
        st = ctypes.c_int()
        lat = ctypes.c_double()
        _lib.check(self._lib.hankel_server_wait(self._h, int(ticket), ctypes.byref(st), ctypes.byref(lat)),
                   "hankel_server_wait")
        self._live.pop(int(ticket), None)
        _lib.check(st.value, "request %d" % ticket)
        return lat.value

    def cancel(self, ticket):
        """Cancel a request still waiting for dispatch; returns True if it was cancelled (it then
        completes with HANKEL_ECANCELED and wait() raises)."""
        done = ctypes.c_int(0)
        _lib.check(self._lib.hankel_server_cancel(self._h, int(ticket), ctypes.byref(done)), "hankel_server_cancel")
        return bool(done.value)

    def status(self, ticket):
        """Block until `ticket` completes; returns (status name, latency ms) without raising."""
        st = ctypes.c_int()
        lat = ctypes.c_double()
        _lib.check(self._lib.hankel_server_wait(self._h, int(ticket), ctypes.byref(st), ctypes.byref(lat)),
                   "hankel_server_wait")
        self._live.pop(int(ticket), None)
        return _lib.STATUS_NAMES.get(st.value, str(st.value)), lat.value

    def drain(self):
        _lib.check(self._lib.hankel_server_drain(self._h), "hankel_server_drain")

    def stats(self):
        out = _lib.ServerStats()
        _lib.check(self._lib.hankel_server_get_stats(self._h, ctypes.byref(out)), "hankel_server_get_stats")
        return out.as_dict()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.hankel_server_destroy(h)
            self._h = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        self.close()
