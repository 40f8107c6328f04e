"""ctypes declarations of the C ABI in include/hankel.h (argument marshalling only)."""
import ctypes
import os

from . import build as _build

_lib = None

HANKEL_OK = 0
STATUS_NAMES = {0: "HANKEL_OK", 1: "HANKEL_EINVAL", 2: "HANKEL_ENOMEM", 3: "HANKEL_ECUDA",
                4: "HANKEL_EUNSUPPORTED", 5: "HANKEL_ETIMEOUT", 6: "HANKEL_ECANCELED"}
FLAG_HOST_ONLY = 1
FLAG_NO_SEGMENT = 2
FLAG_ALL_COLUMNS = 8
FLAG_NO_REFINE = 16
FLAG_NO_LOWRANK = 32
FLAG_UNIFORM_TERMS = 64
FLAG_NO_AUTOTUNE = 128
FLAG_TENSOR_FFT = 256

# Every function include/hankel.h declares.
EXPORTED = [
    "hankel_options_default", "hankel_plan", "hankel_plan_ex", "hankel_exec", "hankel_exec_batched",
    "hankel_exec_host", "hankel_plan_info", "hankel_plan_blocks", "hankel_plan_entry", "hankel_plan_expansion_entry",
    "hankel_exec_inverse", "hankel_dht_inverse_weights",
    "hankel_plan_near_prefix", "hankel_destroy", "hankel_status_string", "hankel_s_nu_M",
    "hankel_t_nu_T", "hankel_neumann_radius", "hankel_p_K", "hankel_q_T", "hankel_params",
    "hankel_j0_zero_offsets", "hankel_plan_set_timing", "hankel_plan_stage_stats", "hankel_exec_static",
    "hankel_server_options_default", "hankel_server_create", "hankel_server_submit", "hankel_server_wait",
    "hankel_server_drain", "hankel_server_get_stats", "hankel_server_destroy",
    "hankel_plan_fft_shapes", "hankel_tune_cache_put", "hankel_tune_cache_get", "hankel_tune_cache_save",
    "hankel_tune_cache_load", "hankel_tune_cache_clear", "hankel_tune_bucket", "hankel_plan_add_context",
    "hankel_exec_batched_ctx", "hankel_server_cancel", "hankel_debug_fail_allocs", "hankel_plan_device_status",
    "hankel_debug_fft_compare",
]
STAGES = ["near", "gen", "fft", "pointwise", "out", "fft_df64", "fft_fp32"]


class Options(ctypes.Structure):
    _fields_ = [("task", ctypes.c_int), ("nu", ctypes.c_int), ("N", ctypes.c_int64), ("eps", ctypes.c_double),
                ("grid", ctypes.c_int), ("gamma", ctypes.c_int64), ("precision", ctypes.c_int),
                ("max_nrhs", ctypes.c_int), ("flags", ctypes.c_uint), ("workspace_limit", ctypes.c_size_t)]


class Info(ctypes.Structure):
    _fields_ = [("task", ctypes.c_int), ("nu", ctypes.c_int), ("grid", ctypes.c_int), ("precision", ctypes.c_int),
                ("N", ctypes.c_int64), ("gamma", ctypes.c_int64), ("eps", ctypes.c_double), ("M", ctypes.c_int),
                ("mu_max", ctypes.c_int), ("s", ctypes.c_double), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("P", ctypes.c_int), ("K", ctypes.c_int), ("T", ctypes.c_int),
                ("K2", ctypes.c_int), ("T2", ctypes.c_int), ("direct_rows", ctypes.c_int64),
                ("direct_cols", ctypes.c_int64), ("nblocks", ctypes.c_int), ("ncols", ctypes.c_int),
                ("npairs", ctypes.c_int), ("near_count", ctypes.c_int64), ("far_count", ctypes.c_int64),
                ("near_zmax", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("workspace_bytes", ctypes.c_size_t), ("block_cols", ctypes.c_int64), ("fft_shapes", ctypes.c_int),
                ("contexts", ctypes.c_int), ("context_bytes", ctypes.c_size_t)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class FftShape(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("log2_len", ctypes.c_int), ("col_bucket", ctypes.c_int),
                ("one_launch", ctypes.c_int), ("npass", ctypes.c_int), ("log2_radix", ctypes.c_int * 4),
                ("tensor_passes", ctypes.c_int), ("ms_default", ctypes.c_double), ("ms_chosen", ctypes.c_double)]

    def as_dict(self):
        return {"precision": self.precision, "log2_len": self.log2_len, "col_bucket": self.col_bucket,
                "one_launch": bool(self.one_launch),
                "radices": [] if self.one_launch else list(self.log2_radix[:self.npass]),
                "tensor_passes": [] if self.one_launch else [bool((self.tensor_passes >> i) & 1)
                                                             for i in range(self.npass)],
                "ms_default": self.ms_default, "ms_chosen": self.ms_chosen}


class StageStat(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("flops", ctypes.c_double), ("entries", ctypes.c_double),
                ("bytes", ctypes.c_double), ("launches", ctypes.c_int64)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("memory_cap", ctypes.c_size_t), ("streams", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("precision", ctypes.c_int), ("pack_requests", ctypes.c_int),
                ("batch_window_us", ctypes.c_int), ("contexts_per_plan", ctypes.c_int),
                ("small_batch", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("vectors", ctypes.c_int64), ("coefficients", ctypes.c_double),
                ("plans_built", ctypes.c_int64), ("plans_evicted", ctypes.c_int64),
                ("graphs_captured", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
                ("contexts_added", ctypes.c_int64), ("cancelled", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Block(ctypes.Structure):
    _fields_ = [("k0", ctypes.c_int64), ("k1", ctypes.c_int64), ("n0", ctypes.c_int64), ("n1", ctypes.c_int64),
                ("fft_len", ctypes.c_int64), ("seg_len", ctypes.c_int64), ("nseg", ctypes.c_int64),
                ("mode", ctypes.c_int), ("ncols", ctypes.c_int), ("dropped", ctypes.c_double),
                ("kept", ctypes.c_int), ("lowrank", ctypes.c_int), ("lowrank_err", ctypes.c_double),
                ("terms_fp64", ctypes.c_int), ("terms_df64", ctypes.c_int), ("terms_fp32", ctypes.c_int)]


def load():
    """Load (building first if needed) libhankel.so. Raises if it cannot be built or loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = ctypes.CDLL(path)
    i32, i64, dbl, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    pplan = ctypes.POINTER(ctypes.c_void_p)
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "hankel_options_default": (i32, [ctypes.POINTER(Options), i32, i32, i64, dbl]),
        "hankel_plan": (i32, [pplan, i32, i32, i64, dbl]),
        "hankel_plan_ex": (i32, [pplan, ctypes.POINTER(Options)]),
        "hankel_exec": (i32, [vp, vp, vp, vp]),
        "hankel_exec_batched": (i32, [vp, vp, i64, vp, i64, i32, vp]),
        "hankel_exec_host": (i32, [vp, dp, i64, dp, i64, i32]),
        "hankel_plan_info": (i32, [vp, ctypes.POINTER(Info)]),
        "hankel_plan_blocks": (i32, [vp, ctypes.POINTER(Block), i32, ctypes.POINTER(i32)]),
        "hankel_plan_entry": (i32, [vp, i64, i64, dp, ctypes.POINTER(i32)]),
        "hankel_plan_expansion_entry": (i32, [vp, i64, i64, dp]),
        "hankel_exec_inverse": (i32, [vp, vp, i64, vp, i64, i32, vp]),
        "hankel_dht_inverse_weights": (i32, [i64, dp]),
        "hankel_plan_near_prefix": (i32, [vp, i64, ctypes.POINTER(i64)]),
        "hankel_destroy": (i32, [vp]),
        "hankel_status_string": (ctypes.c_char_p, [i32]),
        "hankel_s_nu_M": (dbl, [i32, i32, dbl]),
        "hankel_t_nu_T": (dbl, [i32, i32, dbl]),
        "hankel_neumann_radius": (dbl, [i32, dbl]),
        "hankel_p_K": (dbl, [i32, dbl]),
        "hankel_q_T": (dbl, [i32, dbl]),
        "hankel_params": (i32, [ctypes.POINTER(Options), ctypes.POINTER(Info)]),
        "hankel_j0_zero_offsets": (i32, [i64, dp]),
        "hankel_plan_set_timing": (i32, [vp, i32]),
        "hankel_exec_static": (i32, [vp, vp, vp, vp]),
        "hankel_server_options_default": (i32, [ctypes.POINTER(ServerOptions)]),
        "hankel_server_create": (i32, [pplan, ctypes.POINTER(ServerOptions)]),
        "hankel_server_submit": (i32, [vp, i32, i32, i64, dbl, dp, dp, i32, ctypes.POINTER(i64)]),
        "hankel_server_wait": (i32, [vp, i64, ctypes.POINTER(i32), ctypes.POINTER(dbl)]),
        "hankel_server_drain": (i32, [vp]),
        "hankel_server_get_stats": (i32, [vp, ctypes.POINTER(ServerStats)]),
        "hankel_server_destroy": (i32, [vp]),
        "hankel_plan_stage_stats": (i32, [vp, ctypes.POINTER(StageStat)]),
        "hankel_plan_fft_shapes": (i32, [vp, ctypes.POINTER(FftShape), i32, ctypes.POINTER(i32)]),
        "hankel_tune_cache_put": (i32, [ctypes.c_char_p, ctypes.POINTER(FftShape)]),
        "hankel_tune_cache_get": (i32, [ctypes.c_char_p, i32, i32, i32, ctypes.POINTER(FftShape),
                                        ctypes.POINTER(i32)]),
        "hankel_tune_cache_save": (i32, [ctypes.c_char_p]),
        "hankel_tune_cache_load": (i32, [ctypes.c_char_p]),
        "hankel_tune_cache_clear": (i32, []),
        "hankel_tune_bucket": (i32, [i64]),
        "hankel_plan_add_context": (i32, [vp, ctypes.POINTER(i32)]),
        "hankel_exec_batched_ctx": (i32, [vp, i32, vp, i64, vp, i64, i32, vp]),
        "hankel_server_cancel": (i32, [vp, i64, ctypes.POINTER(i32)]),
        "hankel_debug_fail_allocs": (i32, [i64, i64]),
        "hankel_plan_device_status": (i32, [vp]),
        "hankel_debug_fft_compare": (i32, [i32, i32, i32, i32, ctypes.POINTER(i32), i32, dp, dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def library_path():
    return _build.LIB_PATH


def check(status, what):
    if status != HANKEL_OK:
        msg = load().hankel_status_string(status).decode()
        raise RuntimeError("%s failed: %s (%s)" % (what, STATUS_NAMES.get(status, status), msg))


def loaded_path():
    """Path of the shared object this process loaded (None before load())."""
    return os.path.realpath(_build.LIB_PATH) if _lib is not None else None
