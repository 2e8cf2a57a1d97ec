"""ctypes binding of libbsd.so: the C ABI of include/bsd.h under the same names.

Argument marshalling only; every step of decoding runs in the CUDA library.
There is no CPU fallback: if the library is missing or fails to load, the
import of this module's functions raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbsd.so")

BSD_PARAMS_VERSION = 3
BSD_OK = 0
BSD_ERR_INVALID_ARG = -1
BSD_ERR_CUDA = -2
BSD_ERR_OOM = -3
BSD_ERR_TIMEOUT = -4
BSD_ERR_UNSUPPORTED = -5
BSD_ERR_DEVICE = -6
BSD_FP32 = 0
BSD_FP16 = 1
BSD_BF16 = 2
BSD_STATUS_NEAR_TIE = 8
BSD_STATUS_FP32_RERUN = 16
BSD_STATUS_CONVERGED_SEED = 1
BSD_STATUS_CONVERGED_BEAM = 2
BSD_STATUS_FAILED = 4

# every symbol include/bsd.h declares
EXPORTS = ("bsd_params_default", "bsd_params_preset", "bsd_create", "bsd_decode", "bsd_decode_host",
           "bsd_bp_llr", "bsd_sync_error", "bsd_get_info", "bsd_get_batch", "bsd_small_layout", "bsd_generic_layout", "bsd_serve_start", "bsd_serve_decode",
           "bsd_serve_stop", "bsd_profile_enable", "bsd_profile_read",
           "bsd_decode_noalloc", "bsd_set_weights", "bsd_unrolled_workspace", "bsd_unrolled_forward",
           "bsd_unrolled_backward", "bsd_profile_read_kinds", "bsd_autotune", "bsd_get_shape", "bsd_dem_parse",
           "bsd_dem_sizes", "bsd_dem_fill", "bsd_dem_free",
           "bsd_error_string", "bsd_last_cuda_error", "bsd_destroy")
BSD_PROFILE_KINDS = 12
BSD_DEM_MERGE = 1
BSD_ERR_SCRATCH = -7


class bsd_params(C.Structure):
    _fields_ = [("struct_version", C.c_uint32), ("max_rounds", C.c_int32), ("beam_width", C.c_int32),
                ("initial_iters", C.c_int32), ("iters_per_round", C.c_int32), ("num_results", C.c_int32),
                ("ms_scale", C.c_float), ("llr_clamp", C.c_float), ("msg_precision", C.c_int32),
                ("tie_guard_rel", C.c_float), ("workspace_bytes", C.c_int64), ("group_warps", C.c_int32),
                ("small_batch", C.c_int32), ("batch_slots", C.c_int32)]


class bsd_shape_timing(C.Structure):
    _fields_ = [("group_warps", C.c_int32), ("warps_per_block", C.c_int32), ("ms", C.c_float)]


class BsdError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        detail = bsd_last_cuda_error() if code == BSD_ERR_CUDA else ""
        super().__init__(f"{what}: {bsd_error_string(code)} ({code})" + (f" [{detail}]" if detail else ""))


_lib = None


def load(path: str | None = None) -> C.CDLL:
    """Load libbsd.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        from . import _build
        path = _build.build()
    if not os.path.exists(path):
        raise OSError(f"CUDA library not found: {path}")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.bsd_params_default.argtypes = [C.POINTER(bsd_params)]
    lib.bsd_params_preset.argtypes = [C.c_char_p, C.POINTER(bsd_params)]
    lib.bsd_create.argtypes = [C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P, C.POINTER(bsd_params), C.c_int,
                               C.POINTER(P)]
    lib.bsd_decode.argtypes = [P, P, C.c_int64, P, P, P, P, P]
    lib.bsd_decode_host.argtypes = [P, P, C.c_int64, P, P, P, P, P]
    lib.bsd_serve_start.argtypes = [P, C.c_int32]
    lib.bsd_serve_decode.argtypes = [P, P, P, P, P, P]
    lib.bsd_serve_stop.argtypes = [P]
    lib.bsd_bp_llr.argtypes = [P, P, C.c_int64, C.c_int32, P, P, P]
    lib.bsd_sync_error.argtypes = [P]
    lib.bsd_get_info.argtypes = [P] + [C.POINTER(C.c_int32)] * 4 + [C.POINTER(C.c_int64)] * 2
    lib.bsd_get_batch.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.bsd_small_layout.argtypes = [C.c_int32, C.c_int32, P, P, P, P, P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.bsd_generic_layout.argtypes = [C.c_int32, C.c_int32, P, P, P, P, C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32)]
    lib.bsd_decode_noalloc.argtypes = [P, P, C.c_int64, P, P, P, P, P]
    lib.bsd_profile_enable.argtypes = [P, C.c_int]
    lib.bsd_set_weights.argtypes = [P, P, C.c_int32]
    lib.bsd_unrolled_workspace.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, C.POINTER(C.c_int64)]
    lib.bsd_unrolled_forward.argtypes = [P, P, P, C.c_int64, C.c_int32, C.c_int32, P, P, P, P, C.c_int64, P]
    lib.bsd_unrolled_backward.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, P, P, P, P, C.c_int64, P]
    lib.bsd_profile_read.argtypes = [P, P, P, P, P, P]
    lib.bsd_profile_read_kinds.argtypes = [P, P, P]
    lib.bsd_autotune.argtypes = [P, P, C.c_int64, P, P, C.c_int32, C.POINTER(C.c_int32)]
    lib.bsd_get_shape.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.bsd_dem_parse.argtypes = [C.c_char_p, C.c_int64, C.c_int32, C.POINTER(P), C.POINTER(C.c_int64)]
    lib.bsd_dem_sizes.argtypes = [P] + [C.POINTER(C.c_int32)] * 3 + [C.POINTER(C.c_int64)] * 2
    lib.bsd_dem_fill.argtypes = [P, P, P, P, P, P]
    lib.bsd_dem_free.argtypes = [P]
    lib.bsd_dem_free.restype = None
    lib.bsd_error_string.argtypes = [C.c_int]
    lib.bsd_error_string.restype = C.c_char_p
    lib.bsd_last_cuda_error.argtypes = []
    lib.bsd_last_cuda_error.restype = C.c_char_p
    lib.bsd_destroy.argtypes = [P]
    lib.bsd_destroy.restype = None
    for nm in EXPORTS:
        if nm not in ("bsd_error_string", "bsd_last_cuda_error", "bsd_destroy", "bsd_dem_free"):
            getattr(lib, nm).restype = C.c_int
    _lib = lib
    return lib


def check(code: int, what: str) -> None:
    if code != BSD_OK:
        raise BsdError(code, what)


# ---- the C ABI, same names ---------------------------------------------------
def bsd_error_string(code: int) -> str:
    return load().bsd_error_string(int(code)).decode()


def bsd_last_cuda_error() -> str:
    return load().bsd_last_cuda_error().decode()


def bsd_params_default() -> bsd_params:
    p = bsd_params()
    check(load().bsd_params_default(C.byref(p)), "bsd_params_default")
    return p


def bsd_params_preset(name: str) -> bsd_params:
    p = bsd_params()
    check(load().bsd_params_preset(name.encode(), C.byref(p)), f"bsd_params_preset({name})")
    return p


def bsd_create(M, N, K, H_row_ptr, H_col_idx, A_row_ptr, A_col_idx, priors, params: bsd_params,
               device: int = 0) -> int:
    """Pointers are host addresses (ints) of int32 / float64 arrays."""
    h = C.c_void_p()
    check(load().bsd_create(int(M), int(N), int(K), H_row_ptr, H_col_idx, A_row_ptr, A_col_idx, priors,
                            C.byref(params), int(device), C.byref(h)), "bsd_create")
    return h.value


def bsd_decode(dec, d_syndromes, B, d_corrections, d_obs_flips, d_status, d_iters, stream) -> None:
    check(load().bsd_decode(dec, d_syndromes, int(B), d_corrections, d_obs_flips, d_status, d_iters, stream),
          "bsd_decode")


def bsd_decode_noalloc(dec, d_syndromes, B, d_corrections, d_obs_flips, d_status, d_iters, stream) -> int:
    """Allocation-free decode; returns the code (BSD_ERR_SCRATCH is an expected outcome)."""
    return int(load().bsd_decode_noalloc(dec, d_syndromes, int(B), d_corrections, d_obs_flips, d_status,
                                         d_iters, stream))


def bsd_decode_host(dec, h_syndromes, B, h_corrections, h_obs_flips, h_status, h_iters, stream) -> None:
    check(load().bsd_decode_host(dec, h_syndromes, int(B), h_corrections, h_obs_flips, h_status, h_iters, stream),
          "bsd_decode_host")


def bsd_serve_start(dec, idle_ms: int) -> None:
    check(load().bsd_serve_start(dec, int(idle_ms)), "bsd_serve_start")


def bsd_serve_decode(dec, h_syndrome, h_correction, h_obs_flips, h_status, h_iters) -> None:
    """One syndrome through the request loop; host addresses as bsd_decode_host with B = 1."""
    check(load().bsd_serve_decode(dec, h_syndrome, h_correction, h_obs_flips, h_status, h_iters), "bsd_serve_decode")


def bsd_serve_stop(dec) -> None:
    check(load().bsd_serve_stop(dec), "bsd_serve_stop")


def bsd_bp_llr(dec, d_syndromes, B, T, d_llr, d_sum_llr, stream) -> None:
    check(load().bsd_bp_llr(dec, d_syndromes, int(B), int(T), d_llr, d_sum_llr, stream), "bsd_bp_llr")


def bsd_sync_error(dec) -> int:
    return int(load().bsd_sync_error(dec))


def bsd_get_info(dec) -> dict:
    M, N, K, E = (C.c_int32() for _ in range(4))
    cs, wb = C.c_int64(), C.c_int64()
    check(load().bsd_get_info(dec, C.byref(M), C.byref(N), C.byref(K), C.byref(E), C.byref(cs), C.byref(wb)),
          "bsd_get_info")
    return dict(M=M.value, N=N.value, K=K.value, n_edges=E.value, chunk_shots=cs.value, workspace_bytes=wb.value)


def bsd_get_batch(dec) -> dict:
    """Slots of the decoder's batched seed BP (0: none) and whether its launch shape uses them."""
    sl, ac = C.c_int32(), C.c_int32()
    check(load().bsd_get_batch(dec, C.byref(sl), C.byref(ac)), "bsd_get_batch")
    return dict(slots=sl.value, active=bool(ac.value))


def bsd_small_layout(M: int, N: int, row_ptr, col_idx) -> dict:
    """The single-warp engine's shared-memory placement of H's messages (host
    only): plane bases, the word of every CSR edge, the word of the k-th edge
    of every column ([N][3]), the words spanned and the bank loads above three
    left in the error-node pass."""
    import numpy as np
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    plane = np.zeros(3, np.int32)
    ew = np.zeros(int(rp[-1]), np.int32)
    cw = np.zeros(3 * int(N), np.int32)
    ext, exc = C.c_int32(), C.c_int32()
    check(load().bsd_small_layout(int(M), int(N), rp.ctypes.data, ci.ctypes.data, plane.ctypes.data, ew.ctypes.data,
                                  cw.ctypes.data, C.byref(ext), C.byref(exc)), "bsd_small_layout")
    return dict(plane=plane, edge_word=ew, col_word=cw.reshape(int(N), 3), extent=ext.value, excess=exc.value)


def bsd_generic_layout(M: int, N: int, row_ptr, col_idx) -> dict:
    """The generic engines' placement of H's messages (host only): the
    element of every CSR edge, the CSR edge in every (k, column) slot
    ([colK][N], -1 empty), colK and the bank loads above the groups' largest
    degrees left by the search."""
    import numpy as np
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    ew = np.zeros(int(rp[-1]), np.int32)
    se = np.zeros(6 * int(N), np.int32)
    ck, exc = C.c_int32(), C.c_int32()
    check(load().bsd_generic_layout(int(M), int(N), rp.ctypes.data, ci.ctypes.data, ew.ctypes.data, se.ctypes.data,
                                    C.byref(ck), C.byref(exc)), "bsd_generic_layout")
    return dict(edge_word=ew, slot_edge=se[:ck.value * int(N)].reshape(ck.value, int(N)), colK=ck.value,
                excess=exc.value)


def bsd_set_weights(dec, h_weights, T: int) -> None:
    """h_weights: host address of float32 [T][E] (CSR edge order), or None with T = 0."""
    check(load().bsd_set_weights(dec, h_weights, int(T)), "bsd_set_weights")


def bsd_unrolled_workspace(dec, B: int, T: int, ckpt_every: int) -> int:
    n = C.c_int64()
    check(load().bsd_unrolled_workspace(dec, int(B), int(T), int(ckpt_every), C.byref(n)), "bsd_unrolled_workspace")
    return n.value


def bsd_unrolled_forward(dec, d_syndromes, d_errors, B, T, ckpt_every, d_weights, d_loss, d_llr, d_work,
                         work_bytes, stream) -> None:
    check(load().bsd_unrolled_forward(dec, d_syndromes, d_errors, int(B), int(T), int(ckpt_every), d_weights,
                                      d_loss, d_llr, d_work, int(work_bytes), stream), "bsd_unrolled_forward")


def bsd_unrolled_backward(dec, B, T, ckpt_every, d_weights, d_grad_loss, d_grad_weights, d_work, work_bytes,
                          stream) -> None:
    check(load().bsd_unrolled_backward(dec, int(B), int(T), int(ckpt_every), d_weights, d_grad_loss,
                                       d_grad_weights, d_work, int(work_bytes), stream), "bsd_unrolled_backward")


def bsd_profile_enable(dec, enable: bool) -> None:
    check(load().bsd_profile_enable(dec, int(bool(enable))), "bsd_profile_enable")


def bsd_profile_read(dec) -> dict:
    """Kernel times (ms) and launches per kind (seed, round, select), executed full iterations,
    kernel launches, message updates of first-iteration screens."""
    import numpy as np
    ms = np.zeros(3, np.float64)
    ln = np.zeros(3, np.int64)
    it = np.zeros(3, np.uint64)
    kl = np.zeros(1, np.uint64)
    su = np.zeros(1, np.uint64)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    check(load().bsd_profile_read(dec, p(ms), p(ln), p(it), p(kl), p(su)), "bsd_profile_read")
    return dict(ms=ms, launches=ln, exec_iters=it, kernel_launches=int(kl[0]), screen_updates=int(su[0]))


def bsd_profile_read_kinds(dec) -> dict:
    """Event-timed ms and launches of every kernel kind (0 seed, 1 round, 2 select,
    3..6 unrolled check / error / error adjoint / check adjoint, 7 other unrolled,
    8..10 batched seed check / error / retirement, 11 first-iteration screen)."""
    import numpy as np
    ms = np.zeros(BSD_PROFILE_KINDS, np.float64)
    ln = np.zeros(BSD_PROFILE_KINDS, np.int64)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    check(load().bsd_profile_read_kinds(dec, p(ms), p(ln)), "bsd_profile_read_kinds")
    return dict(ms=ms, launches=ln)


def bsd_autotune(dec, d_syndromes, B: int, stream) -> list:
    """Time every launch shape on the sample and keep the fastest; returns [(group_warps, warps_per_block, ms)]."""
    cap = 16
    rep = (bsd_shape_timing * cap)()
    n = C.c_int32()
    check(load().bsd_autotune(dec, d_syndromes, int(B), stream, rep, cap, C.byref(n)), "bsd_autotune")
    return [(rep[k].group_warps, rep[k].warps_per_block, float(rep[k].ms)) for k in range(min(n.value, cap))]


def bsd_get_shape(dec) -> tuple:
    gw, wpb = C.c_int32(), C.c_int32()
    check(load().bsd_get_shape(dec, C.byref(gw), C.byref(wpb)), "bsd_get_shape")
    return gw.value, wpb.value


def bsd_dem_read(text: str, merge: bool = False) -> dict:
    """bsd_dem_parse + bsd_dem_sizes + bsd_dem_fill + bsd_dem_free: a text detector
    error model -> dict(M, N, K, H_row_ptr, H_col_idx, A_row_ptr, A_col_idx, priors)."""
    import numpy as np
    lib = load()
    raw = text.encode()
    h = C.c_void_p()
    line = C.c_int64()
    rc = lib.bsd_dem_parse(raw, len(raw), BSD_DEM_MERGE if merge else 0, C.byref(h), C.byref(line))
    if rc != BSD_OK:
        raise BsdError(rc, f"bsd_dem_parse (line {line.value})")
    try:
        M, N, K = C.c_int32(), C.c_int32(), C.c_int32()
        nh, na = C.c_int64(), C.c_int64()
        check(lib.bsd_dem_sizes(h, C.byref(M), C.byref(N), C.byref(K), C.byref(nh), C.byref(na)), "bsd_dem_sizes")
        out = dict(M=M.value, N=N.value, K=K.value,
                   H_row_ptr=np.zeros(M.value + 1, np.int32), H_col_idx=np.zeros(max(nh.value, 1), np.int32),
                   A_row_ptr=np.zeros(K.value + 1, np.int32), A_col_idx=np.zeros(max(na.value, 1), np.int32),
                   priors=np.zeros(max(N.value, 1), np.float64))
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        check(lib.bsd_dem_fill(h, p(out["H_row_ptr"]), p(out["H_col_idx"]), p(out["A_row_ptr"]),
                               p(out["A_col_idx"]), p(out["priors"])), "bsd_dem_fill")
        out["H_col_idx"] = out["H_col_idx"][:nh.value]
        out["A_col_idx"] = out["A_col_idx"][:na.value]
        out["priors"] = out["priors"][:N.value]
        return out
    finally:
        lib.bsd_dem_free(h)


def bsd_destroy(dec) -> None:
    if dec:
        load().bsd_destroy(dec)
