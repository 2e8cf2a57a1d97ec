"""CPU oracle for the BP-guided beam search decoder (ctypes wrapper).

TEST INFRASTRUCTURE: only tests, the smoke check and the benchmark's CPU
baseline use this package.  The product library never imports it, and it
imports nothing from the product library.  The C source (bsd_oracle.c)
follows the paper's App. A (Eqs. 1-4), Alg. 2 (masked BP) and Alg. 3 with
App. B (beam search); its header lists the readings taken where the paper is
silent.

Two builds of the same source are exposed:
  precision="f64"  the reference arithmetic
  precision="f32"  the same algorithm in single precision, for comparing the
                   integer decisions of a single-precision implementation at
                   that implementation's precision

Problems are passed as any object with attributes M, N, K, H_row_ptr,
H_col_idx, A_row_ptr, A_col_idx and priors (float64 in (0,1)).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

STATUS_SEED = 1
STATUS_BEAM = 2
STATUS_FAILED = 4


class _Params(C.Structure):
    _fields_ = [("max_rounds", C.c_int32), ("beam_width", C.c_int32),
                ("initial_iters", C.c_int32), ("iters_per_round", C.c_int32),
                ("num_results", C.c_int32), ("prune_mode", C.c_int32),
                ("ms_scale", C.c_double), ("llr_clamp", C.c_double),
                ("msg_storage", C.c_int32), ("pad0", C.c_int32), ("tie_guard", C.c_double),
                ("weights", C.c_void_p), ("weights_iters", C.c_int32), ("pad1", C.c_int32)]


class _Trace(C.Structure):
    _fields_ = [("cap", C.c_int32), ("n", C.c_int32)] + \
        [(nm, C.POINTER(C.c_int32)) for nm in
         ("round", "canon", "parent_rank", "val", "pos", "success", "iters", "next_pos", "kept")] + \
        [("score", C.POINTER(C.c_double)),
         ("seed_iters", C.c_int32), ("seed_success", C.c_int32), ("seed_next_pos", C.c_int32),
         ("ret_round", C.c_int32), ("ret_canon", C.c_int32)]


class _DLog(C.Structure):
    _fields_ = [("cap", C.c_int32), ("n", C.c_int32)] + \
        [(nm, C.POINTER(C.c_int32)) for nm in ("call", "round", "t", "kind", "nties")] + \
        [("key", C.POINTER(C.c_uint64)), ("gap", C.POINTER(C.c_double))]


# kinds of decision-log records
LOG_ITER, LOG_ARGMIN, LOG_PRUNE, LOG_RESULT = 0, 1, 2, 3


@dataclass
class Params:
    """Beam search parameters (Alg. 3) plus the readings' constants."""
    max_rounds: int = 10
    beam_width: int = 8
    initial_iters: int = 30
    iters_per_round: int = 20
    num_results: int = 1
    ms_scale: float = 1.0
    llr_clamp: float = 1e4
    prune_mode: int = 0      # 0: bounded insert (App. B), 1: collect then prune (Alg. 3)
    msg_storage: int = 0     # float build: 0 float messages, 1 binary16, 2 bfloat16
    tie_guard: float = 0.0   # near-tie flag (status bit 8) on argmin / pruning margins in (0, tie_guard)
    weights: object = None   # optional float32 [T, E]: w_{e,t} in place of ms_scale (CSR edge order)

    def _c(self) -> _Params:
        w, T = None, 0
        if self.weights is not None:
            self._w32 = np.ascontiguousarray(self.weights, np.float32)
            if self._w32.ndim != 2:
                raise ValueError("weights must be [T, E]")
            w, T = self._w32.ctypes.data, int(self._w32.shape[0])
        return _Params(self.max_rounds, self.beam_width, self.initial_iters, self.iters_per_round,
                       self.num_results, self.prune_mode, float(self.ms_scale), float(self.llr_clamp),
                       int(self.msg_storage), 0, float(self.tie_guard), w, T, 0)


_LIBS: dict[str, C.CDLL] = {}


def _lib(precision: str) -> C.CDLL:
    if precision not in ("f64", "f32"):
        raise ValueError(precision)
    if precision in _LIBS:
        return _LIBS[precision]
    path = os.path.join(HERE, f"liboracle_{precision}.so")
    src = os.path.join(HERE, "bsd_oracle.c")
    if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(src):
        from . import build_oracle
        build_oracle.build()
    _LIBS[precision] = load_library(path, precision)
    return _LIBS[precision]


def load_library(path: str, precision: str) -> C.CDLL:
    """Load a build of bsd_oracle.c at `path` (the packaged ones, or a copy
    compiled elsewhere, e.g. by a test that checks the pins catch a planted
    mistake) and declare its entry points."""
    lib = C.CDLL(path)
    rt = C.c_double if precision == "f64" else C.c_float
    P = C.c_void_p
    lib.oracle_graph_create.restype = P
    lib.oracle_graph_create.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P]
    lib.oracle_graph_destroy.argtypes = [P]
    lib.oracle_decode.argtypes = [P, C.POINTER(_Params), P, P, P, P, P, P, C.POINTER(_Trace)]
    lib.oracle_decode_batch.argtypes = [P, C.POINTER(_Params), P, C.c_int64, P, P, P, P, P, P, C.c_int]
    lib.oracle_decode_logged.argtypes = [P, C.POINTER(_Params), P, P, P, P, P, P, C.POINTER(_DLog)]
    lib.oracle_decode_logged.restype = C.c_int
    lib.oracle_masked_bp.argtypes = [P, C.POINTER(_Params), P, P, P, P, C.c_int, C.c_int,
                                     P, P, P, P, P, P]
    lib.oracle_masked_bp.restype = C.c_int
    lib.oracle_prior_llr.argtypes = [P, P]
    lib.oracle_real_bytes.restype = C.c_int
    lib.oracle_round_storage.argtypes = [P, C.c_int, C.c_int]
    lib._real = rt
    lib._np_real = np.float64 if precision == "f64" else np.float32
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Graph:
    """The oracle's own copy of (H, A, p)."""

    def __init__(self, prob, precision: str = "f64", lib: C.CDLL | None = None):
        self.lib = lib if lib is not None else _lib(precision)
        self.precision = precision
        self.M, self.N, self.K = int(prob.M), int(prob.N), int(prob.K)
        self._keep = [np.ascontiguousarray(prob.H_row_ptr, np.int32),
                      np.ascontiguousarray(prob.H_col_idx, np.int32),
                      np.ascontiguousarray(prob.A_row_ptr, np.int32),
                      np.ascontiguousarray(prob.A_col_idx, np.int32),
                      np.ascontiguousarray(prob.priors, np.float64)]
        self.E = int(self._keep[0][-1])
        self.h = self.lib.oracle_graph_create(self.M, self.N, self.K, *[_ptr(a) for a in self._keep])
        if not self.h:
            raise RuntimeError("oracle_graph_create failed")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.oracle_graph_destroy(h)
            self.h = None

    @property
    def real(self):
        return self.lib._np_real

    def prior_llr(self) -> np.ndarray:
        out = np.zeros(self.N, self.real)
        self.lib.oracle_prior_llr(self.h, _ptr(out))
        return out

    # ---------------------------------------------------------------- decode
    def decode_batch(self, syndromes: np.ndarray, params: Params, nthreads: int = 1) -> dict:
        """Bitpacked syndromes uint32[B, ceil(M/32)] -> dict of outputs."""
        synd = np.ascontiguousarray(syndromes, np.uint32)
        B = synd.shape[0]
        WN, WK = (self.N + 31) // 32, (max(self.K, 1) + 31) // 32
        corr = np.zeros((B, WN), np.uint32)
        obs = np.zeros((B, WK), np.uint32)
        status = np.zeros(B, np.uint32)
        iters = np.zeros(B, np.uint32)
        gap = np.zeros(B, np.float64)
        ties = np.zeros(B, np.int32)
        p = params._c()
        self.lib.oracle_decode_batch(self.h, C.byref(p), _ptr(synd), B, _ptr(corr), _ptr(obs),
                                     _ptr(status), _ptr(iters), _ptr(gap), _ptr(ties), int(nthreads))
        return dict(corrections=corr, obs=obs, status=status, iters=iters, min_gap=gap, ties=ties)

    def decode_one(self, s_bits: np.ndarray, params: Params, trace_cap: int = 4096) -> dict:
        """One syndrome given as M bytes; returns ehat (N bytes), status, iters, gap, trace."""
        s = np.ascontiguousarray(s_bits, np.uint8).reshape(self.M)
        e = np.zeros(self.N, np.uint8)
        st = np.zeros(1, np.int32)
        it = np.zeros(1, np.int64)
        gap = np.zeros(1, np.float64)
        nt = np.zeros(1, np.int32)
        arrs = {nm: np.zeros(trace_cap, np.int32) for nm in
                ("round", "canon", "parent_rank", "val", "pos", "success", "iters", "next_pos", "kept")}
        score = np.zeros(trace_cap, np.float64)
        tr = _Trace()
        tr.cap = trace_cap
        for nm, a in arrs.items():
            setattr(tr, nm, a.ctypes.data_as(C.POINTER(C.c_int32)))
        tr.score = score.ctypes.data_as(C.POINTER(C.c_double))
        p = params._c()
        self.lib.oracle_decode(self.h, C.byref(p), _ptr(s), _ptr(e), _ptr(st), _ptr(it), _ptr(gap),
                               _ptr(nt), C.byref(tr))
        n = tr.n
        trace = {nm: a[:n].copy() for nm, a in arrs.items()}
        trace["score"] = score[:n].copy()
        trace.update(seed_iters=tr.seed_iters, seed_success=tr.seed_success,
                     seed_next_pos=tr.seed_next_pos, ret_round=tr.ret_round, ret_canon=tr.ret_canon)
        return dict(ehat=e, status=int(st[0]), iters=int(it[0]), min_gap=float(gap[0]), ties=int(nt[0]),
                    trace=trace)

    def decode_log(self, s_bits: np.ndarray, params: Params, cap: int = 1 << 16) -> dict:
        """One syndrome (M bytes) with its decision log: one record per BP
        iteration (kind 0: signs of the messages and of e^(t)), per next_pos
        (kind 1), per kept set of a round (kind 2) and per choice among
        results (kind 3), in the sequential algorithm's order.  Each record
        has the call (0 = seed BP, then children in visit order), round,
        iteration, a key of its outcome, its smallest nonzero relative margin
        and its number of exact ties."""
        s = np.ascontiguousarray(s_bits, np.uint8).reshape(self.M)
        e = np.zeros(self.N, np.uint8)
        st = np.zeros(1, np.int32)
        it = np.zeros(1, np.int64)
        gap = np.zeros(1, np.float64)
        nt = np.zeros(1, np.int32)
        ints = {nm: np.zeros(cap, np.int32) for nm in ("call", "round", "t", "kind", "nties")}
        key = np.zeros(cap, np.uint64)
        lg = np.zeros(cap, np.float64)
        d = _DLog()
        d.cap = cap
        for nm, a in ints.items():
            setattr(d, nm, a.ctypes.data_as(C.POINTER(C.c_int32)))
        d.key = key.ctypes.data_as(C.POINTER(C.c_uint64))
        d.gap = lg.ctypes.data_as(C.POINTER(C.c_double))
        p = params._c()
        full = self.lib.oracle_decode_logged(self.h, C.byref(p), _ptr(s), _ptr(e), _ptr(st), _ptr(it), _ptr(gap),
                                             _ptr(nt), C.byref(d))
        if full:
            raise RuntimeError("decision log capacity exceeded")
        n = d.n
        log = {nm: a[:n].copy() for nm, a in ints.items()}
        log.update(key=key[:n].copy(), gap=lg[:n].copy())
        return dict(ehat=e, status=int(st[0]), iters=int(it[0]), min_gap=float(gap[0]), ties=int(nt[0]), log=log)

    # ------------------------------------------------------------- masked BP
    def masked_bp(self, E_in, masked, val, s_bits, max_iters: int, params: Params,
                  stop_on_success: bool = True, record: bool = False) -> dict:
        """Alg. 2 from given edge messages (CSR edge order)."""
        E_in = np.ascontiguousarray(E_in, self.real).reshape(self.E)
        masked = np.ascontiguousarray(masked, np.uint8).reshape(self.N)
        val = np.ascontiguousarray(val, np.uint8).reshape(self.N)
        s = np.ascontiguousarray(s_bits, np.uint8).reshape(self.M)
        e = np.zeros(self.N, np.uint8)
        E_out = np.zeros(max(self.E, 1), self.real)
        sum_llr = np.zeros(self.N, self.real)
        traj = np.zeros((max_iters, self.N), self.real) if record else None
        succ = np.zeros(1, np.int32)
        first = np.zeros(1, np.int32)
        p = params._c()
        it = self.lib.oracle_masked_bp(self.h, C.byref(p), _ptr(E_in), _ptr(masked), _ptr(val), _ptr(s),
                                       int(max_iters), int(bool(stop_on_success)), _ptr(e), _ptr(E_out),
                                       _ptr(sum_llr), _ptr(traj) if record else None,
                                       _ptr(succ), _ptr(first))
        return dict(ehat=e, E_out=E_out[:self.E], sum_llr=sum_llr, llr=traj[:it] if record else None,
                    iters=int(it), success=bool(succ[0]), first_success=int(first[0]))

    def bp(self, s_bits, iters: int, params: Params, stop_on_success: bool = False) -> dict:
        """Plain BP (Eqs. 1-4) from E(0) = Lambda, recording Lambda_j(t) for every t."""
        lam = self.prior_llr()
        col = np.asarray(self._keep[1])
        L = params.llr_clamp
        if self.precision == "f32" and params.msg_storage:
            # E(0) as the decoder stores it: L_MAX and Lambda in the storage format
            L = float(round_storage(np.array([L], np.float32), params.msg_storage)[0])
            E0 = round_storage(np.clip(lam[col], -L, L).astype(np.float32), params.msg_storage)
            E0[E0 == 0] = 0.0
        else:
            E0 = np.clip(lam[col], -L, L).astype(self.real)
        z = np.zeros(self.N, np.uint8)
        return self.masked_bp(E0, z, z, s_bits, iters, params, stop_on_success=stop_on_success, record=True)


def round_storage(x: np.ndarray, mode: int) -> np.ndarray:
    """The float build's rounding of a float32 array to binary16 (mode 1) or bfloat16 (mode 2)."""
    a = np.ascontiguousarray(x, np.float32).copy()
    _lib("f32").oracle_round_storage(_ptr(a), int(a.size), int(mode))
    return a


STATUS_NEAR_TIE = 8


def first_divergence(log_a: dict, log_b: dict) -> int:
    """Index of the first record where two decision logs of the same shot
    differ (call, kind, iteration or outcome key), or the length of the
    shorter one when one is a prefix of the other, or -1 when they are equal."""
    n = min(len(log_a["key"]), len(log_b["key"]))
    for k in range(n):
        if (log_a["call"][k] != log_b["call"][k] or log_a["kind"][k] != log_b["kind"][k]
                or log_a["t"][k] != log_b["t"][k] or log_a["key"][k] != log_b["key"][k]):
            return k
    return -1 if len(log_a["key"]) == len(log_b["key"]) else n


def near_tie_before(log: dict, upto: int, threshold: float) -> bool:
    """Does the log hold a decision with an exact tie or a relative margin
    below threshold among its records 0..upto (inclusive)?"""
    hi = len(log["key"]) if upto < 0 else min(upto + 1, len(log["key"]))
    return bool((log["nties"][:hi] > 0).any() or (log["gap"][:hi] < threshold).any())


# Table I of the paper: (max_rounds, beam_width, initial_iters, iters_per_round, num_results)
PRESETS = {
    "beam8_230iters": (10, 8, 30, 20, 1),
    "beam32_340iters": (10, 32, 40, 30, 1),
    "beam64_640iters": (20, 64, 40, 30, 1),
    "beam64_32res_640iters": (20, 64, 40, 30, 32),
}


def preset(name: str, **kw) -> Params:
    mr, bw, ii, ipr, nr = PRESETS[name]
    return Params(max_rounds=mr, beam_width=bw, initial_iters=ii, iters_per_round=ipr, num_results=nr, **kw)
