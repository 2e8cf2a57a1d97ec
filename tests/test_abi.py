"""The C ABI library: builds, loads, exports every declared symbol, and its
host-only logic (presets, argument validation) works without a GPU."""
import ctypes as C
import json
import os
import re

import numpy as np
import pytest

from paper_2512_07057_gb300 import binding as B
from paper_2512_07057_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "bsd.h")).read()
    return sorted(set(re.findall(r"\b(bsd_[a-z_]+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert sorted(B.EXPORTS) == _declared_symbols()


def test_library_exports_every_declared_symbol():
    lib = B.load()
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_presets_match_table1_golden():
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "table1_presets.json")))
    for name, (mr, bw, ii, ipr, nr) in g["presets"].items():
        p = B.bsd_params_preset(name)
        assert (p.max_rounds, p.beam_width, p.initial_iters, p.iters_per_round, p.num_results) == (mr, bw, ii, ipr, nr)
        assert p.struct_version == B.BSD_PARAMS_VERSION and p.msg_precision == B.BSD_FP32
    with pytest.raises(B.BsdError):
        B.bsd_params_preset("beam7_unknown")


def test_error_strings():
    for code in (0, -1, -2, -3, -4, -5, -6, -99):
        assert isinstance(B.bsd_error_string(code), str)


def _create(prob, params, priors=None, row_ptr=None, col_idx=None):
    hr = np.ascontiguousarray(prob.H_row_ptr if row_ptr is None else row_ptr, np.int32)
    hc = np.ascontiguousarray(prob.H_col_idx if col_idx is None else col_idx, np.int32)
    ar = np.ascontiguousarray(prob.A_row_ptr, np.int32)
    ac = np.ascontiguousarray(prob.A_col_idx, np.int32)
    pr = np.ascontiguousarray(prob.priors if priors is None else priors, np.float64)
    h = C.c_void_p()
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)
    rc = B.load().bsd_create(prob.M, prob.N, prob.K, ptr(hr), ptr(hc), ptr(ar), ptr(ac), ptr(pr),
                             C.byref(params), 0, C.byref(h))
    if rc == 0:
        B.bsd_destroy(h.value)
    return rc


def test_create_rejects_invalid_input_before_touching_the_device():
    prob = W.bb72_code_capacity(0.03)
    good = B.bsd_params_default()
    bad_p = prob.priors.copy()
    bad_p[3] = 1.0
    assert _create(prob, good, priors=bad_p) == B.BSD_ERR_INVALID_ARG
    bad_p[3] = 0.0
    assert _create(prob, good, priors=bad_p) == B.BSD_ERR_INVALID_ARG
    bad_c = prob.H_col_idx.copy()
    bad_c[5] = prob.N
    assert _create(prob, good, col_idx=bad_c) == B.BSD_ERR_INVALID_ARG
    unsorted = prob.H_col_idx.copy()
    unsorted[0], unsorted[1] = unsorted[1], unsorted[0]
    assert _create(prob, good, col_idx=unsorted) == B.BSD_ERR_INVALID_ARG
    for field, val in (("beam_width", 0), ("beam_width", 65), ("num_results", 0), ("initial_iters", 0),
                       ("iters_per_round", 0), ("max_rounds", -1), ("ms_scale", 0.0), ("llr_clamp", -1.0),
                       ("struct_version", 7)):
        p = B.bsd_params_default()
        setattr(p, field, val)
        assert _create(prob, p) == B.BSD_ERR_INVALID_ARG, field
    p = B.bsd_params_default()
    p.msg_precision = 3
    assert _create(prob, p) == B.BSD_ERR_UNSUPPORTED
    lib = B.load()
    assert lib.bsd_decode(None, None, 1, None, None, None, None, None) == B.BSD_ERR_INVALID_ARG
    assert lib.bsd_sync_error(None) == B.BSD_ERR_INVALID_ARG


def _unbound_decoder(M=72, N=144, K=12, device=0):
    """A BeamSearchDecoder shell with sizes but no handle: its checks run on
    the host, so a rejection here happens before any library call."""
    from paper_2512_07057_gb300 import decoder as D

    class _NoCall:
        def __getattr__(self, name):
            raise AssertionError(f"the library was called ({name}) despite a bad tensor")

    dec = D.BeamSearchDecoder.__new__(D.BeamSearchDecoder)
    dec.M, dec.N, dec.K, dec.device, dec.h = M, N, K, device, None
    return dec, _NoCall()


def _good_io(torch, nb=5, M=72, N=144, K=12):
    from paper_2512_07057_gb300 import decoder as D
    w = lambda n: (n + 31) // 32
    synd = torch.zeros((nb, w(M)), dtype=torch.int32)
    out = D.DecodeResult(corrections=torch.zeros((nb, w(N)), dtype=torch.int32),
                         obs_flips=torch.zeros((nb, max(w(K), 1)), dtype=torch.int32),
                         status=torch.zeros(nb, dtype=torch.int32), iters=torch.zeros(nb, dtype=torch.int32))
    return synd, out


@pytest.mark.parametrize("bad", ["synd_words", "synd_1d", "corr_rows", "corr_words", "obs_words", "status_rows",
                                 "iters_rows", "corr_dtype", "status_float", "corr_noncontig", "host_tensors"])
@pytest.mark.parametrize("call", ["decode", "decode_noalloc"])
def test_decoder_rejects_mis_sized_tensors_before_any_launch(bad, call, monkeypatch):
    torch = pytest.importorskip("torch")
    from paper_2512_07057_gb300 import decoder as D
    dec, trap = _unbound_decoder()
    monkeypatch.setattr(D, "B", trap)
    synd, out = _good_io(torch)
    if bad == "synd_words":
        synd = torch.zeros((5, 2), dtype=torch.int32)
    elif bad == "synd_1d":
        synd = torch.zeros(15, dtype=torch.int32)
    elif bad == "corr_rows":
        out.corrections = torch.zeros((4, 5), dtype=torch.int32)
    elif bad == "corr_words":
        out.corrections = torch.zeros((5, 4), dtype=torch.int32)
    elif bad == "obs_words":
        out.obs_flips = torch.zeros((5, 0), dtype=torch.int32)
    elif bad == "status_rows":
        out.status = torch.zeros(4, dtype=torch.int32)
    elif bad == "iters_rows":
        out.iters = torch.zeros(6, dtype=torch.int32)
    elif bad == "corr_dtype":
        out.corrections = torch.zeros((5, 5), dtype=torch.int64)
    elif bad == "status_float":
        out.status = torch.zeros(5, dtype=torch.float32)
    elif bad == "corr_noncontig":
        out.corrections = torch.zeros((5, 10), dtype=torch.int32)[:, ::2]
    # "host_tensors": every size is right, but nothing is on the decoder's device
    with pytest.raises(ValueError):
        if call == "decode":
            dec.decode(synd, out)
        else:
            dec.decode_noalloc(synd, out)


def test_request_loop_entry_points_reject_null_arguments():
    """bsd_serve_*: argument checks come before any device work."""
    lib = B.load()
    assert lib.bsd_serve_start(None, 100) == B.BSD_ERR_INVALID_ARG
    assert lib.bsd_serve_decode(None, None, None, None, None, None) == B.BSD_ERR_INVALID_ARG
    assert lib.bsd_serve_stop(None) == B.BSD_ERR_INVALID_ARG
