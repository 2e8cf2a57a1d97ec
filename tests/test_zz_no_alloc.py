"""bsd_decode_noalloc: decoding with no device allocation in the call.

Some callers cannot allocate device memory when they decode (their memory
belongs to another allocator, or they run a loop that must not take the
driver's allocation locks).  bsd_decode_noalloc serves them from a static
device array instead of the decoder's own workspace.  These tests call it
through the C ABI and check that it returns exactly what bsd_decode
returns, on two calls in a row (the array keeps the previous call's
contents, so the second call checks that each call clears what it must).
This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2512_07057_gb300 import binding as B  # noqa: E402
from paper_2512_07057_gb300 import decoder as D  # noqa: E402
from paper_2512_07057_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _arrays(out):
    return {k: D.from_torch_words(getattr(out, k)).copy() for k in ("corrections", "obs_flips", "status", "iters")}


@pytest.mark.parametrize("case", ["bb144_beam32", "bb72_32res", "phenom_screen"])
def test_noalloc_matches_decode_on_two_calls(case):
    if case == "bb144_beam32":
        prob = W.bb144_code_capacity(0.05)
        params = D.make_params("beam32_340iters", ms_scale=0.625)
        shots = W.sample_shots(prob, 3_000, "noalloc_bb144")
    elif case == "phenom_screen":
        # a generic-engine DEM: the first-iteration screen and its queue run
        # in the static array too, over several chunks
        prob = W.bb_phenomenological(6, 6, 4, 0.01, 0.01)
        params = D.make_params(max_rounds=4, beam_width=8, initial_iters=20, iters_per_round=10, ms_scale=0.625)
        shots = W.sample_shots(prob, 4_000, "noalloc_phenom")
    else:
        prob = W.bb72_code_capacity(0.05)
        params = D.make_params("beam64_32res_640iters", ms_scale=0.625)
        shots = W.sample_shots(prob, 1_000, "noalloc_bb72")
    dec = D.BeamSearchDecoder(prob, params)
    synd = D.to_torch_words(shots.syndromes)
    ref = _arrays(dec.decode(synd))
    torch.cuda.synchronize()
    for call in range(2):
        out = dec.alloc_outputs(shots.B)
        for t in (out.corrections, out.obs_flips, out.status, out.iters):
            t.fill_(-1)
        rc = dec.decode_noalloc(synd, out)
        assert rc == B.BSD_OK, B.bsd_error_string(rc)
        torch.cuda.synchronize()
        got = _arrays(out)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), f"call {call}: {k} differs"
    assert (ref["status"] == 2).sum() > 0          # beam rounds ran, so the scratch was used
    dec.close()


def test_noalloc_rejects_a_shot_larger_than_the_scratch():
    """A 936 x 8800 detector error model at beam width 64 needs two banks of
    128 snapshots of ~35k messages per shot, more than the static array."""
    prob = W.synthetic_dem()
    params = D.make_params("beam64_640iters", ms_scale=0.625, workspace_bytes=1 << 30)
    dec = D.BeamSearchDecoder(prob, params)
    synd = torch.zeros((4, (prob.M + 31) // 32), dtype=torch.int32, device="cuda")
    out = dec.alloc_outputs(4)
    assert dec.decode_noalloc(synd, out) == B.BSD_ERR_SCRATCH
    assert "scratch" in B.bsd_error_string(B.BSD_ERR_SCRATCH)
    dec.close()


def test_noalloc_16bit_messages():
    """16-bit message storage: a decoder that re-runs near-tie shots in single
    precision needs a second decoder's buffers, so the allocation-free call
    refuses it; with the re-runs switched off it returns what bsd_decode
    returns, on two calls in a row."""
    prob = W.bb144_code_capacity(0.05)
    shots = W.sample_shots(prob, 2_000, "noalloc_fp16")
    synd = D.to_torch_words(shots.syndromes)
    with_reruns = D.BeamSearchDecoder(prob, D.make_params("beam32_340iters", ms_scale=0.625,
                                                          msg_precision=B.BSD_FP16, tie_guard_rel=1e-3))
    out = with_reruns.alloc_outputs(shots.B)
    assert with_reruns.decode_noalloc(synd, out) == B.BSD_ERR_UNSUPPORTED
    with_reruns.close()
    dec = D.BeamSearchDecoder(prob, D.make_params("beam32_340iters", ms_scale=0.625,
                                                  msg_precision=B.BSD_FP16, tie_guard_rel=-1.0))
    ref = _arrays(dec.decode(synd))
    torch.cuda.synchronize()
    assert (ref["status"] & 24).sum() == 0        # no near-tie flag, no re-run
    for call in range(2):
        out = dec.alloc_outputs(shots.B)
        for t in (out.corrections, out.obs_flips, out.status, out.iters):
            t.fill_(-1)
        rc = dec.decode_noalloc(synd, out)
        assert rc == B.BSD_OK, B.bsd_error_string(rc)
        torch.cuda.synchronize()
        got = _arrays(out)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), f"call {call}: {k} differs"
    assert (ref["status"] == 2).sum() > 0
    dec.close()
