"""Weighted min-sum in the decoder (bsd_set_weights) against the oracle.

Weights w_{e,t} replace the scale of Eq. 1; iteration t of every BP call uses
row min(t, T) - 1.  Expected: the oracle's single-precision build with the
same float32 weights, bit for bit, through the small engine ([[72,12,6]] and
[[144,12,12]]) and the generic one (irregular code, phenomenological DEM).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2512_07057_gb300 import binding as B  # noqa: E402
from paper_2512_07057_gb300 import decoder as D  # noqa: E402
from paper_2512_07057_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _run(dec, syndromes):
    out = dec.decode(D.to_torch_words(syndromes))
    torch.cuda.synchronize()
    return {k: D.from_torch_words(getattr(out, a)).copy()
            for k, a in (("corrections", "corrections"), ("obs", "obs_flips"), ("status", "status"), ("iters", "iters"))}


def _oracle(prob, base, weights, syndromes):
    g = oracle.Graph(prob, "f32")
    return g.decode_batch(syndromes, oracle.Params(weights=weights, **base), nthreads=8)


def _same(gpu, ref, K):
    for k in ("corrections", "status", "iters"):
        bad = np.nonzero((gpu[k] != ref[k]).reshape(len(ref["status"]), -1).any(1))[0]
        assert bad.size == 0, f"{k} differs on {bad.size} shots, first {bad[:8]}"
    if K > 0:
        assert np.array_equal(gpu["obs"][:, :ref["obs"].shape[1]], ref["obs"])


CASES = {
    "bb72": (lambda: W.bb72_code_capacity(0.04), dict(max_rounds=8, beam_width=8, initial_iters=30, iters_per_round=12)),
    "bb144": (lambda: W.bb144_code_capacity(0.05), dict(max_rounds=6, beam_width=16, initial_iters=30, iters_per_round=15)),
    "irregular": (lambda: W.random_ldpc(24, 48, 3, 0.06, 11, K=3),
                  dict(max_rounds=5, beam_width=4, initial_iters=12, iters_per_round=7, num_results=2)),
    "phenom": (lambda: W.bb_phenomenological(6, 6, 4, 0.01, 0.01),
               dict(max_rounds=4, beam_width=8, initial_iters=20, iters_per_round=10)),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("T", [1, 6])
def test_weighted_decode_matches_oracle(case, T):
    build, base = CASES[case]
    prob = build()
    shots = W.sample_shots(prob, 3000, f"weighted_{case}")
    rng = np.random.default_rng(17 + T)
    w = rng.uniform(0.45, 1.05, size=(T, prob.n_edges)).astype(np.float32)
    dec = D.BeamSearchDecoder(prob, D.make_params(ms_scale=0.625, workspace_bytes=1 << 30, **base))
    dec.set_weights(w)
    gpu = _run(dec, shots.syndromes)
    _same(gpu, _oracle(prob, dict(base, ms_scale=0.625), w, shots.syndromes), prob.K)
    # and back to the scale
    dec.set_weights(None)
    gpu = _run(dec, shots.syndromes)
    _same(gpu, _oracle(prob, dict(base, ms_scale=0.625), None, shots.syndromes), prob.K)
    dec.close()


def test_uniform_weights_equal_scale_on_gpu():
    prob = W.bb144_code_capacity(0.05)
    shots = W.sample_shots(prob, 4000, "weighted_uniform")
    dec = D.BeamSearchDecoder(prob, D.make_params("beam32_340iters", ms_scale=0.625))
    a = _run(dec, shots.syndromes)
    dec.set_weights(np.full((3, prob.n_edges), 0.625, np.float32))
    b = _run(dec, shots.syndromes)
    for k in a:
        assert np.array_equal(a[k], b[k])
    dec.close()


def test_weighted_llr_and_noalloc_match_oracle():
    prob = W.bb_phenomenological(6, 6, 4, 0.01, 0.01)
    shots = W.sample_shots(prob, 64, "weighted_llr")
    rng = np.random.default_rng(5)
    T = 4
    w = rng.uniform(0.5, 1.0, size=(T, prob.n_edges)).astype(np.float32)
    dec = D.BeamSearchDecoder(prob, D.make_params(ms_scale=0.625, max_rounds=3, beam_width=4, initial_iters=15,
                                                  iters_per_round=8))
    dec.set_weights(w)
    llr, _ = dec.bp_llr(D.to_torch_words(shots.syndromes), 7)
    torch.cuda.synchronize()
    llr = llr.cpu().numpy()
    g = oracle.Graph(prob, "f32")
    s_all = W.unpack_bits(shots.syndromes, prob.M)
    for b in range(16):
        ref = g.bp(s_all[b], 7, oracle.Params(weights=w))["llr"][-1]
        assert np.array_equal(llr[b], ref)
    out = dec.alloc_outputs(shots.B)
    rc = dec.decode_noalloc(D.to_torch_words(shots.syndromes), out)
    torch.cuda.synchronize()
    assert rc == 0
    ref = g.decode_batch(shots.syndromes, oracle.Params(weights=w, ms_scale=0.625, max_rounds=3, beam_width=4,
                                                       initial_iters=15, iters_per_round=8), nthreads=4)
    assert np.array_equal(D.from_torch_words(out.corrections), ref["corrections"])
    assert np.array_equal(D.from_torch_words(out.status), ref["status"])
    dec.close()


def test_weights_rejected():
    prob = W.bb72_code_capacity(0.03)
    dec = D.BeamSearchDecoder(prob, D.make_params(ms_scale=0.625))
    bad = np.full((2, prob.n_edges), 0.6, np.float32)
    bad[1, 5] = np.nan
    with pytest.raises(B.BsdError) as ei:
        dec.set_weights(bad)
    assert ei.value.code == B.BSD_ERR_INVALID_ARG
    dec.close()
    d16 = D.BeamSearchDecoder(prob, D.make_params(ms_scale=0.625, msg_precision=B.BSD_FP16))
    with pytest.raises(B.BsdError) as ei:
        d16.set_weights(np.full((1, prob.n_edges), 0.6, np.float32))
    assert ei.value.code == B.BSD_ERR_UNSUPPORTED
    d16.close()
