"""Block groups: a whole block of warps per BP candidate (bsd_params.group_warps).

The block engine computes every row and column on one thread and reduces
exactly, so it must give the single-precision oracle's outputs bit for bit,
like the one-warp engine: checked on the [[72,12,6]] code (forced off its
small engine), an irregular code, the phenomenological DEM and a slice of
the 936 x 8800 synthetic DEM, with single-precision, 16-bit and weighted
messages, and for bsd_bp_llr and the allocation-free path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2512_07057_gb300 import binding as B  # noqa: E402
from paper_2512_07057_gb300 import decoder as D  # noqa: E402
from paper_2512_07057_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _irregular():
    rng = np.random.default_rng(3)
    p = W.random_ldpc(24, 48, 3, 0.06, 11, K=3)
    p.priors = rng.uniform(0.01, 0.2, size=p.N)
    return p


CASES = {
    "bb72": (lambda: W.bb72_code_capacity(0.04), 3000,
             dict(max_rounds=8, beam_width=8, initial_iters=30, iters_per_round=12)),
    "irregular": (_irregular, 3000,
                  dict(max_rounds=5, beam_width=4, initial_iters=12, iters_per_round=7, num_results=2)),
    "phenom": (lambda: W.bb_phenomenological(12, 6, 12, 4e-3, 4e-3), 2000,
               dict(max_rounds=6, beam_width=16, initial_iters=30, iters_per_round=15)),
    "synthetic_dem": (lambda: W.synthetic_dem(), 300,
                      dict(max_rounds=3, beam_width=8, initial_iters=30, iters_per_round=15)),
}


def _run(prob, params, syndromes):
    dec = D.BeamSearchDecoder(prob, params)
    out = dec.decode(D.to_torch_words(syndromes))
    torch.cuda.synchronize()
    res = {k: D.from_torch_words(getattr(out, a)).copy()
           for k, a in (("corrections", "corrections"), ("obs", "obs_flips"), ("status", "status"), ("iters", "iters"))}
    dec.close()
    return res


def _same(gpu, ref, K):
    for k in ("corrections", "status", "iters"):
        bad = np.nonzero((gpu[k] != ref[k]).reshape(len(ref["status"]), -1).any(1))[0]
        assert bad.size == 0, f"{k} differs on {bad.size} shots, first {bad[:8]}"
    if K > 0:
        assert np.array_equal(gpu["obs"][:, :ref["obs"].shape[1]], ref["obs"])


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("gw", [2, 4, 8, 16])
def test_block_engine_matches_oracle(case, gw):
    build, n, base = CASES[case]
    prob = build()
    shots = W.sample_shots(prob, n, f"block_{case}")
    gpu = _run(prob, D.make_params(ms_scale=0.625, workspace_bytes=1 << 30, group_warps=gw, **base),
               shots.syndromes)
    ref = oracle.Graph(prob, "f32").decode_batch(shots.syndromes, oracle.Params(ms_scale=0.625, **base),
                                                 nthreads=8)
    _same(gpu, ref, prob.K)


@pytest.mark.parametrize("prec", [B.BSD_FP16, B.BSD_BF16])
def test_block_engine_16bit_with_reruns(prec):
    prob = W.bb_phenomenological(12, 6, 12, 4e-3, 4e-3)
    shots = W.sample_shots(prob, 2000, "block_16bit")
    base = dict(max_rounds=6, beam_width=16, initial_iters=30, iters_per_round=15)
    gpu = _run(prob, D.make_params(ms_scale=0.625, msg_precision=prec, group_warps=8, **base), shots.syndromes)
    guard, storage = (1e-3, 1) if prec == B.BSD_FP16 else (1e-2, 2)
    g = oracle.Graph(prob, "f32")
    r16 = g.decode_batch(shots.syndromes, oracle.Params(ms_scale=0.625, msg_storage=storage, tie_guard=guard,
                                                        **base), nthreads=8)
    r32 = g.decode_batch(shots.syndromes, oracle.Params(ms_scale=0.625, **base), nthreads=8)
    flag = (r16["status"] & 8) > 0
    exp = {k: r16[k].copy() for k in ("corrections", "obs", "status", "iters")}
    for k in ("corrections", "obs", "iters"):
        exp[k][flag] = r32[k][flag]
    exp["status"][flag] = r32["status"][flag] | 8 | 16
    _same(gpu, exp, prob.K)


def test_block_engine_weights_llr_and_noalloc():
    prob = W.bb_phenomenological(6, 6, 4, 0.01, 0.01)
    shots = W.sample_shots(prob, 500, "block_weighted")
    rng = np.random.default_rng(9)
    w = rng.uniform(0.5, 1.0, size=(4, prob.n_edges)).astype(np.float32)
    base = dict(max_rounds=3, beam_width=4, initial_iters=15, iters_per_round=8)
    dec = D.BeamSearchDecoder(prob, D.make_params(ms_scale=0.625, group_warps=4, **base))
    dec.set_weights(w)
    g = oracle.Graph(prob, "f32")
    out = dec.decode(D.to_torch_words(shots.syndromes))
    torch.cuda.synchronize()
    ref = g.decode_batch(shots.syndromes, oracle.Params(weights=w, ms_scale=0.625, **base), nthreads=4)
    assert np.array_equal(D.from_torch_words(out.corrections), ref["corrections"])
    assert np.array_equal(D.from_torch_words(out.status), ref["status"])
    llr, _ = dec.bp_llr(D.to_torch_words(shots.syndromes[:16]), 6)
    torch.cuda.synchronize()
    llr = llr.cpu().numpy()
    s_all = W.unpack_bits(shots.syndromes, prob.M)
    for b in range(16):
        assert np.array_equal(llr[b], g.bp(s_all[b], 6, oracle.Params(weights=w))["llr"][-1])
    o2 = dec.alloc_outputs(shots.B)
    assert dec.decode_noalloc(D.to_torch_words(shots.syndromes), o2) == 0
    torch.cuda.synchronize()
    assert np.array_equal(D.from_torch_words(o2.corrections), ref["corrections"])
    dec.close()


def test_group_warps_rejected():
    prob = W.bb72_code_capacity(0.03)
    for gw in (17, -1):
        with pytest.raises(B.BsdError) as ei:
            D.BeamSearchDecoder(prob, D.make_params(group_warps=gw))
        assert ei.value.code == B.BSD_ERR_INVALID_ARG
