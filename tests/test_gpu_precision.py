"""16-bit message storage (binary16 / bfloat16) with single-precision re-runs.

The decoder stores every E message in 16 bits and computes in single
precision; a shot whose search meets a near tie (an argmin or pruning margin
inside (0, tie_guard)) is decoded again with single-precision messages.
Expected result per shot, from the oracle's float build:
  * not flagged by the 16-bit oracle run: that run's outputs, bit for bit;
  * flagged: the single-precision run's outputs, status | NEAR_TIE | FP32_RERUN.
The error against double precision is measured on the LLRs and the LER.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2512_07057_gb300 import binding as B  # noqa: E402
from paper_2512_07057_gb300 import decoder as D  # noqa: E402
from paper_2512_07057_gb300 import workloads as W  # noqa: E402
from parity_f64 import check_against_f64  # noqa: E402

pytestmark = pytest.mark.gpu

GUARD = {B.BSD_FP16: 1e-3, B.BSD_BF16: 1e-2}
STORAGE = {B.BSD_FP16: 1, B.BSD_BF16: 2}


def _gpu(prob, params, syndromes):
    dec = D.BeamSearchDecoder(prob, params)
    out = dec.decode(D.to_torch_words(syndromes))
    torch.cuda.synchronize()
    res = {k: D.from_torch_words(getattr(out, a)).copy()
           for k, a in (("corrections", "corrections"), ("obs", "obs_flips"), ("status", "status"), ("iters", "iters"))}
    dec.close()
    return res


def _expected(prob, params, syndromes, prec):
    base = dict(max_rounds=params.max_rounds, beam_width=params.beam_width, initial_iters=params.initial_iters,
                iters_per_round=params.iters_per_round, num_results=params.num_results,
                ms_scale=float(params.ms_scale), llr_clamp=float(params.llr_clamp))
    g = oracle.Graph(prob, "f32")
    r16 = g.decode_batch(syndromes, oracle.Params(msg_storage=STORAGE[prec], tie_guard=GUARD[prec], **base),
                         nthreads=8)
    r32 = g.decode_batch(syndromes, oracle.Params(**base), nthreads=8)
    flag = (r16["status"] & 8) > 0
    exp = {k: r16[k].copy() for k in ("corrections", "obs", "status", "iters")}
    for k in ("corrections", "obs", "iters"):
        exp[k][flag] = r32[k][flag]
    exp["status"][flag] = r32["status"][flag] | 8 | 16
    return exp, flag


def _check(gpu, exp, K):
    for k in ("corrections", "status", "iters"):
        bad = np.nonzero((gpu[k] != exp[k]).reshape(len(exp["status"]), -1).any(1))[0]
        assert bad.size == 0, f"{k} differs on {bad.size} shots, first {bad[:8]}"
    if K > 0:
        assert np.array_equal(gpu["obs"][:, :exp["obs"].shape[1]], exp["obs"])


@pytest.mark.parametrize("prec", [B.BSD_FP16, B.BSD_BF16])
def test_bb72_16bit_messages(prec):
    prob = W.bb72_code_capacity(0.03)
    shots = W.sample_shots(prob, 6000, "bb72_cc_p0.03")
    params = D.make_params(max_rounds=10, beam_width=8, initial_iters=50, iters_per_round=20, ms_scale=0.625,
                           msg_precision=prec)
    gpu = _gpu(prob, params, shots.syndromes)
    exp, flag = _expected(prob, params, shots.syndromes, prec)
    _check(gpu, exp, prob.K)
    assert flag.sum() < 0.05 * shots.B


@pytest.mark.parametrize("prec", [B.BSD_FP16, B.BSD_BF16])
def test_bb144_16bit_messages(prec):
    prob = W.bb144_code_capacity(0.05)
    shots = W.sample_shots(prob, 4000, "bb144_cc_p0.05")
    params = D.make_params("beam32_340iters", ms_scale=0.625, msg_precision=prec)
    gpu = _gpu(prob, params, shots.syndromes)
    exp, flag = _expected(prob, params, shots.syndromes, prec)
    _check(gpu, exp, prob.K)
    assert flag.sum() > 0                                    # the re-run path ran


@pytest.mark.parametrize("prec", [B.BSD_FP16, B.BSD_BF16])
def test_irregular_code_16bit_messages(prec):
    """Irregular column weights run the generic engine."""
    rng = np.random.default_rng(3)
    prob = W.random_ldpc(24, 48, 3, 0.06, 11, K=3)
    prob.priors = rng.uniform(0.01, 0.2, size=prob.N)
    shots = W.sample_shots(prob, 3000, "rand16")
    params = D.make_params(max_rounds=6, beam_width=4, initial_iters=12, iters_per_round=7, num_results=2,
                           ms_scale=0.75, msg_precision=prec)
    gpu = _gpu(prob, params, shots.syndromes)
    exp, _ = _expected(prob, params, shots.syndromes, prec)
    _check(gpu, exp, prob.K)


def test_phenomenological_dem_16bit_small():
    """The phenomenological detector error model (936 x 2592): weight-1 rows
    of the perfect round exercise the empty minimum in every shot."""
    prob = W.bb_phenomenological(12, 6, 12, 2e-3, 2e-3)
    shots = W.sample_shots(prob, 96, "phenom_small")
    params = D.make_params(max_rounds=3, beam_width=4, initial_iters=20, iters_per_round=10, ms_scale=0.625,
                           msg_precision=B.BSD_FP16)
    gpu = _gpu(prob, params, shots.syndromes)
    exp, _ = _expected(prob, params, shots.syndromes, B.BSD_FP16)
    _check(gpu, exp, prob.K)


@pytest.mark.parametrize("prec,tol", [(B.BSD_FP16, 2e-3), (B.BSD_BF16, 2e-2)])
def test_16bit_llr_error_against_double(prec, tol):
    """LLRs with 16-bit messages: bit-exact against the oracle's float build
    with the same storage, and within a stated error of double precision."""
    prob = W.bb144_code_capacity(0.05)
    shots = W.sample_shots(prob, 128, "llr16")
    dec = D.BeamSearchDecoder(prob, D.make_params(ms_scale=0.625, msg_precision=prec))
    llr, _ = dec.bp_llr(D.to_torch_words(shots.syndromes), 10)
    torch.cuda.synchronize()
    llr = llr.cpu().numpy()
    g32, g64 = oracle.Graph(prob, "f32"), oracle.Graph(prob, "f64")
    s_all = W.unpack_bits(shots.syndromes, prob.M)
    rel = []
    for b in range(32):
        r16 = g32.bp(s_all[b], 10, oracle.Params(ms_scale=0.625, msg_storage=STORAGE[prec]))
        assert np.array_equal(llr[b], r16["llr"][-1])
        a = g64.bp(s_all[b], 10, oracle.Params(ms_scale=0.625))["llr"][-1]
        rel.append(np.median(np.abs(llr[b] - a) / np.maximum(1.0, np.abs(a))))
    assert np.median(rel) < tol
    dec.close()


def test_direct_launches_after_later_decoders():
    """Kernel attributes are shared by all decoders: a 16-bit decoder of the
    phenomenological DEM (two warps per block), its single-precision twin
    and a [[72,12,6]] decoder created afterwards (other block shapes) must
    leave the first decoder's direct launches (kernel timing on) valid, with
    the same outputs as its graph launches."""
    prob = W.bb_phenomenological(12, 6, 12, 3e-3, 3e-3)
    shots = W.sample_shots(prob, 3000, "phenom_direct")
    dec = D.BeamSearchDecoder(prob, D.make_params("beam64_640iters", ms_scale=0.625, msg_precision=B.BSD_FP16,
                                                  workspace_bytes=1 << 30))
    other = D.BeamSearchDecoder(W.bb72_code_capacity(0.03), D.make_params(ms_scale=0.625))
    s = D.to_torch_words(shots.syndromes)
    ref = dec.decode(s)
    torch.cuda.synchronize()
    ref = {a: D.from_torch_words(getattr(ref, a)).copy() for a in ("corrections", "status", "iters")}
    dec.profile(True)
    out = dec.decode(s)
    torch.cuda.synchronize()
    prof = dec.profile_read()
    for a in ("corrections", "status", "iters"):
        assert np.array_equal(D.from_torch_words(getattr(out, a)), ref[a])
    assert prof["launches"][0] >= 1
    dec.close()
    other.close()


@pytest.mark.parametrize("prec", [B.BSD_FP32, B.BSD_FP16])
def test_full_size_phenomenological_sampled(prec):
    """The phenomenological DEM at the benchmark's size and launch shape: 10^5
    shots at p = q = 3e-3 with beam64_640iters, autotuned as bench.py runs it;
    1000 sampled shots against the oracle (for 16-bit storage: the 16-bit run,
    or the single-precision run on shots it flags)."""
    prob = W.bb_phenomenological(12, 6, 12, 3e-3, 3e-3)
    shots = W.sample_shots(prob, 100_000, W.shot_seed("bb144_phen_p0.003", 0))
    params = D.make_params("beam64_640iters", ms_scale=0.625, msg_precision=prec, workspace_bytes=16 << 30)
    dec = D.BeamSearchDecoder(prob, params)
    s = D.to_torch_words(shots.syndromes)
    dec.autotune(s[:16384].contiguous())
    out = dec.decode(s)
    torch.cuda.synchronize()
    gpu = {k: D.from_torch_words(getattr(out, a)).copy()
           for k, a in (("corrections", "corrections"), ("obs", "obs_flips"), ("status", "status"), ("iters", "iters"))}
    dec.close()
    idx = np.sort(np.random.default_rng(2).choice(shots.B, size=1000, replace=False))
    sub = {k: v[idx] for k, v in gpu.items()}
    if prec == B.BSD_FP32:
        base = dict(max_rounds=20, beam_width=64, initial_iters=40, iters_per_round=30, num_results=1,
                    ms_scale=0.625, llr_clamp=1e4)
        exp = oracle.Graph(prob, "f32").decode_batch(shots.syndromes[idx], oracle.Params(**base), nthreads=16)
        exp = {k: exp[k] for k in ("corrections", "obs", "status", "iters")}
        check_against_f64(prob, oracle.Params(**base), shots.syndromes[idx], sub, nthreads=16)
    else:
        exp, _ = _expected(prob, params, shots.syndromes[idx], prec)
    _check(sub, exp, prob.K)


def test_full_size_synthetic_dem_fp16_sampled():
    """The 936 x 8800 synthetic DEM with binary16 message storage at 10^6
    shots, autotuned, with near-tie re-runs: the batched seed BP stores its
    messages in 16 bits too.  1000 sampled shots equal the oracle's 16-bit
    run (or, on shots it flags, the single-precision run), bit for bit."""
    prob = W.synthetic_dem()
    shots = W.sample_shots(prob, 1_000_000, "synthetic_dem")
    params = D.make_params("beam32_340iters", ms_scale=0.625, msg_precision=B.BSD_FP16, workspace_bytes=32 << 30)
    dec = D.BeamSearchDecoder(prob, params)
    assert dec.info["batch"]["active"]
    s = D.to_torch_words(shots.syndromes)
    dec.autotune(s[:16384].contiguous())
    out = dec.decode(s)
    torch.cuda.synchronize()
    gpu = {k: D.from_torch_words(getattr(out, a)).copy()
           for k, a in (("corrections", "corrections"), ("obs", "obs_flips"), ("status", "status"), ("iters", "iters"))}
    dec.close()
    idx = np.sort(np.random.default_rng(4).choice(shots.B, size=1000, replace=False))
    sub = {k: v[idx] for k, v in gpu.items()}
    exp, _ = _expected(prob, params, shots.syndromes[idx], B.BSD_FP16)
    _check(sub, exp, prob.K)
