"""The batched seed BP: many shots' first BP runs (Alg. 3) at once, messages
streamed through device memory with the shots contiguous.

It must change nothing: corrections, observable flips, status and iteration
counts equal those of the per-candidate seed kernel (batch_slots = -1) and of
the oracle at single precision, bit for bit, whatever the number of slots --
including shots it hands back to the per-candidate kernel (seeds that fail,
or whose e^ has more ones than a slot lists) and 16-bit message storage.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2512_07057_gb300 import binding as B  # noqa: E402
from paper_2512_07057_gb300 import decoder as D  # noqa: E402
from paper_2512_07057_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

KEYS = ("corrections", "obs_flips", "status", "iters")


def _decode(prob, params, synd_np):
    dec = D.BeamSearchDecoder(prob, params)
    out = dec.decode(D.to_torch_words(synd_np))
    torch.cuda.synchronize()
    assert dec.sync_error() == 0
    res = {k: D.from_torch_words(getattr(out, k)).copy() for k in KEYS}
    res["batch"] = dec.info["batch"]
    # the same kernels launched one by one (the loop flag read back by the host)
    dec.profile(True)
    dec.profile_read()
    out2 = dec.decode(D.to_torch_words(synd_np))
    prof = dec.profile_read()
    for k in KEYS:
        assert np.array_equal(D.from_torch_words(getattr(out2, k)), res[k]), f"direct launches: {k} differs"
    dec.close()
    return res, prof


def _oracle(prob, params, synd_np, storage=0):
    op = oracle.Params(max_rounds=params.max_rounds, beam_width=params.beam_width,
                       initial_iters=params.initial_iters, iters_per_round=params.iters_per_round,
                       num_results=params.num_results, ms_scale=float(params.ms_scale),
                       llr_clamp=float(params.llr_clamp), msg_storage=storage)
    return oracle.Graph(prob, "f32").decode_batch(synd_np, op, nthreads=8)


def _same(a, b, n_rows):
    for k, k2 in (("corrections", "corrections"), ("status", "status"), ("iters", "iters")):
        bad = np.nonzero((a[k] != b[k2]).reshape(n_rows, -1).any(1))[0]
        assert bad.size == 0, f"{k} differs on {bad.size} shots, first {bad[:8]}"


@pytest.mark.parametrize("slots", [256, 2048])
def test_phenomenological_dem_batched_equals_per_candidate_and_oracle(slots):
    """The phenomenological DEM (column degree 2-3) at p = q = 4e-3 with
    beam64_640iters: a few slots (many refills) and the default."""
    prob = W.bb_phenomenological(12, 6, 12, 4e-3, 4e-3)
    shots = W.sample_shots(prob, 20_000, "batch_phen")
    base = dict(ms_scale=0.625, workspace_bytes=4 << 30)
    on, prof = _decode(prob, D.make_params("beam64_640iters", batch_slots=slots, **base), shots.syndromes)
    off, _ = _decode(prob, D.make_params("beam64_640iters", batch_slots=-1, **base), shots.syndromes)
    assert on["batch"]["active"] and not off["batch"]["active"]
    if slots:
        assert on["batch"]["slots"] == slots
    for k in ("corrections", "obs_flips", "status", "iters"):
        assert np.array_equal(on[k], off[k]), k
    ref = _oracle(prob, D.make_params("beam64_640iters", **base), shots.syndromes)
    _same(on, ref, shots.B)
    assert prof["exec_iters"][2] > 0                      # the batch ran seed iterations
    assert (on["status"] == 2).sum() > 0                  # and handed shots on to the beam


def test_synthetic_dem_batched_with_handoffs():
    """The synthetic 936 x 8800 DEM (column degree 2-6) with dense syndromes
    mixed in: 5% of the shots get the syndrome of 60 random error columns, so
    their e^ can exceed a slot's list and their seed BP can fail; every shot
    still decodes exactly as the oracle does."""
    prob = W.synthetic_dem()
    shots = W.sample_shots(prob, 6_000, "batch_syn")
    synd = shots.syndromes.copy()
    rng = np.random.default_rng(5)
    dense = rng.choice(shots.B, size=300, replace=False)
    e = np.zeros((300, prob.N), np.uint8)
    for r in range(300):
        e[r, rng.choice(prob.N, size=60, replace=False)] = 1
    synd[dense] = W.pack_bits(W.syndrome_of(prob, e))
    params = D.make_params("beam8_230iters", ms_scale=0.625, workspace_bytes=2 << 30, batch_slots=512)
    on, prof = _decode(prob, params, synd)
    ref = _oracle(prob, params, synd)
    _same(on, ref, shots.B)
    assert (on["status"][dense] != 1).sum() > 0           # some dense shots left the seed
    assert prof["exec_iters"][0] > prof["exec_iters"][2]  # and the per-candidate kernel ran them again


@pytest.mark.parametrize("prec", [B.BSD_FP16, B.BSD_BF16])
def test_16bit_storage_batched(prec):
    """16-bit message storage in the batch, re-runs of near-tie shots off:
    equal to the oracle's 16-bit run bit for bit."""
    prob = W.bb_phenomenological(12, 6, 12, 3e-3, 3e-3)
    shots = W.sample_shots(prob, 10_000, "batch_16")
    params = D.make_params("beam64_640iters", ms_scale=0.625, msg_precision=prec, tie_guard_rel=-1.0,
                           workspace_bytes=2 << 30, batch_slots=1024)
    on, _ = _decode(prob, params, shots.syndromes)
    assert on["batch"]["active"]
    ref = _oracle(prob, params, shots.syndromes, storage={B.BSD_FP16: 1, B.BSD_BF16: 2}[prec])
    _same(on, ref, shots.B)


def test_high_degree_columns_and_negative_priors():
    """A random code with columns of degree up to 16 (the generic engine's
    largest bound) and some p_j > 1/2 (no screen, no zero-syndrome shortcut):
    the batch starts from every shot of the chunk."""
    rng = np.random.default_rng(3)
    M, N = 60, 150
    H = np.zeros((M, N), np.uint8)
    for j in range(N):
        H[rng.choice(M, size=int(rng.integers(2, 17)), replace=False), j] = 1
    A = (rng.random((3, N)) < 0.1).astype(np.uint8)
    pri = rng.uniform(0.01, 0.1, size=N)
    pri[rng.choice(N, size=5, replace=False)] = 0.6
    prob = W.problem_from_dense(H, A, pri, name="deg16")
    shots = W.sample_shots(prob, 4_000, "batch_deg16")
    params = D.make_params(max_rounds=5, beam_width=8, initial_iters=20, iters_per_round=10, ms_scale=0.7,
                           batch_slots=256)
    on, _ = _decode(prob, params, shots.syndromes)
    assert on["batch"]["active"]
    _same(on, _oracle(prob, params, shots.syndromes), shots.B)


def test_default_slots_follow_the_code_size():
    """By default the batch is used for codes of at least 16384 edges (the
    synthetic DEM), not for smaller ones (the phenomenological DEM)."""
    syn = D.BeamSearchDecoder(W.synthetic_dem(), D.make_params("beam32_340iters", ms_scale=0.625,
                                                               workspace_bytes=2 << 30))
    assert syn.info["batch"]["active"] and syn.info["batch"]["slots"] >= 256
    syn.close()
    phen = D.BeamSearchDecoder(W.bb_phenomenological(12, 6, 12, 2e-3, 2e-3),
                               D.make_params("beam32_340iters", ms_scale=0.625))
    assert not phen.info["batch"]["active"] and phen.info["batch"]["slots"] == 0
    phen.close()


def test_batch_is_off_where_it_does_not_apply():
    """num_results > 1 (a converged seed joins results and the search goes
    on), weighted min-sum and the small engine of the BB codes keep the
    per-candidate seed kernel even when slots are requested."""
    phen = W.bb_phenomenological(6, 6, 4, 0.01, 0.01)
    d = D.BeamSearchDecoder(phen, D.make_params("beam64_32res_640iters", ms_scale=0.625, batch_slots=512))
    assert not d.info["batch"]["active"]
    d.close()
    d = D.BeamSearchDecoder(W.bb144_code_capacity(0.03), D.make_params("beam32_340iters", ms_scale=0.625,
                                                                       batch_slots=512))
    assert not d.info["batch"]["active"]
    d.close()
    d = D.BeamSearchDecoder(phen, D.make_params("beam8_230iters", ms_scale=0.625, batch_slots=512))
    assert d.info["batch"]["active"]
    d.set_weights(np.full((3, phen.n_edges), 0.625, np.float32))
    assert not B.bsd_get_batch(d.h)["active"]
    d.close()
