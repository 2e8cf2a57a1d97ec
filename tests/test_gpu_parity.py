"""GPU parity: the CUDA decoder (through the C ABI) against the CPU oracle.

Two comparisons per workload:
  * against the oracle at the library's precision (single): corrections,
    observable flips, status and iteration counts bit-exact on every shot;
  * against the double-precision oracle: identical on every shot except
    those whose double- and single-precision decision logs first differ at
    or after a decision with a relative margin below 1e-4 or an exact tie
    (counts at 1e-6 and 1e-4 printed); LLRs within 1e-4 relative; logical
    error rates within a 95% Wilson interval of each other.
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


def _oracle_params(p: "D.B.bsd_params", **kw) -> oracle.Params:
    return oracle.Params(max_rounds=p.max_rounds, beam_width=p.beam_width, initial_iters=p.initial_iters,
                         iters_per_round=p.iters_per_round, num_results=p.num_results,
                         ms_scale=float(p.ms_scale), llr_clamp=float(p.llr_clamp), **kw)


def _gpu_decode(prob, params, syndromes):
    dec = D.BeamSearchDecoder(prob, params)
    out = dec.decode(D.to_torch_words(syndromes))
    torch.cuda.synchronize()
    assert dec.sync_error() == 0
    res = dict(corrections=D.from_torch_words(out.corrections), obs=D.from_torch_words(out.obs_flips),
               status=D.from_torch_words(out.status), iters=D.from_torch_words(out.iters), info=dec.info)
    dec.close()
    return res


def _assert_bit_exact(gpu, ref, K):
    for k in ("corrections", "status", "iters"):
        bad = np.nonzero((gpu[k] != ref[k]).reshape(len(gpu["status"]), -1).any(1))[0]
        assert bad.size == 0, f"{k} differs on {bad.size} shots, first {bad[:10]}"
    if K > 0:
        assert np.array_equal(gpu["obs"][:, :ref["obs"].shape[1]], ref["obs"])


def _wilson(k, n, z=1.96):
    p = k / n
    d = 1 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * np.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return c - h, c + h


def _ler(res, shots, K):
    o = W.unpack_bits(res["obs"][:, :(K + 31) // 32], K)
    t = W.unpack_bits(shots.obs, K)
    fail = (o != t).any(1) | (res["status"] == 4)
    return int(fail.sum())


def _check_workload(prob, params, shots, nthreads=8, check_f64=True):
    gpu = _gpu_decode(prob, params, shots.syndromes)
    op = _oracle_params(params)
    ref32 = oracle.Graph(prob, "f32").decode_batch(shots.syndromes, op, nthreads=nthreads)
    _assert_bit_exact(gpu, ref32, prob.K)
    # invariants: H e = s on every converged shot
    e = W.unpack_bits(gpu["corrections"], prob.N).astype(np.int64)
    s = W.unpack_bits(shots.syndromes, prob.M)
    conv = gpu["status"] != 4
    assert np.array_equal(((e @ prob.H_dense().T) % 2)[conv], s[conv])
    if check_f64:
        # a disagreement with double precision must follow a near tie of the
        # double-precision run at or before the first divergent decision, and
        # must be rare
        _, ref64 = check_against_f64(prob, op, shots.syndromes, gpu, nthreads=nthreads)
        k_gpu, k_ref = _ler(gpu, shots, prob.K), _ler(ref64, shots, prob.K)
        lo, hi = _wilson(k_ref, shots.B)
        lo2, hi2 = _wilson(k_gpu, shots.B)
        assert lo2 <= hi and lo <= hi2, (k_gpu, k_ref)
    return gpu


# ----------------------------------------------------------------------------
# the paper's plain method on the [[72,12,6]] BB code (all 10^4 shots)
# ----------------------------------------------------------------------------
def test_bb72_code_capacity_all_shots():
    prob = W.bb72_code_capacity(0.03)
    shots = W.sample_shots(prob, 10_000, "bb72_cc_p0.03")
    params = D.make_params(max_rounds=10, beam_width=8, initial_iters=50, iters_per_round=20, ms_scale=0.625)
    gpu = _check_workload(prob, params, shots)
    assert (gpu["status"] == 2).sum() > 50          # the beam rounds were exercised


@pytest.mark.parametrize("p", [0.01, 0.03, 0.05])
def test_bb144_beam32(p):
    prob = W.bb144_code_capacity(p)
    shots = W.sample_shots(prob, 20_000, f"bb144_cc_p{p}")
    params = D.make_params("beam32_340iters", ms_scale=0.625)
    _check_workload(prob, params, shots)


def test_bb144_alpha1_paper_literal():
    """Eq. 1 without scaling.  With equal priors every message is a small
    integer multiple of Lambda, so many Lambda_j(t) are exactly 0 in exact
    arithmetic and Eq. 4 decides them by the last rounding bit: at p = 0.04
    float(Lambda) has two trailing zero bits and the multiples cancel exactly
    in single precision, while double precision leaves +-1e-16 residues.  The
    two precisions therefore take different branches on many shots; the
    comparison that means something here is the one at equal precision."""
    prob = W.bb144_code_capacity(0.04)
    shots = W.sample_shots(prob, 5_000, "bb144_alpha1")
    params = D.make_params("beam8_230iters", ms_scale=1.0)
    _check_workload(prob, params, shots, check_f64=False)


def test_num_results_32_preset():
    prob = W.bb72_code_capacity(0.05)
    shots = W.sample_shots(prob, 3_000, "bb72_32res")
    params = D.make_params("beam64_32res_640iters", ms_scale=0.625)
    gpu = _check_workload(prob, params, shots)
    assert (gpu["status"] == 2).sum() > 100


# ----------------------------------------------------------------------------
# chunking: a small workspace forces several chunks and a ragged tail
# ----------------------------------------------------------------------------
def test_chunked_batches_match_single_pass():
    prob = W.bb144_code_capacity(0.05)
    shots = W.sample_shots(prob, 7_777, "bb144_chunks")
    small = D.make_params("beam32_340iters", ms_scale=0.625, workspace_bytes=64 << 20)
    big = D.make_params("beam32_340iters", ms_scale=0.625)
    a = _gpu_decode(prob, small, shots.syndromes)
    assert a["info"]["chunk_shots"] < shots.B and shots.B % a["info"]["chunk_shots"] != 0
    b = _gpu_decode(prob, big, shots.syndromes)
    for k in ("corrections", "obs", "status", "iters"):
        assert np.array_equal(a[k], b[k]), k
    ref32 = oracle.Graph(prob, "f32").decode_batch(shots.syndromes, _oracle_params(big), nthreads=8)
    _assert_bit_exact(a, ref32, prob.K)


@pytest.mark.parametrize("gw", [1, 8])
def test_chunked_dem_with_screen_matches_single_pass(gw):
    """The phenomenological DEM (first-iteration screen on) in several chunks
    with a ragged tail: every chunk restarts the screen's queue, and the
    outputs equal one pass over the batch and the oracle, bit for bit."""
    prob = W.bb_phenomenological(6, 6, 4, 0.01, 0.01)
    shots = W.sample_shots(prob, 5_003, "phenom_chunks")
    base = dict(max_rounds=4, beam_width=8, initial_iters=20, iters_per_round=10, ms_scale=0.625, group_warps=gw)
    small = D.make_params(workspace_bytes=24 << 20, **base)
    big = D.make_params(**base)
    a = _gpu_decode(prob, small, shots.syndromes)
    assert a["info"]["chunk_shots"] < shots.B and shots.B % a["info"]["chunk_shots"] != 0
    b = _gpu_decode(prob, big, shots.syndromes)
    for k in ("corrections", "obs", "status", "iters"):
        assert np.array_equal(a[k], b[k]), k
    ref32 = oracle.Graph(prob, "f32").decode_batch(shots.syndromes, _oracle_params(big), nthreads=8)
    _assert_bit_exact(a, ref32, prob.K)
    assert (a["status"] & 7 == 2).any()                # some shots reached the beam


# ----------------------------------------------------------------------------
# edge cases
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(4))
def test_irregular_random_codes(seed):
    rng = np.random.default_rng(seed)
    prob = W.random_ldpc(20, 40, 2 + seed % 2, 0.06, seed, K=3)
    prob.priors = rng.uniform(0.01, 0.2, size=prob.N)
    shots = W.sample_shots(prob, 3_000, f"rand_{seed}")
    params = D.make_params(max_rounds=6, beam_width=4, initial_iters=12, iters_per_round=7,
                           num_results=1 + 2 * (seed % 2), ms_scale=0.75)
    _check_workload(prob, params, shots, check_f64=False)


@pytest.mark.parametrize("M,seed", [(48, 2), (80, 5)])
def test_random_regular_codes_on_the_single_warp_engine(M, seed):
    """Random codes of row degree 6 and column degree 3 run on the single-warp
    engine; unlike the BB codes, their message placement keeps some bank
    conflicts (the search does not reach zero), so the column orders come
    partly from the fallback order.  Bit-exact against the oracle."""
    prob = W.random_regular_36(M, 0.05, seed)
    assert B.bsd_small_layout(prob.M, prob.N, prob.H_row_ptr, prob.H_col_idx)["excess"] > 0
    shots = W.sample_shots(prob, 3_000, f"reg36_{M}")
    params = D.make_params(max_rounds=6, beam_width=8, initial_iters=20, iters_per_round=10, ms_scale=0.625)
    _check_workload(prob, params, shots, check_f64=False)


@pytest.mark.parametrize("gw", [1, 8])
def test_priors_above_one_half(gw):
    """Some p_j above 1/2 (Lambda_j < 0): the zero-syndrome shortcut and the
    first-iteration screen of seed runs both rest on every Lambda_j > 0 and
    must stay off; the outputs equal the oracle's bit for bit, on a random
    code (one warp or a block of 8 per candidate) and including all-zero
    syndromes."""
    rng = np.random.default_rng(11)
    prob = W.random_ldpc(40, 80, 3, 0.05, 21, K=3)
    prob.priors = rng.uniform(0.01, 0.15, size=prob.N)
    prob.priors[rng.choice(prob.N, size=6, replace=False)] = rng.uniform(0.55, 0.7, size=6)
    shots = W.sample_shots(prob, 2_000, "above_half")
    synd = shots.syndromes.copy()
    synd[:50] = 0
    params = D.make_params(max_rounds=5, beam_width=4, initial_iters=15, iters_per_round=8, ms_scale=0.625,
                           group_warps=gw)
    gpu = _gpu_decode(prob, params, synd)
    ref32 = oracle.Graph(prob, "f32").decode_batch(synd, _oracle_params(params), nthreads=8)
    _assert_bit_exact(gpu, ref32, prob.K)


def test_screen_with_many_flipped_detectors():
    """Dense syndromes on a DEM: shots with more than 128 flipped detectors go
    to the seed BP unscreened, others are screened; all-ones, random dense,
    sampled and single-detector syndromes, bit-exact against the oracle."""
    prob = W.bb_phenomenological(12, 6, 4, 0.01, 0.01)         # 360 detectors
    rng = np.random.default_rng(8)
    n = 40
    bits = np.zeros((n, prob.M), np.uint8)
    bits[0] = 1                                                   # every detector flipped
    bits[1:20] = (rng.random((19, prob.M)) < 0.5)                 # about M/2 flipped
    bits[20:30] = W.unpack_bits(W.sample_shots(prob, 10, "dense_real").syndromes, prob.M)   # sampled errors
    for k in range(30, n):
        bits[k, rng.integers(prob.M)] = 1                         # a single detector
    synd = W.pack_bits(bits)
    params = D.make_params(max_rounds=2, beam_width=2, initial_iters=6, iters_per_round=3, ms_scale=0.625)
    gpu = _gpu_decode(prob, params, synd)
    ref32 = oracle.Graph(prob, "f32").decode_batch(synd, _oracle_params(params), nthreads=8)
    _assert_bit_exact(gpu, ref32, prob.K)
    assert (bits.sum(1) > 128).sum() >= 20


def test_first_iteration_screen_accounting():
    """Seed runs on the phenomenological DEM (every Lambda_j > 0, one result):
    a run that converges at t = 1 ends in the first-iteration screen, so the
    device counts its screened message updates and no full iteration for it.
    The full seed iterations are then those of the seeds that converged after
    more than one iteration plus initial_iters for each seed that did not."""
    prob = W.bb_phenomenological(12, 6, 12, 1e-3, 1e-3)
    shots = W.sample_shots(prob, 4_000, "screen_accounting")
    params = D.make_params("beam64_640iters", ms_scale=0.625, group_warps=8)
    dec = D.BeamSearchDecoder(prob, params)
    dec.profile(True)
    dec.profile_read()
    out = dec.decode(D.to_torch_words(shots.syndromes))
    torch.cuda.synchronize()
    rd = dec.profile_read()
    st = D.from_torch_words(out.status) & 7
    it = D.from_torch_words(out.iters).astype(np.int64)
    dec.close()
    seed = st == 1
    assert seed.mean() > 0.99
    assert rd["screen_updates"] > 0
    want = int(it[seed & (it > 1)].sum()) + params.initial_iters * int((~seed).sum())
    assert int(rd["exec_iters"][0]) == want
    ref = oracle.Graph(prob, "f32").decode_batch(shots.syndromes, _oracle_params(params), nthreads=8)
    assert np.array_equal(D.from_torch_words(out.corrections), ref["corrections"])
    assert np.array_equal(D.from_torch_words(out.iters), ref["iters"])


def test_edge_cases_small_problems():
    prob = W.bb72_code_capacity(0.08)
    rng = np.random.default_rng(5)
    WM = (prob.M + 31) // 32
    synd = np.zeros((6, WM), np.uint32)
    synd[1, 0] = 1                                    # a single unsatisfied detector
    synd[2] = W.pack_bits(np.ones(prob.M, np.uint8))  # every detector unsatisfied
    synd[3:] = W.pack_bits(rng.integers(0, 2, size=(3, prob.M)).astype(np.uint8))
    for kw in (dict(max_rounds=0, beam_width=1, initial_iters=5, iters_per_round=1),
               dict(max_rounds=4, beam_width=1, initial_iters=3, iters_per_round=2),
               dict(max_rounds=12, beam_width=64, initial_iters=2, iters_per_round=3, num_results=5),
               dict(max_rounds=3, beam_width=2, initial_iters=1, iters_per_round=1, num_results=64)):
        params = D.make_params(ms_scale=0.625, **kw)
        gpu = _gpu_decode(prob, params, synd)
        ref = oracle.Graph(prob, "f32").decode_batch(synd, _oracle_params(params), nthreads=2)
        _assert_bit_exact(gpu, ref, prob.K)
    # one shot
    params = D.make_params(ms_scale=0.625)
    gpu = _gpu_decode(prob, params, synd[3:4])
    ref = oracle.Graph(prob, "f32").decode_batch(synd[3:4], _oracle_params(params), nthreads=1)
    _assert_bit_exact(gpu, ref, prob.K)


def test_unsatisfiable_detector_and_isolated_nodes():
    """The closed-form example of the oracle pins, through the GPU: a detector
    with no error source (never satisfiable) and isolated error nodes."""
    p = np.array([0.3, 0.35, 0.2, 0.45, 0.1, 0.4])
    H = np.zeros((2, 6), np.uint8)
    H[0, 0] = H[0, 1] = 1
    prob = W.problem_from_dense(H, np.eye(6, dtype=np.uint8)[:2], p)
    synd = W.pack_bits(np.array([[0, 1], [1, 1], [0, 0], [1, 0]], np.uint8))
    params = D.make_params(max_rounds=3, beam_width=3, initial_iters=4, iters_per_round=3, ms_scale=1.0)
    gpu = _gpu_decode(prob, params, synd)
    ref = oracle.Graph(prob, "f32").decode_batch(synd, _oracle_params(params), nthreads=1)
    _assert_bit_exact(gpu, ref, prob.K)
    assert gpu["status"][0] == 4 and gpu["iters"][0] == 4 + 3 * (2 + 4 + 6)


def test_zero_syndromes():
    prob = W.bb144_code_capacity(0.03)
    synd = np.zeros((1000, 3), np.uint32)
    gpu = _gpu_decode(prob, D.make_params("beam32_340iters", ms_scale=0.625), synd)
    assert (gpu["status"] == 1).all() and (gpu["iters"] == 1).all() and (gpu["corrections"] == 0).all()
    # with num_results > 1 the shortcut is off and the seed result opens `results`
    params = D.make_params("beam64_32res_640iters", ms_scale=0.625, max_rounds=2)
    gpu = _gpu_decode(prob, params, synd[:50])
    ref = oracle.Graph(prob, "f32").decode_batch(synd[:50], _oracle_params(params), nthreads=2)
    _assert_bit_exact(gpu, ref, prob.K)


# ----------------------------------------------------------------------------
# LLRs against double precision (App. A, Eqs. 1-3)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("T", [1, 5, 30])
def test_bp_llr_against_f64(T):
    prob = W.bb144_code_capacity(0.05)
    shots = W.sample_shots(prob, 256, "llr_shots")
    params = D.make_params(ms_scale=0.625)
    dec = D.BeamSearchDecoder(prob, params)
    llr, sm = dec.bp_llr(D.to_torch_words(shots.syndromes), T)
    torch.cuda.synchronize()
    llr, sm = llr.cpu().numpy(), sm.cpu().numpy()
    g64, g32 = oracle.Graph(prob, "f64"), oracle.Graph(prob, "f32")
    op = oracle.Params(ms_scale=0.625)
    s_all = W.unpack_bits(shots.syndromes, prob.M)
    worst = 0.0
    for b in range(64):
        r64 = g64.bp(s_all[b], T, op)
        r32 = g32.bp(s_all[b], T, op)
        assert np.array_equal(llr[b], r32["llr"][-1])             # same single-precision arithmetic
        assert np.array_equal(sm[b], r32["sum_llr"])
        rel = np.abs(llr[b] - r64["llr"][-1]) / np.maximum(1.0, np.abs(r64["llr"][-1]))
        worst = max(worst, float(rel.max()))
    assert worst <= 1e-4, worst
    dec.close()


# ----------------------------------------------------------------------------
# host-buffer entry point
# ----------------------------------------------------------------------------
def test_decode_host_matches_device_entry():
    prob = W.bb144_code_capacity(0.05)
    shots = W.sample_shots(prob, 3_000, "host_entry")
    params = D.make_params("beam32_340iters", ms_scale=0.625, workspace_bytes=128 << 20)
    dec = D.BeamSearchDecoder(prob, params)
    h = dec.decode_host(shots.syndromes)
    d = dec.decode(D.to_torch_words(shots.syndromes))
    torch.cuda.synchronize()
    assert np.array_equal(h["corrections"], D.from_torch_words(d.corrections))
    assert np.array_equal(h["status"], D.from_torch_words(d.status))
    assert np.array_equal(h["iters"], D.from_torch_words(d.iters))
    assert np.array_equal(h["obs"], D.from_torch_words(d.obs_flips))
    dec.close()


# ----------------------------------------------------------------------------
# the full-size launch the benchmark times: sampled shots against the oracle
# ----------------------------------------------------------------------------
def test_full_size_bb144_sampled():
    p = 0.05
    prob = W.bb144_code_capacity(p)
    shots = W.sample_shots(prob, 1_000_000, f"bb144_cc_p{p}")
    params = D.make_params("beam32_340iters", ms_scale=0.625, workspace_bytes=32 << 30)
    gpu = _gpu_decode(prob, params, shots.syndromes)
    e = W.unpack_bits(gpu["corrections"], prob.N).astype(np.int64)
    s = W.unpack_bits(shots.syndromes, prob.M)
    conv = gpu["status"] != 4
    assert np.array_equal(((e @ prob.H_dense().T) % 2)[conv], s[conv])
    idx = np.random.default_rng(0).choice(shots.B, size=3000, replace=False)
    idx.sort()
    ref = oracle.Graph(prob, "f32").decode_batch(shots.syndromes[idx], _oracle_params(params), nthreads=8)
    sub = {k: gpu[k][idx] for k in ("corrections", "obs", "status", "iters")}
    _assert_bit_exact(sub, ref, prob.K)
    check_against_f64(prob, _oracle_params(params), shots.syndromes[idx], sub, nthreads=8)


@pytest.mark.parametrize("preset", ["beam8_230iters", "beam32_340iters", "beam64_640iters"])
def test_full_size_synthetic_dem_sampled(preset):
    """The 936 x 8800 synthetic DEM at 10^6 shots, autotuned as the benchmark
    runs it: H e^ = s on every converged shot, sampled shots bit-exact."""
    prob = W.synthetic_dem()
    shots = W.sample_shots(prob, 1_000_000, "synthetic_dem")
    params = D.make_params(preset, ms_scale=0.625, workspace_bytes=32 << 30)
    dec = D.BeamSearchDecoder(prob, params)
    s_t = D.to_torch_words(shots.syndromes)
    dec.autotune(s_t[:16384].contiguous())
    out = dec.decode(s_t)
    torch.cuda.synchronize()
    gpu = {k: D.from_torch_words(getattr(out, a)).copy()
           for k, a in (("corrections", "corrections"), ("obs", "obs_flips"), ("status", "status"), ("iters", "iters"))}
    dec.close()
    # H e^ = s on every converged shot, checked in slices on the GPU with a plain
    # torch product (0/1 entries, integer sums below 2048: exact in float16)
    Ht = torch.from_numpy(prob.H_dense().T.astype(np.float16)).cuda()
    sh32 = torch.arange(32, device="cuda", dtype=torch.int32)

    def bits(words, n):
        w = torch.from_numpy(np.ascontiguousarray(words).view(np.int32)).cuda()
        return ((w.unsqueeze(-1) >> sh32) & 1).reshape(w.shape[0], -1)[:, :n]

    conv = torch.from_numpy(gpu["status"] != 4).cuda()
    for lo in range(0, shots.B, 65536):
        sl = slice(lo, lo + 65536)
        s_hat = (bits(gpu["corrections"][sl], prob.N).half() @ Ht).remainder(2).to(torch.int32)
        bad = ((s_hat != bits(shots.syndromes[sl], prob.M)).any(1) & conv[sl]).sum().item()
        assert bad == 0
    idx = np.random.default_rng(1).choice(shots.B, size=1000, replace=False)
    idx.sort()
    ref = oracle.Graph(prob, "f32").decode_batch(shots.syndromes[idx], _oracle_params(params), nthreads=16)
    sub = {k: gpu[k][idx] for k in ("corrections", "obs", "status", "iters")}
    _assert_bit_exact(sub, ref, prob.K)
    check_against_f64(prob, _oracle_params(params), shots.syndromes[idx], sub, nthreads=16)


@pytest.mark.parametrize("gw", [1, 4])
def test_xyz_decoding_bit_exact(gw):
    """XYZ decoding (both stabilizer types in H, length-4 cycles, degree-6 Y
    columns) of [[72,12,6]] under depolarizing noise, one warp and a block of
    4 warps per candidate."""
    prob = W.bb_xyz_code_capacity(6, 6, 0.08)
    shots = W.sample_shots(prob, 4000, "xyz_parity")
    params = D.make_params("beam32_340iters", ms_scale=0.625, group_warps=gw)
    gpu = _gpu_decode(prob, params, shots.syndromes)
    ref = oracle.Graph(prob, "f32").decode_batch(shots.syndromes, _oracle_params(params), nthreads=8)
    _assert_bit_exact(gpu, ref, prob.K)


def test_dem_text_problem_decodes_bit_exact():
    """A problem read from DEM text (the phenomenological DEM written out and read
    back through bsd_dem_parse) decodes like the oracle on the same arrays."""
    src = W.bb_phenomenological(12, 6, 12, 4e-3, 4e-3)
    prob = W.problem_from_dem_arrays(D.B.bsd_dem_read(W.problem_to_dem(src)), name="dem_text")
    shots = W.sample_shots(prob, 2000, "dem_text")
    params = D.make_params("beam64_640iters", ms_scale=0.625, workspace_bytes=1 << 30)
    gpu = _gpu_decode(prob, params, shots.syndromes)
    ref = oracle.Graph(src, "f32").decode_batch(shots.syndromes, _oracle_params(params), nthreads=8)
    _assert_bit_exact(gpu, ref, prob.K)
