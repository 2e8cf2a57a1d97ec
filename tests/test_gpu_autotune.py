"""The launch-shape autotuner: every shape it times decodes identically, and
it keeps the fastest one it timed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2512_07057_gb300 import decoder as D  # noqa: E402
from paper_2512_07057_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["bb144", "phenom"])
def test_autotune_keeps_results_and_the_fastest_shape(name):
    if name == "bb144":
        prob, params = W.bb144_code_capacity(0.05), D.make_params("beam32_340iters", ms_scale=0.625)
    else:
        prob = W.bb_phenomenological(12, 6, 12, 3e-3, 3e-3)
        params = D.make_params("beam64_640iters", ms_scale=0.625, workspace_bytes=2 << 30)
    shots = W.sample_shots(prob, 8192, f"autotune_{name}")
    s = D.to_torch_words(shots.syndromes)
    dec = D.BeamSearchDecoder(prob, params)
    before = dec.decode(s)
    torch.cuda.synchronize()
    before = {a: D.from_torch_words(getattr(before, a)).copy() for a in ("corrections", "status", "iters")}
    report = dec.autotune(s)
    assert len(report) >= 4                      # warp shapes and block shapes were timed
    assert any(gw >= 2 for gw, _, _ in report) and any(gw == 1 for gw, _, _ in report)
    best = min(report, key=lambda r: r[2])
    assert dec.shape == (best[0], best[1])
    after = dec.decode(s)
    torch.cuda.synchronize()
    for a in ("corrections", "status", "iters"):
        assert np.array_equal(D.from_torch_words(getattr(after, a)), before[a])
    # weights keep the tuned shape
    dec.set_weights(np.full((2, prob.n_edges), 0.625, np.float32))
    assert dec.shape == (best[0], best[1])
    dec.close()


def test_small_chunk_graph_changes_nothing():
    """Chunks of a few shots run a graph with grids sized to them; outputs equal
    the full-grid graph's, for one shot at a time and for a small batch."""
    prob = W.bb144_code_capacity(0.05)
    shots = W.sample_shots(prob, 40, "small_graph")
    s = D.to_torch_words(shots.syndromes)
    res = {}
    for sb in (0, -1):
        dec = D.BeamSearchDecoder(prob, D.make_params("beam32_340iters", ms_scale=0.625, small_batch=sb))
        batch = dec.decode(s[:20])
        single = [dec.decode(s[i:i + 1]) for i in range(20, 40)]
        torch.cuda.synchronize()
        res[sb] = (D.from_torch_words(batch.corrections).copy(), D.from_torch_words(batch.status).copy(),
                   np.concatenate([D.from_torch_words(o.corrections) for o in single]),
                   np.concatenate([D.from_torch_words(o.status) for o in single]))
        dec.close()
    for a, b in zip(res[0], res[-1]):
        assert np.array_equal(a, b)


def test_graph_runs_only_the_rounds_a_chunk_needs():
    """Kernels launched per chunk, counted on the device: a chunk whose shots all
    converge in the seed runs 3 (chunk set-up, seed, pass gate); one that needs
    beam rounds adds the round loop of one pass (start, 3 per round, pass end)
    and no round beyond the last one with children."""
    prob = W.bb144_code_capacity(0.05)
    dec = D.BeamSearchDecoder(prob, D.make_params("beam32_340iters", ms_scale=0.625))
    zero = torch.zeros((64, 3), dtype=torch.int32, device="cuda")
    dec.profile_read()
    dec.decode(zero)
    torch.cuda.synchronize()
    assert dec.profile_read()["kernel_launches"] == 3
    # shots that need rounds: the maximum round any shot reaches bounds the loop
    shots = W.sample_shots(prob, 2000, "graph_rounds")
    out = dec.decode(D.to_torch_words(shots.syndromes))
    torch.cuda.synchronize()
    launches = dec.profile_read()["kernel_launches"]
    st = D.from_torch_words(out.status)
    assert (st & 7 == 2).any()                       # some shots converged in a beam round
    rounds = (launches - 3 - 2) // 3
    assert launches == 3 + 1 + 3 * rounds + 1 and 1 <= rounds <= 10
    dec.close()


@pytest.mark.parametrize("gw", [1, 8])
def test_screen_kernel_runs_before_the_seed_on_dems(gw):
    """A generic-engine decoder with every Lambda_j > 0 and one result runs the
    first-iteration screen before the seed BP: 4 kernels for a seed-only chunk
    (set-up, screen, seed, pass gate).  With per-edge weights the screen is
    off (3 kernels), and so it is with two results (shown without beam
    rounds: set-up and seed only)."""
    prob = W.bb_phenomenological(6, 6, 3, 0.01, 0.01)
    zero = torch.zeros((64, (prob.M + 31) // 32), dtype=torch.int32, device="cuda")
    for nr, rounds, weights, want in ((1, 3, False, 4), (1, 3, True, 3), (2, 0, False, 2), (1, 0, False, 3)):
        dec = D.BeamSearchDecoder(prob, D.make_params(max_rounds=rounds, beam_width=4, initial_iters=10,
                                                      iters_per_round=5, num_results=nr, ms_scale=0.625,
                                                      group_warps=gw))
        if weights:
            dec.set_weights(np.full((2, prob.n_edges), 0.625, np.float32))
        dec.profile_read()
        out = dec.decode(zero)
        torch.cuda.synchronize()
        assert dec.profile_read()["kernel_launches"] == want, (nr, rounds, weights)
        assert np.all(D.from_torch_words(out.status) == 1)
        assert not D.from_torch_words(out.corrections).any()
        dec.close()
