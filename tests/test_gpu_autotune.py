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
