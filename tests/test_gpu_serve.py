"""The single-syndrome request loop (bsd_serve_*): a resident candidate group
answers syndromes posted in host-mapped memory.  Every answer must equal the
regular path's (bsd_decode_host) bit for bit: corrections, observable flips,
status and iteration counts -- for syndromes the loop answers itself (the
seed BP ends the search) and for those it hands to the regular path (the
beam search decides)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2512_07057_gb300 import binding as B  # noqa: E402
from paper_2512_07057_gb300 import decoder as D  # noqa: E402
from paper_2512_07057_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _cases():
    return [
        ("bb144_p0.03", W.bb144_code_capacity(0.03), dict(preset="beam32_340iters", ms_scale=0.625), 600),
        ("bb72_p0.05", W.bb72_code_capacity(0.05), dict(preset="beam8_230iters", ms_scale=0.625), 400),
        ("phen_p0.003", W.bb_phenomenological(12, 6, 12, 3e-3, 3e-3),
         dict(preset="beam32_340iters", ms_scale=0.625), 300),
        ("phen_fp16", W.bb_phenomenological(12, 6, 12, 3e-3, 3e-3),
         dict(preset="beam32_340iters", ms_scale=0.625, msg_precision=B.BSD_FP16), 300),
    ]


def _params(kw):
    kw = dict(kw)
    preset = kw.pop("preset")
    return D.make_params(preset, workspace_bytes=1 << 30, **kw)


@pytest.mark.parametrize("name,prob,kw,n", _cases(), ids=[c[0] for c in _cases()])
def test_answers_equal_the_regular_path(name, prob, kw, n):
    shots = W.sample_shots(prob, n, f"serve_{name}")
    dec = D.BeamSearchDecoder(prob, _params(kw))
    ref = dec.decode_host(shots.syndromes)
    dec.serve_start(idle_ms=1000)
    got = [dec.serve_decode(shots.syndromes[i]) for i in range(shots.B)]
    dec.serve_stop()
    dec.close()
    corr = np.stack([g["corrections"] for g in got])
    obs = np.stack([g["obs"] for g in got])
    status = np.array([g["status"] for g in got], np.uint32)
    iters = np.array([g["iters"] for g in got], np.uint32)
    assert np.array_equal(corr, ref["corrections"])
    assert np.array_equal(obs[:, :ref["obs"].shape[1]], ref["obs"])
    assert np.array_equal(status, ref["status"])
    assert np.array_equal(iters, ref["iters"])
    # both kinds of answer occurred: the loop's own and the regular path's
    assert (status == B.BSD_STATUS_CONVERGED_SEED).any()
    if name.startswith("bb144") or name.startswith("bb72"):
        assert (status != B.BSD_STATUS_CONVERGED_SEED).any()


def test_idle_exit_and_restart():
    """A loop that leaves after its idle limit is started again by the next
    request; answers stay exact."""
    prob = W.bb72_code_capacity(0.05)
    shots = W.sample_shots(prob, 40, "serve_idle")
    dec = D.BeamSearchDecoder(prob, _params(dict(preset="beam8_230iters", ms_scale=0.625)))
    ref = dec.decode_host(shots.syndromes)
    dec.serve_start(idle_ms=2)
    for i in range(shots.B):
        if i % 4 == 0:
            time.sleep(0.02)                      # well past the 2 ms idle limit
        g = dec.serve_decode(shots.syndromes[i])
        assert np.array_equal(g["corrections"], ref["corrections"][i])
        assert g["status"] == ref["status"][i] and g["iters"] == ref["iters"][i]
    dec.serve_stop()
    dec.close()


def test_stop_start_and_close_while_serving():
    prob = W.bb72_code_capacity(0.05)
    shots = W.sample_shots(prob, 8, "serve_stop")
    dec = D.BeamSearchDecoder(prob, _params(dict(preset="beam8_230iters", ms_scale=0.625)))
    ref = dec.decode_host(shots.syndromes)
    dec.serve_start(idle_ms=500)
    dec.serve_start(idle_ms=500)                 # already serving: no-op
    dec.serve_stop()
    dec.serve_stop()                             # not serving: no-op
    with pytest.raises(B.BsdError) as ei:
        dec.serve_decode(shots.syndromes[0])       # not serving
    assert ei.value.code == B.BSD_ERR_INVALID_ARG
    dec.serve_start(idle_ms=500)
    g = dec.serve_decode(shots.syndromes[3])
    assert np.array_equal(g["corrections"], ref["corrections"][3])
    dec.close()                                  # stops the loop first


def test_regular_decodes_run_beside_the_loop():
    """While the loop is resident, a batch decode on another stream runs and
    matches its own earlier result; the loop keeps answering afterwards."""
    prob = W.bb144_code_capacity(0.03)
    shots = W.sample_shots(prob, 4000, "serve_beside")
    dec = D.BeamSearchDecoder(prob, _params(dict(preset="beam32_340iters", ms_scale=0.625)))
    synd = D.to_torch_words(shots.syndromes)
    first = dec.decode(synd)
    torch.cuda.synchronize()
    want = D.from_torch_words(first.corrections).copy()
    dec.serve_start(idle_ms=2000)
    # (a device-wide synchronize would wait for the resident loop until its
    # idle limit: wait for this stream only)
    again = dec.decode(synd)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(D.from_torch_words(again.corrections), want)
    ref = dec.decode_host(shots.syndromes[:16])
    for i in range(16):
        assert np.array_equal(dec.serve_decode(shots.syndromes[i])["corrections"], ref["corrections"][i])
    dec.serve_stop()
    dec.close()


def test_set_weights_stops_the_loop():
    prob = W.bb72_code_capacity(0.05)
    dec = D.BeamSearchDecoder(prob, _params(dict(preset="beam8_230iters", ms_scale=0.625)))
    dec.serve_start(idle_ms=500)
    dec.set_weights(np.full((2, prob.n_edges), 0.625, np.float32))
    with pytest.raises(B.BsdError):
        dec.serve_decode(np.zeros((prob.M + 31) // 32, np.uint32))
    dec.close()
