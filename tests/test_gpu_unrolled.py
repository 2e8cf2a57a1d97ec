"""The unrolled weighted min-sum kernels (forward, loss, adjoint) against the
double-precision autograd reference of oracle/unrolled.py.

Tolerances (single precision against double):
* posteriors Lambda_j(t): |d| <= 1e-4 max(1, |Lambda|), the LLR bar;
* loss terms: 1e-5 relative;
* weight gradients: |d| <= 1e-4 max|g| + 1e-3 |g| per element.  Rounding
  error of 2^-24 grows by at most a factor ~1.25 per iteration of min-sum,
  so after T = 20 iterations it stays near 1e-5 relative; the bars leave an
  order of magnitude above that.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unrolled as U  # noqa: E402
from paper_2512_07057_gb300 import binding as B  # noqa: E402
from paper_2512_07057_gb300 import decoder as D  # noqa: E402
from paper_2512_07057_gb300 import unrolled as G  # noqa: E402
from paper_2512_07057_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _irregular():
    rng = np.random.default_rng(5)
    p = W.random_ldpc(24, 48, 3, 0.06, 11, K=3)
    p.priors = rng.uniform(0.01, 0.2, size=p.N)
    return p


CASES = {
    # name: (problem, B, T, k) -- ragged batches, one and several 512-shot tiles
    "bb72": (lambda: W.bb72_code_capacity(0.04), 37, 8, 3),
    "phenom_small": (lambda: W.bb_phenomenological(6, 6, 2, 0.02, 0.02), 600, 6, 2),
    "irregular": (_irregular, 129, 5, 5),
    "phenom_12_rounds": (lambda: W.bb_phenomenological(12, 6, 12, 2e-3, 2e-3), 64, 20, 5),
    "single_shot": (lambda: W.bb72_code_capacity(0.06), 1, 4, 3),
}


def _weights(prob, T, seed):
    return np.random.default_rng(seed).uniform(0.5, 1.0, size=(T, prob.n_edges)).astype(np.float32)


def _gpu(prob, Bn, T, k, w, tag):
    s_t, e_t, sh = G.batch_tensors(prob, Bn, tag)
    tr = G.UnrolledTrainer(prob, Bn, T, k)
    wt = torch.from_numpy(w).cuda()
    llr = torch.empty((T, Bn, prob.N), dtype=torch.float32, device="cuda")
    loss = tr.forward(wt, s_t, e_t, llr).cpu().numpy().copy()
    grad = tr.backward(wt, torch.ones(1, device="cuda")).cpu().numpy()
    torch.cuda.synchronize()
    return tr, wt, s_t, e_t, sh, loss, llr.cpu().numpy(), grad


@pytest.mark.parametrize("name", list(CASES))
def test_forward_and_gradient_match_fp64(name):
    build, Bn, T, k = CASES[name]
    prob = build()
    w = _weights(prob, T, 7)
    tr, _, _, _, sh, loss, llr, grad = _gpu(prob, Bn, T, k, w, f"unrolled_{name}")
    s, e = W.unpack_bits(sh.syndromes, prob.M), W.unpack_bits(sh.errors, prob.N)
    rl, rg, rpt, rtraj = U.unrolled_grad(U.Tables(prob), s, e, w.astype(np.float64))
    assert np.all(np.abs(llr - rtraj) <= 1e-4 * np.maximum(1.0, np.abs(rtraj)))
    np.testing.assert_allclose(loss[1:], rpt, rtol=1e-5)
    assert abs(loss[0] - rl) <= 1e-5 * rl
    bar = 1e-4 * np.abs(rg).max() + 1e-3 * np.abs(rg)
    bad = np.abs(grad - rg) > bar
    assert not bad.any(), f"{bad.sum()} of {bad.size} weight gradients off"
    tr.close()


def test_checkpoint_interval_and_determinism():
    """Gradients do not depend on the checkpoint interval (the recomputed
    segments are the forward's own values) and repeat bit for bit."""
    prob = W.bb_phenomenological(6, 6, 3, 0.02, 0.02)
    T = 7
    w = _weights(prob, T, 3)
    grads = []
    for k in (1, 3, 7):
        tr, wt, s_t, e_t, _, _, _, g = _gpu(prob, 300, T, k, w, "unrolled_ckpt")
        grads.append(g)
        tr.forward(wt, s_t, e_t)
        again = tr.backward(wt, torch.ones(1, device="cuda")).cpu().numpy()
        assert np.array_equal(g, again)
        tr.close()
    assert np.array_equal(grads[0], grads[1]) and np.array_equal(grads[0], grads[2])


def test_autograd_function_and_upstream_gradient():
    prob = W.bb72_code_capacity(0.05)
    T, Bn = 6, 200
    tr = G.UnrolledTrainer(prob, Bn, T, 2)
    s_t, e_t, _ = G.batch_tensors(prob, Bn, "unrolled_autograd")
    w = torch.from_numpy(_weights(prob, T, 1)).cuda().requires_grad_(True)
    loss = G.unrolled_loss(w, tr, s_t, e_t)[0]
    (3.0 * loss).backward()
    direct = tr.backward(w.detach(), torch.full((1,), 3.0, device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(w.grad, direct)
    # a second forward invalidates the first one's backward
    loss1 = G.unrolled_loss(w, tr, s_t, e_t)
    G.unrolled_loss(w, tr, s_t, e_t)
    with pytest.raises(RuntimeError):
        loss1[0].backward()
    tr.close()


def test_iteration_weighted_objective_matches_fp64():
    """An objective sum_t c_t L_t (here c_t = t / T, weighting the late
    iterations): the adjoint's weight gradient equals the float64 autograd
    gradient of the same objective, and the autograd function gives the same
    through the loss vector."""
    prob = _irregular()
    T, Bn = 6, 300
    w = _weights(prob, T, 5)
    c = np.arange(1, T + 1, dtype=np.float64) / T
    s_t, e_t, sh = G.batch_tensors(prob, Bn, "unrolled_iter_weights")
    tr = G.UnrolledTrainer(prob, Bn, T, 2)
    wt = torch.from_numpy(w).cuda()
    tr.forward(wt, s_t, e_t)
    g = torch.cat([torch.zeros(1), torch.from_numpy(c.astype(np.float32))]).cuda()
    grad = tr.backward(wt, g).cpu().numpy()
    s, e = W.unpack_bits(sh.syndromes, prob.M), W.unpack_bits(sh.errors, prob.N)
    _, rg, _, _ = U.unrolled_grad(U.Tables(prob), s, e, w.astype(np.float64), iter_weights=c)
    bar = 1e-4 * np.abs(rg).max() + 1e-3 * np.abs(rg)
    assert not (np.abs(grad - rg) > bar).any()
    wa = wt.clone().requires_grad_(True)
    (G.unrolled_loss(wa, tr, s_t, e_t)[1:] * torch.from_numpy(c.astype(np.float32)).cuda()).sum().backward()
    torch.cuda.synchronize()
    assert torch.allclose(wa.grad, torch.from_numpy(grad).cuda(), rtol=1e-6, atol=1e-12)
    tr.close()


def test_directional_derivative_by_central_differences():
    """Along the gradient direction, (L(w + h u) - L(w - h u)) / 2h equals |g|
    for a step far below the distance to the nearest kink's effect."""
    prob = W.bb_phenomenological(6, 6, 2, 0.02, 0.02)
    T, Bn = 6, 512
    tr = G.UnrolledTrainer(prob, Bn, T, 3)
    s_t, e_t, _ = G.batch_tensors(prob, Bn, "unrolled_fd")
    w = torch.from_numpy(_weights(prob, T, 9)).cuda()
    tr.forward(w, s_t, e_t)
    g = tr.backward(w, torch.ones(1, device="cuda"))
    u = g / g.norm()
    h = 1e-2
    lp = float(tr.forward(w + h * u, s_t, e_t)[0])
    lm = float(tr.forward(w - h * u, s_t, e_t)[0])
    fd = (lp - lm) / (2 * h)
    assert abs(fd - float(g.norm())) <= 1e-2 * float(g.norm())
    tr.close()


def test_training_lowers_the_loss():
    prob = W.bb72_code_capacity(0.05)
    _, hist = G.train_weights(prob, T=8, ckpt_every=4, batch=1024, steps=40, lr=2e-2, tag="unrolled_train_test")
    assert np.mean(hist[-5:]) < 0.9 * np.mean(hist[:5])


def test_unrolled_errors():
    prob = W.bb72_code_capacity(0.05)
    d16 = D.BeamSearchDecoder(prob, D.make_params(msg_precision=B.BSD_FP16))
    with pytest.raises(B.BsdError) as ei:
        B.bsd_unrolled_workspace(d16.h, 64, 4, 2)
    assert ei.value.code == B.BSD_ERR_UNSUPPORTED
    d16.close()
    tr = G.UnrolledTrainer(prob, 64, 4, 2)
    with pytest.raises(B.BsdError) as ei:
        B.bsd_unrolled_workspace(tr.dec.h, 64, 4, 5)          # k > T
    assert ei.value.code == B.BSD_ERR_INVALID_ARG
    s_t, e_t, _ = G.batch_tensors(prob, 64, "unrolled_err")
    w = torch.full((4, prob.n_edges), 0.6, device="cuda")
    import ctypes as C
    with pytest.raises(B.BsdError) as ei:                     # workspace one byte short
        B.bsd_unrolled_forward(tr.dec.h, C.c_void_p(s_t.data_ptr()), C.c_void_p(e_t.data_ptr()), 64, 4, 2,
                               C.c_void_p(w.data_ptr()), C.c_void_p(tr.loss.data_ptr()), None,
                               C.c_void_p(tr.work.data_ptr()), tr.work.numel() - 1, None)
    assert ei.value.code == B.BSD_ERR_INVALID_ARG
    tr.close()


def test_full_size_training_batch():
    """The benchmark's training configuration (phenomenological DEM, B = 4096,
    T = 20, k = 5): posteriors of 12 sampled shots against the float64
    reference run on those shots alone, the gradient's additivity over two
    half batches (each term is a sum over shots), and central differences of
    the loss along the gradient."""
    prob = W.bb_phenomenological(12, 6, 12, 2e-3, 2e-3)
    Bn, T, k = 4096, 20, 5
    s_t, e_t, sh = G.batch_tensors(prob, Bn, W.shot_seed("unrolled_full_size", 0))
    w = torch.from_numpy(_weights(prob, T, 21)).cuda()
    tr = G.UnrolledTrainer(prob, Bn, T, k)
    llr = torch.empty((T, Bn, prob.N), dtype=torch.float32, device="cuda")
    tr.forward(w, s_t, e_t, llr)
    g = tr.backward(w, torch.ones(1, device="cuda"))
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(4).choice(Bn, size=12, replace=False))
    s = W.unpack_bits(sh.syndromes[idx], prob.M)
    e = W.unpack_bits(sh.errors[idx], prob.N)
    _, _, _, rtraj = U.unrolled_grad(U.Tables(prob), s, e, w.cpu().numpy().astype(np.float64))
    got = llr[:, torch.as_tensor(idx, device="cuda"), :].cpu().numpy()
    assert np.all(np.abs(got - rtraj) <= 1e-4 * np.maximum(1.0, np.abs(rtraj)))
    # additivity: the full-batch gradient is the mean of the two half-batch gradients
    half = []
    for lo in (0, Bn // 2):
        th = G.UnrolledTrainer(prob, Bn // 2, T, k)
        th.forward(w, s_t[lo:lo + Bn // 2].contiguous(), e_t[lo:lo + Bn // 2].contiguous())
        half.append(th.backward(w, torch.ones(1, device="cuda")))
        th.close()
    gh = 0.5 * (half[0] + half[1])
    assert float((g - gh).abs().max()) <= 1e-5 * float(g.abs().max())
    # central differences along the gradient
    u = g / g.norm()
    hstep = 1e-2
    lp = float(tr.forward(w + hstep * u, s_t, e_t)[0])
    lm = float(tr.forward(w - hstep * u, s_t, e_t)[0])
    assert abs((lp - lm) / (2 * hstep) - float(g.norm())) <= 2e-2 * float(g.norm())
    tr.close()
