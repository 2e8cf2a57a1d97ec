"""Pins of the differentiation reference (oracle/unrolled.py) and of the
weighted min-sum in the C oracle.

* the unrolled forward (plain PyTorch) equals the C oracle's BP trajectories,
  with the uniform scale and with per-edge per-iteration weights: two
  independent codings of Eqs. 1-3;
* weights equal to alpha everywhere decode exactly as the scale alpha;
* the autograd gradient equals central finite differences at smooth points;
* at T = 1 the gradient equals its closed form, written out per edge.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import unrolled as U  # noqa: E402
from paper_2512_07057_gb300 import workloads as W  # noqa: E402


def _shots(prob, B, tag):
    sh = W.sample_shots(prob, B, tag, keep_errors=True)
    return W.unpack_bits(sh.syndromes, prob.M), W.unpack_bits(sh.errors, prob.N), sh


def _small_problems():
    rng = np.random.default_rng(5)
    p1 = W.random_ldpc(10, 20, 3, 0.08, 3, K=2)
    p1.priors = rng.uniform(0.02, 0.2, size=p1.N)
    return [W.bb72_code_capacity(0.05), W.bb_phenomenological(6, 6, 2, 0.02, 0.02), p1]


@pytest.mark.parametrize("k", range(3))
@pytest.mark.parametrize("weighted", [False, True])
def test_forward_equals_c_oracle(k, weighted):
    """Posterior trajectories of the unrolled forward against the C oracle
    (double build) for T iterations without the stopping rule."""
    prob = _small_problems()[k]
    T = 7
    s, e, _ = _shots(prob, 6, f"unrolled_fwd{k}")
    rng = np.random.default_rng(11 + k)
    if weighted:
        w32 = rng.uniform(0.3, 1.3, size=(T, prob.n_edges)).astype(np.float32)
    else:
        w32 = np.full((T, prob.n_edges), 0.625, np.float32)
    tab = U.Tables(prob)
    _, _, traj = U.unrolled_loss(tab, s, e, torch.tensor(w32.astype(np.float64)), record=True)
    g = oracle.Graph(prob, "f64")
    prm = oracle.Params(weights=w32) if weighted else oracle.Params(ms_scale=0.625)
    for b in range(s.shape[0]):
        ref = g.bp(s[b], T, prm)["llr"]
        np.testing.assert_allclose(traj[:, b, :].numpy(), ref, rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_uniform_weights_decode_as_scale(precision):
    """w_{e,t} = alpha for every edge and iteration is the scale alpha, bit for
    bit, through the whole beam search (one weight row reused for every t)."""
    prob = W.bb72_code_capacity(0.04)
    sh = W.sample_shots(prob, 300, "unrolled_uniform")
    g = oracle.Graph(prob, precision)
    base = dict(max_rounds=4, beam_width=4, initial_iters=12, iters_per_round=6)
    a = g.decode_batch(sh.syndromes, oracle.Params(ms_scale=0.625, **base), nthreads=4)
    for T in (1, 3):
        b = g.decode_batch(sh.syndromes, oracle.Params(weights=np.full((T, prob.n_edges), 0.625, np.float32),
                                                       **base), nthreads=4)
        for key in ("corrections", "status", "iters"):
            assert np.array_equal(a[key], b[key])


def test_weights_row_per_iteration_and_reuse():
    """Iteration t of every BP call uses weight row min(t, T) - 1: a weight
    set whose rows beyond the first equal the scale reproduces a run whose
    first iteration alone differs."""
    prob = W.bb72_code_capacity(0.05)
    s, _, _ = _shots(prob, 3, "unrolled_rows")
    g = oracle.Graph(prob, "f64")
    E = prob.n_edges
    w = np.full((3, E), 0.625, np.float32)
    w[0] = 0.9
    r = g.bp(s[0], 5, oracle.Params(weights=w))["llr"]
    # the same run in two calls: one iteration with 0.9, then four with 0.625
    lam = g.prior_llr()
    col = np.asarray(prob.H_col_idx)
    z = np.zeros(prob.N, np.uint8)
    first = g.masked_bp(np.clip(lam[col], -1e4, 1e4), z, z, s[0], 1, oracle.Params(ms_scale=float(w[0, 0])),
                        stop_on_success=False, record=True)
    rest = g.masked_bp(first["E_out"], z, z, s[0], 4, oracle.Params(ms_scale=0.625), stop_on_success=False,
                       record=True)
    np.testing.assert_array_equal(r[0], first["llr"][0])
    np.testing.assert_array_equal(r[1:], rest["llr"])


@pytest.mark.parametrize("k", range(3))
def test_gradient_equals_finite_differences(k):
    """torch.autograd.gradcheck (central differences, double precision) at a
    point whose distance from every kink is far above the step."""
    prob = _small_problems()[k]
    T = 4
    s, e, _ = _shots(prob, 3, f"unrolled_fd{k}")
    tab = U.Tables(prob)
    rng = np.random.default_rng(100 + k)
    w0 = rng.uniform(0.4, 1.1, size=(T, prob.n_edges))
    gap, amin, lgap = U.kink_margins(tab, s, w0)
    eps = 1e-6
    assert gap > 1e2 * eps and amin > 1e2 * eps and lgap > 1e2 * eps, (gap, amin, lgap)
    w = torch.tensor(w0, requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: U.unrolled_loss(tab, s, e, x)[0], (w,), eps=eps, atol=1e-8,
                                    rtol=1e-5)


def test_gradient_at_one_iteration_closed_form():
    """T = 1: dloss/dw_e = mean-normalised sum over shots of
    (sigmoid(Lam_j(1)) - 1 + e_j) * (-1)^{s_i} * prod sign * min over the other
    edges of |Lambda| -- written out edge by edge from the definitions."""
    prob = W.bb72_code_capacity(0.05)
    s, e, _ = _shots(prob, 4, "unrolled_t1")
    tab = U.Tables(prob)
    rng = np.random.default_rng(7)
    w0 = rng.uniform(0.5, 1.0, size=(1, prob.n_edges))
    _, grad, _, traj = U.unrolled_grad(tab, s, e, w0)
    lam = tab.lam.numpy()
    rp, ci = np.asarray(prob.H_row_ptr), np.asarray(prob.H_col_idx)
    B, N = s.shape[0], prob.N
    want = np.zeros(prob.n_edges)
    for b in range(B):
        post = traj[0, b]
        for i in range(prob.M):
            for ed in range(rp[i], rp[i + 1]):
                j = ci[ed]
                others = [ci[x] for x in range(rp[i], rp[i + 1]) if x != ed]
                mn = min(abs(lam[j2]) for j2 in others) if others else 1e4
                sg = (-1.0) ** s[b, i] * np.prod([(-1.0 if lam[j2] < 0 else 1.0) for j2 in others])
                dpost = 1.0 / (1.0 + np.exp(-post[j])) - 1.0 + e[b, j]
                want[ed] += dpost * sg * mn / (B * N)
    np.testing.assert_allclose(grad[0], want, rtol=1e-10, atol=1e-14)


def test_loss_is_bce_of_posteriors():
    """The loss is the sum over iterations of the mean binary cross entropy
    between sigmoid(-Lam_j(t)) and e_j, evaluated here from the recorded
    posteriors with the textbook formula."""
    prob = W.bb72_code_capacity(0.05)
    s, e, _ = _shots(prob, 5, "unrolled_bce")
    tab = U.Tables(prob)
    w0 = np.full((3, prob.n_edges), 0.7)
    loss, _, per_t, traj = U.unrolled_grad(tab, s, e, w0)
    q = 1.0 / (1.0 + np.exp(traj))                    # sigmoid(-Lam)
    bce = -(e * np.log(q) + (1 - e) * np.log(1 - q))
    np.testing.assert_allclose(per_t, bce.mean(axis=(1, 2)), rtol=1e-12)
    assert abs(loss - per_t.sum()) < 1e-12


def test_iteration_weighted_objective_is_linear_in_the_terms():
    """sum_t c_t L_t: with c = the t-th unit vector the objective is the t-th
    term, and the gradients of the T unit objectives add up to the gradient
    of the plain total (c = all ones)."""
    prob = W.bb72_code_capacity(0.05)
    sh = W.sample_shots(prob, 20, "iter_weights_ref", keep_errors=True)
    s, e = W.unpack_bits(sh.syndromes, prob.M), W.unpack_bits(sh.errors, prob.N)
    T = 4
    w = np.random.default_rng(2).uniform(0.5, 1.0, size=(T, prob.n_edges))
    tab = U.Tables(prob)
    total, g_all, per_t, _ = U.unrolled_grad(tab, s, e, w)
    acc = np.zeros_like(g_all)
    for t in range(T):
        c = np.zeros(T)
        c[t] = 1.0
        lt, gt, _, _ = U.unrolled_grad(tab, s, e, w, iter_weights=c)
        assert abs(lt - per_t[t]) <= 1e-15 * max(1.0, abs(lt))
        acc += gt
    np.testing.assert_allclose(acc, g_all, rtol=1e-10, atol=1e-15)
