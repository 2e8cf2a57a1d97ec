"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test names the passage it checks.  None of them re-derives the oracle's
own formulas: they use closed forms (min-sum is exact on cycle-free graphs),
hand-worked examples (tests/golden), brute force over all error vectors,
reductions to a simpler problem, library routines (numpy stable sort) and
invariants (H e = s).
"""
import itertools
import json
import os

import numpy as np
import pytest

from paper_2512_07057_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _dense_problem(H, priors, A=None):
    H = np.asarray(H, np.uint8)
    if A is None:
        A = np.eye(H.shape[1], dtype=np.uint8)[:1]
    return W.problem_from_dense(H, A, priors)


# ----------------------------------------------------------------------------
# Table I
# ----------------------------------------------------------------------------
def test_presets_match_table1(oracle_mod):
    g = _golden("table1_presets.json")
    for name, vals in g["presets"].items():
        assert list(oracle_mod.PRESETS[name]) == vals
        mr, bw, ii, ipr, nr = vals
        # the iteration count in the name = initial_iters + max_rounds * iters_per_round
        assert int(name.split("_")[-1].replace("iters", "")) == ii + mr * ipr


# ----------------------------------------------------------------------------
# Eqs. 1-4 on a hand-worked example
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_repetition3_hand_worked(oracle_mod, precision):
    g = _golden("repetition3.json")
    pr = g["problem"]
    prob = _dense_problem(pr["H"], [pr["p"]] * 3)
    G = oracle_mod.Graph(prob, precision)
    lam = np.log(0.9 / 0.1)
    tol = 1e-12 if precision == "f64" else 1e-6
    for key, alpha in (("alpha_1", 1.0), ("alpha_0.625", 0.625)):
        exp = g["expected"][key]
        prm = oracle_mod.Params(ms_scale=alpha)
        r = G.bp(pr["syndrome"], len(exp["llr_over_Lambda"]), prm, stop_on_success=False)
        assert np.allclose(r["llr"] / lam, np.array(exp["llr_over_Lambda"]), atol=tol)
        r2 = G.bp(pr["syndrome"], 10, prm, stop_on_success=True)
        assert r2["iters"] == exp["stop_iter"] and r2["success"]
        assert list(r2["ehat"]) == exp["ehat"]


# ----------------------------------------------------------------------------
# Alg. 2 / Alg. 3 on a hand-worked example
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_single_check_beam_hand_worked(oracle_mod, precision):
    g = _golden("single_check_beam.json")
    pr = g["problem"]
    prob = _dense_problem(pr["H"], pr["p"])
    G = oracle_mod.Graph(prob, precision)
    q = pr["params"]
    for key, nres in (("num_results_1", 1), ("num_results_2", 2)):
        prm = oracle_mod.Params(max_rounds=q["max_rounds"], beam_width=q["beam_width"],
                                initial_iters=q["initial_iters"], iters_per_round=q["iters_per_round"],
                                num_results=nres, ms_scale=q["alpha"], llr_clamp=q["llr_clamp"])
        r = G.decode_one(np.array(pr["syndrome"]), prm)
        exp = g["expected"][key]
        assert list(r["ehat"]) == exp["ehat"]
        assert r["status"] == oracle_mod.STATUS_BEAM
        assert r["iters"] == exp["iters"]
        assert r["trace"]["seed_next_pos"] == 0 and r["trace"]["seed_success"] == 0


# ----------------------------------------------------------------------------
# Tree closed form: min-sum (alpha = 1) is exact min-cost on cycle-free graphs
# ----------------------------------------------------------------------------
def _random_tree(rng, n_vars):
    """Bipartite tree: every check is created with 2-4 variable neighbours."""
    edges = []              # (check, var)
    nv, nc = 1, 0
    while nv < n_vars:
        anchor = int(rng.integers(nv))
        c = nc
        nc += 1
        edges.append((c, anchor))
        k = int(min(rng.integers(1, 4), n_vars - nv))
        for _ in range(k):
            edges.append((c, nv))
            nv += 1
    H = np.zeros((nc, nv), np.uint8)
    for c, v in edges:
        H[c, v] = 1
    return H


def _brute_min_marginals(H, lam, s):
    N = H.shape[1]
    E = np.array(list(itertools.product([0, 1], repeat=N)), dtype=np.uint8)
    ok = ((E.astype(int) @ H.T) % 2 == s).all(1)
    E = E[ok]
    cost = E @ lam
    W1 = np.array([cost[E[:, j] == 1].min() for j in range(N)])
    W0 = np.array([cost[E[:, j] == 0].min() for j in range(N)])
    return W1 - W0


@pytest.mark.parametrize("seed", range(12))
def test_tree_closed_form(oracle_mod, seed):
    """On a Tanner tree, Eq. 3 after enough iterations equals W_j(1) - W_j(0),
    W_j(v) = min{wt(e) : H e = s, e_j = v}, wt(e) = sum_j e_j Lambda_j."""
    rng = np.random.default_rng(seed)
    H = _random_tree(rng, int(rng.integers(5, 14)))
    M, N = H.shape
    p = rng.uniform(0.05, 0.45, size=N)
    lam = np.log((1 - p) / p)
    e = (rng.random(N) < 0.3).astype(np.uint8)
    s = (H.astype(int) @ e) % 2
    prob = _dense_problem(H, p)
    G = oracle_mod.Graph(prob, "f64")
    T = 2 * (M + N) + 2
    r = G.bp(s, T, oracle_mod.Params(ms_scale=1.0), stop_on_success=False)
    exact = _brute_min_marginals(H, lam, s)
    got = r["llr"][-1]
    assert np.allclose(got, exact, rtol=1e-9, atol=1e-9), (got, exact)
    # the hard decision of an exact, tie-free min-marginal is a min-weight solution
    if np.all(np.abs(exact) > 1e-9):
        eh = (got <= 0).astype(np.uint8)
        assert ((H.astype(int) @ eh) % 2 == s).all()


# ----------------------------------------------------------------------------
# Masked BP reduces to plain BP on the column-deleted problem (Alg. 2, App. B)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(10))
def test_masked_bp_equals_reduced_problem(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    prob = W.random_ldpc(8, 16, 3, 0.08, seed)
    H = prob.H_dense()
    M, N = H.shape
    prob.priors = rng.uniform(0.02, 0.3, size=N)
    G = oracle_mod.Graph(prob, "f64")
    prm = oracle_mod.Params(ms_scale=0.625)
    masked = np.zeros(N, np.uint8)
    masked[rng.choice(N, size=int(rng.integers(1, 5)), replace=False)] = 1
    val = (rng.random(N) < 0.5).astype(np.uint8) * masked
    s = rng.integers(0, 2, size=M).astype(np.uint8)
    E0 = rng.normal(0, 3, size=G.E)
    full = G.masked_bp(E0, masked, val, s, 15, prm, stop_on_success=False, record=True)
    # reduced problem: delete masked columns, fold their values into the syndrome
    keep = np.nonzero(masked == 0)[0]
    Hr = H[:, keep]
    sr = (s + H[:, masked == 1].astype(int) @ val[masked == 1]) % 2
    red = W.problem_from_dense(Hr, np.zeros((1, len(keep)), np.uint8), prob.priors[keep])
    Gr = oracle_mod.Graph(red, "f64")
    # edge messages of kept edges, in the reduced CSR order (rows ascending, columns ascending)
    E0r = []
    for i in range(M):
        for e in range(prob.H_row_ptr[i], prob.H_row_ptr[i + 1]):
            if masked[prob.H_col_idx[e]] == 0:
                E0r.append(E0[e])
    z = np.zeros(len(keep), np.uint8)
    rr = Gr.masked_bp(np.array(E0r), z, z, sr, 15, prm, stop_on_success=False, record=True)
    assert np.array_equal(full["llr"][:, keep], rr["llr"])
    assert np.array_equal(full["ehat"][keep], rr["ehat"])
    assert np.array_equal(full["ehat"][masked == 1], val[masked == 1])
    assert full["first_success"] == rr["first_success"]


# ----------------------------------------------------------------------------
# Exhaustive beam search returns a minimum-weight solution
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(6))
def test_unpruned_full_depth_search_is_min_weight(oracle_mod, seed):
    """With beam_width >= 2^max_rounds (no pruning), max_rounds = N (every
    node fixed along every path) and num_results above the number of
    solutions, Alg. 3 visits every assignment and returns min wt(e) over
    {e : H e = s} (App. B weight)."""
    rng = np.random.default_rng(200 + seed)
    N = 9
    prob = W.random_ldpc(5, N, 2, 0.1, seed)
    p = rng.uniform(0.03, 0.3, size=N)
    prob.priors = p
    H = prob.H_dense()
    lam = np.log((1 - p) / p)
    G = oracle_mod.Graph(prob, "f64")
    prm = oracle_mod.Params(max_rounds=N, beam_width=2 ** N, initial_iters=3, iters_per_round=2,
                            num_results=2 ** N + 1, ms_scale=0.625)
    allE = np.array(list(itertools.product([0, 1], repeat=N)), dtype=np.uint8)
    for _ in range(3):
        e = (rng.random(N) < 0.25).astype(np.uint8)
        s = (H.astype(int) @ e) % 2
        r = G.decode_one(s, prm, trace_cap=1 << 12)
        assert r["status"] in (oracle_mod.STATUS_SEED, oracle_mod.STATUS_BEAM)
        eh = r["ehat"]
        assert ((H.astype(int) @ eh) % 2 == s).all()
        ok = ((allE.astype(int) @ H.T) % 2 == s).all(1)
        best = (allE[ok] @ lam).min()
        assert abs(float(eh @ lam) - best) < 1e-9


# ----------------------------------------------------------------------------
# Scores, next_pos and the failure fallback in closed form
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_score_and_next_pos_closed_form(oracle_mod, precision):
    """A problem that never converges (a detector with no error source and
    s = 1) whose posterior LLRs are constant in t: a pair of nodes on one
    check with s = 0 (alpha = 1: Lambda_{0,1}(t) = Lambda_0 + Lambda_1) and
    isolated nodes (Lambda_j(t) = Lambda_j).  Then sum_LLR[j] = iters * c_j,
    every child's score is sum_{j in U} |c_j| (Alg. 3: normalised by iters),
    and next_pos walks the nodes in ascending |c_j| (lowest index on ties)."""
    p = np.array([0.3, 0.35, 0.2, 0.45, 0.1, 0.4])
    lam = np.log((1 - p) / p)
    H = np.zeros((2, 6), np.uint8)
    H[0, 0] = H[0, 1] = 1
    prob = _dense_problem(H, p)
    G = oracle_mod.Graph(prob, precision)
    c = lam.copy()
    c[0] = c[1] = lam[0] + lam[1]
    prm = oracle_mod.Params(max_rounds=3, beam_width=3, initial_iters=4, iters_per_round=3,
                            num_results=1, ms_scale=1.0)
    r = G.decode_one(np.array([0, 1]), prm)
    tr = r["trace"]
    order = sorted(range(6), key=lambda j: (abs(c[j]), j))
    tol = 1e-12 if precision == "f64" else 1e-4
    assert tr["seed_next_pos"] == order[0]
    assert r["status"] == oracle_mod.STATUS_FAILED
    assert r["iters"] == 4 + 3 * (2 + 4 + 6)        # children per round 2, 4, then 2*3 after pruning
    for k in range(len(tr["round"])):
        rd = tr["round"][k]
        U = [j for j in range(6) if j not in order[:rd]]
        assert abs(tr["score"][k] - sum(abs(c[j]) for j in U)) <= tol * max(1, abs(tr["score"][k]))
        assert tr["next_pos"][k] == order[rd]
        assert tr["iters"][k] == 3
    # all scores tie, so pruning keeps canonical order; the fallback is the
    # rank-0 path of the last set: all fixed values 0 and every c_j > 0
    assert list(r["ehat"]) == [0] * 6


# ----------------------------------------------------------------------------
# Pruning: bounded insert (App. B) == stable sort then keep beam_width
# ----------------------------------------------------------------------------
def _bb_shots(p, B, tag):
    prob = W.bb72_code_capacity(p)
    return prob, W.sample_shots(prob, B, tag)


def test_pruning_is_stable_top_w(oracle_mod):
    prob, sh = _bb_shots(0.06, 300, "prune_test")
    G = oracle_mod.Graph(prob, "f64")
    prm = oracle_mod.Params(max_rounds=6, beam_width=4, initial_iters=10, iters_per_round=6,
                            num_results=3, ms_scale=0.625)
    s_all = W.unpack_bits(sh.syndromes, prob.M)
    checked = 0
    for b in range(sh.B):
        r = G.decode_one(s_all[b], prm)
        tr = r["trace"]
        for rd in np.unique(tr["round"]):
            idx = np.nonzero(tr["round"] == rd)[0]
            if rd == tr["ret_round"] or len(idx) == 0:
                continue                                 # stopped early: no pruning took place
            sc = tr["score"][idx]
            # numpy stable sort on (-score); ties keep canonical (visit) order
            order = np.argsort(-sc, kind="stable")
            kept = tr["kept"][idx]
            exp = np.full(len(idx), -1)
            exp[order[:prm.beam_width]] = np.arange(min(prm.beam_width, len(idx)))
            assert np.array_equal(kept, exp)
            # the next round visits parents in that rank order, val 0 then 1
            nxt = np.nonzero(tr["round"] == rd + 1)[0]
            if len(nxt):
                assert np.all(np.diff(tr["canon"][nxt]) > 0)
                assert np.array_equal(tr["canon"][nxt], 2 * tr["parent_rank"][nxt] + tr["val"][nxt])
                # a child branches on its parent's next_pos
                for k in nxt:
                    par = idx[kept == tr["parent_rank"][k]]
                    assert len(par) == 1 and tr["pos"][k] == tr["next_pos"][par[0]]
            checked += 1
    assert checked > 20


@pytest.mark.parametrize("nres", [1, 4])
def test_bounded_insert_equals_collect_then_prune(oracle_mod, nres):
    prob, sh = _bb_shots(0.06, 600, "prune_modes")
    G = oracle_mod.Graph(prob, "f64")
    base = dict(max_rounds=8, beam_width=4, initial_iters=12, iters_per_round=8, num_results=nres,
                ms_scale=0.625)
    a = G.decode_batch(sh.syndromes, oracle_mod.Params(prune_mode=0, **base), nthreads=4)
    b = G.decode_batch(sh.syndromes, oracle_mod.Params(prune_mode=1, **base), nthreads=4)
    for k in ("corrections", "obs", "status", "iters"):
        assert np.array_equal(a[k], b[k]), k


# ----------------------------------------------------------------------------
# Invariants and library reductions on real workloads
# ----------------------------------------------------------------------------
def test_outputs_satisfy_syndrome_and_observables(oracle_mod):
    prob, sh = _bb_shots(0.05, 1500, "invariants")
    G = oracle_mod.Graph(prob, "f64")
    prm = oracle_mod.Params(max_rounds=10, beam_width=8, initial_iters=30, iters_per_round=20,
                            ms_scale=0.625)
    r = G.decode_batch(sh.syndromes, prm, nthreads=4)
    e = W.unpack_bits(r["corrections"], prob.N).astype(int)
    s = W.unpack_bits(sh.syndromes, prob.M)
    conv = r["status"] != oracle_mod.STATUS_FAILED
    assert conv.mean() > 0.9
    assert np.array_equal(((e @ prob.H_dense().T) % 2)[conv], s[conv])            # H e = s
    assert np.array_equal(W.unpack_bits(r["obs"], prob.K), (e @ prob.A_dense().T) % 2)  # A e
    # seed-converged shots: the algorithmic iteration count is the seed's stop time
    seed = r["status"] == oracle_mod.STATUS_SEED
    assert (r["iters"][seed] <= 30).all() and (r["iters"][~seed & conv] > 30).all()


def test_zero_syndrome_converges_at_first_iteration(oracle_mod):
    """s = 0 and every p_j < 1/2: D > 0 everywhere at t = 1, Lambda_j(1) > 0,
    e(1) = 0 and H e(1) = s (Eqs. 1-4), so the seed returns 0 after 1 iteration."""
    prob = W.bb144_code_capacity(0.03)
    G = oracle_mod.Graph(prob, "f64")
    r = G.decode_batch(np.zeros((3, 3), np.uint32), oracle_mod.preset("beam32_340iters", ms_scale=0.625))
    assert (r["status"] == 1).all() and (r["iters"] == 1).all() and (r["corrections"] == 0).all()


def test_ml_bounds_on_tiny_code(oracle_mod):
    """LER(ML) <= LER(beam) <= LER(plain BP) on the smallest BB-family code
    here (l = m = 3, N = 18), ML by enumerating the solution space."""
    prob = W.bb_code_capacity(3, 3, 0.08)
    assert prob.K > 0
    H, A = prob.H_dense(), prob.A_dense()
    sh = W.sample_shots(prob, 3000, "ml_bounds", keep_errors=True)
    G = oracle_mod.Graph(prob, "f64")
    beam = G.decode_batch(sh.syndromes, oracle_mod.Params(max_rounds=10, beam_width=16, initial_iters=20,
                                                          iters_per_round=10, ms_scale=0.625), nthreads=4)
    plain = G.decode_batch(sh.syndromes, oracle_mod.Params(max_rounds=0, beam_width=1, initial_iters=50,
                                                           iters_per_round=1, ms_scale=0.625), nthreads=4)
    obs_true = W.unpack_bits(sh.obs, prob.K)

    def ler(r):
        o = W.unpack_bits(r["obs"], prob.K)
        return float(((o != obs_true).any(1) | (r["status"] == 4)).mean())

    # ML: pick the observable class of largest total probability
    N = prob.N
    allE = np.array(list(itertools.product([0, 1], repeat=N)), dtype=np.uint8)
    synd = (allE.astype(np.int64) @ H.T) % 2
    skey = synd @ (1 << np.arange(H.shape[0]))
    okey = ((allE.astype(np.int64) @ A.T) % 2) @ (1 << np.arange(A.shape[0]))
    wt = allE.sum(1)
    pr = (0.08 ** wt) * (0.92 ** (N - wt))
    s_all = W.unpack_bits(sh.syndromes, prob.M).astype(np.int64) @ (1 << np.arange(H.shape[0]))
    o_all = obs_true.astype(np.int64) @ (1 << np.arange(A.shape[0]))
    ml_fail = 0
    table = {}
    for sk in np.unique(s_all):
        sel = skey == sk
        classes = {}
        for ok_, p_ in zip(okey[sel], pr[sel]):
            classes[ok_] = classes.get(ok_, 0.0) + p_
        table[sk] = max(classes, key=classes.get)
    for sk, ok_ in zip(s_all, o_all):
        ml_fail += table[sk] != ok_
    ler_ml = ml_fail / sh.B
    ler_beam, ler_plain = ler(beam), ler(plain)
    sd = np.sqrt(0.25 / sh.B)
    assert ler_ml <= ler_beam + 3 * sd
    assert ler_beam <= ler_plain + 3 * sd


def test_fp32_build_tracks_fp64(oracle_mod):
    """The single-precision build follows the double one: LLR trajectories
    within 1e-4 relative, and identical decisions on a BB workload sample."""
    prob, sh = _bb_shots(0.03, 1000, "fp32_vs_fp64")
    g64, g32 = oracle_mod.Graph(prob, "f64"), oracle_mod.Graph(prob, "f32")
    prm = oracle_mod.Params(max_rounds=10, beam_width=8, initial_iters=50, iters_per_round=20, ms_scale=0.625)
    s_all = W.unpack_bits(sh.syndromes, prob.M)
    for b in range(40):
        a = g64.bp(s_all[b], 30, prm)["llr"]
        c = g32.bp(s_all[b], 30, prm)["llr"].astype(np.float64)
        assert np.all(np.abs(a - c) <= 1e-4 * np.maximum(1.0, np.abs(a)))
    r64 = g64.decode_batch(sh.syndromes, prm, nthreads=4)
    r32 = g32.decode_batch(sh.syndromes, prm, nthreads=4)
    diff = (r64["corrections"] != r32["corrections"]).any(1) | (r64["status"] != r32["status"])
    # any disagreement must sit on a logged near-tie or exact tie of the double build
    assert np.all((r64["min_gap"][diff] < 1e-4) | (r64["ties"][diff] > 0))
    assert diff.sum() <= 2


# ----------------------------------------------------------------------------
# 16-bit message storage: rounding pinned to library conversions
# ----------------------------------------------------------------------------
def _rounding_cases():
    rng = np.random.default_rng(7)
    x = np.concatenate([
        rng.normal(0, 1, 20000), rng.normal(0, 3000, 20000), rng.uniform(-1e-4, 1e-4, 20000),
        rng.uniform(-1e-7, 1e-7, 5000), np.array([0.0, -0.0, 1e4, -1e4, 65504.0, 65519.0, 2049.0, 2051.0,
                                                  6.103515625e-05, 5.9604644775390625e-08, 1.5 * 2 ** -24])])
    # exact binary16 / bfloat16 halfway points
    h = np.float16(rng.normal(0, 100, 5000)).astype(np.float32)
    halves = (h + np.nextafter(h, np.float32(np.inf)).astype(np.float32)) / 2
    return np.concatenate([x.astype(np.float32), halves]).astype(np.float32)


def test_binary16_rounding_matches_numpy(oracle_mod):
    x = _rounding_cases()
    got = oracle_mod.round_storage(x, 1)
    exp = x.astype(np.float16).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), exp.view(np.uint32))


def test_bfloat16_rounding_matches_torch(oracle_mod):
    torch = pytest.importorskip("torch")
    x = _rounding_cases()
    got = oracle_mod.round_storage(x, 2)
    exp = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(got.view(np.uint32), exp.view(np.uint32))


@pytest.mark.parametrize("mode,tol", [(1, 5e-3), (2, 5e-2)])
def test_16bit_storage_tracks_double(oracle_mod, mode, tol):
    """Messages stored in 16 bits, arithmetic in single precision: the seed
    BP's LLRs stay close to double precision (binary16 keeps 11 significant
    bits, bfloat16 8)."""
    prob, sh = _bb_shots(0.03, 200, "storage16")
    g64, g32 = oracle_mod.Graph(prob, "f64"), oracle_mod.Graph(prob, "f32")
    prm64 = oracle_mod.Params(ms_scale=0.625)
    prm16 = oracle_mod.Params(ms_scale=0.625, msg_storage=mode)
    s_all = W.unpack_bits(sh.syndromes, prob.M)
    med = []
    for b in range(40):
        a = g64.bp(s_all[b], 5, prm64)["llr"]
        c = g32.bp(s_all[b], 5, prm16)["llr"].astype(np.float64)
        med.append(np.median(np.abs(a - c) / np.maximum(1.0, np.abs(a))))
    assert np.median(med) < tol


def test_near_tie_flags(oracle_mod):
    """Status bit 8 marks shots whose beam search met an argmin or pruning
    margin inside (0, tie_guard): none without a guard, only beam shots, and
    more with a wider guard."""
    prob, sh = _bb_shots(0.05, 1500, "near_tie")
    g = oracle_mod.Graph(prob, "f32")
    base = dict(max_rounds=10, beam_width=8, initial_iters=30, iters_per_round=20, ms_scale=0.625, msg_storage=1)
    r0 = g.decode_batch(sh.syndromes, oracle_mod.Params(**base), nthreads=4)
    assert not (r0["status"] & 8).any()
    r1 = g.decode_batch(sh.syndromes, oracle_mod.Params(tie_guard=1e-3, **base), nthreads=4)
    r2 = g.decode_batch(sh.syndromes, oracle_mod.Params(tie_guard=1e-1, **base), nthreads=4)
    f1, f2 = (r1["status"] & 8) > 0, (r2["status"] & 8) > 0
    assert np.all(f2[f1]) and f2.sum() > f1.sum() > 0
    assert np.all((r2["status"][f2] & 3) != 1)           # a shot ending in the seed has no beam decision
    # the flag changes nothing else
    for k in ("corrections", "iters"):
        assert np.array_equal(r0[k], r2[k])
    assert np.array_equal(r0["status"], r2["status"] & ~np.uint32(8))


# ----------------------------------------------------------------------------
# Near-tie logging: hand-worked margins, exact ties and status bit 8
# ----------------------------------------------------------------------------
def _priors(lam):
    """Priors whose Lambda_j = log((1-p_j)/p_j) are the given values."""
    return 1.0 / (1.0 + np.exp(np.asarray(lam, np.float64)))


def _golden_params(oracle_mod, q, guard=0.0):
    return oracle_mod.Params(max_rounds=q["max_rounds"], beam_width=q["beam_width"],
                             initial_iters=q["initial_iters"], iters_per_round=q["iters_per_round"],
                             num_results=1, ms_scale=q["alpha"], llr_clamp=q["llr_clamp"], tie_guard=guard)


def _close(a, b, rel):
    if b == "inf":
        return a == np.inf
    return abs(a - b) <= rel * abs(b)


def _near_tie_sign_margins(oracle_mod, G_for, rel):
    g = _golden("near_tie_sign_margins.json")
    pr = g["problem"]
    for name, case in g["cases"].items():
        G = G_for(_dense_problem(pr["H"], _priors(case["Lambda"])))
        r = G.decode_log(np.array(pr["syndrome"]), _golden_params(oracle_mod, pr["params"]))
        exp = case["expected"]
        assert r["status"] == exp["status"] and list(r["ehat"]) == exp["ehat"] and r["iters"] == exp["iters"], name
        assert _close(r["min_gap"], exp["min_gap"], rel), (name, r["min_gap"])
        assert r["ties"] == exp["ties"], (name, r["ties"])
        lg = r["log"]
        for k, rec in enumerate(exp.get("records", [])):
            assert (lg["kind"][k], lg["call"][k], lg["t"][k], lg["nties"][k]) == \
                (rec["kind"], rec["call"], rec["t"], rec["nties"]), (name, k)
            assert _close(lg["gap"][k], rec["gap"], rel), (name, k, lg["gap"][k])
            if "key" in rec:
                assert int(lg["key"][k]) == rec["key"]


def _near_tie_argmin(oracle_mod, G_for, rel):
    g = _golden("near_tie_argmin.json")
    pr = g["problem"]
    G = G_for(_dense_problem(pr["H"], _priors(pr["Lambda"])))
    exp = g["expected"]
    for guard, st in exp["status_by_guard"].items():
        r = G.decode_log(np.array(pr["syndrome"]), _golden_params(oracle_mod, pr["params"], float(guard)))
        assert r["status"] == st, (guard, r["status"])
        assert list(r["ehat"]) == exp["ehat"] and r["iters"] == exp["iters"]
        assert _close(r["min_gap"], exp["min_gap"], rel), r["min_gap"]
        assert r["ties"] == exp["ties"], r["ties"]
        lg = r["log"]
        am = np.nonzero(lg["kind"] == oracle_mod.LOG_ARGMIN)[0]
        assert len(am) == len(exp["argmin_records"])
        for k, rec in zip(am, exp["argmin_records"]):
            assert lg["call"][k] == rec["call"] and int(lg["key"][k]) == rec["key"]
            assert _close(lg["gap"][k], rec["gap"], rel), (k, lg["gap"][k])
        # the iteration records of every call: t = 1..iters in order
        it = lg["kind"] == oracle_mod.LOG_ITER
        assert list(lg["t"][it]) == [1, 2, 3, 4, 1, 2, 3, 1, 2, 3]


def _near_tie_pruning(oracle_mod, G_for, rel):
    g = _golden("near_tie_pruning.json")
    pr = g["problem"]
    G = G_for(_dense_problem(pr["H"], _priors(pr["Lambda"])))
    exp = g["expected"]
    for guard, st in exp["status_by_guard"].items():
        r = G.decode_log(np.array(pr["syndrome"]), _golden_params(oracle_mod, pr["params"], float(guard)))
        assert r["status"] == st, (guard, r["status"])
        assert list(r["ehat"]) == exp["ehat"] and r["iters"] == exp["iters"]
        assert _close(r["min_gap"], exp["min_gap"], rel), r["min_gap"]
        assert r["ties"] == exp["ties"], r["ties"]
        lg = r["log"]
        pk = np.nonzero(lg["kind"] == oracle_mod.LOG_PRUNE)[0]
        assert len(pk) == len(exp["prune_records"])
        for k, rec in zip(pk, exp["prune_records"]):
            assert lg["round"][k] == rec["round"] and lg["nties"][k] == rec["nties"]
            assert _close(lg["gap"][k], rec["gap"], rel), (rec["round"], lg["gap"][k])
        am = lg["kind"] == oracle_mod.LOG_ARGMIN
        assert [int(x) for x in lg["key"][am]] == exp["argmin_records"]["keys"]
        assert list(lg["nties"][am]) == exp["argmin_records"]["nties"]
        it = np.nonzero(lg["kind"] == oracle_mod.LOG_ITER)[0]
        assert len(it) == len(exp["iteration_gaps"])
        for k, gv in zip(it, exp["iteration_gaps"]):
            assert _close(lg["gap"][k], gv, rel) and lg["nties"][k] == 0, (k, lg["gap"][k])


_NEAR_TIE_PINS = (_near_tie_sign_margins, _near_tie_argmin, _near_tie_pruning)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("pin", _NEAR_TIE_PINS, ids=lambda f: f.__name__[1:])
def test_near_tie_hand_worked(oracle_mod, precision, pin):
    """Sign margins and exact ties (Eqs. 2-4), the argmin runner-up margin
    (Alg. 3), the pruning margin between ranks w-1 and w (App. B), the
    smallest margin, the tie count and status bit 8 against hand-worked
    values; the single-precision build within its rounding (scores on the
    2^-16 grid)."""
    rel = 1e-9 if precision == "f64" else 2e-3
    pin(oracle_mod, lambda prob: oracle_mod.Graph(prob, precision), rel)


# planted mistakes in the near-tie logic: (description, original text, replacement)
_MUTANTS = [
    ("pruning margin between ranks w and w+1",
     "const double s0 = x->rscore[w - 1], s1 = x->rscore[w];",
     "const double s0 = x->rscore[w], s1 = x->rscore[w + 1];"),
    ("pruning margin between ranks w-2 and w-1",
     "const double s0 = x->rscore[w - 1], s1 = x->rscore[w];",
     "const double s0 = x->rscore[w - 2], s1 = x->rscore[w - 1];"),
    ("argmin margin relative to the smallest instead of the runner-up",
     "double s = fabs((double)second) > 1.0 ? fabs((double)second) : 1.0;",
     "double s = fabs((double)bv) > 1.0 ? fabs((double)bv) : 1.0;"),
    ("runner-up = first node seen after the smallest",
     "} else if (!have_second || v < second) {",
     "} else if (!have_second) {"),
    ("sign margin without the message terms in its scale",
     "                scale += fabs((double)w->vbuf[k]);\n",
     ""),
    ("exact ties flagged as near ties",
     "if (x->prm->tie_guard > 0 && gap_rel > 0 && gap_rel < x->prm->tie_guard)",
     "if (x->prm->tie_guard > 0 && gap_rel >= 0 && gap_rel < x->prm->tie_guard)"),
    ("pruning margin not flagged",
     "            tie_check(x, bm);\n",
     ""),
]


@pytest.mark.parametrize("mutant", _MUTANTS, ids=[m[0] for m in _MUTANTS])
def test_near_tie_pins_catch_planted_mistakes(oracle_mod, tmp_path, mutant):
    """Each planted mistake in the oracle's near-tie logic (a copy of the
    source compiled here, on the CPU) makes at least one hand-worked pin fail."""
    from oracle import build_oracle
    _, old, new = mutant
    src = open(build_oracle.SRC).read()
    assert src.count(old) == 1, "the planted mistake no longer matches the source"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib_path = str(tmp_path / "libmutant.so")
    build_oracle.compile_library(str(path), lib_path)
    lib = oracle_mod.load_library(lib_path, "f64")
    failed = 0
    for pin in _NEAR_TIE_PINS:
        try:
            pin(oracle_mod, lambda prob: oracle_mod.Graph(prob, "f64", lib=lib), 1e-9)
        except AssertionError:
            failed += 1
    assert failed > 0


def test_decision_log_summarises_the_run(oracle_mod):
    """The decision log's records reproduce the run's near-tie summary (the
    smallest nonzero margin and the tie count), leave its outputs unchanged,
    and two runs of the same build have equal logs."""
    prob, sh = _bb_shots(0.05, 60, "dlog")
    prm = oracle_mod.Params(max_rounds=10, beam_width=8, initial_iters=50, iters_per_round=20, ms_scale=0.625)
    s_all = W.unpack_bits(sh.syndromes, prob.M)
    for precision in ("f64", "f32"):
        G = oracle_mod.Graph(prob, precision)
        for b in range(sh.B):
            r = G.decode_log(s_all[b], prm)
            r0 = G.decode_one(s_all[b], prm)
            assert (r["status"], r["iters"], list(r["ehat"])) == (r0["status"], r0["iters"], list(r0["ehat"]))
            lg = r["log"]
            assert r["ties"] == r0["ties"] == int(lg["nties"].sum())
            assert r["min_gap"] == r0["min_gap"] == float(lg["gap"].min())
            assert oracle_mod.first_divergence(lg, G.decode_log(s_all[b], prm)["log"]) == -1
            # records: the seed's iterations, its argmin, then per child its
            # iterations and argmin, a kept set per finished round
            assert lg["call"][0] == 0 and lg["kind"][0] == oracle_mod.LOG_ITER and lg["t"][0] == 1
            assert np.all(np.diff(lg["call"]) >= 0)


def test_f64_parity_rule_on_the_single_precision_build(oracle_mod):
    """The rule the GPU tests apply against double precision, checked with the
    oracle's single-precision build in the GPU's place: it holds on the
    [[72,12,6]] workload, and it rejects a mismatch planted on a shot whose
    double-precision run has no near tie."""
    import parity_f64
    prob = W.bb72_code_capacity(0.03)
    sh = W.sample_shots(prob, 10_000, "bb72_cc_p0.03")
    prm = oracle_mod.Params(max_rounds=10, beam_width=8, initial_iters=50, iters_per_round=20, ms_scale=0.625)
    r32 = oracle_mod.Graph(prob, "f32").decode_batch(sh.syndromes, prm, nthreads=8)
    counts, r64 = parity_f64.check_against_f64(prob, prm, sh.syndromes, r32, nthreads=8)
    assert counts["mismatches"] == counts["near_tie_1e4"]
    calm = np.nonzero((r64["min_gap"] > 1e-3) & (r64["ties"] == 0) & (r64["status"] == 2))[0]
    planted = {k: v.copy() for k, v in r32.items()}
    planted["corrections"][calm[0], 0] ^= 1
    with pytest.raises(AssertionError, match="no near tie"):
        parity_f64.check_against_f64(prob, prm, sh.syndromes, planted, ref64=r64)
    # the divergence search itself
    a = dict(call=np.array([0, 0, 1]), kind=np.array([0, 1, 0]), t=np.array([1, 0, 1]),
             key=np.array([5, 7, 9], np.uint64), gap=np.array([0.5, 1e-5, 0.3]), nties=np.array([0, 0, 0]))
    b = {k: v.copy() for k, v in a.items()}
    assert oracle_mod.first_divergence(a, b) == -1
    b["key"][2] = 10
    assert oracle_mod.first_divergence(a, b) == 2
    assert oracle_mod.near_tie_before(a, 0, 1e-4) is False
    assert oracle_mod.near_tie_before(a, 1, 1e-4) is True and oracle_mod.near_tie_before(a, 1, 1e-6) is False
