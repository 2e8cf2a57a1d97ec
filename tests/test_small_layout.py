"""The single-warp engine's shared-memory placement of a code's messages
(host logic, no GPU): every edge gets its own word, each row's six edges fill
the row's three pairs, each column's three edges are read once each, and on
the bivariate bicycle codes every access of both passes touches 32 distinct
banks."""
import numpy as np
import pytest

from paper_2512_07057_gb300 import binding as B
from paper_2512_07057_gb300 import workloads as W


def _codes():
    return [("bb72", W.bb72_code_capacity(0.05)), ("bb144", W.bb144_code_capacity(0.05)),
            ("bb_l9m6", W.bb_code_capacity(9, 6, 0.05))]


@pytest.mark.parametrize("name,prob", _codes())
def test_placement_is_a_conflict_free_bijection(name, prob):
    M, N = prob.M, prob.N
    rp, ci = prob.H_row_ptr, prob.H_col_idx
    lay = B.bsd_small_layout(M, N, rp, ci)
    plane, ew, cw = lay["plane"], lay["edge_word"], lay["col_word"]
    E = int(rp[-1])
    # distinct words inside the extent
    assert len(set(ew.tolist())) == E
    assert ew.min() >= 0 and ew.max() < lay["extent"]
    # planes of the engine's compile-time stride: they do not overlap and
    # each starts on an 8-byte boundary
    P = 64 * ((M + 31) // 32) + 12
    assert plane.tolist() == [0, P, 2 * P] and P >= 2 * M and P % 2 == 0
    assert lay["extent"] == 2 * P + 2 * M
    # row i's edges fill exactly its three pairs plane[h] + 2 i + {0, 1}
    for i in range(M):
        want = {int(plane[h]) + 2 * i + u for h in range(3) for u in range(2)}
        assert set(ew[rp[i]:rp[i + 1]].tolist()) == want
    # column j's three k slots are the words of its three edges
    cols = [[] for _ in range(N)]
    for i in range(M):
        for e in range(rp[i], rp[i + 1]):
            cols[ci[e]].append(int(ew[e]))
    for j in range(N):
        assert sorted(cw[j].tolist()) == sorted(cols[j])
    # both passes conflict-free: the error pass's access (c, k) reads 32
    # words in 32 distinct banks, the detector pass's 8-byte accesses cover
    # 16 distinct bank pairs per half warp
    assert lay["excess"] == 0
    for c in range((N + 31) // 32):
        for k in range(3):
            words = cw[32 * c:32 * c + 32, k]
            assert len(set((words % 32).tolist())) == len(words), (c, k)
    for r in range((M + 31) // 32):
        for h in range(3):
            for half in range(2):
                rows = [i for i in range(32 * r + 16 * half, 32 * r + 16 * half + 16) if i < M]
                pairs = [(int(plane[h]) + 2 * i) // 2 for i in rows]
                assert len(set(p % 16 for p in pairs)) == len(pairs)


def test_the_placement_is_deterministic():
    p = W.bb144_code_capacity(0.05)
    a = B.bsd_small_layout(p.M, p.N, p.H_row_ptr, p.H_col_idx)
    b = B.bsd_small_layout(p.M, p.N, p.H_row_ptr, p.H_col_idx)
    assert np.array_equal(a["edge_word"], b["edge_word"]) and np.array_equal(a["col_word"], b["col_word"])


def test_other_degree_structures_are_unsupported():
    p = W.random_ldpc(40, 80, 4, 0.05, seed=1)
    with pytest.raises(B.BsdError) as ei:
        B.bsd_small_layout(p.M, p.N, p.H_row_ptr, p.H_col_idx)
    assert ei.value.code == B.BSD_ERR_UNSUPPORTED


def test_bad_csr_is_rejected():
    p = W.bb72_code_capacity(0.05)
    ci = p.H_col_idx.copy()
    ci[1] = ci[0]                       # columns of a row not ascending
    with pytest.raises(B.BsdError) as ei:
        B.bsd_small_layout(p.M, p.N, p.H_row_ptr, ci)
    assert ei.value.code == B.BSD_ERR_INVALID_ARG



@pytest.mark.parametrize("M,seed", [(36, 1), (48, 2), (64, 3), (72, 4), (80, 5)])
def test_placement_of_random_regular_codes_is_valid(M, seed):
    """Whatever bank loads the search leaves, the placement is a bijection
    onto the rows' pairs and every column takes k = 0, 1, 2 once; where no
    bank of a column group holds more than three edges, the error pass is
    conflict-free."""
    prob = W.random_regular_36(M, 0.05, seed)
    rp, ci = prob.H_row_ptr, prob.H_col_idx
    lay = B.bsd_small_layout(prob.M, prob.N, rp, ci)
    plane, ew, cw = lay["plane"], lay["edge_word"], lay["col_word"]
    assert len(set(ew.tolist())) == int(rp[-1])
    for i in range(prob.M):
        assert set(ew[rp[i]:rp[i + 1]].tolist()) == {int(plane[h]) + 2 * i + u for h in range(3) for u in range(2)}
    cols = [[] for _ in range(prob.N)]
    for i in range(prob.M):
        for e in range(rp[i], rp[i + 1]):
            cols[ci[e]].append(int(ew[e]))
    for j in range(prob.N):
        assert sorted(cw[j].tolist()) == sorted(cols[j])
    if lay["excess"] == 0:
        for c in range((prob.N + 31) // 32):
            for k in range(3):
                words = cw[32 * c:32 * c + 32, k]
                assert len(set((words % 32).tolist())) == len(words)


# ----------------------------------------------------------------------------
# the generic engines' placement (bsd_generic_layout)
# ----------------------------------------------------------------------------
def _check_generic(prob, lay):
    rp, ci = prob.H_row_ptr, prob.H_col_idx
    ew, se = lay["edge_word"], lay["slot_edge"]
    # each row's edges fill exactly the row's window
    for i in range(prob.M):
        assert sorted(ew[rp[i]:rp[i + 1]].tolist()) == list(range(int(rp[i]), int(rp[i + 1])))
    # every edge sits in exactly one slot, of its own column
    seen = np.zeros(int(rp[-1]), np.int64)
    for k in range(lay["colK"]):
        for j in range(prob.N):
            e = int(se[k, j])
            if e >= 0:
                assert ci[e] == j
                seen[e] += 1
    assert (seen == 1).all()


def _wavefronts(prob, word_of, slot_edge):
    """Bank-conflict wavefronts of the error pass's message accesses: per
    (32-column group, slot), the busiest bank's count."""
    tot = 0
    for c in range((prob.N + 31) // 32):
        for k in range(slot_edge.shape[0]):
            banks = [word_of(int(slot_edge[k, j])) % 32 for j in range(32 * c, min(prob.N, 32 * c + 32))
                     if slot_edge[k, j] >= 0]
            if banks:
                tot += max(np.bincount(banks))
    return tot


@pytest.mark.parametrize("name", ["phenomenological", "synthetic"])
def test_generic_placement_of_the_dems(name):
    prob = W.bb_phenomenological(12, 6, 12, 3e-3, 3e-3) if name == "phenomenological" else W.synthetic_dem()
    lay = B.bsd_generic_layout(prob.M, prob.N, prob.H_row_ptr, prob.H_col_idx)
    _check_generic(prob, lay)
    # the CSR order, slots in the column lists' order, for comparison
    rp, ci = prob.H_row_ptr, prob.H_col_idx
    csr = -np.ones_like(lay["slot_edge"])
    fill = np.zeros(prob.N, np.int64)
    for e in range(int(rp[-1])):
        j = ci[e]
        csr[fill[j], j] = e
        fill[j] += 1
    before = _wavefronts(prob, lambda e: e, csr)
    after = _wavefronts(prob, lambda e: int(lay["edge_word"][e]), lay["slot_edge"])
    assert after < 0.4 * before
    if name == "synthetic":
        # conflict-free: one wavefront per (group, slot) that has an edge
        assert lay["excess"] == 0
        ideal = sum(1 for c in range((prob.N + 31) // 32) for k in range(lay["colK"])
                    if (lay["slot_edge"][k, 32 * c:32 * c + 32] >= 0).any())
        assert after == ideal


@pytest.mark.parametrize("seed", range(4))
def test_generic_placement_of_random_codes_is_valid(seed):
    """Columns of degree 0 to 6 (holes in the slots), rows of any degree
    including 1."""
    rng = np.random.default_rng(100 + seed)
    M, N = 30 + 7 * seed, 150 + 40 * seed
    H = np.zeros((M, N), np.uint8)
    for j in range(N):
        d = int(rng.integers(0, 7 if seed % 2 else 4))
        if d:
            H[rng.choice(M, size=d, replace=False), j] = 1
    prob = W.problem_from_dense(H, np.zeros((1, N), np.uint8), np.full(N, 0.05), name=f"gen_{seed}")
    lay = B.bsd_generic_layout(prob.M, prob.N, prob.H_row_ptr, prob.H_col_idx)
    assert lay["colK"] == (6 if seed % 2 else 3)
    _check_generic(prob, lay)


def test_generic_placement_rejects_higher_degrees():
    rng = np.random.default_rng(7)
    H = (rng.random((40, 60)) < 0.05).astype(np.uint8)
    H[:8, 0] = 1                                   # a column of degree 8
    prob = W.problem_from_dense(H, np.zeros((1, 60), np.uint8), np.full(60, 0.05))
    with pytest.raises(B.BsdError) as ei:
        B.bsd_generic_layout(prob.M, prob.N, prob.H_row_ptr, prob.H_col_idx)
    assert ei.value.code == B.BSD_ERR_UNSUPPORTED
