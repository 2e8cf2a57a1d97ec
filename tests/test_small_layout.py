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
