"""Input generators: code properties, DEM structure, seeded reproducibility."""
import numpy as np
import pytest

from paper_2512_07057_gb300 import workloads as W


@pytest.mark.parametrize("l,m,n,k", [(6, 6, 72, 12), (12, 6, 144, 12)])
def test_bb_code_parameters(l, m, n, k):
    """[[72,12,6]] and [[144,12,12]]: N and k = N - rank H_X - rank H_Z as printed."""
    HX, HZ = W.bb_matrices(l, m, W.BB_A_TERMS, W.BB_B_TERMS)
    assert HX.shape == (n // 2, n)
    assert ((HX.astype(int) @ HZ.T.astype(int)) % 2 == 0).all()       # stabilizers commute
    assert n - W.gf2_rank(HX) - W.gf2_rank(HZ) == k
    assert set(HX.sum(0)) == {3} and set(HX.sum(1)) == {6}             # (3,6)-regular


@pytest.mark.parametrize("maker", [W.bb72_code_capacity, W.bb144_code_capacity])
def test_logical_basis(maker):
    prob = maker(0.03)
    HX, A, HZ = prob.H_dense(), prob.A_dense(), prob.meta["HZ"]
    assert A.shape[0] == 12
    # X logicals commute with Z stabilizers: a Z-stabilizer added to a correction
    # changes neither its syndrome nor its observable flips
    assert ((A.astype(int) @ HZ.T.astype(int)) % 2 == 0).all()
    assert ((HX.astype(int) @ HZ.T.astype(int)) % 2 == 0).all()
    # rank K and independent of rowspace(H_X)
    assert W.gf2_rank(A) == 12
    assert W.gf2_rank(np.vstack([HX, A])) == W.gf2_rank(HX) + 12
    # every Z logical is detected by some row of A: ker(H_X) / rowspace(H_Z) has dimension 12
    ker = W.gf2_nullspace(HX)
    assert W.gf2_rank(np.vstack([HZ, ker])) == W.gf2_rank(HZ) + 12


def test_phenomenological_dem_structure():
    prob = W.bb_phenomenological(12, 6, 12, 2e-3, 2e-3)
    assert (prob.M, prob.N, prob.n_edges) == (936, 2592, 6912)
    H = prob.H_dense()
    cw = H.sum(0)
    assert (cw[:1728] == 3).all() and (cw[1728:] == 2).all()
    rw = H.sum(1)
    assert (rw[:72] == 7).all() and (rw[72:864] == 8).all() and (rw[864:] == 1).all()
    A = prob.A_dense()
    assert (A[:, 1728:] == 0).all()


def test_synthetic_dem_structure_and_seed():
    a = W.synthetic_dem()
    b = W.synthetic_dem()
    assert (a.M, a.N, a.K) == (936, 8800, 12)
    cw = np.diff(np.bincount(a.H_col_idx, minlength=a.N).cumsum(), prepend=0)
    cw = np.bincount(a.H_col_idx, minlength=a.N)
    assert cw.min() == 2 and cw.max() == 6
    assert (a.priors >= 1e-5).all() and (a.priors <= 1e-3).all()
    assert np.array_equal(a.H_col_idx, b.H_col_idx) and np.array_equal(a.priors, b.priors)


def test_shot_sampling_consistent():
    prob = W.bb72_code_capacity(0.05)
    sh = W.sample_shots(prob, 3000, "test_sampling", keep_errors=True)
    e = W.unpack_bits(sh.errors, prob.N)
    s = W.unpack_bits(sh.syndromes, prob.M)
    o = W.unpack_bits(sh.obs, prob.K)
    assert np.array_equal((e.astype(int) @ prob.H_dense().T) % 2, s)
    assert np.array_equal((e.astype(int) @ prob.A_dense().T) % 2, o)
    # Bernoulli(p) marginal: 3000 * 72 draws
    rate = e.mean()
    assert abs(rate - 0.05) < 4 * np.sqrt(0.05 * 0.95 / e.size)
    sh2 = W.sample_shots(prob, 3000, "test_sampling", keep_errors=True)
    assert np.array_equal(sh.syndromes, sh2.syndromes)


def test_pack_roundtrip():
    rng = np.random.default_rng(1)
    for L in (1, 31, 32, 33, 72, 936):
        bits = rng.integers(0, 2, size=(5, L)).astype(np.uint8)
        packed = W.pack_bits(bits)
        assert packed.shape == (5, (L + 31) // 32)
        assert np.array_equal(W.unpack_bits(packed, L), bits)
        if L % 32:
            assert (packed[:, -1] >> np.uint32(L % 32) == 0).all()


def test_xyz_problem_halves_are_the_xz_problems():
    """XYZ decoding's H stacks H_X over H_Z on (X, Z, Y) mechanism columns: the
    two halves of every syndrome and observable vector equal those of the
    XZ components z = Z xor Y (checked by H_X, X-type logicals) and x = X xor Y
    (H_Z, Z-type logicals); Y columns create length-4 cycles."""
    P = W.bb_xyz_code_capacity(6, 6, 0.06)
    zp, xp = W.bb_xz_parts(6, 6, 0.06)
    n = 72
    sh = W.sample_shots(P, 500, "xyz_halves", keep_errors=True)
    e = W.unpack_bits(sh.errors, P.N)
    z, x = e[:, n:2 * n] ^ e[:, 2 * n:], e[:, :n] ^ e[:, 2 * n:]
    s1, s2 = W.split_bits(sh.syndromes, P.M, zp.M)
    o1, o2 = W.split_bits(sh.obs, P.K, zp.K)
    assert np.array_equal(W.unpack_bits(s1, zp.M), (z @ zp.H_dense().T) % 2)
    assert np.array_equal(W.unpack_bits(s2, xp.M), (x @ xp.H_dense().T) % 2)
    assert np.array_equal(W.unpack_bits(o1, zp.K), (z @ zp.A_dense().T) % 2)
    assert np.array_equal(W.unpack_bits(o2, xp.K), (x @ xp.A_dense().T) % 2)
    Hd = P.H_dense().astype(np.int64)
    # a length-4 cycle: two rows sharing two columns (an X check and a Z check through Y columns)
    overlap = Hd @ Hd.T
    np.fill_diagonal(overlap, 0)
    assert overlap.max() >= 2
    assert np.allclose(P.priors, 0.02)
    # the Z-type residual of a Z-type logical operator is detected by the X-type logicals only
    assert zp.K == xp.K == 12
