"""Seeded synthetic decoding problems (H, A, p) and shot sampling.

This module builds inputs only.  It holds none of the decoder's arithmetic
(no belief propagation, no beam search); both the CUDA path and the CPU
oracle read the arrays it returns.

The decoding problem is the triple (H in F2^{MxN}, A in F2^{KxN}, p in (0,1)^N)
of the paper's App. A: columns are error sources, rows of H are detectors and
rows of A are logical observables.  A shot draws e_j ~ Bernoulli(p_j)
independently, and the decoder sees only the syndrome s = H e (mod 2); the
true observable flips A e (mod 2) are kept to score logical failures.

Instances:
  * bivariate bicycle (BB) codes, H_X = [A_poly | B_poly] with
    x = S_l (x) I_m, y = I_l (x) S_m (S_n the n x n cyclic shift),
    decoded for Z flips under code-capacity noise; the observables are a
    basis of X-type logical operators (ker H_Z modulo rowspace H_X);
  * a phenomenological detector error model of a BB code over T noisy
    syndrome rounds followed by one perfect round;
  * a synthetic circuit-shaped detector error model (column weight 2-6,
    log-uniform priors, sparse random observables).

Bit layout used everywhere (device and host): a vector v of length L is
stored in ceil(L/32) little-endian uint32 words, bit i of word i//32 is v_i,
padding bits above L are zero.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ROOT_SEED = 20251207


# ----------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------
@dataclass
class Problem:
    """A decoding problem (H, A, p) in CSR form.

    H_row_ptr/H_col_idx: CSR of H (M x N), column indices ascending per row.
    A_row_ptr/A_col_idx: CSR of A (K x N).
    priors: float64[N], each in (0, 1).
    """
    name: str
    M: int
    N: int
    K: int
    H_row_ptr: np.ndarray
    H_col_idx: np.ndarray
    A_row_ptr: np.ndarray
    A_col_idx: np.ndarray
    priors: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.H_row_ptr[-1])

    def H_dense(self) -> np.ndarray:
        return csr_to_dense(self.H_row_ptr, self.H_col_idx, self.M, self.N)

    def A_dense(self) -> np.ndarray:
        return csr_to_dense(self.A_row_ptr, self.A_col_idx, self.K, self.N)


@dataclass
class Shots:
    """B sampled shots of a problem, bitpacked as described in the module doc."""
    syndromes: np.ndarray      # uint32[B, ceil(M/32)]
    obs: np.ndarray            # uint32[B, ceil(K/32)]  true A e
    errors: np.ndarray | None  # uint32[B, ceil(N/32)]  true e (kept when asked)

    @property
    def B(self) -> int:
        return int(self.syndromes.shape[0])


# ----------------------------------------------------------------------------
# GF(2) helpers (input construction only)
# ----------------------------------------------------------------------------
def words(n: int) -> int:
    return (n + 31) // 32


def dense_to_csr(Hd: np.ndarray):
    Hd = np.asarray(Hd, dtype=np.uint8)
    rows, cols = np.nonzero(Hd)
    row_ptr = np.zeros(Hd.shape[0] + 1, dtype=np.int32)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return row_ptr, cols.astype(np.int32)


def csr_to_dense(row_ptr, col_idx, n_rows, n_cols) -> np.ndarray:
    D = np.zeros((n_rows, n_cols), dtype=np.uint8)
    for r in range(n_rows):
        D[r, col_idx[row_ptr[r]:row_ptr[r + 1]]] = 1
    return D


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """bool/uint8 [..., L] -> uint32 [..., ceil(L/32)] (bit i of word i//32)."""
    bits = np.asarray(bits, dtype=np.uint8)
    L = bits.shape[-1]
    W = words(L)
    pad = W * 32 - L
    if pad:
        bits = np.concatenate([bits, np.zeros(bits.shape[:-1] + (pad,), np.uint8)], axis=-1)
    b = bits.reshape(bits.shape[:-1] + (W, 32)).astype(np.uint64)
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    return (b * weights).sum(axis=-1).astype(np.uint32)


def unpack_bits(packed: np.ndarray, L: int) -> np.ndarray:
    """uint32 [..., W] -> uint8 [..., L]."""
    packed = np.asarray(packed, dtype=np.uint32)
    sh = np.arange(32, dtype=np.uint32)
    b = ((packed[..., :, None] >> sh) & 1).astype(np.uint8)
    return b.reshape(packed.shape[:-1] + (-1,))[..., :L]


def gf2_rank(Mat: np.ndarray) -> int:
    A = (np.asarray(Mat, dtype=np.uint8) & 1).copy()
    r = 0
    rows, cols = A.shape
    for c in range(cols):
        piv = np.nonzero(A[r:, c])[0]
        if piv.size == 0:
            continue
        p = r + piv[0]
        if p != r:
            A[[r, p]] = A[[p, r]]
        others = np.nonzero(A[:, c])[0]
        others = others[others != r]
        A[others] ^= A[r]
        r += 1
        if r == rows:
            break
    return r


def gf2_nullspace(Mat: np.ndarray) -> np.ndarray:
    """Basis (rows) of {x : Mat x = 0} over GF(2)."""
    A = (np.asarray(Mat, dtype=np.uint8) & 1).copy()
    rows, cols = A.shape
    pivots = []
    r = 0
    for c in range(cols):
        if r == rows:
            break
        piv = np.nonzero(A[r:, c])[0]
        if piv.size == 0:
            continue
        p = r + piv[0]
        if p != r:
            A[[r, p]] = A[[p, r]]
        others = np.nonzero(A[:, c])[0]
        others = others[others != r]
        A[others] ^= A[r]
        pivots.append(c)
        r += 1
    free = [c for c in range(cols) if c not in set(pivots)]
    basis = np.zeros((len(free), cols), dtype=np.uint8)
    for k, f in enumerate(free):
        basis[k, f] = 1
        for i, pc in enumerate(pivots):
            if A[i, f]:
                basis[k, pc] = 1
    return basis


# ----------------------------------------------------------------------------
# bivariate bicycle codes
# ----------------------------------------------------------------------------
def _shift(n: int) -> np.ndarray:
    return np.roll(np.eye(n, dtype=np.uint8), 1, axis=1)


def bb_matrices(l: int, m: int, a_terms, b_terms):
    """H_X = [A|B], H_Z = [B^T|A^T] for a BB code.

    a_terms / b_terms are lists of monomials ('x', k) or ('y', k) meaning x^k
    or y^k, with x = S_l (x) I_m and y = I_l (x) S_m.
    """
    x = np.kron(_shift(l), np.eye(m, dtype=np.uint8))
    y = np.kron(np.eye(l, dtype=np.uint8), _shift(m))

    def poly(terms):
        P = np.zeros((l * m, l * m), dtype=np.uint8)
        for var, k in terms:
            base = x if var == "x" else y
            P ^= np.linalg.matrix_power(base.astype(np.int64), k).astype(np.uint8) & 1
        return P

    Ap, Bp = poly(a_terms), poly(b_terms)
    HX = np.concatenate([Ap, Bp], axis=1)
    HZ = np.concatenate([Bp.T, Ap.T], axis=1)
    return HX, HZ


def logical_basis(HX: np.ndarray, HZ: np.ndarray) -> np.ndarray:
    """K vectors of ker(H_Z) independent of rowspace(H_X) (X-type logicals).

    A Z-type residual r with H_X r = 0 is a logical error iff L r != 0 for
    some returned row L.
    """
    ker = gf2_nullspace(HZ)
    basis = []
    cur = HX.copy()
    rk = gf2_rank(cur)
    for v in ker:
        trial = np.vstack([cur, v[None, :]])
        r2 = gf2_rank(trial)
        if r2 > rk:
            basis.append(v)
            cur, rk = trial, r2
    return np.array(basis, dtype=np.uint8).reshape(-1, HX.shape[1])


# The two BB polynomials used by both code-capacity instances:
# A = x^3 + y + y^2, B = y^3 + x + x^2.
BB_A_TERMS = [("x", 3), ("y", 1), ("y", 2)]
BB_B_TERMS = [("y", 3), ("x", 1), ("x", 2)]


def bb_code_capacity(l: int, m: int, p: float, name: str | None = None) -> Problem:
    HX, HZ = bb_matrices(l, m, BB_A_TERMS, BB_B_TERMS)
    L = logical_basis(HX, HZ)
    N = HX.shape[1]
    hr, hc = dense_to_csr(HX)
    ar, ac = dense_to_csr(L)
    return Problem(name=name or f"bb_{N}_cc_p{p}", M=HX.shape[0], N=N, K=L.shape[0],
                   H_row_ptr=hr, H_col_idx=hc, A_row_ptr=ar, A_col_idx=ac,
                   priors=np.full(N, float(p)),
                   meta={"l": l, "m": m, "HZ": HZ, "kind": "bb_code_capacity", "p": p})


def bb_xyz_code_capacity(l: int, m: int, p: float) -> Problem:
    """XYZ decoding problem of a BB code under depolarizing noise.

    Columns are the per-qubit mechanisms X_q (index q), Z_q (n + q) and Y_q
    (2n + q), each with prior p/3.  H stacks both stabilizer types: the
    X-check rows (H_X) see the Z component (Z_q and Y_q), the Z-check rows
    (H_Z, after them) see the X component (X_q and Y_q); the Y columns make
    length-4 cycles.  A holds the X-type logicals on the Z component, then
    the Z-type logicals on the X component.
    """
    HX, HZ = bb_matrices(l, m, BB_A_TERMS, BB_B_TERMS)
    LX = logical_basis(HX, HZ)       # detect Z-type residuals
    LZ = logical_basis(HZ, HX)       # detect X-type residuals
    n = HX.shape[1]
    z = np.zeros_like(HX)
    H = np.block([[z, HX, HX], [HZ, np.zeros_like(HZ), HZ]]).astype(np.uint8)
    A = np.block([[np.zeros_like(LX), LX, LX], [LZ, np.zeros_like(LZ), LZ]]).astype(np.uint8)
    hr, hc = dense_to_csr(H)
    ar, ac = dense_to_csr(A)
    return Problem(name=f"bb_{n}_xyz_p{p}", M=H.shape[0], N=3 * n, K=A.shape[0],
                   H_row_ptr=hr, H_col_idx=hc, A_row_ptr=ar, A_col_idx=ac,
                   priors=np.full(3 * n, p / 3.0),
                   meta={"l": l, "m": m, "kind": "bb_xyz_code_capacity", "p": p, "mx": HX.shape[0],
                         "kx": LX.shape[0]})


def bb_xz_parts(l: int, m: int, p: float):
    """The XZ-decoding counterpart of bb_xyz_code_capacity: the Z component
    decoded with (H_X, X-type logicals) and the X component with (H_Z, Z-type
    logicals), each node with the marginal prior of its component,
    P(Z_q xor Y_q) = 2 (p/3)(1 - p/3)."""
    HX, HZ = bb_matrices(l, m, BB_A_TERMS, BB_B_TERMS)
    q = 2.0 * (p / 3.0) * (1.0 - p / 3.0)
    parts = []
    for Hm, Lm, tag in ((HX, logical_basis(HX, HZ), "z"), (HZ, logical_basis(HZ, HX), "x")):
        hr, hc = dense_to_csr(Hm)
        ar, ac = dense_to_csr(Lm)
        parts.append(Problem(name=f"bb_{Hm.shape[1]}_xz_{tag}_p{p}", M=Hm.shape[0], N=Hm.shape[1], K=Lm.shape[0],
                             H_row_ptr=hr, H_col_idx=hc, A_row_ptr=ar, A_col_idx=ac,
                             priors=np.full(Hm.shape[1], q), meta={"kind": "bb_xz_part", "p": p}))
    return parts


def split_bits(packed: np.ndarray, n_total: int, n_first: int):
    """Bit vectors [B, ceil(n_total/32)] -> (first n_first bits, the rest), repacked."""
    b = unpack_bits(packed, n_total)
    return pack_bits(b[:, :n_first]), pack_bits(b[:, n_first:])


def problem_to_dem(prob: Problem) -> str:
    """The problem (H, A, p) as a text detector error model: one error line per
    column, probabilities written with 17 significant digits (exact round trip),
    then the detector and observable declarations that fix M and K."""
    Hc = [[] for _ in range(prob.N)]
    Ac = [[] for _ in range(prob.N)]
    for i in range(prob.M):
        for e in range(prob.H_row_ptr[i], prob.H_row_ptr[i + 1]):
            Hc[prob.H_col_idx[e]].append(i)
    for k in range(prob.K):
        for e in range(prob.A_row_ptr[k], prob.A_row_ptr[k + 1]):
            Ac[prob.A_col_idx[e]].append(k)
    lines = []
    for j in range(prob.N):
        t = " ".join([f"D{i}" for i in Hc[j]] + [f"L{k}" for k in Ac[j]])
        lines.append(f"error({float(prob.priors[j]):.17g}) {t}".rstrip())
    if prob.M:
        lines.append(f"detector D{prob.M - 1}")
    if prob.K:
        lines.append(f"logical_observable L{prob.K - 1}")
    return "\n".join(lines) + "\n"


def problem_from_dem_arrays(d: dict, name: str = "dem") -> Problem:
    """A Problem from the arrays of a DEM reader (M, N, K, CSR of H and A, priors)."""
    return Problem(name=name, M=int(d["M"]), N=int(d["N"]), K=int(d["K"]),
                   H_row_ptr=np.asarray(d["H_row_ptr"], np.int32), H_col_idx=np.asarray(d["H_col_idx"], np.int32),
                   A_row_ptr=np.asarray(d["A_row_ptr"], np.int32), A_col_idx=np.asarray(d["A_col_idx"], np.int32),
                   priors=np.asarray(d["priors"], np.float64), meta={"kind": "dem"})


def bb72_code_capacity(p: float = 0.03) -> Problem:
    """[[72,12,6]] BB code (l = m = 6), i.i.d. Z flips with probability p."""
    return bb_code_capacity(6, 6, p, name=f"bb72_cc_p{p}")


def bb144_code_capacity(p: float = 0.03) -> Problem:
    """[[144,12,12]] BB code (l = 12, m = 6), i.i.d. Z flips with probability p."""
    return bb_code_capacity(12, 6, p, name=f"bb144_cc_p{p}")


def bb_phenomenological(l: int = 12, m: int = 6, T: int = 12, p: float = 2e-3,
                        q: float | None = None) -> Problem:
    """Phenomenological detector error model of a BB code.

    T noisy syndrome rounds followed by one perfect round: detectors
    (r, c), r = 0..T, are m_r(c) xor m_{r-1}(c) with m_{-1} = 0; a data error
    (r, qb), r < T, flips detectors (r, c) for every check c touching qubit qb;
    a measurement error (r, c), r < T, flips (r, c) and (r+1, c).  Indexing:
    detector r*Mc + c, data column r*Nq + qb, measurement column T*Nq + r*Mc + c.
    The observables of a data column are the logical rows of its qubit;
    measurement columns flip none.
    """
    q = p if q is None else q
    HX, HZ = bb_matrices(l, m, BB_A_TERMS, BB_B_TERMS)
    L = logical_basis(HX, HZ)
    Mc, Nq = HX.shape
    K = L.shape[0]
    M = Mc * (T + 1)
    N = Nq * T + Mc * T
    rows_of_col = []
    for r in range(T):
        for qb in range(Nq):
            rows_of_col.append([r * Mc + c for c in np.nonzero(HX[:, qb])[0]])
    for r in range(T):
        for c in range(Mc):
            rows_of_col.append([r * Mc + c, (r + 1) * Mc + c])
    H = np.zeros((M, N), dtype=np.uint8)
    for j, rs in enumerate(rows_of_col):
        H[rs, j] = 1
    A = np.zeros((K, N), dtype=np.uint8)
    for r in range(T):
        A[:, r * Nq:(r + 1) * Nq] = L
    priors = np.concatenate([np.full(Nq * T, float(p)), np.full(Mc * T, float(q))])
    hr, hc = dense_to_csr(H)
    ar, ac = dense_to_csr(A)
    return Problem(name=f"bb{Nq}_phenom_T{T}_p{p}_q{q}", M=M, N=N, K=K,
                   H_row_ptr=hr, H_col_idx=hc, A_row_ptr=ar, A_col_idx=ac,
                   priors=priors, meta={"kind": "phenomenological", "T": T, "p": p, "q": q})


def synthetic_dem(M: int = 936, N: int = 8800, K: int = 12, wmin: int = 2, wmax: int = 6,
                  pmin: float = 1e-5, pmax: float = 1e-3, obs_density: float = 0.05,
                  seed: int | None = None) -> Problem:
    """Circuit-shaped synthetic detector error model.

    Each column draws a weight uniformly from {wmin..wmax} and that many
    distinct detectors uniformly; priors are log-uniform on [pmin, pmax];
    each observable entry is Bernoulli(obs_density).
    """
    ss = np.random.SeedSequence([ROOT_SEED, 3, M, N] if seed is None else [ROOT_SEED, 3, seed])
    rng = np.random.default_rng(ss)
    H = np.zeros((M, N), dtype=np.uint8)
    wts = rng.integers(wmin, wmax + 1, size=N)
    for j in range(N):
        H[rng.choice(M, size=int(wts[j]), replace=False), j] = 1
    priors = np.exp(rng.uniform(np.log(pmin), np.log(pmax), size=N))
    A = (rng.random((K, N)) < obs_density).astype(np.uint8)
    hr, hc = dense_to_csr(H)
    ar, ac = dense_to_csr(A)
    return Problem(name=f"synthetic_dem_{M}x{N}", M=M, N=N, K=K,
                   H_row_ptr=hr, H_col_idx=hc, A_row_ptr=ar, A_col_idx=ac,
                   priors=priors, meta={"kind": "synthetic_dem"})


def random_ldpc(M: int, N: int, col_weight: int, p: float, seed: int, K: int = 2) -> Problem:
    """Small random LDPC problem (tests): fixed column weight, random observables."""
    rng = np.random.default_rng(np.random.SeedSequence([ROOT_SEED, 7, M, N, col_weight, seed]))
    H = np.zeros((M, N), dtype=np.uint8)
    for j in range(N):
        H[rng.choice(M, size=col_weight, replace=False), j] = 1
    A = (rng.random((K, N)) < 0.3).astype(np.uint8)
    hr, hc = dense_to_csr(H)
    ar, ac = dense_to_csr(A)
    return Problem(name=f"rand_ldpc_{M}x{N}_w{col_weight}_s{seed}", M=M, N=N, K=K,
                   H_row_ptr=hr, H_col_idx=hc, A_row_ptr=ar, A_col_idx=ac,
                   priors=np.full(N, float(p)), meta={"kind": "random_ldpc"})


def random_regular_36(M: int, p: float, seed: int, K: int = 2) -> Problem:
    """Random code with every row of degree 6 and every column of degree 3
    (N = 2 M): a random pairing of the rows' six edge slots with the columns'
    three, drawn again until no column meets a row twice."""
    N = 2 * M
    rng = np.random.default_rng(np.random.SeedSequence([ROOT_SEED, 11, M, seed]))
    while True:
        slots = np.repeat(np.arange(M), 6)
        rng.shuffle(slots)
        cols = slots.reshape(N, 3)
        if all(len(set(c.tolist())) == 3 for c in cols):
            break
    H = np.zeros((M, N), dtype=np.uint8)
    for j in range(N):
        H[cols[j], j] = 1
    A = (rng.random((K, N)) < 0.2).astype(np.uint8)
    hr, hc = dense_to_csr(H)
    ar, ac = dense_to_csr(A)
    return Problem(name=f"regular36_{M}x{N}_s{seed}", M=M, N=N, K=K, H_row_ptr=hr, H_col_idx=hc,
                   A_row_ptr=ar, A_col_idx=ac, priors=np.full(N, float(p)), meta={"kind": "random_regular_36"})


def problem_from_dense(H: np.ndarray, A: np.ndarray, priors, name: str = "dense") -> Problem:
    H = np.asarray(H, np.uint8)
    A = np.asarray(A, np.uint8).reshape(-1, H.shape[1])
    hr, hc = dense_to_csr(H)
    ar, ac = dense_to_csr(A)
    return Problem(name=name, M=H.shape[0], N=H.shape[1], K=A.shape[0],
                   H_row_ptr=hr, H_col_idx=hc, A_row_ptr=ar, A_col_idx=ac,
                   priors=np.asarray(priors, dtype=np.float64).copy(), meta={})


# ----------------------------------------------------------------------------
# shot sampling
# ----------------------------------------------------------------------------
def shot_seed(tag: str, index: int = 0) -> np.random.SeedSequence:
    """Child seed for a (workload tag, shot-range index) pair."""
    key = [ord(ch) for ch in tag]
    return np.random.SeedSequence([ROOT_SEED, index, *key])


def _col_words(prob: Problem, rows: bool):
    """Packed columns of H (rows=True) or A (rows=False): uint32[N, words]."""
    if rows:
        rp, ci, R = prob.H_row_ptr, prob.H_col_idx, prob.M
    else:
        rp, ci, R = prob.A_row_ptr, prob.A_col_idx, prob.K
    W = words(max(R, 1))
    out = np.zeros((prob.N, W), dtype=np.uint32)
    for r in range(R):
        cols = ci[rp[r]:rp[r + 1]]
        out[cols, r // 32] |= np.uint32(1) << np.uint32(r % 32)
    return out


def sample_shots(prob: Problem, B: int, seed: np.random.SeedSequence | int | str,
                 keep_errors: bool = False) -> Shots:
    """Draw B shots: e_j ~ Bernoulli(p_j) independently; s = H e, o = A e (mod 2).

    Sampling is sparse: for each column j the number of shots with e_j = 1 is
    Binomial(B, p_j), and those shots are drawn uniformly without replacement.
    """
    if isinstance(seed, str):
        seed = shot_seed(seed)
    rng = np.random.default_rng(seed)
    Hc = _col_words(prob, True)
    Ac = _col_words(prob, False)
    shot_list, col_list = [], []
    for j in range(prob.N):
        k = int(rng.binomial(B, prob.priors[j]))
        if k:
            shot_list.append(rng.choice(B, size=k, replace=False).astype(np.int64))
            col_list.append(np.full(k, j, dtype=np.int64))
    synd = np.zeros((B, Hc.shape[1]), dtype=np.uint32)
    obs = np.zeros((B, Ac.shape[1]), dtype=np.uint32)
    errs = np.zeros((B, words(prob.N)), dtype=np.uint32) if keep_errors else None
    if shot_list:
        sh = np.concatenate(shot_list)
        co = np.concatenate(col_list)
        for w in range(Hc.shape[1]):
            np.bitwise_xor.at(synd[:, w], sh, Hc[co, w])
        for w in range(Ac.shape[1]):
            np.bitwise_xor.at(obs[:, w], sh, Ac[co, w])
        if keep_errors:
            np.bitwise_or.at(errs, (sh, co // 32), (np.uint32(1) << (co % 32).astype(np.uint32)))
    return Shots(syndromes=synd, obs=obs, errors=errs)


def syndrome_of(prob: Problem, e_bits: np.ndarray) -> np.ndarray:
    """Dense (H e) mod 2 for uint8 e[..., N]."""
    return (e_bits.astype(np.int64) @ prob.H_dense().T.astype(np.int64)) % 2


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
WORKLOADS = {
    # [[72,12,6]] BB, code capacity p = 0.03, beam width 8, 10^4 shots
    "bb72_cc": dict(builder=lambda p: bb72_code_capacity(p), ps=[0.03], shots=10_000),
    # [[144,12,12]] BB, code capacity p in {0.01, 0.03, 0.05}, beam width 32, 10^6 shots per p
    "bb144_cc": dict(builder=lambda p: bb144_code_capacity(p), ps=[0.01, 0.03, 0.05], shots=1_000_000),
    # [[144,12,12]] phenomenological, T = 12 + 1 perfect round, beam width 64
    "bb144_phenom": dict(builder=lambda p: bb_phenomenological(12, 6, 12, p, p),
                         ps=[1e-3, 2e-3, 3e-3], shots=100_000),
    # synthetic circuit-shaped DEM 936 x 8800
    "synthetic_dem": dict(builder=lambda p: synthetic_dem(), ps=[None], shots=1_000_000),
}
