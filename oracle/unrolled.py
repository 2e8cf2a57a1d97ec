"""Unrolled weighted min-sum and its training loss in plain PyTorch (CPU, float64).

TEST INFRASTRUCTURE: the reference that the GPU forward and adjoint kernels
of the unrolled decoder are compared with.  Only tests, the smoke check and
the benchmark's CPU baseline use it; it imports nothing from the product
library.  Gradients come from torch autograd on the plain forward below.

What it computes (App. A, Eqs. 1-3, with a weight per edge and iteration in
place of the constant min-sum scale):
  E_e(0)   = clamp(Lambda_j)                              e = (i, j)
  D_e(t)   = w[t-1, e] * (-1)^{s_i} * prod_{e' in N(i)\\e} sign(E_e'(t-1))
                       * min_{e' in N(i)\\e} |E_e'(t-1)|    (empty min: L_MAX)
  Lam_j(t) = Lambda_j + sum_{e in N(j)} D_e(t)             (Eq. 3)
  E_e(t)   = clamp(Lambda_j + sum_{e' in N(j)\\e} D_e'(t))  (Eq. 2, clamp to [-L_MAX, L_MAX])
  loss     = sum_{t=1..T} mean_{b,j} BCE(sigmoid(-Lam_j(t)), e_j)
           = sum_t mean_{b,j} [ e_j softplus(Lam_j(t)) + (1 - e_j) softplus(-Lam_j(t)) ]
for t = 1..T with no stopping rule.  Readings for the derivative: sign() has
zero derivative; d|x|/dx = sign(x) with 0 at 0; the minimum over the other
edges passes its derivative to the edge holding it, the lowest edge index
among equal magnitudes; a message at +-L_MAX (clamp active or exactly at the
bound) passes none.  The minimum over no other edge is the constant L_MAX.
"""
from __future__ import annotations

import numpy as np
import torch


class Tables:
    """Index tables of H (CSR edge order) for the vectorised forward."""

    def __init__(self, prob):
        rp = np.asarray(prob.H_row_ptr, np.int64)
        ci = np.asarray(prob.H_col_idx, np.int64)
        self.M, self.N = int(prob.M), int(prob.N)
        self.E = int(rp[-1])
        rdeg = np.diff(rp)
        self.rmax = max(1, int(rdeg.max()) if self.M else 1)
        # row table: [M, rmax] CSR edge ids, padding = E (a slot past the last edge)
        self.row_edges = np.full((self.M, self.rmax), self.E, np.int64)
        for i in range(self.M):
            self.row_edges[i, :rdeg[i]] = np.arange(rp[i], rp[i + 1])
        self.row_of_edge = np.repeat(np.arange(self.M), rdeg)
        self.col_of_edge = ci
        cdeg = np.bincount(ci, minlength=self.N)
        self.cmax = max(1, int(cdeg.max()) if self.N else 1)
        # column table: [N, cmax] CSR edge ids of each column in ascending row order, padding = E
        self.col_edges = np.full((self.N, self.cmax), self.E, np.int64)
        fill = np.zeros(self.N, np.int64)
        for e in range(self.E):
            j = ci[e]
            self.col_edges[j, fill[j]] = e
            fill[j] += 1
        # where edge e sits in the flattened tables
        self.row_slot = np.zeros(self.E, np.int64)
        self.col_slot = np.zeros(self.E, np.int64)
        for i in range(self.M):
            for k in range(rdeg[i]):
                self.row_slot[self.row_edges[i, k]] = i * self.rmax + k
        for j in range(self.N):
            for k in range(cdeg[j]):
                self.col_slot[self.col_edges[j, k]] = j * self.cmax + k
        p = np.asarray(prob.priors, np.float64)
        self.lam = torch.tensor(np.log((1.0 - p) / p), dtype=torch.float64)   # App. A prior LLR


def _check_pass(tab: Tables, syn_sign, Em, wt, L: float):
    """Eq. 1 with weights wt [E]: D [B, E] and the row magnitudes [B, M, rmax]."""
    B = Em.shape[0]
    row_edges = torch.as_tensor(tab.row_edges)
    eye_r = torch.eye(tab.rmax, dtype=torch.bool)
    slots_r = torch.arange(tab.rmax)
    mag = torch.cat([Em.abs(), torch.full((B, 1), float("inf"), dtype=torch.float64)], dim=1)  # padding: +inf
    sgn = torch.cat([torch.where(Em < 0, -1.0, 1.0), torch.ones(B, 1, dtype=torch.float64)], dim=1)
    R = mag[:, row_edges]                                                # [B, M, rmax]
    others = R.unsqueeze(2).expand(B, tab.M, tab.rmax, tab.rmax).masked_fill(eye_r, float("inf"))
    mval = others.detach().amin(dim=3, keepdim=True)
    # the lowest slot (= lowest edge id) among equal minima receives the derivative
    first = torch.where(others.detach() == mval, slots_r, tab.rmax).amin(dim=3, keepdim=True)
    mn = torch.gather(others, 3, first.clamp(max=tab.rmax - 1)).squeeze(3)
    mn = torch.where(torch.isinf(mn), torch.full_like(mn, L), mn)         # empty minimum: L_MAX
    par = sgn[:, row_edges].unsqueeze(2).expand(B, tab.M, tab.rmax, tab.rmax).masked_fill(eye_r, 1.0).prod(dim=3)
    wpad = torch.cat([wt, torch.zeros(1, dtype=torch.float64)])
    Dslot = wpad[row_edges] * syn_sign[:, :, None] * par * mn             # [B, M, rmax]
    return Dslot.reshape(B, -1)[:, torch.as_tensor(tab.row_slot)], R.detach()


def _error_pass(tab: Tables, D, L: float):
    """Eq. 3 posterior [B, N], the clamped Eq. 2 messages [B, E] and the
    messages before the clamp."""
    B = D.shape[0]
    eye_c = torch.eye(tab.cmax, dtype=torch.bool)
    Dpad = torch.cat([D, torch.zeros(B, 1, dtype=torch.float64)], dim=1)
    C = Dpad[:, torch.as_tensor(tab.col_edges)]                          # [B, N, cmax]
    post = tab.lam + C.sum(dim=2)
    ext = tab.lam[:, None] + C.unsqueeze(2).expand(B, tab.N, tab.cmax, tab.cmax).masked_fill(eye_c, 0.0).sum(dim=3)
    Enew = ext.reshape(B, -1)[:, torch.as_tensor(tab.col_slot)]
    Em = torch.where(Enew.abs() >= L, (torch.sign(Enew) * L).detach(), Enew)
    return post, Em, Enew


def _initial(tab: Tables, B: int, L: float):
    return torch.clamp(tab.lam[torch.as_tensor(tab.col_of_edge)], -L, L).expand(B, tab.E)


def unrolled_loss(tab: Tables, s_bits: np.ndarray, e_bits: np.ndarray, weights: torch.Tensor,
                  llr_clamp: float = 1e4, record: bool = False, iter_weights=None):
    """Loss of the unrolled decoder on B shots.

    s_bits: uint8 [B, M] syndromes; e_bits: uint8 [B, N] true errors;
    weights: float64 [T, E] (may require grad); iter_weights: optional [T]
    factors c_t of the per-iteration terms (the loss is sum_t c_t L_t; all
    ones by default).  Returns (loss, per-iteration losses [T], posteriors
    [T, B, N] if record else None)."""
    L = float(llr_clamp)
    s = torch.as_tensor(np.asarray(s_bits, np.uint8), dtype=torch.float64)
    y = torch.as_tensor(np.asarray(e_bits, np.uint8), dtype=torch.float64)
    syn_sign = 1.0 - 2.0 * s                                             # (-1)^{s_i}
    Em = _initial(tab, s.shape[0], L)
    total = torch.zeros((), dtype=torch.float64)
    per_t, traj = [], []
    for t in range(weights.shape[0]):
        D, _ = _check_pass(tab, syn_sign, Em, weights[t], L)
        post, Em, _ = _error_pass(tab, D, L)
        # BCE between sigmoid(-Lam(t)) and the true error, averaged over shots and nodes
        lt = (y * torch.nn.functional.softplus(post) + (1.0 - y) * torch.nn.functional.softplus(-post)).mean()
        total = total + (lt if iter_weights is None else float(iter_weights[t]) * lt)
        per_t.append(lt)
        if record:
            traj.append(post.detach())
    return total, torch.stack(per_t), (torch.stack(traj) if record else None)


def unrolled_grad(tab: Tables, s_bits, e_bits, weights: np.ndarray, llr_clamp: float = 1e4, iter_weights=None):
    """(loss, dloss/dweights [T, E], per-iteration losses, posteriors) in float64."""
    w = torch.tensor(np.asarray(weights, np.float64), requires_grad=True)
    loss, per_t, traj = unrolled_loss(tab, s_bits, e_bits, w, llr_clamp, record=True, iter_weights=iter_weights)
    loss.backward()
    return float(loss.detach()), w.grad.numpy().copy(), per_t.detach().numpy(), traj.numpy()


def kink_margins(tab: Tables, s_bits, weights, llr_clamp: float = 1e4):
    """Distance of the forward, as a function of the weights, from the points
    where it is not smooth: the smallest gap between the magnitudes of a row
    that decide a minimum over the other edges (min1 / min2 and min2 / min3 of
    E(t), t >= 1), the smallest |E(t)| (a sign change) and the smallest
    distance of |E(t)| from L_MAX.  Finite differences are meaningful
    only with steps well below these."""
    L = float(llr_clamp)
    with torch.no_grad():
        w = torch.as_tensor(np.asarray(weights, np.float64))
        s = torch.as_tensor(np.asarray(s_bits, np.uint8), dtype=torch.float64)
        Em = _initial(tab, s.shape[0], L)
        gap, amin, lgap = float("inf"), float("inf"), float("inf")
        for t in range(w.shape[0]):
            D, R = _check_pass(tab, 1.0 - 2.0 * s, Em, w[t], L)
            srt = R.sort(dim=2).values
            # E(0) does not depend on the weights, so ties among its magnitudes are no kink
            for k in ((1, 2) if t > 0 else ()):   # min1 vs min2, min2 vs min3
                if tab.rmax > k:
                    d = srt[:, :, k] - srt[:, :, k - 1]
                    d = d[torch.isfinite(d)]
                    if d.numel():
                        gap = min(gap, float(d.min()))
            _, Em, Enew = _error_pass(tab, D, L)
            amin = min(amin, float(Em.abs().min()))
            lgap = min(lgap, float((L - Enew.abs()).abs().min()))
    return gap, amin, lgap
