"""Differentiable unrolled weighted min-sum on the GPU.

T flooding iterations of Eqs. 1-3 with a weight w[t][e] per edge and
iteration in place of the min-sum scale, and the loss terms
    L_t = mean_{b,j} BCE(sigmoid(-Lambda_j(t)), e_j),  loss = sum_t L_t,
computed by bsd_unrolled_forward; the gradient of an objective sum_t c_t L_t
with respect to the weights by the hand-written adjoint bsd_unrolled_backward
(checkpoints every k iterations, segments recomputed).  UnrolledLoss exposes the pair as a
torch.autograd.Function; train_weights fits the weights with Adam, and the
decoder takes the result through BeamSearchDecoder.set_weights.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import binding as B
from . import decoder as D
from . import workloads as W


def _p(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


class UnrolledTrainer:
    """Unrolled decoder for batches of B shots of one problem.

    Owns a decoder handle (H, priors, L_MAX) and the device workspace; one
    forward / backward pair at a time (the backward reads what the forward
    stored)."""

    def __init__(self, prob, batch: int, T: int = 20, ckpt_every: int = 5, device: int = 0,
                 llr_clamp: float = 1e4):
        import torch
        self.prob, self.B, self.T, self.k, self.device = prob, int(batch), int(T), int(ckpt_every), device
        self.dec = D.BeamSearchDecoder(prob, D.make_params(llr_clamp=llr_clamp, max_rounds=0,
                                                           workspace_bytes=64 << 20), device=device)
        nbytes = B.bsd_unrolled_workspace(self.dec.h, self.B, self.T, self.k)
        dev = torch.device("cuda", device)
        self.work = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.loss = torch.empty(self.T + 1, dtype=torch.float32, device=dev)
        self.generation = 0

    @property
    def n_edges(self) -> int:
        return int(self.prob.n_edges)

    def _stream(self):
        import torch
        return C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def forward(self, weights, syndromes, errors, llr=None):
        """weights float32 [T, E]; syndromes / errors int32 bit words [B, ceil(M/32)] / [B, ceil(N/32)];
        llr: optional float32 [T, B, N] output.  Returns the loss vector [T + 1] ([0] = total)."""
        for t, shape in ((weights, (self.T, self.n_edges)), (syndromes, (self.B, (self.prob.M + 31) // 32)),
                         (errors, (self.B, (self.prob.N + 31) // 32))):
            assert t.is_cuda and t.is_contiguous() and tuple(t.shape) == shape, (tuple(t.shape), shape)
        assert weights.dtype.itemsize == 4 and syndromes.element_size() == 4 and errors.element_size() == 4
        if llr is not None:
            assert llr.is_cuda and llr.is_contiguous() and tuple(llr.shape) == (self.T, self.B, self.prob.N)
        B.bsd_unrolled_forward(self.dec.h, _p(syndromes), _p(errors), self.B, self.T, self.k, _p(weights),
                               _p(self.loss), _p(llr) if llr is not None else None, _p(self.work),
                               self.work.numel(), self._stream())
        self.generation += 1
        return self.loss

    def backward(self, weights, grad_loss):
        """grad_loss: float32 CUDA tensor, the objective's derivative with respect
        to the loss vector [T + 1] of the forward ([0] the total, [t] the term of
        iteration t); one element stands for [g, 0, ..., 0].  Returns float32 [T, E]."""
        import torch
        g = grad_loss.reshape(-1).to(torch.float32)
        if g.numel() == 1:
            g = torch.cat([g, torch.zeros(self.T, dtype=torch.float32, device=g.device)])
        assert g.numel() == self.T + 1
        g = g.contiguous()
        out = torch.empty((self.T, self.n_edges), dtype=torch.float32, device=weights.device)
        B.bsd_unrolled_backward(self.dec.h, self.B, self.T, self.k, _p(weights), _p(g), _p(out), _p(self.work),
                                self.work.numel(), self._stream())
        return out

    def close(self):
        self.dec.close()


def _autograd_function():
    import torch

    class UnrolledLoss(torch.autograd.Function):
        """losses = UnrolledLoss.apply(weights, trainer, syndromes, errors): the
        loss vector [T + 1] ([0] the total, [t] the term of iteration t)."""

        @staticmethod
        def forward(ctx, weights, trainer, syndromes, errors):
            w = weights.detach().contiguous()
            loss = trainer.forward(w, syndromes, errors)
            ctx.trainer = trainer
            ctx.generation = trainer.generation
            ctx.save_for_backward(w)
            return loss.clone()

        @staticmethod
        def backward(ctx, grad_out):
            (w,) = ctx.saved_tensors
            if ctx.trainer.generation != ctx.generation:
                raise RuntimeError("the trainer ran another forward before this backward")
            return ctx.trainer.backward(w, grad_out), None, None, None

    return UnrolledLoss


_FN = None


def unrolled_loss(weights, trainer: UnrolledTrainer, syndromes, errors):
    """Differentiable loss vector of the unrolled decoder (torch.autograd):
    [0] the total over iterations, [t] the term of iteration t."""
    global _FN
    if _FN is None:
        _FN = _autograd_function()
    return _FN.apply(weights, trainer, syndromes, errors)


def batch_tensors(prob, batch: int, seed, device: int = 0):
    """A seeded batch of shots as CUDA bit-word tensors (syndromes, errors) plus the Shots record."""
    sh = W.sample_shots(prob, batch, seed, keep_errors=True)
    return D.to_torch_words(sh.syndromes, device), D.to_torch_words(sh.errors, device), sh


def train_weights(prob, T: int = 20, ckpt_every: int = 5, batch: int = 4096, steps: int = 300, lr: float = 1e-2,
                  init: float = 0.625, tag: str = "unrolled_train", device: int = 0, log_every: int = 0,
                  iter_weights=None):
    """Adam on the per-edge, per-iteration weights; a fresh seeded batch every
    step.  The objective is sum_t c_t L_t over the per-iteration loss terms,
    c = iter_weights (default all ones: the total loss).  Returns (weights
    float32 [T, E] as numpy, objective per step)."""
    import torch
    tr = UnrolledTrainer(prob, batch, T, ckpt_every, device)
    w = torch.full((T, prob.n_edges), float(init), dtype=torch.float32, device=f"cuda:{device}",
                   requires_grad=True)
    c = torch.ones(T, dtype=torch.float32, device=f"cuda:{device}") if iter_weights is None else \
        torch.as_tensor(np.asarray(iter_weights, np.float32), device=f"cuda:{device}")
    assert c.numel() == T
    opt = torch.optim.Adam([w], lr=lr)
    hist = []
    for step in range(steps):
        s, e, _ = batch_tensors(prob, batch, W.shot_seed(tag, step), device)
        opt.zero_grad(set_to_none=True)
        loss = (unrolled_loss(w, tr, s, e)[1:] * c).sum()
        loss.backward()
        opt.step()
        hist.append(float(loss.detach()))
        if log_every and step % log_every == 0:
            print(f"step {step} loss {hist[-1]:.6f}", flush=True)
    out = w.detach().cpu().numpy().astype(np.float32)
    tr.close()
    return out, hist
