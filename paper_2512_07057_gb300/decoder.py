"""PyTorch-facing wrapper of the C ABI: device tensors and streams in, tensors out.

PyTorch supplies device memory and the current CUDA stream; every step of the
decoder runs in libbsd.so.  A CUDA device is required: constructing a
BeamSearchDecoder without one raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import binding as B


@dataclass
class DecodeResult:
    corrections: "object"   # torch.int32 [B, ceil(N/32)] (bit words, reinterpret as uint32)
    obs_flips: "object"     # torch.int32 [B, ceil(K/32)]
    status: "object"        # torch.int32 [B]
    iters: "object"         # torch.int32 [B]


def _words(n: int) -> int:
    return (n + 31) // 32


def make_params(preset: str | None = None, **overrides) -> B.bsd_params:
    p = B.bsd_params_preset(preset) if preset else B.bsd_params_default()
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class BeamSearchDecoder:
    """Owns one bsd_decoder handle for a problem (H, A, p)."""

    def __init__(self, prob, params: B.bsd_params, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("BeamSearchDecoder needs a CUDA device")
        B.load()
        self.device = device
        self.M, self.N, self.K = int(prob.M), int(prob.N), int(prob.K)
        hr = np.ascontiguousarray(prob.H_row_ptr, np.int32)
        hc = np.ascontiguousarray(prob.H_col_idx, np.int32)
        ar = np.ascontiguousarray(prob.A_row_ptr, np.int32)
        ac = np.ascontiguousarray(prob.A_col_idx, np.int32)
        pr = np.ascontiguousarray(prob.priors, np.float64)
        if ac.size == 0:
            ac = np.zeros(1, np.int32)
        ptr = lambda a: a.ctypes.data_as(C.c_void_p)
        self.params = params
        self.h = B.bsd_create(self.M, self.N, self.K, ptr(hr), ptr(hc), ptr(ar), ptr(ac), ptr(pr), params, device)
        self.info = B.bsd_get_info(self.h)
        self.info["batch"] = B.bsd_get_batch(self.h)

    def set_weights(self, weights) -> None:
        """Weighted min-sum: float32 [T, E] per-edge, per-iteration weights in
        place of ms_scale (CSR edge order); None returns to ms_scale."""
        if weights is None:
            B.bsd_set_weights(self.h, None, 0)
            return
        w = np.ascontiguousarray(np.asarray(weights, np.float32))
        if w.ndim != 2:
            raise ValueError("weights must be [T, E]")
        B.bsd_set_weights(self.h, w.ctypes.data_as(C.c_void_p), w.shape[0])

    def autotune(self, syndromes, stream=None) -> list:
        """Time the launch shapes on a sample batch (CUDA bit-word tensor) and keep the fastest."""
        assert syndromes.is_cuda and syndromes.is_contiguous() and syndromes.element_size() == 4
        return B.bsd_autotune(self.h, C.c_void_p(syndromes.data_ptr()), syndromes.shape[0], self._stream(stream))

    @property
    def shape(self) -> tuple:
        """(group_warps, warps_per_block) of the current launch shape."""
        return B.bsd_get_shape(self.h)

    def close(self):
        if getattr(self, "h", None):
            B.bsd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # The kernels index every buffer by shot and word with no bounds of their
    # own, so a tensor of the wrong size, type or device would be read or
    # written out of bounds: every tensor is checked before the call.
    def _check_tensor(self, t, name: str, shape: tuple) -> None:
        if tuple(t.shape) != shape:
            raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {shape}")
        if t.element_size() != 4 or t.dtype.is_floating_point:
            raise ValueError(f"{name}: dtype {t.dtype}, expected 32-bit integer words")
        if not t.is_contiguous():
            raise ValueError(f"{name}: not contiguous")
        if not t.is_cuda or t.device.index != self.device:
            raise ValueError(f"{name}: on {t.device}, expected cuda:{self.device}")

    def _check_syndromes(self, syndromes) -> int:
        if syndromes.dim() != 2:
            raise ValueError(f"syndromes: {syndromes.dim()} dimensions, expected [B, {_words(self.M)}]")
        nb = int(syndromes.shape[0])
        self._check_tensor(syndromes, "syndromes", (nb, _words(self.M)))
        return nb

    def _check_outputs(self, out: DecodeResult, nb: int) -> None:
        self._check_tensor(out.corrections, "corrections", (nb, _words(self.N)))
        self._check_tensor(out.obs_flips, "obs_flips", (nb, max(_words(self.K), 1)))
        self._check_tensor(out.status, "status", (nb,))
        if out.iters is not None:
            self._check_tensor(out.iters, "iters", (nb,))

    def _stream(self, stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return C.c_void_p(s.cuda_stream)

    def alloc_outputs(self, nshots: int) -> DecodeResult:
        import torch
        dev = torch.device("cuda", self.device)
        return DecodeResult(
            corrections=torch.empty((nshots, _words(self.N)), dtype=torch.int32, device=dev),
            obs_flips=torch.empty((nshots, max(_words(self.K), 1)), dtype=torch.int32, device=dev),
            status=torch.empty(nshots, dtype=torch.int32, device=dev),
            iters=torch.empty(nshots, dtype=torch.int32, device=dev))

    def decode(self, syndromes, out: DecodeResult | None = None, stream=None, with_iters: bool = True) -> DecodeResult:
        """syndromes: CUDA tensor [B, ceil(M/32)] of 32-bit words (int32 or uint32 bits)."""
        nb = self._check_syndromes(syndromes)
        if out is None:
            out = self.alloc_outputs(nb)
        self._check_outputs(out, nb)
        B.bsd_decode(self.h, C.c_void_p(syndromes.data_ptr()), nb, C.c_void_p(out.corrections.data_ptr()),
                     C.c_void_p(out.obs_flips.data_ptr()), C.c_void_p(out.status.data_ptr()),
                     C.c_void_p(out.iters.data_ptr()) if with_iters and out.iters is not None else None,
                     self._stream(stream))
        return out

    def decode_noalloc(self, syndromes, out: DecodeResult, stream=None) -> int:
        """bsd_decode_noalloc into caller-allocated outputs; returns the C return code."""
        nb = self._check_syndromes(syndromes)
        self._check_outputs(out, nb)
        return B.bsd_decode_noalloc(self.h, C.c_void_p(syndromes.data_ptr()), nb,
                                    C.c_void_p(out.corrections.data_ptr()), C.c_void_p(out.obs_flips.data_ptr()),
                                    C.c_void_p(out.status.data_ptr()),
                                    C.c_void_p(out.iters.data_ptr()) if out.iters is not None else None,
                                    self._stream(stream))

    def decode_host(self, syndromes: np.ndarray, stream=None) -> dict:
        """Host arrays in and out (the copies run inside the call)."""
        synd = np.ascontiguousarray(syndromes, np.uint32)
        nb = synd.shape[0]
        corr = np.zeros((nb, _words(self.N)), np.uint32)
        obs = np.zeros((nb, max(_words(self.K), 1)), np.uint32)
        status = np.zeros(nb, np.uint32)
        iters = np.zeros(nb, np.uint32)
        ptr = lambda a: a.ctypes.data_as(C.c_void_p)
        B.bsd_decode_host(self.h, ptr(synd), nb, ptr(corr), ptr(obs), ptr(status), ptr(iters), self._stream(stream))
        return dict(corrections=corr, obs=obs, status=status, iters=iters)

    def decode_host_ptrs(self, synd_ptr: int, nb: int, corr_ptr: int, obs_ptr: int, status_ptr: int,
                         iters_ptr: int | None, stream=None) -> None:
        """bsd_decode_host on caller-provided (e.g. pinned) host buffers."""
        B.bsd_decode_host(self.h, C.c_void_p(synd_ptr), nb, C.c_void_p(corr_ptr), C.c_void_p(obs_ptr),
                          C.c_void_p(status_ptr), C.c_void_p(iters_ptr) if iters_ptr else None, self._stream(stream))

    # ---- single-syndrome request loop (low latency)
    def serve_start(self, idle_ms: int = 1000) -> None:
        """Keep a request loop resident on the device (bsd_serve_start)."""
        B.bsd_serve_start(self.h, int(idle_ms))
        W = _words
        self._sv = dict(synd=np.zeros(W(self.M), np.uint32), corr=np.zeros(W(self.N), np.uint32),
                        obs=np.zeros(max(W(self.K), 1), np.uint32), status=np.zeros(1, np.uint32),
                        iters=np.zeros(1, np.uint32))
        self._svp = {k: v.ctypes.data_as(C.c_void_p) for k, v in self._sv.items()}

    def serve_decode(self, syndrome: np.ndarray) -> dict:
        """One syndrome (ceil(M/32) words) through the request loop; the same
        outputs as decode_host for B = 1."""
        sv, p = self._sv, self._svp
        sv["synd"][:] = np.asarray(syndrome, np.uint32).reshape(-1)
        B.bsd_serve_decode(self.h, p["synd"], p["corr"], p["obs"], p["status"], p["iters"])
        return dict(corrections=sv["corr"].copy(), obs=sv["obs"].copy(), status=int(sv["status"][0]),
                    iters=int(sv["iters"][0]))

    def serve_stop(self) -> None:
        B.bsd_serve_stop(self.h)

    def bp_llr(self, syndromes, T: int, stream=None):
        """Plain BP for exactly T iterations: (Lambda_j(T), sum_t Lambda_j(t)) as float32 [B, N]."""
        import torch
        nb = syndromes.shape[0]
        llr = torch.empty((nb, self.N), dtype=torch.float32, device=syndromes.device)
        sm = torch.empty((nb, self.N), dtype=torch.float32, device=syndromes.device)
        B.bsd_bp_llr(self.h, C.c_void_p(syndromes.data_ptr()), nb, T, C.c_void_p(llr.data_ptr()),
                     C.c_void_p(sm.data_ptr()), self._stream(stream))
        return llr, sm

    def sync_error(self) -> int:
        return B.bsd_sync_error(self.h)

    def profile(self, enable: bool = True) -> None:
        B.bsd_profile_enable(self.h, enable)

    def profile_read(self) -> dict:
        return B.bsd_profile_read(self.h)

    def profile_read_kinds(self) -> dict:
        return B.bsd_profile_read_kinds(self.h)


def to_torch_words(arr: np.ndarray, device: int = 0):
    """uint32 numpy words -> int32 CUDA tensor with the same bits."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr, np.uint32).view(np.int32)).to(f"cuda:{device}")


def from_torch_words(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)
