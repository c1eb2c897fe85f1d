"""Learned (neural) normalized min-sum decoding: training and logical-error-rate evaluation.

The check-node update of Algorithm 1 (Sec. 2) scales the minimum by a trained weight w[t][e] per
iteration and edge instead of one alpha.  Everything that touches the decoder runs in the
library's CUDA kernels:

* ``NMSLoss`` is a ``torch.autograd.Function`` whose forward is ``qldpc_nms_forward`` (T unrolled
  iterations, per-shot BCE of the soft outputs against the sampled error, or of the soft syndrome
  against the measured one) and whose backward is ``qldpc_nms_backward`` (the reverse sweep,
  recomputing every message from the recorded check state);
* ``NeuralMinSum`` holds the weights, the Adam state (updated by ``qldpc_adam_step``) and the
  device workspace, and trains on shots drawn on the device by ``qldpc_sample_errors``;
* ``evaluate`` decodes fresh device-sampled shots with any mix of plain and learned decoders and
  counts logical failures with ``qldpc_logical_failures``.

torch provides device memory, the autograd plumbing (the mean over shots) and streams only.
"""
from __future__ import annotations

import hashlib
import struct

import numpy as np

from . import gf2, qldpc

_MAGIC = b"QNMS"
_VERSION = 1


def _torch():
    import torch
    return torch


class NMSLoss:
    """Namespace holding the autograd Function (built lazily so importing needs no torch)."""

    _fn = None

    @classmethod
    def apply(cls, weights, graph, syndromes, targets, prior, workspace, loss_weights=None, loss: str = "error"):
        if cls._fn is None:
            torch = _torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, w, g, syn, tg, pr, ws, lw, kind):
                    out, _ = qldpc.nms_forward(g, syn, tg, pr, w.detach().contiguous(), ws, loss_weights=lw,
                                               loss=kind)
                    ctx.graph = g
                    ctx.T = int(w.shape[0])
                    ctx.lw = lw
                    ctx.kind = kind
                    ctx.save_for_backward(syn, tg, pr, ws)   # ws holds the weights and recorded state
                    return out

                @staticmethod
                def backward(ctx, grad_loss):
                    syn, tg, pr, ws = ctx.saved_tensors
                    grad = qldpc.nms_backward(ctx.graph, syn, tg, pr, ctx.T, grad_loss.float().contiguous(), ws,
                                              loss_weights=ctx.lw, loss=ctx.kind)
                    return grad, None, None, None, None, None, None, None

            cls._fn = _F
        return cls._fn.apply(weights, graph, syndromes, targets, prior, workspace, loss_weights, loss)


def code_hash(h) -> bytes:
    """SHA-256 of H's CSR arrays (row_ptr, col_idx as little-endian int32): names the code a
    checkpoint belongs to."""
    sha = hashlib.sha256()
    sha.update(np.ascontiguousarray(h.row_ptr, dtype="<i4").tobytes())
    sha.update(np.ascontiguousarray(h.col_idx, dtype="<i4").tobytes())
    return sha.digest()


class NeuralMinSum:
    """Trainable per-edge, per-iteration weights for one parity-check matrix.

    h: the CSR matrix (workloads.CSR); prior: float [n] LLRs; T: unrolled iterations;
    init: the starting weight (0.75 reproduces normalized min-sum with alpha = 0.75);
    loss_weights: per-iteration loss weights lambda_t ([T]; None: 1/T each);
    loss: "error" (BCE of sigma(-Q) against the sampled error) or "syndrome" (BCE of the soft
    syndrome against the measured one, blind to which error of a coset the outputs point at).
    """

    def __init__(self, h, prior, T: int = 20, init: float = 0.75, max_batch: int = 4096, graph=None,
                 loss_weights=None, loss: str = "error"):
        if loss not in qldpc.LOSSES:
            raise ValueError(f"unknown loss {loss!r}")
        self.loss_kind = loss
        torch = _torch()
        self.h = h
        self.graph = graph if graph is not None else qldpc.Graph.from_csr(h)
        self.T = int(T)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.prior = torch.as_tensor(np.ascontiguousarray(prior, dtype=np.float32), device=dev)
        self.weights = torch.full((self.T, self.graph.nnz), float(init), dtype=torch.float32, device=dev,
                                  requires_grad=True)
        self.exp_avg = torch.zeros_like(self.weights, requires_grad=False)
        self.exp_avg_sq = torch.zeros_like(self.weights, requires_grad=False)
        self.step = 0
        self.max_batch = int(max_batch)
        ws = qldpc.nms_workspace_bytes(self.graph, self.max_batch, self.T)
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=dev)
        self.loss_weights = None if loss_weights is None else torch.as_tensor(
            np.ascontiguousarray(loss_weights, dtype=np.float32).reshape(self.T), device=dev)

    def loss(self, syndromes, targets):
        """Per-shot losses [B] (differentiable with respect to ``weights``)."""
        if syndromes.shape[0] > self.max_batch:
            raise ValueError(f"batch {syndromes.shape[0]} exceeds max_batch {self.max_batch}")
        return NMSLoss.apply(self.weights, self.graph, syndromes, targets, self.prior, self.workspace,
                             self.loss_weights, self.loss_kind)

    def train_step(self, syndromes, targets, lr: float = 1e-3, betas=(0.9, 0.999), eps: float = 1e-8):
        """One Adam step on the mean loss of a batch; returns the mean loss (device scalar)."""
        loss = self.loss(syndromes, targets).mean()
        self.weights.grad = None
        loss.backward()
        self.step += 1
        qldpc.adam_step(self.weights.data, self.weights.grad, self.exp_avg, self.exp_avg_sq, self.step, lr,
                        betas, eps)
        return loss.detach()

    def train(self, shots: int, batch: int = 4096, p_lo: float = 0.02, p_hi: float = 0.06, seed: int = 7,
              lr: float = 1e-3, first_shot: int = 0, record_every: int = 10):
        """Train on ``shots`` device-sampled shots (rate uniform in [p_lo, p_hi) per shot).

        Returns the mean losses of every ``record_every``-th step (one host sync at the end)."""
        torch = _torch()
        steps = shots // batch
        rec = []
        for i in range(steps):
            err, syn = qldpc.sample_errors(self.graph, seed, first_shot + i * batch, batch, p_lo, p_hi)
            l = self.train_step(syn, err, lr)
            if i % record_every == 0 or i == steps - 1:
                rec.append(l)
        return torch.stack(rec).cpu().numpy() if rec else np.zeros(0, dtype=np.float32)

    def publish(self) -> None:
        """Copy the current weights into the graph for learned decoding."""
        self.graph.set_weights(self.weights.detach())

    # -- checkpoint: little-endian header + weights + Adam state ----------------------------------
    def save(self, path: str) -> None:
        header = _MAGIC + struct.pack("<I", _VERSION) + code_hash(self.h) + struct.pack(
            "<iiiiq", self.graph.m, self.graph.n, self.graph.nnz, self.T, self.step)
        with open(path, "wb") as f:
            f.write(header)
            for t in (self.weights.detach(), self.exp_avg, self.exp_avg_sq):
                f.write(t.cpu().numpy().astype("<f4").tobytes())

    def load(self, path: str) -> None:
        with open(path, "rb") as f:
            blob = f.read()
        hdr = 4 + 4 + 32 + struct.calcsize("<iiiiq")
        if blob[:4] != _MAGIC or struct.unpack("<I", blob[4:8])[0] != _VERSION:
            raise ValueError("not a learned min-sum checkpoint")
        if blob[8:40] != code_hash(self.h):
            raise ValueError("checkpoint belongs to another parity-check matrix")
        m, n, nnz, T, step = struct.unpack("<iiiiq", blob[40:hdr])
        if (m, n, nnz, T) != (self.graph.m, self.graph.n, self.graph.nnz, self.T):
            raise ValueError("checkpoint shape differs")
        count = T * nnz
        arrs = np.frombuffer(blob[hdr:], dtype="<f4")
        if arrs.size != 3 * count:
            raise ValueError("truncated checkpoint")
        torch = _torch()
        with torch.no_grad():
            for dst, k in ((self.weights, 0), (self.exp_avg, 1), (self.exp_avg_sq, 2)):
                dst.copy_(torch.from_numpy(arrs[k * count:(k + 1) * count].reshape(T, nnz).copy()))
        self.step = step


def z_logicals(code):
    """Logical operators that detect X-error residuals of a CSS code (uint8 [k, n])."""
    return gf2.logical_basis(code.hx_csr.dense(), code.hz_csr.dense())


def evaluate(graph, prior, logicals, decoders: dict, shots: int, batch: int = 65536, p_lo: float = 0.02,
             p_hi=None, seed: int = 11, first_shot: int = 0, alpha: float = 0.75, paired=()):
    """Logical error rates of several decoders on the same device-sampled shots.

    decoders: name -> (max_iter, learned).  A learned decoder uses the graph's weights and then
    plain min-sum for up to max_iter iterations.  Returns name -> dict(failures, ler, mean_iters,
    unconverged) over ``shots`` shots (rate uniform in [p_lo, p_hi), or p_lo if p_hi is None).

    paired: pairs (a, b) of decoder names compared shot by shot on the same shots.  out["paired"]
    ["a|b"] holds the discordant counts (a_only: shots a fails and b decodes, b_only: the reverse),
    the LER difference ler_a - ler_b and its 95 % confidence interval from the paired (McNemar)
    variance of the per-shot difference.
    """
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    L = torch.as_tensor(np.ascontiguousarray(logicals, dtype=np.uint8), device=dev)
    pr = torch.as_tensor(np.ascontiguousarray(prior, dtype=np.float32), device=dev)
    acc = {k: torch.zeros(3, dtype=torch.int64, device=dev) for k in decoders}
    disc = {pair: torch.zeros(2, dtype=torch.int64, device=dev) for pair in paired}
    done = 0
    while done < shots:
        b = min(batch, shots - done)
        err, syn = qldpc.sample_errors(graph, seed, first_shot + done, b, p_lo, p_hi)
        fails = {}
        for name, (max_iter, learned) in decoders.items():
            dec, iters, ok, _ = qldpc.decode(graph, syn, pr, int(max_iter), alpha, learned=bool(learned))
            fail = qldpc.logical_failures(L, err, dec, ok)
            fails[name] = fail.bool()
            acc[name] += torch.stack([fail.sum(dtype=torch.int64), iters.sum(dtype=torch.int64),
                                      (ok == 0).sum(dtype=torch.int64)])
        for (a, c) in paired:
            disc[(a, c)] += torch.stack([(fails[a] & ~fails[c]).sum(dtype=torch.int64),
                                         (fails[c] & ~fails[a]).sum(dtype=torch.int64)])
        done += b
    out = {}
    for name, a in acc.items():
        f, it, unc = (int(x) for x in a.cpu())
        out[name] = {"failures": f, "ler": f / shots, "mean_iters": it / shots, "unconverged": unc}
    if paired:
        out["paired"] = {}
        for (a, c), d in disc.items():
            n_a, n_c = (int(x) for x in d.cpu())
            diff = (n_a - n_c) / shots
            var = ((n_a + n_c) / shots - diff * diff) / shots
            half = 1.959964 * float(np.sqrt(max(var, 0.0)))
            out["paired"][f"{a}|{c}"] = {"a_only": n_a, "b_only": n_c, "ler_diff": diff,
                                         "ci95": [diff - half, diff + half]}
    return out
