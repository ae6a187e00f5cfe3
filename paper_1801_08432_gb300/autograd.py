"""Differentiation of y = H(theta) x and of Lanczos eigenvalues w.r.t. the
interaction theta = (SPEs, TBMEs), for fitting interactions.

The products with H and their adjoints run in the library's kernels
(forward bs_apply_H, adjoint bs_apply_H_backward, Lanczos bs_lanczos); torch
supplies the tape.  The one exception is lanczos_k_loss: the dot products,
vector updates and norms of its K-step recurrence are torch operations on the
device, because the tape has to see them to differentiate through the steps
(only its H v products go through the library).  theta is a CPU float64
tensor: the SPEs (one per orbit) followed
by the TBME values in the order of the label list the operator was built
with.

* HxFunction: y = H(theta) x with the hand-written adjoint
  (gx = H gy, gtheta_t = sum gy^T dH/dtheta_t x).
* LowestEigenvalues: E_n(theta) from bs_lanczos with dE/dtheta by
  Hellmann-Feynman, dE/dtheta_t = psi^T (dH/dtheta_t) psi (the paper's
  "diagonal" two-body densities X_J(ab,cd) = dE/dV_J(ab,cd)).
* lanczos_k_loss: the lowest eigenvalue of the K-step Lanczos matrix T_K,
  differentiated through the K steps with the vectors recomputed rather than
  stored: only every ceil(sqrt(K))-th pair (v_{i-1}, v_i) is kept, and each
  segment is replayed in the backward pass (torch.utils.checkpoint).  The
  recurrence is the three-term one of Sec. "Standard Lanczos algorithm",
  steps (1)-(6), plus one local reorthogonalization against v_i and v_{i-1}
  (full reorthogonalization would make every step depend on every stored
  vector, which a recompute scheme cannot avoid storing).
"""
from __future__ import annotations

import math

import numpy as np
import torch
from torch.utils.checkpoint import checkpoint

from . import _native as N


class HamiltonianOp:
    """A bs context whose interaction follows a theta tensor."""

    def __init__(self, orbits, Z, Nn, twoM, parity, spe, tbmes, device=0):
        self.ctx = N.make(orbits, spe, tbmes, Z, Nn, twoM, parity, device=device)
        self.labels = [tuple(t[:6]) for t in tbmes]
        self.n_spe = len(spe)
        self.n_theta = self.n_spe + len(self.labels)
        self.dim = self.ctx.dim
        self._theta = np.concatenate([np.asarray(spe, dtype=np.float64), [t[6] for t in tbmes]])

    def theta0(self):
        return torch.from_numpy(self._theta.copy())

    def set_theta(self, theta):
        th = theta.detach().cpu().double().numpy()
        if not np.array_equal(th, self._theta):
            spe = th[:self.n_spe]
            tb = [(*lab, float(v)) for lab, v in zip(self.labels, th[self.n_spe:])]
            self.ctx.load_interaction(spe, tb)
            self._theta = th.copy()

    @staticmethod
    def _kind(x):
        return N.BS_F64 if x.dtype == torch.float64 else N.BS_F32

    def apply(self, x):
        y = torch.empty_like(x)
        self.ctx.apply_H(x, y, x.shape[1], self._kind(x), torch.cuda.current_stream().cuda_stream)
        return y


class HxFunction(torch.autograd.Function):
    """y = H(theta) x; x: CUDA tensor [dim][k] (float32 or float64)."""

    @staticmethod
    def forward(ctx, op, theta, x):
        op.set_theta(theta)
        x = x.contiguous()
        ctx.op = op
        ctx.save_for_backward(theta, x)
        return op.apply(x)

    @staticmethod
    def backward(ctx, gy):
        theta, x = ctx.saved_tensors
        op = ctx.op
        op.set_theta(theta)
        gy = gy.contiguous()
        gx = torch.empty_like(gy)
        need_theta = ctx.needs_input_grad[1]
        g = op.ctx.apply_H_backward(x, gy, gx, x.shape[1], op._kind(x),
                                    n_theta=op.n_theta if need_theta else None,
                                    stream=torch.cuda.current_stream().cuda_stream)
        gtheta = torch.from_numpy(g).to(theta.dtype) if need_theta else None
        return None, gtheta, gx


def hx(op, theta, x):
    return HxFunction.apply(op, theta, x)


class LowestEigenvalues(torch.autograd.Function):
    """The n lowest eigenvalues of H(theta) (FP64 Lanczos with FP64 refinement),
    differentiated by Hellmann-Feynman."""

    @staticmethod
    def forward(ctx, op, theta, n, niter, k, dtype, seed):
        op.set_theta(theta)
        rng = np.random.Generator(np.random.PCG64(seed))
        piv = torch.from_numpy(rng.standard_normal((op.dim, k))).to(
            "cuda", torch.float64 if dtype == N.BS_F64 else torch.float32)
        evecs = torch.zeros((op.dim, n), device="cuda", dtype=torch.float64)
        ev, rep = op.ctx.lanczos(piv, k, dtype, niter, n, refine=True, evecs=evecs,
                                 stream=torch.cuda.current_stream().cuda_stream)
        ctx.op = op
        ctx.save_for_backward(theta, evecs)
        ctx.report = rep
        return torch.from_numpy(ev[:n].copy())

    @staticmethod
    def backward(ctx, gE):
        theta, evecs = ctx.saved_tensors
        op = ctx.op
        op.set_theta(theta)
        gtheta = np.zeros(op.n_theta)
        for m in range(evecs.shape[1]):
            w = float(gE[m])
            if w == 0.0:
                continue
            psi = evecs[:, m:m + 1].contiguous()
            psi = psi / torch.linalg.norm(psi)
            gx = torch.empty_like(psi)
            gtheta += w * op.ctx.apply_H_backward(psi, psi, gx, 1, N.BS_F64, n_theta=op.n_theta,
                                                  stream=torch.cuda.current_stream().cuda_stream)
        return None, torch.from_numpy(gtheta).to(theta.dtype), None, None, None, None, None


def lowest_eigenvalues(op, theta, n=1, niter=200, k=1, dtype=N.BS_F64, seed=180108433):
    return LowestEigenvalues.apply(op, theta, n, niter, k, dtype, seed)


def _lanczos_segment(op, theta, v_prev, v, beta_prev, nsteps):
    """nsteps steps of the three-term recurrence with local reorthogonalization.
    Returns (alphas, betas, v_prev, v) as tensors."""
    alphas, betas = [], []
    for _ in range(nsteps):
        w = hx(op, theta, v)
        a = (v * w).sum()
        w = w - a * v - beta_prev * v_prev
        # local reorthogonalization against the two vectors the recurrence uses
        w = w - (v * w).sum() * v - (v_prev * w).sum() * v_prev
        b = torch.sqrt((w * w).sum())
        alphas.append(a)
        betas.append(b)
        v_prev, v, beta_prev = v, w / b, b
    return torch.stack(alphas), torch.stack(betas), v_prev, v


def lanczos_k_loss(op, theta, pivot, K, segment=None):
    """Lowest eigenvalue of the K x K Lanczos matrix T_K built from `pivot`
    (CUDA float64 [dim][1]), differentiable in theta; the Lanczos vectors of
    each segment of ceil(sqrt(K)) steps are recomputed in the backward pass."""
    seg = segment or max(1, int(math.ceil(math.sqrt(K))))
    v = pivot / torch.sqrt((pivot * pivot).sum())
    v_prev = torch.zeros_like(v)
    beta_prev = torch.zeros((), dtype=v.dtype, device=v.device)
    alphas, betas = [], []
    done = 0
    while done < K:
        n = min(seg, K - done)

        def run(th, vp, vv, bp, n=n):
            return _lanczos_segment(op, th, vp, vv, bp, n)

        a, b, v_prev, v = checkpoint(run, theta, v_prev, v, beta_prev, use_reentrant=False)
        alphas.append(a)
        betas.append(b)
        beta_prev = b[-1]
        done += n
    alpha = torch.cat(alphas)
    beta = torch.cat(betas)[:K - 1]
    T = torch.diag(alpha) + torch.diag(beta, 1) + torch.diag(beta, -1)
    return torch.linalg.eigvalsh(T.cpu())[0]
