"""torch.autograd patterns over the CUDA path.

  * HxFunction: gx = H gy and gtheta; L(theta) = gy . H(theta) x is linear in
    theta, so L = theta . dL/dtheta exactly (Euler).
  * LowestEigenvalues: autograd gradient equals the direct Hellmann-Feynman
    adjoint call.
  * lanczos_k_loss (K Lanczos steps, vectors recomputed in backward):
      - the forward value equals the same unrolled recurrence run in numpy on
        the oracle's explicit FP64 matrix (sd 4p4n);
      - the gradient equals central finite differences;
      - H is linear in theta and the Lanczos vectors do not change when H is
        scaled, so L(c theta) = c L(theta) and theta . dL/dtheta = L (checked
        at pf 4p4n with K = 50);
      - fewer than K vectors are alive at once (memory).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1801_08432_gb300 import _native as N
from paper_1801_08432_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_08432_gb300 import autograd as AG  # noqa: E402


def make_op(name, Z, Nn):
    orbits, spe, tb = I.space(name)
    return AG.HamiltonianOp(orbits, Z, Nn, 0, +1, spe, tb), orbits, spe, tb


def test_hx_function_gradients():
    op, orbits, spe, tb = make_op("sd", 4, 4)
    theta = op.theta0().requires_grad_(True)
    x = torch.from_numpy(I.random_block(op.dim, 2, seed=1)).cuda()
    gy = torch.from_numpy(I.random_block(op.dim, 2, seed=2)).cuda()
    xr = x.clone().requires_grad_(True)
    y = AG.hx(op, theta, xr)
    L = (gy * y).sum()
    L.backward()
    Lv = float(L.detach())
    assert abs(float((theta.detach() * theta.grad).sum()) - Lv) < 1e-10 * max(1.0, abs(Lv))
    gx_ref = op.apply(gy)
    assert torch.max(torch.abs(xr.grad - gx_ref)) < 1e-12 * torch.max(torch.abs(gx_ref))


def test_lowest_eigenvalues_gradient_is_hellmann_feynman():
    op, orbits, spe, tb = make_op("sd", 4, 4)
    theta = op.theta0().requires_grad_(True)
    E = AG.lowest_eigenvalues(op, theta, n=2, niter=250)
    comb = E[0] + 2.0 * E[1]
    comb.backward()
    g = theta.grad.numpy()
    cv, e0 = float(comb.detach()), float(E[0].detach())
    # Euler identity for the combination
    assert abs(float(theta.detach() @ theta.grad) - cv) < 1e-8 * abs(e0)
    assert abs(g[:3].sum() - 3.0 * 8.0) < 1e-8


def oracle_k_loss(o, pivot, K):
    """The same unrolled recurrence in numpy on the oracle's explicit matrix."""
    H = o.matrix()
    v = pivot / np.linalg.norm(pivot)
    vp = np.zeros_like(v)
    bp = 0.0
    al, be = [], []
    for _ in range(K):
        w = H @ v
        a = v @ w
        w = w - a * v - bp * vp
        w = w - (v @ w) * v - (vp @ w) * vp
        b = np.linalg.norm(w)
        al.append(a)
        be.append(b)
        vp, v, bp = v, w / b, b
    T = np.diag(al) + np.diag(be[:K - 1], 1) + np.diag(be[:K - 1], -1)
    return np.linalg.eigvalsh(T)[0]


def test_k_step_loss_matches_oracle_and_finite_differences():
    op, orbits, spe, tb = make_op("sd", 4, 4)
    o = O.Oracle(orbits, 4, 4, 0, 0).set_interaction(spe, tb)
    K = 20
    piv = I.random_block(op.dim, 1, seed=I.PIVOT_SEED)
    pv = torch.from_numpy(piv).cuda()
    theta = op.theta0().requires_grad_(True)
    L = AG.lanczos_k_loss(op, theta, pv, K)
    ref = oracle_k_loss(o, piv[:, 0], K)
    assert abs(float(L) - ref) < 1e-10 * abs(ref)
    L.backward()
    g = theta.grad.numpy()
    h = 1e-5
    for t in [0, 2, 5, 30, len(g) - 1]:
        th = op.theta0()
        vals = []
        for s in (1, -1):
            tp = th.clone()
            tp[t] += s * h
            with torch.no_grad():
                vals.append(float(AG.lanczos_k_loss(op, tp, pv, K)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[t]) <= 1e-5 * max(1.0, abs(g[t])), (t, fd, g[t])


def test_k50_loss_pf4p4n_euler_and_recompute_memory():
    op, orbits, spe, tb = make_op("pf", 4, 4)
    K = 50
    pv = torch.from_numpy(I.random_block(op.dim, 1, seed=I.PIVOT_SEED)).cuda()
    peaks, grads, losses = {}, {}, {}
    for seg in (None, K):     # ceil(sqrt(K))-step segments vs one segment holding all K steps
        theta = op.theta0().requires_grad_(True)
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        L = AG.lanczos_k_loss(op, theta, pv, K, segment=seg)
        L.backward()
        peaks[seg] = torch.cuda.max_memory_allocated() - base
        grads[seg] = theta.grad.numpy().copy()
        losses[seg] = float(L.detach())
        # L(c theta) = c L(theta): theta . dL/dtheta = L
        assert abs(float(theta.detach() @ theta.grad) - losses[seg]) < 1e-8 * abs(losses[seg])
    assert math.isfinite(losses[None])
    assert abs(losses[None] - losses[K]) < 1e-12 * abs(losses[K])
    assert np.max(np.abs(grads[None] - grads[K])) < 1e-9 * np.max(np.abs(grads[K]))
    # recomputing segments keeps far fewer vectors alive than replaying all K steps at once
    assert peaks[None] < 0.4 * peaks[K], (peaks[None] / (op.dim * 8), peaks[K] / (op.dim * 8))
