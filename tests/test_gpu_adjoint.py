"""Adjoint of y = H(theta) x on the GPU (bs_apply_H_backward) against the oracle.

  * gx = H gy equals the forward product.
  * gtheta_t = gy^T (dH/dtheta_t) x for every SPE and TBME equals the oracle's
    explicit unit-parameter matrices: H_t built by the oracle from a single
    nonzero parameter (the paper's "expectation value of a Hamiltonian with
    exactly one matrix element V_J(ab,cd) = 1"), for random x, gy.
  * Hellmann-Feynman on eigenstates: Euler's identity E = sum_t theta_t dE/dtheta_t
    (H is linear in theta), sum_a dE/de_a = A, and central finite differences
    of FP64 Lanczos eigenvalues.
"""
import numpy as np
import pytest

import oracle as O
from paper_1801_08432_gb300 import _native as N
from paper_1801_08432_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def unit_oracle_matrix(orbits, Z, Nn, twoM, spe, tb, t):
    """Oracle H_t for parameter t (SPEs first, then TBMEs in list order)."""
    ns = len(spe)
    o = O.Oracle(orbits, Z, Nn, twoM, 0)
    if t < ns:
        e = np.zeros(ns)
        e[t] = 1.0
        o.set_interaction(e, [])
    else:
        a, b, c, d, J, T, _ = tb[t - ns]
        o.set_interaction(np.zeros(ns), [(a, b, c, d, J, T, 1.0)])
    return o.matrix()


@pytest.mark.parametrize("k,dtype", [(1, N.BS_F64), (2, N.BS_F64), (4, N.BS_F32)])
def test_transition_densities_sd22_all_parameters(k, dtype):
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 2, 2, 0, +1, device=0)
    dim = c.dim
    x = I.random_block(dim, k, seed=51)
    gy = I.random_block(dim, k, seed=52)
    tdt = torch.float64 if dtype == N.BS_F64 else torch.float32
    if dtype == N.BS_F32:
        x = x.astype(np.float32).astype(np.float64)
        gy = gy.astype(np.float32).astype(np.float64)
    gx = torch.empty((dim, k), device="cuda", dtype=tdt)
    g = c.apply_H_backward(dev(x, tdt), dev(gy, tdt), gx, k, dtype, n_theta=len(spe) + len(tb))
    o = O.Oracle(orbits, 2, 2, 0, 0).set_interaction(spe, tb)
    assert np.max(np.abs(gx.double().cpu().numpy() - o.spmv(gy))) <= (1e-12 if dtype == N.BS_F64 else 1e-5) * 10
    ref = np.array([np.sum(gy * (unit_oracle_matrix(orbits, 2, 2, 0, spe, tb, t) @ x))
                    for t in range(len(spe) + len(tb))])
    tol = 1e-11 if dtype == N.BS_F64 else 2e-6
    assert np.max(np.abs(g - ref)) <= tol * max(1.0, np.max(np.abs(ref))), np.max(np.abs(g - ref))


def test_transition_densities_sd44_all_slots():
    """Every one of the 66 parameter slots (3 SPEs, 63 TBMEs) at sd 4p4n
    (dim 28,503) against the oracle's unit-parameter matrix."""
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 4, 4, 0, +1, device=0)
    dim = c.dim
    x = I.random_block(dim, 1, seed=61)
    gy = I.random_block(dim, 1, seed=62)
    gx = torch.empty((dim, 1), device="cuda", dtype=torch.float64)
    g = c.apply_H_backward(dev(x), dev(gy), gx, 1, N.BS_F64, n_theta=len(spe) + len(tb))
    assert len(g) == 66
    for t in range(len(spe) + len(tb)):
        ref = float(np.sum(gy * (unit_oracle_matrix(orbits, 4, 4, 0, spe, tb, t) @ x)))
        assert abs(g[t] - ref) <= 1e-11 * max(1.0, abs(ref)), (t, g[t], ref)


def eig_grad(c, spe, tb, n_ev, niter, dtype=N.BS_F64, k=1):
    p = I.random_block(c.dim, k, seed=I.PIVOT_SEED)
    tdt = torch.float64 if dtype == N.BS_F64 else torch.float32
    evecs = torch.zeros((c.dim, n_ev), device="cuda", dtype=torch.float64)
    ev, rep = c.lanczos(dev(p, tdt), k, dtype, niter, n_ev, refine=True, evecs=evecs)
    grads = []
    for m in range(n_ev):
        psi = evecs[:, m:m + 1].contiguous()
        psi = psi / torch.linalg.norm(psi)
        gx = torch.empty_like(psi)
        grads.append(c.apply_H_backward(psi, psi, gx, 1, N.BS_F64, n_theta=len(spe) + len(tb)))
    return ev, np.array(grads), rep


def test_hellmann_feynman_identities_sd44():
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 4, 4, 0, +1, device=0)
    ev, G, rep = eig_grad(c, spe, tb, 3, 300)
    theta = np.concatenate([spe, [t[6] for t in tb]])
    for m in range(3):
        assert abs(theta @ G[m] - ev[m]) < 1e-8 * abs(ev[m])        # Euler: H linear in theta
        assert abs(np.sum(G[m][:len(spe)]) - 8.0) < 1e-9             # sum_a dE/de_a = A


@pytest.mark.parametrize("pf", [False, True])
def test_hellmann_feynman_vs_finite_differences(pf):
    name, Z, Nn = ("pf", 4, 4) if pf else ("sd", 4, 4)
    orbits, spe, tb = I.space(name)
    c = N.make(orbits, spe, tb, Z, Nn, 0, +1, device=0)
    niter = 300 if pf else 250
    ev, G, rep = eig_grad(c, spe, tb, 3, niter)
    assert max(rep["residual"]) < 1e-6
    h = 1e-4
    params = [1, len(spe) + 0, len(spe) + len(tb) // 2, len(spe) + len(tb) - 1]
    for t in params:
        vals = []
        for s in (+1, -1):
            sp = list(spe)
            tbb = list(tb)
            if t < len(spe):
                sp[t] += s * h
            else:
                a, b, cc, d, J, T, v = tbb[t - len(spe)]
                tbb[t - len(spe)] = (a, b, cc, d, J, T, v + s * h)
            c.load_interaction(sp, tbb)
            e, r = c.lanczos(dev(I.random_block(c.dim, 1, seed=I.PIVOT_SEED)), 1, N.BS_F64, niter, 3, refine=True)
            vals.append(e)
        fd = (vals[0] - vals[1]) / (2 * h)
        for m in range(3):
            assert abs(fd[m] - G[m][t]) <= 1e-5 * max(1.0, abs(G[m][t])), (t, m, fd[m], G[m][t])
    c.load_interaction(spe, tb)


def test_48cr_gradients_fp64_and_fp32_vectors_vs_finite_differences():
    """The differentiation workload: pf 4p4n (48Cr, dim 1,963,461), dE/dtheta of
    the 3 lowest levels over 4 SPEs + 195 TBMEs, against central finite
    differences (h = 1e-4 MeV) of FP64 Lanczos eigenvalues for 14 parameters
    (every SPE and 10 seeded random TBME slots).  Gradients are accumulated
    in FP64 from (a) FP64 Ritz vectors (relative error <= 1e-5) and (b) Ritz
    vectors of FP32 block Lanczos with k = 4, combined in FP64 (the FP32 path
    of the configuration), whose error is first order in the vector error:
    it is held to 10 (r / gap) relative, r the level's FP64 residual and gap
    its distance to the nearest other level, and at most 1e-3."""
    orbits, spe, tb = I.space("pf")
    c = N.make(orbits, spe, tb, 4, 4, 0, +1, device=0)
    ev64, G64, rep64 = eig_grad(c, spe, tb, 3, 300)
    assert max(rep64["residual"]) < 1e-6
    ev32, G32, rep32 = eig_grad(c, spe, tb, 3, 100, dtype=N.BS_F32, k=4)
    r32 = np.array(rep32["residual"][:3])
    ev5 = c.lanczos(dev(I.random_block(c.dim, 1, seed=I.PIVOT_SEED)), 1, N.BS_F64, 300, 5, refine=True)[0]
    gap = np.array([np.min(np.abs(np.delete(ev5, m) - ev5[m])) for m in range(3)])
    rng = np.random.default_rng(48)
    nsp = len(spe)
    params = list(range(nsp)) + sorted(rng.choice(np.arange(nsp, nsp + len(tb)), 10, replace=False).tolist())
    h = 1e-4
    worst32 = np.zeros(3)
    for t in params:
        vals = []
        for sgn in (+1, -1):
            sp, tbb = list(spe), list(tb)
            if t < nsp:
                sp[t] += sgn * h
            else:
                a, b, cc, d, J, T, v = tbb[t - nsp]
                tbb[t - nsp] = (a, b, cc, d, J, T, v + sgn * h)
            c.load_interaction(sp, tbb)
            e, _ = c.lanczos(dev(I.random_block(c.dim, 1, seed=I.PIVOT_SEED)), 1, N.BS_F64, 300, 3, refine=True)
            vals.append(e)
        fd = (vals[0] - vals[1]) / (2 * h)
        for m in range(3):
            scale = max(1.0, abs(fd[m]))
            assert abs(fd[m] - G64[m][t]) <= 1e-5 * scale, (t, m, fd[m], G64[m][t])
            worst32[m] = max(worst32[m], abs(fd[m] - G32[m][t]) / scale)
    c.load_interaction(spe, tb)
    print("48Cr FP32 k=4 vectors: worst relative gradient error per level", worst32, "residuals", r32, "gaps", gap)
    assert np.all(worst32 <= np.minimum(1e-3, np.maximum(1e-5, 10 * r32 / gap))), (worst32, r32, gap)
