"""Strength function on the GPU (bs_strength) against the FP64 oracle's block
strength function (Sec. "Generating strength function distributions",
Sec. "Block strength function").

  * FP64, sd 4p4n (dim 28,503), k = 1 and 4, pivots of unequal norms: every
    energy and strength of T equals the oracle's from the same pivot; the
    moments sum_r E_r^p S_ir equal <w_i|H^p|w_i> of the oracle's explicit H
    for p < 2 niter.
  * FP32 k = 8, 48Cr (pf 4p4n, dim 1,963,461): the sum rules for p = 0, 1, 2
    against FP64 products H w by the library.
  * argument checks: rank-deficient pivot, n_out < 1.
"""
import numpy as np
import pytest

import oracle as O
from paper_1801_08432_gb300 import _native as N
from paper_1801_08432_gb300 import inputs as I

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sd44():
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 4, 4, 0, +1, device=0)
    o = O.Oracle(orbits, 4, 4, 0, 0).set_interaction(spe, tb)
    return c, o


def scaled_pivot(dim, k, seed):
    return I.random_block(dim, k, seed=seed) * np.array([1.0, 2.5, 0.3, 1.7, 0.9, 1.1, 3.0, 0.5][:k])


@pytest.mark.gpu
@pytest.mark.parametrize("k,niter", [(1, 12), (4, 6)])
def test_fp64_strength_equals_oracle_and_moments(sd44, k, niter):
    c, o = sd44
    W0 = scaled_pivot(o.dim, k, 11)
    E_o, S_o = o.strength(W0, niter)
    n_out = niter * k
    E, S, rep = c.strength(torch.from_numpy(W0).cuda(), k, N.BS_F64, niter, n_out)
    assert rep["iterations"] == niter
    assert np.max(np.abs(E - E_o)) < 1e-8
    norms = (W0 * W0).sum(axis=0)
    assert np.max(np.abs(S - S_o) / norms[:, None]) < 1e-9
    H = o.matrix()
    HpW = W0.copy()
    for p in range(2 * niter):
        ref = np.einsum("ai,ai->i", W0, HpW)
        got = (S * E ** p).sum(axis=1)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-9, p
        HpW = H @ HpW
    c.sync_status()


@pytest.mark.gpu
def test_fp32_strength_48cr_sum_rules():
    orbits, spe, tb = I.space("pf")
    c = N.make(orbits, spe, tb, 4, 4, 0, +1, device=0)
    k, niter = 8, 40
    W0 = torch.from_numpy(scaled_pivot(c.dim, k, 12)).cuda()
    E, S, rep = c.strength(W0.float(), k, N.BS_F32, niter, niter * k)
    assert np.all(np.isfinite(E)) and np.all(S >= 0)
    # <w|w>, <w|H|w>, <w|H^2|w> = |H w|^2 with FP64 products by the library
    Wd = W0.float().double().contiguous()   # the FP32 pivot the run saw, in FP64
    HW = torch.empty_like(Wd)
    c.apply_H(Wd, HW, k, N.BS_F64)
    m0 = (Wd * Wd).sum(dim=0).cpu().numpy()
    m1 = (Wd * HW).sum(dim=0).cpu().numpy()
    m2 = (HW * HW).sum(dim=0).cpu().numpy()
    for p, ref in ((0, m0), (1, m1), (2, m2)):
        got = (S * E ** p).sum(axis=1)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 2e-5, (p, got, ref)
    c.sync_status()


@pytest.mark.gpu
def test_strength_argument_checks(sd44):
    c, o = sd44
    W0 = scaled_pivot(o.dim, 4, 13)
    W0[:, 3] = W0[:, 1]                       # rank-deficient pivot block
    with pytest.raises(N.BSError) as e:
        c.strength(torch.from_numpy(W0).cuda(), 4, N.BS_F64, 5, 10)
    assert e.value.code == -1
    with pytest.raises(N.BSError) as e:
        c.strength(torch.from_numpy(scaled_pivot(o.dim, 1, 14)).cuda(), 1, N.BS_F64, 5, 0)
    assert e.value.code == -1
