"""One-body transition densities on the GPU (bs_density) against the FP64
oracle's densities from the definition <F| a+_i a_l |X> (bit operations on
the basis).

  * sd 4p4n (dim 28,503), k = 1, 2, 4, 8 blocks of random vectors, and sd 6p6n
    (dim 93,710), k = 2: every proton and neutron entry equals the oracle's.
  * 48Cr (pf 4p4n, dim 1,963,461), Lanczos eigenvectors: the diagonal gives the
    oracle's occupations (bit counts) and the particle numbers, and
    rho_FX(i, l) = rho_XF(l, i).
"""
import numpy as np
import pytest

import oracle as O
from paper_1801_08432_gb300 import _native as N
from paper_1801_08432_gb300 import inputs as I

torch = pytest.importorskip("torch")


def ns_of(orbits):
    return sum(o.twoj + 1 for o in orbits)


@pytest.mark.gpu
@pytest.mark.parametrize("Z,k", [(4, 1), (4, 2), (4, 4), (4, 8), (6, 2)])
def test_density_equals_oracle(Z, k):
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, Z, Z, 0, +1, device=0)
    o = O.Oracle(orbits, Z, Z, 0, 0)
    rng = np.random.default_rng(50 + Z + k)
    F = rng.standard_normal((c.dim, k))
    X = rng.standard_normal((c.dim, k))
    ns = ns_of(orbits)
    rho = c.density(torch.from_numpy(F).cuda(), torch.from_numpy(X).cuda(), k, ns)
    pairs = [(f, j) for f in range(k) for j in range(k)]
    if len(pairs) > 6:
        pairs = pairs[:3] + pairs[-3:]
    for f, j in pairs:
        ref = o.density(F[:, f], X[:, j])
        got = rho[:, :, :, f, j]
        scale = np.sqrt((F[:, f] ** 2).sum() * (X[:, j] ** 2).sum())
        assert np.max(np.abs(got - ref)) <= 1e-12 * scale, (f, j)
    c.sync_status()


@pytest.mark.gpu
def test_density_48cr_occupations_and_symmetry():
    orbits, spe, tb = I.space("pf")
    c = N.make(orbits, spe, tb, 4, 4, 0, +1, device=0)
    p = torch.from_numpy(I.random_block(c.dim, 1, seed=I.PIVOT_SEED)).to("cuda", torch.float64)
    X = torch.zeros((c.dim, 2), device="cuda", dtype=torch.float64)
    ev, rep = c.lanczos(p, 1, N.BS_F64, 120, 2, refine=True, evecs=X)
    ns = ns_of(orbits)
    rho = c.density(X, X, 2, ns)
    o = O.Oracle(orbits, 4, 4, 0, 0)
    st = o.sp_states()
    Xh = X.cpu().numpy()
    nrm = (Xh * Xh).sum(axis=0)
    for m in range(2):
        r = rho[:, :, :, m, m] / nrm[m]
        assert abs(np.trace(r[0]) - 4.0) < 1e-10 and abs(np.trace(r[1]) - 4.0) < 1e-10
        n = np.zeros(len(orbits))
        for i, (a, tm) in enumerate(st):
            n[a] += r[0, i, i] + r[1, i, i]
        assert np.max(np.abs(n - o.occupations(Xh[:, m]))) < 1e-10
    # <F_f|a+_i a_l|X_j> = <X_j|a+_l a_i|F_f> for real vectors
    assert np.max(np.abs(rho - rho.transpose(0, 2, 1, 4, 3))) < 1e-12
    # transition density between two different eigenstates: traceless
    assert abs(np.trace(rho[0, :, :, 0, 1])) < 1e-9 * np.sqrt(nrm[0] * nrm[1])
    c.sync_status()
