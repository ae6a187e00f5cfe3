"""<J^2> as an operator in the interaction format (observables.j2_operator),
applied by the library's kernels, pinned against the oracle's independent
route |J+ psi|^2 + M(M+1) (J+ applied by bit operations into the 2M+2 basis).

  * CPU: the J^2 table loaded into the oracle gives, for random vectors, the
    same <J^2> as the J+ route, and its explicit matrix has the eigenvalues
    J(J+1) (integer J for even A, half-integer for odd A) only.
  * GPU: <J^2> of GPU Lanczos eigenvectors, through a J^2 context on the same
    basis (H x kernels + block inner products), equals the oracle's J+ route
    on the same vectors, and is J(J+1) for the converged ones.
"""
import numpy as np
import pytest

import oracle as O
from paper_1801_08432_gb300 import inputs as I
from paper_1801_08432_gb300 import observables as OB


# (space, Z, N, 2M, parity: 0 = +, 1 = -); all p-shell orbits are odd, so
# 2p3n has negative parity
@pytest.mark.parametrize("name,Z,Nn,twoM,par", [("sd", 2, 2, 0, 0), ("sd", 2, 2, 2, 0), ("sd", 3, 2, 1, 0), ("p", 2, 3, 1, 1)])
def test_j2_operator_matches_jplus_route_and_has_jj1_spectrum(name, Z, Nn, twoM, par):
    orbits, _, _ = I.space(name)
    spe, tb = OB.j2_operator(orbits)
    oj = O.Oracle(orbits, Z, Nn, twoM, par).set_interaction(spe, tb)
    up = O.Oracle(orbits, Z, Nn, twoM + 2, par)
    assert oj.dim > 0
    rng = np.random.default_rng(3 + twoM)
    for _ in range(3):
        psi = rng.standard_normal(oj.dim)
        via_table = float(psi @ oj.spmv(psi)) / float(psi @ psi)
        assert abs(via_table - oj.j2(psi, up)) <= 1e-10 * max(1.0, abs(via_table))
    ev = np.linalg.eigvalsh(oj.dense())
    J = OB.j_from_j2(ev)
    twoJ = np.rint(2 * J)
    assert np.max(np.abs(2 * J - twoJ)) < 1e-8
    assert np.all((twoJ - twoM) % 2 == 0) and np.all(twoJ >= abs(twoM))


@pytest.mark.gpu
@pytest.mark.parametrize("twoM", [0, 2])
def test_gpu_j2_of_lanczos_eigenvectors(twoM):
    torch = pytest.importorskip("torch")
    from paper_1801_08432_gb300 import _native as N
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 4, 4, twoM, +1, device=0)
    cj = OB.j2_context(orbits, 4, 4, twoM, device=0)
    nkeep = 4
    p = torch.from_numpy(I.random_block(c.dim, 1, seed=I.PIVOT_SEED)).to("cuda", torch.float64)
    X = torch.zeros((c.dim, nkeep), device="cuda", dtype=torch.float64)
    ev, rep = c.lanczos(p, 1, N.BS_F64, 120, nkeep, refine=True, evecs=X)
    j2 = np.diag(OB.expectation(cj, X, nkeep, N.BS_F64))
    orc = O.Oracle(orbits, 4, 4, twoM, 0)
    up = O.Oracle(orbits, 4, 4, twoM + 2, 0)
    Xh = X.cpu().numpy()
    ref = np.array([orc.j2(Xh[:, m].copy(), up) for m in range(nkeep)])
    assert np.max(np.abs(j2 - ref)) <= 1e-9 * np.max(np.abs(ref))
    for m in range(nkeep):
        if rep["residual"][m] <= 1e-6:
            J = OB.j_from_j2(j2[m])
            assert abs(J - round(J)) < 1e-5 and round(J) >= twoM // 2
    c.close()
    cj.close()
