"""<J^2> and <T^2> as operators in the interaction format
(observables.j2_operator, t2_operator) and orbit occupations from the adjoint
(observables.occupations), applied by the library's kernels.  <J^2> is
pinned against the oracle's independent route |J+ psi|^2 + M(M+1) (J+
applied by bit operations into the 2M+2 basis); T^2 against isospin
multiplet counting; occupations against finite differences of the
eigenvalue in the SPEs (Hellmann-Feynman), the particle number and the
filling of a pure one-body Hamiltonian.

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


@pytest.mark.parametrize("Z,Nn", [(2, 2), (3, 2), (3, 1)])
def test_t2_operator_spectrum_counts_isospin_multiplets(Z, Nn):
    # every isospin multiplet with T >= t has exactly one member with
    # Tz = t, so the number of states with isospin T in the basis of
    # (Z, N) is dim(Tz = T) - dim(Tz = T + 1) at the same A, 2M, parity
    orbits, spe, tb = I.space("sd")
    A, twoM = Z + Nn, (Z + Nn) % 2
    st, tt = OB.t2_operator(orbits)
    ot = O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(st, tt)
    T2 = ot.dense()
    w = np.linalg.eigvalsh(T2)
    twoT = np.rint(2 * OB.j_from_j2(w)).astype(int)
    assert np.max(np.abs(2 * OB.j_from_j2(w) - twoT)) < 1e-9

    def dim_tz(twoTz):   # 2Tz = Z' - N' >= 0, 0 if no such nucleus in the space
        Zp = (A + twoTz) // 2
        if Zp > 12 or A - Zp < 0:
            return 0
        try:
            return O.Oracle(orbits, Zp, A - Zp, twoM, 0).dim
        except O.OracleError:
            return 0

    for t2 in sorted(set(twoT)):
        assert np.sum(twoT == t2) == dim_tz(t2) - dim_tz(t2 + 2), t2
    assert min(twoT) == abs(Z - Nn)
    H = O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(spe, tb).dense()
    assert np.max(np.abs(H @ T2 - T2 @ H)) < 1e-12 * np.max(np.abs(H))   # isospin-conserving H


def test_oracle_occupations_pins():
    orbits, spe, tb = I.space("sd")
    o = O.Oracle(orbits, 2, 2, 0, 0).set_interaction(spe, tb)
    ev, X = o.eigh(3)
    n0 = o.occupations(X[:, 0])
    for m in range(3):
        assert abs(o.occupations(X[:, m]).sum() - 4.0) < 1e-12
    # Hellmann-Feynman: n_a = dE_0 / de_a, central differences on dense eigh
    h = 1e-4
    for a in range(len(orbits)):
        e = []
        for sgn in (1, -1):
            sp = list(spe)
            sp[a] += sgn * h
            e.append(O.Oracle(orbits, 2, 2, 0, 0).set_interaction(sp, tb).eigh(1)[0][0])
        assert abs((e[0] - e[1]) / (2 * h) - n0[a]) < 1e-7, a
    # one-body only: the lowest level fills the lowest orbit (0d5/2 takes 4)
    o1 = O.Oracle(orbits, 2, 2, 0, 0).set_interaction(spe, [])
    ev1, X1 = o1.eigh(1)
    assert np.allclose(o1.occupations(X1[:, 0]), [4.0, 0.0, 0.0], atol=1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("name,Z", [("sd", 4), ("pf", 4)])
def test_gpu_occupations_and_t2_of_lanczos_eigenvectors(name, Z):
    """sd 4p4n and 48Cr (pf 4p4n, dim 1,963,461), FP64 Lanczos eigenvectors:
    occupations from the adjoint equal the oracle's bit counts on the same
    vectors and sum to A; <T^2> through a T^2 context equals the oracle's
    explicit T^2 (sd) and is T(T+1) with integer T >= 0 for converged levels."""
    torch = pytest.importorskip("torch")
    from paper_1801_08432_gb300 import _native as N
    orbits, spe, tb = I.space(name)
    c = N.make(orbits, spe, tb, Z, Z, 0, +1, device=0)
    ct = OB.t2_context(orbits, Z, Z, 0, device=0)
    nkeep = 3
    p = torch.from_numpy(I.random_block(c.dim, 1, seed=I.PIVOT_SEED)).to("cuda", torch.float64)
    X = torch.zeros((c.dim, nkeep), device="cuda", dtype=torch.float64)
    ev, rep = c.lanczos(p, 1, N.BS_F64, 150, nkeep, refine=True, evecs=X)
    occ = OB.occupations(c, X, N.BS_F64)
    orc = O.Oracle(orbits, Z, Z, 0, 0)
    Xh = X.cpu().numpy()
    for m in range(nkeep):
        ref = orc.occupations(Xh[:, m])
        assert np.max(np.abs(occ[m] - ref)) < 1e-9, (m, occ[m], ref)
        assert abs(occ[m].sum() - 2 * Z) < 1e-9
    t2 = np.diag(OB.expectation(ct, X, nkeep, N.BS_F64))
    if name == "sd":
        st, tt = OB.t2_operator(orbits)
        ot = O.Oracle(orbits, Z, Z, 0, 0).set_interaction(st, tt)
        ref = np.array([Xh[:, m] @ ot.spmv(Xh[:, m]) / (Xh[:, m] @ Xh[:, m]) for m in range(nkeep)])
        assert np.max(np.abs(t2 - ref)) < 1e-9
    for m in range(nkeep):
        if rep["residual"][m] <= 1e-6:
            T = OB.j_from_j2(t2[m])
            assert abs(T - round(T)) < 1e-5
    c.close()
    ct.close()


def test_product_clebsch_gordan_matches_sympy():
    sympy = pytest.importorskip("sympy")
    from sympy.physics.wigner import clebsch_gordan as cg_exact
    H = sympy.Rational(1, 2)
    worst = 0.0
    for tj1 in range(0, 8):
        for tj2 in range(0, 8):
            for tJ in range(abs(tj1 - tj2), tj1 + tj2 + 1, 2):
                for tm1 in range(-tj1, tj1 + 1, 2):
                    for tm2 in range(-tj2, tj2 + 1, 2):
                        if abs(tm1 + tm2) > tJ:
                            continue
                        ref = float(cg_exact(tj1 * H, tj2 * H, tJ * H, tm1 * H, tm2 * H, (tm1 + tm2) * H))
                        worst = max(worst, abs(OB.clebsch_gordan(tj1, tm1, tj2, tm2, tJ, tm1 + tm2) - ref))
    assert worst < 1e-12


@pytest.mark.gpu
def test_gpu_reduced_densities_of_lanczos_eigenvectors():
    """sd 4p4n at M = 1: M-scheme densities of GPU Lanczos eigenvectors from
    bs_density, reduced by observables.reduced_densities, equal the oracle's
    reduction of its own densities of the same vectors (diagonal and
    transitions); the reduced J of every converged level is sqrt(J(J+1)(2J+1))."""
    torch = pytest.importorskip("torch")
    from paper_1801_08432_gb300 import _native as N
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 4, 4, 2, +1, device=0)
    cj = OB.j2_context(orbits, 4, 4, 2, device=0)
    nkeep = 4
    p = torch.from_numpy(I.random_block(c.dim, 1, seed=I.PIVOT_SEED)).to("cuda", torch.float64)
    X = torch.zeros((c.dim, nkeep), device="cuda", dtype=torch.float64)
    ev, rep = c.lanczos(p, 1, N.BS_F64, 200, nkeep, refine=True, evecs=X)
    assert max(rep["residual"]) < 1e-6
    J = [int(round(float(v))) for v in OB.j_from_j2(np.diag(OB.expectation(cj, X, nkeep, N.BS_F64)))]
    ns = sum(o.twoj + 1 for o in orbits)
    rho = c.density(X, X, nkeep, ns)
    Xh = X.cpu().numpy()
    orc = O.Oracle(orbits, 4, 4, 2, 0)
    for f, i in [(0, 0), (1, 1), (0, 1), (2, 3), (3, 0)]:
        got = OB.reduced_densities(rho[:, :, :, f, i], orbits, 2, 2 * J[f], 2 * J[i])
        ref = orc.reduced_density(orc.density(Xh[:, f], Xh[:, i]), 2 * J[f], 2 * J[i])
        for key, v in ref.items():
            assert np.isnan(v) == np.isnan(got[key])
            if np.isfinite(v):
                assert abs(got[key] - v) < 1e-9, (f, i, key)
    for m in range(nkeep):
        r = OB.reduced_densities(rho[:, :, :, m, m], orbits, 2, 2 * J[m], 2 * J[m])
        s = sum(np.sqrt(o.twoj / 2 * (o.twoj / 2 + 1) * (o.twoj + 1)) * (r[(0, a, a, 2)] + r[(1, a, a, 2)])
                for a, o in enumerate(orbits))
        assert abs(s - np.sqrt(J[m] * (J[m] + 1) * (2 * J[m] + 1))) < 1e-6
    c.close()
    cj.close()
