"""Pins of the FP64 oracle to facts other than itself.

Each test ties one part of the oracle to something the paper or mathematics
fixes, so that a dropped term, a wrong phase or a transposed index fails:

  * Clebsch-Gordan: sympy's exact routine, orthogonality;
  * sign rule: the paper's worked bitstring examples (Sec. "Representation of
    the basis");
  * basis: dimensions and SD/sector counts printed in the paper
    (tests/golden/basis_dims.txt), Table al27 row by row
    (tests/golden/al27_sectors.txt), brute-force enumeration;
  * decoupling, TBME phases, pn isospin combination (Eq. xpndef), sign rule:
    one proton + one neutron gives exactly the union over (J,T) of the coupled
    two-body channel spectra; two like particles give the T=1 channels;
  * SPE path: with no TBMEs the spectrum is the multiset of SPE sums;
  * rotational invariance of the whole chain: eig(M=1) inside eig(M=0) and
    integer J from <J^2> = |J+ psi|^2 + M(M+1);
  * assembly: H = H^T, trace from occupation counts, reading in any label order;
  * products: the on-the-fly rows (apply_rows, k = 1 and 4, and the |H| |x|
    bound) equal rows of the explicit matrix times x, and spmv (k = 1, 2, 4,
    8) and its sampled-row form (spmv_rows) equal the matrix times x, on sd
    4p4n M = 0 and M = 1 and sd 5p6n,
    random rows plus the first and last rows of every block and of its
    proton rows (the row path is the checker of the large-space GPU tests);
  * Lanczos: dense diagonalization;
  * thick-restart block Lanczos: T = Q^T H Q after restarts, convergence to
    dense, Ritz values that never rise, the no-restart limit, the targeted
    run's levels nearest the target;
  * strength function: the Lanczos moment identities, converged overlaps;
  * one-body densities: the independent J+ route, occupations, particle
    numbers; reduced densities: K = 0 occupations, the reduced J, M
    independence, the transition symmetry;
  * W truncation: the single-orbit limit, rotational invariance, the
    untruncated limit.
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O
from paper_1801_08432_gb300 import inputs as I
from tests.helpers import channel_spectrum, match_subset, scrambled_tbmes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- CG
def test_cg_matches_sympy():
    sympy = pytest.importorskip("sympy")
    from sympy.physics.wigner import clebsch_gordan
    H = sympy.Rational(1, 2)
    worst = 0.0
    for tj1 in range(1, 8, 2):
        for tj2 in range(1, 8, 2):
            for tJ in range(abs(tj1 - tj2), tj1 + tj2 + 1, 2):
                for tm1 in range(-tj1, tj1 + 1, 2):
                    for tm2 in range(-tj2, tj2 + 1, 2):
                        tM = tm1 + tm2
                        if abs(tM) > tJ:
                            continue
                        ref = float(clebsch_gordan(tj1 * H, tj2 * H, tJ * H, tm1 * H, tm2 * H, tM * H))
                        worst = max(worst, abs(O.cg(tj1, tm1, tj2, tm2, tJ, tM) - ref))
    assert worst < 1e-13


def test_cg_orthogonality():
    for tj1, tj2 in [(7, 5), (5, 5), (3, 1), (7, 7)]:
        for tM in range(-(tj1 + tj2), tj1 + tj2 + 1, 2):
            Js = [tJ for tJ in range(abs(tj1 - tj2), tj1 + tj2 + 1, 2) if abs(tM) <= tJ]
            ms = [(m1, tM - m1) for m1 in range(-tj1, tj1 + 1, 2) if abs(tM - m1) <= tj2]
            C = np.array([[O.cg(tj1, m1, tj2, m2, tJ, tM) for (m1, m2) in ms] for tJ in Js])
            assert C.shape[0] == C.shape[1]
            assert np.allclose(C @ C.T, np.eye(len(Js)), atol=1e-13)


def test_cg_closed_forms():
    # <j m j -m | 0 0> = (-1)^(j-m) / sqrt(2j+1); stretched state = 1
    for tj in (1, 3, 5, 7):
        for tm in range(-tj, tj + 1, 2):
            assert abs(O.cg(tj, tm, tj, -tm, 0, 0) - (-1) ** ((tj - tm) // 2) / np.sqrt(tj + 1)) < 1e-14
        assert abs(O.cg(tj, tj, 5, 5, tj + 5, tj + 5) - 1.0) < 1e-14


# ----------------------------------------------------------------- sign rule
def _m(s):
    return sum(1 << i for i, c in enumerate(s) if c == "1")


def test_sign_rule_paper_examples():
    # a_2 |110101> = -|100101> (states counted from 1 at the left)
    assert O.apply_string(_m("110101"), [("-", 1)]) == (-1, _m("100101"))
    # a_2 |100111> = 0
    assert O.apply_string(_m("100111"), [("-", 1)])[0] == 0
    # a+_3 |110001> = |110101> and a+_3 |100101> = 0: these two examples count
    # states from 0 at the left (the paper mixes the two countings).
    assert O.apply_string(_m("110001"), [("+", 3)]) == (1, _m("110101"))
    assert O.apply_string(_m("100101"), [("+", 3)])[0] == 0
    # a+_3 a+_5 a_4 a_1 |1101011> = -a+_3 a+_5 |0100011>, and the full string is negative
    assert O.apply_string(_m("1101011"), [("-", 3), ("-", 0)]) == (-1, _m("0100011"))
    sg, _ = O.apply_string(_m("1101011"), [("+", 2), ("+", 4), ("-", 3), ("-", 0)])
    assert sg == -1


# ----------------------------------------------------------------- basis
def _golden_dims():
    rows = []
    for line in open(os.path.join(GOLD, "basis_dims.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((f[0], *[int(v) for v in f[1:6]], *(None if v == "-" else int(v) for v in f[6:9])))
    return rows


@pytest.mark.parametrize("row", _golden_dims(), ids=lambda r: "%s-%dp%dn-2M%d" % (r[0], r[1], r[2], r[3]))
def test_basis_dimensions_from_paper(row):
    name, Z, N, twoM, par, dim, npsd, nnsd_used, npsec = row
    orbits, _ = I.SPACES[name]
    o = O.Oracle(orbits, Z, N, twoM, par)
    assert o.dim == dim
    B = o.basis()
    if npsd is not None:
        assert o.n_psd == npsd
    if nnsd_used is not None:
        used = sum(int(B["n_sec"][b[1]][3]) for b in B["blocks"])
        assert used == nnsd_used
    if npsec is not None:
        assert o.n_psec == npsec


def test_al27_sector_table():
    rows = [tuple(int(v) for v in l.split()) for l in open(os.path.join(GOLD, "al27_sectors.txt"))
            if l.strip() and not l.startswith("#")]
    o = O.Oracle(I.SD_ORBITS, 5, 6, 1, 0)
    B = o.basis()
    got = set()
    for (ps, ns_, off) in B["blocks"]:
        mp, _, _, cp = B["p_sec"][ps]
        mn, _, _, cn = B["n_sec"][ns_]
        got.add((int(mp), int(cp), int(mn), int(cn), int(cp * cn)))
    assert got == set(rows)
    assert sum(r[4] for r in rows) == 80115 == o.dim


def test_ne20_first_proton_sector():
    # 20Ne .bas example: first proton sector 2Jz = -8, parity +, two proton SDs
    o = O.Oracle(I.SD_ORBITS, 2, 2, 0, 0)
    B = o.basis()
    assert tuple(B["p_sec"][0][:2]) == (-8, 0) and B["p_sec"][0][3] == 2
    assert o.n_psec == 9 and o.n_psd == 66


@pytest.mark.parametrize("Z,N,twoM", [(2, 1, 1), (1, 2, -1), (3, 2, 3), (0, 2, 0), (2, 0, 2)])
def test_basis_brute_force(Z, N, twoM):
    orbits = I.SD_ORBITS
    st = [(a, tm) for a, o in enumerate(orbits) for tm in range(-o.twoj, o.twoj + 1, 2)]
    par = [orbits[a].l % 2 for a, _ in st]

    def key(c):
        return sum(st[s][1] for s in c), sum(par[s] for s in c) % 2

    states = set()
    for cp in itertools.combinations(range(len(st)), Z):
        for cn in itertools.combinations(range(len(st)), N):
            if key(cp)[0] + key(cn)[0] == twoM and (key(cp)[1] + key(cn)[1]) % 2 == 0:
                states.add((sum(1 << s for s in cp), sum(1 << s for s in cn)))
    o = O.Oracle(orbits, Z, N, twoM, 0)
    P, Nn = o.states()
    got = list(zip(P.tolist(), Nn.tolist()))
    assert len(got) == len(set(got)) == len(states)
    assert set(got) == states
    # proton index outer, neutron inner; sectors by 2M ascending; bitmask order inside
    B = o.basis()
    for s in range(o.n_psec):
        _, _, st0, c = B["p_sec"][s]
        assert np.all(np.diff(B["p_bits"][st0:st0 + c].astype(np.int64)) > 0)
    assert np.all(np.diff(B["p_sec"][:, 0] * 2 + B["p_sec"][:, 1]) > 0)


# ----------------------------------------------------------------- two-body closed forms
@pytest.mark.parametrize("name,twoM", [("sd", 0), ("sd", 2), ("pf", 0), ("pf", 4), ("p", 0)])
def test_one_proton_one_neutron_closed_form(name, twoM):
    orbits, spe, tb = I.space(name)
    o = O.Oracle(orbits, 1, 1, twoM, 0)
    o.set_interaction(spe, tb)
    ev = np.linalg.eigvalsh(o.dense())
    ref = []
    jmax = max(x.twoj for x in orbits)
    for T in (0, 1):
        for J in range(abs(twoM) // 2, jmax + 1):
            ref.extend(channel_spectrum(orbits, spe, tb, J, T))
    ref = np.sort(ref)
    assert len(ref) == o.dim
    assert np.max(np.abs(ev - ref)) < 1e-11


@pytest.mark.parametrize("name,Z,N", [("sd", 2, 0), ("sd", 0, 2), ("pf", 2, 0)])
def test_two_like_particles_closed_form(name, Z, N):
    orbits, spe, tb = I.space(name)
    o = O.Oracle(orbits, Z, N, 0, 0)
    o.set_interaction(spe, tb)
    ev = np.linalg.eigvalsh(o.dense())
    jmax = max(x.twoj for x in orbits)
    ref = np.sort(np.concatenate([channel_spectrum(orbits, spe, tb, J, 1) for J in range(0, jmax + 1)]))
    assert len(ref) == o.dim
    assert np.max(np.abs(ev - ref)) < 1e-11


def test_one_body_only_spectrum():
    orbits, spe, _ = I.space("sd")
    o = O.Oracle(orbits, 2, 3, 1, 0)
    o.set_interaction(spe, [])
    H = o.dense()
    assert np.count_nonzero(H - np.diag(np.diag(H))) == 0
    P, Nn = o.states()
    st_e = [spe[a] for a, x in enumerate(orbits) for _ in range(x.twoj + 1)]
    ref = [sum(st_e[s] for s in range(12) if (int(p) >> s) & 1) + sum(st_e[s] for s in range(12) if (int(n) >> s) & 1)
           for p, n in zip(P, Nn)]
    assert np.allclose(np.sort(np.linalg.eigvalsh(H)), np.sort(ref), atol=1e-13)
    # lowest = best M-allowed filling
    assert abs(np.min(ref) - np.linalg.eigvalsh(H)[0]) < 1e-13


# ----------------------------------------------------------------- assembly
@pytest.fixture(scope="module")
def sd22():
    orbits, spe, tb = I.space("sd")
    o = O.Oracle(orbits, 2, 2, 0, 0).set_interaction(spe, tb)
    return o


def test_matrix_symmetric(sd22):
    H = sd22.dense()
    assert np.max(np.abs(H - H.T)) <= 1e-13 * np.max(np.abs(H))


def test_any_label_order_same_matrix(sd22):
    orbits, spe, tb = I.space("sd")
    o2 = O.Oracle(orbits, 2, 2, 0, 0).set_interaction(spe, scrambled_tbmes(tb, orbits))
    assert np.max(np.abs(o2.dense() - sd22.dense())) < 1e-13


def test_rejects_invalid_elements():
    orbits, spe, tb = I.space("sd")
    o = O.Oracle(orbits, 2, 2, 0, 0)
    for bad in [(1, 1, 1, 1, 1, 1, 1.0),     # d5/2^2 with J+T even (Pauli)
                (1, 2, 1, 2, 0, 1, 1.0),     # d5/2 s1/2 cannot couple to J=0
                (1, 1, 1, 4, 1, 0, 1.0),     # orbit 4 does not exist
                (1, 1, 1, 1, 1, 2, 1.0)]:    # T = 2
        with pytest.raises(O.OracleError):
            o.set_interaction(spe, [bad])
    with pytest.raises(O.OracleError):       # same element twice, once in another label order
        a, b, c, d, J, T, v = tb[5]
        o.set_interaction(spe, [tb[5], (c, d, a, b, J, T, v)])
    mixed = (I.Orbit(0, 2, 5), I.Orbit(0, 3, 7))
    with pytest.raises(O.OracleError):       # parity change d5/2 f7/2 -> d5/2 d5/2
        O.Oracle(mixed, 2, 0, 0, 0).set_interaction([0.0, 0.0], [(1, 2, 1, 1, 2, 1, 1.0)])


def test_trace_from_occupation_counts():
    orbits, spe, tb = I.space("sd")
    o = O.Oracle(orbits, 4, 3, 1, 0).set_interaction(spe, tb)
    wpp, wpn = o.w_tables()
    P, Nn = o.states()
    ns = o.ns
    occP = ((P[:, None] >> np.arange(ns, dtype=np.uint64)) & np.uint64(1)).astype(np.float64)
    occN = ((Nn[:, None] >> np.arange(ns, dtype=np.uint64)) & np.uint64(1)).astype(np.float64)
    st_e = np.array([spe[a] for a, x in enumerate(orbits) for _ in range(x.twoj + 1)])
    tr = st_e @ occP.sum(0) + st_e @ occN.sum(0)
    pairP = occP.T @ occP
    pairN = occN.T @ occN
    pn = occP.T @ occN
    for s in range(ns):
        for t in range(s + 1, ns):
            tr += wpp[s, t, s, t] * (pairP[s, t] + pairN[s, t])
    for i in range(ns):
        for j in range(ns):
            tr += wpn[i, j, i, j] * pn[i, j]
    assert abs(o.trace() - tr) < 1e-9 * max(1.0, abs(tr))


# ----------------------------------------------------------------- products
@pytest.fixture(scope="module", params=[(4, 4, 0), (4, 4, 2), (5, 6, 1)], ids=lambda c: "sd-%dp%dn-2M%d" % c)
def sd_product_case(request):
    Z, Nn, twoM = request.param
    orbits, spe, tb = I.space("sd")
    return O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(spe, tb)


def _boundary_rows(o, rng, n_random=3000):
    """Random rows plus the first and last rows of every block and of the first
    and last proton rows inside it."""
    B = o.basis()
    rows = set(rng.integers(0, o.dim, n_random).tolist())
    for (ps, nsi, off) in B["blocks"]:
        pc, nc = int(B["p_sec"][ps][3]), int(B["n_sec"][nsi][3])
        for ip in {0, 1, pc - 2, pc - 1}:
            if 0 <= ip < pc:
                rows.update((int(off) + ip * nc, int(off) + ip * nc + nc - 1))
    return np.array(sorted(rows), dtype=np.int64)


@pytest.mark.parametrize("k", [1, 4])
def test_apply_rows_equal_matrix_rows(sd_product_case, k):
    o = sd_product_case
    rng = np.random.default_rng(11 + k)
    rows = _boundary_rows(o, rng)
    x = rng.standard_normal((o.dim, k))
    H = o.matrix()
    ref = H[rows] @ x
    got = o.apply_rows(rows, x)
    assert got.shape == (len(rows), k)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    # the |H| |x| bound, row by row
    ref_abs = abs(H[rows]) @ np.abs(x)
    got_abs = o.apply_rows(rows, x, absval=True)
    assert np.max(np.abs(got_abs - ref_abs)) <= 1e-13 * np.max(ref_abs)
    assert np.all(got_abs >= np.abs(got) - 1e-12 * np.max(ref_abs))
    # a single vector passed as [dim] gives [nrows]
    one = o.apply_rows(rows, x[:, 0])
    assert one.shape == (len(rows),) and np.array_equal(one, got[:, 0])


@pytest.mark.parametrize("k", [1, 4])
def test_sampled_stored_rows_equal_matrix_rows(sd_product_case, k):
    o = sd_product_case
    rng = np.random.default_rng(30 + k)
    rows = _boundary_rows(o, rng, 1000)
    x = rng.standard_normal((o.dim, k))
    H = o.matrix()
    nnz = o.build_rows(rows)
    assert nnz == H[rows].nnz
    ref = H[rows] @ x
    got = o.spmv_rows(x)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_spmv_equals_matrix_product(sd_product_case, k):
    o = sd_product_case
    x = np.random.default_rng(20 + k).standard_normal((o.dim, k))
    ref = o.matrix() @ x
    got = o.spmv(x)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    if k == 1:
        assert np.max(np.abs(o.spmv(x[:, 0]) - ref[:, 0])) <= 1e-13 * np.max(np.abs(ref))


# ----------------------------------------------------------------- rotational invariance
def test_m1_spectrum_inside_m0(sd22):
    orbits, spe, tb = I.space("sd")
    o1 = O.Oracle(orbits, 2, 2, 2, 0).set_interaction(spe, tb)
    e0 = np.linalg.eigvalsh(sd22.dense())
    e1 = np.linalg.eigvalsh(o1.dense())
    worst, left = match_subset(e1, e0, 1e-9)
    assert worst < 1e-9
    assert len(left) == sd22.dim - o1.dim


def test_j2_integer(sd22):
    orbits, spe, tb = I.space("sd")
    up = O.Oracle(orbits, 2, 2, 2, 0)
    ev, X = np.linalg.eigh(sd22.dense())
    for n in range(12):
        j2 = sd22.j2(X[:, n], up)
        J = O.j_from_j2(j2)
        assert abs(J - round(J)) < 1e-8, (n, ev[n], j2)


# ----------------------------------------------------------------- Lanczos
def test_lanczos_matches_dense(sd22):
    piv = I.random_block(sd22.dim, 1)[:, 0]
    ev_l = sd22.lanczos(piv, 200, nkeep=5)
    ev_d = np.linalg.eigvalsh(sd22.dense())[:5]
    assert np.max(np.abs(ev_l - ev_d)) < 1e-9


def test_lanczos_ritz_vectors_are_eigenvectors(sd22):
    piv = I.random_block(sd22.dim, 1)[:, 0]
    ev, X = sd22.lanczos(piv, 200, nkeep=3, return_vectors=True)
    H = sd22.matrix()
    for n in range(3):
        r = H @ X[:, n] - ev[n] * X[:, n]
        assert np.linalg.norm(r) < 1e-8


# ------------------------------------------------------ thick-restart block Lanczos
@pytest.mark.parametrize("k,niter,nthick", [(1, 12, 3), (2, 8, 4), (4, 6, 8)])
def test_thick_restart_converges_to_dense(sd22, k, niter, nthick):
    piv = I.random_block(sd22.dim, k)
    ev, hist = sd22.block_lanczos_thick(piv, niter, nthick, 25, nkeep=3)
    ev_d = np.linalg.eigvalsh(sd22.dense())[:3]
    assert np.max(np.abs(ev - ev_d)) < 1e-9


@pytest.mark.parametrize("k,niter,nthick", [(1, 10, 3), (2, 7, 4), (4, 5, 8)])
def test_thick_restart_matrix_is_the_projection(sd22, k, niter, nthick):
    # the arrow-shaped T after restarts (Ritz values, coupling r = B U_last,
    # then the block-tridiagonal part) must equal Q^T H Q over the stored
    # orthonormal basis Q, whatever the restart formulas are
    piv = I.random_block(sd22.dim, k)
    for restarts in (1, 3):
        ev, hist, Q, T = sd22.block_lanczos_thick(piv, niter, nthick, restarts, return_state=True)
        H = sd22.matrix()
        assert np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1]))) < 1e-12
        assert np.max(np.abs(T - Q.T @ (H @ Q))) < 1e-11
        assert np.max(np.abs(T[:nthick, :nthick] - np.diag(np.diag(T[:nthick, :nthick])))) == 0.0


def test_thick_restart_ritz_values_never_rise(sd22):
    # the subspace after a restart contains the kept Ritz vectors, so by
    # Courant-Fischer the i-th lowest Ritz value (i < nthick) cannot rise
    piv = I.random_block(sd22.dim, 2)
    ev, hist = sd22.block_lanczos_thick(piv, 6, 4, 12)
    h = np.array([x[:4] for x in hist])
    assert np.all(np.diff(h, axis=0) <= 1e-11)
    assert np.all(h[-1] >= np.linalg.eigvalsh(sd22.dense())[:4] - 1e-11)


def test_thick_restart_without_restart_is_lanczos(sd22):
    # no restart, k = 1: the same Krylov space as the single-vector routine
    piv = I.random_block(sd22.dim, 1)
    ev_t, _ = sd22.block_lanczos_thick(piv, 15, 2, 0)
    ev_l = sd22.lanczos(piv[:, 0], 15)
    assert np.max(np.abs(ev_t - ev_l)) < 1e-10


# ------------------------------------------------------ strength function
@pytest.mark.parametrize("k,niter", [(1, 6), (3, 5)])
def test_strength_moments_equal_matrix_powers(sd22, k, niter):
    # Lanczos reproduces the moments sum_r E_r^p |<w_i|E_r>|^2 = <w_i|H^p|w_i>
    # exactly for p < 2 niter (k = 1; block: the diagonal of the moment
    # matrices), whatever the pivot's norm
    W0 = I.random_block(sd22.dim, k, seed=5) * np.array([1.0, 2.5, 0.3][:k])
    E, S = sd22.strength(W0, niter)
    H = sd22.dense()
    Hp = np.eye(sd22.dim)
    for p in range(2 * niter):
        lhs = (S * E ** p).sum(axis=1)
        rhs = np.einsum("ai,ai->i", W0, Hp @ W0)
        assert np.max(np.abs(lhs - rhs) / np.abs(rhs)) < 1e-12, p
        Hp = H @ Hp


def test_strength_converged_levels_equal_dense_overlaps(sd22):
    W0 = I.random_block(sd22.dim, 3, seed=6) * np.array([1.0, 2.5, 0.3])
    E, S = sd22.strength(W0, 60)
    ev, X = np.linalg.eigh(sd22.dense())
    assert np.max(np.abs(E[:2] - ev[:2])) < 1e-9
    assert np.max(np.abs(S[:, 0] - (X[:, 0] @ W0) ** 2)) < 1e-12


# ------------------------------------------------------ one-body densities
@pytest.mark.parametrize("name,Z,Nn,twoM,par", [("sd", 2, 3, 1, 0), ("sd", 2, 2, 0, 0), ("p", 2, 3, -1, 1)])
def test_density_contracts_to_the_jplus_route(name, Z, Nn, twoM, par):
    # <F|J+|X> = sum_ik (j+)_ik rho_FX(i, k) with (j+) = sqrt(j(j+1) - m(m+1))
    # between neighbouring m of one orbit, J+ applied by the oracle's C code
    orbits, spe, tb = I.space(name)
    o = O.Oracle(orbits, Z, Nn, twoM, par)
    up = O.Oracle(orbits, Z, Nn, twoM + 2, par)
    rng = np.random.default_rng(17 + twoM)
    X, F = rng.standard_normal(o.dim), rng.standard_normal(up.dim)
    out = np.zeros(up.dim)
    assert O.lib().orc_jplus(o.h, up.h, O._p(np.ascontiguousarray(X), O.f64p), O._p(out, O.f64p)) == 0
    rho = o.density(F, X, other=up)
    st = o.sp_states()
    jp = np.zeros((o.ns, o.ns))
    for i, (a, tm) in enumerate(st):
        for k, (b, tm2) in enumerate(st):
            if a == b and tm == tm2 + 2:
                tj = orbits[a].twoj
                jp[i, k] = 0.5 * np.sqrt((tj - tm2) * (tj + tm2 + 2.0))
    ref = float(F @ out)
    assert abs(np.sum(jp * (rho[0] + rho[1])) - ref) <= 1e-12 * max(1.0, abs(ref))


def test_density_diagonal_gives_occupations_and_particle_numbers(sd22):
    ev, X = sd22.eigh(3)
    st = sd22.sp_states()
    for m in range(3):
        rho = sd22.density(X[:, m], X[:, m])
        assert abs(np.trace(rho[0]) - 2.0) < 1e-12 and abs(np.trace(rho[1]) - 2.0) < 1e-12
        n = np.zeros(3)
        for i, (a, tm) in enumerate(st):
            n[a] += rho[0, i, i] + rho[1, i, i]
        assert np.max(np.abs(n - sd22.occupations(X[:, m]))) < 1e-12
        assert np.max(np.abs(rho - rho.transpose(0, 2, 1))) < 1e-13   # real symmetric for F = X
    # transition densities: rho_fi(i, k) = rho_if(k, i)
    r01, r10 = sd22.density(X[:, 0], X[:, 1]), sd22.density(X[:, 1], X[:, 0])
    assert np.max(np.abs(r01 - r10.transpose(0, 2, 1))) < 1e-13


# ------------------------------------------------------ reduced densities
def _levels_with_j(o, nlev):
    up = O.Oracle(o.orbits, o.Z, o.N, o.twoM + 2, o.parity)
    ev, X = o.eigh(nlev)
    J = [int(round(O.j_from_j2(o.j2(X[:, m], up)))) for m in range(nlev)]
    return ev, X, J


@pytest.fixture(scope="module")
def sd22_m1():
    orbits, spe, tb = I.space("sd")
    return O.Oracle(orbits, 2, 2, 2, 0).set_interaction(spe, tb)


def test_reduced_density_k0_is_scaled_occupation(sd22):
    # (a+ a~)_00 = n_a / [j_a], so rho_0(a+ a) = [J] n_a / [j_a] per species
    ev, X, J = _levels_with_j(sd22, 5)
    st = sd22.sp_states()
    for m in range(5):
        rho = sd22.density(X[:, m], X[:, m])
        r = sd22.reduced_density(rho, 2 * J[m], 2 * J[m])
        for t in range(2):
            for a, o in enumerate(sd22.orbits):
                n = sum(rho[t, i, i] for i, (oa, _) in enumerate(st) if oa == a)
                assert abs(r[(t, a, a, 0)] - np.sqrt(2 * J[m] + 1.0) * n / np.sqrt(o.twoj + 1.0)) < 1e-12


def test_reduced_density_k1_gives_reduced_j(sd22_m1):
    # <J||J||J> = sqrt(J(J+1)(2J+1)) = sum_a <a||j||a> (rho_1^p + rho_1^n)(a+ a),
    # <a||j||a> = sqrt(j(j+1)(2j+1)) (Edmonds); M = 1, so every J >= 1 counts
    o = sd22_m1
    ev, X, J = _levels_with_j(o, 5)
    for m in range(5):
        rho = o.density(X[:, m], X[:, m])
        r = o.reduced_density(rho, 2 * J[m], 2 * J[m])
        s = sum(np.sqrt(orb.twoj / 2 * (orb.twoj / 2 + 1) * (orb.twoj + 1)) * (r[(0, a, a, 2)] + r[(1, a, a, 2)])
                for a, orb in enumerate(o.orbits))
        assert abs(s - np.sqrt(J[m] * (J[m] + 1) * (2 * J[m] + 1))) < 1e-11, (m, J[m])


def test_reduced_density_independent_of_m(sd22, sd22_m1):
    # Wigner-Eckart: the same levels at M = 0 and M = 1 give the same rho_K
    ev0, X0, J0 = _levels_with_j(sd22, 6)
    ev1, X1, J1 = _levels_with_j(sd22_m1, 5)
    checked = 0
    for m1 in range(5):
        m0 = int(np.argmin(np.abs(ev0 - ev1[m1])))
        if abs(ev0[m0] - ev1[m1]) > 1e-8 or J0[m0] != J1[m1]:
            continue
        r0 = sd22.reduced_density(sd22.density(X0[:, m0], X0[:, m0]), 2 * J0[m0], 2 * J0[m0])
        r1 = sd22_m1.reduced_density(sd22_m1.density(X1[:, m1], X1[:, m1]), 2 * J1[m1], 2 * J1[m1])
        for key, v in r0.items():
            if np.isfinite(v) and np.isfinite(r1[key]):
                assert abs(v - r1[key]) < 1e-11, key
                checked += 1
    assert checked > 50


def test_reduced_transition_density_symmetry(sd22_m1):
    # Edmonds' convention, real states: rho^{if}_K(b+ a) =
    # (-1)^(J_f - J_i + j_a - j_b) rho^{fi}_K(a+ b); the other coupling order
    # of the Wigner-Eckart theorem would scale one side by [J_i] / [J_f]
    o = sd22_m1
    ev, X, J = _levels_with_j(o, 6)
    n = 0
    for f, i in [(0, 1), (1, 3), (0, 3), (2, 4)]:
        rfi = o.reduced_density(o.density(X[:, f], X[:, i]), 2 * J[f], 2 * J[i])
        rif = o.reduced_density(o.density(X[:, i], X[:, f]), 2 * J[i], 2 * J[f])
        for (t, a, b, tk), v in rfi.items():
            w = rif[(t, b, a, tk)]
            if np.isfinite(v) and np.isfinite(w):
                ph = (-1) ** ((J[f] - J[i]) + (o.orbits[a].twoj - o.orbits[b].twoj) // 2)
                assert abs(w - ph * v) < 1e-12
                n += 1
    assert n > 100 and len({J[0], J[1], J[3], J[4]}) > 2


def test_targeted_thick_restart_finds_levels_nearest_the_target(sd22):
    # thick restart on (H - E_bar)^2: the Ritz vectors of its lowest levels
    # are the eigenvectors of H nearest E_bar (dense diagonalization)
    ev = np.linalg.eigvalsh(sd22.dense())
    H = sd22.matrix()
    for idx, niter, restarts in ((8, 40, 60), (100, 60, 100)):
        Eb = 0.5 * (ev[idx] + ev[idx + 1]) + 0.013
        piv = I.random_block(sd22.dim, 2)
        e2, hist, X = sd22.block_lanczos_thick(piv, niter, 8, restarts, nkeep=3, return_vectors=True, target=Eb)
        rq = np.sort([X[:, m] @ (H @ X[:, m]) / (X[:, m] @ X[:, m]) for m in range(3)])
        near = np.sort(ev[np.argsort(np.abs(ev - Eb))[:3]])
        assert np.max(np.abs(rq - near)) < 1e-9
        assert np.max(np.abs(np.sort(e2) - np.sort((near - Eb) ** 2))) < 1e-9


# ------------------------------------------------------ W truncation
@pytest.mark.parametrize("Z,Nn,twoM", [(2, 2, 0), (3, 2, 1)])
def test_w_truncation_without_excitation_is_the_single_orbit_space(Z, Nn, twoM):
    # w = 0 on 0d5/2 and 1 on 1s1/2, 0d3/2, no excitation: every nucleon
    # stays in 0d5/2, so the truncated H is the single-orbit problem, built
    # independently on the orbit list (0d5/2) with its (0d5/2)^2 elements
    orbits, spe, tb = I.space("sd")
    o = O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(spe, tb)
    ev_t = np.linalg.eigvalsh(o.truncated_matrix((0, 1, 1), 0).toarray())
    tb1 = [t for t in tb if t[:4] == (1, 1, 1, 1)]
    o1 = O.Oracle([orbits[0]], Z, Nn, twoM, 0).set_interaction([spe[0]], tb1)
    ev1 = np.linalg.eigvalsh(o1.dense())
    assert len(ev_t) == len(ev1)
    assert np.max(np.abs(ev_t - ev1)) < 1e-11


def test_w_truncation_keeps_rotational_invariance():
    # w is a property of the orbit, so the truncated space is closed under
    # J+-: each M = 1 level of a truncated space is a level of the M = 0 one
    orbits, spe, tb = I.space("sd")
    o0 = O.Oracle(orbits, 2, 2, 0, 0).set_interaction(spe, tb)
    o1 = O.Oracle(orbits, 2, 2, 2, 0).set_interaction(spe, tb)
    for E in (1, 2):
        e0 = np.linalg.eigvalsh(o0.truncated_matrix((0, 1, 1), E).toarray())
        e1 = np.linalg.eigvalsh(o1.truncated_matrix((0, 1, 1), E).toarray())
        assert len(e1) < len(e0)
        worst, _ = match_subset(e1, e0, 1e-9)
        assert worst < 1e-9, (E, worst)


def test_w_truncation_limits():
    orbits, spe, tb = I.space("sd")
    o = O.Oracle(orbits, 3, 2, 1, 0).set_interaction(spe, tb)
    dims = []
    for E in range(0, 7):
        mask, w_min, e_max = o.truncation_mask((0, 1, 1), E)
        dims.append(int(mask.sum()))
    assert (w_min, e_max) == (0, 5)
    assert dims == sorted(dims) and dims[5] == dims[6] == o.dim
    full = np.linalg.eigvalsh(o.truncated_matrix((0, 1, 1), e_max).toarray())
    assert np.max(np.abs(full - np.linalg.eigvalsh(o.dense()))) < 1e-11
    # equal weights: no truncation possible
    assert o.truncation_mask((2, 2, 2), 0)[0].all()


# ------------------------------------------------------ isospin densities
def _t2_tables(orbits):
    # T^2 as SPE 3/4 and diagonal pair elements T(T+1) - 3/2 (test helper)
    return ([0.75] * len(orbits),
            [(a, b, c, d, J, T, T * (T + 1.0) - 1.5) for (a, b, c, d, J, T) in I.tbme_labels(orbits) if (a, b) == (c, d)])


def _levels_jt(Z, Nn, twoM, nlev):
    orbits, spe, tb = I.space("sd")
    o = O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(spe, tb)
    up = O.Oracle(orbits, Z, Nn, twoM + 2, 0)
    ot = O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(*_t2_tables(orbits))
    ev, X = o.eigh(nlev)
    twoJ = [int(round(2 * O.j_from_j2(o.j2(X[:, m], up)))) for m in range(nlev)]
    twoT = [int(round(2 * O.j_from_j2(X[:, m] @ ot.spmv(X[:, m])))) for m in range(nlev)]
    return o, ev, X, twoJ, twoT


@pytest.mark.parametrize("Z,Nn,twoM", [(3, 2, 1), (3, 1, 0), (2, 2, 0)])
def test_isospin_density_special_case_and_occupations(Z, Nn, twoM):
    # T_f = T_i: rho_{T=0} = [T]/sqrt2 (rho^p + rho^n), rho_{T=1} = [T]/sqrt2
    # (rho^p - rho^n) sqrt(T(T+1)) / (sqrt3 T_z); and the proton and neutron
    # occupations n = [1/2][j] / ([J][T]) 1/2 (rho_00 +- T_z sqrt3 /
    # sqrt(T(T+1)) rho_01), against bit counts
    o, ev, X, twoJ, twoT = _levels_jt(Z, Nn, twoM, 4)
    Tz = (Z - Nn) / 2.0
    st = o.sp_states()
    for m in range(4):
        T = twoT[m] / 2.0
        rho = o.density(X[:, m], X[:, m])
        red = o.reduced_density(rho, twoJ[m], twoJ[m])
        iso = o.isospin_density(red, twoT[m], twoT[m])
        for (a, b, tk, TT), v in iso.items():
            rp, rn = red[(0, a, b, tk)], red[(1, a, b, tk)]
            if not (np.isfinite(v) and np.isfinite(rp)):
                continue
            if TT == 0:
                ref = np.sqrt(twoT[m] + 1.0) / np.sqrt(2.0) * (rp + rn)
            else:
                ref = np.sqrt(twoT[m] + 1.0) / np.sqrt(2.0) * (rp - rn) * np.sqrt(T * (T + 1)) / (np.sqrt(3.0) * Tz)
            assert abs(v - ref) < 1e-12, (a, b, tk, TT)
        for a, orb in enumerate(o.orbits):
            n_p = sum(rho[0, i, i] for i, (oa, _) in enumerate(st) if oa == a)
            n_n = sum(rho[1, i, i] for i, (oa, _) in enumerate(st) if oa == a)
            pre = np.sqrt(2.0) * np.sqrt(orb.twoj + 1.0) / (np.sqrt(twoJ[m] + 1.0) * np.sqrt(twoT[m] + 1.0)) * 0.5
            r0, r1 = iso[(a, a, 0, 0)], iso[(a, a, 0, 1)]
            assert abs(2 * pre * r0 - (n_p + n_n)) < 1e-12
            if Tz != 0:
                assert abs(pre * (r0 + Tz * np.sqrt(3.0) / np.sqrt(T * (T + 1)) * r1) - n_p) < 1e-12
                assert abs(pre * (r0 - Tz * np.sqrt(3.0) / np.sqrt(T * (T + 1)) * r1) - n_n) < 1e-12


def test_isospin_transition_density_symmetry():
    # rho^{if}_{K,T}(ba) = (-1)^(j_a - j_b + J_i - J_f + T_i - T_f) rho^{fi}_{K,T}(ab)
    o, ev, X, twoJ, twoT = _levels_jt(3, 2, 1, 5)
    n = 0
    for f, i in [(0, 1), (1, 3), (0, 2), (2, 4)]:
        rfi = o.isospin_density(o.reduced_density(o.density(X[:, f], X[:, i]), twoJ[f], twoJ[i]), twoT[f], twoT[i])
        rif = o.isospin_density(o.reduced_density(o.density(X[:, i], X[:, f]), twoJ[i], twoJ[f]), twoT[i], twoT[f])
        for (a, b, tk, TT), v in rfi.items():
            w = rif[(b, a, tk, TT)]
            if np.isfinite(v) and np.isfinite(w):
                ph = (-1) ** ((o.orbits[a].twoj - o.orbits[b].twoj + twoJ[i] - twoJ[f] + twoT[i] - twoT[f]) // 2)
                assert abs(w - ph * v) < 1e-12
                n += 1
    assert n > 50
