"""Host-side logic that needs no GPU: the bench's compulsory-byte counts for
the Lanczos vector work, and the observables' operator tables and reduction
conventions."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1801_08432_gb300 import inputs as I  # noqa: E402
from paper_1801_08432_gb300 import observables as OB  # noqa: E402


def test_reorth_bytes_count_blocks():
    # iteration n: alpha (read 2, read 2 + write 1), per pass dots (n + 2)
    # and update (n + 2 read, 1 write), Gram (1), normalization (2)
    dim, k, s = 1000, 4, 4
    blk = dim * k * s
    assert bench.reorth_bytes(dim, k, s, 1, 2) == (8 + 2 * 5) * blk
    assert bench.reorth_bytes(dim, k, s, 3, 1) == sum(8 + (2 * n + 5) for n in range(3)) * blk
    # no restart: the thick-restart count is the plain one
    assert bench.reorth_bytes_thick(dim, k, s, 6, 2, 0, 2) == bench.reorth_bytes(dim, k, s, 6, 2)
    # one restart: iterations tb..niter-1 again, plus forming tb Ritz blocks
    # from niter stored ones and moving tb + 1 blocks
    one = bench.reorth_bytes_thick(dim, k, s, 6, 2, 1, 2) - bench.reorth_bytes(dim, k, s, 6, 2)
    assert one == (sum(8 + 2 * (2 * n + 5) for n in range(2, 6)) + 2 * (6 + 2) + 2 * 3) * blk


@pytest.mark.parametrize("name", ["sd", "pf", "p"])
def test_j2_and_t2_tables_cover_every_diagonal_pair_state(name):
    orbits, _, _ = I.space(name)
    labels = [t for t in I.tbme_labels(orbits) if t[:2] == t[2:4]]
    for op in (OB.j2_operator, OB.t2_operator):
        spe, tb = op(orbits)
        assert len(spe) == len(orbits)
        assert sorted(t[:6] for t in tb) == sorted(labels)
    spe, tb = OB.t2_operator(orbits)
    assert all(v == 0.75 for v in spe)
    assert {t[6] for t in tb} <= {-1.5, 0.5}
    assert all(t[6] == (-1.5 if t[5] == 0 else 0.5) for t in tb)
    spe, tb = OB.j2_operator(orbits)
    for (a, b, c, d, J, T, v) in tb:
        ja, jb = orbits[a - 1].twoj / 2.0, orbits[b - 1].twoj / 2.0
        assert v == J * (J + 1.0) - ja * (ja + 1) - jb * (jb + 1)


def test_reduced_densities_nan_where_the_coupling_vanishes():
    # at M = 0 with J_f = J_i = J, (J 0, K 0 | J 0) = 0 for odd K: those
    # reduced densities are undefined at this M and come back as NaN
    orbits, _, _ = I.space("sd")
    ns = sum(o.twoj + 1 for o in orbits)
    rho = np.random.default_rng(1).standard_normal((2, ns, ns))
    r = OB.reduced_densities(rho, orbits, 0, 4, 4)
    for (t, a, b, twoK), v in r.items():
        assert np.isnan(v) == ((twoK // 2) % 2 == 1), (a, b, twoK)
    # at M = 1 with J = 2 every K <= 2J = 4 is defined (odd K too); only
    # K = 5 (0d5/2 with itself or 0d3/2) breaks the triangle with J = 2
    r1 = OB.reduced_densities(rho, orbits, 2, 4, 4)
    for (t, a, b, twoK), v in r1.items():
        assert np.isnan(v) == (twoK > 8), (a, b, twoK)


def test_isospin_densities_equal_the_oracle():
    # the product's conversion (own Clebsch-Gordan) against the oracle's on
    # the same reduced proton-neutron densities: levels and transitions of
    # sd 3p2n (T_z = 1/2) and sd 2p2n (T_z = 0)
    import oracle as O
    orbits, spe, tb = I.space("sd")
    t2 = ([0.75] * len(orbits),
          [(a, b, c, d, J, T, T * (T + 1.0) - 1.5) for (a, b, c, d, J, T) in I.tbme_labels(orbits) if (a, b) == (c, d)])
    for Z, Nn, twoM in ((3, 2, 1), (2, 2, 0)):
        o = O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(spe, tb)
        up = O.Oracle(orbits, Z, Nn, twoM + 2, 0)
        ot = O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(*t2)
        ev, X = o.eigh(4)
        twoJ = [int(round(2 * O.j_from_j2(o.j2(X[:, m], up)))) for m in range(4)]
        twoT = [int(round(2 * O.j_from_j2(X[:, m] @ ot.spmv(X[:, m])))) for m in range(4)]
        for f, i in [(0, 0), (1, 1), (0, 1), (2, 3)]:
            red = o.reduced_density(o.density(X[:, f], X[:, i]), twoJ[f], twoJ[i])
            ref = o.isospin_density(red, twoT[f], twoT[i])
            got = OB.isospin_densities(red, Z, Nn, twoT[f], twoT[i])
            assert set(ref) == set(got)
            for key, v in ref.items():
                assert np.isnan(v) == np.isnan(got[key])
                if np.isfinite(v):
                    assert abs(got[key] - v) < 1e-12, key


def test_embed_single_orbit_eigenvectors_into_the_sd_space():
    # the sd H restricted to states with every nucleon in 0d5/2 is the
    # single-orbit H (see the W-truncation pins), so an embedded eigenvector
    # of the 0d5/2 problem keeps its norm and its energy in the sd space
    import oracle as O
    from paper_1801_08432_gb300 import _native as N
    orbits, spe, tb = I.space("sd")
    small = [orbits[0]]
    tb1 = [t for t in tb if t[:4] == (1, 1, 1, 1)]
    for Z, Nn, twoM in ((2, 2, 0), (3, 2, 1)):
        cs = N.Context(-1).build_basis(small, Z, Nn, twoM, +1)
        cb = N.Context(-1).build_basis(orbits, Z, Nn, twoM, +1)
        o1 = O.Oracle(small, Z, Nn, twoM, 0).set_interaction([spe[0]], tb1)
        ob = O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(spe, tb)
        ev, X = np.linalg.eigh(o1.dense())
        Xb = OB.embed(X[:, :4], cs, small, cb, orbits)
        H = ob.matrix()
        assert np.allclose(np.linalg.norm(Xb, axis=0), 1.0)
        rq = np.einsum("ai,ai->i", Xb, H @ Xb)
        assert np.max(np.abs(rq - ev[:4])) < 1e-11
        with pytest.raises(ValueError):
            OB.embed(X[:, :1], cs, small, cb, list(reversed(orbits)))
