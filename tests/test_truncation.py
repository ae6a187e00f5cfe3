"""W truncation (Sec. "Truncation of the many-body space") on the library's
host side, against the FP64 oracle (no GPU).

The oracle keeps the states of its full basis with W_p + W_n <= W_min +
max_excite and restricts its explicit H to them (pinned in
test_oracle_pins.py).  The library builds the truncated basis directly, with
sectors keyed by (2M, parity, W) and several conjugate neutron sectors per
proton sector; its order differs from the oracle's filtered order, so states
are matched by their (proton, neutron) bitstrings:

  * basis: the same set of states, bit for bit; every sector's W is the sum
    of its SDs' weights; sectors sorted by (2M, parity, W); blocks in the
    basis-file order (proton sector, then its conjugate neutron sectors) and
    only with W_p + W_n <= W_max; SDs sorted inside a sector;
  * tables: H x rebuilt in numpy from the exported tables (same-sector
    like-particle lists, like-particle links between blocks, pn links) equals
    the oracle's truncated H times x, for particle-hole weights in the sd and
    pf shells at 0 to 3 excitations, even and odd A, both parities.
"""
import numpy as np
import pytest

import oracle as O
from paper_1801_08432_gb300 import _native as N
from paper_1801_08432_gb300 import inputs as I
from tests.test_host_tables import tables_matvec

SD_W = (I.Orbit(0, 2, 5, 0), I.Orbit(1, 0, 1, 1), I.Orbit(0, 2, 3, 1))            # 1p-1h weights over 0d5/2
PF_W = (I.Orbit(0, 3, 7, 0), I.Orbit(1, 1, 3, 1), I.Orbit(0, 3, 5, 1), I.Orbit(1, 1, 1, 1))
SD_NMAX = (I.Orbit(0, 2, 5, 0), I.Orbit(1, 0, 1, 2), I.Orbit(0, 2, 3, 3))          # uneven weights
SPACES = {"sd": (SD_W, I.SD_SPE), "pf": (PF_W, I.PF_SPE), "sd_uneven": (SD_NMAX, I.SD_SPE)}

CASES = [("sd", 4, 4, 0, +1, 0), ("sd", 4, 4, 0, +1, 1), ("sd", 4, 4, 0, +1, 2), ("sd", 2, 3, 1, +1, 3),
         ("pf", 2, 2, 0, +1, 1), ("pf", 2, 2, 0, +1, 2), ("pf", 3, 2, 1, -1, 0), ("pf", 3, 2, 1, -1, 2),
         ("sd_uneven", 3, 3, 0, +1, 2), ("sd_uneven", 3, 3, 0, +1, 4)]


def _tbmes(name):
    base = "pf" if name == "pf" else "sd"
    return I.space(base)[2]


def oracle_case(name, Z, Nn, twoM, par, mx):
    orbits, spe = SPACES[name]
    o = O.Oracle(orbits, Z, Nn, twoM, 0 if par > 0 else 1).set_interaction(spe, _tbmes(name))
    mask, wmin, _ = o.truncation_mask([x.w for x in orbits], mx)
    return o, mask, wmin


def lib_case(name, Z, Nn, twoM, par, mx):
    orbits, spe = SPACES[name]
    c = N.Context(-1).build_basis(orbits, Z, Nn, twoM, par, max_excite=mx)
    return c.load_interaction(spe, _tbmes(name))


def lib_states(c):
    """(proton bits, neutron bits) of every basis index of a library basis."""
    B = c.export_basis()
    P = np.zeros(c.dim, dtype=np.uint64)
    Q = np.zeros(c.dim, dtype=np.uint64)
    for (ps, nsi, off) in B["blocks"]:
        _, _, p0, pc = B["p_sec"][ps]
        _, _, n0, nc = B["n_sec"][nsi]
        P[off:off + pc * nc] = np.repeat(B["p_bits"][p0:p0 + pc], nc)
        Q[off:off + pc * nc] = np.tile(B["n_bits"][n0:n0 + nc], pc)
    return P, Q


def sd_weight(bits, w_state):
    return sum(w_state[s] for s in range(len(w_state)) if int(bits) >> s & 1)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-%dp%dn-2M%d-par%+d-x%d" % c)
def test_truncated_basis_bit_exact(case):
    name, Z, Nn, twoM, par, mx = case
    o, mask, wmin = oracle_case(*case)
    c = lib_case(*case)
    assert c.dim == int(mask.sum())
    P, Q = lib_states(c)
    Po, Qo = o.states()
    assert set(zip(P.tolist(), Q.tolist())) == set(zip(Po[mask].tolist(), Qo[mask].tolist()))
    assert len(set(zip(P.tolist(), Q.tolist()))) == c.dim
    orbits, _ = SPACES[name]
    w_state = [x.w for x in orbits for _ in range(x.twoj + 1)]
    B = c.export_basis()
    wmax = wmin + mx
    for t, key in ((0, "p"), (1, "n")):
        sec = B[key + "_sec"]
        sw = c.table(key + "_sec_w", np.int64)
        bits = B[key + "_bits"]
        assert len(sw) == len(sec)
        for s, (tm, pa, st, cnt) in enumerate(sec):
            assert all(sd_weight(b, w_state) == sw[s] for b in bits[st:st + cnt])
            assert np.all(np.diff(bits[st:st + cnt].astype(np.int64)) > 0)
        keys = [(int(tm), int(pa), int(w)) for (tm, pa, _, _), w in zip(sec, sw)]
        assert keys == sorted(keys) and len(set(keys)) == len(keys)
    psw, nsw = c.table("p_sec_w", np.int64), c.table("n_sec_w", np.int64)
    blk = [(int(ps), int(ns_)) for (ps, ns_, _) in B["blocks"]]
    assert blk == sorted(blk)
    assert all(psw[ps] + nsw[ns_] <= wmax for (ps, ns_) in blk)
    offs = [int(off) for (_, _, off) in B["blocks"]]
    sizes = [int(B["p_sec"][ps][3] * B["n_sec"][ns_][3]) for (ps, ns_) in blk]
    assert offs == list(np.cumsum([0] + sizes[:-1]))


def truncated_tables_matvec(c, x):
    """tables_matvec plus the like-particle links between blocks."""
    y = tables_matvec(c, x)
    B = c.export_basis()
    blocks = B["blocks"]
    ll = c.table("llinks", np.int64).reshape(-1, 4)
    px = (c.table("ppx_ptr", np.int64), c.table("ppx_src", np.int32), c.table("ppx_coef", np.float64))
    nx = (c.table("nnx_ptr", np.int64), c.table("nnx_src", np.int32), c.table("nnx_coef", np.float64))

    def blk(b):
        ps, ns_, off = blocks[b]
        return int(off), int(B["p_sec"][ps][3]), int(B["n_sec"][ns_][3])

    for (d, s, species, po) in ll:
        offd, nPd, nNd = blk(d)
        offs, nPs, nNs = blk(s)
        Xs = x[offs:offs + nPs * nNs].reshape(nPs, nNs)
        Yd = y[offd:offd + nPd * nNd].reshape(nPd, nNd)
        ptr, src, coef = px if species == 0 else nx
        if species == 0:
            assert nNs == nNd
            for r in range(nPd):
                for e in range(ptr[po + r], ptr[po + r + 1]):
                    Yd[r] += coef[e] * Xs[src[e]]
        else:
            assert nPs == nPd
            for q in range(nNd):
                for e in range(ptr[po + q], ptr[po + q + 1]):
                    Yd[:, q] += coef[e] * Xs[:, src[e]]
    return y


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-%dp%dn-2M%d-par%+d-x%d" % c)
def test_truncated_tables_reproduce_oracle_matrix(case):
    name, Z, Nn, twoM, par, mx = case
    o, mask, _ = oracle_case(*case)
    c = lib_case(*case)
    orbits, _ = SPACES[name]
    H = o.truncated_matrix([x.w for x in orbits], mx)
    P, Q = lib_states(c)
    Po, Qo = o.states()
    idx = np.nonzero(mask)[0]
    pos = {(int(a), int(b)): j for j, (a, b) in enumerate(zip(Po[idx], Qo[idx]))}
    perm = np.array([pos[(int(a), int(b))] for a, b in zip(P, Q)])   # library index -> oracle kept position
    x = I.random_block(c.dim, 1, seed=7)[:, 0]
    xo = np.zeros(c.dim)
    xo[perm] = x
    y_ref = (H @ xo)[perm]
    y = truncated_tables_matvec(c, x)
    assert np.max(np.abs(y - y_ref)) <= 1e-12 * np.max(np.abs(y_ref))
    if mx > 0:
        assert len(c.table("llinks", np.int64)) > 0   # W-changing moves exist and are linked


def test_untruncated_limit_and_arguments():
    # the largest excitation keeps every state of the full basis, in the
    # W-sorted sector order
    c = lib_case("sd", 2, 3, 1, +1, 5)
    o = O.Oracle(SD_W, 2, 3, 1, 0)
    assert c.dim == o.dim
    with pytest.raises(N.BSError) as e:
        N.Context(-1).build_basis(SD_W, 2, 2, 0, +1, max_excite=-2)
    assert e.value.code == -1
    bad = (I.Orbit(0, 2, 5, -1), I.Orbit(1, 0, 1, 0))
    with pytest.raises(N.BSError):
        N.Context(-1).build_basis(bad, 1, 1, 0, +1, max_excite=0)
    # weights are ignored without truncation: the basis equals the plain one
    a = N.Context(-1).build_basis(SD_NMAX, 2, 2, 0, +1)
    b = N.Context(-1).build_basis(I.SD_ORBITS, 2, 2, 0, +1)
    assert a.dim == b.dim == 640
    ea, eb = a.export_basis(), b.export_basis()
    assert all(np.array_equal(ea[k], eb[k]) for k in ea)
