"""CPU checks of the library's host side (no GPU): basis, decoupling and jump
tables from a host-only context (bs_create(-1)) against the FP64 oracle.

The product H*x is rebuilt here in numpy from the exported tables, with the
same meaning the CUDA kernel gives them (pp/nn destination lists; pn as
proton one-body jump x neutron one-body jump with W_pn), and compared with
the oracle's explicit matrix.  Also: bit-exact basis, bit-exact one-body jump
indices and signs against the oracle's operator strings, and error codes.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1801_08432_gb300 import _native as N
from paper_1801_08432_gb300 import inputs as I
from tests.helpers import scrambled_tbmes


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_1801_08432_gb300 import build
    build.build()


def host_ctx(name, Z, Nn, twoM, parity=+1, tb=None):
    orbits, spe, tbm = I.space(name)
    c = N.Context(-1).build_basis(orbits, Z, Nn, twoM, parity)
    c.load_interaction(spe, tbm if tb is None else tb)
    return c


def tables_matvec(c, x):
    """y = H x from the exported host tables (test-side numpy)."""
    B = c.export_basis()
    y = np.zeros_like(x)
    pp_ptr, pp_src, pp_c = c.table("pp_ptr", np.int64), c.table("pp_src", np.int32), c.table("pp_coef", np.float64)
    nn_ptr, nn_src, nn_c = c.table("nn_ptr", np.int64), c.table("nn_src", np.int32), c.table("nn_coef", np.float64)
    p1_ptr, p1_ent = c.table("p1_ptr", np.int64), c.table("p1_ent", np.uint32)
    n1_ptr, n1_ent = c.table("n1_ptr", np.int64), c.table("n1_ent", np.uint32)
    p1_cls = c.table("p1_cls", np.int64).reshape(-1, 4)
    n1_cls = c.table("n1_cls", np.int64).reshape(-1, 4)
    links = c.table("links", np.int64).reshape(-1, 6)
    wpn = c.table("wpn", np.float64)
    blocks = B["blocks"]

    def blk(b):
        ps, ns_, off = blocks[b]
        return int(off), int(B["p_sec"][ps][2]), int(B["p_sec"][ps][3]), int(B["n_sec"][ns_][2]), int(B["n_sec"][ns_][3])

    for b in range(len(blocks)):
        off, p0, nP, n0, nN = blk(b)
        X = x[off:off + nP * nN].reshape(nP, nN)
        Y = y[off:off + nP * nN].reshape(nP, nN)
        for r in range(nP):
            for e in range(pp_ptr[p0 + r], pp_ptr[p0 + r + 1]):
                Y[r] += pp_c[e] * X[pp_src[e]]
        for col in range(nN):
            for e in range(nn_ptr[n0 + col], nn_ptr[n0 + col + 1]):
                Y[:, col] += nn_c[e] * X[:, nn_src[e]]
    for (d, s, pc, nc, w_off, nb) in links:
        offd, _, nPd, _, nNd = blk(d)
        offs, _, nPs, _, nNs = blk(s)
        Xs = x[offs:offs + nPs * nNs].reshape(nPs, nNs)
        Yd = y[offd:offd + nPd * nNd].reshape(nPd, nNd)
        pptr = p1_cls[pc][3]
        nptr = n1_cls[nc][3]
        # proton side as (row, src, op, sign), neutron side as (col, src, op, sign)
        pr = [(r, e & 0xFFFF, (e >> 16) & 0x7FFF, -1.0 if e >> 31 else 1.0)
              for r in range(nPd) for e in p1_ent[p1_ptr[pptr + r]:p1_ptr[pptr + r + 1]]]
        ncl = [(q, e & 0xFFFF, (e >> 16) & 0x7FFF, -1.0 if e >> 31 else 1.0)
               for q in range(nNd) for e in n1_ent[n1_ptr[nptr + q]:n1_ptr[nptr + q + 1]]]
        if not pr or not ncl:
            continue
        na = max(a for (_, _, a, _) in pr) + 1
        W = wpn[w_off:w_off + na * nb].reshape(na, nb) if na * nb else None
        ncl = np.array(ncl, dtype=np.float64)
        for a in range(na):
            rows = [(r, src, sg) for (r, src, aa, sg) in pr if aa == a]
            if not rows:
                continue
            P = sp.csr_matrix(([g for (_, _, g) in rows], ([r for (r, _, _) in rows], [s_ for (_, s_, _) in rows])),
                              shape=(nPd, nPs))
            vals = ncl[:, 3] * W[a, ncl[:, 2].astype(int)]
            Oa = sp.csr_matrix((vals, (ncl[:, 0].astype(int), ncl[:, 1].astype(int))), shape=(nNd, nNs))
            Yd += P @ (Oa @ Xs.T).T
    return y


@pytest.mark.parametrize("name,Z,Nn,twoM", [("sd", 2, 2, 0), ("sd", 3, 2, 1), ("sd", 1, 1, 0), ("sd", 2, 0, 0),
                                            ("sd", 0, 3, 3), ("pf", 2, 2, 0), ("p", 4, 4, 0), ("sd", 4, 4, 2)])
def test_host_tables_reproduce_oracle_matrix(name, Z, Nn, twoM):
    orbits, spe, tb = I.space(name)
    o = O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(spe, tb)
    c = host_ctx(name, Z, Nn, twoM)
    assert c.dim == o.dim
    x = I.random_block(o.dim, 1)[:, 0]
    y_ref = o.spmv(x)
    y = tables_matvec(c, x)
    assert np.max(np.abs(y - y_ref)) <= 1e-12 * np.max(np.abs(y_ref))


@pytest.mark.parametrize("name,Z,Nn,twoM,par", [("sd", 2, 2, 0, 1), ("sd", 4, 4, 0, 1), ("sd", 5, 6, 1, 1),
                                                ("pf", 4, 4, 0, 1), ("pf", 3, 2, -1, -1), ("p", 4, 4, 0, 1),
                                                ("sd", 0, 2, 0, 1)])
def test_basis_bit_exact(name, Z, Nn, twoM, par):
    orbits, _ = I.SPACES[name]
    o = O.Oracle(orbits, Z, Nn, twoM, 0 if par > 0 else 1)
    c = N.Context(-1).build_basis(orbits, Z, Nn, twoM, par)
    A, Bo = c.export_basis(), o.basis()
    for key in ("p_bits", "n_bits", "p_sec", "n_sec", "blocks"):
        assert np.array_equal(A[key], Bo[key]), key


def test_mixed_parity_basis_bit_exact():
    # sd + f7/2: sectors of both parities
    orbits = (I.Orbit(0, 2, 5), I.Orbit(1, 0, 1), I.Orbit(0, 3, 7))
    for par in (+1, -1):
        o = O.Oracle(orbits, 2, 3, 1, 0 if par > 0 else 1)
        c = N.Context(-1).build_basis(orbits, 2, 3, 1, par)
        A, Bo = c.export_basis(), o.basis()
        for key in ("p_bits", "n_bits", "p_sec", "n_sec", "blocks"):
            assert np.array_equal(A[key], Bo[key]), key


@pytest.mark.parametrize("species", [0, 1])
def test_onebody_jumps_bit_exact(species):
    """Every one-body jump a+_i a_k (index, source, destination, sign) of the
    library equals the oracle's operator string on the same bitstrings."""
    name, Z, Nn, twoM = "sd", 3, 2, 1
    orbits, _ = I.SPACES[name]
    c = host_ctx(name, Z, Nn, twoM)
    B = c.export_basis()
    sec = B["p_sec"] if species == 0 else B["n_sec"]
    bits = B["p_bits"] if species == 0 else B["n_bits"]
    pre = "p1" if species == 0 else "n1"
    ptr, ent = c.table(pre + "_ptr", np.int64), c.table(pre + "_ent", np.uint32)
    cls = c.table(pre + "_cls", np.int64).reshape(-1, 4)
    ops = c.table("ops", np.int64).reshape(-1, 5)
    op_lists = c.table("op_lists", np.int64)
    starts = np.concatenate([[0], np.cumsum(ops[:, 4])])
    ns = 12
    lib = set()
    for (ssrc, sdst, g, po) in cls:
        for dl in range(sec[sdst][3]):
            for e in ent[ptr[po + dl]:ptr[po + dl + 1]]:
                src = int(bits[sec[ssrc][2] + (e & 0xFFFF)])
                dst = int(bits[sec[sdst][2] + dl])
                op = int(op_lists[starts[g] + ((e >> 16) & 0x7FFF)])
                lib.add((src, dst, op // ns, op % ns, -1 if e >> 31 else 1))
    ref = set()
    for src in bits:
        for k in range(ns):
            for i in range(ns):
                sg, dst = O.apply_string(int(src), [("+", i), ("-", k)])
                if sg:
                    ref.add((int(src), dst, i, k, sg))
    assert lib == ref


def test_scrambled_labels_same_tables():
    orbits, spe, tb = I.space("sd")
    a = host_ctx("sd", 2, 2, 0)
    b = host_ctx("sd", 2, 2, 0, tb=scrambled_tbmes(tb, orbits, seed=11))
    for name in ("pp_coef", "nn_coef", "wpn"):
        assert np.max(np.abs(a.table(name, np.float64) - b.table(name, np.float64))) < 1e-13


def test_error_codes():
    orbits, spe, tb = I.space("sd")
    c = N.Context(-1)
    with pytest.raises(N.BSError) as e:
        c.load_interaction(spe, tb)
    assert e.value.code == -2                                  # BS_ENOBASIS
    for args in [(orbits, 2, 2, 1, 1),                          # 2M odd for even A
                 (orbits, 13, 2, 0, 1),                         # Z > states
                 (orbits, 2, 2, 0, 0),                          # parity not +-1
                 (orbits, 2, 2, 40, 1)]:                        # empty basis
        with pytest.raises(N.BSError) as e:
            c.build_basis(*args)
        assert e.value.code == -1
    bad_orb = [I.Orbit(0, 2, 4)]
    with pytest.raises(N.BSError):
        c.build_basis(bad_orb, 1, 1, 0, 1)
    c.build_basis(orbits, 2, 2, 0, 1)
    for bad in [(1, 1, 1, 1, 1, 1, 1.0), (1, 2, 1, 2, 0, 1, 1.0), (1, 1, 1, 4, 1, 0, 1.0), (1, 1, 1, 1, 1, 2, 1.0)]:
        with pytest.raises(N.BSError) as e:
            c.load_interaction(spe, [bad])
        assert e.value.code == -1
    a, b, cc, d, J, T, v = tb[5]
    with pytest.raises(N.BSError):
        c.load_interaction(spe, [tb[5], (cc, d, a, b, J, T, v)])
    with pytest.raises(N.BSError):
        c.load_interaction(spe[:2], tb)
    c.load_interaction(spe, [])                                  # SPE only is legal
    x = np.zeros(c.dim)
    with pytest.raises(N.BSError):                               # host-only context cannot apply
        c.apply_H_host(x, x.copy(), 1, N.BS_F64)


def test_abi_exports_every_declared_symbol():
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "bigstick_gpu.h")).read()
    names = set(re.findall(r"^\s*(?:const\s+)?(?:int|void|char\s*\*|const char\s*\*)\s*\**\s*(bs_\w+)\s*\(", hdr, re.M))
    assert names, "no declarations found"
    L = N.load()
    for n in sorted(names):
        assert hasattr(L, n), n
    assert names <= set(N.EXPORTED) | {"bs_apply_H_backward", "bs_lanczos"}


def ell_lists(c, prefix, base_rows, ncols_of, packed=True):
    """Per-column lists rebuilt from an ELL export: {(class, column): sorted entries}."""
    col = c.table(prefix + "_col", np.int32)
    ln = c.table(prefix + "_len", np.int32)
    soff = c.table(prefix + "_soff", np.int64)
    if packed:
        ent = c.table(prefix + "_ent", np.uint32)
    else:
        src = c.table(prefix + "_src", np.int32)
        cf = c.table(prefix + "_coef", np.float64)
    out = {}
    for cls, (col0, sl0) in enumerate(base_rows):
        n = ncols_of(cls)
        seen = set()
        for i in range(n):
            base = soff[sl0 + i // 32] + i % 32
            items = []
            for v in range(ln[col0 + i]):
                e = base + 32 * v
                items.append(int(ent[e]) if packed else (int(src[e]), float(cf[e])))
            cc = int(col[col0 + i])
            seen.add(cc)
            out[(cls, cc)] = sorted(items)
        assert seen == set(range(n))
    return out


def test_ell_forms_match_csr_lists():
    c = host_ctx("pf", 2, 3, 1, parity=-1)
    B = c.export_basis()
    n1_ptr, n1_ent = c.table("n1_ptr", np.int64), c.table("n1_ent", np.uint32)
    cls = c.table("n1_cls", np.int64).reshape(-1, 4)
    base = c.table("n1e_base", np.int64).reshape(-1, 2)
    ws = int(c.table("stats", np.int64)[7])
    got = ell_lists(c, "n1e", base, lambda k: int(B["n_sec"][cls[k][1]][3]))
    # ELL entries are src | (op + ws * sign) << 16; back to src | op << 16 | sign << 31
    def unpack(e):
        bi = e >> 16
        return (e & 0xFFFF) | ((bi % ws) << 16) | ((bi // ws) << 31)
    got = {key: sorted(unpack(e) for e in val) for key, val in got.items()}
    for k, (ssrc, sdst, g, po) in enumerate(cls):
        for col in range(B["n_sec"][sdst][3]):
            ref = sorted(int(e) for e in n1_ent[n1_ptr[po + col]:n1_ptr[po + col + 1]])
            assert got[(k, col)] == ref
    nn_ptr, nn_src, nn_c = c.table("nn_ptr", np.int64), c.table("nn_src", np.int32), c.table("nn_coef", np.float64)
    nbase = c.table("nne_base", np.int64).reshape(-1, 2)
    got = ell_lists(c, "nne", nbase, lambda s: int(B["n_sec"][s][3]), packed=False)
    for s, (_, _, st, cnt) in enumerate(B["n_sec"]):
        for col in range(cnt):
            g = st + col
            ref = sorted((int(a), float(b)) for a, b in zip(nn_src[nn_ptr[g]:nn_ptr[g + 1]], nn_c[nn_ptr[g]:nn_ptr[g + 1]]))
            assert got[(s, col)] == ref


def pipe_tables_matvec(c, x):
    """y = H x from the pipelined kernel's tables (one column order per neutron
    sector, sliced ELL with +W/-W indices, pre-signed W rows), test-side numpy."""
    B = c.export_basis()
    blocks = B["blocks"]
    nsec = len(B["n_sec"])
    st = c.table("stats", np.int64)
    ws = int(st[7])
    base = c.table("pe_base", np.int64)
    sec_base = base[:3 * nsec].reshape(-1, 3)
    cls_base = base[3 * nsec:].reshape(-1, 2)
    perm = c.table("pe_perm", np.int32)
    sinfo = c.table("pe_sinfo", np.int32)
    ent = c.table("pe_ent", np.uint32)
    nsrc, ncoef, nsinfo = c.table("pe_nn_src", np.int32), c.table("pe_nn_coef", np.float64), c.table("pe_nn_sinfo", np.int32)
    ww = c.table("ww", np.float64)
    ww_off = c.table("ww_off", np.int64)
    pp_ptr, pp_src, pp_c = c.table("pp_ptr", np.int64), c.table("pp_src", np.int32), c.table("pp_coef", np.float64)
    p1_ptr, p1_ent = c.table("p1_ptr", np.int64), c.table("p1_ent", np.uint32)
    p1_cls = c.table("p1_cls", np.int64).reshape(-1, 4)
    links = c.table("links", np.int64).reshape(-1, 6)
    y = np.zeros_like(x)

    def blk(b):
        ps, ns_, off = blocks[b]
        return int(off), int(B["p_sec"][ps][2]), int(B["p_sec"][ps][3]), int(ns_), int(B["n_sec"][ns_][3])

    for b in range(len(blocks)):
        off, p0, nP, ns_, nN = blk(b)
        X = x[off:off + nP * nN].reshape(nP, nN)
        Y = y[off:off + nP * nN].reshape(nP, nN)
        for r in range(nP):
            for e in range(pp_ptr[p0 + r], pp_ptr[p0 + r + 1]):
                Y[r] += pp_c[e] * X[pp_src[e]]
        po, ne0, ns0 = sec_base[ns_]
        for p in range(nN):
            col = perm[po + p]
            o, lmax = nsinfo[ns0 + 2 * (p // 32)], nsinfo[ns0 + 2 * (p // 32) + 1]
            idx = ne0 + o + 32 * np.arange(lmax) + p % 32
            Y[:, col] += X[:, nsrc[idx]] @ ncoef[idx]
    for (d, s, pc, nc, w_off, nb) in links:
        offd, _, nPd, nsd, nNd = blk(d)
        offs, _, nPs, _, nNs = blk(s)
        Xs = x[offs:offs + nPs * nNs].reshape(nPs, nNs)
        Yd = y[offd:offd + nPd * nNd].reshape(nPd, nNd)
        pptr = p1_cls[pc][3]
        wo = ww_off[p1_cls[pc][2]]
        ce, cs = cls_base[nc]
        po = sec_base[nsd][0]
        for r in range(nPd):
            for e in p1_ent[p1_ptr[pptr + r]:p1_ptr[pptr + r + 1]]:
                ip, a, sp_ = int(e & 0xFFFF), int((e >> 16) & 0x7FFF), int(e >> 31)
                wrow = ww[wo + (2 * a + sp_) * 2 * ws: wo + (2 * a + sp_ + 1) * 2 * ws]
                for p in range(nNd):
                    col = perm[po + p]
                    o, lmax = sinfo[cs + 2 * (p // 32)], sinfo[cs + 2 * (p // 32) + 1]
                    es = ent[ce + o + 32 * np.arange(lmax) + p % 32]
                    Yd[r, col] += np.dot(wrow[(es >> 16) & 0x7FFF], Xs[ip, es & 0xFFFF])
    return y


@pytest.mark.parametrize("name,Z,Nn,twoM", [("sd", 2, 2, 0), ("sd", 3, 2, 1), ("sd", 0, 3, 3), ("sd", 1, 1, 0),
                                            ("pf", 2, 2, 0)])
def test_pipe_tables_reproduce_oracle_matrix(name, Z, Nn, twoM):
    orbits, spe, tb = I.space(name)
    o = O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(spe, tb)
    c = host_ctx(name, Z, Nn, twoM)
    x = I.random_block(o.dim, 1, seed=9)[:, 0]
    y_ref = o.spmv(x)
    y = pipe_tables_matvec(c, x)
    assert np.max(np.abs(y - y_ref)) <= 1e-12 * np.max(np.abs(y_ref))


CORE_UNIT = np.dtype([("dblock", np.int32), ("nsrc", np.int32), ("src0", np.int64),
                      ("drow", np.int32, 4), ("meta", np.int32, 4),
                      ("nN", np.int32), ("perm_off", np.int32), ("doff", np.int64)])
CORE_SRC = np.dtype([("x_elem", np.int64), ("nN", np.int32), ("wtab", np.uint32),
                     ("ent_base", np.int64), ("sinfo_base", np.int64)])


PPG = 8
PP_UNIT = np.dtype([("dblock", np.int32), ("nsrc", np.int32), ("src0", np.int64),
                    ("drow", np.int32, PPG), ("part", np.int32, PPG),
                    ("nN", np.int32), ("pad", np.int32), ("doff", np.int64)])


def core_tables_matvec(c, x, Z, pp_core=False):
    """y = H x with the pn term taken from the core-grouped tables: one partial
    vector per rank t of the removed proton state, summed at the end; the
    like-particle terms from the pipelined kernel's tables.  Test-side numpy.
    Also returns how often each (row, t) slot of the partial vectors was written."""
    B = c.export_basis()
    blocks = B["blocks"]
    nsec = len(B["n_sec"])
    ws = int(c.table("stats", np.int64)[7])
    base = c.table("pe_base", np.int64)
    sec_base = base[:3 * nsec].reshape(-1, 3)
    cls_base = base[3 * nsec:].reshape(-1, 2)
    perm = c.table("pe_perm", np.int32)
    sinfo = c.table("pe_sinfo", np.int32)
    ent = c.table("core_ent", np.uint32)
    assert len(ent) == len(c.table("pe_ent", np.uint32))
    links = c.table("links", np.int64).reshape(-1, 6)
    units = np.frombuffer(c.table("core_units", np.uint8).tobytes(), dtype=CORE_UNIT)
    srcs = np.frombuffer(c.table("core_src", np.uint8).tobytes(), dtype=CORE_SRC)
    wc = c.table("wc", np.float64).reshape(-1, 2 * ws * 4)   # one [2 wsign][4] slot per table
    dim = len(x)
    nz = Z + (Z * (Z - 1) // 2 if pp_core else 0)
    part = np.zeros((nz, dim))
    written = np.zeros((nz, dim), dtype=np.int64)

    def blk(b):
        ps, ns_, off = blocks[b]
        return int(off), int(B["p_sec"][ps][3]), int(ns_), int(B["n_sec"][ns_][3])

    for u in units:
        offd, nPd, nsd, nNd = blk(u["dblock"])
        assert (u["nN"], u["doff"], u["perm_off"]) == (nNd, offd, sec_base[nsd][0])   # the record's header copies
        acc = np.zeros((4, nNd))
        po = sec_base[nsd][0]
        # weight rows of R floats at the front of the slot: R = 1, 2 or 4 by the unit's rows
        R = 1 if u["drow"][1] < 0 else 2 if u["drow"][2] < 0 else 4
        for q in range(u["nsrc"]):
            xe, nNs, wt, ce, cs = srcs[u["src0"] + q]
            xs = x[xe: xe + nNs]
            assert (int(wt) & 1) == (int(wt) >> 31)        # the table of a -1 sign of a_k has its halves swapped
            W = np.zeros((2 * ws, 4))
            W[:, :R] = wc[int(wt) & 0x7FFFFFFF][:2 * ws * R].reshape(2 * ws, R)
            for p in range(nNd):
                col = perm[po + p]
                o, lmax = sinfo[cs + 2 * (p // 32)], sinfo[cs + 2 * (p // 32) + 1]
                es = ent[ce + o + 32 * np.arange(lmax) + p % 32].astype(np.int64)
                acc[:, col] += W[es >> 16].T @ xs[es & 0xFFFF]
        for p4 in range(4):
            r = u["drow"][p4]
            if r < 0:
                continue
            t, sg = u["meta"][p4] & 255, (-1.0 if u["meta"][p4] & 256 else 1.0)
            part[t, offd + r * nNd: offd + (r + 1) * nNd] = sg * acc[p4]
            written[t, offd + r * nNd: offd + (r + 1) * nNd] += 1
    if pp_core:
        ppu = np.frombuffer(c.table("pp_units", np.uint8).tobytes(), dtype=PP_UNIT)
        prow = c.table("pps_row", np.int32)
        pw = c.table("pps_w", np.float64).reshape(-1, PPG)
        for u in ppu:
            offd, nPd, nsd, nNd = blk(u["dblock"])
            acc = np.zeros((PPG, nNd))
            for q in range(u["nsrc"]):
                sr = prow[u["src0"] + q]
                acc += np.outer(pw[u["src0"] + q], x[offd + sr * nNd: offd + (sr + 1) * nNd])
            for p8 in range(PPG):
                r = u["drow"][p8]
                if r < 0:
                    continue
                part[u["part"][p8], offd + r * nNd: offd + (r + 1) * nNd] = acc[p8]
                written[u["part"][p8], offd + r * nNd: offd + (r + 1) * nNd] += 1
    # like-particle terms (pp by rows, nn by the sector's lists)
    y = np.zeros_like(x)
    pp_ptr, pp_src, pp_c = c.table("pp_ptr", np.int64), c.table("pp_src", np.int32), c.table("pp_coef", np.float64)
    pdiag = c.table("pdiag", np.float64)
    nsrc_, ncoef, nsinfo = c.table("pe_nn_src", np.int32), c.table("pe_nn_coef", np.float64), c.table("pe_nn_sinfo", np.int32)
    for b in range(len(blocks)):
        ps, ns_, off = blocks[b]
        p0, nP, nN = int(B["p_sec"][ps][2]), int(B["p_sec"][ps][3]), int(B["n_sec"][ns_][3])
        X = x[off:off + nP * nN].reshape(nP, nN)
        Y = y[off:off + nP * nN].reshape(nP, nN)
        for r in range(nP):
            if pp_core:
                Y[r] += pdiag[p0 + r] * X[r]
            else:
                for e in range(pp_ptr[p0 + r], pp_ptr[p0 + r + 1]):
                    Y[r] += pp_c[e] * X[pp_src[e]]
        po, ne0, ns0 = sec_base[ns_]
        for p in range(nN):
            col = perm[po + p]
            o, lmax = nsinfo[ns0 + 2 * (p // 32)], nsinfo[ns0 + 2 * (p // 32) + 1]
            idx = ne0 + o + 32 * np.arange(lmax) + p % 32
            Y[:, col] += X[:, nsrc_[idx]] @ ncoef[idx]
    for t in range(nz):
        y += part[t]
    return y, written


@pytest.mark.parametrize("name,Z,Nn,twoM", [("sd", 2, 2, 0), ("sd", 3, 2, 1), ("sd", 1, 1, 0), ("sd", 1, 3, 0),
                                            ("pf", 2, 2, 2), ("p", 2, 2, 2), ("p", 3, 3, 0)])
@pytest.mark.parametrize("pp_core", [False, True])
def test_core_tables_reproduce_oracle_matrix(name, Z, Nn, twoM, pp_core):
    """The pn term regrouped by (Z-1)-proton cores and (optionally) the pp term
    by (Z-2)-proton cores: every proton jump belongs to exactly one core, every
    destination row gets exactly one partial per rank t (and per pair of its
    states), and the sum reproduces the oracle's H x."""
    orbits, spe, tb = I.space(name)
    o = O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(spe, tb)
    c = host_ctx(name, Z, Nn, twoM)
    x = I.random_block(o.dim, 1, seed=11)[:, 0]
    y_ref = o.spmv(x)
    y, written = core_tables_matvec(c, x, Z, pp_core)
    assert np.all(written == 1)
    assert np.max(np.abs(y - y_ref)) <= 1e-12 * np.max(np.abs(y_ref))


def test_core_weight_rows_match_the_unit_row_count():
    """The weight table a pn-core source names has rows of R floats, R = 1, 2
    or 4 for units with one, two, or three and four destination rows, packed
    at the front of its [2 wsign][4] slot: every nonzero weight lies in the
    first 2 wsign R floats, and row p of entry o sits at o R + p (the
    layout the kernel indexes).  Checked against the slot read in the
    4-float layout of the operator rows: the packed table equals it column
    by column."""
    c = host_ctx("sd", 4, 4, 0)
    ws = int(c.table("stats", np.int64)[7])
    units = np.frombuffer(c.table("core_units", np.uint8).tobytes(), dtype=CORE_UNIT)
    srcs = np.frombuffer(c.table("core_src", np.uint8).tobytes(), dtype=CORE_SRC)
    wc = c.table("wc", np.float64).reshape(-1, 2 * ws * 4)
    tabs = {}   # table -> (R, real rows) of the units that name it
    for u in units:
        nreal = int((u["drow"] >= 0).sum())
        assert np.all(u["drow"][:nreal] >= 0) and np.all(u["drow"][nreal:] < 0)   # packed to the front
        R = 1 if nreal == 1 else 2 if nreal == 2 else 4
        for t in (srcs["wtab"][u["src0"]: u["src0"] + u["nsrc"]].astype(np.int64) & 0x7FFFFFFF).tolist():
            assert tabs.setdefault(t, (R, nreal)) == (R, nreal)   # one layout per table
    assert {r for r, _ in tabs.values()} == {1, 2, 4}
    for t, (R, nreal) in tabs.items():
        slot = wc[t]
        assert not np.any(slot[2 * ws * R:]), (t, R)   # nothing past the packed rows
        rows = slot[:2 * ws * R].reshape(2 * ws, R)
        assert not np.any(rows[:, nreal:]), (t, R)     # the padded fourth column of 3-row units
        # the +W and -W halves: table 2 j + 1 is table 2 j with its halves swapped
        mate = wc[t ^ 1][:2 * ws * R].reshape(2 * ws, R)
        assert np.array_equal(rows, np.roll(mate, ws, axis=0))


def test_core_units_structure():
    """Each unit: one core c (Z-1 states) shared by its destination rows and
    sources; destination states of one (2m, parity); the stored rank t and the
    fermion signs of a+_i on c and of a_k on c + k, recomputed from bitmasks."""
    name, Z, Nn = "sd", 3, 3
    c = host_ctx(name, Z, Nn, 2)
    B = c.export_basis()
    pbits = B["p_bits"]
    units = np.frombuffer(c.table("core_units", np.uint8).tobytes(), dtype=CORE_UNIT)
    srcs = np.frombuffer(c.table("core_src", np.uint8).tobytes(), dtype=CORE_SRC)
    orbits, _, _ = I.space(name)
    twom = [tm for o_ in orbits for tm in range(-o_.twoj, o_.twoj + 1, 2)]
    ns = len(twom)

    def sd_bits(blk, row):
        ps = B["blocks"][blk][0]
        return int(pbits[B["p_sec"][ps][2] + row])

    def below(m, s):
        return -1 if bin(m & ((1 << s) - 1)).count("1") % 2 else 1

    def sd_of_elem(xe):
        # the proton SD of the source row starting at basis index xe
        for b_, (ps, ns_, off) in enumerate(B["blocks"]):
            nN = int(B["n_sec"][ns_][3])
            nP = int(B["p_sec"][ps][3])
            if off <= xe < off + nP * nN:
                assert (xe - off) % nN == 0
                return sd_bits(b_, (xe - off) // nN)
        raise AssertionError(xe)

    for u in units:
        cores, keys = set(), set()
        nr = int(np.sum(u["drow"] >= 0))
        assert nr >= 1 and np.all(u["drow"][:nr] >= 0) and np.all(u["drow"][nr:] < 0)   # rows packed to the front
        for p in range(4):
            if u["drow"][p] < 0:
                continue
            r = sd_bits(u["dblock"], u["drow"][p])
            t = u["meta"][p] & 255
            i = [s for s in range(ns) if r >> s & 1][t]
            core = r & ~(1 << i)
            cores.add(core)
            keys.add(twom[i])
            assert (u["meta"][p] & 256 != 0) == (below(core, i) < 0)
        assert len(cores) == 1 and len(keys) == 1
        core = cores.pop()
        assert bin(core).count("1") == Z - 1
        for q in range(u["nsrc"]):
            xe, nNs, wt, _, _ = srcs[u["src0"] + q]
            s = sd_of_elem(int(xe))
            k_bits = s & ~core
            assert s & core == core and bin(k_bits).count("1") == 1
            k = k_bits.bit_length() - 1
            assert ((int(wt) & 0x7FFFFFFF) >> 1) % ns == k
            assert ((int(wt) >> 31) != 0) == (below(core, k) < 0) == ((int(wt) & 1) != 0)


def test_abi_struct_layout_matches_header(tmp_path):
    # the ctypes structures of the binding against sizeof / offsetof of the
    # C declarations, compiled from the public header by the host compiler
    import os
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no host C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")
    structs = [N.bs_orbit, N.bs_tbme, N.bs_lanczos_opts, N.bs_lanczos_report]
    body = []
    for S in structs:
        body.append('printf("%s %%zu\\n", sizeof(%s));' % (S.__name__, S.__name__))
        for f in S._fields_:
            body.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (S.__name__, f[0], S.__name__, f[0]))
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include <stdint.h>\n#include \"bigstick_gpu.h\"\n"
                   "int main(void) {\n" + "\n".join(body) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for S in structs:
        assert int(got[S.__name__]) == ctypes_sizeof(S), S.__name__
        for f in S._fields_:
            assert int(got[S.__name__ + "." + f[0]]) == getattr(S, f[0]).offset, (S.__name__, f[0])


def ctypes_sizeof(S):
    import ctypes
    return ctypes.sizeof(S)


_ORDER_SCRIPT = r"""
import hashlib, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1801_08432_gb300 import _native as N, inputs as I
o, s, t = I.space("sd")
c = N.Context(-1).build_basis(o, 6, 6, 0, 1).load_interaction(s, t)
h = hashlib.sha256()
for name, dt in (("core_ent", np.uint32), ("pe_ent", np.uint32), ("pe_nn_src", np.int32), ("pe_nn_coef", np.float64)):
    h.update(c.table(name, dt).tobytes())
print(h.hexdigest())
"""


def test_list_orders_do_not_depend_on_the_thread_count():
    """The list step orders (greedy, then the seeded annealing of each slice,
    run in parallel) are the same for any number of host threads, so the
    product is bit-reproducible across machines: sd 6p6n (28Si) tables built
    with 1 and with 4 OpenMP threads, in fresh processes."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = []
    for nt in (1, 4):
        env = dict(os.environ, OMP_NUM_THREADS=str(nt))
        r = subprocess.run([sys.executable, "-c", _ORDER_SCRIPT, root], env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        out.append(r.stdout.strip().splitlines()[-1])
    assert out[0] == out[1]
