"""Scalar observables: J^2 and T^2 as one- plus two-body operators in the
interaction format, orbit occupations from the adjoint, and reduced one-body
densities (proton-neutron and isospin form) from the GPU's M-scheme
densities.

The total angular momentum squared is J^2 = sum_i j_i^2 + sum_{i != j} j_i . j_j.
Its single-particle part is j_a (j_a + 1) on every particle in orbit a, and
its two-body part sum_{i < j} 2 j_i . j_j is diagonal in the normalized
coupled pair states:

    <ab; J T | 2 j_1 . j_2 | ab; J T> = J (J + 1) - j_a (j_a + 1) - j_b (j_b + 1),

for every Pauli-allowed (a <= b, J, T), the same for T = 0 and T = 1.  Written
as single-particle energies and TBMEs V_JT(ab, ab), it loads into a context
like any interaction (Sec. "Interaction files"): on the same basis the
library's H x kernels then apply J^2, and <J^2> of a block of vectors comes
from one product and one block inner product, all on the GPU.  This is how
the paper evaluates J^2, as an expectation value after the diagonalization.
"""
from __future__ import annotations

import numpy as np

from . import _native as N
from .inputs import tbme_labels


def j2_operator(orbits):
    """(spe, tbmes) of J^2 for the orbits (labels 1-based, the interaction format)."""
    jj = [o.twoj * (o.twoj + 2) / 4.0 for o in orbits]   # j (j + 1)
    spe = list(jj)
    tb = []
    for (a, b, c, d, J, T) in tbme_labels(orbits):
        if (a, b) != (c, d):
            continue
        tb.append((a, b, c, d, J, T, J * (J + 1.0) - jj[a - 1] - jj[b - 1]))
    return spe, tb


def t2_operator(orbits):
    """(spe, tbmes) of the isospin squared T^2 = sum_i t_i^2 + sum_{i<j} 2 t_i . t_j:
    3/4 on every particle, and <ab; J T| 2 t_1 . t_2 |ab; J T> = T (T + 1) - 3/2
    on every pair state (isospin only, so diagonal in (ab, J))."""
    spe = [0.75] * len(orbits)
    tb = [(a, b, c, d, J, T, T * (T + 1.0) - 1.5) for (a, b, c, d, J, T) in tbme_labels(orbits)
          if (a, b) == (c, d)]
    return spe, tb


def t2_context(orbits, Z, Nn, twoM, parity=+1, device=0):
    """A context on the (orbits, Z, N, 2M, parity) basis whose "interaction" is T^2."""
    spe, tb = t2_operator(orbits)
    return N.make(orbits, spe, tb, Z, Nn, twoM, parity, device=device)


def occupations(ctx, psi, dtype, stream=None):
    """Orbit occupations n_a = <psi|N_a|psi> / <psi|psi> of the columns of psi
    (CUDA tensor [dim][k] in dtype), as a k x (number of orbits) numpy array.  The SPEs
    enter H as sum_a e_a N_a, so n_a = dE/de_a (Hellmann-Feynman): the
    adjoint's SPE derivatives psi^T (dH/de_a) psi from the GPU's transition
    densities, one column at a time, over psi^T psi from bs_block_dots."""
    import torch

    k = psi.shape[1]
    n_spe = ctx.n_spe
    n_theta = n_spe + ctx.n_tbme
    out = np.zeros((k, n_spe))
    gx = torch.empty((psi.shape[0], 1), device=psi.device, dtype=psi.dtype)
    nrm = torch.zeros(1, device=psi.device, dtype=torch.float64)
    for m in range(k):
        x = psi[:, m:m + 1].contiguous()
        g = ctx.apply_H_backward(x, x, gx, 1, dtype, n_theta=n_theta, stream=stream)
        ctx.block_dots(x, 1, x, 1, dtype, nrm, stream)
        out[m] = g[:n_spe] / float(nrm.cpu()[0])
    return out


def clebsch_gordan(tj1, tm1, tj2, tm2, tJ, tM):
    """<j1 m1 j2 m2 | J M>, all arguments doubled, by Racah's closed formula
    (a finite alternating sum of factorial ratios)."""
    from math import factorial as fac, sqrt
    if tm1 + tm2 != tM or abs(tm1) > tj1 or abs(tm2) > tj2 or abs(tM) > tJ:
        return 0.0
    if (tj1 + tm1) % 2 or (tj2 + tm2) % 2 or (tJ + tM) % 2 or (tj1 + tj2 + tJ) % 2:
        return 0.0
    if tJ > tj1 + tj2 or tJ < abs(tj1 - tj2):
        return 0.0
    a, b, c = (tj1 + tj2 - tJ) // 2, (tj1 - tj2 + tJ) // 2, (-tj1 + tj2 + tJ) // 2
    pre = sqrt((tJ + 1) * fac(a) * fac(b) * fac(c) / fac((tj1 + tj2 + tJ) // 2 + 1))
    pre *= sqrt(fac((tj1 + tm1) // 2) * fac((tj1 - tm1) // 2) * fac((tj2 + tm2) // 2) * fac((tj2 - tm2) // 2)
                * fac((tJ + tM) // 2) * fac((tJ - tM) // 2))
    s = 0.0
    for k in range(0, a + 1):
        d = [k, a - k, (tj1 - tm1) // 2 - k, (tj2 + tm2) // 2 - k, (tJ - tj2 + tm1) // 2 + k,
             (tJ - tj1 - tm2) // 2 + k]
        if min(d) < 0:
            continue
        den = 1
        for x in d:
            den *= fac(x)
        s += (-1.0 if k % 2 else 1.0) / den
    return pre * s


def reduced_densities(rho, orbits, twoM, twoJf, twoJi):
    """Reduced one-body densities in proton-neutron form (Sec. "One-body
    density matrices and occupations") from the M-scheme densities of one
    pair of states of one basis (rho[t][i][l] = <f| a+_i a_l |i>, species t,
    as bs_density returns them per column pair; M_f = M_i = M):

        rho_K(a+ b) = [K]^-1 [J_f] <J_f M| (a+ b~)_K0 |J_i M> / (J_i M, K 0 | J_f M),
        (a+ b~)_K0 = sum_m (j_a m, j_b -m | K 0) (-1)^(j_b - m) a+_{a m} b_{b m},

    [x] = sqrt(2x + 1), Edmonds' Wigner-Eckart convention.  Returns
    {(t, a, b, 2K): value}; NaN where (J_i M, K 0 | J_f M) vanishes (choose
    another M for those K)."""
    st = []
    for a, o in enumerate(orbits):
        st += [(a, tm) for tm in range(-o.twoj, o.twoj + 1, 2)]
    first = {}
    for i, (a, tm) in enumerate(st):
        first.setdefault(a, i)
    out = {}
    for t in range(2):
        for a, oa in enumerate(orbits):
            for b, ob in enumerate(orbits):
                ja, jb = oa.twoj, ob.twoj
                for twoK in range(abs(ja - jb), ja + jb + 1, 2):
                    s = 0.0
                    for tm in range(-min(ja, jb), min(ja, jb) + 1, 2):
                        i = first[a] + (tm + ja) // 2
                        l = first[b] + (tm + jb) // 2
                        ph = -1.0 if ((jb - tm) // 2) % 2 else 1.0
                        s += clebsch_gordan(ja, tm, jb, -tm, twoK, 0) * ph * rho[t][i][l]
                    c = clebsch_gordan(twoJi, twoM, twoK, 0, twoJf, twoM)
                    out[(t, a, b, twoK)] = (float("nan") if abs(c) < 1e-12 else
                                            np.sqrt(twoJf + 1.0) * s / c / np.sqrt(twoK + 1.0))
    return out


def isospin_densities(red, Z, Nn, twoTf, twoTi):
    """Doubly reduced one-body densities (J and isospin) from the reduced
    proton-neutron densities ``red`` of reduced_densities, for states of good
    isospin T_f, T_i (Sec. "Conversion from proton-neutron to isospin"),
    with protons at m_t = +1/2, T_z = (Z - N)/2, and the isospin
    time-reversal phase (-1)^(1/2 - m_t) of the annihilation operator:

        rho_T = [T_f] / (T_i T_z, T 0 | T_f T_z) [T]^-1
                sum_{m_t} (-1)^(1/2 - m_t) (1/2 m_t, 1/2 -m_t | T 0) rho_{m_t}.

    For T_f = T_i this is rho_0 = [T](rho^p + rho^n)/sqrt2 and
    rho_1 = [T](rho^p - rho^n) sqrt(T(T+1)) / (sqrt3 T_z).  Returns
    {(a, b, 2K, T): value}, NaN where (T_i T_z, T 0 | T_f T_z) vanishes (T = 1
    between equal T at T_z = 0)."""
    tTz = Z - Nn
    out = {}
    for (t, a, b, tk) in red:
        if t != 0:
            continue
        for T in (0, 1):
            c = clebsch_gordan(twoTi, tTz, 2 * T, 0, twoTf, tTz)
            if abs(c) < 1e-12:
                out[(a, b, tk, T)] = float("nan")
                continue
            s = (clebsch_gordan(1, 1, 1, -1, 2 * T, 0) * red[(0, a, b, tk)]
                 - clebsch_gordan(1, -1, 1, 1, 2 * T, 0) * red[(1, a, b, tk)])
            out[(a, b, tk, T)] = np.sqrt(twoTf + 1.0) / c / np.sqrt(2 * T + 1.0) * s
    return out


def basis_states(ctx):
    """(proton bits, neutron bits) of every basis state of a context, in
    basis order (block offset + proton row x neutron count + neutron column)."""
    B = ctx.export_basis()
    P = np.zeros(ctx.dim, dtype=np.uint64)
    Nb = np.zeros(ctx.dim, dtype=np.uint64)
    for ps, ns_, off in B["blocks"]:
        p0, pc = B["p_sec"][ps][2], B["p_sec"][ps][3]
        n0, nc = B["n_sec"][ns_][2], B["n_sec"][ns_][3]
        P[off:off + pc * nc] = np.repeat(B["p_bits"][p0:p0 + pc], nc)
        Nb[off:off + pc * nc] = np.tile(B["n_bits"][n0:n0 + nc], pc)
    return P, Nb


def embed(X, ctx_small, orbits_small, ctx_big, orbits_big):
    """Vectors of a smaller model space as vectors of a larger one with the
    same Z, N, 2M and parity, e.g. to start block Lanczos from approximate
    eigenvectors of the smaller space (Sec. "Block Lanczos": a bootstrapped
    pivot).  Every orbit of the small space must appear in the big one
    (same n, l, 2j) in the same relative order.  Single-particle states are
    numbered orbit-major, 2m ascending, so the renaming of states is then
    increasing and keeps the order of the creation operators (no sign); each
    small-space SD is a big-space basis state.  X: numpy [dim_small] or
    [dim_small][k]; returns numpy [dim_big](, k)."""
    where = []
    for o in orbits_small:
        hits = [b for b, q in enumerate(orbits_big) if (q.n, q.l, q.twoj) == (o.n, o.l, o.twoj)]
        if len(hits) != 1:
            raise ValueError("embed: orbit (n=%d, l=%d, 2j=%d) not found once in the big space" % (o.n, o.l, o.twoj))
        where.append(hits[0])
    if where != sorted(where):
        raise ValueError("embed: the small space's orbits must keep their order in the big space")
    first_big, off = [], 0
    for q in orbits_big:
        first_big.append(off)
        off += q.twoj + 1
    smap = []   # small state -> big state
    for a, o in enumerate(orbits_small):
        smap += [first_big[where[a]] + i for i in range(o.twoj + 1)]

    def remap(bits):
        out = np.zeros_like(bits)
        for s_small, s_big in enumerate(smap):
            on = (bits >> np.uint64(s_small)) & np.uint64(1)
            out |= on << np.uint64(s_big)
        return out

    Ps, Ns = basis_states(ctx_small)
    Pb, Nb = basis_states(ctx_big)
    if off > 32:
        raise ValueError("embed: at most 32 single-particle states per species (64-bit state keys)")
    nsb = np.uint64(off)
    key_b = (Pb << nsb) | Nb
    order = np.argsort(key_b)
    key_s = (remap(Ps) << nsb) | remap(Ns)
    pos = np.searchsorted(key_b[order], key_s)
    if np.any(pos >= len(order)) or np.any(key_b[order][np.minimum(pos, len(order) - 1)] != key_s):
        raise ValueError("embed: a small-space state is not in the big basis (Z, N, 2M or parity differ)")
    idx = order[pos]
    X = np.asarray(X)
    out = np.zeros((ctx_big.dim,) + X.shape[1:], dtype=X.dtype)
    out[idx] = X
    return out


def j2_context(orbits, Z, Nn, twoM, parity=+1, device=0):
    """A context on the (orbits, Z, N, 2M, parity) basis whose "interaction" is J^2."""
    spe, tb = j2_operator(orbits)
    return N.make(orbits, spe, tb, Z, Nn, twoM, parity, device=device)


def expectation(ctx_op, psi, k, dtype, stream=None):
    """<psi_i | O | psi_j> / sqrt(<psi_i|psi_i> <psi_j|psi_j>), a k x k numpy
    array, for the k <= 8 columns of psi (a CUDA tensor [dim][k] of the dtype),
    with O the operator loaded into ctx_op: O psi by its H x kernels, the
    inner products by bs_block_dots (extended precision)."""
    import torch

    if not 1 <= k <= 8:
        raise ValueError("expectation: 1 <= k <= 8 columns")
    kk = 1 if k == 1 else 2 if k == 2 else 4 if k <= 4 else 8   # the kernels' block sizes
    if kk != k:   # zero columns up to the next block size; only the k x k corner is returned
        psi = torch.cat([psi[:, :k], torch.zeros((psi.shape[0], kk - k), device=psi.device, dtype=psi.dtype)],
                        dim=1).contiguous()
    y = torch.empty_like(psi)
    ctx_op.apply_H(psi, y, kk, dtype, stream)
    num = torch.zeros(kk * kk, device=psi.device, dtype=torch.float64)
    den = torch.zeros(kk * kk, device=psi.device, dtype=torch.float64)
    ctx_op.block_dots(psi, 1, y, kk, dtype, num, stream)
    ctx_op.block_dots(psi, 1, psi, kk, dtype, den, stream)
    num = num.cpu().numpy().reshape(kk, kk)[:k, :k]
    nrm = np.sqrt(np.diag(den.cpu().numpy().reshape(kk, kk))[:k])
    return num / np.outer(nrm, nrm)


def j_from_j2(j2):
    """J from J (J + 1)."""
    return 0.5 * (-1.0 + np.sqrt(1.0 + 4.0 * np.asarray(j2)))
