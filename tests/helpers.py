"""Test-side helpers (no method arithmetic of the library or the oracle)."""
from __future__ import annotations

import numpy as np

from paper_1801_08432_gb300.inputs import SplitMix64


def scrambled_tbmes(tbmes, orbits, seed: int = 7):
    """The same interaction written with scrambled labels.

    Each element gets its orbits inside a pair exchanged and/or its two pairs
    swapped, with the exchange phase of the isospin-coupled symmetry relation
    (Sec. "Symmetries of matrix elements"): V_JT(ba,cd) = (-1)^(ja+jb+J+T) V_JT(ab,cd),
    and V_JT(cd,ab) = V_JT(ab,cd).  The list order is permuted too.
    """
    rng = SplitMix64(seed)
    out = []
    for (a, b, c, d, J, T, v) in tbmes:
        r = rng.next_u64()
        if r & 1 and a != b:
            v = v * (-1) ** ((orbits[a - 1].twoj + orbits[b - 1].twoj) // 2 + J + T)
            a, b = b, a
        if r & 2 and c != d:
            v = v * (-1) ** ((orbits[c - 1].twoj + orbits[d - 1].twoj) // 2 + J + T)
            c, d = d, c
        if r & 4:
            a, b, c, d = c, d, a, b
        out.append((a, b, c, d, J, T, v))
    keys = [SplitMix64(seed * 1000 + i).next_u64() for i in range(len(out))]
    return [out[i] for i in np.argsort(keys, kind="stable")]


def channel_spectrum(orbits, spe, tbmes, J, T, species="pn"):
    """Eigenvalues of one coupled two-body channel (J, T):
    matrix (e_a + e_b) delta + V_JT(ab, cd) over pairs a <= b that couple to J
    (same-orbit pairs need J + T odd).  The TBMEs are read in their canonical
    label form (a <= b, c <= d), as the seeded generator writes them."""
    pairs = []
    for a in range(len(orbits)):
        for b in range(a, len(orbits)):
            ja, jb = orbits[a].twoj, orbits[b].twoj
            if not (abs(ja - jb) <= 2 * J <= ja + jb):
                continue
            if a == b and (J + T) % 2 == 0:
                continue
            pairs.append((a, b))
    n = len(pairs)
    if n == 0:
        return np.zeros(0)
    idx = {p: i for i, p in enumerate(pairs)}
    M = np.zeros((n, n))
    for i, (a, b) in enumerate(pairs):
        M[i, i] += spe[a] + spe[b]
    for (a, b, c, d, JJ, TT, v) in tbmes:
        if JJ != J or TT != T:
            continue
        p, q = (a - 1, b - 1), (c - 1, d - 1)
        assert p[0] <= p[1] and q[0] <= q[1]
        M[idx[p], idx[q]] += v
        if p != q:
            M[idx[q], idx[p]] += v
    return np.linalg.eigvalsh(M)


def match_subset(small, big, tol):
    """Greedy nearest matching of every value of `small` to a distinct value of
    `big`; returns (max distance, unmatched values of big)."""
    big = list(np.sort(big))
    worst = 0.0
    for v in np.sort(small):
        j = int(np.argmin([abs(v - b) for b in big]))
        worst = max(worst, abs(v - big[j]))
        big.pop(j)
    return worst, np.array(big)
