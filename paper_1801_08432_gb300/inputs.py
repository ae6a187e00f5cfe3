"""Seeded synthetic inputs: model spaces, single-particle energies, random
isospin-coupled two-body matrix elements and random vectors.

This module is shared by the CUDA path, the tests and the oracle.  It holds
none of the method's arithmetic (no Clebsch-Gordan coefficients, no
decoupling, no Slater determinants): it only lists the orbits of a valence
space, enumerates the labels (a b c d J T) of the two-body matrix elements a
file of the paper's format would hold (Sec. "Interaction files": normalized
two-body states, a,b,c,d 1-based orbit labels, any order accepted) and draws
their values from a published counter-based generator.

Generator: SplitMix64 (Steele, Lea & Flood 2014) gives 64-bit words; a word w
maps to a uniform double (w >> 11) * 2**-53; a Gaussian is one Box-Muller
draw from two such uniforms, sqrt(-2 ln(1-u1)) * cos(2 pi u2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1


@dataclass(frozen=True)
class Orbit:
    """One single-particle orbit (n, l, 2j); w is the truncation weight."""
    n: int
    l: int
    twoj: int
    w: int = 0


# The valence spaces of the configurations.  Orbit order is the order the
# labels of the interaction refer to (1-based).
SD_ORBITS = (Orbit(0, 2, 5), Orbit(1, 0, 1), Orbit(0, 2, 3))          # 0d5/2 1s1/2 0d3/2
SD_SPE = (-3.95, -3.16, 1.65)
PF_ORBITS = (Orbit(0, 3, 7), Orbit(1, 1, 3), Orbit(0, 3, 5), Orbit(1, 1, 1))  # 0f7/2 1p3/2 0f5/2 1p1/2
PF_SPE = (0.0, 2.0, 6.5, 4.0)
P_ORBITS = (Orbit(0, 1, 3), Orbit(0, 1, 1))                          # 0p3/2 0p1/2
P_SPE = (0.0, 1.0)

SPACES = {
    "sd": (SD_ORBITS, SD_SPE),
    "pf": (PF_ORBITS, PF_SPE),
    "p": (P_ORBITS, P_SPE),
}

TBME_SEED = 180108432
PIVOT_SEED = 180108433


class SplitMix64:
    """SplitMix64 word stream."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def gauss(self) -> float:
        u1 = self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)


def tbme_labels(orbits):
    """All Pauli-allowed, parity-conserving isospin-coupled TBME labels.

    Returned as 1-based (a, b, c, d, J, T) with a <= b, c <= d and
    (a, b) <= (c, d), in the order: T ascending, J ascending, bra pair
    ascending, ket pair ascending.  A pair (a, b) couples to J when
    |j_a - j_b| <= J <= j_a + j_b; a pair a == b needs J + T odd.
    """
    n = len(orbits)
    pairs = [(a, b) for a in range(n) for b in range(a, n)]
    out = []
    jmax = max(o.twoj for o in orbits)
    for T in (0, 1):
        for J in range(0, jmax + 1):
            chan = []
            for (a, b) in pairs:
                ja, jb = orbits[a].twoj, orbits[b].twoj
                if not (abs(ja - jb) <= 2 * J <= ja + jb):
                    continue
                if a == b and (J + T) % 2 == 0:
                    continue
                chan.append((a, b))
            for x in range(len(chan)):
                a, b = chan[x]
                pab = (orbits[a].l + orbits[b].l) % 2
                for y in range(x, len(chan)):
                    c, d = chan[y]
                    if (orbits[c].l + orbits[d].l) % 2 != pab:
                        continue
                    out.append((a + 1, b + 1, c + 1, d + 1, J, T))
    return out


def random_tbmes(orbits, seed: int = TBME_SEED, sigma: float = 1.0, sigma_diag: float = 2.0):
    """Seeded Gaussian V_JT(ab,cd) with mean 0: std sigma_diag when (ab)==(cd), else sigma.

    Returns a list of (a, b, c, d, J, T, V) tuples, labels 1-based.
    """
    rng = SplitMix64(seed)
    out = []
    for (a, b, c, d, J, T) in tbme_labels(orbits):
        s = sigma_diag if (a, b) == (c, d) else sigma
        out.append((a, b, c, d, J, T, s * rng.gauss()))
    return out


def space(name: str, seed: int = TBME_SEED):
    """(orbits, spe, tbmes) of a named valence space with seeded random TBMEs."""
    orbits, spe = SPACES[name]
    return list(orbits), list(spe), random_tbmes(orbits, seed)


def random_block(dim: int, k: int, seed: int = PIVOT_SEED, dtype=np.float64):
    """A [dim][k] block (k fastest) of N(0,1) entries, columns normalized.

    Drawn with numpy's PCG64 (these are bench/test vectors, not part of the
    method; the Lanczos pivot is passed to both sides as data).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal((dim, k))
    nrm = np.sqrt((x * x).sum(axis=0))
    nrm[nrm == 0] = 1.0
    return (x / nrm).astype(dtype)
