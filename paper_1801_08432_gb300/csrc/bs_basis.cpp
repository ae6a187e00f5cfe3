// M-scheme basis of proton x neutron Slater determinants.
//
// Sec. "Factorization of the basis" and Table al27: each species' SDs are
// occupation bitstrings grouped into sectors by (2M, parity); a proton sector
// pairs with the one neutron sector that completes M_p + M_n = M and the total
// parity, and every SD of the one combines with every SD of the other.  The
// basis-file pseudocode fixes proton index outer, neutron index inner
// ("pstart(ip) + nstart(jn)").  Sector order and SD order inside a sector are
// not fixed by the paper; here sectors go by 2M ascending then parity +/-,
// SDs by bitmask ascending.
#include <algorithm>
#include <map>

#include "bs_internal.h"

namespace bs {

int Species::find_sector(int twoM, int par) const
{
    // sectors are sorted by (twoM, par): binary search
    int lo = 0, hi = (int)sec.size() - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        const Sector &s = sec[mid];
        if (s.twoM == twoM && s.par == par) return mid;
        if (s.twoM < twoM || (s.twoM == twoM && s.par < par)) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

namespace {

// Depth-first enumeration of all n-subsets of the first ns states.
void enumerate(int ns, int n, int first, uint64_t mask, int twoM, int par, const std::vector<SpState> &st,
               std::map<std::pair<int, int>, std::vector<uint64_t>> &out)
{
    if (n == 0) {
        out[{twoM, par}].push_back(mask);
        return;
    }
    for (int s = first; s <= ns - n; ++s)
        enumerate(ns, n - 1, s + 1, mask | (1ULL << s), twoM + st[s].twom, par ^ st[s].par, st, out);
}

void build_species(const std::vector<SpState> &st, int n, Species &S)
{
    std::map<std::pair<int, int>, std::vector<uint64_t>> groups;
    enumerate((int)st.size(), n, 0, 0ULL, 0, 0, st, groups);
    S = Species();
    S.nparticles = n;
    for (auto &kv : groups) {
        std::vector<uint64_t> &v = kv.second;
        std::sort(v.begin(), v.end());
        Sector sec;
        sec.twoM = kv.first.first;
        sec.par = kv.first.second;
        sec.start = (int64_t)S.bits.size();
        sec.count = (int64_t)v.size();
        int sid = (int)S.sec.size();
        S.sec.push_back(sec);
        for (uint64_t m : v) {
            S.index.emplace(m, (int64_t)S.bits.size());
            S.bits.push_back(m);
            S.sec_of_sd.push_back(sid);
        }
    }
}

}  // namespace

int build_basis(Basis &B, const bs_orbit *orbits, int n_orbits, int Z, int N, int twoM, int parity, std::string &err)
{
    B = Basis();
    if (n_orbits <= 0 || !orbits) { err = "build_basis: no orbits"; return BS_EINVAL; }
    for (int a = 0; a < n_orbits; ++a) {
        if (orbits[a].twoj <= 0 || (orbits[a].twoj % 2) == 0) { err = "build_basis: 2j must be odd and positive"; return BS_EINVAL; }
        if (orbits[a].l < 0) { err = "build_basis: negative l"; return BS_EINVAL; }
        if (orbits[a].w != orbits[0].w) { err = "build_basis: W truncation is not supported (all w must be equal)"; return BS_EINVAL; }
        B.orb_l.push_back(orbits[a].l);
        B.orb_twoj.push_back(orbits[a].twoj);
        for (int tm = -orbits[a].twoj; tm <= orbits[a].twoj; tm += 2)
            B.st.push_back(SpState{a, tm, orbits[a].l & 1});
    }
    int ns = (int)B.st.size();
    if (ns > 64) { err = "build_basis: more than 64 single-particle states per species"; return BS_EINVAL; }
    if (Z < 0 || N < 0 || Z > ns || N > ns) { err = "build_basis: Z or N out of range"; return BS_EINVAL; }
    if (((twoM + Z + N) & 1) != 0) { err = "build_basis: 2M must have the parity of A = Z + N"; return BS_EINVAL; }
    if (parity != 1 && parity != -1) { err = "build_basis: parity must be +1 or -1"; return BS_EINVAL; }
    B.Z = Z; B.N = N; B.twoM = twoM; B.par = parity < 0 ? 1 : 0;
    build_species(B.st, Z, B.sp[0]);
    build_species(B.st, N, B.sp[1]);
    B.block_of_psec.assign(B.sp[0].sec.size(), -1);
    int64_t off = 0;
    for (size_t s = 0; s < B.sp[0].sec.size(); ++s) {
        const Sector &P = B.sp[0].sec[s];
        int n = B.sp[1].find_sector(twoM - P.twoM, B.par ^ P.par);
        if (n < 0) continue;
        Block b;
        b.ps = (int)s; b.ns = n; b.off = off;
        b.nP = P.count; b.nN = B.sp[1].sec[n].count;
        B.block_of_psec[s] = (int)B.blocks.size();
        B.blocks.push_back(b);
        off += b.nP * b.nN;
    }
    B.dim = off;
    if (B.dim == 0) { err = "build_basis: empty basis"; return BS_EINVAL; }
    for (int sp = 0; sp < 2; ++sp)
        for (const Sector &s : B.sp[sp].sec)
            if (s.count > 65535) { err = "build_basis: a sector holds more than 65535 SDs"; return BS_EINVAL; }
    return BS_OK;
}

}  // namespace bs
