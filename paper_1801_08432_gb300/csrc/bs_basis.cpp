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
//
// W truncation (Sec. "Truncation of the many-body space"): every orbit has a
// non-negative integer weight w, an SD's W is the sum over its occupied
// states, and the kept states have W_p + W_n <= W_min + the allowed
// excitation, W_min being the smallest total any Z-proton, N-neutron state
// can have.  Sectors are then keyed by (2M, parity, W) (the .bas description
// of sectors) and sorted by 2M, parity, then W; a proton sector pairs with
// every conjugate neutron sector whose W fits ("# of conjugate sectors"), in
// neutron-sector order, which is the basis-file loop order (proton sector,
// its conjugate neutron sectors, proton SDs, neutron SDs).
#include <algorithm>
#include <map>
#include <tuple>

#include "bs_internal.h"

namespace bs {

int Species::find_sector(int twoM, int par, int W) const
{
    // sectors are sorted by (twoM, par, W): binary search
    int lo = 0, hi = (int)sec.size() - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        const Sector &s = sec[mid];
        if (s.twoM == twoM && s.par == par && s.W == W) return mid;
        if (s.twoM < twoM || (s.twoM == twoM && (s.par < par || (s.par == par && s.W < W)))) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

int Basis::block_of(int ps, int ns) const
{
    if (ps < 0 || ns < 0 || ps >= (int)sp[0].sec.size() || ns >= (int)sp[1].sec.size()) return -1;
    return blk_of_pair[(size_t)ps * sp[1].sec.size() + (size_t)ns];
}

namespace {

// Depth-first enumeration of all n-subsets of the first ns states, keyed by
// (2M, parity, W); with wcap >= 0, subsets whose W exceeds wcap are dropped
// (they cannot appear in any kept state).  W is 0 unless `weighted`.
void enumerate(int ns, int n, int first, uint64_t mask, int twoM, int par, int W, bool weighted, int wcap,
               const std::vector<SpState> &st, std::map<std::tuple<int, int, int>, std::vector<uint64_t>> &out)
{
    if (wcap >= 0 && W > wcap) return;
    if (n == 0) {
        out[{twoM, par, W}].push_back(mask);
        return;
    }
    for (int s = first; s <= ns - n; ++s)
        enumerate(ns, n - 1, s + 1, mask | (1ULL << s), twoM + st[s].twom, par ^ st[s].par,
                  weighted ? W + st[s].w : 0, weighted, wcap, st, out);
}

void build_species(const std::vector<SpState> &st, int n, bool weighted, int wcap, Species &S)
{
    std::map<std::tuple<int, int, int>, std::vector<uint64_t>> groups;
    enumerate((int)st.size(), n, 0, 0ULL, 0, 0, 0, weighted, wcap, st, groups);
    S = Species();
    S.nparticles = n;
    for (auto &kv : groups) {
        std::vector<uint64_t> &v = kv.second;
        std::sort(v.begin(), v.end());
        Sector sec;
        sec.twoM = std::get<0>(kv.first);
        sec.par = std::get<1>(kv.first);
        sec.W = std::get<2>(kv.first);
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

int build_basis(Basis &B, const bs_orbit *orbits, int n_orbits, int Z, int N, int twoM, int parity, int max_excite,
                std::string &err)
{
    B = Basis();
    if (n_orbits <= 0 || !orbits) { err = "build_basis: no orbits"; return BS_EINVAL; }
    for (int a = 0; a < n_orbits; ++a) {
        if (orbits[a].twoj <= 0 || (orbits[a].twoj % 2) == 0) { err = "build_basis: 2j must be odd and positive"; return BS_EINVAL; }
        if (orbits[a].l < 0) { err = "build_basis: negative l"; return BS_EINVAL; }
        if (max_excite >= 0 && orbits[a].w < 0) { err = "build_basis: truncation weights w must be non-negative"; return BS_EINVAL; }
        B.orb_l.push_back(orbits[a].l);
        B.orb_twoj.push_back(orbits[a].twoj);
        for (int tm = -orbits[a].twoj; tm <= orbits[a].twoj; tm += 2)
            B.st.push_back(SpState{a, tm, orbits[a].l & 1, orbits[a].w});
    }
    int ns = (int)B.st.size();
    if (ns > 64) { err = "build_basis: more than 64 single-particle states per species"; return BS_EINVAL; }
    if (Z < 0 || N < 0 || Z > ns || N > ns) { err = "build_basis: Z or N out of range"; return BS_EINVAL; }
    if (((twoM + Z + N) & 1) != 0) { err = "build_basis: 2M must have the parity of A = Z + N"; return BS_EINVAL; }
    if (parity != 1 && parity != -1) { err = "build_basis: parity must be +1 or -1"; return BS_EINVAL; }
    B.Z = Z; B.N = N; B.twoM = twoM; B.par = parity < 0 ? 1 : 0;
    B.trunc = max_excite >= 0;
    int wcap_p = -1, wcap_n = -1;
    if (B.trunc) {
        // W_min: the lowest-w states filled, for each species
        std::vector<int> ws;
        for (const SpState &t : B.st) ws.push_back(t.w);
        std::sort(ws.begin(), ws.end());
        int wmin_p = 0, wmin_n = 0;
        for (int i = 0; i < Z; ++i) wmin_p += ws[(size_t)i];
        for (int i = 0; i < N; ++i) wmin_n += ws[(size_t)i];
        B.w_max = wmin_p + wmin_n + max_excite;
        wcap_p = B.w_max - wmin_n;   // no proton SD above this fits any neutron SD
        wcap_n = B.w_max - wmin_p;
    }
    build_species(B.st, Z, B.trunc, wcap_p, B.sp[0]);
    build_species(B.st, N, B.trunc, wcap_n, B.sp[1]);
    const size_t nps = B.sp[0].sec.size(), nns = B.sp[1].sec.size();
    B.block_of_psec.assign(nps, -1);
    B.blk_of_pair.assign(nps * nns, -1);
    int64_t off = 0;
    for (size_t s = 0; s < nps; ++s) {
        const Sector &P = B.sp[0].sec[s];
        for (size_t n = 0; n < nns; ++n) {
            const Sector &Q = B.sp[1].sec[n];
            if (Q.twoM != twoM - P.twoM || Q.par != (B.par ^ P.par)) continue;
            if (B.trunc && P.W + Q.W > B.w_max) continue;
            Block b;
            b.ps = (int)s; b.ns = (int)n; b.off = off;
            b.nP = P.count; b.nN = Q.count;
            if (B.block_of_psec[s] < 0) B.block_of_psec[s] = (int)B.blocks.size();
            B.blk_of_pair[s * nns + n] = (int)B.blocks.size();
            B.blocks.push_back(b);
            off += b.nP * b.nN;
        }
    }
    B.dim = off;
    if (B.dim == 0) { err = "build_basis: empty basis"; return BS_EINVAL; }
    for (int sp = 0; sp < 2; ++sp)
        for (const Sector &s : B.sp[sp].sec)
            if (s.count > 65535) { err = "build_basis: a sector holds more than 65535 SDs"; return BS_EINVAL; }
    return BS_OK;
}

}  // namespace bs
