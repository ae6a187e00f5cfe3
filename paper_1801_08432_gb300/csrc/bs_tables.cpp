// Jump tables (Sec. "The Lanczos algorithm and computational cost", jumps and
// Table jumps): the proton-only and neutron-only parts of H are stored as
// species-local sparse matrices (two-body moves, with the SPE and the
// like-particle diagonal folded in), the pn part as one-body jumps of each
// species that a kernel multiplies on the fly with the decoupled W_pn.
//
// Everything is stored by DESTINATION (the paper stores one direction and
// applies its transpose for the "back" half; here both directions are kept so
// that every output element has one owner and no atomics are needed).
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>

#include "bs_internal.h"

namespace bs {

namespace {

// Fermion sign of a_s or a+_s on bitmask m (the paper's rule): (-1)^(number of
// occupied states below s).
inline int sign_below(uint64_t m, int s)
{
    return (__builtin_popcountll(m & ((1ULL << s) - 1ULL)) & 1) ? -1 : 1;
}

// Like-particle part of one species: sum_{i<j,k<l} W(ij,kl) a+_i a+_j a_l a_k
// plus sum_s e_s n_s, as a destination CSR over the species' SDs.  The
// operator is real symmetric (W(ij,kl) = W(kl,ij)), so the row of SD g,
// <g|V|m>, is read off V|g> = sum_m <m|V|g> |m>: every row is built from its
// own SD, in parallel, with no scatter.  Moves that stay in g's sector go to
// L (source as a local index in the sector); in a W-truncated basis a move
// can change W, and those go to X, one class per (source, destination)
// sector pair.
void like_jumps(const Basis &B, const Interaction &I, int spc, LikeJumps &L, LikeCross &X, int64_t &nent)
{
    const Species &S = B.sp[spc];
    const int ns = (int)B.st.size();
    const int64_t nsd = (int64_t)S.bits.size();
    std::vector<std::vector<std::pair<int64_t, double>>> rows((size_t)nsd);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t g = 0; g < nsd; ++g) {
        const uint64_t X = S.bits[g];
        std::vector<std::pair<int64_t, double>> &r = rows[(size_t)g];
        double e = 0.0;
        for (int s = 0; s < ns; ++s)
            if (X >> s & 1) e += I.spe_state[s];
        r.emplace_back(g, e);
        for (int k = 0; k < ns; ++k) {
            if (!(X >> k & 1)) continue;
            for (int l = k + 1; l < ns; ++l) {
                if (!(X >> l & 1)) continue;
                const int q = I.pair_id[(size_t)k * ns + l];
                // a_l a_k
                int sg = sign_below(X, k);
                uint64_t m1 = X & ~(1ULL << k);
                sg *= sign_below(m1, l);
                m1 &= ~(1ULL << l);
                for (int p : I.pairs_by_key[I.key_of_pair[q]]) {
                    const double w = I.Wpp[(size_t)p * I.npairs + q];
                    if (w == 0.0) continue;
                    const int i = I.pair_i[p], j = I.pair_j[p];
                    if ((m1 >> i & 1) || (m1 >> j & 1)) continue;
                    // a+_i a+_j
                    int s2 = sign_below(m1, j);
                    uint64_t m2 = m1 | (1ULL << j);
                    s2 *= sign_below(m2, i);
                    m2 |= (1ULL << i);
                    const auto it = S.index.find(m2);
                    if (it == S.index.end()) continue;   // above the W cap of a truncated basis
                    r.emplace_back(it->second, sg * s2 * w);
                }
            }
        }
        std::sort(r.begin(), r.end(), [](const std::pair<int64_t, double> &a, const std::pair<int64_t, double> &b) {
            return a.first < b.first;
        });
        size_t w = 0;
        for (size_t t = 0; t < r.size(); ++t) {
            if (w > 0 && r[w - 1].first == r[t].first) r[w - 1].second += r[t].second;
            else r[w++] = r[t];
        }
        r.resize(w);
    }
    // same-sector moves
    L.ptr.assign((size_t)nsd + 1, 0);
    for (int64_t g = 0; g < nsd; ++g) {
        int64_t n = 0;
        for (const auto &e : rows[(size_t)g]) n += S.sec_of_sd[(size_t)e.first] == S.sec_of_sd[(size_t)g];
        L.ptr[(size_t)g + 1] = L.ptr[(size_t)g] + n;
    }
    L.src.resize((size_t)L.ptr[(size_t)nsd]);
    L.coef.resize((size_t)L.ptr[(size_t)nsd]);
    const size_t nsec = S.sec.size();
    std::map<std::pair<int, int>, std::vector<std::pair<int64_t, std::pair<int32_t, double>>>> cross;
    for (int64_t g = 0; g < nsd; ++g) {
        int64_t o = L.ptr[(size_t)g];
        const int sd = S.sec_of_sd[(size_t)g];
        for (const auto &e : rows[(size_t)g]) {
            const int ss = S.sec_of_sd[(size_t)e.first];
            const int32_t loc = (int32_t)(e.first - S.sec[(size_t)ss].start);
            if (ss == sd) {
                L.src[(size_t)o] = loc;
                L.coef[(size_t)o] = e.second;
                ++o;
            } else {
                cross[{ss, sd}].push_back({g - S.sec[(size_t)sd].start, {loc, e.second}});
            }
        }
        std::vector<std::pair<int64_t, double>>().swap(rows[(size_t)g]);
    }
    nent = L.ptr[(size_t)nsd];
    // moves between sectors, one class per (source, destination) pair
    X = LikeCross();
    (void)nsec;
    for (auto &kv : cross) {
        LikeCrossClass c;
        c.s_src = kv.first.first;
        c.s_dst = kv.first.second;
        c.ptr_off = (int64_t)X.ptr.size();
        const int64_t nd = S.sec[(size_t)c.s_dst].count;
        const auto &v = kv.second;   // in destination order (rows were visited in order)
        size_t t = 0;
        for (int64_t dl = 0; dl <= nd; ++dl) {
            while (t < v.size() && v[t].first < dl) {
                X.src.push_back(v[t].second.first);
                X.coef.push_back(v[t].second.second);
                ++t;
            }
            X.ptr.push_back((int64_t)X.src.size());
        }
        X.cls.push_back(c);
        nent += (int64_t)v.size();
    }
}

// One-body jumps a+_i a_k of one species (i == k included: the number
// operator), grouped by (source sector, destination sector), destination CSR.
// For destination d the incoming jumps come from s = a+_k a_i d with i
// occupied in d; <d|a+_i a_k|s> = <s|a+_k a_i|d> is the sign of a_i then a+_k
// on d.  The stored operator index is that of a+_i a_k.
void onebody_jumps(const Basis &B, const Interaction &I, int spc, OneBodyJumps &J, int64_t &nent)
{
    const Species &S = B.sp[spc];
    const int ns = (int)B.st.size();
    const int nsec = (int)S.sec.size();
    struct E { int32_t dst_loc; uint32_t packed; };
    std::vector<std::vector<E>> bucket((size_t)nsec * nsec);
    std::vector<int> grp((size_t)nsec * nsec, -1);
    for (int64_t d = 0; d < (int64_t)S.bits.size(); ++d) {
        const uint64_t X = S.bits[d];
        const int sdst = S.sec_of_sd[d];
        const int32_t dloc = (int32_t)(d - S.sec[sdst].start);
        for (int i = 0; i < ns; ++i) {
            if (!(X >> i & 1)) continue;
            const int s1 = sign_below(X, i);
            const uint64_t m1 = X & ~(1ULL << i);
            for (int k = 0; k < ns; ++k) {
                if (m1 >> k & 1) continue;
                const int s2 = sign_below(m1, k);
                const auto it = S.index.find(m1 | (1ULL << k));
                if (it == S.index.end()) continue;   // above the W cap of a truncated basis
                const int64_t gs = it->second;
                const int ssrc = S.sec_of_sd[gs];
                const int op = i * ns + k;
                const uint32_t sloc = (uint32_t)(gs - S.sec[ssrc].start);
                const uint32_t packed = sloc | ((uint32_t)I.ops.local_of_op[op] << 16) | ((s1 * s2 < 0) ? 0x80000000u : 0u);
                bucket[(size_t)ssrc * nsec + sdst].push_back(E{dloc, packed});
                grp[(size_t)ssrc * nsec + sdst] = I.ops.group_of_op[op];
            }
        }
    }
    J.cls.clear();
    J.ptr.clear();
    J.ent.clear();
    for (int a = 0; a < nsec; ++a)
        for (int b = 0; b < nsec; ++b) {
            auto &v = bucket[(size_t)a * nsec + b];
            if (v.empty()) continue;
            OneBodyClass c;
            c.s_src = a;
            c.s_dst = b;
            c.group = grp[(size_t)a * nsec + b];
            c.ptr_off = (int64_t)J.ptr.size();
            const int64_t nd = S.sec[b].count;
            size_t t = 0;
            for (int64_t dl = 0; dl <= nd; ++dl) {
                while (t < v.size() && v[t].dst_loc < dl) J.ent.push_back(v[t++].packed);
                J.ptr.push_back((int64_t)J.ent.size());
            }
            J.cls.push_back(c);
            std::vector<E>().swap(v);
        }
    nent = (int64_t)J.ent.size();
}

// Order the entries of the (at most 32) lists of one ELL slice so that at every
// step the lanes' source columns spread over the eight residues mod 8: a warp
// then gathers from all shared-memory bank groups at once.  key(e) gives the
// source column of entry e.  Any order of a list sums the same terms; this one
// is fixed at build time, so results stay bit-reproducible.
template <typename Entry, typename Key>
void bank_order(std::vector<std::vector<Entry>> &lists, Key key)
{
    // key(entry, lane) -> residue class to balance
    size_t lmax = 0;
    for (auto &l : lists) lmax = std::max(lmax, l.size());
    std::vector<std::vector<Entry>> out(lists.size());
    // a 16-byte shared-memory load is served a quarter warp (8 lanes) at a
    // time: balance the residues inside each quarter
    for (size_t v = 0; v < lmax; ++v) {
        int cnt[4][8] = {};
        for (size_t lane = 0; lane < lists.size(); ++lane) {
            auto &l = lists[lane];
            if (l.empty()) continue;
            size_t best = 0;
            const int ln = (int)lane;
            int *c = cnt[(lane >> 3) & 3];
            for (size_t t = 1; t < l.size(); ++t)
                if (c[key(l[t], ln) & 7] < c[key(l[best], ln) & 7]) best = t;
            c[key(l[best], ln) & 7]++;
            out[lane].push_back(l[best]);
            l.erase(l.begin() + (long)best);
        }
    }
    lists.swap(out);
}

// Step order of the neutron one-body lists of one 32-column slice for the
// kernels that read a 32-byte element (k = 8 floats) as two 16-byte chunks
// and a 16-byte weight quadruple per entry.  Every entry also gets a rotation
// bit (bit 31): which chunk its lane loads first.  At every step and in every
// quarter warp (the lanes one 16-byte shared-memory load serves together) the
// greedy picks, lane by lane (longest remaining list first), the entry and
// rotation that add the fewest bank conflicts: a new chunk address in an
// occupied residue mod 8 costs its occupancy + 1, a new weight row
// (index (e >> 16) & 0x7FFF, residue mod 8) half as much.  Lists shorter than
// the slice's longest are padded with `pad` (a zero weight), which also gets a
// rotation.  Output: lists[lane] of length lmax, in step order.
void bank_schedule_rot(std::vector<std::vector<uint32_t>> &lists, uint32_t pad)
{
    size_t lmax = 0;
    for (auto &l : lists) lmax = std::max(lmax, l.size());
    std::vector<std::vector<uint32_t>> rem = lists, out(lists.size());
    for (size_t v = 0; v < lmax; ++v)
        for (size_t q = 0; q * 8 < lists.size(); ++q) {
            std::vector<size_t> lanes;
            for (size_t l = q * 8; l < std::min(lists.size(), q * 8 + 8); ++l) lanes.push_back(l);
            std::stable_sort(lanes.begin(), lanes.end(), [&](size_t a, size_t b) { return rem[a].size() > rem[b].size(); });
            int ares[8] = {}, wres[8] = {};
            std::vector<uint32_t> used_a, used_w;
            for (size_t l : lanes) {
                const bool has = !rem[l].empty();
                const size_t nc = has ? rem[l].size() : 1;
                double best = 1e30;
                size_t bt = 0;
                uint32_t br = 0;
                for (size_t t = 0; t < nc; ++t) {
                    const uint32_t e = has ? rem[l][t] : pad;
                    const uint32_t w = (e >> 16) & 0x7FFFu;
                    for (uint32_t r = 0; r < 2; ++r) {
                        const uint32_t a = 2 * (e & 0xFFFFu) + r;
                        const bool na = std::find(used_a.begin(), used_a.end(), a) == used_a.end();
                        const bool nw = std::find(used_w.begin(), used_w.end(), w) == used_w.end();
                        const double c = (na ? ares[a & 7] + 1 : 0) + 0.5 * (nw ? wres[w & 7] + 1 : 0);
                        if (c < best) { best = c; bt = t; br = r; }
                    }
                }
                const uint32_t e = has ? rem[l][bt] : pad;
                if (has) rem[l].erase(rem[l].begin() + (long)bt);
                const uint32_t a = 2 * (e & 0xFFFFu) + br, w = (e >> 16) & 0x7FFFu;
                if (std::find(used_a.begin(), used_a.end(), a) == used_a.end()) { used_a.push_back(a); ares[a & 7]++; }
                if (std::find(used_w.begin(), used_w.end(), w) == used_w.end()) { used_w.push_back(w); wres[w & 7]++; }
                out[l].push_back(e | (br << 31));
            }
        }
    lists.swap(out);
}

// Step order of the neutron one-body lists of one 32-column slice for the
// pn-core kernel, whose lanes read a 32-byte element's two 16-byte chunks in
// a fixed per-lane order (lane bit 2 picks the chunk first read), so that the
// registers need no per-entry reordering.  A quarter warp's first loads then
// avoid each other's bank groups when its lanes 0-3 (and 4-7) use source
// columns of distinct residues mod 4; at every step the greedy picks, lane by
// lane (longest remaining list first), the entry that adds the fewest
// conflicts, counting a new chunk address in an occupied bank group by its
// occupancy + 1 and a new weight row (residue mod 8) half as much.  Shorter
// lists are padded with `pad`.  Output: lists[lane] of length lmax.
// Cost of one quarter warp's step: the wavefronts of the two chunk loads
// (the most distinct addresses in one bank group) plus half those of the
// weight-row load.
void quarter_terms(const uint32_t *e, const uint32_t *rot, int n, double &chunks, double &weights)
{
    double tot = 0.0;
    for (uint32_t chunk = 0; chunk < 2; ++chunk) {
        uint32_t addr[8];
        int cnt[8] = {}, mx = 0;
        for (int i = 0; i < n; ++i) {
            const uint32_t a = 2 * (e[i] & 0xFFFFu) + (rot[i] ^ chunk);
            bool seen = false;
            for (int j = 0; j < i; ++j) seen = seen || addr[j] == a;
            addr[i] = a;
            if (!seen) mx = std::max(mx, ++cnt[a & 7]);
        }
        tot += mx;
    }
    uint32_t wrow[8];
    int cnt[8] = {}, mx = 0;
    for (int i = 0; i < n; ++i) {
        const uint32_t w = (e[i] >> 16) & 0x7FFFu;
        bool seen = false;
        for (int j = 0; j < i; ++j) seen = seen || wrow[j] == w;
        wrow[i] = w;
        if (!seen) mx = std::max(mx, ++cnt[w & 7]);
    }
    chunks = tot;
    weights = mx;
}

double quarter_cost(const uint32_t *e, const uint32_t *rot, int n)
{
    double x, w;
    quarter_terms(e, rot, n, x, w);
    return x + 0.5 * w;
}

// Wavefronts of one quarter warp's element load when an element is one
// 16-byte chunk (k = 4 FP32 vectors): the most distinct source columns that
// share a bank group (src mod 8).
double quarter_cost_k4(const uint32_t *e, int n)
{
    uint32_t addr[8];
    int cnt[8] = {}, mx = 0;
    for (int i = 0; i < n; ++i) {
        const uint32_t a = e[i] & 0xFFFFu;
        bool seen = false;
        for (int j = 0; j < i; ++j) seen = seen || addr[j] == a;
        addr[i] = a;
        if (!seen) mx = std::max(mx, ++cnt[a & 7]);
    }
    return mx;
}


// Wavefronts of one quarter warp's loads for the step orders (8 lanes, entries
// src | weight row << 16): m0 for each of the two k = 8 chunk loads, m4 for
// the k = 4 element load, mw for the weight-row load; each is the most
// distinct addresses that share one of the 8 bank groups.  The second chunk's
// addresses are the first's with the low bit flipped (a lane reads the other
// half of its element), a bijection that maps bank group g to g ^ 1, so both
// chunk loads take the same count; one pass over the lane pairs finds all
// three (the values of quarter_terms and quarter_cost_k4, at a third of the
// comparisons).
inline void quarter_counts(const uint32_t *e, const uint32_t *rot, int &m0, int &m4, int &mw)
{
    uint32_t s[8], w[8];
    for (int i = 0; i < 8; ++i) {
        s[i] = e[i] & 0xFFFFu;
        w[i] = (e[i] >> 16) & 0x7FFFu;
    }
    int c0[8] = {}, c4[8] = {}, cw[8] = {};
    m0 = m4 = mw = 0;
    for (int i = 0; i < 8; ++i) {
        bool d0 = false, d4 = false, dw = false;
        for (int j = 0; j < i; ++j) {
            const bool eq = s[j] == s[i];
            d4 = d4 || eq;
            d0 = d0 || (eq && rot[j] == rot[i]);
            dw = dw || w[j] == w[i];
        }
        if (!d0) m0 = std::max(m0, ++c0[(2 * s[i] + rot[i]) & 7]);
        if (!d4) m4 = std::max(m4, ++c4[s[i] & 7]);
        if (!dw) mw = std::max(mw, ++cw[w[i] & 7]);
    }
}

// The annealing objective of the pn-core order: the k = 8 chunk loads, the
// weight load counted in full and half the k = 4 element load, so that one
// order serves both block widths the product runs at.
double pn_order_cost(const uint32_t *e, const uint32_t *rot)
{
    int m0, m4, mw;
    quarter_counts(e, rot, m0, m4, mw);
    return 2.0 * m0 + mw + 0.5 * m4;
}

void bank_schedule_lane(std::vector<std::vector<uint32_t>> &lists, uint32_t pad)
{
    size_t lmax = 0;
    for (auto &l : lists) lmax = std::max(lmax, l.size());
    std::vector<std::vector<uint32_t>> rem = lists, out(lists.size());
    for (size_t v = 0; v < lmax; ++v)
        for (size_t q = 0; q * 8 < lists.size(); ++q) {
            std::vector<size_t> lanes;
            for (size_t l = q * 8; l < std::min(lists.size(), q * 8 + 8); ++l) lanes.push_back(l);
            std::stable_sort(lanes.begin(), lanes.end(), [&](size_t a, size_t b) { return rem[a].size() > rem[b].size(); });
            int ares[8] = {}, wres[8] = {};
            std::vector<uint32_t> used_a, used_w;
            std::vector<uint32_t> pick(lanes.size());
            uint32_t rots[8];
            for (size_t k = 0; k < lanes.size(); ++k) {
                const size_t l = lanes[k];
                const bool has = !rem[l].empty();
                const size_t nc = has ? rem[l].size() : 1;
                const uint32_t r = (uint32_t)(l >> 2) & 1u;
                rots[k] = r;
                double best = 1e30;
                size_t bt = 0;
                for (size_t t = 0; t < nc; ++t) {
                    const uint32_t e = has ? rem[l][t] : pad;
                    const uint32_t w = (e >> 16) & 0x7FFFu;
                    const uint32_t a = 2 * (e & 0xFFFFu) + r;
                    const bool na = std::find(used_a.begin(), used_a.end(), a) == used_a.end();
                    const bool nw = std::find(used_w.begin(), used_w.end(), w) == used_w.end();
                    const double c = (na ? ares[a & 7] + 1 : 0) + 0.5 * (nw ? wres[w & 7] + 1 : 0);
                    if (c < best) { best = c; bt = t; }
                }
                const uint32_t e = has ? rem[l][bt] : pad;
                pick[k] = e;
                const uint32_t a = 2 * (e & 0xFFFFu) + r, w = (e >> 16) & 0x7FFFu;
                if (std::find(used_a.begin(), used_a.end(), a) == used_a.end()) { used_a.push_back(a); ares[a & 7]++; }
                if (std::find(used_w.begin(), used_w.end(), w) == used_w.end()) { used_w.push_back(w); wres[w & 7]++; }
            }
            // then single-lane exchanges while they lower the quarter's cost
            double cur = quarter_cost(pick.data(), rots, (int)pick.size());
            for (int it = 0; it < 3; ++it) {
                bool better = false;
                for (size_t k = 0; k < lanes.size(); ++k) {
                    const size_t l = lanes[k];
                    for (uint32_t e : rem[l]) {
                        if (e == pick[k]) continue;
                        const uint32_t old = pick[k];
                        pick[k] = e;
                        const double c = quarter_cost(pick.data(), rots, (int)pick.size());
                        if (c < cur - 1e-9) { cur = c; better = true; }
                        else pick[k] = old;
                    }
                }
                if (!better) break;
            }
            for (size_t k = 0; k < lanes.size(); ++k) {
                const size_t l = lanes[k];
                if (!rem[l].empty()) rem[l].erase(std::find(rem[l].begin(), rem[l].end(), pick[k]));
                out[l].push_back(pick[k]);
            }
        }
    lists.swap(out);
}

// Whole-slice refinement of the pn-core step order (lmax steps x 32 lanes at E,
// [step][lane]) under pn_order_cost: per quarter warp, a move
// either swaps one lane's entries at two steps or, for a padding entry (zero
// weight row), sets its source column to 0..3 (when the source row has 4 or
// more), so that it takes a free bank group.  Moves are accepted by the
// Metropolis rule under a temperature falling linearly from 0.3 wavefronts to
// zero, and the best order seen is kept.  The stepwise greedy above cannot
// trade entries between steps; this can.  Deterministic: a splitmix64 stream
// seeded per slice.
// ipe = moves per entry.
void anneal_slice(uint32_t *E, size_t lmax, uint32_t pad, int64_t nsrc, uint64_t seed, int ipe)
{
    if (lmax < 1 || ipe < 1) return;
    uint64_t st = seed;
    auto next = [&st]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto unif = [&next]() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); };
    const uint32_t rots[8] = {0, 0, 0, 0, 1, 1, 1, 1};
    std::vector<uint32_t> q8(lmax * 8), best(lmax * 8);
    std::vector<double> cost(lmax);
    for (size_t q = 0; q < 4; ++q) {
        for (size_t v = 0; v < lmax; ++v)
            for (size_t k = 0; k < 8; ++k) q8[v * 8 + k] = E[v * 32 + q * 8 + k];
        double cur = 0.0;
        for (size_t v = 0; v < lmax; ++v) cur += (cost[v] = pn_order_cost(&q8[v * 8], rots));
        double bestc = cur;
        best = q8;
        const int64_t n = (int64_t)ipe * (int64_t)lmax * 8;
        for (int64_t it = 0; it < n; ++it) {
            const double T = 0.3 * (1.0 - (double)it / (double)n) + 1e-3;
            const size_t k = (size_t)(next() % 8), v1 = (size_t)(next() % lmax);
            uint32_t &a = q8[v1 * 8 + k];
            if ((a >> 16) == (pad >> 16) && nsrc >= 4 && next() % 10 < 3) {   // a padding entry's source column
                const uint32_t old = a;
                a = pad | (uint32_t)(next() % 4);
                const double c1 = pn_order_cost(&q8[v1 * 8], rots), d = c1 - cost[v1];
                if (d < 0 || unif() < std::exp(-d / T)) {
                    cost[v1] = c1;
                    cur += d;
                    if (cur < bestc - 1e-9) { bestc = cur; best = q8; }
                } else {
                    a = old;
                }
                continue;
            }
            const size_t v2 = (size_t)(next() % lmax);
            uint32_t &b = q8[v2 * 8 + k];
            if (v1 == v2 || a == b) continue;
            std::swap(a, b);
            const double c1 = pn_order_cost(&q8[v1 * 8], rots), c2 = pn_order_cost(&q8[v2 * 8], rots);
            const double d = c1 + c2 - cost[v1] - cost[v2];
            if (d < 0 || unif() < std::exp(-d / T)) {
                cost[v1] = c1;
                cost[v2] = c2;
                cur += d;
                if (cur < bestc - 1e-9) { bestc = cur; best = q8; }
            } else {
                std::swap(a, b);
            }
        }
        for (size_t v = 0; v < lmax; ++v)
            for (size_t k = 0; k < 8; ++k) E[v * 32 + q * 8 + k] = best[v * 8 + k];
    }
}

// The like-particle lists (src, coef) of one quarter warp q (lanes 8q .. 8q+7)
// of one 32-column slice, [step][lane]: the same refinement for the kernels
// that read a 32-byte element's chunks lane parity first (k = 8) or a
// 16-byte element (k = 4), at the cost of the quarter's two chunk loads plus
// its k = 4 element load (no weights); src and coef move together.
// Quarters touch disjoint lanes, so they can run in parallel.
void anneal_nn_quarter(int32_t *src, double *coef, size_t lmax, size_t q, uint64_t seed, int ipe)
{
    if (lmax < 2 || ipe < 1) return;
    uint64_t st = seed;
    auto next = [&st]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto unif = [&next]() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); };
    const uint32_t rots[8] = {0, 1, 0, 1, 0, 1, 0, 1};
    auto cost8 = [&rots](const uint32_t *e) {   // k = 8 chunk loads + the k = 4 element load
        int m0, m4, mw;
        quarter_counts(e, rots, m0, m4, mw);
        return 2.0 * m0 + m4;
    };
    std::vector<uint32_t> q8(lmax * 8), best(lmax * 8);
    std::vector<uint32_t> idx(lmax * 8), bidx(lmax * 8);   // the entries' original steps, to move coef
    std::vector<double> cost(lmax);
    for (size_t v = 0; v < lmax; ++v)
        for (size_t k = 0; k < 8; ++k) {
            q8[v * 8 + k] = (uint32_t)src[v * 32 + q * 8 + k] & 0xFFFFu;
            idx[v * 8 + k] = (uint32_t)v;
        }
    double cur = 0.0;
    for (size_t v = 0; v < lmax; ++v) cur += (cost[v] = cost8(&q8[v * 8]));
    double bestc = cur;
    best = q8;
    bidx = idx;
    const int64_t n = (int64_t)ipe * (int64_t)lmax * 8;
    for (int64_t it = 0; it < n; ++it) {
        const double T = 0.6 * (1.0 - (double)it / (double)n) + 1e-3;
        const size_t k = (size_t)(next() % 8), v1 = (size_t)(next() % lmax), v2 = (size_t)(next() % lmax);
        if (v1 == v2 || q8[v1 * 8 + k] == q8[v2 * 8 + k]) continue;
        std::swap(q8[v1 * 8 + k], q8[v2 * 8 + k]);
        std::swap(idx[v1 * 8 + k], idx[v2 * 8 + k]);
        const double a = cost8(&q8[v1 * 8]), b = cost8(&q8[v2 * 8]);
        const double d = a + b - cost[v1] - cost[v2];
        if (d < 0 || unif() < std::exp(-d / T)) {
            cost[v1] = a;
            cost[v2] = b;
            cur += d;
            if (cur < bestc - 1e-9) { bestc = cur; best = q8; bidx = idx; }
        } else {
            std::swap(q8[v1 * 8 + k], q8[v2 * 8 + k]);
            std::swap(idx[v1 * 8 + k], idx[v2 * 8 + k]);
        }
    }
    std::vector<int32_t> s2(lmax * 8);
    std::vector<double> c2(lmax * 8);
    for (size_t v = 0; v < lmax; ++v)
        for (size_t k = 0; k < 8; ++k) {
            const size_t from = (size_t)bidx[v * 8 + k] * 32 + q * 8 + k;
            s2[v * 8 + k] = src[from];
            c2[v * 8 + k] = coef[from];
        }
    for (size_t v = 0; v < lmax; ++v)
        for (size_t k = 0; k < 8; ++k) {
            src[v * 32 + q * 8 + k] = s2[v * 8 + k];
            coef[v * 32 + q * 8 + k] = c2[v * 8 + k];
        }
}

// Length-sorted, 32-column-sliced ELL of packed one-body lists given as a CSR
// (ptr[0..ncols]).  put(csr_index) returns one entry.
template <typename Put>
void append_ell(Ell &E, int64_t ncols, const int64_t *ptr, Put put, int64_t &col_off, int64_t &slice_base,
                uint32_t pad)
{
    col_off = (int64_t)E.col.size();
    slice_base = (int64_t)E.soff.size();
    std::vector<int32_t> order((size_t)ncols);
    for (int64_t c = 0; c < ncols; ++c) order[(size_t)c] = (int32_t)c;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return (ptr[a + 1] - ptr[a]) > (ptr[b + 1] - ptr[b]);
    });
    for (int64_t i = 0; i < ncols; ++i) {
        E.col.push_back(order[(size_t)i]);
        E.len.push_back((int32_t)(ptr[order[(size_t)i] + 1] - ptr[order[(size_t)i]]));
    }
    for (int64_t s0 = 0; s0 < ncols; s0 += 32) {
        const int64_t base = (int64_t)E.ent.size();
        E.soff.push_back(base);
        const int32_t lmax = E.len[(size_t)(col_off + s0)];   // longest first
        E.ent.resize((size_t)(base + (int64_t)lmax * 32), pad);
        std::vector<std::vector<uint32_t>> lists;
        for (int64_t lane = 0; lane < 32 && s0 + lane < ncols; ++lane) {
            const int32_t c = order[(size_t)(s0 + lane)];
            lists.emplace_back();
            for (int64_t v = 0; v < ptr[c + 1] - ptr[c]; ++v) lists.back().push_back(put(ptr[c] + v));
        }
        // the row kernel reads a 32-byte element (k = 8 floats) as two 16-byte
        // chunks, lane-parity first: balance (2 src + lane parity) mod 8
        bank_order(lists, [](uint32_t e, int ln) { return 2 * (int)(e & 0xFFFFu) + (ln & 1); });
        for (size_t lane = 0; lane < lists.size(); ++lane)
            for (size_t v = 0; v < lists[lane].size(); ++v) E.ent[(size_t)(base + (int64_t)v * 32 + (int64_t)lane)] = lists[lane][v];
    }
}

// Lists of the pipelined kernel (see PermEll) and its pre-signed W rows.
void build_perm_ell(const Basis &B, const Interaction &I, Tables &T)
{
    PermEll &P = T.pe;
    P = PermEll();
    const uint32_t ws = (uint32_t)T.wsign;
    auto repack = [ws](uint32_t e) -> uint32_t {
        return (e & 0xFFFFu) | ((((e >> 16) & 0x7FFFu) + ((e >> 31) ? ws : 0u)) << 16);
    };
    const Species &NS = B.sp[1];
    const size_t nsec = NS.sec.size();
    std::vector<std::vector<int>> into(nsec);
    for (size_t c = 0; c < T.n1.cls.size(); ++c) into[(size_t)T.n1.cls[c].s_dst].push_back((int)c);
    P.perm_off.assign(nsec, 0);
    P.cls_ent.assign(T.n1.cls.size(), 0);
    P.cls_sinfo.assign(T.n1.cls.size(), 0);
    P.sec_nn_ent.assign(nsec, 0);
    P.sec_nn_sinfo.assign(nsec, 0);
    struct CoreSlice {
        size_t base, lmax;
        int64_t nsrc;
    };
    std::vector<CoreSlice> core_slices, nn_slices;
    for (size_t s = 0; s < nsec; ++s) {
        const int64_t n = NS.sec[s].count;
        // column order: lexicographic (descending) by the per-class list lengths
        std::vector<int32_t> order((size_t)n);
        for (int64_t c = 0; c < n; ++c) order[(size_t)c] = (int32_t)c;
        auto len = [&](int cls, int32_t col) {
            const int64_t po = T.n1.cls[(size_t)cls].ptr_off;
            return T.n1.ptr[(size_t)(po + col + 1)] - T.n1.ptr[(size_t)(po + col)];
        };
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
            for (int cls : into[s]) {
                const int64_t la = len(cls, a), lb = len(cls, b);
                if (la != lb) return la > lb;
            }
            return false;
        });
        while (P.perm.size() % 4) P.perm.push_back(0);
        P.perm_off[s] = (int64_t)P.perm.size();
        P.perm.insert(P.perm.end(), order.begin(), order.end());
        const int64_t nsl = (n + 31) / 32;
        // one-body classes into this sector
        for (int cls : into[s]) {
            while (P.sinfo.size() % 4) P.sinfo.push_back(0);
            P.cls_ent[(size_t)cls] = (int64_t)P.ent.size();
            P.cls_sinfo[(size_t)cls] = (int64_t)P.sinfo.size();
            const int64_t po = T.n1.cls[(size_t)cls].ptr_off;
            for (int64_t sl = 0; sl < nsl; ++sl) {
                std::vector<std::vector<uint32_t>> lists;
                size_t lmax = 0;
                for (int64_t lane = 0; lane < 32; ++lane) {
                    lists.emplace_back();
                    const int64_t pos = sl * 32 + lane;
                    if (pos >= n) continue;
                    const int32_t col = order[(size_t)pos];
                    for (int64_t e = T.n1.ptr[(size_t)(po + col)]; e < T.n1.ptr[(size_t)(po + col + 1)]; ++e)
                        lists.back().push_back(repack(T.n1.ent[(size_t)e]));
                    lmax = std::max(lmax, lists.back().size());
                }
                std::vector<std::vector<uint32_t>> lists_core = lists;
                bank_schedule_rot(lists, (ws - 1u) << 16);   // padding: a zero W entry, source column 0
                bank_schedule_lane(lists_core, (ws - 1u) << 16);
                core_slices.push_back({P.ent.size(), lmax, B.sp[1].sec[(size_t)T.n1.cls[(size_t)cls].s_src].count});
                P.sinfo.push_back((int32_t)((int64_t)P.ent.size() - P.cls_ent[(size_t)cls]));
                P.sinfo.push_back((int32_t)lmax);
                const size_t base = P.ent.size();
                P.ent.resize(base + lmax * 32, (ws - 1u) << 16);
                P.core_ent.resize(base + lmax * 32, (ws - 1u) << 16);
                for (size_t lane = 0; lane < 32; ++lane)
                    for (size_t v = 0; v < lists[lane].size(); ++v) {
                        P.ent[base + v * 32 + lane] = lists[lane][v];
                        P.core_ent[base + v * 32 + lane] = lists_core[lane][v];
                    }
            }
        }
        // like-particle lists of the sector, same order
        while (P.nn_sinfo.size() % 4) P.nn_sinfo.push_back(0);
        P.sec_nn_ent[s] = (int64_t)P.nn_src.size();
        P.sec_nn_sinfo[s] = (int64_t)P.nn_sinfo.size();
        const int64_t *ptr = T.nn.ptr.data() + NS.sec[s].start;
        for (int64_t sl = 0; sl < nsl; ++sl) {
            std::vector<std::vector<std::pair<int32_t, double>>> lists;
            size_t lmax = 0;
            for (int64_t lane = 0; lane < 32; ++lane) {
                lists.emplace_back();
                const int64_t pos = sl * 32 + lane;
                if (pos >= n) continue;
                const int32_t col = order[(size_t)pos];
                for (int64_t e = ptr[col]; e < ptr[col + 1]; ++e)
                    lists.back().emplace_back(T.nn.src[(size_t)e], T.nn.coef[(size_t)e]);
                lmax = std::max(lmax, lists.back().size());
            }
            bank_order(lists, [](const std::pair<int32_t, double> &e, int ln) { return 2 * (int)e.first + (ln & 1); });
            P.nn_sinfo.push_back((int32_t)((int64_t)P.nn_src.size() - P.sec_nn_ent[s]));
            P.nn_sinfo.push_back((int32_t)lmax);
            const size_t base = P.nn_src.size();
            nn_slices.push_back({base, lmax, 0});
            P.nn_src.resize(base + lmax * 32, 0);
            P.nn_coef.resize(base + lmax * 32, 0.0);
            for (size_t lane = 0; lane < 32; ++lane)
                for (size_t v = 0; v < lists[lane].size(); ++v) {
                    P.nn_src[base + v * 32 + lane] = lists[lane][v].first;
                    P.nn_coef[base + v * 32 + lane] = lists[lane][v].second;
                }
        }
    }
    // whole 16-byte groups at the end: kernels copy slice info in 16-byte pieces
    while (P.sinfo.size() % 4) P.sinfo.push_back(0);
    while (P.ent.size() % 4) P.ent.push_back((ws - 1u) << 16);
    P.core_ent.resize(P.ent.size(), (ws - 1u) << 16);
    {   // refine the pn-core and like-particle orders, slices in parallel: up to 200
        // (pn) and 100 (like-particle) moves per entry, fewer for large tables (at
        // most ~1.5e8 moves for each); below 10 moves per entry the search gains
        // nothing and is skipped
        auto moves = [](size_t n, double cap) {
            const double m = std::min(cap, 1.5e8 / (double)std::max<size_t>(n, 1));
            return m < 10.0 ? 0 : (int)m;
        };
        const int ipe = moves(P.core_ent.size(), 200.0);
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t i = 0; i < (int64_t)core_slices.size(); ++i) {
            const CoreSlice &c = core_slices[(size_t)i];
            anneal_slice(P.core_ent.data() + c.base, c.lmax, (ws - 1u) << 16, c.nsrc,
                         0x5DEECE66Dull * (uint64_t)(i + 1), ipe);
        }
        const int ipn = moves(P.nn_src.size(), 100.0);
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t i = 0; i < 4 * (int64_t)nn_slices.size(); ++i) {
            const CoreSlice &c = nn_slices[(size_t)(i / 4)];
            anneal_nn_quarter(P.nn_src.data() + c.base, P.nn_coef.data() + c.base, c.lmax, (size_t)(i % 4),
                              0x2545F4914F6CDD1Dull * (uint64_t)(i + 1), ipn);
        }
    }
    // pre-signed W rows: group g, operator a, proton sign sp -> [ sp W[a][.] | -sp W[a][.] ]
    const size_t ng = I.ops.ops.size();
    T.ww_off.assign(ng, 0);
    T.ww.clear();
    for (size_t g = 0; g < ng; ++g) {
        T.ww_off[g] = (int64_t)T.ww.size();
        const int h = I.conj_group[g];
        if (h < 0) continue;
        const size_t na = I.ops.ops[g].size(), nb = I.ops.ops[(size_t)h].size();
        for (size_t a = 0; a < na; ++a)
            for (int sp = 0; sp < 2; ++sp) {
                const double sg = sp ? -1.0 : 1.0;
                const size_t base = T.ww.size();
                T.ww.resize(base + 2 * (size_t)ws, 0.0);
                for (size_t b = 0; b < nb; ++b) {
                    const double w = sg * I.Wpn[(size_t)I.wpn_off[g] + a * nb + b];
                    T.ww[base + b] = w;
                    T.ww[base + ws + b] = -w;
                }
            }
    }
}


// Units of the core-grouped pn kernel (see CoreUnit): every (Z-1)-proton core
// c that some basis SD contains, times every chunk of <= 4 states of one
// (2m, parity) key.  Sources of a unit: the SDs c + k for every state k not in
// c whose block is linked to the unit's destination block, ordered by the key
// of k so that consecutive sources share one link (one set of neutron lists).
// Order of units for a persistent kernel whose CTA b takes units b, b + G,
// b + 2G, ... (G = grid): the units come sorted by decreasing cost, and each
// round of G goes heaviest first to the CTAs with the least cost so far, so
// that the CTAs end within about one unit of each other (round-robin on the
// sorted list gives CTA 0 the heaviest unit of every round).  Every CTA keeps
// the same number of units (one more for the first n mod G), so the result is
// again a round-robin layout: position j G + b holds CTA b's j-th unit.
template <typename U>
void balance_round_robin(std::vector<U> &units, int G)
{
    const size_t n = units.size(), g = (size_t)std::max(1, G);
    if (n <= g) return;
    std::vector<std::vector<size_t>> cta(g);
    std::vector<double> load(g, 0.0);
    std::vector<size_t> by(g);
    for (size_t r0 = 0; r0 < n; r0 += g) {
        const size_t m = std::min(g, n - r0);
        for (size_t b = 0; b < g; ++b) by[b] = b;
        std::stable_sort(by.begin(), by.end(), [&](size_t a, size_t b) { return load[a] < load[b]; });
        for (size_t j = 0; j < m; ++j) {
            cta[by[j]].push_back(r0 + j);
            load[by[j]] += units[r0 + j].cost;
        }
    }
    // the CTAs with the extra unit take the first labels
    std::vector<size_t> lab(g);
    for (size_t b = 0; b < g; ++b) lab[b] = b;
    std::stable_sort(lab.begin(), lab.end(), [&](size_t a, size_t b) { return cta[a].size() > cta[b].size(); });
    std::vector<U> out;
    out.reserve(n);
    for (size_t j = 0; out.size() < n; ++j)
        for (size_t b = 0; b < g; ++b)
            if (j < cta[lab[b]].size()) out.push_back(std::move(units[cta[lab[b]][j]]));
    units.swap(out);
}

void build_core_units(const Basis &B, const Interaction &I, Tables &T)
{
    T.cunits.clear();
    T.csrc.clear();
    T.wc.clear();
    T.n_wtab = 0;
    T.gathers_pn = 0.0;
    const Species &P = B.sp[0];
    const int ns = (int)B.st.size();
    if (P.nparticles < 1 || T.links.empty()) return;
    // keys and chunks
    std::vector<std::pair<int, int>> keys;
    std::vector<int> key_of(ns);
    for (int s = 0; s < ns; ++s) {
        const std::pair<int, int> kk{B.st[s].twom, B.st[s].par};
        auto it = std::find(keys.begin(), keys.end(), kk);
        key_of[s] = (int)(it - keys.begin());
        if (it == keys.end()) keys.push_back(kk);
    }
    std::vector<std::vector<int>> chunks;
    for (size_t q = 0; q < keys.size(); ++q) {
        std::vector<int> st;
        for (int s = 0; s < ns; ++s)
            if (key_of[s] == (int)q) st.push_back(s);
        for (size_t a = 0; a < st.size(); a += 4)
            chunks.emplace_back(st.begin() + (long)a, st.begin() + (long)std::min(st.size(), a + 4));
    }
    std::vector<int> by_key(ns);
    std::iota(by_key.begin(), by_key.end(), 0);
    std::stable_sort(by_key.begin(), by_key.end(), [&](int a, int b) { return key_of[a] < key_of[b]; });
    // Weights per (chunk, subset of its states, k): column j of table row idx is
    // the pre-signed W row of op a+_i a_k (+ variant, then - variant) for the
    // j-th state i of the subset.  A unit's destination rows are the chunk
    // states its core leaves free, packed to the front, so that the kernel
    // can skip the padded rows of units with one or two of them.  Rows are
    // R = 1, 2 or 4 floats apart (one, two, three or four states), packed at
    // the front of the table: a lane's 4- or 8-byte weight load then meets
    // 32 or 16 bank positions across the rows instead of the 8 that a
    // 16-byte row stride leaves.  Tables are made on first use, ns of them
    // (one per k) per (chunk, subset).
    const size_t ws2 = 2 * (size_t)T.wsign;
    std::map<std::pair<size_t, int>, int> tab_of;   // (chunk, subset mask) -> first table
    // Table 2 (t0 + k) + f holds them with the +W and -W halves swapped when
    // f = 1 (the sign of a_k on the source row is -1), so the kernel reads
    // row (op + wsign * neutron sign) of the table its source names, with no
    // per-entry sign arithmetic.
    auto tables_for = [&](size_t q, int mask) -> int {
        auto it = tab_of.find({q, mask});
        if (it != tab_of.end()) return it->second;
        const int t0 = T.n_wtab;
        T.n_wtab += ns;
        T.wc.resize((size_t)T.n_wtab * 2 * ws2 * 4, 0.0);
        const size_t ws = ws2 / 2;
        const int cnt = __builtin_popcount((unsigned)mask);
        const size_t rs = cnt <= 1 ? 1 : cnt == 2 ? 2 : 4;   // floats per table row
        for (int k = 0; k < ns; ++k) {
            int j = 0;
            for (size_t p = 0; p < chunks[q].size(); ++p) {
                if (!(mask >> p & 1)) continue;
                const int col = j++;
                const int op = chunks[q][p] * ns + k;
                const int g = I.ops.group_of_op[(size_t)op];
                if (g < 0 || I.conj_group[(size_t)g] < 0) continue;
                const size_t row = (size_t)T.ww_off[(size_t)g] + 2 * (size_t)I.ops.local_of_op[(size_t)op] * ws2;
                double *dst = T.wc.data() + 2 * ((size_t)t0 + (size_t)k) * ws2 * 4;
                for (size_t idx = 0; idx < ws2; ++idx) {
                    dst[idx * rs + col] = T.ww[row + idx];
                    dst[ws2 * 4 + (idx ^ ws) * rs + col] = T.ww[row + idx];
                }
            }
        }
        tab_of[{q, mask}] = t0;
        return t0;
    };
    // cores
    std::vector<uint64_t> cores;
    cores.reserve(P.bits.size() * (size_t)P.nparticles);
    for (uint64_t r : P.bits)
        for (int i = 0; i < ns; ++i)
            if (r >> i & 1) cores.push_back(r & ~(1ULL << i));
    std::sort(cores.begin(), cores.end());
    cores.erase(std::unique(cores.begin(), cores.end()), cores.end());
    auto locate = [&](uint64_t m, int &blk, int &row) {
        blk = row = -1;
        auto it = P.index.find(m);
        if (it == P.index.end()) return;
        const int sec = P.sec_of_sd[(size_t)it->second];
        blk = B.block_of_psec[(size_t)sec];
        row = (int)(it->second - P.sec[(size_t)sec].start);
    };
    auto link_of = [&](int d, int s) {
        for (int64_t l = T.links_of_block[(size_t)d]; l < T.links_of_block[(size_t)d + 1]; ++l)
            if (T.links[(size_t)l].src_block == s) return (int)l;
        return -1;
    };
    struct U { double cost; CoreUnit u; std::vector<CoreSrc> src; };
    std::vector<U> units;
    for (uint64_t c : cores)
        for (size_t q = 0; q < chunks.size(); ++q) {
            U x;
            x.u.dblock = -1;
            for (int p = 0; p < 4; ++p) { x.u.drow[p] = -1; x.u.meta[p] = 0; }
            int mask = 0, nr = 0;
            for (size_t p = 0; p < chunks[q].size(); ++p) {
                const int i = chunks[q][p];
                if (c >> i & 1) continue;
                int blk, row;
                locate(c | (1ULL << i), blk, row);
                if (blk < 0) continue;
                x.u.dblock = blk;
                x.u.drow[nr] = row;
                x.u.meta[nr] = __builtin_popcountll(c & ((1ULL << i) - 1ULL)) | (sign_below(c, i) < 0 ? 256 : 0);
                mask |= 1 << p;
                ++nr;
            }
            if (x.u.dblock < 0) continue;
            const int tq = tables_for(q, mask);
            const int i0 = chunks[q][0];
            for (int k : by_key) {
                if (c >> k & 1) continue;
                const int g = I.ops.group_of_op[(size_t)(i0 * ns + k)];
                if (g < 0 || I.conj_group[(size_t)g] < 0) continue;
                int blk, row;
                locate(c | (1ULL << k), blk, row);
                if (blk < 0) continue;
                const int l = link_of(x.u.dblock, blk);
                if (l < 0) continue;
                const Block &Sb = B.blocks[(size_t)blk];
                const int ncl = T.links[(size_t)l].ncls;
                const uint32_t f = sign_below(c, k) < 0 ? 1u : 0u;
                x.src.push_back(CoreSrc{Sb.off + (int64_t)row * Sb.nN, (int32_t)Sb.nN,
                                        (2u * (uint32_t)(tq + k) + f) | (f << 31),
                                        T.pe.cls_ent[(size_t)ncl], T.pe.cls_sinfo[(size_t)ncl]});
            }
            x.u.nsrc = (int)x.src.size();
            x.u.nN = (int)B.blocks[(size_t)x.u.dblock].nN;
            x.u.perm_off = (int)T.pe.perm_off[(size_t)B.blocks[(size_t)x.u.dblock].ns];
            x.u.doff = B.blocks[(size_t)x.u.dblock].off;
            {   // cost: per source and tile of 18 column slices, the longest list (all warps
                // wait for it) weighted by the shared-memory wavefronts of a step with this
                // many rows (entry + element + weights: 10, 11, 13), plus a slot overhead
                const int nN = (int)B.blocks[(size_t)x.u.dblock].nN, nsl = (nN + 31) / 32;
                const double rf = nr <= 1 ? 1.0 : nr == 2 ? 1.1 : 1.3;
                x.cost = 0.0;
                for (const CoreSrc &cs : x.src)
                    for (int t0 = 0; t0 < nsl; t0 += 18) {
                        int lm = 0;
                        for (int sl = t0; sl < std::min(nsl, t0 + 18); ++sl)
                            lm = std::max(lm, (int)T.pe.sinfo[(size_t)(cs.sinfo_base + 2 * sl + 1)]);
                        x.cost += rf * lm + 4.0;
                    }
            }
            for (int k : by_key) {
                if (c >> k & 1) continue;
                const int g = I.ops.group_of_op[(size_t)(i0 * ns + k)];
                if (g < 0 || I.conj_group[(size_t)g] < 0) continue;
                int blk, row;
                locate(c | (1ULL << k), blk, row);
                if (blk < 0) continue;
                const int l = link_of(x.u.dblock, blk);
                if (l < 0) continue;
                const OneBodyClass &NC = T.n1.cls[(size_t)T.links[(size_t)l].ncls];
                const int nN = B.blocks[(size_t)x.u.dblock].nN;
                T.gathers_pn += (double)(T.n1.ptr[NC.ptr_off + nN] - T.n1.ptr[NC.ptr_off]);
            }
            units.push_back(std::move(x));
        }
    std::stable_sort(units.begin(), units.end(), [](const U &a, const U &b) { return a.cost > b.cost; });
    balance_round_robin(units, T.grid);
    for (U &x : units) {
        x.u.src0 = (int64_t)T.csrc.size();
        T.csrc.insert(T.csrc.end(), x.src.begin(), x.src.end());
        T.cunits.push_back(x.u);
    }
}

// Units of the core-grouped pp kernel (see PPUnit) and the per-SD proton
// single-particle diagonal it leaves out.
void build_pp_units(const Basis &B, const Interaction &I, Tables &T)
{
    T.ppunits.clear();
    T.pps_row.clear();
    T.pps_w.clear();
    const Species &P = B.sp[0];
    const int ns = (int)B.st.size();
    const int Z = P.nparticles;
    T.pdiag.assign(P.bits.size(), 0.0);
    for (size_t g = 0; g < P.bits.size(); ++g)
        for (int s = 0; s < ns; ++s)
            if (P.bits[g] >> s & 1) T.pdiag[g] += I.spe_state[(size_t)s];
    if (Z < 2) return;
    std::vector<uint64_t> cores;
    for (uint64_t r : P.bits)
        for (int a = 0; a < ns; ++a)
            if (r >> a & 1)
                for (int b = a + 1; b < ns; ++b)
                    if (r >> b & 1) cores.push_back(r & ~(1ULL << a) & ~(1ULL << b));
    std::sort(cores.begin(), cores.end());
    cores.erase(std::unique(cores.begin(), cores.end()), cores.end());
    // rank of pair (a-th, b-th occupied state), a < b, among the C(Z,2) pairs
    auto pair_rank = [Z](int a, int b) { return a * (2 * Z - a - 1) / 2 + (b - a - 1); };
    struct U { double cost; PPUnit u; std::vector<int32_t> row; std::vector<double> w; };
    std::vector<U> units;
    for (uint64_t c2 : cores)
        for (const std::vector<int> &keyp : I.pairs_by_key) {
            std::vector<int> av;   // pairs of the key outside the core
            for (int q : keyp)
                if (!(c2 >> I.pair_i[(size_t)q] & 1) && !(c2 >> I.pair_j[(size_t)q] & 1)) av.push_back(q);
            if (av.empty()) continue;
            // all rows of the unit share one proton sector
            int blk = -1, sec = -1;
            std::vector<int> rowof(av.size(), -1);
            for (size_t t = 0; t < av.size(); ++t) {
                const uint64_t m = c2 | (1ULL << I.pair_i[(size_t)av[t]]) | (1ULL << I.pair_j[(size_t)av[t]]);
                auto it = P.index.find(m);
                if (it == P.index.end()) continue;
                sec = P.sec_of_sd[(size_t)it->second];
                blk = B.block_of_psec[(size_t)sec];
                rowof[t] = (int)(it->second - P.sec[(size_t)sec].start);
            }
            if (blk < 0) continue;
            for (size_t d0 = 0; d0 < av.size(); d0 += kPPG) {
                U x;
                x.u.dblock = blk;
                bool any = false;
                for (int p = 0; p < kPPG; ++p) {
                    x.u.drow[p] = -1;
                    x.u.part[p] = 0;
                    const size_t t = d0 + (size_t)p;
                    if (t >= av.size() || rowof[t] < 0) continue;
                    const int i = I.pair_i[(size_t)av[t]], j = I.pair_j[(size_t)av[t]];
                    const uint64_t r = c2 | (1ULL << i) | (1ULL << j);
                    const int ra = __builtin_popcountll(r & ((1ULL << i) - 1ULL));
                    const int rb = __builtin_popcountll(r & ((1ULL << j) - 1ULL));
                    x.u.drow[p] = rowof[t];
                    x.u.part[p] = Z + pair_rank(ra, rb);
                    any = true;
                }
                if (!any) continue;
                for (size_t t = 0; t < av.size(); ++t) {
                    if (rowof[t] < 0) continue;
                    const int k = I.pair_i[(size_t)av[t]], l = I.pair_j[(size_t)av[t]];
                    const uint64_t X = c2 | (1ULL << k) | (1ULL << l);
                    // a_l a_k on the source, then a+_j a+_i (i < j, k < l)
                    int sg = sign_below(X, k);
                    uint64_t m1 = X & ~(1ULL << k);
                    sg *= sign_below(m1, l);
                    m1 &= ~(1ULL << l);
                    double w[kPPG] = {};
                    bool nz = false;
                    for (int p = 0; p < kPPG; ++p) {
                        if (x.u.drow[p] < 0) continue;
                        const int q = av[d0 + (size_t)p];
                        const int i = I.pair_i[(size_t)q], j = I.pair_j[(size_t)q];
                        int s2 = sign_below(m1, j);
                        const uint64_t m2 = m1 | (1ULL << j);
                        s2 *= sign_below(m2, i);
                        w[p] = sg * s2 * I.Wpp[(size_t)q * I.npairs + (size_t)av[t]];
                        nz = nz || w[p] != 0.0;
                    }
                    if (!nz) continue;
                    x.row.push_back(rowof[t]);
                    x.w.insert(x.w.end(), w, w + kPPG);
                }
                x.u.nsrc = (int)x.row.size();
                x.u.nN = (int)B.blocks[(size_t)blk].nN;
                x.u.pad = 0;
                x.u.doff = B.blocks[(size_t)blk].off;
                // cost: one slot per source and tile of 576 columns (one element per
                // thread each), plus the stores of the unit's rows
                x.cost = (double)(x.u.nsrc + 3) * (double)((B.blocks[(size_t)blk].nN + 575) / 576);
                units.push_back(std::move(x));
            }
        }
    std::stable_sort(units.begin(), units.end(), [](const U &a, const U &b) { return a.cost > b.cost; });
    balance_round_robin(units, T.grid);
    for (U &x : units) {
        x.u.src0 = (int64_t)T.pps_row.size();
        T.pps_row.insert(T.pps_row.end(), x.row.begin(), x.row.end());
        T.pps_w.insert(T.pps_w.end(), x.w.begin(), x.w.end());
        T.ppunits.push_back(x.u);
    }
}
}  // namespace

int build_tables(const Basis &B, const Interaction &I, Tables &T, std::string &err, int grid)
{
    (void)err;
    T = Tables();
    T.grid = std::max(1, grid);
    like_jumps(B, I, 0, T.pp, T.ppx, T.n_pp);
    like_jumps(B, I, 1, T.nn, T.nnx, T.n_nn);
    onebody_jumps(B, I, 0, T.p1, T.n_p1);
    onebody_jumps(B, I, 1, T.n1, T.n_n1);
    // ELL forms of the neutron-side lists for the row kernel.  One-body
    // entries are repacked as src | (op + wsign * sign) << 16, an index into a
    // shared-memory row holding +W at [0, wsign) and -W at [wsign, 2 wsign).
    size_t gmax = 1;
    for (const auto &g : I.ops.ops) gmax = std::max(gmax, g.size());
    T.wsign = 1;
    while ((size_t)T.wsign < gmax + 1) T.wsign <<= 1;
    const uint32_t ws = (uint32_t)T.wsign;
    auto repack = [ws](uint32_t e) -> uint32_t {
        return (e & 0xFFFFu) | ((((e >> 16) & 0x7FFFu) + ((e >> 31) ? ws : 0u)) << 16);
    };
    T.n1e_col.resize(T.n1.cls.size());
    T.n1e_slice.resize(T.n1.cls.size());
    for (size_t c = 0; c < T.n1.cls.size(); ++c) {
        const OneBodyClass &K = T.n1.cls[c];
        const int64_t ncols = B.sp[1].sec[K.s_dst].count;
        // padding entries point at index wsign - 1 (always a zero W entry) and source column 0
        const uint32_t pad = (ws - 1u) << 16;
        append_ell(T.n1e, ncols, T.n1.ptr.data() + K.ptr_off,
                   [&](int64_t i) { return repack(T.n1.ent[(size_t)i]); }, T.n1e_col[c], T.n1e_slice[c], pad);
    }
    T.nne_col.resize(B.sp[1].sec.size());
    T.nne_slice.resize(B.sp[1].sec.size());
    for (size_t s = 0; s < B.sp[1].sec.size(); ++s) {
        const Sector &S = B.sp[1].sec[s];
        const int64_t *ptr = T.nn.ptr.data() + S.start;
        // the same layout for (source column, coefficient) lists
        Ell &E = T.nne;
        int64_t col_off = (int64_t)E.col.size(), slice_base = (int64_t)E.soff.size();
        std::vector<int32_t> order((size_t)S.count);
        for (int64_t c = 0; c < S.count; ++c) order[(size_t)c] = (int32_t)c;
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return (ptr[a + 1] - ptr[a]) > (ptr[b + 1] - ptr[b]); });
        for (int64_t i = 0; i < S.count; ++i) {
            E.col.push_back(order[(size_t)i]);
            E.len.push_back((int32_t)(ptr[order[(size_t)i] + 1] - ptr[order[(size_t)i]]));
        }
        for (int64_t s0 = 0; s0 < S.count; s0 += 32) {
            const int64_t base = (int64_t)E.src.size();
            E.soff.push_back(base);
            const int64_t need = base + (int64_t)E.len[(size_t)(col_off + s0)] * 32;
            E.src.resize((size_t)need, 0);
            E.coef.resize((size_t)need, 0.0);
            std::vector<std::vector<std::pair<int32_t, double>>> lists;
            for (int64_t lane = 0; lane < 32 && s0 + lane < S.count; ++lane) {
                const int32_t c = order[(size_t)(s0 + lane)];
                lists.emplace_back();
                for (int64_t v = 0; v < ptr[c + 1] - ptr[c]; ++v)
                    lists.back().emplace_back(T.nn.src[(size_t)(ptr[c] + v)], T.nn.coef[(size_t)(ptr[c] + v)]);
            }
            bank_order(lists, [](const std::pair<int32_t, double> &e, int ln) { return 2 * (int)e.first + (ln & 1); });
            for (size_t lane = 0; lane < lists.size(); ++lane)
                for (size_t v = 0; v < lists[lane].size(); ++v) {
                    E.src[(size_t)(base + (int64_t)v * 32 + (int64_t)lane)] = lists[lane][v].first;
                    E.coef[(size_t)(base + (int64_t)v * 32 + (int64_t)lane)] = lists[lane][v].second;
                }
        }
        T.nne_col[s] = col_off;
        T.nne_slice[s] = slice_base;
    }
    build_perm_ell(B, I, T);
    // pn links: destination block <- source block
    const int nb = (int)B.blocks.size();
    const int nps = (int)B.sp[0].sec.size(), nns = (int)B.sp[1].sec.size();
    std::vector<int> pcls((size_t)nps * nps, -1), ncls((size_t)nns * nns, -1);
    for (size_t c = 0; c < T.p1.cls.size(); ++c) pcls[(size_t)T.p1.cls[c].s_src * nps + T.p1.cls[c].s_dst] = (int)c;
    for (size_t c = 0; c < T.n1.cls.size(); ++c) ncls[(size_t)T.n1.cls[c].s_src * nns + T.n1.cls[c].s_dst] = (int)c;
    T.links_of_block.assign((size_t)nb + 1, 0);
    T.llinks_of_block.assign((size_t)nb + 1, 0);
    double ops = 0.0;
    for (int d = 0; d < nb; ++d) {
        const Block &D = B.blocks[d];
        for (int s = 0; s < nb; ++s) {
            const Block &S = B.blocks[s];
            int pc = pcls[(size_t)S.ps * nps + D.ps], nc = ncls[(size_t)S.ns * nns + D.ns];
            if (pc < 0 || nc < 0) continue;
            int g = T.p1.cls[pc].group;
            int h = I.conj_group[g];
            if (h < 0 || T.n1.cls[nc].group != h) continue;
            PnLink L;
            L.dst_block = d;
            L.src_block = s;
            L.pcls = pc;
            L.ncls = nc;
            L.w_off = I.wpn_off[g];
            L.nb = (int)I.ops.ops[h].size();
            T.links.push_back(L);
            const OneBodyClass &P = T.p1.cls[pc], &N = T.n1.cls[nc];
            double np_ = (double)(T.p1.ptr[P.ptr_off + D.nP] - T.p1.ptr[P.ptr_off]);
            double nn_ = (double)(T.n1.ptr[N.ptr_off + D.nN] - T.n1.ptr[N.ptr_off]);
            ops += np_ * nn_;
            T.ops_pn += np_ * nn_;
        }
        T.links_of_block[(size_t)d + 1] = (int64_t)T.links.size();
        // like-particle work of this block
        const Sector &PS = B.sp[0].sec[D.ps], &NS = B.sp[1].sec[D.ns];
        double opp = (double)(T.pp.ptr[PS.start + PS.count] - T.pp.ptr[PS.start]) * (double)D.nN;
        double onn = (double)(T.nn.ptr[NS.start + NS.count] - T.nn.ptr[NS.start]) * (double)D.nP;
        // moves from other sectors (W-truncated bases): pp from block (s_src, D.ns),
        // nn from block (D.ps, s_src), where those blocks are in the basis
        for (const LikeCrossClass &c : T.ppx.cls) {
            if (c.s_dst != D.ps) continue;
            const int sb = B.block_of(c.s_src, D.ns);
            if (sb < 0) continue;
            T.llinks.push_back(LikeLink{d, sb, 0, c.ptr_off});
            opp += (double)(T.ppx.ptr[(size_t)(c.ptr_off + D.nP)] - T.ppx.ptr[(size_t)c.ptr_off]) * (double)D.nN;
        }
        for (const LikeCrossClass &c : T.nnx.cls) {
            if (c.s_dst != D.ns) continue;
            const int sb = B.block_of(D.ps, c.s_src);
            if (sb < 0) continue;
            T.llinks.push_back(LikeLink{d, sb, 1, c.ptr_off});
            onn += (double)(T.nnx.ptr[(size_t)(c.ptr_off + D.nN)] - T.nnx.ptr[(size_t)c.ptr_off]) * (double)D.nP;
        }
        T.llinks_of_block[(size_t)d + 1] = (int64_t)T.llinks.size();
        ops += opp + onn;
        T.ops_pp += opp;
        T.ops_nn += onn;
    }
    T.ops_per_vector = ops;
    if (B.trunc) return BS_OK;   // the core-grouped tables assume one neutron sector per proton sector
    {   // the pp-core kernel packs a destination row and its partial rank into one int
        const int Z = B.sp[0].nparticles;
        int64_t maxsec = 0;
        for (const Sector &S : B.sp[0].sec) maxsec = std::max<int64_t>(maxsec, (int64_t)S.count);
        if (Z + Z * (Z - 1) / 2 > 255 || maxsec >= (int64_t)1 << 23) return BS_OK;
    }
    build_core_units(B, I, T);
    build_pp_units(B, I, T);
    return BS_OK;
}

}  // namespace bs
