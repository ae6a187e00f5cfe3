// Isospin-coupled SPEs and TBMEs -> M-scheme (decoupled) matrix elements, FP64.
//
// Eq. (hamdef): H = sum_a e_a n_a + 1/4 sum_abcd zeta_ab zeta_cd sum_J V_J(ab,cd)
//   sum_M A+_JM(ab) A_JM(cd), with A+_JM(ab) = (a+ x b+)_JM (Eq. angmomcoupling,
//   Eq. Adagger, Edmonds' Clebsch-Gordan coefficients) and A_JM its adjoint.
// Like particles: restricting to i<j, k<l (states ordered orbit-major), the
//   overlap <ij|A+_JM(ab)|0>/zeta_ab equals zeta_ab <ja mi jb mj|JM>, so
//   W(ij,kl) = sum_J P_J(ij) P_J(kl) V_J,T=1(ab,cd) with P_J(ij) = zeta_ab CG.
// Proton-neutron: Eq. (xpndef), V^pn_J = sqrt((1+d_ab)(1+d_cd))/2 (V_J0 + V_J1),
//   between the normalized states sum CG a+_p b+_n |0>, so
//   W_pn(ij,kl) = sum_J Q_J(ij) Q_J(kl) V^pn_J(ab,cd), Q_J(ij) = CG, with i,k
//   proton states and j,l neutron states; the operator is (a+_i a_k)_p (a+_j a_l)_n.
// Input elements may come in any label order; the symmetries of Sec.
// "Symmetries of matrix elements" map them to a <= b, c <= d, (ab) <= (cd):
//   V_JT(ab,cd) = (-1)^(ja+jb+J+T) V_JT(ba,cd), same for (cd), V(ab,cd) = V(cd,ab).
#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>

#include "bs_internal.h"

namespace bs {

namespace {

// log n! table
struct LogFact {
    std::vector<double> t;
    LogFact() : t(200, 0.0)
    {
        for (size_t n = 1; n < t.size(); ++n) t[n] = t[n - 1] + std::log((double)n);
    }
    double operator()(int n) const { return t[(size_t)n]; }
};

const LogFact &lf()
{
    static LogFact f;
    return f;
}

// Wigner 3j symbol (j1 j2 j3; m1 m2 m3), doubled arguments, Racah's sum in
// log form; the CG coefficient follows from
// <j1 m1 j2 m2|J M> = (-1)^(j1-j2+M) sqrt(2J+1) (j1 j2 J; m1 m2 -M).
double threej(int a, int b, int c, int x, int y, int z)
{
    if (x + y + z != 0) return 0.0;
    if (std::abs(x) > a || std::abs(y) > b || std::abs(z) > c) return 0.0;
    if (c < std::abs(a - b) || c > a + b || ((a + b + c) & 1)) return 0.0;
    if (((a + x) & 1) || ((b + y) & 1) || ((c + z) & 1)) return 0.0;
    const LogFact &L = lf();
    int t1 = (a + b - c) / 2, t2 = (a - b + c) / 2, t3 = (-a + b + c) / 2, t4 = (a + b + c) / 2 + 1;
    double tri = 0.5 * (L(t1) + L(t2) + L(t3) - L(t4));
    double ms = 0.5 * (L((a + x) / 2) + L((a - x) / 2) + L((b + y) / 2) + L((b - y) / 2) + L((c + z) / 2) + L((c - z) / 2));
    int kmin = std::max(0, std::max((b - c - x) / 2, (a - c + y) / 2));
    int kmax = std::min(t1, std::min((a - x) / 2, (b + y) / 2));
    double s = 0.0;
    for (int k = kmin; k <= kmax; ++k) {
        double lg = L(k) + L(t1 - k) + L((a - x) / 2 - k) + L((b + y) / 2 - k) + L((c - b + x) / 2 + k) + L((c - a - y) / 2 + k);
        double term = std::exp(tri + ms - lg);
        s += (k & 1) ? -term : term;
    }
    int ph = (a - b - z) / 2;
    return (ph & 1) ? -s : s;
}

double clebsch(int j1, int m1, int j2, int m2, int J, int M)
{
    if (m1 + m2 != M) return 0.0;
    double t = threej(j1, j2, J, m1, m2, -M);
    int ph = (j1 - j2 + M) / 2;
    return ((ph & 1) ? -1.0 : 1.0) * std::sqrt((double)J + 1.0) * t;
}

using Key = std::tuple<int, int, int, int, int, int>;   // T, J, a, b, c, d (canonical)

struct Tbme {
    const Basis *B;
    std::map<Key, double> v;

    int phase(int a, int b, int J, int T) const
    {
        int x = (B->orb_twoj[a] + B->orb_twoj[b]) / 2 + J + T;
        return (x & 1) ? -1 : 1;
    }
    // V_JT(ab,cd) in any label order
    double get(int T, int J, int a, int b, int c, int d) const
    {
        double ph = 1.0;
        if (a > b) { ph *= phase(a, b, J, T); std::swap(a, b); }
        if (c > d) { ph *= phase(c, d, J, T); std::swap(c, d); }
        if (std::make_pair(a, b) > std::make_pair(c, d)) { std::swap(a, c); std::swap(b, d); }
        auto it = v.find(Key(T, J, a, b, c, d));
        return it == v.end() ? 0.0 : ph * it->second;
    }
};

}  // namespace

int OpGroups::find(int dtwom, int dpar) const
{
    for (size_t g = 0; g < g_dtwom.size(); ++g)
        if (g_dtwom[g] == dtwom && g_dpar[g] == dpar) return (int)g;
    return -1;
}

int build_interaction(const Basis &B, const double *spe, int n_spe, const bs_tbme *tbme, int n_tbme,
                      Interaction &I, std::string &err)
{
    I = Interaction();
    const int no = (int)B.orb_twoj.size();
    const int ns = (int)B.st.size();
    if (n_spe != no || !spe) { err = "load_interaction: need one SPE per orbit"; return BS_EINVAL; }
    if (n_tbme < 0 || (n_tbme > 0 && !tbme)) { err = "load_interaction: bad TBME list"; return BS_EINVAL; }
    Tbme V;
    V.B = &B;
    for (int t = 0; t < n_tbme; ++t) {
        int a = tbme[t].a - 1, b = tbme[t].b - 1, c = tbme[t].c - 1, d = tbme[t].d - 1;
        int J = tbme[t].J, T = tbme[t].T;
        char buf[160];
        std::snprintf(buf, sizeof buf, "load_interaction: element %d (%d %d %d %d J=%d T=%d) ", t,
                      tbme[t].a, tbme[t].b, tbme[t].c, tbme[t].d, J, T);
        if (a < 0 || b < 0 || c < 0 || d < 0 || a >= no || b >= no || c >= no || d >= no) { err = std::string(buf) + "has an orbit label out of range"; return BS_EINVAL; }
        if (T != 0 && T != 1) { err = std::string(buf) + "has T not 0 or 1"; return BS_EINVAL; }
        int ja = B.orb_twoj[a], jb = B.orb_twoj[b], jc = B.orb_twoj[c], jd = B.orb_twoj[d];
        if (J < 0 || 2 * J < std::abs(ja - jb) || 2 * J > ja + jb || 2 * J < std::abs(jc - jd) || 2 * J > jc + jd) { err = std::string(buf) + "violates the triangle rule"; return BS_EINVAL; }
        if ((a == b || c == d) && ((J + T) % 2) == 0) { err = std::string(buf) + "is Pauli-forbidden (same orbits, J+T even)"; return BS_EINVAL; }
        if (((B.orb_l[a] + B.orb_l[b] + B.orb_l[c] + B.orb_l[d]) & 1) != 0) { err = std::string(buf) + "changes parity"; return BS_EINVAL; }
        double val = tbme[t].v;
        if (a > b) { val *= V.phase(a, b, J, T); std::swap(a, b); }
        if (c > d) { val *= V.phase(c, d, J, T); std::swap(c, d); }
        if (std::make_pair(a, b) > std::make_pair(c, d)) { std::swap(a, c); std::swap(b, d); }
        if (!V.v.emplace(Key(T, J, a, b, c, d), val).second) { err = std::string(buf) + "is given twice"; return BS_EINVAL; }
    }
    const std::vector<SpState> &st = B.st;
    auto tj = [&](int s) { return B.orb_twoj[st[s].orb]; };
    I.spe_state.resize(ns);
    for (int s = 0; s < ns; ++s) I.spe_state[s] = spe[st[s].orb];
    int Jmax2 = 0;
    for (int a = 0; a < no; ++a) Jmax2 = std::max(Jmax2, 2 * B.orb_twoj[a]);

    // ---- like particles: pairs i<j grouped by (2M, parity)
    I.pair_id.assign((size_t)ns * ns, -1);
    std::map<std::pair<int, int>, int> keyid;
    for (int i = 0; i < ns; ++i)
        for (int j = i + 1; j < ns; ++j) {
            int id = I.npairs++;
            I.pair_i.push_back(i);
            I.pair_j.push_back(j);
            I.pair_id[(size_t)i * ns + j] = id;
            std::pair<int, int> key(st[i].twom + st[j].twom, st[i].par ^ st[j].par);
            auto it = keyid.find(key);
            int kid;
            if (it == keyid.end()) { kid = (int)I.pairs_by_key.size(); keyid[key] = kid; I.pairs_by_key.emplace_back(); }
            else kid = it->second;
            I.pairs_by_key[kid].push_back(id);
            I.key_of_pair.push_back(kid);
        }
    // pair amplitudes P_J(ij) = zeta_ab <ja mi jb mj | J M>
    int nJ = Jmax2 / 2 + 1;
    std::vector<double> P((size_t)I.npairs * nJ, 0.0);
    for (int p = 0; p < I.npairs; ++p) {
        int i = I.pair_i[p], j = I.pair_j[p];
        double z = st[i].orb == st[j].orb ? std::sqrt(2.0) : 1.0;
        for (int J = 0; J < nJ; ++J)
            P[(size_t)p * nJ + J] = z * clebsch(tj(i), st[i].twom, tj(j), st[j].twom, 2 * J, st[i].twom + st[j].twom);
    }
    I.Wpp.assign((size_t)I.npairs * I.npairs, 0.0);
    for (const std::vector<int> &grp : I.pairs_by_key)
        for (int p : grp)
            for (int q : grp) {
                int a = st[I.pair_i[p]].orb, b = st[I.pair_j[p]].orb;
                int c = st[I.pair_i[q]].orb, d = st[I.pair_j[q]].orb;
                double w = 0.0;
                for (int J = 0; J < nJ; ++J) {
                    double pp = P[(size_t)p * nJ + J], qq = P[(size_t)q * nJ + J];
                    if (pp == 0.0 || qq == 0.0) continue;
                    w += pp * qq * V.get(1, J, a, b, c, d);
                }
                I.Wpp[(size_t)p * I.npairs + q] = w;
            }

    // ---- one-body operator groups a+_i a_k by (2m_i - 2m_k, par_i ^ par_k)
    OpGroups &G = I.ops;
    G.group_of_op.assign((size_t)ns * ns, -1);
    G.local_of_op.assign((size_t)ns * ns, -1);
    std::map<std::pair<int, int>, std::vector<int>> byk;
    for (int i = 0; i < ns; ++i)
        for (int k = 0; k < ns; ++k)
            byk[{st[i].twom - st[k].twom, st[i].par ^ st[k].par}].push_back(i * ns + k);
    for (auto &kv : byk) {
        int g = (int)G.ops.size();
        G.g_dtwom.push_back(kv.first.first);
        G.g_dpar.push_back(kv.first.second);
        G.ops.push_back(kv.second);
        for (size_t t = 0; t < kv.second.size(); ++t) {
            G.group_of_op[kv.second[t]] = g;
            G.local_of_op[kv.second[t]] = (int)t;
        }
    }
    int ng = (int)G.ops.size();
    I.conj_group.assign(ng, -1);
    I.wpn_off.assign(ng + 1, 0);
    for (int g = 0; g < ng; ++g) {
        I.conj_group[g] = G.find(-G.g_dtwom[g], G.g_dpar[g]);
        int h = I.conj_group[g];
        I.wpn_off[g + 1] = I.wpn_off[g] + (h < 0 ? 0 : (int64_t)G.ops[g].size() * (int64_t)G.ops[h].size());
    }
    // pn amplitudes Q_J(ij) = <ja mi jb mj | J M>, i proton, j neutron
    std::vector<double> Q((size_t)ns * ns * nJ, 0.0);
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j)
            for (int J = 0; J < nJ; ++J)
                Q[((size_t)i * ns + j) * nJ + J] = clebsch(tj(i), st[i].twom, tj(j), st[j].twom, 2 * J, st[i].twom + st[j].twom);
    I.Wpn.assign((size_t)I.wpn_off[ng], 0.0);
    for (int g = 0; g < ng; ++g) {
        int h = I.conj_group[g];
        if (h < 0) continue;
        int nb = (int)G.ops[h].size();
        for (size_t ia = 0; ia < G.ops[g].size(); ++ia) {
            int i = G.ops[g][ia] / ns, k = G.ops[g][ia] % ns;
            for (int ib = 0; ib < nb; ++ib) {
                int j = G.ops[h][ib] / ns, l = G.ops[h][ib] % ns;
                int a = st[i].orb, b = st[j].orb, c = st[k].orb, d = st[l].orb;
                double zz = 0.5 * (a == b ? std::sqrt(2.0) : 1.0) * (c == d ? std::sqrt(2.0) : 1.0);
                double w = 0.0;
                for (int J = 0; J < nJ; ++J) {
                    double q1 = Q[((size_t)i * ns + j) * nJ + J], q2 = Q[((size_t)k * ns + l) * nJ + J];
                    if (q1 == 0.0 || q2 == 0.0) continue;
                    w += q1 * q2 * zz * (V.get(0, J, a, b, c, d) + V.get(1, J, a, b, c, d));
                }
                I.Wpn[(size_t)I.wpn_off[g] + ia * nb + ib] = w;
            }
        }
    }
    return BS_OK;
}

}  // namespace bs
