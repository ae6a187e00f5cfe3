/*
 * bs_oracle.c -- plain FP64 reference for the M-scheme shell-model Hamiltonian.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg load this code; the library never does, and the two share
 * no source.  It is written for obviousness, not speed: every matrix element
 * is produced by applying creation/annihilation operators to occupation
 * bitstrings, as the paper defines them.
 *
 * What it follows (BIGSTICK manual, arXiv:1801.08432):
 *   - occupation bitstrings and the fermion sign of a^dagger / a
 *     (Sec. "Representation of the basis");
 *   - M-scheme basis of proton x neutron Slater determinants with
 *     M_p + M_n = M, sectors labelled by (M, parity), every proton SD of a
 *     sector combined with every neutron SD of the conjugate sector, proton
 *     index outer and neutron index inner (Sec. "Factorization of the basis",
 *     Table al27, and the basis-file description);
 *   - the Hamiltonian of Eq. (hamdef): H = sum_a e_a n_a +
 *     1/4 sum_abcd zeta_ab zeta_cd sum_J V_J(ab,cd) sum_M A^dag_JM(ab) A_JM(cd),
 *     with A^dag_JM(ab) = (a^dag x b^dag)_JM coupled with Edmonds' Clebsch-
 *     Gordan coefficients (Eq. angmomcoupling, Eq. Adagger);
 *   - the TBME symmetries with isospin (Sec. "Symmetries of matrix elements");
 *   - the proton-neutron matrix element built from isospin-coupled ones,
 *     Eq. (xpndef): V^pn_J = sqrt((1+d_ab)(1+d_cd))/2 [V_J,T=0 + V_J,T=1].
 *
 * Single-particle state order (the paper leaves it open): orbit after orbit in
 * input order, m ascending inside an orbit.  Slater determinants inside a
 * sector are sorted by bitmask; sectors by 2M ascending, parity + before -.
 *
 * Decoupled operator (derived in the comments of decouple() from Eq. hamdef):
 *   V_pp = sum_{i<j, k<l} W_pp(ij,kl) a+_i a+_j a_l a_k        (T = 1 elements)
 *   V_pn = sum_{i,k in p; j,l in n} W_pn(ij,kl) (a+_i a_k)_p (a+_j a_l)_n
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EINVAL (-1)
#define OR_ENOMEM (-4)
#define MAXJ2 64   /* largest 2J of a pair handled */

/* ------------------------------------------------------------------ */
/* Clebsch-Gordan coefficient <j1 m1 j2 m2 | J M>, all arguments doubled.   */
/* Racah's closed formula (Edmonds 1957, Eq. 3.6.11), in double.          */
/* ------------------------------------------------------------------ */
static double fact(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

double orc_cg(int tj1, int tm1, int tj2, int tm2, int tJ, int tM)
{
    if (tm1 + tm2 != tM) return 0.0;
    if (abs(tm1) > tj1 || abs(tm2) > tj2 || abs(tM) > tJ) return 0.0;
    if (tJ < abs(tj1 - tj2) || tJ > tj1 + tj2) return 0.0;
    if (((tj1 + tm1) & 1) || ((tj2 + tm2) & 1) || ((tJ + tM) & 1)) return 0.0;
    if (((tj1 + tj2 + tJ) & 1)) return 0.0;
    /* integer combinations */
    int a = (tj1 + tj2 - tJ) / 2, b = (tj1 - tj2 + tJ) / 2, c = (-tj1 + tj2 + tJ) / 2;
    int d = (tj1 + tj2 + tJ) / 2 + 1;
    double pre = sqrt((tJ + 1) * fact(a) * fact(b) * fact(c) / fact(d));
    pre *= sqrt(fact((tj1 + tm1) / 2) * fact((tj1 - tm1) / 2) * fact((tj2 + tm2) / 2) *
                fact((tj2 - tm2) / 2) * fact((tJ + tM) / 2) * fact((tJ - tM) / 2));
    double sum = 0.0;
    for (int k = 0; k <= d; ++k) {
        int e1 = a - k;                       /* j1+j2-J-k  */
        int e2 = (tj1 - tm1) / 2 - k;         /* j1-m1-k    */
        int e3 = (tj2 + tm2) / 2 - k;         /* j2+m2-k    */
        int e4 = (tJ - tj2 + tm1) / 2 + k;    /* J-j2+m1+k  */
        int e5 = (tJ - tj1 - tm2) / 2 + k;    /* J-j1-m2+k  */
        if (e1 < 0 || e2 < 0 || e3 < 0 || e4 < 0 || e5 < 0) continue;
        double t = 1.0 / (fact(k) * fact(e1) * fact(e2) * fact(e3) * fact(e4) * fact(e5));
        sum += (k & 1) ? -t : t;
    }
    return pre * sum;
}

/* ------------------------------------------------------------------ */
/* bit operations: the sign rule of the paper.  a_s or a^dag_s acting on */
/* |b> = prod_{t in b, ascending} a^dag_t |0> picks up (-1)^(number of   */
/* occupied states t < s).                                              */
/* ------------------------------------------------------------------ */
static int popc(uint64_t x) { return __builtin_popcountll(x); }

static int annihilate(uint64_t *m, int s)
{
    uint64_t bit = 1ULL << s;
    if (!(*m & bit)) return 0;
    int sg = (popc(*m & (bit - 1)) & 1) ? -1 : 1;
    *m &= ~bit;
    return sg;
}

static int create(uint64_t *m, int s)
{
    uint64_t bit = 1ULL << s;
    if (*m & bit) return 0;
    int sg = (popc(*m & (bit - 1)) & 1) ? -1 : 1;
    *m |= bit;
    return sg;
}

/* ------------------------------------------------------------------ */
/* context                                                              */
/* ------------------------------------------------------------------ */
typedef struct {
    int twoM, par;     /* key */
    int64_t start;     /* first SD of the sector in the species list */
    int64_t count;
} or_sector;

typedef struct {
    int nsd, nsec;
    uint64_t *bits;    /* [nsd] sorted by sector then bitmask */
    or_sector *sec;    /* [nsec] */
    int *sec_of_key;   /* [(twoM+keyoff)*2+par] -> sector or -1 */
    int keyoff, nkey;
} or_species;

typedef struct orc {
    int norb, ns;
    int *orb_l, *orb_twoj;
    int st_orb[64], st_twom[64], st_par[64];
    int Z, N, twoM, parity;
    or_species sp[2];                 /* 0 = protons, 1 = neutrons */
    int nblk;
    int *blk_psec, *blk_nsec;         /* [nblk] */
    int64_t *blk_off;                 /* [nblk+1] */
    int *blk_of_psec;                 /* [psec] -> block or -1 */
    int64_t dim;
    /* interaction */
    int have_int;
    double spe_state[64];
    double *V;     /* V[T][J][a][b][c][d] full table, orbit-ordered labels as given by symmetries */
    double *Wpp;   /* [ns^4] W_pp(i,j,k,l), used for i<j, k<l */
    double *Wpn;   /* [ns^4] W_pn(i,j,k,l), i,k proton; j,l neutron */
    /* explicit matrix (CSC of H; equal to CSR because H is symmetric) */
    int64_t *colptr, *rowidx;
    double *val;
    int64_t nnz;
    /* the stored rows of a row sample (same format, rows listed in sub_rows) */
    int64_t *sub_rows, *sub_ptr, *sub_idx;
    double *sub_val;
    int64_t nsub, sub_nnz;
} orc;

static int nsd_choose(int n, int k)
{
    if (k < 0 || k > n) return 0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return (int)(r + 0.5);
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Enumerate every N-particle bitstring over ns states and group by (2M, parity). */
static int build_species(orc *o, int nparticles, or_species *S)
{
    int ns = o->ns;
    int total = nsd_choose(ns, nparticles);
    if (total <= 0) return OR_EINVAL;
    uint64_t *all = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)total);
    int *tm = (int *)malloc(sizeof(int) * (size_t)total);
    int *pr = (int *)malloc(sizeof(int) * (size_t)total);
    if (!all || !tm || !pr) return OR_ENOMEM;
    /* plain enumeration of all subsets of size nparticles, in increasing bitmask order */
    int cnt = 0;
    uint64_t lim = (ns == 64) ? ~0ULL : ((1ULL << ns) - 1);
    if (nparticles == 0) {
        all[cnt++] = 0;
    } else {
        uint64_t v = (1ULL << nparticles) - 1;
        while (1) {
            all[cnt++] = v;
            /* next larger integer with the same popcount */
            uint64_t t = v | (v - 1);
            uint64_t w = (t + 1) | (((~t & -~t) - 1) >> (__builtin_ctzll(v) + 1));
            if (w > lim || w <= v) break;
            v = w;
        }
    }
    if (cnt != total) { free(all); free(tm); free(pr); return OR_EINVAL; }
    int maxM = 0;
    for (int s = 0; s < ns; ++s) maxM += abs(o->st_twom[s]);
    S->keyoff = maxM;
    S->nkey = 2 * (2 * maxM + 1);
    S->sec_of_key = (int *)malloc(sizeof(int) * (size_t)S->nkey);
    int64_t *kcount = (int64_t *)calloc((size_t)S->nkey, sizeof(int64_t));
    for (int i = 0; i < cnt; ++i) {
        int M = 0, p = 0;
        for (int s = 0; s < ns; ++s)
            if (all[i] >> s & 1) { M += o->st_twom[s]; p ^= o->st_par[s]; }
        tm[i] = M; pr[i] = p;
        kcount[(M + maxM) * 2 + p]++;
    }
    /* sectors in key order: 2M ascending, parity + (0) before - (1) */
    S->nsec = 0;
    for (int k = 0; k < S->nkey; ++k) S->sec_of_key[k] = -1;
    for (int k = 0; k < S->nkey; ++k)
        if (kcount[k] > 0) S->sec_of_key[k] = S->nsec++;
    S->sec = (or_sector *)malloc(sizeof(or_sector) * (size_t)S->nsec);
    int64_t run = 0;
    for (int k = 0; k < S->nkey; ++k) {
        int s = S->sec_of_key[k];
        if (s < 0) continue;
        S->sec[s].twoM = k / 2 - maxM;
        S->sec[s].par = k % 2;
        S->sec[s].start = run;
        S->sec[s].count = kcount[k];
        run += kcount[k];
    }
    S->nsd = cnt;
    S->bits = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)cnt);
    int64_t *fill = (int64_t *)calloc((size_t)S->nsec, sizeof(int64_t));
    for (int i = 0; i < cnt; ++i) {
        int s = S->sec_of_key[(tm[i] + maxM) * 2 + pr[i]];
        S->bits[S->sec[s].start + fill[s]++] = all[i];
    }
    for (int s = 0; s < S->nsec; ++s)
        qsort(S->bits + S->sec[s].start, (size_t)S->sec[s].count, sizeof(uint64_t), cmp_u64);
    free(all); free(tm); free(pr); free(kcount); free(fill);
    return 0;
}

static int sector_of(const or_species *S, int twoM, int par)
{
    int k = (twoM + S->keyoff) * 2 + par;
    if (k < 0 || k >= S->nkey) return -1;
    return S->sec_of_key[k];
}

/* local index of bitstring m inside sector s, or -1 */
static int64_t local_index(const or_species *S, int s, uint64_t m)
{
    int64_t lo = 0, hi = S->sec[s].count - 1;
    const uint64_t *b = S->bits + S->sec[s].start;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (b[mid] == m) return mid;
        if (b[mid] < m) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

static void mask_quantum(const orc *o, uint64_t m, int *twoM, int *par)
{
    int M = 0, p = 0;
    for (int s = 0; s < o->ns; ++s)
        if (m >> s & 1) { M += o->st_twom[s]; p ^= o->st_par[s]; }
    *twoM = M; *par = p;
}

/* global basis index of (proton bits, neutron bits), or -1 if not in the basis */
static int64_t basis_index(const orc *o, uint64_t P, uint64_t Nb)
{
    int Mp, pp, Mn, pn;
    mask_quantum(o, P, &Mp, &pp);
    mask_quantum(o, Nb, &Mn, &pn);
    if (Mp + Mn != o->twoM || (pp ^ pn) != o->parity) return -1;
    int sp = sector_of(&o->sp[0], Mp, pp);
    int sn = sector_of(&o->sp[1], Mn, pn);
    if (sp < 0 || sn < 0) return -1;
    int b = o->blk_of_psec[sp];
    if (b < 0 || o->blk_nsec[b] != sn) return -1;
    int64_t ip = local_index(&o->sp[0], sp, P);
    int64_t jn = local_index(&o->sp[1], sn, Nb);
    if (ip < 0 || jn < 0) return -1;
    return o->blk_off[b] + ip * o->sp[1].sec[sn].count + jn;
}

/* parity is 0 for +, 1 for - */
int orc_create(orc **out, const int *orb_l, const int *orb_twoj, int norb,
               int Z, int N, int twoM, int parity)
{
    *out = NULL;
    if (norb <= 0 || Z < 0 || N < 0) return OR_EINVAL;
    orc *o = (orc *)calloc(1, sizeof(orc));
    o->norb = norb;
    o->orb_l = (int *)malloc(sizeof(int) * (size_t)norb);
    o->orb_twoj = (int *)malloc(sizeof(int) * (size_t)norb);
    int ns = 0;
    for (int a = 0; a < norb; ++a) {
        o->orb_l[a] = orb_l[a];
        o->orb_twoj[a] = orb_twoj[a];
        if (orb_twoj[a] <= 0 || !(orb_twoj[a] & 1)) return OR_EINVAL;
        for (int tm = -orb_twoj[a]; tm <= orb_twoj[a]; tm += 2) {
            if (ns >= 64) return OR_EINVAL;
            o->st_orb[ns] = a;
            o->st_twom[ns] = tm;
            o->st_par[ns] = orb_l[a] & 1;
            ns++;
        }
    }
    o->ns = ns;
    if (Z > ns || N > ns) return OR_EINVAL;
    o->Z = Z; o->N = N; o->twoM = twoM; o->parity = parity;
    int rc;
    if ((rc = build_species(o, Z, &o->sp[0])) != 0) return rc;
    if ((rc = build_species(o, N, &o->sp[1])) != 0) return rc;
    /* blocks: each proton sector with its conjugate neutron sector */
    int np = o->sp[0].nsec;
    o->blk_psec = (int *)malloc(sizeof(int) * (size_t)np);
    o->blk_nsec = (int *)malloc(sizeof(int) * (size_t)np);
    o->blk_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(np + 1));
    o->blk_of_psec = (int *)malloc(sizeof(int) * (size_t)np);
    o->nblk = 0;
    int64_t off = 0;
    for (int s = 0; s < np; ++s) {
        o->blk_of_psec[s] = -1;
        int sn = sector_of(&o->sp[1], twoM - o->sp[0].sec[s].twoM, parity ^ o->sp[0].sec[s].par);
        if (sn < 0) continue;
        int b = o->nblk++;
        o->blk_psec[b] = s;
        o->blk_nsec[b] = sn;
        o->blk_off[b] = off;
        o->blk_of_psec[s] = b;
        off += o->sp[0].sec[s].count * o->sp[1].sec[sn].count;
    }
    o->blk_off[o->nblk] = off;
    o->dim = off;
    *out = o;
    return 0;
}

int64_t orc_dim(const orc *o) { return o->dim; }
int orc_ns(const orc *o) { return o->ns; }

void orc_sizes(const orc *o, int *out /* [5] */)
{
    out[0] = o->sp[0].nsd; out[1] = o->sp[1].nsd;
    out[2] = o->sp[0].nsec; out[3] = o->sp[1].nsec;
    out[4] = o->nblk;
}

/* Copies the basis out.  sec arrays hold (2M, parity, start, count) per sector,
 * blocks hold (proton sector, neutron sector, offset) per block. */
void orc_export_basis(const orc *o, uint64_t *pbits, uint64_t *nbits,
                      int64_t *psec, int64_t *nsec, int64_t *blocks)
{
    memcpy(pbits, o->sp[0].bits, sizeof(uint64_t) * (size_t)o->sp[0].nsd);
    memcpy(nbits, o->sp[1].bits, sizeof(uint64_t) * (size_t)o->sp[1].nsd);
    for (int s = 0; s < o->sp[0].nsec; ++s) {
        psec[4 * s] = o->sp[0].sec[s].twoM; psec[4 * s + 1] = o->sp[0].sec[s].par;
        psec[4 * s + 2] = o->sp[0].sec[s].start; psec[4 * s + 3] = o->sp[0].sec[s].count;
    }
    for (int s = 0; s < o->sp[1].nsec; ++s) {
        nsec[4 * s] = o->sp[1].sec[s].twoM; nsec[4 * s + 1] = o->sp[1].sec[s].par;
        nsec[4 * s + 2] = o->sp[1].sec[s].start; nsec[4 * s + 3] = o->sp[1].sec[s].count;
    }
    for (int b = 0; b < o->nblk; ++b) {
        blocks[3 * b] = o->blk_psec[b]; blocks[3 * b + 1] = o->blk_nsec[b];
        blocks[3 * b + 2] = o->blk_off[b];
    }
}

/* ------------------------------------------------------------------ */
/* interaction                                                          */
/* ------------------------------------------------------------------ */
#define VIDX(o, T, J, a, b, c, d) \
    (((((((size_t)(T) * (MAXJ2 / 2 + 1) + (J)) * (o)->norb + (a)) * (o)->norb + (b)) * (o)->norb + (c)) * (o)->norb + (d)))

/* V_JT(ab,cd) for any orbit order, from the stored table.  The table holds
 * every order already (filled by orc_set_interaction with the symmetry
 * phases), so this is a plain lookup. */
static double vlook(const orc *o, int T, int J, int a, int b, int c, int d)
{
    if (J < 0 || J > MAXJ2 / 2) return 0.0;
    return o->V[VIDX(o, T, J, a, b, c, d)];
}

/*
 * Reads the isospin-coupled elements (a b c d J T V), labels 1-based, any
 * order, and fills V_JT for every label order with the phases of the paper:
 *   V_JT(ab,cd) = (-1)^(j_a+j_b+J+T) V_JT(ba,cd)      (from -(-1)^(x+1) = (-1)^x)
 *   V_JT(ab,cd) = (-1)^(j_c+j_d+J+T) V_JT(ab,dc)
 *   V_JT(ab,cd) = V_JT(cd,ab)                          (real elements)
 * Rejects labels out of range, a J outside a pair's triangle, a same-orbit
 * pair with J+T even (Pauli), parity change, and an element given twice.
 * Then decouples (see decouple()).
 */
static void decouple(orc *o);

int orc_set_interaction(orc *o, const double *spe, const int *lab, const double *v, int ntb)
{
    int no = o->norb;
    size_t nv = (size_t)2 * (MAXJ2 / 2 + 1) * no * no * no * no;
    free(o->V);
    o->V = (double *)calloc(nv, sizeof(double));
    char *seen = (char *)calloc(nv, 1);
    if (!o->V || !seen) return OR_ENOMEM;
    for (int s = 0; s < o->ns; ++s) o->spe_state[s] = spe[o->st_orb[s]];
    for (int t = 0; t < ntb; ++t) {
        int a = lab[6 * t] - 1, b = lab[6 * t + 1] - 1, c = lab[6 * t + 2] - 1, d = lab[6 * t + 3] - 1;
        int J = lab[6 * t + 4], T = lab[6 * t + 5];
        if (a < 0 || b < 0 || c < 0 || d < 0 || a >= no || b >= no || c >= no || d >= no) { free(seen); return OR_EINVAL; }
        if (T != 0 && T != 1) { free(seen); return OR_EINVAL; }
        if (J < 0 || 2 * J > MAXJ2) { free(seen); return OR_EINVAL; }
        int ja = o->orb_twoj[a], jb = o->orb_twoj[b], jc = o->orb_twoj[c], jd = o->orb_twoj[d];
        if (2 * J < abs(ja - jb) || 2 * J > ja + jb || 2 * J < abs(jc - jd) || 2 * J > jc + jd) { free(seen); return OR_EINVAL; }
        if ((a == b || c == d) && ((J + T) % 2 == 0)) { free(seen); return OR_EINVAL; }
        if (((o->orb_l[a] + o->orb_l[b] + o->orb_l[c] + o->orb_l[d]) & 1) != 0) { free(seen); return OR_EINVAL; }
        /* an element given twice (in any label order) is an error */
        int ca = a < b ? a : b, cb = a < b ? b : a, cc = c < d ? c : d, cd = c < d ? d : c;
        if (ca > cc || (ca == cc && cb > cd)) { int t0 = ca, t1 = cb; ca = cc; cb = cd; cc = t0; cd = t1; }
        size_t key = VIDX(o, T, J, ca, cb, cc, cd);
        if (seen[key]) { free(seen); return OR_EINVAL; }
        seen[key] = 1;
        /* store every label order: (ab) or (ba), (cd) or (dc), and the two pair orders */
        int pab = (((ja + jb) / 2 + J + T) & 1) ? -1 : 1;   /* (-1)^(ja+jb+J+T) */
        int pcd = (((jc + jd) / 2 + J + T) & 1) ? -1 : 1;
        int A[2] = {a, b}, B[2] = {c, d};
        for (int x = 0; x < 2; ++x)
            for (int y = 0; y < 2; ++y) {
                double val = v[t] * (x ? pab : 1) * (y ? pcd : 1);
                int aa = A[x], bb = A[1 - x], cc2 = B[y], dd = B[1 - y];
                o->V[VIDX(o, T, J, aa, bb, cc2, dd)] = val;
                o->V[VIDX(o, T, J, cc2, dd, aa, bb)] = val;
            }
    }
    free(seen);
    decouple(o);
    o->have_int = 1;
    return 0;
}

/*
 * Decoupling to the M-scheme (Eq. hamdef with Eq. Adagger and the pair
 * annihilator A_JM = (A^dag_JM)^dag).
 *
 * Like particles.  The sum over all a,b,c,d with 1/4 zeta_ab zeta_cd equals a
 * sum over a<=b, c<=d of V_J(ab,cd) (A^dag/zeta_ab)(A/zeta_cd), because
 * swapping a,b changes V and A^dag by the same phase.  The overlap of the
 * two-particle determinant |ij> = a+_i a+_j|0> (i<j, so orb(i) <= orb(j)) with
 * the normalized pair state is zeta_ab <j_a m_i j_b m_j|J M> (the factor 2 of
 * a same-orbit pair cancels the 1/sqrt2).  Hence
 *   W_pp(ij,kl) = zeta_ab zeta_cd sum_J <ja mi jb mj|JM><jc mk jd ml|JM> V_J,T=1(ab,cd),
 * a=orb(i), b=orb(j), c=orb(k), d=orb(l), M = mi+mj = mk+ml.
 *
 * Proton-neutron.  The pn pair state |a_p b_n; JM> = sum <ja ma jb mb|JM>
 * a+_p b+_n|0> is normalized without zeta, and its element is Eq. (xpndef):
 *   W_pn(ij,kl) = sum_J <ja mi jb mj|JM><jc mk jd ml|JM> * 1/2 zeta_ab zeta_cd (V_J0 + V_J1)(ab,cd)
 * with i,k proton states and j,l neutron states (a,c proton orbits, b,d
 * neutron orbits, in that order).  The operator a+_i b+_j b_l a_k equals
 * (a+_i a_k)(b+_j b_l).
 */
static void decouple(orc *o)
{
    int ns = o->ns;
    size_t n4 = (size_t)ns * ns * ns * ns;
    free(o->Wpp); free(o->Wpn);
    o->Wpp = (double *)calloc(n4, sizeof(double));
    o->Wpn = (double *)calloc(n4, sizeof(double));
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j)
            for (int k = 0; k < ns; ++k)
                for (int l = 0; l < ns; ++l) {
                    int tM = o->st_twom[i] + o->st_twom[j];
                    if (tM != o->st_twom[k] + o->st_twom[l]) continue;
                    int a = o->st_orb[i], b = o->st_orb[j], c = o->st_orb[k], d = o->st_orb[l];
                    int ja = o->orb_twoj[a], jb = o->orb_twoj[b], jc = o->orb_twoj[c], jd = o->orb_twoj[d];
                    double zab = (a == b) ? sqrt(2.0) : 1.0;
                    double zcd = (c == d) ? sqrt(2.0) : 1.0;
                    double wpp = 0.0, wpn = 0.0;
                    for (int tJ = 0; tJ <= MAXJ2; tJ += 2) {
                        double c1 = orc_cg(ja, o->st_twom[i], jb, o->st_twom[j], tJ, tM);
                        double c2 = orc_cg(jc, o->st_twom[k], jd, o->st_twom[l], tJ, tM);
                        if (c1 == 0.0 || c2 == 0.0) continue;
                        int J = tJ / 2;
                        wpp += zab * zcd * c1 * c2 * vlook(o, 1, J, a, b, c, d);
                        wpn += c1 * c2 * 0.5 * zab * zcd *
                               (vlook(o, 0, J, a, b, c, d) + vlook(o, 1, J, a, b, c, d));
                    }
                    size_t idx = (((size_t)i * ns + j) * ns + k) * ns + l;
                    if (i < j && k < l) o->Wpp[idx] = wpp;
                    o->Wpn[idx] = wpn;
                }
}

void orc_get_w(const orc *o, double *wpp, double *wpn)
{
    size_t n4 = (size_t)o->ns * o->ns * o->ns * o->ns;
    memcpy(wpp, o->Wpp, n4 * sizeof(double));
    memcpy(wpn, o->Wpn, n4 * sizeof(double));
}

/* ------------------------------------------------------------------ */
/* H applied to one basis state: the column H|alpha>                    */
/* ------------------------------------------------------------------ */
typedef struct { int64_t idx; double v; } entry;

typedef struct { entry *e; int64_t n, cap; } elist;

static void push(elist *L, int64_t idx, double v)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 1024;
        L->e = (entry *)realloc(L->e, sizeof(entry) * (size_t)L->cap);
    }
    L->e[L->n].idx = idx;
    L->e[L->n].v = v;
    L->n++;
}

static int cmp_entry(const void *a, const void *b)
{
    int64_t x = ((const entry *)a)->idx, y = ((const entry *)b)->idx;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Emits every (target, value) of H|P,N>; duplicates are summed by the caller. */
static void apply_H_state(const orc *o, uint64_t P, uint64_t Nb, elist *L)
{
    int ns = o->ns;
    /* one-body: sum_s e_s n_s, both species (diagonal) */
    double d = 0.0;
    for (int s = 0; s < ns; ++s) {
        if (P >> s & 1) d += o->spe_state[s];
        if (Nb >> s & 1) d += o->spe_state[s];
    }
    push(L, basis_index(o, P, Nb), d);
    /* like-particle two-body, protons (species 0) then neutrons (species 1):
     * a+_i a+_j a_l a_k with i<j, k<l, applied right to left */
    for (int sp = 0; sp < 2; ++sp) {
        uint64_t X = sp == 0 ? P : Nb;
        for (int k = 0; k < ns; ++k)
            for (int l = k + 1; l < ns; ++l) {
                if (!(X >> k & 1) || !(X >> l & 1)) continue;
                for (int i = 0; i < ns; ++i)
                    for (int j = i + 1; j < ns; ++j) {
                        double w = o->Wpp[(((size_t)i * ns + j) * ns + k) * ns + l];
                        if (w == 0.0) continue;
                        uint64_t m = X;
                        int sg = annihilate(&m, k);
                        if (!sg) continue;
                        int s2 = annihilate(&m, l);
                        if (!s2) continue;
                        sg *= s2;
                        s2 = create(&m, j);
                        if (!s2) continue;
                        sg *= s2;
                        s2 = create(&m, i);
                        if (!s2) continue;
                        sg *= s2;
                        int64_t t = sp == 0 ? basis_index(o, m, Nb) : basis_index(o, P, m);
                        if (t >= 0) push(L, t, sg * w);
                    }
            }
    }
    /* proton-neutron: (a+_i a_k)_p (a+_j a_l)_n */
    for (int k = 0; k < ns; ++k)
        for (int i = 0; i < ns; ++i) {
            uint64_t mp = P;
            int sp = annihilate(&mp, k);
            if (!sp) continue;
            int s2 = create(&mp, i);
            if (!s2) continue;
            sp *= s2;
            for (int l = 0; l < ns; ++l)
                for (int j = 0; j < ns; ++j) {
                    double w = o->Wpn[(((size_t)i * ns + j) * ns + k) * ns + l];
                    if (w == 0.0) continue;
                    uint64_t mn = Nb;
                    int sn = annihilate(&mn, l);
                    if (!sn) continue;
                    int s3 = create(&mn, j);
                    if (!s3) continue;
                    sn *= s3;
                    int64_t t = basis_index(o, mp, mn);
                    if (t >= 0) push(L, t, sp * sn * w);
                }
        }
}

static void state_of_index(const orc *o, int64_t alpha, uint64_t *P, uint64_t *Nb)
{
    int b = 0;
    while (b + 1 < o->nblk && o->blk_off[b + 1] <= alpha) ++b;
    int sp = o->blk_psec[b], sn = o->blk_nsec[b];
    int64_t nn = o->sp[1].sec[sn].count;
    int64_t r = alpha - o->blk_off[b];
    *P = o->sp[0].bits[o->sp[0].sec[sp].start + r / nn];
    *Nb = o->sp[1].bits[o->sp[1].sec[sn].start + r % nn];
}

/* sorts and merges duplicates of a column list; returns the merged length */
static int64_t merge_list(elist *L)
{
    qsort(L->e, (size_t)L->n, sizeof(entry), cmp_entry);
    int64_t w = 0;
    for (int64_t r = 0; r < L->n; ++r) {
        if (w > 0 && L->e[w - 1].idx == L->e[r].idx) L->e[w - 1].v += L->e[r].v;
        else L->e[w++] = L->e[r];
    }
    L->n = w;
    return w;
}

/* Builds the columns of H at the basis indices cols[0..n) (CSC; a column is
 * also the row of the same index, H being symmetric): *ptr[n+1], *idx[nnz],
 * *val[nnz], allocated here.  Returns nnz or a negative error. */
static int64_t build_columns(const orc *o, const int64_t *cols, int64_t n, int64_t **ptr_out, int64_t **idx_out,
                             double **val_out)
{
    int64_t *ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    entry **cl = (entry **)calloc((size_t)(n ? n : 1), sizeof(entry *));
    int64_t *clen = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
    if (!ptr || !cl || !clen) { free(ptr); free(cl); free(clen); return OR_ENOMEM; }
#pragma omp parallel
    {
        elist L = {0, 0, 0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < n; ++r) {
            uint64_t P, Nb;
            state_of_index(o, cols ? cols[r] : r, &P, &Nb);
            L.n = 0;
            apply_H_state(o, P, Nb, &L);
            merge_list(&L);
            cl[r] = (entry *)malloc(sizeof(entry) * (size_t)(L.n ? L.n : 1));
            memcpy(cl[r], L.e, sizeof(entry) * (size_t)L.n);
            clen[r] = L.n;
        }
        free(L.e);
    }
    for (int64_t r = 0; r < n; ++r) ptr[r + 1] = ptr[r] + clen[r];
    const int64_t nnz = ptr[n];
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz ? nnz : 1));
    double *val = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    for (int64_t r = 0; r < n; ++r) {
        for (int64_t t = 0; t < clen[r]; ++t) {
            idx[ptr[r] + t] = cl[r][t].idx;
            val[ptr[r] + t] = cl[r][t].v;
        }
        free(cl[r]);
    }
    free(cl); free(clen);
    *ptr_out = ptr; *idx_out = idx; *val_out = val;
    return nnz;
}

/* Builds every column of H (CSC).  Returns nnz or a negative error. */
int64_t orc_build_matrix(orc *o)
{
    if (!o->have_int) return OR_EINVAL;
    free(o->colptr); free(o->rowidx); free(o->val);
    o->colptr = NULL; o->rowidx = NULL; o->val = NULL;
    const int64_t nnz = build_columns(o, NULL, o->dim, &o->colptr, &o->rowidx, &o->val);
    if (nnz < 0) return nnz;
    o->nnz = nnz;
    return nnz;
}

/* Stores the rows rows[0..n) of H (a sample of the explicit matrix, built as
 * orc_build_matrix builds every row).  Returns their element count or a
 * negative error. */
int64_t orc_build_rows(orc *o, const int64_t *rows, int64_t n)
{
    if (!o->have_int) return OR_EINVAL;
    free(o->sub_rows); free(o->sub_ptr); free(o->sub_idx); free(o->sub_val);
    o->sub_rows = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    if (!o->sub_rows) return OR_ENOMEM;
    memcpy(o->sub_rows, rows, sizeof(int64_t) * (size_t)n);
    o->sub_ptr = NULL; o->sub_idx = NULL; o->sub_val = NULL;
    const int64_t nnz = build_columns(o, rows, n, &o->sub_ptr, &o->sub_idx, &o->sub_val);
    if (nnz < 0) return nnz;
    o->nsub = n;
    o->sub_nnz = nnz;
    return nnz;
}

void orc_export_matrix(const orc *o, int64_t *colptr, int64_t *rowidx, double *val)
{
    memcpy(colptr, o->colptr, sizeof(int64_t) * (size_t)(o->dim + 1));
    memcpy(rowidx, o->rowidx, sizeof(int64_t) * (size_t)o->nnz);
    memcpy(val, o->val, sizeof(double) * (size_t)o->nnz);
}

/* y[r] = sum_t val[t] x[idx[t]] over the stored row r (ptr[r] <= t <
 * ptr[r+1]), for n rows, x [dim][k], y [n][k]. */
static void csr_apply(const int64_t *ptr, const int64_t *idx, const double *val, int64_t n, const double *x,
                      double *y, int k)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < n; ++r) {
        for (int c = 0; c < k; ++c) {
            double s = 0.0;
            for (int64_t t = ptr[r]; t < ptr[r + 1]; ++t)
                s += val[t] * x[idx[t] * k + c];
            y[r * k + c] = s;
        }
    }
}

/* y = H x with the stored matrix, x and y [dim][k].  Uses H = H^T, so the
 * stored columns are rows. */
void orc_spmv(const orc *o, const double *x, double *y, int k)
{
    csr_apply(o->colptr, o->rowidx, o->val, o->dim, x, y, k);
}

/* The sampled rows of y = H x (orc_build_rows): y [nsub][k], x [dim][k]. */
void orc_spmv_rows(const orc *o, const double *x, double *y, int k)
{
    csr_apply(o->sub_ptr, o->sub_idx, o->sub_val, o->nsub, x, y, k);
}

/* Selected rows of y = H x computed on the fly, without the matrix:
 * <alpha|H|x> = sum_beta x_beta <beta|H|alpha> (H Hermitian, real). */
void orc_apply_rows_ex(const orc *o, const int64_t *rows, int64_t nrows, const double *x, int k, double *yrows,
                       int absval)
{
#pragma omp parallel
    {
        elist L = {0, 0, 0};
#pragma omp for schedule(dynamic, 4)
        for (int64_t r = 0; r < nrows; ++r) {
            uint64_t P, Nb;
            state_of_index(o, rows[r], &P, &Nb);
            L.n = 0;
            apply_H_state(o, P, Nb, &L);
            merge_list(&L);
            for (int c = 0; c < k; ++c) {
                double s = 0.0;
                for (int64_t t = 0; t < L.n; ++t)
                    s += absval ? fabs(L.e[t].v) * fabs(x[L.e[t].idx * k + c]) : L.e[t].v * x[L.e[t].idx * k + c];
                yrows[r * k + c] = s;
            }
        }
        free(L.e);
    }
}

/* Selected rows of y = H x (absval = 0) or of |H| |x| (absval = 1, for
 * rounding-error bounds), on the fly. */
void orc_apply_rows(const orc *o, const int64_t *rows, int64_t nrows, const double *x, int k, double *yrows)
{
    orc_apply_rows_ex(o, rows, nrows, x, k, yrows, 0);
}

/* out = J+ psi, psi in basis `from` (2M), out in basis `to` (2M+2), both
 * species: J+ = sum_s sqrt(j(j+1) - m(m+1)) a+_{m+1} a_m within each orbit. */
int orc_jplus(const orc *from, const orc *to, const double *psi, double *out)
{
    if (to->twoM != from->twoM + 2 || to->ns != from->ns) return OR_EINVAL;
    memset(out, 0, sizeof(double) * (size_t)to->dim);
    int ns = from->ns;
    for (int64_t a = 0; a < from->dim; ++a) {
        uint64_t P, Nb;
        state_of_index(from, a, &P, &Nb);
        for (int sp = 0; sp < 2; ++sp) {
            for (int s = 0; s + 1 < ns; ++s) {
                if (from->st_orb[s + 1] != from->st_orb[s]) continue;
                double tj = from->orb_twoj[from->st_orb[s]], tm = from->st_twom[s];
                double c = 0.5 * sqrt((tj - tm) * (tj + tm + 2.0));   /* sqrt(j(j+1)-m(m+1)) */
                uint64_t m = sp == 0 ? P : Nb;
                int sg = annihilate(&m, s);
                if (!sg) continue;
                int s2 = create(&m, s + 1);
                if (!s2) continue;
                int64_t t = sp == 0 ? basis_index(to, m, Nb) : basis_index(to, P, m);
                if (t >= 0) out[t] += sg * s2 * c * psi[a];
            }
        }
    }
    return 0;
}

void orc_destroy(orc *o)
{
    if (!o) return;
    for (int s = 0; s < 2; ++s) {
        free(o->sp[s].bits); free(o->sp[s].sec); free(o->sp[s].sec_of_key);
    }
    free(o->orb_l); free(o->orb_twoj);
    free(o->blk_psec); free(o->blk_nsec); free(o->blk_off); free(o->blk_of_psec);
    free(o->V); free(o->Wpp); free(o->Wpn);
    free(o->colptr); free(o->rowidx); free(o->val);
    free(o->sub_rows); free(o->sub_ptr); free(o->sub_idx); free(o->sub_val);
    free(o);
}

/* Applies a string of operators to a bitstring, rightmost first.  ops[t] > 0
 * means a^dag_{ops[t]-1}, ops[t] < 0 means a_{-ops[t]-1}.  Returns the sign
 * (+1/-1) and the result in *out, or 0 if the state vanishes.  Exposed so the
 * sign rule can be checked against the paper's worked examples. */
int orc_apply_string(uint64_t mask, const int *ops, int nops, uint64_t *out)
{
    int sg = 1;
    for (int t = nops - 1; t >= 0; --t) {
        int s = ops[t] > 0 ? ops[t] - 1 : -ops[t] - 1;
        int r = ops[t] > 0 ? create(&mask, s) : annihilate(&mask, s);
        if (!r) return 0;
        sg *= r;
    }
    *out = mask;
    return sg;
}
