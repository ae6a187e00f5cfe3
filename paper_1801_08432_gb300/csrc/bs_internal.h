// Internal data structures of libbsgpu: host-side basis, interaction and jump
// tables, and the device mirror the kernels read.
#pragma once

#include <cuda_runtime.h>
#include <vector_types.h>

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "bigstick_gpu.h"

namespace bs {

// ---------------------------------------------------------------- basis
struct SpState {
    int orb;     // orbit index (0-based, input order)
    int twom;    // 2 m
    int par;     // 0 for +, 1 for -
    int w;       // truncation weight of the orbit (used only by a W-truncated basis)
};

struct Sector {
    int twoM, par;
    int64_t start;   // first SD of the sector in the species list
    int64_t count;
    int W = 0;       // summed weight of its SDs (0 in an untruncated basis)
};

struct Species {
    int nparticles = 0;
    std::vector<uint64_t> bits;            // sorted by sector, then bitmask
    std::vector<Sector> sec;
    std::vector<int> sec_of_sd;            // sector of every SD
    std::unordered_map<uint64_t, int64_t> index;  // bitmask -> global SD index
    int find_sector(int twoM, int par, int W = 0) const;
};

struct Block {
    int ps, ns;        // proton and neutron sector
    int64_t off;       // first basis index
    int64_t nP, nN;    // sector sizes
};

struct Basis {
    std::vector<int> orb_l, orb_twoj;
    std::vector<SpState> st;
    int Z = 0, N = 0, twoM = 0, par = 0;
    Species sp[2];
    std::vector<Block> blocks;
    std::vector<int> block_of_psec;        // first block of a proton sector, -1 when it has no conjugate
    int64_t dim = 0;
    // W truncation (Sec. "Truncation of the many-body space"): sectors are keyed
    // by (2M, parity, W) and a proton sector pairs with every conjugate neutron
    // sector whose W keeps W_p + W_n <= w_max, so it may head several blocks
    bool trunc = false;
    int w_max = 0;                         // W_min + the allowed excitation
    int block_of(int ps, int ns) const;    // block of a (proton, neutron) sector pair, or -1
    std::vector<int> blk_of_pair;          // [n_psec * n_nsec]
};

// ---------------------------------------------------------------- interaction
// A one-body operator a+_i a_k of one species, grouped by the change it makes
// to (2M, parity): key = (2m_i - 2m_k, par_i ^ par_k).  Inside a group the
// operators get compact indices 0..n-1.
struct OpGroups {
    std::vector<int> group_of_op;     // [ns*ns] op (i*ns+k) -> group
    std::vector<int> local_of_op;     // [ns*ns] op -> index inside its group
    std::vector<int> g_dtwom, g_dpar; // per group
    std::vector<std::vector<int>> ops; // per group: list of ops
    int find(int dtwom, int dpar) const;
};

struct Interaction {
    // like-particle two-body elements W(ij,kl), i<j, k<l, keyed by pair ids
    int npairs = 0;
    std::vector<int> pair_i, pair_j;            // pair id -> states
    std::vector<int> pair_id;                   // [ns*ns] (i<j) -> id
    std::vector<std::vector<int>> pairs_by_key; // pairs grouped by (2M, parity)
    std::vector<int> key_of_pair;
    std::vector<double> Wpp;                    // [npairs*npairs]
    std::vector<double> spe_state;              // [ns]
    OpGroups ops;                               // proton and neutron one-body groups (same space)
    // W_pn for group pair (g for protons, conj(g) for neutrons): dense [n_g x n_conj]
    std::vector<int> conj_group;                // g -> neutron group with opposite 2m change
    std::vector<int64_t> wpn_off;               // per group offset into Wpn
    std::vector<double> Wpn;
};

// ---------------------------------------------------------------- jumps
// Destination-ordered sparse lists ("both directions stored, sorted by destination").
struct LikeJumps {          // pp or nn, same sector, diagonal included (SPE folded in)
    std::vector<int64_t> ptr;     // [nsd+1] by destination SD (global index)
    std::vector<int32_t> src;     // source SD, local index inside the sector
    std::vector<double> coef;
};

// Like-particle jumps that change the sector (only in a W-truncated basis,
// where a two-body move can change an SD's W but not its 2M and parity):
// per (source sector, destination sector) a destination CSR over the SDs of
// s_dst with source SDs as local indices in s_src.
struct LikeCrossClass {
    int s_src, s_dst;
    int64_t ptr_off;        // into LikeCross::ptr, |S_dst|+1 entries
};

struct LikeCross {
    std::vector<LikeCrossClass> cls;
    std::vector<int64_t> ptr;
    std::vector<int32_t> src;
    std::vector<double> coef;
};

// A like-particle link: destination block <- source block of the same
// neutron sector (pp, species 0) or the same proton sector (nn, species 1)
// through one LikeCross class.
struct LikeLink {
    int dst_block, src_block, species;
    int64_t ptr_off;
};

struct OneBodyClass {       // one-body jumps from sector s_src into sector s_dst
    int s_src, s_dst;
    int group;              // operator group (change of 2m, parity)
    int64_t ptr_off;        // into OneBodyJumps::ptr, |S_dst|+1 entries
};

struct OneBodyJumps {
    std::vector<OneBodyClass> cls;
    std::vector<int64_t> ptr;
    std::vector<uint32_t> ent;    // packed: src local (bits 0..15) | op local (bits 16..30) | sign (bit 31)
};

// One pn "opbundle": destination block <- source block through proton class
// pc and neutron class nc.
struct PnLink {
    int dst_block, src_block;
    int pcls, ncls;
    int64_t w_off;      // offset of the W_pn group matrix
    int nb;             // row length of that matrix (neutron ops of the conjugate group)
};

// Per-column lists laid out for the warps of the row kernel: the columns of a
// sector are sorted by list length (longest first) and cut into slices of 32;
// entry v of the lane-th column of a slice sits at soff[slice] + 32 v + lane,
// so a warp reads 128 contiguous bytes per step and runs about as many steps
// as its longest list, which sorting keeps close to the others.
struct Ell {
    std::vector<int32_t> col, len;     // per sorted position: column id, list length
    std::vector<int64_t> soff;         // per slice: first entry
    std::vector<uint32_t> ent;         // one-body lists: packed (src | op << 16 | sign << 31)
    std::vector<int32_t> src;          // like-particle lists: source column
    std::vector<double> coef;          //                      coefficient
};

// The same neutron-side lists for the pipelined kernel: the columns of each
// neutron sector in ONE fixed order shared by every list kind (sorted
// lexicographically by the column's list lengths over the incoming classes,
// so neighbouring columns have similar lengths), cut into 32-column slices;
// per class and slice: offset of the slice's first entry and its longest list.
struct PermEll {
    std::vector<int32_t> perm;          // per sector: position -> column (sector offset in perm_off)
    std::vector<int64_t> perm_off;      // per neutron sector
    std::vector<uint32_t> ent;          // one-body entries, packed like Tables::n1e, plus a rotation bit (31)
    std::vector<uint32_t> core_ent;     // the same lists at the same positions for the pn-core kernel:
                                        // src | W row << 16, in a step order scheduled for the fixed
                                        // per-lane chunk order of that kernel (no rotation bit)
    std::vector<int32_t> sinfo;         // per class and slice: (entry offset from class base, lmax)
    std::vector<int64_t> cls_ent, cls_sinfo;   // per one-body class: base of its entries / slice info
    std::vector<int32_t> nn_src;        // like-particle lists in the same order
    std::vector<double> nn_coef;
    std::vector<int32_t> nn_sinfo;      // per sector and slice: (entry offset, lmax)
    std::vector<int64_t> sec_nn_ent, sec_nn_sinfo;
};

// pn term by (Z-1)-proton cores.  Every proton one-body jump a+_i a_k from
// SD s into SD r passes through exactly one core c = a_k s (a Z-1 proton SD),
// with r = a+_i c: a+_i a_k restricted to Z protons is sum_c a+_i|c><c|a_k.
// A unit is one core c and a chunk of at most 4 states i of one (2m, parity)
// key; its destination rows r_i = c + i share one proton sector, hence one
// neutron sector and the same neutron jump lists, so one staged source row
// c + k and one 16-byte load of the four weights W(i_p j, k l) feed four
// destination rows.  Each destination row receives one such partial per core
// (Z of them); they are summed in a fixed order afterwards.
struct CoreUnit {
    int dblock;            // destination block
    int nsrc;              // source slots of the unit
    int64_t src0;          // first slot in Tables::csrc
    int drow[4];           // destination proton row (local in the sector), -1 if absent
    int meta[4];           // rank t of i in r (0..Z-1) | 256 if the sign of a+_i on c is -1
    int nN;                // the destination block's columns, its column order (PermEll offset)
    int perm_off;          //   and first basis index: copied here so that the kernel reads one
    int64_t doff;          //   record per unit
};

struct CoreSrc {           // 32 bytes: staged with its source row
    int64_t x_elem;        // first basis index of the source row c + k (block offset + row * nN)
    int32_t nN;            // its length (the source block's neutron sector)
    uint32_t wtab;         // W table 2 (chunk, k) + f, f = 1 if the sign of a_k on c + k is -1 (that
                           // table has the +W and -W halves swapped); bit 31 repeats f
    int64_t ent_base;      // neutron lists of the link dst block <- src block: first entry of the
    int64_t sinfo_base;    // class in PermEll::ent and its per-slice (offset, longest list)
};

// pp term by (Z-2)-proton cores: a two-body term a+_i a+_j a_l a_k taking
// SD s to r belongs to exactly one core c2 = s - {k,l} = r - {i,j}.  A unit is
// one core, one (2M, parity) key of pairs and up to eight destination pairs
// (i,j); its destination rows r_p = c2 + {i_p,j_p} and its sources
// c2 + {k,l} all lie in one proton sector, so a staged source row serves eight
// destination rows with eight CTA-uniform weights (the fermion sign folded in).
// Row r gets one partial per pair of its states (C(Z,2) of them); the proton
// single-particle energies are left to a per-row diagonal.
constexpr int kPPG = 8;    // destination pairs per pp unit
struct PPUnit {
    int dblock;
    int nsrc;
    int64_t src0;          // first source in Tables::pps_row / pps_w
    int drow[kPPG];        // destination proton row, -1 if absent
    int part[kPPG];        // partial vector of the destination row (Z + pair rank)
    int nN;                // the destination block's columns and first basis index (one record per unit)
    int pad;
    int64_t doff;
};

struct Tables {
    int grid = 152;                      // CTAs of the persistent core-grouped kernels (units are balanced for it)
    LikeJumps pp, nn;                    // moves inside a sector (diagonal and SPE included)
    LikeCross ppx, nnx;                  // moves between sectors (W-truncated bases only)
    std::vector<LikeLink> llinks;        // sorted by dst block
    std::vector<int64_t> llinks_of_block;   // [nblocks+1]
    PermEll pe;                          // pipelined kernel's neutron lists
    std::vector<double> ww;              // per group g, op a, proton sign: a row of 2*wsign W values
    std::vector<int64_t> ww_off;         // per group
    Ell n1e;                             // neutron one-body classes, ELL form, entries packed as
                                         // src | (op + wsign * sign) << 16 (index into a +W/-W row)
    int wsign = 0;                       // power of two > largest operator group: offset of -W
    Ell nne;                             // neutron like-particle lists, ELL form
    std::vector<int64_t> n1e_col, n1e_slice;   // per neutron one-body class: offsets into n1e
    std::vector<int64_t> nne_col, nne_slice;   // per neutron sector: offsets into nne
    OneBodyJumps p1, n1;
    std::vector<PnLink> links;           // sorted by dst block
    std::vector<int64_t> links_of_block; // [nblocks+1]
    int64_t n_pp = 0, n_nn = 0, n_p1 = 0, n_n1 = 0;
    double ops_per_vector = 0.0;         // multiply-adds of one H*x (structural)
    double ops_pn = 0.0, ops_pp = 0.0, ops_nn = 0.0;   // its split by term
    double gathers_pn = 0.0;   // source elements the pn-core kernel gathers per vector (one per neutron
                               // one-body jump of each source record; each feeds the unit's rows)
    // core-grouped pn term
    std::vector<CoreUnit> cunits;        // sorted by work, largest first
    std::vector<CoreSrc> csrc;
    std::vector<double> wc;              // per (chunk, k): [2 wsign][R] weights W(i_p ., k .), +W then -W, R = 1, 2, 4
                                         // by the unit's rows, at the front of a [2 wsign][4] slot
    int n_wtab = 0;
    // core-grouped pp term
    std::vector<PPUnit> ppunits;         // sorted by work, largest first
    std::vector<int32_t> pps_row;        // per source: proton row c2 + {k,l}
    std::vector<double> pps_w;           // per source: kPPG signed weights
    std::vector<double> pdiag;           // per proton SD: sum of its single-particle energies
};

// ---------------------------------------------------------------- device mirror
struct DevBlock {
    int64_t off;
    int nP, nN;
    int p_start, n_start;   // global SD index of the first SD of each sector
    int link_begin, link_end;
    int llink_begin, llink_end;   // like-particle links from other blocks (W-truncated bases)
    int64_t nne_col, nne_slice;   // ELL of the neutron like-particle lists of this block's neutron sector
    int64_t perm_off;             // pipelined kernel: column order of the neutron sector
    int64_t pe_nn_ent, pe_nn_sinfo;
};

struct DevLink {
    int src_block;
    int nb;
    int64_t p_ptr_off;      // proton class CSR (|S_p dst|+1)
    int64_t n_ptr_off;      // neutron class CSR (|S_n dst|+1)
    int64_t w_off;
    int64_t n1e_col, n1e_slice;   // ELL of the neutron class
    int64_t pe_ent, pe_sinfo;     // pipelined kernel: class entries and slice info
    int64_t ww_off;               // pipelined kernel: signed W rows of the proton group
};

struct DevLLink {
    int src_block;
    int species;            // 0: pp (rows of the source block), 1: nn (columns)
    int64_t ptr_off;        // class CSR in ppx_ptr / nnx_ptr
};

struct DevTask {            // one CTA: destination block, proton row, column tile
    int block;
    int row;
    int col0;
    int pad;
};

template <typename T>
struct DevCoefs {
    T *pp_coef = nullptr, *nn_coef = nullptr, *wpn = nullptr, *nne_coef = nullptr;
    T *ppx_coef = nullptr, *nnx_coef = nullptr;
};

struct RowTask {            // row kernel: one CTA per destination proton row
    int block;
    int row;
};

struct Device {
    int dev = 0;
    bool trunc = false;       // W-truncated basis: only the tiled kernel applies
    DevBlock *blocks = nullptr;
    DevLink *links = nullptr;
    DevLLink *llinks = nullptr;
    int64_t *ppx_ptr = nullptr, *nnx_ptr = nullptr;
    int32_t *ppx_src = nullptr, *nnx_src = nullptr;
    DevTask *tasks = nullptr;
    int ntasks = 0;
    int tile = 0;
    int64_t *pp_ptr = nullptr, *nn_ptr = nullptr;
    int32_t *pp_src = nullptr, *nn_src = nullptr;
    int64_t *p1_ptr = nullptr, *n1_ptr = nullptr;
    uint32_t *p1_ent = nullptr, *n1_ent = nullptr;
    DevCoefs<double> c64;
    DevCoefs<float> c32;
    // row kernel
    RowTask *rtasks = nullptr;
    int nrtasks = 0;
    int32_t *n1e_col = nullptr, *n1e_len = nullptr, *nne_col = nullptr, *nne_len = nullptr, *nne_src = nullptr;
    int64_t *n1e_soff = nullptr, *nne_soff = nullptr;
    uint32_t *n1e_ent = nullptr;
    int max_nN = 0, max_nb = 0, max_pu = 0, wsign = 0;   // widest neutron sector, widest W row, most proton jumps per (row, link)
    int *err = nullptr;                       // device status word (BS_ETIMEOUT from bounded waits)
    int *core_next = nullptr;                 // unit counters of the persistent core-grouped kernels: pn, pp
    // pipelined kernel
    int32_t *pe_perm = nullptr, *pe_sinfo = nullptr, *pe_nn_src = nullptr, *pe_nn_sinfo = nullptr;
    uint32_t *pe_ent = nullptr;
    double *pe_nn_coef64 = nullptr, *ww64 = nullptr;
    float *pe_nn_coef32 = nullptr, *ww32 = nullptr;
    // core-grouped pn kernel
    CoreUnit *cunits = nullptr;
    CoreSrc *csrc = nullptr;
    uint32_t *core_ent = nullptr;
    float *wc32 = nullptr;
    int ncunits = 0, nz = 0;
    int64_t core_list_max[2] = {0, 0};   // largest list block of one column tile (18, 10 warps), entries
    PPUnit *ppunits = nullptr;
    int32_t *pps_row = nullptr;
    float *pps_w32 = nullptr, *pdiag32 = nullptr;
    int nppunits = 0, nzpp = 0;
    // neutron like-particle kernel over tiles of R proton rows (R = 2, 4): (block, first row)
    int2 *nntasks2 = nullptr, *nntasks4 = nullptr;
    int nnntasks2 = 0, nnntasks4 = 0;
    std::vector<void *> owned;   // every cudaMalloc above
};

}  // namespace bs

struct bs_ctx {
    int device = 0;
    std::string err;
    bool have_basis = false, have_int = false;
    bs::Basis basis;
    bs::Interaction inter;
    bs::Tables tab;
    bs::Device dev;
    // host-buffer entry point workspace
    void *hx_x = nullptr, *hx_y = nullptr;
    size_t hx_bytes = 0;
    // asynchronous host-buffer entry point: two staging slots, the event that ends
    // each slot's last use, and the event that ends the last product
    void *hxa_x[2] = {nullptr, nullptr}, *hxa_y[2] = {nullptr, nullptr};
    size_t hxa_bytes = 0;
    cudaEvent_t hxa_free[2] = {nullptr, nullptr}, hxa_prod = nullptr;
    int hx_mode = 0;         // 0: autotuned, 1: tiled kernel, 2 + v: row kernel variant v, then pipelined, then core
    // partial sums of the core-grouped pn kernel: nz x dim x k elements, grown on demand
    mutable void *core_part = nullptr;
    mutable size_t core_part_bytes = 0;
    // event pairs around the dominant kernel of each product (bs_time_kernel)
    std::vector<cudaEvent_t> tev;
    mutable int tev_used = 0;
    int tuned[2][4] = {};    // autotuned mode per (dtype, k slot); 0 = not tuned
    // the loaded interaction as given (for the parameter derivatives of the adjoint)
    std::vector<double> spe_in;
    std::vector<bs_tbme> tbme_in;
    // adjoint: derivative of the decoupled tables w.r.t. each TBME, sparse, built on first use
    bool have_dW = false;
    std::vector<std::vector<std::pair<int64_t, double>>> dWpp, dWpn;
    // adjoint device buffers
    double *adj_gpp = nullptr, *adj_gnn = nullptr, *adj_rho = nullptr;
};

// ---------------------------------------------------------------- builders (host)
namespace bs {
int build_basis(Basis &B, const bs_orbit *orbits, int n_orbits, int Z, int N, int twoM, int parity, int max_excite,
                std::string &err);
int build_interaction(const Basis &B, const double *spe, int n_spe, const bs_tbme *tbme, int n_tbme,
                      Interaction &I, std::string &err);
int build_tables(const Basis &B, const Interaction &I, Tables &T, std::string &err, int grid = 152);
int upload(const Basis &B, const Interaction &I, const Tables &T, Device &D, std::string &err);
void release(Device &D);
int launch_hx(const bs_ctx *ctx, const void *x, void *y, int k, bs_dtype dt, void *stream, std::string &err);
int row_variants();
int run_block_dots(bs_ctx *c, const void *V, int nb, const void *W, int k, bs_dtype dt, double *C, void *stream);
int run_block_update(bs_ctx *c, const void *V, int nb, const double *C, void *W, int k, bs_dtype dt, void *stream);
int run_backward(bs_ctx *c, const void *x, const void *gy, void *gx, double *gtheta, int k, bs_dtype dt,
                 void *stream);
// strength-function outputs of a Lanczos run (host): the lowest n_out
// eigenvalues of T and |<w_i|E_r>|^2 per pivot column i ([k][n_out])
struct StrengthReq {
    int n_out;
    double *E;
    double *S;
};
int run_lanczos(bs_ctx *c, const bs_lanczos_opts &o, const void *pivot, double *evals, double *evecs,
                bs_lanczos_report *rep, const StrengthReq *sreq = nullptr);
int run_density(bs_ctx *c, const double *F, const double *X, int k, double *rho_host, void *stream);
int run_gather_ceiling(int device, int where, int k, int rows, double *gflops, void *stream, std::string &err);
int run_wait_expiry(int device, uint32_t limit, int *err, void *stream, std::string &msg);
uint32_t tma_wait_limit();   // iteration limit of the kernels' bounded mbarrier waits
int pipe_variants();
int core_variants();
// allocates what launch_hx needs for (k, dtype) outside any stream capture
int prepare_hx(const bs_ctx *ctx, int k, bs_dtype dt, std::string &err);
}  // namespace bs
