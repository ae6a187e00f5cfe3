// The C ABI (include/bigstick_gpu.h): context, error codes, basis and
// interaction set-up, device upload, and the host-buffer entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <cstring>
#include <new>

#include "bs_internal.h"

using namespace bs;

namespace {

int cuda_fail(bs_ctx *c, cudaError_t e, const char *what)
{
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? BS_ENOMEM : BS_ECUDA;
}

template <typename F>
int guarded(bs_ctx *c, F &&f)
{
    if (!c) return BS_EINVAL;
    try {
        return f();
    } catch (const std::bad_alloc &) {
        c->err = "host allocation failed";
        return BS_ENOMEM;
    } catch (const std::exception &e) {
        c->err = e.what();
        return BS_EINVAL;
    } catch (...) {
        c->err = "unknown error";
        return BS_EINVAL;
    }
}

template <typename T>
int put(Device &D, T *&dst, const T *src, size_t n, std::string &err)
{
    dst = nullptr;
    size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)&dst, bytes);
    if (e != cudaSuccess) { err = std::string("cudaMalloc: ") + cudaGetErrorString(e); return e == cudaErrorMemoryAllocation ? BS_ENOMEM : BS_ECUDA; }
    D.owned.push_back(dst);
    if (n) {
        e = cudaMemcpy(dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { err = std::string("cudaMemcpy: ") + cudaGetErrorString(e); return BS_ECUDA; }
    }
    return BS_OK;
}

template <typename T>
std::vector<T> cast(const std::vector<double> &v)
{
    return std::vector<T>(v.begin(), v.end());
}

}  // namespace

namespace bs {

void release(Device &D)
{
    for (void *p : D.owned) cudaFree(p);
    D.owned.clear();
    int dev = D.dev;
    D = Device();
    D.dev = dev;
}

// Task list for the fused kernel: one CTA per (destination block, proton row,
// tile of neutron columns), ordered by estimated work, largest first, so the
// hardware's in-order CTA dispatch approximates longest-processing-time
// scheduling.
static void make_tasks(const Basis &B, const Tables &T, int tile, std::vector<DevTask> &tasks)
{
    struct C { double cost; DevTask t; };
    std::vector<C> v;
    for (size_t b = 0; b < B.blocks.size(); ++b) {
        const Block &D = B.blocks[b];
        const Sector &PS = B.sp[0].sec[D.ps], &NS = B.sp[1].sec[D.ns];
        double nn_avg = (double)(T.nn.ptr[NS.start + NS.count] - T.nn.ptr[NS.start]) / (double)std::max<int64_t>(1, NS.count);
        for (int64_t r = 0; r < D.nP; ++r) {
            double per_col = (double)(T.pp.ptr[PS.start + r + 1] - T.pp.ptr[PS.start + r]) + nn_avg;
            for (int64_t L = T.links_of_block[b]; L < T.links_of_block[b + 1]; ++L) {
                const PnLink &lk = T.links[(size_t)L];
                const OneBodyClass &P = T.p1.cls[(size_t)lk.pcls], &N = T.n1.cls[(size_t)lk.ncls];
                double np_ = (double)(T.p1.ptr[(size_t)(P.ptr_off + r + 1)] - T.p1.ptr[(size_t)(P.ptr_off + r)]);
                double nn_ = (double)(T.n1.ptr[(size_t)(N.ptr_off + D.nN)] - T.n1.ptr[(size_t)N.ptr_off]) / (double)D.nN;
                per_col += np_ * nn_;
            }
            for (int64_t c0 = 0; c0 < D.nN; c0 += tile) {
                int64_t cols = std::min<int64_t>(tile, D.nN - c0);
                v.push_back(C{per_col * (double)cols, DevTask{(int)b, (int)r, (int)c0, 0}});
            }
        }
    }
    std::stable_sort(v.begin(), v.end(), [](const C &a, const C &b) { return a.cost > b.cost; });
    tasks.resize(v.size());
    for (size_t i = 0; i < v.size(); ++i) tasks[i] = v[i].t;
}

// One CTA per destination proton row for the row kernel, largest work first.
static void make_row_tasks(const Basis &B, const Tables &T, std::vector<RowTask> &tasks, int &max_pu)
{
    struct C { double cost; RowTask t; };
    std::vector<C> v;
    max_pu = 0;
    for (size_t b = 0; b < B.blocks.size(); ++b) {
        const Block &D = B.blocks[b];
        const Sector &PS = B.sp[0].sec[D.ps], &NS = B.sp[1].sec[D.ns];
        double nn_avg = (double)(T.nn.ptr[NS.start + NS.count] - T.nn.ptr[NS.start]) / (double)std::max<int64_t>(1, NS.count);
        for (int64_t r = 0; r < D.nP; ++r) {
            double per_col = (double)(T.pp.ptr[PS.start + r + 1] - T.pp.ptr[PS.start + r]) + nn_avg;
            for (int64_t L = T.links_of_block[b]; L < T.links_of_block[b + 1]; ++L) {
                const PnLink &lk = T.links[(size_t)L];
                const OneBodyClass &P = T.p1.cls[(size_t)lk.pcls], &N = T.n1.cls[(size_t)lk.ncls];
                int64_t np_ = T.p1.ptr[(size_t)(P.ptr_off + r + 1)] - T.p1.ptr[(size_t)(P.ptr_off + r)];
                max_pu = std::max<int>(max_pu, (int)np_);
                double nn_ = (double)(T.n1.ptr[(size_t)(N.ptr_off + D.nN)] - T.n1.ptr[(size_t)N.ptr_off]) / (double)D.nN;
                per_col += (double)np_ * nn_;
            }
            v.push_back(C{per_col * (double)D.nN, RowTask{(int)b, (int)r}});
        }
    }
    std::stable_sort(v.begin(), v.end(), [](const C &a, const C &b) { return a.cost > b.cost; });
    tasks.resize(v.size());
    for (size_t i = 0; i < v.size(); ++i) tasks[i] = v[i].t;
}

int upload(const Basis &B, const Interaction &I, const Tables &T, Device &D, std::string &err)
{
    release(D);
    cudaError_t e = cudaSetDevice(D.dev);
    if (e != cudaSuccess) { err = std::string("cudaSetDevice: ") + cudaGetErrorString(e); return BS_ECUDA; }
    int rc;
    std::vector<DevBlock> blocks(B.blocks.size());
    for (size_t b = 0; b < B.blocks.size(); ++b) {
        const Block &s = B.blocks[b];
        blocks[b].off = s.off;
        blocks[b].nP = (int)s.nP;
        blocks[b].nN = (int)s.nN;
        blocks[b].p_start = (int)B.sp[0].sec[s.ps].start;
        blocks[b].n_start = (int)B.sp[1].sec[s.ns].start;
        blocks[b].link_begin = (int)T.links_of_block[b];
        blocks[b].link_end = (int)T.links_of_block[b + 1];
        blocks[b].llink_begin = (int)T.llinks_of_block[b];
        blocks[b].llink_end = (int)T.llinks_of_block[b + 1];
        blocks[b].nne_col = T.nne_col[(size_t)s.ns];
        blocks[b].nne_slice = T.nne_slice[(size_t)s.ns];
        blocks[b].perm_off = T.pe.perm_off[(size_t)s.ns];
        blocks[b].pe_nn_ent = T.pe.sec_nn_ent[(size_t)s.ns];
        blocks[b].pe_nn_sinfo = T.pe.sec_nn_sinfo[(size_t)s.ns];
    }
    std::vector<DevLink> links(T.links.size());
    for (size_t l = 0; l < T.links.size(); ++l) {
        const PnLink &L = T.links[l];
        links[l].src_block = L.src_block;
        links[l].p_ptr_off = T.p1.cls[(size_t)L.pcls].ptr_off;
        links[l].n_ptr_off = T.n1.cls[(size_t)L.ncls].ptr_off;
        links[l].w_off = L.w_off;
        links[l].nb = L.nb;
        links[l].n1e_col = T.n1e_col[(size_t)L.ncls];
        links[l].n1e_slice = T.n1e_slice[(size_t)L.ncls];
        links[l].pe_ent = T.pe.cls_ent[(size_t)L.ncls];
        links[l].pe_sinfo = T.pe.cls_sinfo[(size_t)L.ncls];
        links[l].ww_off = T.ww_off[(size_t)T.p1.cls[(size_t)L.pcls].group];
    }
    std::vector<DevLLink> llinks(T.llinks.size());
    for (size_t l = 0; l < T.llinks.size(); ++l)
        llinks[l] = DevLLink{T.llinks[l].src_block, T.llinks[l].species, T.llinks[l].ptr_off};
    D.trunc = B.trunc;
    D.tile = 128;
    std::vector<DevTask> tasks;
    make_tasks(B, T, D.tile, tasks);
    D.ntasks = (int)tasks.size();
    if ((rc = put(D, D.blocks, blocks.data(), blocks.size(), err))) return rc;
    if ((rc = put(D, D.links, links.data(), links.size(), err))) return rc;
    if ((rc = put(D, D.tasks, tasks.data(), tasks.size(), err))) return rc;
    if ((rc = put(D, D.pp_ptr, T.pp.ptr.data(), T.pp.ptr.size(), err))) return rc;
    if ((rc = put(D, D.pp_src, T.pp.src.data(), T.pp.src.size(), err))) return rc;
    if ((rc = put(D, D.nn_ptr, T.nn.ptr.data(), T.nn.ptr.size(), err))) return rc;
    if ((rc = put(D, D.nn_src, T.nn.src.data(), T.nn.src.size(), err))) return rc;
    if ((rc = put(D, D.p1_ptr, T.p1.ptr.data(), T.p1.ptr.size(), err))) return rc;
    if ((rc = put(D, D.p1_ent, T.p1.ent.data(), T.p1.ent.size(), err))) return rc;
    if ((rc = put(D, D.n1_ptr, T.n1.ptr.data(), T.n1.ptr.size(), err))) return rc;
    if ((rc = put(D, D.n1_ent, T.n1.ent.data(), T.n1.ent.size(), err))) return rc;
    if ((rc = put(D, D.c64.pp_coef, T.pp.coef.data(), T.pp.coef.size(), err))) return rc;
    if ((rc = put(D, D.c64.nn_coef, T.nn.coef.data(), T.nn.coef.size(), err))) return rc;
    if ((rc = put(D, D.c64.wpn, I.Wpn.data(), I.Wpn.size(), err))) return rc;
    // like-particle moves between sectors (W-truncated bases; empty otherwise)
    if ((rc = put(D, D.llinks, llinks.data(), llinks.size(), err))) return rc;
    if ((rc = put(D, D.ppx_ptr, T.ppx.ptr.data(), T.ppx.ptr.size(), err))) return rc;
    if ((rc = put(D, D.ppx_src, T.ppx.src.data(), T.ppx.src.size(), err))) return rc;
    if ((rc = put(D, D.nnx_ptr, T.nnx.ptr.data(), T.nnx.ptr.size(), err))) return rc;
    if ((rc = put(D, D.nnx_src, T.nnx.src.data(), T.nnx.src.size(), err))) return rc;
    if ((rc = put(D, D.c64.ppx_coef, T.ppx.coef.data(), T.ppx.coef.size(), err))) return rc;
    if ((rc = put(D, D.c64.nnx_coef, T.nnx.coef.data(), T.nnx.coef.size(), err))) return rc;
    std::vector<float> f;
    f = cast<float>(T.ppx.coef);
    if ((rc = put(D, D.c32.ppx_coef, f.data(), f.size(), err))) return rc;
    f = cast<float>(T.nnx.coef);
    if ((rc = put(D, D.c32.nnx_coef, f.data(), f.size(), err))) return rc;
    f = cast<float>(T.pp.coef);
    if ((rc = put(D, D.c32.pp_coef, f.data(), f.size(), err))) return rc;
    f = cast<float>(T.nn.coef);
    if ((rc = put(D, D.c32.nn_coef, f.data(), f.size(), err))) return rc;
    f = cast<float>(I.Wpn);
    if ((rc = put(D, D.c32.wpn, f.data(), f.size(), err))) return rc;
    // row kernel
    std::vector<RowTask> rt;
    make_row_tasks(B, T, rt, D.max_pu);
    D.nrtasks = (int)rt.size();
    D.max_nN = 0;
    for (const Sector &S : B.sp[1].sec) D.max_nN = std::max<int>(D.max_nN, (int)S.count);
    D.max_nb = 1;
    for (const PnLink &L : T.links) D.max_nb = std::max(D.max_nb, L.nb);
    D.wsign = T.wsign;
    if ((rc = put(D, D.rtasks, rt.data(), rt.size(), err))) return rc;
    if ((rc = put(D, D.n1e_col, T.n1e.col.data(), T.n1e.col.size(), err))) return rc;
    if ((rc = put(D, D.n1e_len, T.n1e.len.data(), T.n1e.len.size(), err))) return rc;
    if ((rc = put(D, D.n1e_soff, T.n1e.soff.data(), T.n1e.soff.size(), err))) return rc;
    if ((rc = put(D, D.n1e_ent, T.n1e.ent.data(), T.n1e.ent.size(), err))) return rc;
    if ((rc = put(D, D.nne_col, T.nne.col.data(), T.nne.col.size(), err))) return rc;
    if ((rc = put(D, D.nne_len, T.nne.len.data(), T.nne.len.size(), err))) return rc;
    if ((rc = put(D, D.nne_soff, T.nne.soff.data(), T.nne.soff.size(), err))) return rc;
    if ((rc = put(D, D.nne_src, T.nne.src.data(), T.nne.src.size(), err))) return rc;
    if ((rc = put(D, D.c64.nne_coef, T.nne.coef.data(), T.nne.coef.size(), err))) return rc;
    f = cast<float>(T.nne.coef);
    if ((rc = put(D, D.c32.nne_coef, f.data(), f.size(), err))) return rc;
    int zero = 0;
    if ((rc = put(D, D.err, &zero, 1, err))) return rc;
    const int zeros[4] = {0, 0, 0, 0};
    if ((rc = put(D, D.core_next, zeros, 4, err))) return rc;
    // pipelined kernel
    if ((rc = put(D, D.pe_perm, T.pe.perm.data(), T.pe.perm.size(), err))) return rc;
    if ((rc = put(D, D.pe_sinfo, T.pe.sinfo.data(), T.pe.sinfo.size(), err))) return rc;
    if ((rc = put(D, D.pe_ent, T.pe.ent.data(), T.pe.ent.size(), err))) return rc;
    if ((rc = put(D, D.pe_nn_src, T.pe.nn_src.data(), T.pe.nn_src.size(), err))) return rc;
    if ((rc = put(D, D.pe_nn_sinfo, T.pe.nn_sinfo.data(), T.pe.nn_sinfo.size(), err))) return rc;
    if ((rc = put(D, D.pe_nn_coef64, T.pe.nn_coef.data(), T.pe.nn_coef.size(), err))) return rc;
    f = cast<float>(T.pe.nn_coef);
    if ((rc = put(D, D.pe_nn_coef32, f.data(), f.size(), err))) return rc;
    if ((rc = put(D, D.ww64, T.ww.data(), T.ww.size(), err))) return rc;
    // core-grouped pn kernel
    D.ncunits = (int)T.cunits.size();
    D.nz = D.ncunits ? B.sp[0].nparticles : 0;
    if ((rc = put(D, D.cunits, T.cunits.data(), T.cunits.size(), err))) return rc;
    if ((rc = put(D, D.csrc, T.csrc.data(), T.csrc.size(), err))) return rc;
    if ((rc = put(D, D.core_ent, T.pe.core_ent.data(), T.pe.core_ent.size(), err))) return rc;
    f = cast<float>(T.wc);
    if ((rc = put(D, D.wc32, f.data(), f.size(), err))) return rc;
    // largest list block one column tile of the pn-core kernel stages (18 or 10 warps of 32 columns)
    for (int vi = 0; vi < 2; ++vi) {
        const int nw = vi == 0 ? 18 : 10;
        int64_t mx = 0;
        for (size_t cl = 0; cl < T.n1.cls.size(); ++cl) {
            const int64_t n = B.sp[1].sec[(size_t)T.n1.cls[cl].s_dst].count;
            const int64_t nsl = (n + 31) / 32;
            const int32_t *si = T.pe.sinfo.data() + T.pe.cls_sinfo[cl];
            for (int64_t s0 = 0; s0 < nsl; s0 += nw) {
                const int64_t s1 = std::min(nsl, s0 + nw) - 1;
                mx = std::max<int64_t>(mx, (int64_t)si[2 * s1] + 32 * (int64_t)si[2 * s1 + 1] - si[2 * s0]);
            }
        }
        D.core_list_max[vi] = mx;
    }
    // core-grouped pp kernel
    D.nppunits = (int)T.ppunits.size();
    D.nzpp = D.nppunits ? B.sp[0].nparticles * (B.sp[0].nparticles - 1) / 2 : 0;
    if ((rc = put(D, D.ppunits, T.ppunits.data(), T.ppunits.size(), err))) return rc;
    if ((rc = put(D, D.pps_row, T.pps_row.data(), T.pps_row.size(), err))) return rc;
    f = cast<float>(T.pps_w);
    if ((rc = put(D, D.pps_w32, f.data(), f.size(), err))) return rc;
    f = cast<float>(T.pdiag);
    if ((rc = put(D, D.pdiag32, f.data(), f.size(), err))) return rc;
    for (int R : {2, 4}) {
        // row tiles of the neutron like-particle kernel, widest sectors first
        std::vector<int2> nt;
        std::vector<size_t> ord(B.blocks.size());
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b2) { return B.blocks[a].nN > B.blocks[b2].nN; });
        for (size_t b2 : ord)
            for (int64_t r = 0; r < B.blocks[b2].nP; r += R) nt.push_back(make_int2((int)b2, (int)r));
        int2 *&dst = R == 2 ? D.nntasks2 : D.nntasks4;
        (R == 2 ? D.nnntasks2 : D.nnntasks4) = (int)nt.size();
        if ((rc = put(D, dst, nt.data(), nt.size(), err))) return rc;
    }
    f = cast<float>(T.ww);
    if ((rc = put(D, D.ww32, f.data(), f.size(), err))) return rc;
    return BS_OK;
}

}  // namespace bs

extern "C" {

int bs_create(bs_ctx **out, int cuda_device)
{
    if (!out) return BS_EINVAL;
    *out = nullptr;
    bs_ctx *c = new (std::nothrow) bs_ctx();
    if (!c) return BS_ENOMEM;
    c->device = cuda_device;
    c->dev.dev = cuda_device;
    if (cuda_device >= 0) {
        int n = 0;
        cudaError_t e = cudaGetDeviceCount(&n);
        if (e != cudaSuccess || cuda_device >= n) {
            delete c;
            return e != cudaSuccess ? BS_ECUDA : BS_EINVAL;
        }
    }
    *out = c;
    return BS_OK;
}

void bs_destroy(bs_ctx *c)
{
    if (!c) return;
    if (c->device >= 0) {
        cudaSetDevice(c->device);
        release(c->dev);
        if (c->adj_gpp) cudaFree(c->adj_gpp);
        if (c->adj_gnn) cudaFree(c->adj_gnn);
        if (c->adj_rho) cudaFree(c->adj_rho);
        if (c->hx_x) cudaFree(c->hx_x);
        if (c->hx_y) cudaFree(c->hx_y);
        for (int i = 0; i < 2; ++i) {
            if (c->hxa_x[i]) cudaFree(c->hxa_x[i]);
            if (c->hxa_y[i]) cudaFree(c->hxa_y[i]);
            if (c->hxa_free[i]) cudaEventDestroy(c->hxa_free[i]);
        }
        if (c->hxa_prod) cudaEventDestroy(c->hxa_prod);
        if (c->core_part) cudaFree(c->core_part);
        for (cudaEvent_t ev : c->tev) cudaEventDestroy(ev);
    }
    delete c;
}

const char *bs_last_error(const bs_ctx *c) { return c ? c->err.c_str() : "null context"; }

int bs_build_basis_trunc(bs_ctx *c, const bs_orbit *orbits, int n_orbits, int Z, int N, int twoM, int parity,
                         int max_excite)
{
    return guarded(c, [&]() -> int {
        c->have_basis = c->have_int = false;
        if (c->device >= 0) release(c->dev);
        if (max_excite < -1) { c->err = "build_basis: max_excite must be -1 (no truncation) or >= 0"; return BS_EINVAL; }
        int rc = build_basis(c->basis, orbits, n_orbits, Z, N, twoM, parity, max_excite, c->err);
        if (rc) return rc;
        c->have_basis = true;
        c->err.clear();
        return BS_OK;
    });
}

int bs_build_basis(bs_ctx *c, const bs_orbit *orbits, int n_orbits, int Z, int N, int twoM, int parity)
{
    return bs_build_basis_trunc(c, orbits, n_orbits, Z, N, twoM, parity, -1);
}

int bs_basis_info(bs_ctx *c, int64_t *dim, int *n_psec, int *n_nsec, int *n_psd, int *n_nsd, int *n_blocks)
{
    return guarded(c, [&]() -> int {
        if (!c->have_basis) { c->err = "no basis"; return BS_ENOBASIS; }
        const Basis &B = c->basis;
        if (dim) *dim = B.dim;
        if (n_psec) *n_psec = (int)B.sp[0].sec.size();
        if (n_nsec) *n_nsec = (int)B.sp[1].sec.size();
        if (n_psd) *n_psd = (int)B.sp[0].bits.size();
        if (n_nsd) *n_nsd = (int)B.sp[1].bits.size();
        if (n_blocks) *n_blocks = (int)B.blocks.size();
        return BS_OK;
    });
}

int bs_export_basis(bs_ctx *c, uint64_t *p_bits, uint64_t *n_bits, int64_t *p_sec, int64_t *n_sec, int64_t *blocks)
{
    return guarded(c, [&]() -> int {
        if (!c->have_basis) { c->err = "no basis"; return BS_ENOBASIS; }
        const Basis &B = c->basis;
        uint64_t *bits[2] = {p_bits, n_bits};
        int64_t *sec[2] = {p_sec, n_sec};
        for (int s = 0; s < 2; ++s) {
            if (bits[s]) std::memcpy(bits[s], B.sp[s].bits.data(), B.sp[s].bits.size() * sizeof(uint64_t));
            if (sec[s])
                for (size_t t = 0; t < B.sp[s].sec.size(); ++t) {
                    sec[s][4 * t] = B.sp[s].sec[t].twoM;
                    sec[s][4 * t + 1] = B.sp[s].sec[t].par;
                    sec[s][4 * t + 2] = B.sp[s].sec[t].start;
                    sec[s][4 * t + 3] = B.sp[s].sec[t].count;
                }
        }
        if (blocks)
            for (size_t b = 0; b < B.blocks.size(); ++b) {
                blocks[3 * b] = B.blocks[b].ps;
                blocks[3 * b + 1] = B.blocks[b].ns;
                blocks[3 * b + 2] = B.blocks[b].off;
            }
        return BS_OK;
    });
}

int bs_load_interaction(bs_ctx *c, const double *spe, int n_spe, const bs_tbme *tbme, int n_tbme)
{
    return guarded(c, [&]() -> int {
        if (!c->have_basis) { c->err = "no basis"; return BS_ENOBASIS; }
        c->have_int = false;
        int rc = build_interaction(c->basis, spe, n_spe, tbme, n_tbme, c->inter, c->err);
        if (rc == BS_OK) {
            std::vector<bs_tbme> tb(tbme, tbme + std::max(0, n_tbme));
            bool same_labels = tb.size() == c->tbme_in.size() && c->spe_in.size() == (size_t)n_spe;
            for (size_t i = 0; same_labels && i < tb.size(); ++i)
                same_labels = tb[i].a == c->tbme_in[i].a && tb[i].b == c->tbme_in[i].b && tb[i].c == c->tbme_in[i].c &&
                              tb[i].d == c->tbme_in[i].d && tb[i].J == c->tbme_in[i].J && tb[i].T == c->tbme_in[i].T;
            if (!same_labels) c->have_dW = false;   // derivative tables depend on the labels only
            c->spe_in.assign(spe, spe + n_spe);
            c->tbme_in.swap(tb);
        }
        if (rc) return rc;
        int nsm = 152;   // the persistent kernels run one CTA per SM: balance their units for this device
        if (c->device >= 0 && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
            (void)cudaGetLastError();
            nsm = 152;
        }
        rc = build_tables(c->basis, c->inter, c->tab, c->err, nsm);
        if (rc) return rc;
        if (c->device >= 0) {
            if (c->adj_gpp) { cudaFree(c->adj_gpp); cudaFree(c->adj_gnn); cudaFree(c->adj_rho); }
            c->adj_gpp = c->adj_gnn = c->adj_rho = nullptr;
            rc = upload(c->basis, c->inter, c->tab, c->dev, c->err);
            if (rc) { release(c->dev); return rc; }
        }
        c->have_int = true;
        c->err.clear();
        return BS_OK;
    });
}

static int check_apply(bs_ctx *c, int k, bs_dtype dt)
{
    if (!c->have_basis) { c->err = "no basis"; return BS_ENOBASIS; }
    if (!c->have_int) { c->err = "no interaction"; return BS_ENOINT; }
    if (c->device < 0) { c->err = "context has no device"; return BS_EINVAL; }
    if (k != 1 && k != 2 && k != 4 && k != 8) { c->err = "k must be 1, 2, 4 or 8"; return BS_EINVAL; }
    if (dt != BS_F64 && dt != BS_F32) { c->err = "bad dtype"; return BS_EINVAL; }
    return BS_OK;
}

int bs_apply_H(bs_ctx *c, const void *x, void *y, int k, bs_dtype dt, void *stream)
{
    return guarded(c, [&]() -> int {
        int rc = check_apply(c, k, dt);
        if (rc) return rc;
        if (!x || !y || x == y) { c->err = "x and y must be distinct device buffers"; return BS_EINVAL; }
        if (((uintptr_t)x | (uintptr_t)y) & 15) { c->err = "x and y must be 16-byte aligned"; return BS_EINVAL; }
        return launch_hx(c, x, y, k, dt, stream, c->err);
    });
}

int bs_apply_H_host(bs_ctx *c, const void *xh, void *yh, int k, bs_dtype dt, void *stream)
{
    return guarded(c, [&]() -> int {
        int rc = check_apply(c, k, dt);
        if (rc) return rc;
        if (!xh || !yh) { c->err = "null host buffer"; return BS_EINVAL; }
        size_t bytes = (size_t)c->basis.dim * (size_t)k * (dt == BS_F64 ? 8 : 4);
        cudaError_t e;
        if (bytes > c->hx_bytes) {
            if (c->hx_x) cudaFree(c->hx_x);
            if (c->hx_y) cudaFree(c->hx_y);
            c->hx_x = c->hx_y = nullptr;
            c->hx_bytes = 0;
            if ((e = cudaMalloc(&c->hx_x, bytes)) != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
            if ((e = cudaMalloc(&c->hx_y, bytes)) != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
            c->hx_bytes = bytes;
        }
        cudaStream_t s = (cudaStream_t)stream;
        if ((e = cudaMemcpyAsync(c->hx_x, xh, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync");
        if ((rc = launch_hx(c, c->hx_x, c->hx_y, k, dt, stream, c->err))) return rc;
        if ((e = cudaMemcpyAsync(yh, c->hx_y, bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
        return BS_OK;
    });
}

int bs_apply_H_host_async(bs_ctx *c, const void *xh, void *yh, int k, bs_dtype dt, void *stream, int slot)
{
    return guarded(c, [&]() -> int {
        int rc = check_apply(c, k, dt);
        if (rc) return rc;
        if (!xh || !yh) { c->err = "null host buffer"; return BS_EINVAL; }
        if (slot < 0 || slot > 1) { c->err = "host async: slot must be 0 or 1"; return BS_EINVAL; }
        const size_t bytes = (size_t)c->basis.dim * (size_t)k * (dt == BS_F64 ? 8 : 4);
        cudaError_t e;
        for (int i = 0; i < 2; ++i)
            if (!c->hxa_free[i] && (e = cudaEventCreateWithFlags(&c->hxa_free[i], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(c, e, "cudaEventCreate");
        if (!c->hxa_prod && (e = cudaEventCreateWithFlags(&c->hxa_prod, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(c, e, "cudaEventCreate");
        if (bytes > c->hxa_bytes) {
            // larger blocks: wait for every use of the old buffers, then replace them
            for (int i = 0; i < 2; ++i)
                if ((e = cudaEventSynchronize(c->hxa_free[i])) != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize");
            for (int i = 0; i < 2; ++i) {
                if (c->hxa_x[i]) cudaFree(c->hxa_x[i]);
                if (c->hxa_y[i]) cudaFree(c->hxa_y[i]);
                c->hxa_x[i] = c->hxa_y[i] = nullptr;
            }
            c->hxa_bytes = 0;
            for (int i = 0; i < 2; ++i) {
                if ((e = cudaMalloc(&c->hxa_x[i], bytes)) != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
                if ((e = cudaMalloc(&c->hxa_y[i], bytes)) != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
            }
            c->hxa_bytes = bytes;
        }
        cudaStream_t s = (cudaStream_t)stream;
        // the slot's previous use (its copy out) has ended; then x in, which may run while
        // another stream's product does
        if ((e = cudaStreamWaitEvent(s, c->hxa_free[slot], 0)) != cudaSuccess) return cuda_fail(c, e, "cudaStreamWaitEvent");
        if ((e = cudaMemcpyAsync(c->hxa_x[slot], xh, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(c, e, "cudaMemcpyAsync");
        // the previous product has ended: products share the context's workspace
        if ((e = cudaStreamWaitEvent(s, c->hxa_prod, 0)) != cudaSuccess) return cuda_fail(c, e, "cudaStreamWaitEvent");
        if ((rc = launch_hx(c, c->hxa_x[slot], c->hxa_y[slot], k, dt, stream, c->err))) return rc;
        if ((e = cudaEventRecord(c->hxa_prod, s)) != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
        if ((e = cudaMemcpyAsync(yh, c->hxa_y[slot], bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(c, e, "cudaMemcpyAsync");
        if ((e = cudaEventRecord(c->hxa_free[slot], s)) != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
        return BS_OK;
    });
}

int bs_block_dots(bs_ctx *c, const void *V, int nb, const void *W, int k, bs_dtype dt, double *C, void *stream)
{
    return guarded(c, [&]() -> int {
        int rc = check_apply(c, k, dt);
        if (rc) return rc;
        if (!V || !W || !C || nb < 1) { c->err = "block dots: need V, W, C and nb >= 1"; return BS_EINVAL; }
        return run_block_dots(c, V, nb, W, k, dt, C, stream);
    });
}

int bs_block_update(bs_ctx *c, const void *V, int nb, const double *C, void *W, int k, bs_dtype dt, void *stream)
{
    return guarded(c, [&]() -> int {
        int rc = check_apply(c, k, dt);
        if (rc) return rc;
        if (!V || !W || !C || nb < 1) { c->err = "block update: need V, C, W and nb >= 1"; return BS_EINVAL; }
        const size_t es = dt == BS_F64 ? 8 : 4, blk = (size_t)c->basis.dim * (size_t)k * es;
        const uintptr_t v0 = (uintptr_t)V, v1 = v0 + (size_t)nb * blk, w0 = (uintptr_t)W, w1 = w0 + blk;
        if (w0 < v1 && v0 < w1) { c->err = "block update: W overlaps V"; return BS_EINVAL; }
        return run_block_update(c, V, nb, C, W, k, dt, stream);
    });
}

int bs_apply_H_backward(bs_ctx *c, const void *x, const void *gy, void *gx, double *gtheta, int k, bs_dtype dt,
                        void *stream)
{
    return guarded(c, [&]() -> int {
        int rc = check_apply(c, k, dt);
        if (rc) return rc;
        if (c->basis.trunc) { c->err = "backward: not available on a W-truncated basis"; return BS_EINVAL; }
        if (!x || !gy || !gx || gy == gx) { c->err = "x, gy and gx must be device buffers, gy != gx"; return BS_EINVAL; }
        if (((uintptr_t)x | (uintptr_t)gy | (uintptr_t)gx) & 15) { c->err = "buffers must be 16-byte aligned"; return BS_EINVAL; }
        return run_backward(c, x, gy, gx, gtheta, k, dt, stream);
    });
}

int bs_lanczos(bs_ctx *c, const bs_lanczos_opts *o, const void *pivot, double *evals, double *evecs,
               bs_lanczos_report *rep)
{
    return guarded(c, [&]() -> int {
        if (!o) { c->err = "null options"; return BS_EINVAL; }
        int rc = check_apply(c, o->k, o->dtype);
        if (rc) return rc;
        if (o->niter < 1 || o->nkeep < 1 || o->nkeep > 64 || !pivot || !evals) {
            c->err = "lanczos: need niter >= 1, 1 <= nkeep <= 64, a pivot and an evals array";
            return BS_EINVAL;
        }
        if (o->nthick < 0 || o->max_restarts < 0 || !(o->tol >= 0.0) ||
            (o->nthick > 0 && (o->nthick % o->k || o->nthick / o->k + 1 >= o->niter))) {
            c->err = "lanczos: thick restart needs nthick a multiple of k with nthick / k + 1 < niter, "
                     "max_restarts >= 0, tol >= 0";
            return BS_EINVAL;
        }
        if (o->targeted && (!o->refine || o->nkeep > 8 || !std::isfinite(o->target))) {
            c->err = "lanczos: a targeted run needs refine = 1, nkeep <= 8 and a finite target";
            return BS_EINVAL;
        }
        if (rep) std::memset(rep, 0, sizeof(*rep));
        return run_lanczos(c, *o, pivot, evals, evecs, rep);
    });
}

int bs_strength(bs_ctx *c, const bs_lanczos_opts *o, const void *pivot, int n_out, double *energies,
                double *strengths, bs_lanczos_report *rep)
{
    return guarded(c, [&]() -> int {
        if (!o) { c->err = "null options"; return BS_EINVAL; }
        int rc = check_apply(c, o->k, o->dtype);
        if (rc) return rc;
        if (o->niter < 1 || n_out < 1 || !pivot || !energies || !strengths || o->nthick != 0) {
            c->err = "strength: need niter >= 1, n_out >= 1, a pivot, output arrays and no thick restart";
            return BS_EINVAL;
        }
        bs_lanczos_opts so = *o;
        so.targeted = 0;
        so.refine = 0;
        so.nkeep = 1;
        so.max_restarts = 0;
        double e0 = 0.0;
        StrengthReq req{n_out, energies, strengths};
        if (rep) std::memset(rep, 0, sizeof(*rep));
        return run_lanczos(c, so, pivot, &e0, nullptr, rep, &req);
    });
}

int bs_density(bs_ctx *c, const double *F, const double *X, int k, double *rho, void *stream)
{
    return guarded(c, [&]() -> int {
        int rc = check_apply(c, k, BS_F64);
        if (rc) return rc;
        if (c->basis.trunc) { c->err = "density: not available on a W-truncated basis"; return BS_EINVAL; }
        if (!F || !X || !rho) { c->err = "density: null pointer"; return BS_EINVAL; }
        return run_density(c, F, X, k, rho, stream);
    });
}

int bs_gather_ceiling(bs_ctx *c, int where, int k, int rows, double *gflops, void *stream)
{
    return guarded(c, [&]() -> int {
        if (c->device < 0) { c->err = "context has no device"; return BS_EINVAL; }
        if ((where != 0 && where != 1) || (k != 4 && k != 8) || (rows != 1 && rows != 2 && rows != 4) || !gflops) {
            c->err = "gather ceiling: where 0 or 1, k 4 or 8, rows 1, 2 or 4, and an output";
            return BS_EINVAL;
        }
        return run_gather_ceiling(c->device, where, k, rows, gflops, stream, c->err);
    });
}

int bs_debug_wait_expiry(bs_ctx *c, int limit, void *stream)
{
    return guarded(c, [&]() -> int {
        int rc = check_apply(c, 1, BS_F64);
        if (rc) return rc;
        if (limit < 1 || limit > (int)tma_wait_limit()) {
            c->err = "wait expiry: limit must be in 1 .. the kernels' own limit";
            return BS_EINVAL;
        }
        return run_wait_expiry(c->device, (uint32_t)limit, c->dev.err, stream, c->err);
    });
}

int bs_set_kernel(bs_ctx *c, int mode)
{
    return guarded(c, [&]() -> int {
        if (mode < 0 || mode > BS_KERNEL_MODES) { c->err = "unknown kernel mode"; return BS_EINVAL; }
        c->hx_mode = mode;
        return BS_OK;
    });
}

int bs_autotune(bs_ctx *c, int k, bs_dtype dt, void *stream, int *mode_out, float *ms_out)
{
    return guarded(c, [&]() -> int {
        int rc = check_apply(c, k, dt);
        if (rc) return rc;
        const size_t bytes = (size_t)c->basis.dim * (size_t)k * (dt == BS_F64 ? 8 : 4);
        void *x = nullptr, *y = nullptr;
        cudaError_t e;
        if ((e = cudaMalloc(&x, bytes)) != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
        if ((e = cudaMalloc(&y, bytes)) != cudaSuccess) { cudaFree(x); return cuda_fail(c, e, "cudaMalloc"); }
        cudaStream_t s = (cudaStream_t)stream;
        cudaMemsetAsync(x, 0, bytes, s);
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        const int saved = c->hx_mode;
        int best = 1;
        float best_ms = 1e30f;
        for (int mode = 1; mode <= BS_KERNEL_MODES && rc == BS_OK; ++mode) {
            c->hx_mode = mode;
            rc = launch_hx(c, x, y, k, dt, stream, c->err);       // warm-up
            if (rc) break;
            cudaEventRecord(a, s);
            for (int r = 0; r < 3 && rc == BS_OK; ++r) rc = launch_hx(c, x, y, k, dt, stream, c->err);
            cudaEventRecord(b, s);
            if ((e = cudaEventSynchronize(b)) != cudaSuccess) { rc = cuda_fail(c, e, "autotune"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            ms /= 3.0f;
            if (ms_out) ms_out[mode - 1] = ms;
            if (ms < best_ms) { best_ms = ms; best = mode; }
        }
        c->hx_mode = saved;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        cudaFree(x);
        cudaFree(y);
        if (rc) return rc;
        c->tuned[dt == BS_F64 ? 0 : 1][k == 1 ? 0 : k == 2 ? 1 : k == 4 ? 2 : 3] = best;
        if (mode_out) *mode_out = best;
        return BS_OK;
    });
}

int bs_set_tuned(bs_ctx *c, int k, bs_dtype dt, int mode)
{
    return guarded(c, [&]() -> int {
        if ((k != 1 && k != 2 && k != 4 && k != 8) || (dt != BS_F64 && dt != BS_F32) || mode < 1 ||
            mode > BS_KERNEL_MODES) {
            c->err = "set_tuned: need k in {1, 2, 4, 8}, a known dtype and a mode in 1..BS_KERNEL_MODES";
            return BS_EINVAL;
        }
        c->tuned[dt == BS_F64 ? 0 : 1][k == 1 ? 0 : k == 2 ? 1 : k == 4 ? 2 : 3] = mode;
        return BS_OK;
    });
}

int bs_sync_status(bs_ctx *c, void *stream)
{
    return guarded(c, [&]() -> int {
        if (c->device < 0 || !c->dev.err) return BS_OK;
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
        int flag = 0;
        if ((e = cudaMemcpy(&flag, c->dev.err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy");
        if (flag != 0) {
            int zero = 0;
            cudaMemcpy(c->dev.err, &zero, sizeof(int), cudaMemcpyHostToDevice);
            c->err = "a device-side wait ran out of its iteration budget";
            return flag;
        }
        return BS_OK;
    });
}

int bs_time_kernel(bs_ctx *c, int n)
{
    return guarded(c, [&]() -> int {
        if (n < 0 || n > BS_TIME_MAX) { c->err = "bs_time_kernel: n out of range"; return BS_EINVAL; }
        if (c->device < 0) { c->err = "bs_time_kernel: host-only context"; return BS_EINVAL; }
        cudaError_t e = cudaSetDevice(c->device);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
        for (cudaEvent_t ev : c->tev) cudaEventDestroy(ev);
        c->tev.clear();
        c->tev_used = 0;
        for (int i = 0; i < 2 * n; ++i) {
            cudaEvent_t ev;
            if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(c, e, "cudaEventCreate");
            c->tev.push_back(ev);
        }
        return BS_OK;
    });
}

int bs_kernel_times(bs_ctx *c, float *ms, int *n)
{
    return guarded(c, [&]() -> int {
        if (!n) { c->err = "bs_kernel_times: null count"; return BS_EINVAL; }
        const int m = c->tev_used;
        *n = m;
        for (int i = 0; i < m; ++i) {
            cudaError_t e = cudaEventSynchronize(c->tev[2 * i + 1]);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize");
            float t = 0.f;
            if ((e = cudaEventElapsedTime(&t, c->tev[2 * i], c->tev[2 * i + 1])) != cudaSuccess)
                return cuda_fail(c, e, "cudaEventElapsedTime");
            if (ms) ms[i] = t;
        }
        return BS_OK;
    });
}

// Host copies of the built tables, by name, for tests that check the host
// builders without a GPU.  With out == NULL only *nbytes is set.
int bs_debug_table(bs_ctx *c, const char *name, void *out, int64_t *nbytes)
{
    return guarded(c, [&]() -> int {
        if (!c->have_int) { c->err = "no interaction"; return BS_ENOINT; }
        const Tables &T = c->tab;
        const Interaction &I = c->inter;
        std::vector<int64_t> tmp;
        const void *src = nullptr;
        size_t n = 0;
        std::string s(name ? name : "");
        auto use = [&](const void *p, size_t b) { src = p; n = b; };
        if (s == "pp_ptr") use(T.pp.ptr.data(), T.pp.ptr.size() * 8);
        else if (s == "pp_src") use(T.pp.src.data(), T.pp.src.size() * 4);
        else if (s == "pp_coef") use(T.pp.coef.data(), T.pp.coef.size() * 8);
        else if (s == "nn_ptr") use(T.nn.ptr.data(), T.nn.ptr.size() * 8);
        else if (s == "nn_src") use(T.nn.src.data(), T.nn.src.size() * 4);
        else if (s == "nn_coef") use(T.nn.coef.data(), T.nn.coef.size() * 8);
        else if (s == "ppx_ptr") use(T.ppx.ptr.data(), T.ppx.ptr.size() * 8);
        else if (s == "ppx_src") use(T.ppx.src.data(), T.ppx.src.size() * 4);
        else if (s == "ppx_coef") use(T.ppx.coef.data(), T.ppx.coef.size() * 8);
        else if (s == "nnx_ptr") use(T.nnx.ptr.data(), T.nnx.ptr.size() * 8);
        else if (s == "nnx_src") use(T.nnx.src.data(), T.nnx.src.size() * 4);
        else if (s == "nnx_coef") use(T.nnx.coef.data(), T.nnx.coef.size() * 8);
        else if (s == "p1_ptr") use(T.p1.ptr.data(), T.p1.ptr.size() * 8);
        else if (s == "p1_ent") use(T.p1.ent.data(), T.p1.ent.size() * 4);
        else if (s == "n1_ptr") use(T.n1.ptr.data(), T.n1.ptr.size() * 8);
        else if (s == "n1_ent") use(T.n1.ent.data(), T.n1.ent.size() * 4);
        else if (s == "wpn") use(I.Wpn.data(), I.Wpn.size() * 8);
        else if (s == "n1e_col") use(T.n1e.col.data(), T.n1e.col.size() * 4);
        else if (s == "n1e_len") use(T.n1e.len.data(), T.n1e.len.size() * 4);
        else if (s == "n1e_soff") use(T.n1e.soff.data(), T.n1e.soff.size() * 8);
        else if (s == "n1e_ent") use(T.n1e.ent.data(), T.n1e.ent.size() * 4);
        else if (s == "nne_col") use(T.nne.col.data(), T.nne.col.size() * 4);
        else if (s == "nne_len") use(T.nne.len.data(), T.nne.len.size() * 4);
        else if (s == "nne_soff") use(T.nne.soff.data(), T.nne.soff.size() * 8);
        else if (s == "nne_src") use(T.nne.src.data(), T.nne.src.size() * 4);
        else if (s == "nne_coef") use(T.nne.coef.data(), T.nne.coef.size() * 8);
        else if (s == "pe_perm") use(T.pe.perm.data(), T.pe.perm.size() * 4);
        else if (s == "pe_sinfo") use(T.pe.sinfo.data(), T.pe.sinfo.size() * 4);
        else if (s == "pe_ent") use(T.pe.ent.data(), T.pe.ent.size() * 4);
        else if (s == "pe_nn_src") use(T.pe.nn_src.data(), T.pe.nn_src.size() * 4);
        else if (s == "pe_nn_coef") use(T.pe.nn_coef.data(), T.pe.nn_coef.size() * 8);
        else if (s == "pe_nn_sinfo") use(T.pe.nn_sinfo.data(), T.pe.nn_sinfo.size() * 4);
        else if (s == "ww") use(T.ww.data(), T.ww.size() * 8);
        else if (s == "pe_base") {   // per neutron sector: perm_off, nn_ent, nn_sinfo; then per class: ent, sinfo
            for (size_t k = 0; k < T.pe.perm_off.size(); ++k) { tmp.push_back(T.pe.perm_off[k]); tmp.push_back(T.pe.sec_nn_ent[k]); tmp.push_back(T.pe.sec_nn_sinfo[k]); }
            for (size_t k = 0; k < T.pe.cls_ent.size(); ++k) { tmp.push_back(T.pe.cls_ent[k]); tmp.push_back(T.pe.cls_sinfo[k]); }
            use(tmp.data(), tmp.size() * 8);
        } else if (s == "ww_off") use(T.ww_off.data(), T.ww_off.size() * 8);
        else if (s == "core_units") use(T.cunits.data(), T.cunits.size() * sizeof(CoreUnit));
        else if (s == "core_src") use(T.csrc.data(), T.csrc.size() * sizeof(CoreSrc));
        else if (s == "wc") use(T.wc.data(), T.wc.size() * 8);
        else if (s == "core_ent") use(T.pe.core_ent.data(), T.pe.core_ent.size() * 4);
        else if (s == "pp_units") use(T.ppunits.data(), T.ppunits.size() * sizeof(PPUnit));
        else if (s == "pps_row") use(T.pps_row.data(), T.pps_row.size() * 4);
        else if (s == "pps_w") use(T.pps_w.data(), T.pps_w.size() * 8);
        else if (s == "pdiag") use(T.pdiag.data(), T.pdiag.size() * 8);
        else if (s == "n1e_base") {
            for (size_t k = 0; k < T.n1e_col.size(); ++k) { tmp.push_back(T.n1e_col[k]); tmp.push_back(T.n1e_slice[k]); }
            use(tmp.data(), tmp.size() * 8);
        } else if (s == "nne_base") {
            for (size_t k = 0; k < T.nne_col.size(); ++k) { tmp.push_back(T.nne_col[k]); tmp.push_back(T.nne_slice[k]); }
            use(tmp.data(), tmp.size() * 8);
        }
        else if (s == "p1_cls" || s == "n1_cls") {
            const OneBodyJumps &J = s[0] == 'p' ? T.p1 : T.n1;
            for (const OneBodyClass &k : J.cls) { tmp.push_back(k.s_src); tmp.push_back(k.s_dst); tmp.push_back(k.group); tmp.push_back(k.ptr_off); }
            use(tmp.data(), tmp.size() * 8);
        } else if (s == "links") {
            for (const PnLink &L : T.links) {
                tmp.push_back(L.dst_block); tmp.push_back(L.src_block); tmp.push_back(L.pcls);
                tmp.push_back(L.ncls); tmp.push_back(L.w_off); tmp.push_back(L.nb);
            }
            use(tmp.data(), tmp.size() * 8);
        } else if (s == "ops") {   // per group: dtwom, dpar, conj group, wpn offset, n ops; then op lists
            for (size_t g = 0; g < I.ops.ops.size(); ++g) {
                tmp.push_back(I.ops.g_dtwom[g]); tmp.push_back(I.ops.g_dpar[g]); tmp.push_back(I.conj_group[g]);
                tmp.push_back(I.wpn_off[g]); tmp.push_back((int64_t)I.ops.ops[g].size());
            }
            use(tmp.data(), tmp.size() * 8);
        } else if (s == "op_lists") {
            for (const auto &g : I.ops.ops) for (int op : g) tmp.push_back(op);
            use(tmp.data(), tmp.size() * 8);
        } else if (s == "p_sec_w" || s == "n_sec_w") {   // W of every sector
            for (const Sector &q : c->basis.sp[s[0] == 'p' ? 0 : 1].sec) tmp.push_back(q.W);
            use(tmp.data(), tmp.size() * 8);
        } else if (s == "llinks") {
            for (const LikeLink &L : T.llinks) {
                tmp.push_back(L.dst_block); tmp.push_back(L.src_block); tmp.push_back(L.species); tmp.push_back(L.ptr_off);
            }
            use(tmp.data(), tmp.size() * 8);
        } else if (s == "stats") {
            tmp = {T.n_pp, T.n_nn, T.n_p1, T.n_n1, (int64_t)T.links.size(), (int64_t)T.ops_per_vector, (int64_t)c->dev.ntasks,
                   (int64_t)T.wsign, (int64_t)T.ops_pn, (int64_t)T.ops_pp, (int64_t)T.ops_nn,
                   (int64_t)T.gathers_pn};
            use(tmp.data(), tmp.size() * 8);
        } else {
            c->err = "unknown table " + s;
            return BS_EINVAL;
        }
        if (nbytes) *nbytes = (int64_t)n;
        if (out && n) std::memcpy(out, src, n);
        return BS_OK;
    });
}

}  // extern "C"
