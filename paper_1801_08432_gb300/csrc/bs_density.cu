// One-body transition densities of one basis (Sec. "One-body density
// matrices and occupations", the M-scheme matrix elements that the reduced
// densities <J_f||(a+ b)_K||J_i> are built from):
//
//     rho_t(i, k)[f][j] = <F_f| a+_i a_k |X_j>,   t = protons, neutrons,
//
// for the k columns of two FP64 blocks on the same (2M, parity) basis, so
// 2m_i = 2m_k and the operator keeps every sector: its jumps are the
// one-body jump class (s -> s) of each sector, already on the device for the
// pn term.  One warp takes one destination SD of one species in one block;
// per incoming jump (source SD, operator, sign) its lanes run over the other
// species' SDs of the block, accumulate the k x k products F[dst] X[src] in
// FP64, reduce them across the warp and add them to the operator's k x k
// slot (FP64 atomics: the summation order, and so the last bits, may vary
// between runs).
#include <cuda_runtime.h>

#include <vector>

#include "bs_internal.h"

namespace bs {
namespace {

struct DensItem {
    int64_t off;   // first basis index of the block
    int64_t ptr;   // index into the species' jump pointers: this SD's entries
    int nP, nN;    // block shape (proton rows x neutron columns)
    int r;         // destination SD, local in its sector
    int spc;       // 0: proton SD (lanes over neutron columns), 1: neutron SD (lanes over proton rows)
};

template <int K>
__global__ void __launch_bounds__(128) density_kernel(const DensItem *__restrict__ items, int nitems,
                                                      const int64_t *__restrict__ pptr, const uint32_t *__restrict__ pent,
                                                      const int64_t *__restrict__ nptr, const uint32_t *__restrict__ nent,
                                                      const int *__restrict__ op_of_local, const double *__restrict__ F,
                                                      const double *__restrict__ X, double *__restrict__ rho, int nops)
{
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int it = warp; it < nitems; it += nwarps) {
        const DensItem d = items[it];
        const int64_t *ptr = d.spc ? nptr : pptr;
        const uint32_t *ent = d.spc ? nent : pent;
        const int n_other = d.spc ? d.nP : d.nN;
        const int64_t e1 = ptr[d.ptr + 1];
        for (int64_t e = ptr[d.ptr]; e < e1; ++e) {
            const uint32_t pk = ent[e];
            const int64_t src = (int64_t)(pk & 0xFFFFu);
            const int op = op_of_local[(pk >> 16) & 0x7FFFu];
            double acc[K][K];
#pragma unroll
            for (int f = 0; f < K; ++f)
#pragma unroll
                for (int j = 0; j < K; ++j) acc[f][j] = 0.0;
            for (int q = lane; q < n_other; q += 32) {
                const int64_t a_dst = d.spc ? d.off + (int64_t)q * d.nN + d.r : d.off + (int64_t)d.r * d.nN + q;
                const int64_t a_src = d.spc ? d.off + (int64_t)q * d.nN + src : d.off + src * d.nN + q;
                double fv[K], xv[K];
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    fv[j] = F[a_dst * K + j];
                    xv[j] = X[a_src * K + j];
                }
#pragma unroll
                for (int f = 0; f < K; ++f)
#pragma unroll
                    for (int j = 0; j < K; ++j) acc[f][j] = fma(fv[f], xv[j], acc[f][j]);
            }
#pragma unroll
            for (int f = 0; f < K; ++f)
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    double v = acc[f][j];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    acc[f][j] = v;
                }
            if (lane == 0) {
                const double sg = (pk >> 31) ? -1.0 : 1.0;
                double *out = rho + ((int64_t)d.spc * nops + op) * K * K;
#pragma unroll
                for (int f = 0; f < K; ++f)
#pragma unroll
                    for (int j = 0; j < K; ++j) atomicAdd(out + f * K + j, sg * acc[f][j]);
            }
        }
    }
}

}  // namespace

int run_density(bs_ctx *c, const double *F, const double *X, int k, double *rho_host, void *stream)
{
    const Basis &B = c->basis;
    const Tables &T = c->tab;
    const Interaction &I = c->inter;
    const Device &D = c->dev;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return BS_ECUDA; }
    cudaStream_t s = (cudaStream_t)stream;
    const int ns = (int)B.st.size();
    const int nops = ns * ns;
    const size_t nrho = (size_t)2 * nops * k * k;
    // operators that keep (2m, parity): their group and local numbering
    int g0 = -1;
    for (size_t g = 0; g < I.ops.g_dtwom.size(); ++g)
        if (I.ops.g_dtwom[g] == 0 && I.ops.g_dpar[g] == 0) g0 = (int)g;
    std::vector<double> zero(nrho, 0.0);
    if (g0 < 0) {
        std::copy(zero.begin(), zero.end(), rho_host);
        return BS_OK;
    }
    const std::vector<int> &opmap = I.ops.ops[(size_t)g0];
    // the (s -> s) jump class of every sector, per species
    std::vector<int64_t> pcls(B.sp[0].sec.size(), -1), ncls(B.sp[1].sec.size(), -1);
    for (const OneBodyClass &cl : T.p1.cls)
        if (cl.s_src == cl.s_dst) pcls[(size_t)cl.s_dst] = cl.ptr_off;
    for (const OneBodyClass &cl : T.n1.cls)
        if (cl.s_src == cl.s_dst) ncls[(size_t)cl.s_dst] = cl.ptr_off;
    std::vector<DensItem> items;
    for (const Block &b : B.blocks) {
        if (pcls[(size_t)b.ps] >= 0)
            for (int64_t r = 0; r < b.nP; ++r)
                items.push_back(DensItem{b.off, pcls[(size_t)b.ps] + r, (int)b.nP, (int)b.nN, (int)r, 0});
        if (ncls[(size_t)b.ns] >= 0)
            for (int64_t r = 0; r < b.nN; ++r)
                items.push_back(DensItem{b.off, ncls[(size_t)b.ns] + r, (int)b.nP, (int)b.nN, (int)r, 1});
    }
    DensItem *d_items = nullptr;
    int *d_op = nullptr;
    double *d_rho = nullptr;
    auto fail = [&](cudaError_t err, const char *what) {
        cudaFree(d_items);
        cudaFree(d_op);
        cudaFree(d_rho);
        c->err = std::string("density: ") + what + ": " + cudaGetErrorString(err);
        return err == cudaErrorMemoryAllocation ? BS_ENOMEM : BS_ECUDA;
    };
    if ((e = cudaMalloc(&d_items, std::max<size_t>(items.size(), 1) * sizeof(DensItem))) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&d_op, std::max<size_t>(opmap.size(), 1) * sizeof(int))) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&d_rho, nrho * sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc");
    cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(DensItem), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_op, opmap.data(), opmap.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(d_rho, 0, nrho * sizeof(double), s);
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int nitems = (int)items.size();
    const int grid = std::max(1, std::min(8 * nsm, (nitems + 3) / 4));   // 4 warps per CTA
    switch (k) {
    case 1: density_kernel<1><<<grid, 128, 0, s>>>(d_items, nitems, D.p1_ptr, D.p1_ent, D.n1_ptr, D.n1_ent, d_op, F, X, d_rho, nops); break;
    case 2: density_kernel<2><<<grid, 128, 0, s>>>(d_items, nitems, D.p1_ptr, D.p1_ent, D.n1_ptr, D.n1_ent, d_op, F, X, d_rho, nops); break;
    case 4: density_kernel<4><<<grid, 128, 0, s>>>(d_items, nitems, D.p1_ptr, D.p1_ent, D.n1_ptr, D.n1_ent, d_op, F, X, d_rho, nops); break;
    default: density_kernel<8><<<grid, 128, 0, s>>>(d_items, nitems, D.p1_ptr, D.p1_ent, D.n1_ptr, D.n1_ent, d_op, F, X, d_rho, nops); break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "launch");
    cudaMemcpyAsync(rho_host, d_rho, nrho * sizeof(double), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "run");
    cudaFree(d_items);
    cudaFree(d_op);
    cudaFree(d_rho);
    return BS_OK;
}

}  // namespace bs
