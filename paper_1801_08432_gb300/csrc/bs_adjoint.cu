// Adjoint of y = H(theta) x (sm_103a).
//
// H is real symmetric, so the input adjoint is gx = H gy (the forward
// kernels).  H is linear in theta = (SPEs, TBMEs) through the decoupling of
// Eq. (hamdef) / Eq. (xpndef), so
//   d/dtheta_t (gy . H x) = sum over jumps of (dc_jump / dtheta_t) gy[dst] . x[src].
// The kernels here reduce gy . x over the jumps into transition densities:
//   pp: one value per pp jump (destination SD row . source SD row),
//   nn: one value per nn jump (summed over the proton rows of the block),
//   pn: one value per (proton operator a, neutron operator b) of a W_pn
//       group, summed over all proton jump x neutron jump pairs using (a, b);
// the host then splits pp/nn values into two-body moves and contracts
// everything with dW/dtheta.  Products of FP32 vectors are formed in FP32
// and summed in FP64; pn densities use FP64 atomics (the order of those
// additions, and so the last bits, may differ from run to run).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "bs_internal.h"

namespace bs {

namespace {

template <typename T, int K>
__device__ __forceinline__ double dotk(const T *__restrict__ a, const T *__restrict__ b)
{
    double s = 0.0;
    if constexpr (sizeof(T) == 4) {
        float f = 0.f;   // K <= 8 products of FP32 values
#pragma unroll
        for (int q = 0; q < K; ++q) f = fmaf(a[q], b[q], f);
        s = (double)f;
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) s = fma(a[q], b[q], s);
    }
    return s;
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;   // valid in thread 0
}

// pp: G[e] = gy[row ip'] . x[row ip_e] over the block's columns and k vectors
template <typename T, int K>
__global__ void adj_pp(const RowTask *tasks, const DevBlock *blocks, const int64_t *pp_ptr, const int32_t *pp_src,
                       const T *__restrict__ x, const T *__restrict__ gy, double *__restrict__ G)
{
    __shared__ double red[32];
    const RowTask t = tasks[blockIdx.x];
    const DevBlock D = blocks[t.block];
    const int g = D.p_start + t.row;
    const T *gr = gy + (D.off + (int64_t)t.row * D.nN) * K;
    for (int64_t e = pp_ptr[g]; e < pp_ptr[g + 1]; ++e) {
        const T *xr = x + (D.off + (int64_t)pp_src[e] * D.nN) * K;
        double s = 0.0;
        for (int c = threadIdx.x; c < D.nN; c += blockDim.x) s += dotk<T, K>(gr + (int64_t)c * K, xr + (int64_t)c * K);
        s = block_sum(s, red);
        if (threadIdx.x == 0) G[e] = s;
    }
}

// nn: G[e] = sum over the block's rows ip of gy[ip, jn'] . x[ip, jn_e]; one CTA per (block, column jn')
template <typename T, int K>
__global__ void adj_nn(const DevBlock *blocks, const int *col_block, const int *col_local, const int64_t *nn_ptr,
                       const int32_t *nn_src, const T *__restrict__ x, const T *__restrict__ gy,
                       double *__restrict__ G)
{
    __shared__ double red[32];
    const DevBlock D = blocks[col_block[blockIdx.x]];
    const int jc = col_local[blockIdx.x];
    const int g = D.n_start + jc;
    for (int64_t e = nn_ptr[g]; e < nn_ptr[g + 1]; ++e) {
        const int js = nn_src[e];
        double s = 0.0;
        for (int r = threadIdx.x; r < D.nP; r += blockDim.x) {
            const int64_t base = D.off + (int64_t)r * D.nN;
            s += dotk<T, K>(gy + (base + jc) * K, x + (base + js) * K);
        }
        s = block_sum(s, red);
        if (threadIdx.x == 0) G[e] = s;
    }
}

// pn: rho[w_off + a nb + b] += phi_u sum_{jn'} sum_{v: b_v = b} phi_v gy[ip', jn'] . x_s[ip_u, jn_v]
template <typename T, int K>
__global__ void adj_pn(const RowTask *tasks, const DevBlock *blocks, const DevLink *links, const int64_t *p1_ptr,
                       const uint32_t *p1_ent, const int64_t *n1_ptr, const uint32_t *n1_ent,
                       const T *__restrict__ x, const T *__restrict__ gy, double *__restrict__ rho)
{
    extern __shared__ double acc[];   // [nb]
    const RowTask t = tasks[blockIdx.x];
    const DevBlock D = blocks[t.block];
    const T *gr = gy + (D.off + (int64_t)t.row * D.nN) * K;
    for (int L = D.link_begin; L < D.link_end; ++L) {
        const DevLink lk = links[L];
        const int64_t pb = p1_ptr[lk.p_ptr_off + t.row], pe = p1_ptr[lk.p_ptr_off + t.row + 1];
        if (pb == pe) continue;
        const DevBlock S = blocks[lk.src_block];
        for (int64_t u = pb; u < pe; ++u) {
            for (int b = threadIdx.x; b < lk.nb; b += blockDim.x) acc[b] = 0.0;
            __syncthreads();
            const uint32_t ep = p1_ent[u];
            const T *xr = x + (S.off + (int64_t)(ep & 0xFFFFu) * S.nN) * K;
            for (int c = threadIdx.x; c < D.nN; c += blockDim.x) {
                const T *gc = gr + (int64_t)c * K;
                for (int64_t v = n1_ptr[lk.n_ptr_off + c]; v < n1_ptr[lk.n_ptr_off + c + 1]; ++v) {
                    const uint32_t en = n1_ent[v];
                    const double d = dotk<T, K>(gc, xr + (int64_t)(en & 0xFFFFu) * K);
                    atomicAdd(&acc[(en >> 16) & 0x7FFFu], (en >> 31) ? -d : d);
                }
            }
            __syncthreads();
            const double sp = (ep >> 31) ? -1.0 : 1.0;
            const int64_t row0 = lk.w_off + (int64_t)((ep >> 16) & 0x7FFFu) * lk.nb;
            for (int b = threadIdx.x; b < lk.nb; b += blockDim.x)
                if (acc[b] != 0.0) atomicAdd(&rho[row0 + b], sp * acc[b]);
            __syncthreads();
        }
    }
}

inline int sgn_below(uint64_t m, int s) { return (__builtin_popcountll(m & ((1ULL << s) - 1ULL)) & 1) ? -1 : 1; }

// sign of a+_i a+_j a_l a_k on X (k<l occupied, i<j empty after removal)
int move_sign(uint64_t X, int i, int j, int k, int l)
{
    int s = sgn_below(X, k);
    uint64_t m = X & ~(1ULL << k);
    s *= sgn_below(m, l);
    m &= ~(1ULL << l);
    s *= sgn_below(m, j);
    m |= 1ULL << j;
    s *= sgn_below(m, i);
    return s;
}

// Splits the per-jump overlaps G of one species (destination-CSR like the
// pp/nn lists) into two-body move densities rho2[p*npairs+q] and the
// one-body number densities rho1[s].
void split_like(const Basis &B, const Interaction &I, int spc, const LikeJumps &Lj, const std::vector<double> &G,
                std::vector<double> &rho2, std::vector<double> &rho1)
{
    const Species &S = B.sp[spc];
    const int ns = (int)B.st.size();
    for (int64_t g = 0; g < (int64_t)S.bits.size(); ++g) {
        const uint64_t dst = S.bits[(size_t)g];
        const int64_t s0 = S.sec[(size_t)S.sec_of_sd[(size_t)g]].start;
        for (int64_t e = Lj.ptr[(size_t)g]; e < Lj.ptr[(size_t)g + 1]; ++e) {
            const double v = G[(size_t)e];
            if (v == 0.0) continue;
            const uint64_t src = S.bits[(size_t)(s0 + Lj.src[(size_t)e])];
            const uint64_t diff = src ^ dst;
            const int nd = __builtin_popcountll(diff);
            if (nd == 0) {
                for (int a = 0; a < ns; ++a) {
                    if (!(src >> a & 1)) continue;
                    rho1[a] += v;
                    for (int b = a + 1; b < ns; ++b)
                        if (src >> b & 1) {
                            const int p = I.pair_id[(size_t)a * ns + b];
                            rho2[(size_t)p * I.npairs + p] += v;
                        }
                }
            } else if (nd == 2) {
                const int k = __builtin_ctzll(src & diff), i = __builtin_ctzll(dst & diff);
                for (int x = 0; x < ns; ++x) {
                    if (x == k || !(src >> x & 1)) continue;
                    const int kk = std::min(k, x), ll = std::max(k, x), ii = std::min(i, x), jj = std::max(i, x);
                    const int q = I.pair_id[(size_t)kk * ns + ll], p = I.pair_id[(size_t)ii * ns + jj];
                    rho2[(size_t)p * I.npairs + q] += v * move_sign(src, ii, jj, kk, ll);
                }
            } else if (nd == 4) {
                const uint64_t out = src & diff, in = dst & diff;
                const int k = __builtin_ctzll(out), l = 63 - __builtin_clzll(out);
                const int i = __builtin_ctzll(in), j = 63 - __builtin_clzll(in);
                const int q = I.pair_id[(size_t)k * ns + l], p = I.pair_id[(size_t)i * ns + j];
                rho2[(size_t)p * I.npairs + q] += v * move_sign(src, i, j, k, l);
            }
        }
    }
}

template <typename T, int K>
int launch_adj(bs_ctx *c, const T *x, const T *gy, cudaStream_t s, std::vector<int> &cb, std::vector<int> &cl)
{
    const Device &D = c->dev;
    adj_pp<T, K><<<D.nrtasks, 128, 0, s>>>(D.rtasks, D.blocks, D.pp_ptr, D.pp_src, x, gy, c->adj_gpp);
    if (!cb.empty()) {
        int *dcb = nullptr, *dcl = nullptr;
        cudaMallocAsync((void **)&dcb, cb.size() * sizeof(int), s);
        cudaMallocAsync((void **)&dcl, cl.size() * sizeof(int), s);
        cudaMemcpyAsync(dcb, cb.data(), cb.size() * sizeof(int), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dcl, cl.data(), cl.size() * sizeof(int), cudaMemcpyHostToDevice, s);
        adj_nn<T, K><<<(int)cb.size(), 128, 0, s>>>(D.blocks, dcb, dcl, D.nn_ptr, D.nn_src, x, gy, c->adj_gnn);
        cudaFreeAsync(dcb, s);
        cudaFreeAsync(dcl, s);
    }
    adj_pn<T, K><<<D.nrtasks, 128, (size_t)std::max(1, D.max_nb) * sizeof(double), s>>>(
        D.rtasks, D.blocks, D.links, D.p1_ptr, D.p1_ent, D.n1_ptr, D.n1_ent, x, gy, c->adj_rho);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("adjoint launch: ") + cudaGetErrorString(e);
        return BS_ECUDA;
    }
    return BS_OK;
}

// dWpp/dWpn of every TBME as given (unit interactions through the same decoupling)
int build_derivatives(bs_ctx *c)
{
    const int nt = (int)c->tbme_in.size();
    c->dWpp.assign(nt, {});
    c->dWpn.assign(nt, {});
    std::vector<double> zero(c->spe_in.size(), 0.0);
    for (int t = 0; t < nt; ++t) {
        bs_tbme one = c->tbme_in[(size_t)t];
        one.v = 1.0;
        Interaction U;
        std::string err;
        int rc = build_interaction(c->basis, zero.data(), (int)zero.size(), &one, 1, U, err);
        if (rc) { c->err = err; return rc; }
        for (size_t i = 0; i < U.Wpp.size(); ++i)
            if (U.Wpp[i] != 0.0) c->dWpp[(size_t)t].emplace_back((int64_t)i, U.Wpp[i]);
        for (size_t i = 0; i < U.Wpn.size(); ++i)
            if (U.Wpn[i] != 0.0) c->dWpn[(size_t)t].emplace_back((int64_t)i, U.Wpn[i]);
    }
    c->have_dW = true;
    return BS_OK;
}

}  // namespace

int run_backward(bs_ctx *c, const void *x, const void *gy, void *gx, double *gtheta, int k, bs_dtype dt,
                 void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_hx(c, gy, gx, k, dt, stream, c->err);   // gx = H gy (H symmetric)
    if (rc || !gtheta) return rc;
    if (!c->have_dW && (rc = build_derivatives(c))) return rc;
    const Tables &T = c->tab;
    const Interaction &I = c->inter;
    cudaError_t e;
    if (!c->adj_gpp) {
        if ((e = cudaMalloc(&c->adj_gpp, std::max<size_t>(1, T.pp.src.size()) * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&c->adj_gnn, std::max<size_t>(1, T.nn.src.size()) * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&c->adj_rho, std::max<size_t>(1, I.Wpn.size()) * sizeof(double))) != cudaSuccess) {
            c->err = std::string("adjoint: ") + cudaGetErrorString(e);
            return BS_ENOMEM;
        }
    }
    cudaMemsetAsync(c->adj_gpp, 0, std::max<size_t>(1, T.pp.src.size()) * sizeof(double), s);
    cudaMemsetAsync(c->adj_gnn, 0, std::max<size_t>(1, T.nn.src.size()) * sizeof(double), s);
    cudaMemsetAsync(c->adj_rho, 0, std::max<size_t>(1, I.Wpn.size()) * sizeof(double), s);
    // one CTA per (block, neutron column) for the nn densities
    std::vector<int> cb, cl;
    for (size_t b = 0; b < c->basis.blocks.size(); ++b)
        for (int64_t j = 0; j < c->basis.blocks[b].nN; ++j) { cb.push_back((int)b); cl.push_back((int)j); }
    if (dt == BS_F64) {
        const double *xi = (const double *)x, *gi = (const double *)gy;
        switch (k) {
        case 1: rc = launch_adj<double, 1>(c, xi, gi, s, cb, cl); break;
        case 2: rc = launch_adj<double, 2>(c, xi, gi, s, cb, cl); break;
        case 4: rc = launch_adj<double, 4>(c, xi, gi, s, cb, cl); break;
        default: rc = launch_adj<double, 8>(c, xi, gi, s, cb, cl); break;
        }
    } else {
        const float *xi = (const float *)x, *gi = (const float *)gy;
        switch (k) {
        case 1: rc = launch_adj<float, 1>(c, xi, gi, s, cb, cl); break;
        case 2: rc = launch_adj<float, 2>(c, xi, gi, s, cb, cl); break;
        case 4: rc = launch_adj<float, 4>(c, xi, gi, s, cb, cl); break;
        default: rc = launch_adj<float, 8>(c, xi, gi, s, cb, cl); break;
        }
    }
    if (rc) return rc;
    std::vector<double> gpp(T.pp.src.size()), gnn(T.nn.src.size()), rho(I.Wpn.size());
    cudaMemcpyAsync(gpp.data(), c->adj_gpp, gpp.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(gnn.data(), c->adj_gnn, gnn.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(rho.data(), c->adj_rho, rho.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
        c->err = std::string("adjoint: ") + cudaGetErrorString(e);
        return BS_ECUDA;
    }
    const int ns = (int)c->basis.st.size();
    std::vector<double> rho2((size_t)I.npairs * I.npairs, 0.0), rho1p(ns, 0.0), rho1n(ns, 0.0);
    split_like(c->basis, I, 0, T.pp, gpp, rho2, rho1p);
    split_like(c->basis, I, 1, T.nn, gnn, rho2, rho1n);
    const int no = (int)c->spe_in.size();
    for (int st = 0; st < ns; ++st) gtheta[c->basis.st[(size_t)st].orb] += rho1p[st] + rho1n[st];
    for (size_t t = 0; t < c->tbme_in.size(); ++t) {
        double g = 0.0;
        for (const auto &kv : c->dWpp[t]) g += rho2[(size_t)kv.first] * kv.second;
        for (const auto &kv : c->dWpn[t]) g += rho[(size_t)kv.first] * kv.second;
        gtheta[no + t] += g;
    }
    return BS_OK;
}

}  // namespace bs
