// Fused on-the-fly y = H x over k interleaved vectors (sm_103a).
//
// One CTA owns one destination proton row ip' of one basis block (sector pair
// s' = (s_p', s_n')) and a tile of its neutron columns jn'; every thread owns
// one column (its k values).  The thread sums, in a fixed order,
//   pp: sum over pp jumps into ip' (diagonal and SPE included) c * x[ip, jn']
//   nn: sum over nn jumps into jn' (diagonal and SPE included) c * x[ip', jn]
//   pn: for every source block s linked to s' (a proton one-body class
//       s_p -> s_p' and the matching neutron class s_n -> s_n'),
//       sum over proton jumps (ip, a, phi_p) into ip'
//         phi_p * sum over neutron jumps (jn, b, phi_n) into jn'
//           phi_n * W_pn[a][b] * x_s[ip, jn]
// and writes y once.  This is the paper's factorization (pn = proton one-body
// jump x neutron one-body jump, Sec. on jumps and Table jumps) applied as a
// gather: each y element has one owner, so there are no atomics and the
// result is bit-reproducible.  In a W-truncated basis (Sec. "Truncation of
// the many-body space") a like-particle move may change an SD's W and so its
// sector: those moves come from other blocks through like-particle links,
// and the pn links already join any pair of blocks.
#include <cuda_runtime.h>

#include "bs_internal.h"

namespace bs {

namespace {

template <typename T, int K>
struct Acc {
    T v[K];
};

// load k contiguous values (16-byte vectors where the width allows)
template <typename T, int K>
__device__ __forceinline__ void ldk(const T *__restrict__ p, T (&r)[K])
{
    if constexpr (sizeof(T) * K >= 16) {
        constexpr int W = 16 / sizeof(T);
#pragma unroll
        for (int c = 0; c < K; c += W) {
            if constexpr (sizeof(T) == 4) {
                float4 q = __ldg(reinterpret_cast<const float4 *>(p + c));
                r[c] = q.x; r[c + 1] = q.y; r[c + 2] = q.z; r[c + 3] = q.w;
            } else {
                double2 q = __ldg(reinterpret_cast<const double2 *>(p + c));
                r[c] = q.x; r[c + 1] = q.y;
            }
        }
    } else if constexpr (sizeof(T) == 4 && K == 2) {
        float2 q = __ldg(reinterpret_cast<const float2 *>(p));
        r[0] = q.x; r[1] = q.y;
    } else {
#pragma unroll
        for (int c = 0; c < K; ++c) r[c] = __ldg(p + c);
    }
}

template <typename T, int K>
__device__ __forceinline__ void stk(T *__restrict__ p, const T (&r)[K])
{
    if constexpr (sizeof(T) * K >= 16) {
        constexpr int W = 16 / sizeof(T);
#pragma unroll
        for (int c = 0; c < K; c += W) {
            if constexpr (sizeof(T) == 4) *reinterpret_cast<float4 *>(p + c) = make_float4(r[c], r[c + 1], r[c + 2], r[c + 3]);
            else *reinterpret_cast<double2 *>(p + c) = make_double2(r[c], r[c + 1]);
        }
    } else if constexpr (sizeof(T) == 4 && K == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(r[0], r[1]);
    } else {
#pragma unroll
        for (int c = 0; c < K; ++c) p[c] = r[c];
    }
}

struct HxArgs {
    const DevTask *tasks;
    const DevBlock *blocks;
    const DevLink *links;
    const int64_t *pp_ptr, *nn_ptr, *p1_ptr, *n1_ptr;
    const int32_t *pp_src, *nn_src;
    const uint32_t *p1_ent, *n1_ent;
    const DevLLink *llinks;
    const int64_t *ppx_ptr, *nnx_ptr;
    const int32_t *ppx_src, *nnx_src;
};

template <typename T, int K>
__global__ void __launch_bounds__(128) hx_fused_kernel(HxArgs A, const T *__restrict__ pp_coef,
                                                       const T *__restrict__ nn_coef, const T *__restrict__ wpn,
                                                       const T *__restrict__ ppx_coef, const T *__restrict__ nnx_coef,
                                                       const T *__restrict__ x, T *__restrict__ y)
{
    const DevTask t = A.tasks[blockIdx.x];
    const DevBlock D = A.blocks[t.block];
    const int col = t.col0 + (int)threadIdx.x;
    if (col >= D.nN) return;
    T acc[K];
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = T(0);
    T xv[K];

    // pp (same block): rows ip of x, column col
    {
        const int g = D.p_start + t.row;
        const int64_t e1 = A.pp_ptr[g + 1];
        const T *xc = x + (D.off + col) * K;
        for (int64_t e = A.pp_ptr[g]; e < e1; ++e) {
            const T c = pp_coef[e];
            ldk<T, K>(xc + (int64_t)A.pp_src[e] * D.nN * K, xv);
#pragma unroll
            for (int q = 0; q < K; ++q) acc[q] = fma(c, xv[q], acc[q]);
        }
    }
    // nn (same block): row ip', columns jn
    {
        const int g = D.n_start + col;
        const int64_t e1 = A.nn_ptr[g + 1];
        const T *xr = x + (D.off + (int64_t)t.row * D.nN) * K;
        for (int64_t e = A.nn_ptr[g]; e < e1; ++e) {
            const T c = nn_coef[e];
            ldk<T, K>(xr + (int64_t)A.nn_src[e] * K, xv);
#pragma unroll
            for (int q = 0; q < K; ++q) acc[q] = fma(c, xv[q], acc[q]);
        }
    }
    // like-particle moves from other blocks (W-truncated bases): pp moves from
    // the block of another proton sector with this neutron sector (same
    // column), nn moves from the block of another neutron sector with this
    // proton sector (same row)
    for (int L = D.llink_begin; L < D.llink_end; ++L) {
        const DevLLink lk = A.llinks[L];
        const DevBlock S = A.blocks[lk.src_block];
        if (lk.species == 0) {
            const int64_t e1 = A.ppx_ptr[lk.ptr_off + t.row + 1];
            const T *xc = x + (S.off + col) * K;
            for (int64_t e = A.ppx_ptr[lk.ptr_off + t.row]; e < e1; ++e) {
                const T c = ppx_coef[e];
                ldk<T, K>(xc + (int64_t)A.ppx_src[e] * S.nN * K, xv);
#pragma unroll
                for (int q = 0; q < K; ++q) acc[q] = fma(c, xv[q], acc[q]);
            }
        } else {
            const int64_t e1 = A.nnx_ptr[lk.ptr_off + col + 1];
            const T *xr = x + (S.off + (int64_t)t.row * S.nN) * K;
            for (int64_t e = A.nnx_ptr[lk.ptr_off + col]; e < e1; ++e) {
                const T c = nnx_coef[e];
                ldk<T, K>(xr + (int64_t)A.nnx_src[e] * K, xv);
#pragma unroll
                for (int q = 0; q < K; ++q) acc[q] = fma(c, xv[q], acc[q]);
            }
        }
    }
    // pn: proton one-body jump x neutron one-body jump, per linked source block
    for (int L = D.link_begin; L < D.link_end; ++L) {
        const DevLink lk = A.links[L];
        const int64_t pb = A.p1_ptr[lk.p_ptr_off + t.row], pe = A.p1_ptr[lk.p_ptr_off + t.row + 1];
        if (pb == pe) continue;
        const int64_t nb0 = A.n1_ptr[lk.n_ptr_off + col], ne0 = A.n1_ptr[lk.n_ptr_off + col + 1];
        if (nb0 == ne0) continue;
        const DevBlock S = A.blocks[lk.src_block];
        const T *W = wpn + lk.w_off;
        for (int64_t u = pb; u < pe; ++u) {
            const uint32_t ep = A.p1_ent[u];
            const T *xr = x + (S.off + (int64_t)(ep & 0xFFFFu) * S.nN) * K;
            const T *Wa = W + (int64_t)((ep >> 16) & 0x7FFFu) * lk.nb;
            T part[K];
#pragma unroll
            for (int q = 0; q < K; ++q) part[q] = T(0);
            for (int64_t v = nb0; v < ne0; ++v) {
                const uint32_t en = A.n1_ent[v];
                T w = __ldg(Wa + ((en >> 16) & 0x7FFFu));
                if (en >> 31) w = -w;
                ldk<T, K>(xr + (int64_t)(en & 0xFFFFu) * K, xv);
#pragma unroll
                for (int q = 0; q < K; ++q) part[q] = fma(w, xv[q], part[q]);
            }
            if (ep >> 31) {
#pragma unroll
                for (int q = 0; q < K; ++q) acc[q] -= part[q];
            } else {
#pragma unroll
                for (int q = 0; q < K; ++q) acc[q] += part[q];
            }
        }
    }
    stk<T, K>(y + (D.off + (int64_t)t.row * D.nN + col) * K, acc);
}

template <typename T, int K>
cudaError_t launch(const Device &Dv, const DevCoefs<T> &C, const T *x, T *y, cudaStream_t s)
{
    HxArgs A{Dv.tasks, Dv.blocks, Dv.links, Dv.pp_ptr, Dv.nn_ptr, Dv.p1_ptr, Dv.n1_ptr,
             Dv.pp_src, Dv.nn_src, Dv.p1_ent, Dv.n1_ent, Dv.llinks, Dv.ppx_ptr, Dv.nnx_ptr, Dv.ppx_src, Dv.nnx_src};
    hx_fused_kernel<T, K><<<Dv.ntasks, Dv.tile, 0, s>>>(A, C.pp_coef, C.nn_coef, C.wpn, C.ppx_coef, C.nnx_coef, x, y);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_hx_row(const bs_ctx *c, const void *x, void *y, int k, bs_dtype dt, cudaStream_t s, int variant,
                          bool &used);

cudaError_t launch_hx_pipe(const bs_ctx *c, const void *x, void *y, int k, bs_dtype dt, cudaStream_t s, int v,
                           bool &used);
cudaError_t launch_hx_core(const bs_ctx *c, const void *x, void *y, int k, bs_dtype dt, cudaStream_t s, int v,
                           bool &used, cudaEvent_t t0, cudaEvent_t t1);

static int kslot(int k)
{
    return k == 1 ? 0 : k == 2 ? 1 : k == 4 ? 2 : 3;
}

// Kernel choice: mode 1 = tiled kernel; mode 2 + v = row kernel variant v;
// mode 2 + R + v = pipelined kernel variant v (R = number of row variants);
// mode 0 = the variant the autotuner picked for (k, dtype), else the first
// pipelined variant, else the first row variant.  A row or pipelined variant
// that does not fit the basis falls back to the tiled kernel.
int launch_hx(const bs_ctx *c, const void *x, void *y, int k, bs_dtype dt, void *stream, std::string &err)
{
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(c->device);
    bool used = false;
    int mode = c->hx_mode;
    // bs_time_kernel: events around the dominant kernel of this product
    const bool timing = c->tev_used < (int)c->tev.size() / 2;
    cudaEvent_t t0 = timing ? c->tev[2 * (size_t)c->tev_used] : nullptr;
    cudaEvent_t t1 = timing ? c->tev[2 * (size_t)c->tev_used + 1] : nullptr;
    bool core_used = false;
    if (timing && e == cudaSuccess) e = cudaEventRecord(t0, s);
    const int R = row_variants();
    if (mode == 0) mode = c->tuned[dt == BS_F64 ? 0 : 1][kslot(k)];
    if (mode == 0 && e == cudaSuccess) {
        // not tuned: the core-grouped path where it applies, else the first
        // pipelined variant, else the first row variant
        e = launch_hx_core(c, x, y, k, dt, s, 2, used, t0, t1);
        core_used = used;
        if (e == cudaSuccess && !used) e = launch_hx_pipe(c, x, y, k, dt, s, 0, used);
        if (!used) mode = 2;
    }
    const int P = pipe_variants();
    if (e == cudaSuccess && !used && mode >= 2 + R + P) {
        e = launch_hx_core(c, x, y, k, dt, s, mode - 2 - R - P, used, t0, t1);
        core_used = used;
    }
    if (e == cudaSuccess && !used && mode >= 2 + R && mode < 2 + R + P)
        e = launch_hx_pipe(c, x, y, k, dt, s, mode - 2 - R, used);
    if (e == cudaSuccess && !used && mode >= 2 && mode < 2 + R) e = launch_hx_row(c, x, y, k, dt, s, mode - 2, used);
    if (e == cudaSuccess && !used) {
        if (dt == BS_F64) {
            const double *xi = (const double *)x;
            double *yo = (double *)y;
            switch (k) {
            case 1: e = launch<double, 1>(c->dev, c->dev.c64, xi, yo, s); break;
            case 2: e = launch<double, 2>(c->dev, c->dev.c64, xi, yo, s); break;
            case 4: e = launch<double, 4>(c->dev, c->dev.c64, xi, yo, s); break;
            default: e = launch<double, 8>(c->dev, c->dev.c64, xi, yo, s); break;
            }
        } else {
            const float *xi = (const float *)x;
            float *yo = (float *)y;
            switch (k) {
            case 1: e = launch<float, 1>(c->dev, c->dev.c32, xi, yo, s); break;
            case 2: e = launch<float, 2>(c->dev, c->dev.c32, xi, yo, s); break;
            case 4: e = launch<float, 4>(c->dev, c->dev.c32, xi, yo, s); break;
            default: e = launch<float, 8>(c->dev, c->dev.c32, xi, yo, s); break;
            }
        }
    }
    if (timing && e == cudaSuccess) {
        if (!core_used) e = cudaEventRecord(t1, s);
        ++c->tev_used;
    }
    if (e != cudaSuccess) {
        err = std::string("hx launch: ") + cudaGetErrorString(e);
        return BS_ECUDA;
    }
    return BS_OK;
}

}  // namespace bs
