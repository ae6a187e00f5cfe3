// Pipelined row kernel for y = H x (sm_103a), warp-specialized.
//
// One CTA per destination proton row ip' of a basis block.  Warp NW is the
// producer: one lane walks the row's chunk sequence and fills a ring of S
// shared-memory slots with TMA bulk copies (cp.async.bulk + mbarrier):
//   nn chunk:  the row x[ip', :] itself;
//   pp chunks: up to uc source rows x[ip, :] of the pp jumps into ip';
//   pn chunks: up to uc source rows x_s[ip_u, :] of the proton one-body
//              jumps u into ip' from one linked source block, plus the
//              pre-signed rows phi_u (+W, -W)[a_u][.] of the decoupled W_pn.
// Warps 0..NW-1 consume the slots in the same order.  Each consumer thread
// owns CPT fixed columns of the row (positions warp + NW j of the sector's
// column order, one 32-column slice per warp step) and keeps their sums in
// registers for the whole row:
//   nn: y[jn'] += sum_v c_v x[ip', jn_v]
//   pp: y[jn'] += sum_u c_u x[ip_u, jn']
//   pn: y[jn'] += sum_u sum_v (+-W)[u][b_v] x_s[ip_u, jn_v]
// then writes them once.  Slots are recycled through "empty" mbarriers (one
// arrival per consumer warp), so no CTA-wide barrier is needed after set-up.
// This is the paper's factorization of the pn term (a proton one-body jump
// times a neutron one-body jump) evaluated as a destination-owned gather: no
// atomics, a fixed summation order, bit-reproducible results.  Every mbarrier
// wait is bounded; on expiry the CTA records BS_ETIMEOUT and returns.
#include <cuda_runtime.h>

#include "bs_internal.h"
#include "bs_tma.cuh"

namespace bs {

using namespace tma;

namespace {

constexpr int kPipeMaxList = 16;

}  // namespace

struct PipeArgs {
    const RowTask *tasks;
    const DevBlock *blocks;
    const DevLink *links;
    const int64_t *pp_ptr;
    const int32_t *pp_src;
    const int64_t *p1_ptr;
    const uint32_t *p1_ent;
    const int32_t *perm;
    const int32_t *sinfo;
    const uint32_t *ent;
    const int32_t *nn_src;
    const int32_t *nn_sinfo;
    int *err;
    int S;            // slots in the ring
    int uc;           // source rows per slot
    int row_stride;   // elements per staged row
    int wrow;         // elements per signed W row (2 * wsign)
    int slot_elems;   // elements per slot: uc rows, then uc W rows
    int skip_pn;      // 1: pn chunks are left out (the core-grouped kernel computed them) ...
    int skip_pp;      // 1: pp chunks are left out, the proton single-particle diagonal is added instead ...
    int nz;           // ... and these partial vectors are added at the end, or
    int out_slot;     // (>= 0) the row is written to this partial vector instead of y
    int64_t part_stride;
};

// One step of a row's chunk sequence: nn (own row), pp chunks, pn chunks.
struct PChunk {
    int kind;        // 0 nn, 1 pp, 2 pn, 3 end
    int L;           // link (pn)
    int64_t e0;      // first entry (pp: pp entry, pn: proton one-body entry)
    int cu;          // rows in the chunk
};

struct PStream {
    int kind;
    int L;
    int64_t e, e1;
};

__device__ __forceinline__ PChunk pnext(PStream &s, const PipeArgs &A, const DevBlock &D, int row)
{
    if (s.kind == 0) {
        s.kind = 1;
        const int g = D.p_start + row;
        s.e = A.pp_ptr[g];
        s.e1 = A.skip_pp ? s.e : A.pp_ptr[g + 1];
        return PChunk{0, -1, 0, 1};
    }
    if (s.kind == 1) {
        if (s.e < s.e1) {
            const int cu = (int)min((int64_t)A.uc, s.e1 - s.e);
            const PChunk c{1, -1, s.e, cu};
            s.e += cu;
            return c;
        }
        if (A.skip_pn) {
            s.kind = 3;
            return PChunk{3, 0, 0, 0};
        }
        s.kind = 2;
        s.L = D.link_begin - 1;
        s.e = s.e1 = 0;
    }
    if (s.kind == 2) {
        while (s.e >= s.e1) {
            if (++s.L >= D.link_end) {
                s.kind = 3;
                return PChunk{3, 0, 0, 0};
            }
            const int64_t po = A.links[s.L].p_ptr_off;
            s.e = A.p1_ptr[po + row];
            s.e1 = A.p1_ptr[po + row + 1];
        }
        const int cu = (int)min((int64_t)A.uc, s.e1 - s.e);
        const PChunk c{2, s.L, s.e, cu};
        s.e += cu;
        return c;
    }
    return PChunk{3, 0, 0, 0};
}

template <typename T, int K, int NW, int CPT>
__global__ void __launch_bounds__((NW + 1) * 32, NW <= 8 ? 2 : 1) hx_pipe_kernel(PipeArgs A, const T *__restrict__ pp_coef,
                                                                const T *__restrict__ nn_coef,
                                                                const T *__restrict__ ww, const T *__restrict__ x,
                                                                T *__restrict__ y, const T *__restrict__ part,
                                                                const T *__restrict__ pdiag)
{
    extern __shared__ __align__(128) unsigned char smem[];
    T *slots = reinterpret_cast<T *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(slots + (size_t)A.S * A.slot_elems);
    const uint32_t full0 = su32(bars), empty0 = su32(bars + A.S);

    const RowTask task = A.tasks[blockIdx.x];
    const DevBlock D = A.blocks[task.block];
    const int nN = D.nN;
    const int row = task.row;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < A.S; ++s) {
            bar_init(full0 + 8u * s, 1);
            bar_init(empty0 + 8u * s, NW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == NW) {
        // ---------------- producer
        if (lane != 0) return;
        PStream st{0, 0, 0, 0};
        for (int c = 0;; ++c) {
            const PChunk ch = pnext(st, A, D, row);
            if (ch.kind == 3) break;
            const int s = c % A.S;
            const int round = c / A.S;
            if (round > 0 && bar_wait(empty0 + 8u * s, (uint32_t)(round - 1) & 1u)) {
                atomicExch(A.err, BS_ETIMEOUT);
                drain_ring(full0, A.S, c);
                return;
            }
            T *dst = slots + (size_t)s * A.slot_elems;
            const uint32_t fb = full0 + 8u * s;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (ch.kind == 0) {
                const uint32_t bytes = (uint32_t)(nN * K * sizeof(T));
                bar_expect_tx(fb, bytes);
                bulk_copy(su32(dst), x + (D.off + (int64_t)row * nN) * K, bytes, fb);
            } else if (ch.kind == 1) {
                const uint32_t bytes = (uint32_t)(nN * K * sizeof(T));
                bar_expect_tx(fb, bytes * (uint32_t)ch.cu);
                for (int u = 0; u < ch.cu; ++u)
                    bulk_copy(su32(dst + (size_t)u * A.row_stride), x + (D.off + (int64_t)A.pp_src[ch.e0 + u] * nN) * K,
                              bytes, fb);
            } else {
                const DevLink lk = A.links[ch.L];
                const DevBlock S = A.blocks[lk.src_block];
                const uint32_t bytes = (uint32_t)(S.nN * K * sizeof(T));
                const uint32_t wbytes = (uint32_t)(A.wrow * sizeof(T));
                bar_expect_tx(fb, (bytes + wbytes) * (uint32_t)ch.cu);
                T *wdst = dst + (size_t)A.uc * A.row_stride;
                for (int u = 0; u < ch.cu; ++u) {
                    const uint32_t ep = A.p1_ent[ch.e0 + u];
                    bulk_copy(su32(dst + (size_t)u * A.row_stride), x + (S.off + (int64_t)(ep & 0xFFFFu) * S.nN) * K,
                              bytes, fb);
                    const int64_t wi = lk.ww_off + (int64_t)(2 * (int)((ep >> 16) & 0x7FFFu) + (int)(ep >> 31)) * A.wrow;
                    bulk_copy(su32(wdst + (size_t)u * A.wrow), ww + wi, wbytes, fb);
                }
            }
        }
        return;
    }

    // ---------------- consumers
    const int rot = prot<T, K>(lane);
    T acc[CPT][K];
    int col[CPT];
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
#pragma unroll
        for (int q = 0; q < K; ++q) acc[j][q] = T(0);
        const int p = (warp + NW * j) * 32 + lane;
        col[j] = p < nN ? A.perm[D.perm_off + p] : -1;
    }
    T xv[K];
    PStream st{0, 0, 0, 0};
    bool hung = false;
    for (int c = 0;; ++c) {
        const PChunk ch = pnext(st, A, D, row);
        if (ch.kind == 3) break;
        const int s = c % A.S;
        const int round = c / A.S;
        if (__any_sync(0xffffffffu, bar_wait(full0 + 8u * s, (uint32_t)round & 1u))) {
            hung = true;
            break;
        }
        const T *Xs = slots + (size_t)s * A.slot_elems;
        if (ch.kind == 0) {
            if (A.skip_pp) {
                // proton single-particle energies of this row (the pp two-body
                // terms come as partial vectors)
                const T pd = pdiag[D.p_start + row];
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    if (col[j] < 0) continue;
                    pld<T, K>(Xs, col[j], rot, xv);
#pragma unroll
                    for (int q = 0; q < K; ++q) acc[j][q] = fma(pd, xv[q], acc[j][q]);
                }
            }
            // nn: lists in the sector's column order, sliced by 32
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const int sl = warp + NW * j;
                if (sl * 32 >= nN) break;
                const int off = A.nn_sinfo[D.pe_nn_sinfo + 2 * sl], lmax = A.nn_sinfo[D.pe_nn_sinfo + 2 * sl + 1];
                const int64_t base = D.pe_nn_ent + off + lane;
                for (int v = 0; v < lmax; ++v) {
                    const int64_t e = base + 32 * (int64_t)v;
                    const T cf = nn_coef[e];
                    pld<T, K>(Xs, A.nn_src[e], rot, xv);
#pragma unroll
                    for (int q = 0; q < K; ++q) acc[j][q] = fma(cf, xv[q], acc[j][q]);
                }
            }
        } else if (ch.kind == 1) {
            // pp: whole source rows, same column
            for (int u = 0; u < ch.cu; ++u) {
                const T cf = pp_coef[ch.e0 + u];
                const T *Xu = Xs + (size_t)u * A.row_stride;
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    if (col[j] < 0) continue;
                    pld<T, K>(Xu, col[j], rot, xv);
#pragma unroll
                    for (int q = 0; q < K; ++q) acc[j][q] = fma(cf, xv[q], acc[j][q]);
                }
            }
        } else {
            // pn: proton jumps u of this chunk x neutron jumps v of each column
            const DevLink lk = A.links[ch.L];
            const T *W0 = Xs + (size_t)A.uc * A.row_stride;
            const int cu = ch.cu;
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const int sl = warp + NW * j;
                if (sl * 32 >= nN) break;
                const int off = A.sinfo[lk.pe_sinfo + 2 * sl], lmax = A.sinfo[lk.pe_sinfo + 2 * sl + 1];
                if (lmax == 0) continue;
                const int64_t base = lk.pe_ent + off + lane;
                if (lmax <= kPipeMaxList) {
                    // entries past the slice's longest list point at a zero weight
                    const uint32_t pad = (uint32_t)(A.wrow / 2 - 1) << 16;
                    uint32_t ev[kPipeMaxList];
#pragma unroll
                    for (int v = 0; v < kPipeMaxList; ++v) ev[v] = v < lmax ? A.ent[base + 32 * v] : pad;
                    for (int u = 0; u < cu; ++u) {
                        const T *Xu = Xs + (size_t)u * A.row_stride;
                        const T *Wu = W0 + (size_t)u * A.wrow;
#pragma unroll
                        for (int v0 = 0; v0 < kPipeMaxList; v0 += 2) {
                            if (v0 >= lmax) break;
#pragma unroll
                            for (int dv = 0; dv < 2; ++dv) {
                                const uint32_t en = ev[v0 + dv];
                                const T w = Wu[(en >> 16) & 0x7FFFu];
                                pld<T, K>(Xu, (int)(en & 0xFFFFu), rot, xv);
#pragma unroll
                                for (int q = 0; q < K; ++q) acc[j][q] = fma(w, xv[q], acc[j][q]);
                            }
                        }
                    }
                } else {
                    for (int v = 0; v < lmax; ++v) {
                        const uint32_t en = A.ent[base + 32 * (int64_t)v];
                        for (int u = 0; u < cu; ++u) {
                            const T w = W0[(size_t)u * A.wrow + ((en >> 16) & 0x7FFFu)];
                            pld<T, K>(Xs + (size_t)u * A.row_stride, (int)(en & 0xFFFFu), rot, xv);
#pragma unroll
                            for (int q = 0; q < K; ++q) acc[j][q] = fma(w, xv[q], acc[j][q]);
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) bar_arrive(empty0 + 8u * s);
    }
    if (hung) {
        if (lane == 0) atomicExch(A.err, BS_ETIMEOUT);
        return;
    }
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
        if (col[j] < 0) continue;
        prot_fix<T, K>(acc[j], rot);
        const int64_t at = (D.off + (int64_t)row * nN + col[j]) * K;
        for (int t = 0; t < A.nz; ++t) {
            // partial sums of the core-grouped kernels, added in a fixed order
            T pv[K];
            pld<T, K>(part + t * A.part_stride + at, 0, 0, pv);
#pragma unroll
            for (int q = 0; q < K; ++q) acc[j][q] += pv[q];
        }
        pst<T, K>((A.out_slot >= 0 ? const_cast<T *>(part) + A.out_slot * A.part_stride : y) + at, acc[j]);
    }
}

namespace {

struct PipeVariant {
    int nw, cpt, S;
    size_t target;
};

template <typename T, int K, int NW, int CPT>
cudaError_t launch_pipe_t(const Device &Dv, const DevCoefs<T> &C, const T *ww, const T *nn_coef, const T *x, T *y,
                          cudaStream_t s, int S, size_t target, bool &used, const T *part, int nz, int64_t dim,
                          const T *pdiag)
{
    const size_t es = sizeof(T);
    const int row_elems = Dv.max_nN * K;
    const int row_stride = (int)(((row_elems * es + 127) / 128) * 128 / es);
    const int wrow = 2 * Dv.wsign;
    const size_t hard = 227 * 1024;
    const size_t per_u = (size_t)row_stride * es + (size_t)wrow * es;
    const size_t bars = 16 * (size_t)S + 16;
    int uc = (int)((target > bars ? target - bars : 0) / ((size_t)S * per_u));
    if (uc < 1) uc = (int)((hard > bars ? hard - bars : 0) / ((size_t)S * per_u));
    // TMA rows need 16-byte elements (k values of one basis state)
    used = uc >= 1 && (size_t)NW * CPT * 32 >= (size_t)Dv.max_nN && (K * es) % 16 == 0;
    if (!used || !x) return cudaSuccess;   // x == nullptr: only report whether the variant fits
    uc = std::min(uc, std::max(1, std::max(Dv.max_pu, 1)));
    uc = std::min(uc, 8);
    const int slot_elems = uc * row_stride + uc * wrow;
    const size_t smem = (size_t)S * slot_elems * es + bars;
    auto kern = hx_pipe_kernel<T, K, NW, CPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    PipeArgs A{Dv.rtasks, Dv.blocks, Dv.links, Dv.pp_ptr, Dv.pp_src, Dv.p1_ptr, Dv.p1_ent, Dv.pe_perm, Dv.pe_sinfo,
               Dv.pe_ent, Dv.pe_nn_src, Dv.pe_nn_sinfo, Dv.err, S, uc, row_stride, wrow, slot_elems,
               part ? 1 : 0, pdiag ? 1 : 0, part && nz < 0 ? 0 : (part ? nz : 0), part && nz < 0 ? -nz - 1 : -1, dim * K};
    kern<<<Dv.nrtasks, (NW + 1) * 32, smem, s>>>(A, C.pp_coef, nn_coef, ww, x, y, part, pdiag);
    return cudaGetLastError();
}

// variants: consumer warps, columns per thread (largest sector must fit), ring slots, smem target
constexpr PipeVariant kPipeVariants[] = {
    {8, 3, 3, 110 * 1024}, {8, 4, 3, 110 * 1024}, {16, 2, 3, 110 * 1024}, {16, 8, 2, 200 * 1024}, {8, 1, 3, 75 * 1024},
};
constexpr int kNumPipe = 5;

template <typename T, int K>
cudaError_t launch_pipe_k(const Device &Dv, const DevCoefs<T> &C, const T *ww, const T *nn_coef, const T *x, T *y,
                          cudaStream_t s, int v, bool &used, const T *part = nullptr, int nz = 0, int64_t dim = 0,
                          const T *pdiag = nullptr)
{
    const PipeVariant P = kPipeVariants[v];
    if (P.nw == 8 && P.cpt == 3)
        return launch_pipe_t<T, K, 8, 3>(Dv, C, ww, nn_coef, x, y, s, P.S, P.target, used, part, nz, dim, pdiag);
    if (P.nw == 8 && P.cpt == 4)
        return launch_pipe_t<T, K, 8, 4>(Dv, C, ww, nn_coef, x, y, s, P.S, P.target, used, part, nz, dim, pdiag);
    if (P.nw == 16 && P.cpt == 2)
        return launch_pipe_t<T, K, 16, 2>(Dv, C, ww, nn_coef, x, y, s, P.S, P.target, used, part, nz, dim, pdiag);
    if (P.nw == 16 && P.cpt == 8)
        return launch_pipe_t<T, K, 16, 8>(Dv, C, ww, nn_coef, x, y, s, P.S, P.target, used, part, nz, dim, pdiag);
    return launch_pipe_t<T, K, 8, 1>(Dv, C, ww, nn_coef, x, y, s, P.S, P.target, used, part, nz, dim, pdiag);
}

}  // namespace

int pipe_variants() { return kNumPipe; }

// The pipelined kernel without its pn chunks (and, with skip_pp, without its
// pp chunks but with the proton single-particle diagonal), adding nz partial
// vectors (FP32, k = 4 or 8) of the core-grouped kernels; with nz = -1 - t it
// adds none and writes its rows to partial vector t instead of y.  x ==
// nullptr only checks whether variant v fits.
cudaError_t launch_hx_pipe_combine(const bs_ctx *c, const void *x, void *y, int k, bs_dtype dt, cudaStream_t s, int v,
                                   const void *part, int nz, bool skip_pp, bool &used)
{
    const Device &D = c->dev;
    used = false;
    if (D.trunc || dt != BS_F32 || (k != 4 && k != 8)) return cudaSuccess;
    const float *xi = (const float *)x;
    float *yo = (float *)y;
    const float *pi = (const float *)part;
    const float *pd = skip_pp ? D.pdiag32 : nullptr;
    if (k == 4)
        return launch_pipe_k<float, 4>(D, D.c32, D.ww32, D.pe_nn_coef32, xi, yo, s, v, used, pi, nz, c->basis.dim, pd);
    return launch_pipe_k<float, 8>(D, D.c32, D.ww32, D.pe_nn_coef32, xi, yo, s, v, used, pi, nz, c->basis.dim, pd);
}

// Pipelined kernel, variant v; `used` is false when it does not fit (row too
// wide for the variant's columns or shared memory).
cudaError_t launch_hx_pipe(const bs_ctx *c, const void *x, void *y, int k, bs_dtype dt, cudaStream_t s, int v,
                           bool &used)
{
    const Device &D = c->dev;
    used = false;
    if (D.trunc) return cudaSuccess;   // like-particle moves inside a block only
    if (dt == BS_F64) {
        const double *xi = (const double *)x;
        double *yo = (double *)y;
        switch (k) {
        case 1: return launch_pipe_k<double, 1>(D, D.c64, D.ww64, D.pe_nn_coef64, xi, yo, s, v, used);
        case 2: return launch_pipe_k<double, 2>(D, D.c64, D.ww64, D.pe_nn_coef64, xi, yo, s, v, used);
        case 4: return launch_pipe_k<double, 4>(D, D.c64, D.ww64, D.pe_nn_coef64, xi, yo, s, v, used);
        default: return launch_pipe_k<double, 8>(D, D.c64, D.ww64, D.pe_nn_coef64, xi, yo, s, v, used);
        }
    }
    const float *xi = (const float *)x;
    float *yo = (float *)y;
    switch (k) {
    case 1: return launch_pipe_k<float, 1>(D, D.c32, D.ww32, D.pe_nn_coef32, xi, yo, s, v, used);
    case 2: return launch_pipe_k<float, 2>(D, D.c32, D.ww32, D.pe_nn_coef32, xi, yo, s, v, used);
    case 4: return launch_pipe_k<float, 4>(D, D.c32, D.ww32, D.pe_nn_coef32, xi, yo, s, v, used);
    default: return launch_pipe_k<float, 8>(D, D.c32, D.ww32, D.pe_nn_coef32, xi, yo, s, v, used);
    }
}

}  // namespace bs
