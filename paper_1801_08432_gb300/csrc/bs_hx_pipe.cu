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

namespace bs {

namespace {

constexpr uint32_t kPipeWaitLimit = 1u << 22;
constexpr int kPipeMaxList = 16;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(n) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint32_t b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint32_t b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}

__device__ __forceinline__ bool bar_try(uint32_t b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; true if it expired
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity)
{
    uint32_t spins = 0;
    while (!bar_try(b, parity))
        if (++spins > kPipeWaitLimit) return true;
    return false;
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t b)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}

// K values of element jn of a staged row.  32- and 64-byte elements are read
// in 16-byte chunks starting at chunk `rot` (fixed per lane) so that the
// first load of a quarter warp spreads over the bank groups; the registers
// then hold the values rotated by `rot` and prot_fix() restores the order of
// a finished sum.
template <typename T, int K>
__device__ __forceinline__ void pld(const T *row, int jn, int rot, T (&r)[K])
{
    constexpr int E = K * (int)sizeof(T);
    if constexpr (E == 32 || E == 64) {
        constexpr int NC = E / 16, W = 16 / (int)sizeof(T);
        const char *p = reinterpret_cast<const char *>(row) + (size_t)jn * E;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const float4 q = *reinterpret_cast<const float4 *>(p + 16 * ((c + rot) & (NC - 1)));
            if constexpr (sizeof(T) == 4) {
                r[4 * c] = q.x; r[4 * c + 1] = q.y; r[4 * c + 2] = q.z; r[4 * c + 3] = q.w;
            } else {
                const double2 d = *reinterpret_cast<const double2 *>(&q);
                r[W * c] = d.x; r[W * c + 1] = d.y;
            }
        }
    } else if constexpr (E == 16) {
        const float4 q = *reinterpret_cast<const float4 *>(row + (size_t)jn * K);
        if constexpr (sizeof(T) == 4) {
            r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
        } else {
            const double2 d = *reinterpret_cast<const double2 *>(&q);
            r[0] = d.x; r[1] = d.y;
        }
    } else if constexpr (E == 8 && sizeof(T) == 4) {
        const float2 q = *reinterpret_cast<const float2 *>(row + (size_t)jn * K);
        r[0] = q.x; r[1] = q.y;
    } else {
        r[0] = row[jn];
    }
}

template <typename T, int K>
__device__ __forceinline__ int prot(int lane)
{
    constexpr int E = K * (int)sizeof(T);
    return E == 32 ? (lane & 1) : E == 64 ? (lane & 3) : 0;
}

template <typename T, int K>
__device__ __forceinline__ void prot_fix(T (&r)[K], int rot)
{
    constexpr int E = K * (int)sizeof(T);
    if constexpr (E == 32 || E == 64) {
        constexpr int NC = E / 16, W = 16 / (int)sizeof(T);
        T t[K];
#pragma unroll
        for (int i = 0; i < K; ++i) t[i] = r[i];
#pragma unroll
        for (int j = 0; j < NC; ++j)
#pragma unroll
            for (int w = 0; w < W; ++w) {
                T v = t[w];
#pragma unroll
                for (int c = 1; c < NC; ++c) v = (((c + rot) & (NC - 1)) == j) ? t[W * c + w] : v;
                r[W * j + w] = v;
            }
    }
}

template <typename T, int K>
__device__ __forceinline__ void pst(T *p, const T (&r)[K])
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
        s.e1 = A.pp_ptr[g + 1];
        return PChunk{0, -1, 0, 1};
    }
    if (s.kind == 1) {
        if (s.e < s.e1) {
            const int cu = (int)min((int64_t)A.uc, s.e1 - s.e);
            const PChunk c{1, -1, s.e, cu};
            s.e += cu;
            return c;
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
                                                                T *__restrict__ y)
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
                                const T w = Wu[en >> 16];
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
                            const T w = W0[(size_t)u * A.wrow + (en >> 16)];
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
        pst<T, K>(y + (D.off + (int64_t)row * nN + col[j]) * K, acc[j]);
    }
}

namespace {

struct PipeVariant {
    int nw, cpt, S;
    size_t target;
};

template <typename T, int K, int NW, int CPT>
cudaError_t launch_pipe_t(const Device &Dv, const DevCoefs<T> &C, const T *ww, const T *nn_coef, const T *x, T *y,
                          cudaStream_t s, int S, size_t target, bool &used)
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
    if (!used) return cudaSuccess;
    uc = std::min(uc, std::max(1, std::max(Dv.max_pu, 1)));
    uc = std::min(uc, 8);
    const int slot_elems = uc * row_stride + uc * wrow;
    const size_t smem = (size_t)S * slot_elems * es + bars;
    auto kern = hx_pipe_kernel<T, K, NW, CPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    PipeArgs A{Dv.rtasks, Dv.blocks, Dv.links, Dv.pp_ptr, Dv.pp_src, Dv.p1_ptr, Dv.p1_ent, Dv.pe_perm, Dv.pe_sinfo,
               Dv.pe_ent, Dv.pe_nn_src, Dv.pe_nn_sinfo, Dv.err, S, uc, row_stride, wrow, slot_elems};
    kern<<<Dv.nrtasks, (NW + 1) * 32, smem, s>>>(A, C.pp_coef, nn_coef, ww, x, y);
    return cudaGetLastError();
}

// variants: consumer warps, columns per thread (largest sector must fit), ring slots, smem target
constexpr PipeVariant kPipeVariants[] = {
    {8, 3, 3, 110 * 1024}, {8, 4, 3, 110 * 1024}, {16, 2, 3, 110 * 1024}, {16, 8, 2, 200 * 1024}, {8, 1, 3, 75 * 1024},
};
constexpr int kNumPipe = 5;

template <typename T, int K>
cudaError_t launch_pipe_k(const Device &Dv, const DevCoefs<T> &C, const T *ww, const T *nn_coef, const T *x, T *y,
                          cudaStream_t s, int v, bool &used)
{
    const PipeVariant P = kPipeVariants[v];
    if (P.nw == 8 && P.cpt == 3) return launch_pipe_t<T, K, 8, 3>(Dv, C, ww, nn_coef, x, y, s, P.S, P.target, used);
    if (P.nw == 8 && P.cpt == 4) return launch_pipe_t<T, K, 8, 4>(Dv, C, ww, nn_coef, x, y, s, P.S, P.target, used);
    if (P.nw == 16 && P.cpt == 2) return launch_pipe_t<T, K, 16, 2>(Dv, C, ww, nn_coef, x, y, s, P.S, P.target, used);
    if (P.nw == 16 && P.cpt == 8) return launch_pipe_t<T, K, 16, 8>(Dv, C, ww, nn_coef, x, y, s, P.S, P.target, used);
    return launch_pipe_t<T, K, 8, 1>(Dv, C, ww, nn_coef, x, y, s, P.S, P.target, used);
}

}  // namespace

int pipe_variants() { return kNumPipe; }

// Pipelined kernel, variant v; `used` is false when it does not fit (row too
// wide for the variant's columns or shared memory).
cudaError_t launch_hx_pipe(const bs_ctx *c, const void *x, void *y, int k, bs_dtype dt, cudaStream_t s, int v,
                           bool &used)
{
    const Device &D = c->dev;
    used = false;
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
