// pn term of y = H x grouped by (Z-1)-proton cores (sm_103a).
//
// The proton one-body operator restricted to Z-proton SDs factors through the
// Z-1 proton SDs ("cores"): a+_i a_k = sum_c a+_i |c><c| a_k, so every proton
// jump s -> r of the paper's pn factorization (a proton one-body jump times a
// neutron one-body jump, Eq. xpndef) belongs to exactly one core c, with
// s = a+_k c and r = a+_i c.  A unit (see CoreUnit) is one core and up to four
// states i of one (2m, parity): its destination rows r_p = a+_{i_p} c lie in
// one block, so they share the neutron columns and the neutron jump lists of
// every link.  For each source row c + k staged in shared memory, a thread that
// owns destination column n' gathers x[c+k][n_v] once per neutron jump v and
// applies it to all four rows with one 16-byte load of the weights
// (W(i_0 j_v, k l_v), ..., W(i_3 j_v, k l_v)): four times the multiply-adds of
// the row-by-row kernel per shared-memory element read.
//
// Persistent and warp-specialized: warp NW is the producer (one lane fills a
// ring of S slots, each one source row plus its [2 wsign][4] weight table, by
// TMA bulk copies completing on an mbarrier); warps 0..NW-1 consume, one
// destination column per thread, the column tile's accumulators in registers.
// The result for row r through core c goes to partial vector t (the rank of
// the removed state in r), so every element of every partial vector has one
// writer; the pipelined like-particle kernel then adds the Z partials in the
// order t = 0..Z-1.  No atomics, bit-reproducible.  Every mbarrier wait is
// bounded; on expiry the CTA records BS_ETIMEOUT and returns.
#include <cuda_runtime.h>

#include <algorithm>

#include "bs_internal.h"
#include "bs_tma.cuh"

namespace bs {

using namespace tma;

cudaError_t launch_hx_pipe_combine(const bs_ctx *c, const void *x, void *y, int k, bs_dtype dt, cudaStream_t s, int v,
                                   const void *part, int nz, bool skip_pp, bool &used);

namespace {

constexpr int kCoreMaxList = 16;

struct CoreArgs {
    const CoreUnit *units;
    const CoreSrc *src;
    const DevBlock *blocks;
    const DevLink *links;
    const int32_t *perm;
    const int32_t *sinfo;
    const uint32_t *ent;
    int *err;
    int nunits;
    int S;             // ring slots
    int row_stride;    // floats per staged row (multiple of 32)
    int wtab;          // floats per weight table (2 wsign x 4)
    int slot_elems;    // row_stride + wtab
    uint32_t ws;       // wsign
    int64_t part_stride;   // dim * K
};

template <int K, int NW, int MINB>
__global__ void __launch_bounds__((NW + 1) * 32, MINB)
    hx_core_kernel(CoreArgs A, const float *__restrict__ wc, const float *__restrict__ x, float *__restrict__ part)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float *slots = reinterpret_cast<float *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(slots + (size_t)A.S * A.slot_elems);
    const uint32_t full0 = su32(bars), empty0 = su32(bars + A.S);
    constexpr int C = NW * 32;   // columns per tile
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
        // ---------------- producer: one lane streams every unit's sources, tile by tile
        if (lane != 0) return;
        int c = 0;
        for (int u = blockIdx.x; u < A.nunits; u += gridDim.x) {
            const CoreUnit U = A.units[u];
            const int ntile = (A.blocks[U.dblock].nN + C - 1) / C;
            for (int tile = 0; tile < ntile; ++tile)
                for (int q = 0; q < U.nsrc; ++q, ++c) {
                    const int s = c % A.S;
                    const int round = c / A.S;
                    if (round > 0 && bar_wait(empty0 + 8u * s, (uint32_t)(round - 1) & 1u)) {
                        atomicExch(A.err, BS_ETIMEOUT);
                        return;
                    }
                    const CoreSrc cs = A.src[U.src0 + q];
                    const DevBlock Sb = A.blocks[cs.sblock];
                    const uint32_t bytes = (uint32_t)(Sb.nN * K * (int)sizeof(float));
                    const uint32_t wbytes = (uint32_t)(A.wtab * (int)sizeof(float));
                    float *dst = slots + (size_t)s * A.slot_elems;
                    const uint32_t fb = full0 + 8u * s;
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bar_expect_tx(fb, bytes + wbytes);
                    bulk_copy(su32(dst), x + (Sb.off + (int64_t)cs.srow * Sb.nN) * K, bytes, fb);
                    bulk_copy(su32(dst + A.row_stride), wc + (size_t)(cs.wtab & 0x7FFFFFFFu) * A.wtab, wbytes, fb);
                }
        }
        return;
    }

    // ---------------- consumers
    const int rot = prot<float, K>(lane);
    int c = 0;
    for (int u = blockIdx.x; u < A.nunits; u += gridDim.x) {
        const CoreUnit U = A.units[u];
        const DevBlock D = A.blocks[U.dblock];
        const int nN = D.nN;
        const int ntile = (nN + C - 1) / C;
        for (int tile = 0; tile < ntile; ++tile) {
            const int pos0 = tile * C + warp * 32;   // warp-uniform
            const bool active = pos0 < nN;
            const int pos = pos0 + lane;
            const int sl = pos0 >> 5;
            const int col = pos < nN ? A.perm[D.perm_off + pos] : -1;
            float acc[4][K];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < K; ++q) acc[p][q] = 0.0f;
            int prev = -1, lmax = 0;
            int64_t base = 0;
            uint32_t ev[kCoreMaxList];
#pragma unroll
            for (int v = 0; v < kCoreMaxList; ++v) ev[v] = 0;
            for (int q = 0; q < U.nsrc; ++q, ++c) {
                const int s = c % A.S;
                const int round = c / A.S;
                if (__any_sync(0xffffffffu, bar_wait(full0 + 8u * s, (uint32_t)round & 1u))) {
                    if (lane == 0) atomicExch(A.err, BS_ETIMEOUT);
                    return;
                }
                if (active) {
                    const CoreSrc cs = A.src[U.src0 + q];
                    if (cs.link != prev) {
                        // a new link: this warp's slice of its neutron lists
                        prev = cs.link;
                        const DevLink lk = A.links[cs.link];
                        const int off = A.sinfo[lk.pe_sinfo + 2 * sl];
                        lmax = A.sinfo[lk.pe_sinfo + 2 * sl + 1];
                        base = lk.pe_ent + off + lane;
                        if (lmax <= kCoreMaxList) {
                            const uint32_t pad = (A.ws - 1u) << 16;   // a zero weight, source column 0
#pragma unroll
                            for (int v = 0; v < kCoreMaxList; ++v) ev[v] = v < lmax ? A.ent[base + 32 * v] : pad;
                        }
                    }
                    const float *Xs = slots + (size_t)s * A.slot_elems;
                    const float *Wt = Xs + A.row_stride;
                    const uint32_t flip = (cs.wtab >> 31) ? A.ws : 0u;   // sign of a_k on c + k: swap the +W / -W halves
                    float xv[K];
                    if (lmax <= kCoreMaxList) {
#pragma unroll
                        for (int v = 0; v < kCoreMaxList; ++v) {
                            if (v >= lmax) break;
                            const uint32_t en = ev[v];
                            const float4 w = *reinterpret_cast<const float4 *>(Wt + 4 * ((en >> 16) ^ flip));
                            pld<float, K>(Xs, (int)(en & 0xFFFFu), rot, xv);
#pragma unroll
                            for (int qq = 0; qq < K; ++qq) {
                                acc[0][qq] = fmaf(w.x, xv[qq], acc[0][qq]);
                                acc[1][qq] = fmaf(w.y, xv[qq], acc[1][qq]);
                                acc[2][qq] = fmaf(w.z, xv[qq], acc[2][qq]);
                                acc[3][qq] = fmaf(w.w, xv[qq], acc[3][qq]);
                            }
                        }
                    } else {
                        for (int v = 0; v < lmax; ++v) {
                            const uint32_t en = A.ent[base + 32 * (int64_t)v];
                            const float4 w = *reinterpret_cast<const float4 *>(Wt + 4 * ((en >> 16) ^ flip));
                            pld<float, K>(Xs, (int)(en & 0xFFFFu), rot, xv);
#pragma unroll
                            for (int qq = 0; qq < K; ++qq) {
                                acc[0][qq] = fmaf(w.x, xv[qq], acc[0][qq]);
                                acc[1][qq] = fmaf(w.y, xv[qq], acc[1][qq]);
                                acc[2][qq] = fmaf(w.z, xv[qq], acc[2][qq]);
                                acc[3][qq] = fmaf(w.w, xv[qq], acc[3][qq]);
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) bar_arrive(empty0 + 8u * s);
            }
            if (col >= 0) {
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    if (U.drow[p] < 0) continue;
                    prot_fix<float, K>(acc[p], rot);
                    if (U.meta[p] & 256)
#pragma unroll
                        for (int qq = 0; qq < K; ++qq) acc[p][qq] = -acc[p][qq];
                    pst<float, K>(part + (int64_t)(U.meta[p] & 255) * A.part_stride +
                                      (D.off + (int64_t)U.drow[p] * nN + col) * K,
                                  acc[p]);
                }
            }
        }
    }
}

struct PPArgs {
    const PPUnit *units;
    const int32_t *srow;
    const float *w;        // kPPG weights per source
    const DevBlock *blocks;
    int *err;
    int nunits;
    int S;
    int row_stride;
    int slot_elems;        // row_stride + kPPG
    int64_t part_stride;
};

// pp term by (Z-2)-proton cores.  The same ring as above; a slot holds one
// source row and its kPPG signed weights (CTA-uniform: read as broadcasts).
// Each thread owns one destination column in natural order (a quarter warp
// reads eight consecutive 32-byte elements: conflict-free with the lane
// rotation (lane >> 2) & 1) and applies the element to kPPG destination rows.
template <int K, int NW, int MINB>
__global__ void __launch_bounds__((NW + 1) * 32, MINB)
    hx_ppcore_kernel(PPArgs A, const float *__restrict__ x, float *__restrict__ part)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float *slots = reinterpret_cast<float *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(slots + (size_t)A.S * A.slot_elems);
    const uint32_t full0 = su32(bars), empty0 = su32(bars + A.S);
    constexpr int C = NW * 32;
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
        if (lane != 0) return;
        int c = 0;
        for (int u = blockIdx.x; u < A.nunits; u += gridDim.x) {
            const PPUnit U = A.units[u];
            const DevBlock D = A.blocks[U.dblock];
            const int ntile = (D.nN + C - 1) / C;
            const uint32_t bytes = (uint32_t)(D.nN * K * (int)sizeof(float));
            const uint32_t wbytes = (uint32_t)(kPPG * sizeof(float));
            for (int tile = 0; tile < ntile; ++tile)
                for (int q = 0; q < U.nsrc; ++q, ++c) {
                    const int s = c % A.S;
                    const int round = c / A.S;
                    if (round > 0 && bar_wait(empty0 + 8u * s, (uint32_t)(round - 1) & 1u)) {
                        atomicExch(A.err, BS_ETIMEOUT);
                        return;
                    }
                    const uint32_t fb = full0 + 8u * s;
                    float *dst = slots + (size_t)s * A.slot_elems;
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bar_expect_tx(fb, bytes + wbytes);
                    bulk_copy(su32(dst), x + (D.off + (int64_t)A.srow[U.src0 + q] * D.nN) * K, bytes, fb);
                    bulk_copy(su32(dst + A.row_stride), A.w + (U.src0 + q) * kPPG, wbytes, fb);
                }
        }
        return;
    }

    constexpr int E = K * (int)sizeof(float);
    const int rot = E == 32 ? ((lane >> 2) & 1) : 0;
    int c = 0;
    for (int u = blockIdx.x; u < A.nunits; u += gridDim.x) {
        const PPUnit U = A.units[u];
        const DevBlock D = A.blocks[U.dblock];
        const int nN = D.nN;
        const int ntile = (nN + C - 1) / C;
        for (int tile = 0; tile < ntile; ++tile) {
            const int col = tile * C + warp * 32 + lane;
            const bool active = tile * C + warp * 32 < nN;
            const int cl = col < nN ? col : nN - 1;
            float acc[kPPG][K];
#pragma unroll
            for (int p = 0; p < kPPG; ++p)
#pragma unroll
                for (int q = 0; q < K; ++q) acc[p][q] = 0.0f;
            for (int q = 0; q < U.nsrc; ++q, ++c) {
                const int s = c % A.S;
                const int round = c / A.S;
                if (__any_sync(0xffffffffu, bar_wait(full0 + 8u * s, (uint32_t)round & 1u))) {
                    if (lane == 0) atomicExch(A.err, BS_ETIMEOUT);
                    return;
                }
                if (active) {
                    const float *Xs = slots + (size_t)s * A.slot_elems;
                    float w[kPPG];
#pragma unroll
                    for (int p = 0; p < kPPG; p += 4) {
                        const float4 w4 = *reinterpret_cast<const float4 *>(Xs + A.row_stride + p);
                        w[p] = w4.x; w[p + 1] = w4.y; w[p + 2] = w4.z; w[p + 3] = w4.w;
                    }
                    float xv[K];
                    pld<float, K>(Xs, cl, rot, xv);
#pragma unroll
                    for (int p = 0; p < kPPG; ++p)
#pragma unroll
                        for (int qq = 0; qq < K; ++qq) acc[p][qq] = fmaf(w[p], xv[qq], acc[p][qq]);
                }
                __syncwarp();
                if (lane == 0) bar_arrive(empty0 + 8u * s);
            }
            if (col < nN) {
#pragma unroll
                for (int p = 0; p < kPPG; ++p) {
                    if (U.drow[p] < 0) continue;
                    prot_fix<float, K>(acc[p], rot);
                    pst<float, K>(part + (int64_t)U.part[p] * A.part_stride + (D.off + (int64_t)U.drow[p] * nN + col) * K,
                                  acc[p]);
                }
            }
        }
    }
}

struct NNArgs {
    const int2 *tasks;
    const DevBlock *blocks;
    const int32_t *perm;
    const int32_t *src;
    const float *coef;
    const int32_t *sinfo;
    const float *pdiag;
    int *err;
    int row_stride;
};

// Neutron like-particle term plus the proton single-particle diagonal over a
// tile of R consecutive proton rows of one block: y[r][n'] = e_p(r) x[r][n'] +
// sum_v c_v x[r][n_v].  The neutron lists are the same for every proton row,
// so each thread (one destination column, in the sector's list order) loads
// an entry once and applies it to the R staged rows.  The R rows arrive by
// TMA bulk copies on one mbarrier (bounded wait).  Output: partial vector.
template <int K, int R, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB)
    hx_nn_rows_kernel(NNArgs A, const float *__restrict__ x, float *__restrict__ out)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float *rows = reinterpret_cast<float *>(smem);
    uint64_t *bar = reinterpret_cast<uint64_t *>(rows + (size_t)R * A.row_stride);
    const uint32_t b0 = su32(bar);
    const int2 task = A.tasks[blockIdx.x];
    const DevBlock D = A.blocks[task.x];
    const int nN = D.nN;
    const int r0 = task.y;
    const int nr = min(R, D.nP - r0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        bar_init(b0, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)(nN * K * (int)sizeof(float));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bar_expect_tx(b0, bytes * (uint32_t)nr);
        for (int r = 0; r < nr; ++r)
            bulk_copy(su32(rows + (size_t)r * A.row_stride), x + (D.off + (int64_t)(r0 + r) * nN) * K, bytes, b0);
    }
    float pd[R];
#pragma unroll
    for (int r = 0; r < R; ++r) pd[r] = r < nr ? A.pdiag[D.p_start + r0 + r] : 0.0f;
    const int p = warp * 32 + lane;
    const int sl = warp;
    const bool active = sl * 32 < nN;   // warp-uniform
    const int col = p < nN ? A.perm[D.perm_off + p] : -1;
    int off = 0, lmax = 0;
    if (active) {
        off = A.sinfo[D.pe_nn_sinfo + 2 * sl];
        lmax = A.sinfo[D.pe_nn_sinfo + 2 * sl + 1];
    }
    if (__any_sync(0xffffffffu, bar_wait(b0, 0u))) {
        if (lane == 0) atomicExch(A.err, BS_ETIMEOUT);
        return;
    }
    if (!active) return;
    const int rot = prot<float, K>(lane);
    float acc[R][K], xv[K];
    const int cc = col >= 0 ? col : 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        pld<float, K>(rows + (size_t)r * A.row_stride, cc, rot, xv);
#pragma unroll
        for (int q = 0; q < K; ++q) acc[r][q] = pd[r] * xv[q];
    }
    const int64_t base = D.pe_nn_ent + off + lane;
#pragma unroll 2
    for (int v = 0; v < lmax; ++v) {
        const float c = A.coef[base + 32 * (int64_t)v];
        const int s = A.src[base + 32 * (int64_t)v];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            pld<float, K>(rows + (size_t)r * A.row_stride, s, rot, xv);
#pragma unroll
            for (int q = 0; q < K; ++q) acc[r][q] = fmaf(c, xv[q], acc[r][q]);
        }
    }
    if (col < 0) return;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r >= nr) break;
        prot_fix<float, K>(acc[r], rot);
        pst<float, K>(out + (D.off + (int64_t)(r0 + r) * nN + col) * K, acc[r]);
    }
}

// y = sum_t part[t], t = 0..n-1 in order, float4 at a time (the fixed order
// keeps the product bit-reproducible).
__global__ void __launch_bounds__(256) hx_sum_partials(const float4 *__restrict__ part, int n, int64_t n4,
                                                       float4 *__restrict__ y)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x) {
        float4 a = part[e];
        for (int t = 1; t < n; ++t) {
            const float4 b = part[t * n4 + e];
            a.x += b.x;
            a.y += b.y;
            a.z += b.z;
            a.w += b.w;
        }
        y[e] = a;
    }
}

struct CoreVariant {
    int nw, minb;
    size_t target;   // shared-memory budget per CTA
    bool pp;         // pp term by (Z-2)-proton cores, nn by row tiles of nn_rows rows
    int nn_rows;
};

constexpr CoreVariant kCoreVariants[] = {
    {18, 1, 200 * 1024, false, 0}, {10, 2, 105 * 1024, false, 0}, {18, 1, 200 * 1024, true, 4}, {18, 1, 200 * 1024, true, 2}};
constexpr int kNumCore = 4;

template <int K, int R, int MINB>
cudaError_t launch_nn_t(const bs_ctx *ctx, const float *x, float *out, cudaStream_t s, bool &used)
{
    const Device &Dv = ctx->dev;
    constexpr int NW = 18;
    const int row_stride = ((Dv.max_nN * K + 31) / 32) * 32;
    const size_t smem = (size_t)R * row_stride * sizeof(float) + 16;
    used = Dv.max_nN <= NW * 32 && smem <= 200 * 1024;
    if (!used || !x) return cudaSuccess;
    auto kern = hx_nn_rows_kernel<K, R, NW, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    NNArgs A{R == 2 ? Dv.nntasks2 : Dv.nntasks4, Dv.blocks, Dv.pe_perm, Dv.pe_nn_src, Dv.pe_nn_coef32, Dv.pe_nn_sinfo,
             Dv.pdiag32, Dv.err, row_stride};
    kern<<<R == 2 ? Dv.nnntasks2 : Dv.nnntasks4, NW * 32, smem, s>>>(A, x, out);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_nn_k(const bs_ctx *ctx, const float *x, float *out, cudaStream_t s, int R, bool &used)
{
    return R == 2 ? launch_nn_t<K, 2, 2>(ctx, x, out, s, used) : launch_nn_t<K, 4, 1>(ctx, x, out, s, used);
}

template <int K, int NW, int MINB>
cudaError_t launch_core_t(const bs_ctx *ctx, const float *x, float *part, cudaStream_t s, size_t target, bool &used)
{
    const Device &Dv = ctx->dev;
    const int row_stride = ((Dv.max_nN * K + 31) / 32) * 32;
    const int wtab = 8 * Dv.wsign;
    const int slot_elems = row_stride + wtab;
    const size_t slot_bytes = (size_t)slot_elems * sizeof(float) + 16;
    int S = (int)std::min<size_t>(8, target / slot_bytes);
    used = S >= 2;
    if (!used) return cudaSuccess;
    const size_t smem = (size_t)S * slot_elems * sizeof(float) + 16 * (size_t)S;
    auto kern = hx_core_kernel<K, NW, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 0, per = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, Dv.dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, (NW + 1) * 32, smem)) != cudaSuccess) return e;
    const int grid = std::max(1, std::min(Dv.ncunits, nsm * std::max(per, 1)));
    CoreArgs A{Dv.cunits, Dv.csrc, Dv.blocks, Dv.links, Dv.pe_perm, Dv.pe_sinfo, Dv.pe_ent, Dv.err,
               Dv.ncunits, S, row_stride, wtab, slot_elems, (uint32_t)Dv.wsign, (int64_t)ctx->basis.dim * K};
    kern<<<grid, (NW + 1) * 32, smem, s>>>(A, Dv.wc32, x, part);
    return cudaGetLastError();
}

template <int K, int NW, int MINB>
cudaError_t launch_pp_t(const bs_ctx *ctx, const float *x, float *part, cudaStream_t s, size_t target, bool &used)
{
    const Device &Dv = ctx->dev;
    const int row_stride = ((Dv.max_nN * K + 31) / 32) * 32;
    const int slot_elems = row_stride + 32;   // row, kPPG weights, padded to 128 bytes
    const size_t slot_bytes = (size_t)slot_elems * sizeof(float) + 16;
    const int S = (int)std::min<size_t>(8, target / slot_bytes);
    used = S >= 2;
    if (!used) return cudaSuccess;
    const size_t smem = (size_t)S * slot_elems * sizeof(float) + 16 * (size_t)S;
    auto kern = hx_ppcore_kernel<K, NW, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 0, per = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, Dv.dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, (NW + 1) * 32, smem)) != cudaSuccess) return e;
    const int grid = std::max(1, std::min(Dv.nppunits, nsm * std::max(per, 1)));
    PPArgs A{Dv.ppunits, Dv.pps_row, Dv.pps_w32, Dv.blocks, Dv.err, Dv.nppunits, S, row_stride, slot_elems,
             (int64_t)ctx->basis.dim * K};
    kern<<<grid, (NW + 1) * 32, smem, s>>>(A, x, part);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_core_k(const bs_ctx *ctx, const float *x, float *part, cudaStream_t s, int v, bool &used)
{
    const CoreVariant P = kCoreVariants[v];
    if (P.nw == 18) return launch_core_t<K, 18, 1>(ctx, x, part, s, P.target, used);
    return launch_core_t<K, 10, 2>(ctx, x, part, s, P.target, used);
}

// partial vectors: Z of the pn kernel, C(Z,2) of the pp kernel, one of the
// like-particle kernel
size_t part_bytes(const bs_ctx *c, int k)
{
    return (size_t)(c->dev.nz + c->dev.nzpp + 1) * (size_t)c->basis.dim * (size_t)k * sizeof(float);
}

bool core_applies(const bs_ctx *c, int k, bs_dtype dt)
{
    return dt == BS_F32 && (k == 4 || k == 8) && c->dev.ncunits > 0 && c->dev.nz > 0;
}

}  // namespace

int core_variants() { return kNumCore; }

int prepare_hx(const bs_ctx *c, int k, bs_dtype dt, std::string &err)
{
    if (!core_applies(c, k, dt)) return BS_OK;
    const size_t need = part_bytes(c, k);
    if (c->core_part_bytes >= need) return BS_OK;
    if (c->core_part) cudaFree(c->core_part);
    c->core_part = nullptr;
    c->core_part_bytes = 0;
    cudaError_t e = cudaMalloc(&c->core_part, need);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        c->core_part = nullptr;
        err = std::string("core partial buffer: ") + cudaGetErrorString(e);
        return BS_ENOMEM;
    }
    c->core_part_bytes = need;
    return BS_OK;
}

// Core-grouped pn kernel variant v followed by the pipelined like-particle
// kernel (variant 0) that adds the partials; `used` is false when the path
// does not apply (FP64, k < 4, no cores) or does not fit.
cudaError_t launch_hx_core(const bs_ctx *c, const void *x, void *y, int k, bs_dtype dt, cudaStream_t s, int v,
                           bool &used, cudaEvent_t t0, cudaEvent_t t1)
{
    used = false;
    if (!core_applies(c, k, dt) || v < 0 || v >= kNumCore) return cudaSuccess;
    if (c->core_part_bytes < part_bytes(c, k)) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(s, &cap);
        if (e != cudaSuccess) return e;
        std::string err;
        if (cap != cudaStreamCaptureStatusNone || prepare_hx(c, k, dt, err) != BS_OK) return cudaSuccess;
    }
    const bool pp = kCoreVariants[v].pp;
    const int R = kCoreVariants[v].nn_rows;
    bool fits = false;
    cudaError_t e = R ? (k == 8 ? launch_nn_k<8>(c, nullptr, nullptr, s, R, fits) : launch_nn_k<4>(c, nullptr, nullptr, s, R, fits))
                      : launch_hx_pipe_combine(c, nullptr, nullptr, k, dt, s, 0, nullptr, 0, pp, fits);
    if (e != cudaSuccess || !fits) return e;
    float *part = (float *)c->core_part;
    const float *xf = (const float *)x;
    if (t0 && (e = cudaEventRecord(t0, s)) != cudaSuccess) return e;
    e = k == 8 ? launch_core_k<8>(c, xf, part, s, v, used) : launch_core_k<4>(c, xf, part, s, v, used);
    if (e != cudaSuccess || !used) return e;
    if (t1 && (e = cudaEventRecord(t1, s)) != cudaSuccess) return e;
    int nz = c->dev.nz;
    if (pp) {
        if (c->dev.nppunits > 0) {
            e = k == 8 ? launch_pp_t<8, 18, 1>(c, xf, part, s, kCoreVariants[v].target, used)
                       : launch_pp_t<4, 18, 1>(c, xf, part, s, kCoreVariants[v].target, used);
            if (e != cudaSuccess) return e;
            if (!used) return cudaErrorInvalidConfiguration;   // the pn kernel with the same budget fitted
        }
        nz += c->dev.nzpp;
    }
    // remaining like-particle terms into partial vector nz, then the ordered sum
    float *last = part + (size_t)nz * (size_t)c->basis.dim * (size_t)k;
    e = R ? (k == 8 ? launch_nn_k<8>(c, xf, last, s, R, used) : launch_nn_k<4>(c, xf, last, s, R, used))
          : launch_hx_pipe_combine(c, x, y, k, dt, s, 0, part, -1 - nz, pp, used);
    if (e != cudaSuccess || !used) return e;
    const int64_t n4 = c->basis.dim * k / 4;
    int nsm = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->dev.dev)) != cudaSuccess) return e;
    const int64_t want = (n4 + 255) / 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * 8));
    hx_sum_partials<<<grid, 256, 0, s>>>(reinterpret_cast<const float4 *>(part), nz + 1, n4, reinterpret_cast<float4 *>(y));
    return cudaGetLastError();
}

}  // namespace bs
