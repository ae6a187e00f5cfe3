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
                                   const void *part, int nz, bool &used);

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

struct CoreVariant {
    int nw, minb;
    size_t target;   // shared-memory budget per CTA
};

constexpr CoreVariant kCoreVariants[] = {{18, 1, 200 * 1024}, {10, 2, 105 * 1024}};
constexpr int kNumCore = 2;

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

template <int K>
cudaError_t launch_core_k(const bs_ctx *ctx, const float *x, float *part, cudaStream_t s, int v, bool &used)
{
    const CoreVariant P = kCoreVariants[v];
    if (P.nw == 18) return launch_core_t<K, 18, 1>(ctx, x, part, s, P.target, used);
    return launch_core_t<K, 10, 2>(ctx, x, part, s, P.target, used);
}

size_t part_bytes(const bs_ctx *c, int k) { return (size_t)c->dev.nz * (size_t)c->basis.dim * (size_t)k * sizeof(float); }

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
                           bool &used)
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
    bool fits = false;
    cudaError_t e = launch_hx_pipe_combine(c, nullptr, nullptr, k, dt, s, 0, nullptr, c->dev.nz, fits);
    if (e != cudaSuccess || !fits) return e;
    float *part = (float *)c->core_part;
    e = k == 8 ? launch_core_k<8>(c, (const float *)x, part, s, v, used)
                           : launch_core_k<4>(c, (const float *)x, part, s, v, used);
    if (e != cudaSuccess || !used) return e;
    return launch_hx_pipe_combine(c, x, y, k, dt, s, 0, part, c->dev.nz, used);
}

}  // namespace bs
