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
#include <type_traits>

#include "bs_internal.h"
#include "bs_tma.cuh"

namespace bs {

using namespace tma;

cudaError_t launch_hx_pipe_combine(const bs_ctx *c, const void *x, void *y, int k, bs_dtype dt, cudaStream_t s, int v,
                                   const void *part, int nz, bool skip_pp, bool &used);

namespace {

// One list entry of one destination column: the gathered element of the
// staged source row times the weights of the entry's weight row, for the
// unit's first R destination rows (its rows are packed to the front; R = 4
// also serves units with three).  The source's weight table has rows of R
// floats.  Entries are src | W row << 16.  For K = 8
// the lane reads the element's 16-byte chunks in its own fixed order (XA
// and XB are the staged row shifted to the lane's first and second chunk),
// so the accumulators hold the components in that order and are put back
// in order once, at the store.
template <int K, int R = 4>
__device__ __forceinline__ void core_step(const float *XA, const float *XB, const float *Wt, uint32_t en,
                                          float2 (&acc)[4][K / 2])
{
    const float *wr = Wt + R * (en >> 16);
    const uint32_t src = en & 0xFFFFu;
    float2 xv[K / 2];
    {
        const float4 a = *reinterpret_cast<const float4 *>(XA + (size_t)src * K);
        xv[0] = make_float2(a.x, a.y);
        xv[1] = make_float2(a.z, a.w);
        if constexpr (K == 8) {
            const float4 b = *reinterpret_cast<const float4 *>(XB + (size_t)src * K);
            xv[2] = make_float2(b.x, b.y);
            xv[3] = make_float2(b.z, b.w);
        }
    }
    // two correctly rounded fused multiply-adds per instruction
    if constexpr (R == 1) {
        const float w = *wr;
        const float2 w0 = make_float2(w, w);
#pragma unroll
        for (int qq = 0; qq < K / 2; ++qq) acc[0][qq] = __ffma2_rn(w0, xv[qq], acc[0][qq]);
    } else if constexpr (R == 2) {
        const float2 w = *reinterpret_cast<const float2 *>(wr);
        const float2 w0 = make_float2(w.x, w.x), w1 = make_float2(w.y, w.y);
#pragma unroll
        for (int qq = 0; qq < K / 2; ++qq) {
            acc[0][qq] = __ffma2_rn(w0, xv[qq], acc[0][qq]);
            acc[1][qq] = __ffma2_rn(w1, xv[qq], acc[1][qq]);
        }
    } else {
        const float4 w = *reinterpret_cast<const float4 *>(wr);
        const float2 w0 = make_float2(w.x, w.x), w1 = make_float2(w.y, w.y);
        const float2 w2 = make_float2(w.z, w.z), w3 = make_float2(w.w, w.w);
#pragma unroll
        for (int qq = 0; qq < K / 2; ++qq) {
            acc[0][qq] = __ffma2_rn(w0, xv[qq], acc[0][qq]);
            acc[1][qq] = __ffma2_rn(w1, xv[qq], acc[1][qq]);
            acc[2][qq] = __ffma2_rn(w2, xv[qq], acc[2][qq]);
            acc[3][qq] = __ffma2_rn(w3, xv[qq], acc[3][qq]);
        }
    }
}

// Stage c % S and round c / S of a running slot counter c, kept up to date
// without integer divisions (S is a launch parameter).
struct SlotRing {
    int s = 0, round = 0;
    __device__ __forceinline__ void next(int S)
    {
        if (++s == S) {
            s = 0;
            ++round;
        }
    }
};

struct CoreArgs {
    int *next;         // units claimed beyond the first grid's worth (zeroed before the launch), or null: static
    const CoreUnit *units;
    const CoreSrc *src;
    const int32_t *perm;
    const int32_t *sinfo;
    const uint32_t *ent;
    int *err;
    int nunits;
    int S;             // ring slots
    int row_stride;    // floats per staged row (multiple of 32)
    int wtab;          // floats per weight table (2 wsign x 4)
    int slot_elems;    // row_stride + wtab + 16 (the slot's CoreSrc, then the unit's rows and ranks)
    int list_elems;    // entries per list buffer (multiple of 32)
    int nlb;           // list buffers (2..4)
    uint32_t ws;       // wsign
    int64_t part_stride;   // dim * K
};

// Shared memory: S slots [source row | weight table | CoreSrc | the unit's
// drow and meta (only in a tile's last slot, which the consumers keep until
// they have stored the tile)], nlb list buffers (one link's neutron lists for
// the tile's slices) with their slice info, then the barriers: full[S],
// empty[S], list_empty[nlb], then one int per slot: the next unit (written
// into a unit's first slot).  A "group" is a
// run of slots of one tile that share a link; its lists arrive with its first
// slot, in buffer (group % nlb), and each consumer warp releases the buffer
// when it starts the next group, so the producer can run nlb - 1 groups ahead.
// CPT = 1: consumer warp w owns 32-column slice w of the tile; CPT = 2: it
// owns slices w and ns - 1 - w (ns slices in the tile), a long and a short
// list in the sector's list-length order, which balances the warps' work.
template <int K, int NW, int MINB, int CPT>
__global__ void __launch_bounds__((NW + 1) * 32, MINB)
    hx_core_kernel(CoreArgs A, const float *__restrict__ wc, const float *__restrict__ x, float *__restrict__ part)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int SL = NW * CPT;                      // slices per tile
    constexpr int C = SL * 32;                        // columns per tile
    constexpr int SI = ((2 * SL + 3) / 4) * 4;        // slice-info ints per buffer
    float *slots = reinterpret_cast<float *>(smem);
    uint32_t *lists = reinterpret_cast<uint32_t *>(slots + (size_t)A.S * A.slot_elems);
    int32_t *sinf = reinterpret_cast<int32_t *>(lists + (size_t)A.nlb * A.list_elems);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sinf + A.nlb * SI);
    int *uidp = reinterpret_cast<int *>(bars + 2 * A.S + A.nlb);   // per slot: the unit after the current one
    const uint32_t full0 = su32(bars), empty0 = su32(bars + A.S), lempty0 = su32(bars + 2 * A.S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < A.S; ++s) {
            bar_init(full0 + 8u * s, 1);
            bar_init(empty0 + 8u * s, NW);
        }
        for (int b = 0; b < A.nlb; ++b) bar_init(lempty0 + 8u * b, NW);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == NW) {
        // ---------------- producer: lane 0 streams every unit's sources, tile by tile;
        // the warp's 32 lanes fetch the metadata of 32 sources at a time
        SlotRing rg;
        int gb = 0, ground = 0;   // list buffer and its use number for the next group (g + 1)
        // the unit record is read one unit ahead
        int hn = 0, hN = 0;
        int64_t hs = 0;
        if (blockIdx.x < A.nunits) {
            hn = A.units[blockIdx.x].nsrc;
            hN = A.units[blockIdx.x].nN;
            hs = A.units[blockIdx.x].src0;
        }
        // units: blockIdx.x first, then each one claims the next (a counter shared by
        // the CTAs, offset by the grid, or blockIdx.x + grid, + 2 grid, ... without
        // one); the next unit rides in the current unit's first slot to the consumers
        for (int u = blockIdx.x, un = 0; u < A.nunits; u = un) {
            const int nsrc = hn, nN = hN;
            const int64_t src0 = hs;
            {
                int v = 0;
                if (lane == 0) v = A.next ? (int)gridDim.x + atomicAdd(A.next, 1) : u + (int)gridDim.x;
                un = __shfl_sync(0xffffffffu, v, 0);
            }
            if (un < A.nunits) {
                hn = A.units[un].nsrc;
                hN = A.units[un].nN;
                hs = A.units[un].src0;
            }
            const int nsl = (nN + 31) / 32;
            const int ntile = (nN + C - 1) / C;
            for (int tile = 0; tile < ntile; ++tile) {
                const int sl0 = tile * SL, sl1 = min(nsl, sl0 + SL);
                int64_t prev = -1;
                if (nsrc == 0) {   // no sources: one empty slot per tile (the first carries the next unit)
                    int bad = 0;
                    if (lane == 0) {
                        const int s = rg.s;
                        if (rg.round > 0 && bar_wait(empty0 + 8u * s, (uint32_t)(rg.round - 1) & 1u)) {
                            bad = 1;
                        } else {   // the slot brings the unit's rows and partial ranks (the store needs them)
                            uidp[s] = un;
                            const uint32_t fb = full0 + 8u * s;
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                            bar_expect_tx(fb, 32u);
                            bulk_copy(su32(slots + (size_t)s * A.slot_elems + A.row_stride + A.wtab + 8), A.units[u].drow, 32u,
                                      fb);
                        }
                    }
                    if (__shfl_sync(0xffffffffu, bad, 0)) {
                        if (lane == 0) {
                            atomicExch(A.err, BS_ETIMEOUT);
                            drain_ring(full0, A.S, (int64_t)rg.round * A.S + rg.s);
                        }
                        return;
                    }
                    rg.next(A.S);
                }
                for (int q0 = 0; q0 < nsrc; q0 += 32) {
                    const int qm = q0 + lane;
                    int64_t mx = 0, msb = -1, mof = 0, mol = 0;
                    int mn = 0, mlm = 0;
                    uint32_t mw = 0;
                    if (qm < nsrc) {
                        const CoreSrc cs = A.src[src0 + qm];
                        mx = cs.x_elem;
                        mn = cs.nN;
                        mw = cs.wtab;
                        msb = cs.sinfo_base;
                        mof = cs.ent_base + A.sinfo[cs.sinfo_base + 2 * sl0];
                        mol = A.sinfo[cs.sinfo_base + 2 * sl0];
                        mlm = A.sinfo[cs.sinfo_base + 2 * (sl1 - 1)] + 32 * A.sinfo[cs.sinfo_base + 2 * (sl1 - 1) + 1];
                    }
                    const int cnt = min(32, nsrc - q0);
                    for (int j = 0; j < cnt; ++j, rg.next(A.S)) {
                        const int64_t xe = __shfl_sync(0xffffffffu, mx, j);
                        const int sn = __shfl_sync(0xffffffffu, mn, j);
                        const uint32_t wt = __shfl_sync(0xffffffffu, mw, j);
                        const int64_t sb = __shfl_sync(0xffffffffu, msb, j);
                        const int64_t lsrc = __shfl_sync(0xffffffffu, mof, j);   // first list entry of the tile
                        const int64_t o0 = __shfl_sync(0xffffffffu, mol, j);
                        const int lend = __shfl_sync(0xffffffffu, mlm, j);        // end of the tile's list block
                        const bool newg = sb != prev;
                        int bad = 0;
                        if (lane == 0) {
                            const int s = rg.s;
                            const int round = rg.round;
                            if (round > 0 && bar_wait(empty0 + 8u * s, (uint32_t)(round - 1) & 1u)) bad = 1;
                            uint32_t lbytes = 0, sbytes = 0;
                            const int b = gb;
                            if (!bad && newg) {
                                // use `ground` of buffer b waits for the consumers' release of use ground - 1
                                if (ground > 0 && bar_wait(lempty0 + 8u * b, (uint32_t)(ground - 1) & 1u)) bad = 1;
                                lbytes = (uint32_t)((lend - o0) * 4);
                                sbytes = (uint32_t)(((2 * (sl1 - sl0) + 3) / 4) * 16);
                            }
                            if (!bad) {
                                const uint32_t bytes = (uint32_t)(sn * K * (int)sizeof(float));
                                const uint32_t wbytes = (uint32_t)(A.wtab * (int)sizeof(float));
                                float *dst = slots + (size_t)s * A.slot_elems;
                                const uint32_t fb = full0 + 8u * s;
                                if (tile == 0 && q0 + j == 0) uidp[s] = un;   // published by the arrive below
                                // the tile's last slot also brings the unit's rows and partial ranks
                                const uint32_t rbytes = q0 + j == nsrc - 1 ? 32u : 0u;
                                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                                bar_expect_tx(fb, bytes + wbytes + 32u + rbytes + lbytes + sbytes);
                                bulk_copy(su32(dst), x + xe * K, bytes, fb);
                                bulk_copy(su32(dst + A.row_stride), wc + (size_t)(wt & 0x7FFFFFFFu) * A.wtab, wbytes, fb);
                                bulk_copy(su32(dst + A.row_stride + A.wtab), A.src + src0 + q0 + j, 32u, fb);
                                if (rbytes) bulk_copy(su32(dst + A.row_stride + A.wtab + 8), A.units[u].drow, rbytes, fb);
                                if (newg) {
                                    if (lbytes) bulk_copy(su32(lists + (size_t)b * A.list_elems), A.ent + lsrc, lbytes, fb);
                                    bulk_copy(su32(sinf + b * SI), A.sinfo + sb + 2 * sl0, sbytes, fb);
                                }
                            }
                        }
                        if (__shfl_sync(0xffffffffu, bad, 0)) {
                            if (lane == 0) {
                                atomicExch(A.err, BS_ETIMEOUT);
                                drain_ring(full0, A.S, (int64_t)rg.round * A.S + rg.s);
                            }
                            return;
                        }
                        if (newg) {
                            prev = sb;
                            if (++gb == A.nlb) {
                                gb = 0;
                                ++ground;
                            }
                        }
                    }
                }
            }
        }
        return;
    }

    // ---------------- consumers
    SlotRing rg;
    int cb = -1;   // list buffer of the current group (none yet)
    const int rot = K == 8 ? (lane >> 2) & 1 : 0;   // this lane's first 16-byte chunk of an element
    // the unit record, read one unit ahead (consumed only in the next unit)
    int hn = 0, hN = 0, hp = 0, hd1 = -1, hd2 = -1;
    int64_t ho = 0;
    if (blockIdx.x < A.nunits) {
        const CoreUnit *U = A.units + blockIdx.x;
        hn = U->nsrc; hN = U->nN; hp = U->perm_off; ho = U->doff; hd1 = U->drow[1]; hd2 = U->drow[2];
    }
    for (int u = blockIdx.x, un = A.nunits; u < A.nunits; u = un) {
        const int nsrc = hn, nN = hN, perm_off = hp;
        const int64_t doff = ho;
        // destination rows of the unit (packed to the front): 1, 2 or more
        const int nrow = hd1 < 0 ? 1 : hd2 < 0 ? 2 : 4;
        const int nsl = (nN + 31) / 32;
        const int ntile = (nN + C - 1) / C;
        for (int tile = 0; tile < ntile; ++tile) {
            const int nst = min(SL, nsl - tile * SL);   // slices in this tile
            // this warp's slices (warp-uniform): sa always, sb only when CPT = 2
            const int sa = warp, sb = CPT == 2 ? nst - 1 - warp : -1;
            const bool hasA = CPT == 2 ? sa <= sb : sa < nst;
            const bool hasB = CPT == 2 && sa < sb;
            const int posA = tile * C + sa * 32 + lane, posB = tile * C + sb * 32 + lane;
            const int colA = hasA && posA < nN ? A.perm[perm_off + posA] : -1;
            const int colB = hasB && posB < nN ? A.perm[perm_off + posB] : -1;
            // packed accumulators: acc[p][j] holds components 2j, 2j+1 of destination row p
            // (for K = 8 in the lane's chunk order)
            float2 accA[4][K / 2], accB[4][K / 2];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < K / 2; ++q) accA[p][q] = accB[p][q] = make_float2(0.0f, 0.0f);
            int64_t prev = -1;
            int la = 0, lb = 0;
            const uint32_t *lstA = lists, *lstB = lists;
            int ls = 0;   // the tile's last slot: kept until the store, which reads the unit's rows from it
            // a unit without sources still takes one (empty) slot per tile; the first has the next unit
            for (int q = 0; q < nsrc || (nsrc == 0 && q == 0); ++q, rg.next(A.S)) {
                const int s = rg.s;
                if (__any_sync(0xffffffffu, bar_wait(full0 + 8u * s, (uint32_t)rg.round & 1u))) {
                    if (lane == 0) atomicExch(A.err, BS_ETIMEOUT);
                    return;
                }
                if (tile == 0 && q == 0) {   // the next unit: read its record now, use it after this one
                    un = uidp[s];
                    if (un < A.nunits) {
                        const CoreUnit *U = A.units + un;
                        hn = U->nsrc; hN = U->nN; hp = U->perm_off; ho = U->doff; hd1 = U->drow[1]; hd2 = U->drow[2];
                    }
                }
                const bool last = q == (nsrc > 0 ? nsrc : 1) - 1;
                if (last) ls = s;
                if (nsrc == 0) continue;
                const float *Xs = slots + (size_t)s * A.slot_elems;
                const float *Wt = Xs + A.row_stride;
                const CoreSrc *cs = reinterpret_cast<const CoreSrc *>(Wt + A.wtab);
                const int64_t sbase = cs->sinfo_base;
                const float *XA = Xs + 4 * rot, *XB = Xs + 4 * (rot ^ 1);
                if (sbase != prev) {
                    // a new group: release the previous group's list buffer, read this one
                    __syncwarp();
                    if (cb >= 0 && lane == 0) bar_arrive(lempty0 + 8u * cb);
                    cb = cb + 1 == A.nlb ? 0 : cb + 1;
                    prev = sbase;
                    const int b = cb;
                    const int32_t *si = sinf + b * SI;
                    const uint32_t *lb0 = lists + (size_t)b * A.list_elems - si[0] + lane;
                    la = hasA ? si[2 * sa + 1] : 0;
                    lb = hasB ? si[2 * sb + 1] : 0;
                    lstA = lb0 + (hasA ? si[2 * sa] : 0);
                    lstB = lb0 + (hasB ? si[2 * sb] : 0);
                }
                // entries straight from the staged lists (32 lanes, 128 contiguous bytes per step)
                if constexpr (CPT == 1) {
                    // one slice: the plain loop, for the unit's number of rows
                    if (nrow == 1) {
#pragma unroll 4
                        for (int v = 0; v < la; ++v) core_step<K, 1>(XA, XB, Wt, lstA[32 * v], accA);
                    } else if (nrow == 2) {
#pragma unroll 4
                        for (int v = 0; v < la; ++v) core_step<K, 2>(XA, XB, Wt, lstA[32 * v], accA);
                    } else {
#pragma unroll 4
                        for (int v = 0; v < la; ++v) core_step<K, 4>(XA, XB, Wt, lstA[32 * v], accA);
                    }
                } else {
                    // two slices, for the unit's number of rows (the weight rows are R floats)
                    auto run = [&](auto rt) {
                        constexpr int R = decltype(rt)::value;
                        const int lm = min(la, lb);
                        int v = 0;
                        for (; v < lm; ++v) {
                            core_step<K, R>(XA, XB, Wt, lstA[32 * v], accA);
                            core_step<K, R>(XA, XB, Wt, lstB[32 * v], accB);
                        }
#pragma unroll 2
                        for (int va = v; va < la; ++va) core_step<K, R>(XA, XB, Wt, lstA[32 * va], accA);
#pragma unroll 2
                        for (int vb = v; vb < lb; ++vb) core_step<K, R>(XA, XB, Wt, lstB[32 * vb], accB);
                    };
                    if (nrow == 1) run(std::integral_constant<int, 1>{});
                    else if (nrow == 2) run(std::integral_constant<int, 2>{});
                    else run(std::integral_constant<int, 4>{});
                }
                if (last) continue;   // released after the store
                __syncwarp();
                if (lane == 0) bar_arrive(empty0 + 8u * s);
            }
            // the unit's destination rows and partial ranks, brought by its last slot
            const int *rec = reinterpret_cast<const int *>(slots + (size_t)ls * A.slot_elems + A.row_stride + A.wtab + 8);
            auto store = [&](int col, float2 (&acc)[4][K / 2]) {
                if (col < 0) return;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const int drow = rec[p], meta = rec[4 + p];
                    if (drow < 0) continue;
                    const float sg = (meta & 256) ? -1.0f : 1.0f;
                    float o[K];
#pragma unroll
                    for (int qq = 0; qq < K / 2; ++qq) {
                        // K = 8: the lane's chunk order back to component order
                        const float2 a = K == 8 ? (rot ? acc[p][qq ^ 2] : acc[p][qq]) : acc[p][qq];
                        o[2 * qq] = sg * a.x;
                        o[2 * qq + 1] = sg * a.y;
                    }
                    pst<float, K>(part + (int64_t)(meta & 255) * A.part_stride + (doff + (int64_t)drow * nN + col) * K, o);
                }
            };
            store(colA, accA);
            if (CPT == 2) store(colB, accB);
            __syncwarp();
            if (lane == 0) bar_arrive(empty0 + 8u * ls);   // the last slot, now that its record is read
        }
    }
}

struct PPArgs {
    int *next;             // as CoreArgs::next
    const PPUnit *units;
    const int32_t *srow;
    const float *w;        // kPPG weights per source
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
    int *uidp = reinterpret_cast<int *>(bars + 2 * A.S);   // per slot: the unit after the current one
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
        // lane 0 issues the copies; the warp's lanes fetch the source rows of
        // 32 sources at a time, so no copy waits on a dependent global load
        SlotRing rg;
        // the unit record is read one unit ahead
        int hn = 0, hN = 0;
        int64_t hs = 0, ho = 0;
        if (blockIdx.x < A.nunits) {
            hn = A.units[blockIdx.x].nsrc; hN = A.units[blockIdx.x].nN;
            hs = A.units[blockIdx.x].src0; ho = A.units[blockIdx.x].doff;
        }
        // units claimed as in the pn kernel; the next one rides in the first slot
        for (int u = blockIdx.x, un = 0; u < A.nunits; u = un) {
            const int nsrc = hn, nN = hN;
            const int64_t src0 = hs, doff = ho;
            {
                int v = 0;
                if (lane == 0) v = A.next ? (int)gridDim.x + atomicAdd(A.next, 1) : u + (int)gridDim.x;
                un = __shfl_sync(0xffffffffu, v, 0);
            }
            if (un < A.nunits) {
                hn = A.units[un].nsrc; hN = A.units[un].nN;
                hs = A.units[un].src0; ho = A.units[un].doff;
            }
            if (nsrc == 0) {   // no sources: one empty slot carries the next unit
                int bad = 0;
                if (lane == 0) {
                    const int s = rg.s;
                    if (rg.round > 0 && bar_wait(empty0 + 8u * s, (uint32_t)(rg.round - 1) & 1u)) {
                        bad = 1;
                    } else {
                        uidp[s] = un;
                        bar_arrive(full0 + 8u * s);
                    }
                }
                if (__shfl_sync(0xffffffffu, bad, 0)) {
                    if (lane == 0) {
                        atomicExch(A.err, BS_ETIMEOUT);
                        drain_ring(full0, A.S, (int64_t)rg.round * A.S + rg.s);
                    }
                    return;
                }
                rg.next(A.S);
            }
            const int ntile = (nN + C - 1) / C;
            const uint32_t bytes = (uint32_t)(nN * K * (int)sizeof(float));
            const uint32_t wbytes = (uint32_t)(kPPG * sizeof(float));
            for (int tile = 0; tile < ntile; ++tile)
                for (int q0 = 0; q0 < nsrc; q0 += 32) {
                    const int32_t myrow = q0 + lane < nsrc ? A.srow[src0 + q0 + lane] : 0;
                    const int cnt = min(32, nsrc - q0);
                    for (int j = 0; j < cnt; ++j, rg.next(A.S)) {
                        const int32_t row = __shfl_sync(0xffffffffu, myrow, j);
                        int bad = 0;
                        if (lane == 0) {
                            const int s = rg.s;
                            const int round = rg.round;
                            if (round > 0 && bar_wait(empty0 + 8u * s, (uint32_t)(round - 1) & 1u)) {
                                bad = 1;
                            } else {
                                const uint32_t fb = full0 + 8u * s;
                                float *dst = slots + (size_t)s * A.slot_elems;
                                if (tile == 0 && q0 + j == 0) uidp[s] = un;   // published by the arrive below
                                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                                bar_expect_tx(fb, bytes + wbytes);
                                bulk_copy(su32(dst), x + (doff + (int64_t)row * nN) * K, bytes, fb);
                                bulk_copy(su32(dst + A.row_stride), A.w + (src0 + q0 + j) * kPPG, wbytes, fb);
                            }
                        }
                        if (__shfl_sync(0xffffffffu, bad, 0)) {
                            if (lane == 0) {
                                atomicExch(A.err, BS_ETIMEOUT);
                                drain_ring(full0, A.S, (int64_t)rg.round * A.S + rg.s);
                            }
                            return;
                        }
                    }
                }
        }
        return;
    }

    constexpr int E = K * (int)sizeof(float);
    const int rot = E == 32 ? ((lane >> 2) & 1) : 0;
    SlotRing rg;
    // the unit record is read one unit ahead; lane p < kPPG keeps destination
    // row p and its partial rank, packed as drow << 8 | part (-1: no row; the
    // host keeps drow < 2^23 and part < 256), until the store
    auto packed = [&](const PPUnit *U) {
        if (lane >= kPPG) return 0;
        const int d = U->drow[lane];
        return d < 0 ? -1 : (d << 8) | U->part[lane];
    };
    int hn = 0, hN = 0, hrec = 0;
    int64_t ho = 0;
    if (blockIdx.x < A.nunits) {
        const PPUnit *U = A.units + blockIdx.x;
        hn = U->nsrc; hN = U->nN; ho = U->doff;
        hrec = packed(U);
    }
    for (int u = blockIdx.x, un = A.nunits; u < A.nunits; u = un) {
        const int nsrc = hn, nN = hN, rec = hrec;
        const int64_t doff = ho;
        const int ntile = (nN + C - 1) / C;
        for (int tile = 0; tile < ntile; ++tile) {
            const int col = tile * C + warp * 32 + lane;
            const bool active = tile * C + warp * 32 < nN;
            const int cl = col < nN ? col : nN - 1;
            float2 acc[kPPG][K / 2];   // packed: components 2j, 2j+1 (in the lane's rotated order)
#pragma unroll
            for (int p = 0; p < kPPG; ++p)
#pragma unroll
                for (int q = 0; q < K / 2; ++q) acc[p][q] = make_float2(0.0f, 0.0f);
            // a unit without sources still takes one (empty) slot: the one with the next unit
            for (int q = 0; q < nsrc || (nsrc == 0 && tile == 0 && q == 0); ++q, rg.next(A.S)) {
                const int s = rg.s;
                if (__any_sync(0xffffffffu, bar_wait(full0 + 8u * s, (uint32_t)rg.round & 1u))) {
                    if (lane == 0) atomicExch(A.err, BS_ETIMEOUT);
                    return;
                }
                if (tile == 0 && q == 0) {   // the next unit: read its record now, use it after this one
                    un = uidp[s];
                    if (un < A.nunits) {
                        const PPUnit *U = A.units + un;
                        hn = U->nsrc; hN = U->nN; ho = U->doff;
                        hrec = packed(U);
                    }
                }
                if (active && nsrc > 0) {
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
                    for (int p = 0; p < kPPG; ++p) {
                        const float2 wp = make_float2(w[p], w[p]);
#pragma unroll
                        for (int qq = 0; qq < K / 2; ++qq)
                            acc[p][qq] = __ffma2_rn(wp, make_float2(xv[2 * qq], xv[2 * qq + 1]), acc[p][qq]);
                    }
                }
                __syncwarp();
                if (lane == 0) bar_arrive(empty0 + 8u * s);
            }
            // every lane takes part in the shuffles; only columns inside the block store
#pragma unroll
            for (int p = 0; p < kPPG; ++p) {
                const int pk = __shfl_sync(0xffffffffu, rec, p);
                if (col < nN) {
                    if (pk < 0) continue;
                    const int drow = pk >> 8, prt = pk & 255;
                    float o[K];
#pragma unroll
                    for (int qq = 0; qq < K / 2; ++qq) {
                        o[2 * qq] = acc[p][qq].x;
                        o[2 * qq + 1] = acc[p][qq].y;
                    }
                    prot_fix<float, K>(o, rot);
                    pst<float, K>(part + (int64_t)prt * A.part_stride + (doff + (int64_t)drow * nN + col) * K, o);
                }
            }
        }
    }
}

struct NNArgs {
    int stage;           // 1: results staged in shared memory, then summed and stored in column order
    const int2 *tasks;
    const DevBlock *blocks;
    const int32_t *perm;
    const int32_t *src;
    const float *coef;
    const int32_t *sinfo;
    const float *pdiag;
    int *err;
    int row_stride;
    const float *part;   // the other terms' partial vectors (nz of them, pstride apart), summed in, or null
    int nz;
    int64_t pstride;
};

// Neutron like-particle term plus the proton single-particle diagonal over a
// tile of R consecutive proton rows of one block: y[r][n'] = e_p(r) x[r][n'] +
// sum_v c_v x[r][n_v].  The neutron lists are the same for every proton row,
// so each thread (one destination column, in the sector's list order) loads
// an entry once and applies it to the R staged rows.  The R rows arrive by
// TMA bulk copies on one mbarrier (bounded wait).  Output: y itself when the
// other terms' partial vectors are given (their ordered sum, then this term:
// the order of hx_sum_partials, so the result is bit-identical to a separate
// summation pass), else a partial vector.  Threads own columns in the
// sector's list order; with A.stage the tile's results go to shared memory
// first, so that the partial vectors are read and y written in column
// order (whole 128-byte lines per quarter warp instead of scattered 32-byte
// elements).
template <int K, int R, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB)
    hx_nn_rows_kernel(NNArgs A, const float *__restrict__ x, float *__restrict__ out)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float *rows = reinterpret_cast<float *>(smem);
    float *res = rows + (size_t)R * A.row_stride;   // used when A.stage
    uint64_t *bar = reinterpret_cast<uint64_t *>(res + (A.stage ? (size_t)R * A.row_stride : 0));
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
    // one decision for the whole CTA, so that no thread leaves before the
    // barrier of the staged epilogue
    if (__syncthreads_or(bar_wait(b0, 0u) ? 1 : 0)) {
        if (threadIdx.x == 0) {
            atomicExch(A.err, BS_ETIMEOUT);
            (void)bar_wait(b0, 0u);   // the rows' copies: no copy left in flight at exit
        }
        return;
    }
    const int rot = prot<float, K>(lane);
    // column tiles of NW * 32 (one column per thread) over the staged rows
    for (int c0 = 0; c0 < nN; c0 += NW * 32) {
        const int p = c0 + warp * 32 + lane;
        const int sl = c0 / 32 + warp;
        if (sl * 32 >= nN) break;   // warp-uniform
        const int col = p < nN ? A.perm[D.perm_off + p] : -1;
        const int off = A.sinfo[D.pe_nn_sinfo + 2 * sl];
        const int lmax = A.sinfo[D.pe_nn_sinfo + 2 * sl + 1];
        float2 acc[R][K / 2];   // packed, in the lane's rotated component order
        float xv[K];
        const int cc = col >= 0 ? col : 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            pld<float, K>(rows + (size_t)r * A.row_stride, cc, rot, xv);
#pragma unroll
            for (int q = 0; q < K / 2; ++q) acc[r][q] = make_float2(pd[r] * xv[2 * q], pd[r] * xv[2 * q + 1]);
        }
        const int64_t base = D.pe_nn_ent + off + lane;
        // the list streams from global memory (L2): NB entries are loaded at a
        // time, all before any is used, so that NB loads are in flight
        constexpr int NB = (K == 8 || R == 2) ? 4 : 8;
        for (int v0 = 0; v0 < lmax; v0 += NB) {
            float cb[NB];
            int sb[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const bool in = v0 + j < lmax;
                cb[j] = in ? A.coef[base + 32 * (int64_t)(v0 + j)] : 0.0f;
                sb[j] = in ? A.src[base + 32 * (int64_t)(v0 + j)] : 0;
            }
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                if (v0 + j >= lmax) break;
                const float2 c2 = make_float2(cb[j], cb[j]);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    pld<float, K>(rows + (size_t)r * A.row_stride, sb[j], rot, xv);
#pragma unroll
                    for (int q = 0; q < K / 2; ++q) acc[r][q] = __ffma2_rn(c2, make_float2(xv[2 * q], xv[2 * q + 1]), acc[r][q]);
                }
            }
        }
        if (col < 0) continue;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r >= nr) break;
            float o[K];
#pragma unroll
            for (int q = 0; q < K / 2; ++q) {
                o[2 * q] = acc[r][q].x;
                o[2 * q + 1] = acc[r][q].y;
            }
            prot_fix<float, K>(o, rot);
            if (A.stage) {
                pst<float, K>(res + (size_t)r * A.row_stride + (size_t)col * K, o);
                continue;
            }
            const int64_t e = (D.off + (int64_t)(r0 + r) * nN + col) * K;
            if (A.nz > 0) {
                // the partials' sum in the order t = 0 .. nz - 1, with the loads of
                // four partials in flight at a time (the adds stay in order)
                float4 a[K / 4];
#pragma unroll
                for (int q = 0; q < K / 4; ++q) a[q] = __ldg(reinterpret_cast<const float4 *>(A.part + e) + q);
                int t = 1;
                for (; t + 4 <= A.nz; t += 4) {
                    float4 v[4][K / 4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int q = 0; q < K / 4; ++q)
                            v[u][q] = __ldg(reinterpret_cast<const float4 *>(A.part + (int64_t)(t + u) * A.pstride + e) + q);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int q = 0; q < K / 4; ++q) {
                            a[q].x += v[u][q].x; a[q].y += v[u][q].y; a[q].z += v[u][q].z; a[q].w += v[u][q].w;
                        }
                }
                for (; t < A.nz; ++t) {
#pragma unroll
                    for (int q = 0; q < K / 4; ++q) {
                        const float4 v = __ldg(reinterpret_cast<const float4 *>(A.part + (int64_t)t * A.pstride + e) + q);
                        a[q].x += v.x; a[q].y += v.y; a[q].z += v.z; a[q].w += v.w;
                    }
                }
#pragma unroll
                for (int q = 0; q < K / 4; ++q) {
                    o[4 * q] = a[q].x + o[4 * q];
                    o[4 * q + 1] = a[q].y + o[4 * q + 1];
                    o[4 * q + 2] = a[q].z + o[4 * q + 2];
                    o[4 * q + 3] = a[q].w + o[4 * q + 3];
                }
            }
            pst<float, K>(out + e, o);
        }
    }
    if (!A.stage) return;
    __syncthreads();
    // column order, 16 bytes per thread (a warp reads 512 contiguous bytes of
    // every partial): the other terms' partials in the order t = 0 .. nz - 1,
    // then this term (the same additions as the direct path)
    const int n4 = nN * (K / 4);   // float4 units of one row
    for (int r = 0; r < nr; ++r) {
        const int64_t e0 = (D.off + (int64_t)(r0 + r) * nN) * K;
        for (int i = threadIdx.x; i < n4; i += NW * 32) {
            float4 o = *reinterpret_cast<const float4 *>(res + (size_t)r * A.row_stride + 4 * (size_t)i);
            const int64_t e = e0 + 4 * (int64_t)i;
            if (A.nz > 0) {
                float4 a = __ldg(reinterpret_cast<const float4 *>(A.part + e));
                int t = 1;
                for (; t + 4 <= A.nz; t += 4) {
                    float4 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) v[u] = __ldg(reinterpret_cast<const float4 *>(A.part + (int64_t)(t + u) * A.pstride + e));
#pragma unroll
                    for (int u = 0; u < 4; ++u) { a.x += v[u].x; a.y += v[u].y; a.z += v[u].z; a.w += v[u].w; }
                }
                for (; t < A.nz; ++t) {
                    const float4 v = __ldg(reinterpret_cast<const float4 *>(A.part + (int64_t)t * A.pstride + e));
                    a.x += v.x; a.y += v.y; a.z += v.z; a.w += v.w;
                }
                o.x = a.x + o.x; o.y = a.y + o.y; o.z = a.z + o.z; o.w = a.w + o.w;
            }
            *reinterpret_cast<float4 *>(out + e) = o;
        }
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
    int nw, cpt;     // consumer warps, 32-column slices per warp
    size_t target;   // shared-memory budget per CTA
    bool pp;         // pp term by (Z-2)-proton cores, nn by row tiles of nn_rows rows
    int nn_rows;
    int nlb;         // neutron-list buffers (0: three if the ring keeps seven slots, else two)
};

// Modes 11.. in this order.  The last two spend the whole 227 KB on three or
// four list buffers: the producer can then run two or three link groups
// ahead of the slowest consumer warp instead of one.
// Modes 17, 18 also spend 227 KB, with two list buffers, and leave the
// like-particle terms (17: pp and nn; 18: nn, after the pp-core kernel) to
// the first pipelined variant that fits the basis: for source rows of up to
// ~64 KB (pf 6p6n: 3,952 columns of 16 bytes at k = 4).  Mode 19 is 18 with
// the nn term in row tiles of 2 rows (two CTAs per SM); mode 20 pairs those
// 2-row tiles with the three list buffers of mode 15.
constexpr CoreVariant kCoreVariants[] = {{18, 1, 200 * 1024, false, 0, 0}, {9, 2, 200 * 1024, false, 0, 0},
                                         {18, 1, 200 * 1024, true, 4, 0},  {9, 2, 200 * 1024, true, 4, 0},
                                         {18, 1, 227 * 1024, true, 4, 3},  {18, 1, 227 * 1024, true, 4, 4},
                                         {18, 1, 227 * 1024, false, 0, 2}, {18, 1, 227 * 1024, true, 0, 2},
                                         {18, 1, 227 * 1024, true, 2, 2},  {18, 1, 227 * 1024, true, 2, 3}};
constexpr int kNumCore = 10;

template <int K, int R, int MINB>
cudaError_t launch_nn_t(const bs_ctx *ctx, const float *x, float *out, cudaStream_t s, bool &used,
                        const float *part = nullptr, int nz = 0)
{
    const Device &Dv = ctx->dev;
    constexpr int NW = 18;
    const int row_stride = ((Dv.max_nN * K + 31) / 32) * 32;
    const size_t rows_bytes = (size_t)R * row_stride * sizeof(float);
    used = rows_bytes + 16 <= 200 * 1024;   // wider sectors than NW * 32 columns run in column tiles
    if (!used || !x) return cudaSuccess;
    // the results staged beside the rows where both fit one SM's 227 KB
    const int stage = 2 * rows_bytes + 16 <= 227 * 1024 ? 1 : 0;
    const size_t smem = (stage ? 2 : 1) * rows_bytes + 16;
    auto kern = hx_nn_rows_kernel<K, R, NW, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    NNArgs A{stage, R == 2 ? Dv.nntasks2 : Dv.nntasks4, Dv.blocks, Dv.pe_perm, Dv.pe_nn_src, Dv.pe_nn_coef32,
             Dv.pe_nn_sinfo, Dv.pdiag32, Dv.err, row_stride, part, part ? nz : 0, ctx->basis.dim * K};
    kern<<<R == 2 ? Dv.nnntasks2 : Dv.nnntasks4, NW * 32, smem, s>>>(A, x, out);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_nn_k(const bs_ctx *ctx, const float *x, float *out, cudaStream_t s, int R, bool &used,
                       const float *part = nullptr, int nz = 0)
{
    return R == 2 ? launch_nn_t<K, 2, 2>(ctx, x, out, s, used, part, nz)
                  : launch_nn_t<K, 4, 1>(ctx, x, out, s, used, part, nz);
}

template <int K, int NW, int MINB, int CPT>
cudaError_t launch_core_t(const bs_ctx *ctx, const float *x, float *part, cudaStream_t s, size_t target, int nlb_req,
                          bool &used)
{
    const Device &Dv = ctx->dev;
    const int row_stride = ((Dv.max_nN * K + 31) / 32) * 32;
    const int wtab = 8 * Dv.wsign;
    const int slot_elems = row_stride + wtab + 16;   // + the source record (8 floats) and the unit's rows (8)
    const size_t slot_bytes = (size_t)slot_elems * sizeof(float) + 16;
    static_assert(NW * CPT == 18 || NW * CPT == 10, "list bounds are built for tiles of 18 or 10 slices");
    const int64_t lmaxe = Dv.core_list_max[NW * CPT == 18 ? 0 : 1];
    const int list_elems = (int)(((std::max<int64_t>(lmaxe, 32) + 31) / 32) * 32);
    constexpr int SI = ((2 * NW * CPT + 3) / 4) * 4;
    // list buffers: three when the ring still keeps seven slots, else two (a
    // deeper ring pays more than a third buffer)
    int nlb = nlb_req > 0 ? nlb_req : 3, S = 0;
    for (; nlb >= 2; --nlb) {
        const size_t fixed = (size_t)nlb * list_elems * 4 + (size_t)nlb * SI * 4 + 8 * (size_t)nlb + 64;
        S = target > fixed ? (int)std::min<size_t>(8, (target - fixed) / slot_bytes) : 0;
        if (nlb_req > 0 || S >= 7 || nlb == 2) break;
    }
    // (+ 64 bytes: the slots' next-unit words after the barriers, S <= 8)
    const size_t fixed = (size_t)nlb * list_elems * 4 + (size_t)nlb * SI * 4 + 8 * (size_t)nlb + 64;
    used = S >= 2;
    if (!used) return cudaSuccess;
    const size_t smem = (size_t)S * slot_elems * sizeof(float) + fixed + 16 * (size_t)S;
    auto kern = hx_core_kernel<K, NW, MINB, CPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 0, per = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, Dv.dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, (NW + 1) * 32, smem)) != cudaSuccess) return e;
    const int grid = std::max(1, std::min(Dv.ncunits, nsm * std::max(per, 1)));
    CoreArgs A{Dv.core_next, Dv.cunits, Dv.csrc, Dv.pe_perm, Dv.pe_sinfo, Dv.core_ent, Dv.err, Dv.ncunits, S,
               row_stride, wtab, slot_elems, list_elems, nlb, (uint32_t)Dv.wsign, (int64_t)ctx->basis.dim * K};
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
    const int S = target > 64 ? (int)std::min<size_t>(8, (target - 64) / slot_bytes) : 0;
    used = S >= 2;
    if (!used) return cudaSuccess;
    const size_t smem = (size_t)S * slot_elems * sizeof(float) + 16 * (size_t)S + 64;   // + the slots' next-unit words
    auto kern = hx_ppcore_kernel<K, NW, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 0, per = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, Dv.dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, (NW + 1) * 32, smem)) != cudaSuccess) return e;
    const int grid = std::max(1, std::min(Dv.nppunits, nsm * std::max(per, 1)));
    PPArgs A{Dv.core_next ? Dv.core_next + 1 : nullptr, Dv.ppunits, Dv.pps_row, Dv.pps_w32, Dv.err, Dv.nppunits, S, row_stride, slot_elems,
             (int64_t)ctx->basis.dim * K};
    kern<<<grid, (NW + 1) * 32, smem, s>>>(A, x, part);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_core_k(const bs_ctx *ctx, const float *x, float *part, cudaStream_t s, int v, bool &used)
{
    const CoreVariant P = kCoreVariants[v];
    if (P.cpt == 2) return launch_core_t<K, 9, 1, 2>(ctx, x, part, s, P.target, P.nlb, used);
    return launch_core_t<K, 18, 1, 1>(ctx, x, part, s, P.target, P.nlb, used);
}

// partial vectors: Z of the pn kernel, C(Z,2) of the pp kernel, one of the
// like-particle kernel
size_t part_bytes(const bs_ctx *c, int k)
{
    return (size_t)(c->dev.nz + c->dev.nzpp + 1) * (size_t)c->basis.dim * (size_t)k * sizeof(float);
}

bool core_applies(const bs_ctx *c, int k, bs_dtype dt)
{
    return !c->dev.trunc && dt == BS_F32 && (k == 4 || k == 8) && c->dev.ncunits > 0 && c->dev.nz > 0;
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
    cudaError_t e = cudaSuccess;
    int pv = 0;   // pipelined variant for the like-particle terms: the first that fits
    if (R) {
        e = k == 8 ? launch_nn_k<8>(c, nullptr, nullptr, s, R, fits) : launch_nn_k<4>(c, nullptr, nullptr, s, R, fits);
    } else {
        for (; pv < pipe_variants() && e == cudaSuccess; ++pv) {
            e = launch_hx_pipe_combine(c, nullptr, nullptr, k, dt, s, pv, nullptr, 0, pp, fits);
            if (fits) break;
        }
    }
    if (e != cudaSuccess || !fits) return e;
    float *part = (float *)c->core_part;
    const float *xf = (const float *)x;
    // the pn and pp kernels' unit counters start at zero for every product (a memset
    // node in a captured graph), before the timed window of the dominant kernel
    if (c->dev.core_next && (e = cudaMemsetAsync(c->dev.core_next, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
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
    // remaining like-particle terms: the row-tile kernel adds the nz partial
    // vectors in order and writes y itself; else they go into partial
    // vector nz, followed by the ordered sum
    if (R) {
        float *yf = (float *)y;
        e = k == 8 ? launch_nn_k<8>(c, xf, yf, s, R, used, part, nz) : launch_nn_k<4>(c, xf, yf, s, R, used, part, nz);
        if (e != cudaSuccess) return e;
        return used ? cudaGetLastError() : cudaSuccess;
    }
    e = launch_hx_pipe_combine(c, x, y, k, dt, s, pv, part, -1 - nz, pp, used);
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
