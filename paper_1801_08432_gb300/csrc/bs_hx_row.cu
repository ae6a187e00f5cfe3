// Row kernel for y = H x (sm_103a): one CTA per destination proton row ip'
// of a basis block, all neutron columns of that row.
//
// The row of y is accumulated in shared memory and written once.  In order:
//   pp  y[ip',jn'] += sum_{pp jumps ip -> ip'} c x[ip, jn']            (rows of x, coalesced)
//   nn  y[ip',jn'] += sum_{nn jumps jn -> jn'} c x[ip', jn]            (x[ip',:] staged in smem)
//   pn  for each linked source block s (proton class s_p -> s_p', neutron class s_n -> s_n'):
//         y[ip',jn'] += sum_u phi_u sum_v phi_v W[a_u][b_v] x_s[ip_u, jn_v]
//       with the source rows x_s[ip_u, :] of the proton jumps u staged in shared
//       memory by TMA bulk copies (cp.async.bulk + mbarrier), the rows W[a_u][:]
//       (proton sign folded in) in shared memory, and the neutron jumps v of
//       every column read from a length-sorted 32-column ELL so the lanes of a
//       warp run lists of similar length.
// This is the paper's factorization of the pn term (proton one-body jump x
// neutron one-body jump), evaluated as a gather so every output has one owner:
// no atomics, fixed summation order, bit-reproducible results.
//
// Every mbarrier wait is bounded; on expiry the CTA records BS_ETIMEOUT in the
// device status word and returns.
#include <cuda_runtime.h>

#include "bs_internal.h"

namespace bs {

namespace {

constexpr uint32_t kWaitLimit = 1u << 22;   // try_wait rounds before a wait is declared hung
constexpr int kMaxList = 24;                 // neutron lists up to this length are held in registers

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}

// one bulk copy global -> shared, completion counted on the mbarrier
__device__ __forceinline__ void tma_row(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

template <typename T, int K>
__device__ __forceinline__ void ld_vec(const T *p, T (&r)[K])
{
    if constexpr (sizeof(T) * K >= 16) {
        constexpr int W = 16 / sizeof(T);
#pragma unroll
        for (int c = 0; c < K; c += W) {
            if constexpr (sizeof(T) == 4) {
                float4 q = *reinterpret_cast<const float4 *>(p + c);
                r[c] = q.x; r[c + 1] = q.y; r[c + 2] = q.z; r[c + 3] = q.w;
            } else {
                double2 q = *reinterpret_cast<const double2 *>(p + c);
                r[c] = q.x; r[c + 1] = q.y;
            }
        }
    } else if constexpr (sizeof(T) == 4 && K == 2) {
        float2 q = *reinterpret_cast<const float2 *>(p);
        r[0] = q.x; r[1] = q.y;
    } else {
#pragma unroll
        for (int c = 0; c < K; ++c) r[c] = p[c];
    }
}

template <typename T, int K>
__device__ __forceinline__ void ldg_vec(const T *p, T (&r)[K])
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
__device__ __forceinline__ void st_vec(T *p, const T (&r)[K])
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

template <typename T>
__device__ __forceinline__ T flip(T w, uint32_t neg)
{
    return neg ? -w : w;
}

// Elements of 32 (64) bytes are read as 2 (4) 16-byte chunks starting at
// chunk `rot` of the element; rot is fixed per lane (lane parity, or lane mod
// 4), so a warp's first load spreads over all eight 16-byte bank groups.  The
// values land in registers rotated by `rot` and are accumulated that way;
// unrot() puts a finished sum back in order.
template <typename T, int K>
__device__ __forceinline__ int chunk_rot(int lane)
{
    constexpr int E = K * (int)sizeof(T);
    return E == 32 ? (lane & 1) : E == 64 ? (lane & 3) : 0;
}

template <typename T, int K>
__device__ __forceinline__ void ld_rot(const T *row, int jn, int rot, T (&r)[K])
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
    } else {
        ld_vec<T, K>(row + (size_t)jn * K, r);
    }
}

template <typename T, int K>
__device__ __forceinline__ void unrot(T (&r)[K], int rot)
{
    constexpr int E = K * (int)sizeof(T);
    if constexpr (E == 32 || E == 64) {
        constexpr int NC = E / 16, W = 16 / (int)sizeof(T);
        T t[K];
#pragma unroll
        for (int i = 0; i < K; ++i) t[i] = r[i];
        // register chunk c holds element chunk (c + rot) mod NC
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

}  // namespace

struct RowArgs {
    const RowTask *tasks;
    const DevBlock *blocks;
    const DevLink *links;
    const int64_t *pp_ptr;
    const int32_t *pp_src;
    const int64_t *p1_ptr;
    const uint32_t *p1_ent;
    const int32_t *n1e_col, *n1e_len;
    const int64_t *n1e_soff;
    const uint32_t *n1e_ent;
    const int32_t *nne_col, *nne_len, *nne_src;
    const int64_t *nne_soff;
    int *err;
    int uc;           // source rows per staged chunk
    int row_stride;   // elements per staged row slot
    int nb_stride;    // elements per W row slot
    int acc_elems;    // elements of the accumulator row
    int wsign;        // offset of -W inside a W row slot
};

// Position in the sequence of staged chunks of one destination row: link L,
// proton jumps u0 .. u0+cu-1 of that link (pb = first jump's entry index).
struct Chunk {
    int L, u0, cu;
    int64_t pb;
};

template <typename T, int K, int NT>
__global__ void __launch_bounds__(NT) hx_row_kernel(RowArgs A, const T *__restrict__ pp_coef,
                                                    const T *__restrict__ nne_coef, const T *__restrict__ wpn,
                                                    const T *__restrict__ x, T *__restrict__ y)
{
    constexpr bool kBulk = (K * sizeof(T)) % 16 == 0;
    extern __shared__ __align__(128) unsigned char smem[];
    T *Xs = reinterpret_cast<T *>(smem);                          // [2][uc][row_stride]
    T *acc = Xs + (size_t)2 * A.uc * A.row_stride;                 // [acc_elems]
    T *Ws = acc + A.acc_elems;                                     // [2][uc][nb_stride]
    uint64_t *bar = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(Ws + (size_t)2 * A.uc * A.nb_stride) + 15) & ~uintptr_t(15));
    const uint32_t ubar0 = smem_u32(bar);   // slot s uses the mbarrier at ubar0 + 8 s
    int *next_slice = reinterpret_cast<int *>(bar + 2);   // work counter of the current phase
    const int lane = threadIdx.x & 31;
    const int rot = chunk_rot<T, K>(lane);

    const RowTask task = A.tasks[blockIdx.x];
    const DevBlock D = A.blocks[task.block];
    const int nN = D.nN;
    const int row = task.row;
    const int tid = threadIdx.x;

    for (int i = tid; i < nN * K; i += NT) acc[i] = T(0);
    if (tid == 0) {
        mbar_init(ubar0, 1);
        mbar_init(ubar0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0u;   // bit s: parity to wait for on slot s

    // start copying n rows into slot `slot`; row u starts at src_of(u)
    auto issue_rows = [&](int slot, int n, int nelem, auto src_of) {
        T *dst = Xs + (size_t)slot * A.uc * A.row_stride;
        if constexpr (kBulk) {
            if (tid == 0) {
                const uint32_t bytes = (uint32_t)(nelem * K * sizeof(T));
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const uint32_t ub = ubar0 + 8u * (uint32_t)slot;
                mbar_expect_tx(ub, bytes * (uint32_t)n);
                for (int u = 0; u < n; ++u) tma_row(smem_u32(dst + (size_t)u * A.row_stride), src_of(u), bytes, ub);
            }
        } else {
            for (int u = 0; u < n; ++u) {
                const T *s = src_of(u);
                T *d = dst + (size_t)u * A.row_stride;
                for (int i = tid; i < nelem * K; i += NT) d[i] = __ldg(s + i);
            }
        }
    };
    // wait for slot `slot`; true if the bounded wait expired
    auto wait_rows = [&](int slot) -> bool {
        if constexpr (kBulk) {
            uint32_t spins = 0;
            bool hung = false;
            const uint32_t ub = ubar0 + 8u * (uint32_t)slot;
            while (!mbar_try_wait(ub, (phase >> slot) & 1u)) {
                if (++spins > kWaitLimit) { hung = true; break; }
            }
            phase ^= 1u << slot;
            return hung;
        } else {
            return false;
        }
    };
    // after a wait on `slot` ran out: wait once more (bounded) for that
    // slot's copies, so that none is in flight when the CTA exits
    auto drain_rows = [&](int slot) {
        if constexpr (kBulk) {
            const uint32_t ub = ubar0 + 8u * (uint32_t)slot;
            const uint32_t par = ((phase >> slot) & 1u) ^ 1u;   // the phase wait_rows gave up on
            uint32_t spins = 0;
            while (!mbar_try_wait(ub, par) && ++spins <= kWaitLimit) {
            }
        }
    };

    // ---- pp: coalesced reads of whole rows of x
    {
        const int g = D.p_start + row;
        const int64_t e0 = A.pp_ptr[g], e1 = A.pp_ptr[g + 1];
        for (int c = tid; c < nN; c += NT) {
            T part[K], xv[K];
#pragma unroll
            for (int q = 0; q < K; ++q) part[q] = T(0);
            const T *xc = x + (D.off + c) * K;
            for (int64_t e = e0; e < e1; ++e) {
                const T cf = pp_coef[e];
                ldg_vec<T, K>(xc + (int64_t)A.pp_src[e] * nN * K, xv);
#pragma unroll
                for (int q = 0; q < K; ++q) part[q] = fma(cf, xv[q], part[q]);
            }
#pragma unroll
            for (int q = 0; q < K; ++q) acc[c * K + q] += part[q];
        }
    }

    // ---- nn: own row of x staged in slot 0, gathers from shared memory
    {
        const T *src = x + (D.off + (int64_t)row * nN) * K;
        issue_rows(0, 1, nN, [&](int) { return src; });
        if (tid == 0) *next_slice = 0;
        const bool hung = wait_rows(0);
        if (__syncthreads_or(hung)) {
            if (tid == 0) {
                atomicExch(A.err, BS_ETIMEOUT);
                drain_rows(0);
            }
            return;
        }
        const int nslices = (nN + 31) >> 5;
        for (;;) {
            // warps claim 32-column slices (sorted longest first) one at a time
            int sl = 0;
            if (lane == 0) sl = atomicAdd(next_slice, 1);
            sl = __shfl_sync(0xffffffffu, sl, 0);
            if (sl >= nslices) break;
            const int i = sl * 32 + lane;
            if (i >= nN) continue;
            const int col = A.nne_col[D.nne_col + i];
            const int len = A.nne_len[D.nne_col + i];
            const int64_t base = A.nne_soff[D.nne_slice + sl] + lane;
            T part[K], xv[K];
#pragma unroll
            for (int q = 0; q < K; ++q) part[q] = T(0);
            for (int v = 0; v < len; ++v) {
                const int64_t e = base + 32 * (int64_t)v;
                const T cf = nne_coef[e];
                ld_rot<T, K>(Xs, A.nne_src[e], rot, xv);
#pragma unroll
                for (int q = 0; q < K; ++q) part[q] = fma(cf, xv[q], part[q]);
            }
            unrot<T, K>(part, rot);
#pragma unroll
            for (int q = 0; q < K; ++q) acc[col * K + q] += part[q];
        }
        __syncthreads();
    }

    // ---- pn: chunks of source rows, double-buffered across links
    auto next_chunk = [&](int L, int u0) -> Chunk {
        while (L < D.link_end) {
            const int64_t po = A.links[L].p_ptr_off;
            const int64_t pb = A.p1_ptr[po + row], pe = A.p1_ptr[po + row + 1];
            const int U = (int)(pe - pb);
            if (u0 < U) return Chunk{L, u0, min(A.uc, U - u0), pb};
            ++L;
            u0 = 0;
        }
        return Chunk{D.link_end, 0, 0, 0};
    };
    auto issue_chunk = [&](const Chunk &ch, int slot) {
        const DevLink lk = A.links[ch.L];
        const DevBlock S = A.blocks[lk.src_block];
        const int nb = lk.nb;
        T *W = Ws + (size_t)slot * A.uc * A.nb_stride;
        // row u: [0, wsign) = phi_u W[a_u][b] (zero for b >= nb), [wsign, 2 wsign) = its negative
        const int ws = A.wsign;
        for (int i = tid; i < ch.cu * ws; i += NT) {
            const int u = i / ws, b = i - u * ws;
            const uint32_t ep = A.p1_ent[ch.pb + ch.u0 + u];
            const T w = b < nb ? flip(wpn[lk.w_off + (int64_t)((ep >> 16) & 0x7FFFu) * nb + b], ep >> 31) : T(0);
            W[u * A.nb_stride + b] = w;
            W[u * A.nb_stride + ws + b] = -w;
        }
        issue_rows(slot, ch.cu, S.nN, [&](int u) {
            const uint32_t ep = A.p1_ent[ch.pb + ch.u0 + u];
            return x + (S.off + (int64_t)(ep & 0xFFFFu) * S.nN) * K;
        });
    };

    Chunk cur = next_chunk(D.link_begin, 0);
    int slot = 0;
    if (cur.L < D.link_end) issue_chunk(cur, slot);
    while (cur.L < D.link_end) {
        const Chunk nxt = next_chunk(cur.L, cur.u0 + cur.cu);
        if (nxt.L < D.link_end) issue_chunk(nxt, slot ^ 1);
        if (tid == 0) *next_slice = 0;
        const bool hung = wait_rows(slot);
        if (__syncthreads_or(hung)) {
            if (tid == 0) {
                atomicExch(A.err, BS_ETIMEOUT);
                drain_rows(slot);
            }
            // let the other slot's copy land before the CTA exits (bounded)
            if (nxt.L < D.link_end) wait_rows(slot ^ 1);
            return;
        }
        const DevLink lk = A.links[cur.L];
        const T *X0 = Xs + (size_t)slot * A.uc * A.row_stride;
        const T *W0 = Ws + (size_t)slot * A.uc * A.nb_stride;
        const int cu = cur.cu;
        const uint32_t pad = (uint32_t)(A.wsign - 1) << 16;   // a zero W entry, source column 0
        const int nslices = (nN + 31) >> 5;
        for (;;) {
            // warps claim 32-column slices one at a time; slices are sorted
            // longest first, so this is longest-processing-time scheduling
            int sl = 0;
            if (lane == 0) sl = atomicAdd(next_slice, 1);
            sl = __shfl_sync(0xffffffffu, sl, 0);
            if (sl >= nslices) break;
            // lists of a slice are sorted longest first: lane 0's length is
            // the slice's (warp-uniform) trip count; shorter lists are padded
            // with zero-weight entries
            const int lmax = A.n1e_len[lk.n1e_col + sl * 32];
            if (lmax == 0) break;   // every later slice is empty too
            const int i = sl * 32 + lane;
            const bool live = i < nN;
            const int col = live ? A.n1e_col[lk.n1e_col + i] : 0;
            const int64_t base = A.n1e_soff[lk.n1e_slice + sl] + lane;
            T part[K], xv[K];
#pragma unroll
            for (int q = 0; q < K; ++q) part[q] = T(0);
            if (lmax <= kMaxList) {
                uint32_t ev[kMaxList];
#pragma unroll
                for (int v = 0; v < kMaxList; ++v) ev[v] = v < lmax ? A.n1e_ent[base + 32 * v] : pad;
                for (int u = 0; u < cu; ++u) {
                    const T *Xu = X0 + (size_t)u * A.row_stride;
                    const T *Wu = W0 + (size_t)u * A.nb_stride;
#pragma unroll
                    for (int v0 = 0; v0 < kMaxList; v0 += 2) {
                        if (v0 >= lmax) break;
#pragma unroll
                        for (int dv = 0; dv < 2; ++dv) {
                            const uint32_t en = ev[v0 + dv];
                            const T w = Wu[en >> 16];
                            ld_rot<T, K>(Xu, (int)(en & 0xFFFFu), rot, xv);
#pragma unroll
                            for (int q = 0; q < K; ++q) part[q] = fma(w, xv[q], part[q]);
                        }
                    }
                }
            } else {
                for (int v = 0; v < lmax; ++v) {
                    const uint32_t en = A.n1e_ent[base + 32 * (int64_t)v];
                    for (int u = 0; u < cu; ++u) {
                        const T w = W0[u * A.nb_stride + (en >> 16)];
                        ld_rot<T, K>(X0 + (size_t)u * A.row_stride, (int)(en & 0xFFFFu), rot, xv);
#pragma unroll
                        for (int q = 0; q < K; ++q) part[q] = fma(w, xv[q], part[q]);
                    }
                }
            }
            unrot<T, K>(part, rot);
            if (live) {
#pragma unroll
                for (int q = 0; q < K; ++q) acc[col * K + q] += part[q];
            }
        }
        __syncthreads();
        cur = nxt;
        slot ^= 1;
    }

    // ---- write the row once
    for (int c = tid; c < nN; c += NT) {
        T r[K];
#pragma unroll
        for (int q = 0; q < K; ++q) r[q] = acc[c * K + q];
        st_vec<T, K>(y + (D.off + (int64_t)row * nN + c) * K, r);
    }
}

namespace {

// variant v: (threads per CTA, shared-memory target per CTA)
struct RowVariant {
    int threads;
    size_t target;
};
constexpr RowVariant kVariants[] = {{256, 100 * 1024}, {512, 200 * 1024}, {256, 200 * 1024}, {128, 70 * 1024}};
constexpr int kNumVariants = 4;

template <typename T, int K, int NT>
cudaError_t launch_row_nt(const Device &Dv, const DevCoefs<T> &C, const T *x, T *y, cudaStream_t s, size_t target,
                          bool &used)
{
    const size_t es = sizeof(T);
    const int row_elems = Dv.max_nN * K;
    const int row_stride = (int)(((row_elems * es + 127) / 128) * 128 / es);   // 128-byte aligned slots
    const int nb_stride = 2 * Dv.wsign;    // +W and -W halves
    const size_t fixed = (size_t)row_elems * es + 96;   // + mbarriers and the work counter
    const size_t per_u = 2 * ((size_t)row_stride * es + (size_t)nb_stride * es);
    const size_t hard = 227 * 1024;
    int uc = (int)((target > fixed ? target - fixed : 0) / per_u);
    if (uc < 1) uc = (int)((hard > fixed ? hard - fixed : 0) / per_u);
    used = uc >= 1;
    if (!used) return cudaSuccess;
    uc = std::min(uc, std::max(1, Dv.max_pu));
    uc = std::min(uc, 16);
    const size_t smem = (size_t)uc * per_u + fixed + 32;
    auto kern = hx_row_kernel<T, K, NT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    RowArgs A{Dv.rtasks, Dv.blocks, Dv.links, Dv.pp_ptr, Dv.pp_src, Dv.p1_ptr, Dv.p1_ent, Dv.n1e_col, Dv.n1e_len,
              Dv.n1e_soff, Dv.n1e_ent, Dv.nne_col, Dv.nne_len, Dv.nne_src, Dv.nne_soff, Dv.err,
              uc, row_stride, nb_stride, row_elems, Dv.wsign};
    kern<<<Dv.nrtasks, NT, smem, s>>>(A, C.pp_coef, C.nne_coef, C.wpn, x, y);
    return cudaGetLastError();
}

template <typename T, int K>
cudaError_t launch_row(const Device &Dv, const DevCoefs<T> &C, const T *x, T *y, cudaStream_t s, int variant,
                       bool &used)
{
    const RowVariant v = kVariants[variant];
    switch (v.threads) {
    case 128: return launch_row_nt<T, K, 128>(Dv, C, x, y, s, v.target, used);
    case 512: return launch_row_nt<T, K, 512>(Dv, C, x, y, s, v.target, used);
    default: return launch_row_nt<T, K, 256>(Dv, C, x, y, s, v.target, used);
    }
}

}  // namespace

int row_variants() { return kNumVariants; }

// Launches the row kernel (variant `variant`); `used` is false when a row
// does not fit in shared memory (the caller then runs the tiled kernel).
cudaError_t launch_hx_row(const bs_ctx *c, const void *x, void *y, int k, bs_dtype dt, cudaStream_t s, int variant,
                          bool &used)
{
    const Device &D = c->dev;
    used = false;
    if (D.trunc) return cudaSuccess;   // one neutron sector per proton row is assumed
    if (dt == BS_F64) {
        const double *xi = (const double *)x;
        double *yo = (double *)y;
        switch (k) {
        case 1: return launch_row<double, 1>(D, D.c64, xi, yo, s, variant, used);
        case 2: return launch_row<double, 2>(D, D.c64, xi, yo, s, variant, used);
        case 4: return launch_row<double, 4>(D, D.c64, xi, yo, s, variant, used);
        default: return launch_row<double, 8>(D, D.c64, xi, yo, s, variant, used);
        }
    }
    const float *xi = (const float *)x;
    float *yo = (float *)y;
    switch (k) {
    case 1: return launch_row<float, 1>(D, D.c32, xi, yo, s, variant, used);
    case 2: return launch_row<float, 2>(D, D.c32, xi, yo, s, variant, used);
    case 4: return launch_row<float, 4>(D, D.c32, xi, yo, s, variant, used);
    default: return launch_row<float, 8>(D, D.c32, xi, yo, s, variant, used);
    }
}

}  // namespace bs
