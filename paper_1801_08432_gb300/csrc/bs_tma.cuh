// Shared device helpers of the pipelined kernels (sm_103a): mbarrier waits
// with an iteration limit, TMA bulk copies global -> shared, and the k-wide
// element loads/stores of a staged row.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace bs {
namespace tma {

constexpr uint32_t kWaitLimit = 1u << 22;

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

// bounded wait; true if it expired (after `limit` unsuccessful tries)
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity, uint32_t limit = kWaitLimit)
{
    uint32_t spins = 0;
    while (!bar_try(b, parity))
        if (++spins > limit) return true;
    return false;
}

// For a producer that gives up after a wait ran out: waits (bounded again)
// for the last copy it issued into each of its S ring stages (fills = copies
// issued so far, stage = fill index mod S, full barrier of stage s at full0 +
// 8 s), so that no copy into the CTA's shared memory is in flight when the
// CTA exits.
__device__ __forceinline__ void drain_ring(uint32_t full0, int S, int64_t fills)
{
    for (int s = 0; s < S && s < fills; ++s) {
        const int64_t n = (fills - s + S - 1) / S;   // fills of stage s
        (void)bar_wait(full0 + 8u * (uint32_t)s, (uint32_t)((n - 1) & 1));
    }
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

}  // namespace tma
}  // namespace bs
