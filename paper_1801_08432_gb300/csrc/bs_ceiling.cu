// Measured on-chip ceilings of the H x kernels (a measurement aid with no
// counterpart in the paper).  Every multiply-add of the product gathers one
// k-float element of a source vector, at an index read from a list, and
// applies it to one or more destination rows.  These kernels time exactly
// that and nothing else: a list of seeded random indices walked by every
// thread in turn (coalesced reads), one gathered element per entry, and
// packed FP32 FMAs into R row accumulators.  The table lives in shared memory
// (96 KB) or in global memory (64 MB, L2-resident); the rate they reach is
// the ceiling that the gather-bound H x kernels are measured against.
// The gathers get the best pattern the product's kernels use: the index of
// list position v has the residue of its lane modulo 4 (32-byte elements) or
// 8 (16-byte elements), and for 32-byte elements the second half of each
// quarter warp loads the element's 16-byte halves in swapped order, so a
// quarter warp's 16-byte loads hit eight distinct bank groups; four entries
// per thread are in flight at a time.
#include <cuda_runtime.h>

#include <vector>

#include "bs_internal.h"
#include "bs_tma.cuh"

namespace bs {
namespace {

constexpr int kCeilThreads = 576;     // 18 warps, as the pn-core kernel's consumers
constexpr int kCeilList = 8192;       // indices per list (32 KB of shared memory)
constexpr int kCeilSmemBytes = 96 * 1024;
constexpr int64_t kCeilL2Bytes = 64ll << 20;

// the element's 16-byte parts in the order rot, rot ^ 1 (K = 8) or as is
template <int K>
__device__ __forceinline__ void load_elem(const float *p, int rot, float (&v)[K])
{
#pragma unroll
    for (int q = 0; q < K; q += 4) {
        const int h = K == 8 ? ((q >> 2) ^ rot) << 2 : q;
        const float4 t = *reinterpret_cast<const float4 *>(p + h);
        v[q] = t.x; v[q + 1] = t.y; v[q + 2] = t.z; v[q + 3] = t.w;
    }
}

template <int K>
__device__ __forceinline__ void load_elem_global(const float *p, int rot, float (&v)[K])
{
#pragma unroll
    for (int q = 0; q < K; q += 4) {
        const int h = K == 8 ? ((q >> 2) ^ rot) << 2 : q;
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p + h));
        v[q] = t.x; v[q + 1] = t.y; v[q + 2] = t.z; v[q + 3] = t.w;
    }
}

// SHARED: the table is copied to shared memory first; else gathered from
// global memory.  Every index is < n_elem (the host draws them so).
template <int K, int R, bool SHARED>
__global__ void __launch_bounds__(kCeilThreads, 1)
    gather_fma_kernel(const uint32_t *__restrict__ ids_g, const float *__restrict__ table, int n_elem_smem, int iters,
                      float *__restrict__ sink)
{
    extern __shared__ __align__(16) unsigned char sm[];
    uint32_t *ids = reinterpret_cast<uint32_t *>(sm);
    float *tab = reinterpret_cast<float *>(sm + kCeilList * sizeof(uint32_t));
    for (int i = threadIdx.x; i < kCeilList; i += blockDim.x) ids[i] = ids_g[i];
    if (SHARED)
        for (int i = threadIdx.x; i < n_elem_smem * K; i += blockDim.x) tab[i] = table[i];
    __syncthreads();
    float2 acc[R][K / 2];
    float w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        w[r] = 1.0f + 0.125f * (float)(r + 1);
#pragma unroll
        for (int q = 0; q < K / 2; ++q) acc[r][q] = make_float2(0.0f, 0.0f);
    }
    const int rot = ((threadIdx.x & 31) >> 2) & 1;
    for (int it = 0; it < iters; ++it) {
#pragma unroll 4
        for (int v = threadIdx.x; v < kCeilList; v += blockDim.x) {
            const uint32_t e = ids[v];
            float xv[K];
            if (SHARED) load_elem<K>(tab + (size_t)e * K, rot, xv);
            else load_elem_global<K>(table + (size_t)e * K, rot, xv);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 w2 = make_float2(w[r], w[r]);
#pragma unroll
                for (int q = 0; q < K / 2; ++q) acc[r][q] = __ffma2_rn(w2, make_float2(xv[2 * q], xv[2 * q + 1]), acc[r][q]);
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = 0; q < K / 2; ++q) s += acc[r][q].x + acc[r][q].y;
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void fill_table(float *t, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = 0.001f * (float)(i % 997);
}

template <int K, int R, bool SHARED>
cudaError_t time_ceiling(int nsm, const uint32_t *ids, const float *table, int n_elem_smem, float *sink,
                         cudaStream_t s, double &gflops)
{
    const size_t smem = kCeilList * sizeof(uint32_t) + (SHARED ? (size_t)n_elem_smem * K * sizeof(float) : 0);
    auto kern = gather_fma_kernel<K, R, SHARED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int iters = SHARED ? 400 : 200;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int w = 0; w < 2; ++w) kern<<<nsm, kCeilThreads, smem, s>>>(ids, table, n_elem_smem, iters, sink);
    const int reps = 5;
    cudaEventRecord(a, s);
    for (int r = 0; r < reps; ++r) kern<<<nsm, kCeilThreads, smem, s>>>(ids, table, n_elem_smem, iters, sink);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return e;
    const double fma = (double)nsm * kCeilList * (double)iters * reps * K * R;
    gflops = 2.0 * fma / (ms * 1e-3) / 1e9;
    return cudaGetLastError();
}

template <int K>
cudaError_t ceiling_k(int nsm, int where, int rows, const uint32_t *ids, const float *table, int n_elem_smem,
                      float *sink, cudaStream_t s, double &g)
{
    if (where == 0) {
        switch (rows) {
        case 1: return time_ceiling<K, 1, true>(nsm, ids, table, n_elem_smem, sink, s, g);
        case 2: return time_ceiling<K, 2, true>(nsm, ids, table, n_elem_smem, sink, s, g);
        default: return time_ceiling<K, 4, true>(nsm, ids, table, n_elem_smem, sink, s, g);
        }
    }
    switch (rows) {
    case 1: return time_ceiling<K, 1, false>(nsm, ids, table, 0, sink, s, g);
    case 2: return time_ceiling<K, 2, false>(nsm, ids, table, 0, sink, s, g);
    default: return time_ceiling<K, 4, false>(nsm, ids, table, 0, sink, s, g);
    }
}

// Test aid: one warp waits on an mbarrier that nothing arrives at, through
// the same bounded wait the TMA kernels use, with a short limit.  No copy is
// issued, so none is in flight when the wait gives up; the expiry is
// recorded in the context's status word exactly as a product kernel records
// it, and the kernel returns.
__global__ void wait_expiry_kernel(uint32_t limit, int *err)
{
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = tma::su32(&bar);
    if (threadIdx.x == 0) {
        tma::bar_init(b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (__any_sync(0xffffffffu, tma::bar_wait(b, 0u, limit))) {
        if (threadIdx.x == 0) atomicExch(err, BS_ETIMEOUT);
        return;
    }
}

}  // namespace

uint32_t tma_wait_limit() { return tma::kWaitLimit; }

int run_wait_expiry(int device, uint32_t limit, int *err, void *stream, std::string &msg)
{
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) {
        wait_expiry_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(limit, err);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) { msg = std::string("wait expiry: ") + cudaGetErrorString(e); return BS_ECUDA; }
    return BS_OK;
}

int run_gather_ceiling(int device, int where, int k, int rows, double *gflops, void *stream, std::string &err)
{
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { err = cudaGetErrorString(e); return BS_ECUDA; }
    cudaStream_t s = (cudaStream_t)stream;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    const int elem_bytes = k * (int)sizeof(float);
    const int64_t n_elem = where == 0 ? kCeilSmemBytes / elem_bytes : kCeilL2Bytes / elem_bytes;
    // seeded random indices in [0, n_elem) (SplitMix64)
    std::vector<uint32_t> ids(kCeilList);
    uint64_t z = 0x2545F4914F6CDD1Dull;
    for (int i = 0; i < kCeilList; ++i) {
        z += 0x9E3779B97F4A7C15ull;
        uint64_t v = z;
        v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
        v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
        v ^= v >> 31;
        // residue of the lane (position i is read by lane i mod 32)
        const uint64_t m = k == 8 ? 4 : 8;
        ids[(size_t)i] = (uint32_t)((v % ((uint64_t)n_elem / m)) * m + (uint64_t)(i & 31) % m);
    }
    uint32_t *d_ids = nullptr;
    float *d_tab = nullptr, *d_sink = nullptr;
    auto done = [&](cudaError_t er, const char *what) {
        cudaFree(d_ids);
        cudaFree(d_tab);
        cudaFree(d_sink);
        if (er == cudaSuccess) return BS_OK;
        err = std::string("gather ceiling: ") + what + ": " + cudaGetErrorString(er);
        return er == cudaErrorMemoryAllocation ? BS_ENOMEM : BS_ECUDA;
    };
    if ((e = cudaMalloc(&d_ids, ids.size() * sizeof(uint32_t))) != cudaSuccess) return done(e, "cudaMalloc");
    if ((e = cudaMalloc(&d_tab, (size_t)n_elem * elem_bytes)) != cudaSuccess) return done(e, "cudaMalloc");
    if ((e = cudaMalloc(&d_sink, (size_t)nsm * kCeilThreads * sizeof(float))) != cudaSuccess) return done(e, "cudaMalloc");
    cudaMemcpyAsync(d_ids, ids.data(), ids.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    fill_table<<<4 * nsm, 256, 0, s>>>(d_tab, n_elem * k);
    double g = 0.0;
    e = k == 8 ? ceiling_k<8>(nsm, where, rows, d_ids, d_tab, (int)(where == 0 ? n_elem : 0), d_sink, s, g)
               : ceiling_k<4>(nsm, where, rows, d_ids, d_tab, (int)(where == 0 ? n_elem : 0), d_sink, s, g);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *gflops = g;
    return done(e, "run");
}

}  // namespace bs
