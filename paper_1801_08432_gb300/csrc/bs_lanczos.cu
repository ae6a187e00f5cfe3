// Block Lanczos with full reorthogonalization on the GPU (sm_103a).
//
// Sec. "Standard Lanczos algorithm" and Sec. "Block Lanczos": for block n,
//   W   = H V_n                        (the H x kernels, k vectors at once)
//   A_n = V_n^T W,   W -= V_n A_n       (alpha first)
//   W  -= V_m (V_m^T W) for every stored block m <= n, twice
//                                      (full reorthogonalization, classical
//                                       Gram-Schmidt repeated once)
//   O   = W^T W = U Lambda U^T,  B_n = Lambda^(1/2) U^T,
//   V_{n+1} = W U Lambda^(-1/2)
// and T (A_n on the diagonal, B_n below, B_n^T above) is diagonalized in FP64
// on the host.  k = 1 is the standard Lanczos of steps (1)-(6), with
// beta_n = sqrt(O).
//
// Precision.  Vectors are stored in the caller's dtype (FP32: the paper's
// single-precision Lanczos vectors; FP64).  Every inner product (A_n, O and
// the reorthogonalization coefficients) is accumulated in extended precision:
// FP64 vectors use FP64 fused multiply-adds; FP32 vectors form each product
// exactly (a*b and the fma residual) and sum it in a double-float (hi + lo
// FP32) accumulator, which carries about 48 bits -- FP64-grade dots at FP32
// throughput on a part whose FP64 rate is a small fraction of its FP32 rate.
// Block results are reduced across CTAs in FP64 in a fixed order.  Updates of
// the stored vectors run in their own precision.  The small eigenproblems
// (O, k <= 8, on the device; T on the host) are FP64.
//
// Reading of the paper where it is silent: the pivot block is the caller's
// (random) block, orthonormalized; a Gram eigenvalue below 1e-24 of the
// largest marks a breakdown: that column is replaced by a counter-based
// random vector orthogonalized against every stored block.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "bs_internal.h"
#include "bs_tma.cuh"

namespace bs {

bool host_eigh(int n, const double *A, double *w, double *Z, int nvec);
bool host_eigh_banded(int n, int bw, const double *A, int nval, double *w, double *Z, int nvec);

namespace {

constexpr int kDotThreads = 256;

// ---- extended-precision accumulation
struct DF {   // double-float: value = hi + lo
    float hi, lo;
};

__device__ __forceinline__ double df_value(const DF &a) { return (double)a.hi + (double)a.lo; }

// hi + lo += a * b exactly up to the final rounding of lo: the product is
// split as p + e (fma) and p added by a two-sum
__device__ __forceinline__ void df_add_prod(DF &acc, float a, float b)
{
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float s = acc.hi + p;
    const float bb = s - acc.hi;
    const float err = (acc.hi - (s - bb)) + (p - bb);
    acc.hi = s;
    acc.lo += err + e;
}

// hi + lo += s (two-sum: the rounding error of the addition is kept in lo)
__device__ __forceinline__ void df_add(DF &acc, float s)
{
    const float t = acc.hi + s;
    const float bb = t - acc.hi;
    const float err = (acc.hi - (t - bb)) + (s - bb);
    acc.hi = t;
    acc.lo += err;
}

// Extended-precision sums of products.  FP32, EXACT: every product exactly
// (p + e) into a double-float accumulator (~48 bits), for the entries of T and
// for bs_block_dots.  FP32, not EXACT (the Gram-Schmidt coefficients):
// products summed in FP32 over chunks of kChunk rows, each chunk sum added to
// a double-float accumulator; a chunk's rounding error is at most
// kChunk * 2^-24 of its sum of |products|, below the 2^-24 relative rounding
// of the FP32 vectors, and the second Gram-Schmidt pass removes what the
// first leaves.  FP64: FP64 FMAs.
constexpr int kChunk = 16;
template <typename T, bool EXACT>
struct Accum;
template <>
struct Accum<float, true> {
    DF v{0.f, 0.f};
    __device__ __forceinline__ void add(float a, float b) { df_add_prod(v, a, b); }
    __device__ __forceinline__ void flush() {}
    __device__ __forceinline__ double get() const { return df_value(v); }
};
template <>
struct Accum<float, false> {
    DF v{0.f, 0.f};
    float c = 0.f;
    __device__ __forceinline__ void add(float a, float b) { c = fmaf(a, b, c); }
    __device__ __forceinline__ void flush()
    {
        df_add(v, c);
        c = 0.f;
    }
    __device__ __forceinline__ double get() const { return df_value(v) + (double)c; }
};
template <bool EXACT>
struct Accum<double, EXACT> {
    double v = 0.0;
    __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ void flush() {}
    __device__ __forceinline__ double get() const { return v; }
};

// K consecutive values (one basis state of a [dim][K] block), vector loads
template <typename T, int K>
__device__ __forceinline__ void ldrow(const T *p, T (&v)[K])
{
    if constexpr (sizeof(T) * K >= 16) {
        constexpr int W = 16 / sizeof(T);
#pragma unroll
        for (int c = 0; c < K; c += W) {
            if constexpr (sizeof(T) == 4) {
                const float4 q = *reinterpret_cast<const float4 *>(p + c);
                v[c] = q.x; v[c + 1] = q.y; v[c + 2] = q.z; v[c + 3] = q.w;
            } else {
                const double2 q = *reinterpret_cast<const double2 *>(p + c);
                v[c] = q.x; v[c + 1] = q.y;
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < K; ++c) v[c] = p[c];
    }
}

// partial[cta][b][i][j] = sum over this CTA's rows alpha of V_b[alpha][i] * W[alpha][j]
// for the nb blocks V_b of the stored basis (stride `bstride` elements).
// Thread (row slot r, column j): K threads share a row, one W column each.
// Blocks are taken BG = 16 / K at a time, so W is read once per group and a
// thread carries BG x K extended-precision sums.
template <typename T, int K, bool EXACT = true>
__global__ void __launch_bounds__(kDotThreads) blk_dots(const T *__restrict__ V, int64_t bstride, int nb,
                                                        const T *__restrict__ W, int64_t dim,
                                                        double *__restrict__ partial, const int *__restrict__ nb_iter)
{
    if (nb_iter) nb = *nb_iter + 1;   // graph replay: blocks 0..n of iteration n
    constexpr int BG = 16 / K;
    constexpr int RPS = kDotThreads / K;   // rows per CTA step
    __shared__ double red[kDotThreads / 32][BG * K * K];
    const int tid = threadIdx.x, j = tid % K, r = tid / K;
    const int warp = tid >> 5, lane = tid & 31;
    for (int b0 = 0; b0 < nb; b0 += BG) {
        const int nbg = min(BG, nb - b0);
        Accum<T, EXACT> acc[BG][K];
        int cnt = 0;
        for (int64_t a = (int64_t)blockIdx.x * RPS + r; a < dim; a += (int64_t)gridDim.x * RPS) {
            const T w = W[a * K + j];
#pragma unroll
            for (int g = 0; g < BG; ++g) {
                if (g < nbg) {
                    T v[K];
                    ldrow<T, K>(V + (int64_t)(b0 + g) * bstride + a * K, v);
#pragma unroll
                    for (int i = 0; i < K; ++i) acc[g][i].add(v[i], w);
                }
            }
            if (++cnt == kChunk) {
                cnt = 0;
#pragma unroll
                for (int g = 0; g < BG; ++g)
#pragma unroll
                    for (int i = 0; i < K; ++i) acc[g][i].flush();
            }
        }
        // reduce over the rows of the warp (lanes with equal j), then over warps
#pragma unroll
        for (int g = 0; g < BG; ++g) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                double sv = acc[g][i].get();
#pragma unroll
                for (int o = 16; o >= K; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
                if (lane < K) red[warp][(g * K + i) * K + j] = sv;
            }
        }
        __syncthreads();
        for (int e = tid; e < nbg * K * K; e += kDotThreads) {
            double t = 0.0;
            for (int w2 = 0; w2 < kDotThreads / 32; ++w2) t += red[w2][e];
            partial[((int64_t)blockIdx.x * nb + b0) * K * K + e] = t;
        }
        __syncthreads();
    }
}

// out[e] = sum over CTAs of partial[cta][e], e < n, in a fixed order: thread
// (slice q, e) adds the CTAs q, q + kRedSl, ... in turn, then the kRedSl
// slices are added in order.
__device__ __forceinline__ double part_value(double p) { return p; }
__device__ __forceinline__ double part_value(float2 p) { return (double)p.x + (double)p.y; }
constexpr int kRedE = 32;   // outputs per CTA
constexpr int kRedSl = 8;   // slices of the partials per output

template <typename P>
__global__ void __launch_bounds__(kRedE * kRedSl) dots_reduce(const P *__restrict__ partial, int ncta, int n,
                                                              double *__restrict__ out, const int *__restrict__ nb_iter,
                                                              const int *__restrict__ out_iter, int kk)
{
    if (nb_iter) n = (*nb_iter + 1) * kk;       // graph replay: n+1 blocks of k x k
    if (out_iter) out += (int64_t)(*out_iter) * kk;   // graph replay: block n of a history array
    __shared__ double sl[kRedSl][kRedE];
    const int el = threadIdx.x % kRedE, q = threadIdx.x / kRedE;
    const int e = blockIdx.x * kRedE + el;
    double t = 0.0;
    if (e < n)
        for (int c = q; c < ncta; c += kRedSl) t += part_value(partial[(int64_t)c * n + e]);
    sl[q][el] = t;
    __syncthreads();
    if (q == 0 && e < n) {
        double u = sl[0][el];
        for (int r = 1; r < kRedSl; ++r) u += sl[r][el];
        out[e] = u;
    }
}

// n_launch: the largest n the launch may see (graph replay reads n from nb_iter)
template <typename P>
void reduce_parts(const P *partial, int ncta, int n_launch, int n, double *out, const int *nb_iter, const int *out_iter,
                  int kk, cudaStream_t s)
{
    dots_reduce<P><<<(n_launch + kRedE - 1) / kRedE, kRedE * kRedSl, 0, s>>>(partial, ncta, n, out, nb_iter, out_iter, kk);
}

// W[alpha][j] -= sum_b sum_i V_b[alpha][i] C[b][i][j]   (C: nb blocks of K x K, FP64)
template <typename T, int K>
__global__ void blk_update(const T *__restrict__ V, int64_t bstride, int nb, const double *__restrict__ C,
                           T *__restrict__ W, int64_t dim, const int *__restrict__ nb_iter,
                           const int *__restrict__ c_iter)
{
    if (nb_iter) nb = *nb_iter + 1;
    if (c_iter) C += (int64_t)(*c_iter) * K * K;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T *Cs = reinterpret_cast<T *>(sm_raw);
    for (int e = threadIdx.x; e < nb * K * K; e += blockDim.x) Cs[e] = (T)C[e];
    __syncthreads();
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < dim; a += (int64_t)gridDim.x * blockDim.x) {
        T w[K];
        ldrow<T, K>(W + a * K, w);
        for (int b = 0; b < nb; ++b) {
            T v[K];
            ldrow<T, K>(V + (int64_t)b * bstride + a * K, v);
            const T *c = Cs + b * K * K;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                T ci[K];
                ldrow<T, K>(c + i * K, ci);
#pragma unroll
                for (int j = 0; j < K; ++j) w[j] = fma(-v[i], ci[j], w[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < K; ++j) W[a * K + j] = w[j];
    }
}

// Vout[alpha][:] = W[alpha][:] M   (M: K x K, FP64)
template <typename T, int K>
__global__ void blk_scale(const T *__restrict__ W, const double *__restrict__ M, T *__restrict__ Vout, int64_t dim,
                          const int *__restrict__ iter, int64_t bstride, T *__restrict__ Vout2)
{
    if (iter) Vout += (int64_t)(*iter + 1) * bstride;   // graph replay: block n+1
    __shared__ T Ms[K * K];
    if (threadIdx.x < K * K) Ms[threadIdx.x] = (T)M[threadIdx.x];
    __syncthreads();
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < dim; a += (int64_t)gridDim.x * blockDim.x) {
        T w[K], o[K];
#pragma unroll
        for (int i = 0; i < K; ++i) { w[i] = W[a * K + i]; o[i] = T(0); }
#pragma unroll
        for (int i = 0; i < K; ++i)
#pragma unroll
            for (int j = 0; j < K; ++j) o[j] = fma(w[i], Ms[i * K + j], o[j]);
#pragma unroll
        for (int j = 0; j < K; ++j) Vout[a * K + j] = o[j];
        if (Vout2) {
#pragma unroll
            for (int j = 0; j < K; ++j) Vout2[a * K + j] = o[j];
        }
    }
}

__global__ void iter_advance(int *iter)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) ++*iter;
}

__global__ void iter_set(int *iter, int v)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *iter = v;
}

// y[e] += a x[e], e < n (the shift of the targeted operator (H - E_bar)^2)
template <typename T>
__global__ void vec_axpy(T *__restrict__ y, const T *__restrict__ x, T a, int64_t n)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = fma(a, x[e], y[e]);
}

// X[alpha][m] = sum_b sum_i V_b[alpha][i] Y[b*K+i][m], m < nm, FP64 output [dim][ldx]
template <typename T, int K>
__global__ void blk_combine(const T *__restrict__ V, int64_t bstride, int nb, const double *__restrict__ Y, int nm,
                            double *__restrict__ X, int ldx, int64_t dim)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < dim; a += (int64_t)gridDim.x * blockDim.x) {
        double o[8];
        for (int m = 0; m < 8; ++m) o[m] = 0.0;
        for (int b = 0; b < nb; ++b) {
            const T *v = V + (int64_t)b * bstride + a * K;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const double vi = (double)v[i];
                const double *y = Y + (int64_t)(b * K + i) * nm;
                for (int m = 0; m < nm; ++m) o[m] = fma(vi, y[m], o[m]);
            }
        }
        for (int m = 0; m < nm; ++m) X[a * ldx + m] = o[m];
    }
}

// R[alpha][m] -= e[m] X[alpha][m] for m < nm, row length ld (FP64): the
// residual H psi - E psi formed in place of H psi
__global__ void resid_inplace(double *__restrict__ R, const double *__restrict__ X, const double *__restrict__ e,
                              int nm, int ld, int64_t dim)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < dim; a += (int64_t)gridDim.x * blockDim.x)
        for (int m = 0; m < nm; ++m) R[a * ld + m] -= e[m] * X[a * ld + m];
}

// One warp: symmetric Jacobi on the K x K Gram matrix O (FP64), K = 1, 2, 4
// or 8.  Each round applies K/2 disjoint rotations at once (round-robin pair
// schedule: state 0 fixed, the others cycled), one (pair, index) per lane,
// so a sweep of all K(K-1)/2 pairs takes K-1 rounds.  Writes M = U
// Lambda^(-1/2) (to normalize) and B = Lambda^(1/2) U^T; columns whose
// eigenvalue is below rel * max are flagged (bit i of *flags) and get a zero
// column in M and a zero row in B.  Also symmetrizes A in place when given.
__global__ void __launch_bounds__(32) small_gram(int K, const double *__restrict__ O, double rel,
                                                 double *__restrict__ M, double *__restrict__ B,
                                                 int *__restrict__ flags, double *__restrict__ A,
                                                 const int *__restrict__ iter)
{
    __shared__ double a[64], u[64], cs[4][2];
    __shared__ int pq[4][2];
    const int lane = threadIdx.x;
    if (iter) {   // graph replay: B_n and A_n of iteration n
        B += (int64_t)(*iter) * K * K;
        if (A) A += (int64_t)(*iter) * K * K;
    }
    for (int e = lane; e < K * K; e += 32) {
        const int i = e / K, jj = e % K;
        a[e] = 0.5 * (O[i * K + jj] + O[jj * K + i]);
        u[e] = i == jj ? 1.0 : 0.0;
    }
    if (A) {   // one lane per pair (i < jj): every read before any write
        double sv[2];   // K * K <= 64: two elements per lane
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = lane + 32 * h, i = e / K, jj = e % K;
            sv[h] = e < K * K && i < jj ? 0.5 * (A[i * K + jj] + A[jj * K + i]) : 0.0;
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = lane + 32 * h, i = e / K, jj = e % K;
            if (e < K * K && i < jj) A[i * K + jj] = A[jj * K + i] = sv[h];
        }
    }
    __syncwarp();
    const int np = K / 2;                  // rotations per round
    const int m = lane / K, r = lane % K;  // this lane: rotation m, index r (m < np)
    for (int sweep = 0; sweep < 30 && K > 1; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = lane; e < K * K; e += 32) {
            const double v2 = a[e] * a[e];
            tot += v2;
            if (e / K != e % K) off += v2;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        // off-diagonal at ~1e-15 of the matrix: rounding level.  (The column and row
        // updates round differently, so the lower triangle keeps ~1e-16 residues that
        // no rotation removes; a tighter test would run every remaining sweep.)
        if (off <= 1e-30 * tot) break;
        for (int t = 0; t < K - 1; ++t) {
            if (lane < np) {
                // circle method: position i holds state 0 (i = 0) or 1 + (i - 1 + t) mod (K - 1)
                auto st = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + t) % (K - 1); };
                int p = st(lane), q = st(K - 1 - lane);
                if (p > q) { const int x = p; p = q; q = x; }
                pq[lane][0] = p;
                pq[lane][1] = q;
                const double apq = a[p * K + q];
                double c = 1.0, sn = 0.0;
                const float apq32 = (float)apq;
                if (apq32 != 0.0f) {
                    // The angle that zeroes a[p][q], in FP32: the rotation leaves a[p][q] at
                    // ~1e-7 of itself and the next sweep removes the rest (the stopping test
                    // stays in FP64).  FP64 divisions and square roots are slow here.
                    const float th = 0.5f * (float)(a[q * K + q] - a[p * K + p]) / apq32;
                    const float tt = copysignf(1.0f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));   // 0 for huge th
                    const float c32 = rsqrtf(fmaf(tt, tt, 1.0f));
                    // (c, s) made orthonormal in FP64: two Newton steps of 1 / sqrt(c^2 + s^2)
                    // from 1 (c^2 + s^2 is within ~1e-7 of 1), so U stays orthogonal to FP64 rounding
                    c = (double)c32;
                    sn = (double)(tt * c32);
#pragma unroll
                    for (int it = 0; it < 2; ++it) {
                        const double g = fma(-0.5, fma(c, c, sn * sn), 1.5);
                        c *= g;
                        sn *= g;
                    }
                }
                cs[lane][0] = c;
                cs[lane][1] = sn;
            }
            __syncwarp();
            const bool on = m < np;
            int p = 0, q = 0;
            double c = 1.0, sn = 0.0;
            if (on) {
                p = pq[m][0];
                q = pq[m][1];
                c = cs[m][0];
                sn = cs[m][1];
            }
            // columns p, q of A and U (row r)
            double arp = 0, arq = 0, urp = 0, urq = 0;
            if (on) {
                arp = a[r * K + p]; arq = a[r * K + q];
                urp = u[r * K + p]; urq = u[r * K + q];
            }
            __syncwarp();
            if (on) {
                a[r * K + p] = c * arp - sn * arq;
                a[r * K + q] = sn * arp + c * arq;
                u[r * K + p] = c * urp - sn * urq;
                u[r * K + q] = sn * urp + c * urq;
            }
            __syncwarp();
            // rows p, q of A (column r)
            double apr = 0, aqr = 0;
            if (on) {
                apr = a[p * K + r];
                aqr = a[q * K + r];
            }
            __syncwarp();
            if (on) {
                a[p * K + r] = c * apr - sn * aqr;
                a[q * K + r] = sn * apr + c * aqr;
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        double lmax = 0.0;
        for (int i = 0; i < K; ++i) lmax = fmax(lmax, a[i * K + i]);
        int fl = 0;
        for (int i = 0; i < K; ++i) {
            const double lam = a[i * K + i];
            const bool bad = !(lam > rel * lmax) || !(lam > 0.0);
            if (bad) fl |= 1 << i;
        }
        *flags = fl;
        pq[0][0] = fl;
    }
    __syncwarp();
    const int fl = pq[0][0];
    for (int e = lane; e < K * K; e += 32) {
        const int rr = e / K, i = e % K;   // M[rr][i], B[i][rr]
        const double lam = a[i * K + i];
        const bool bad = (fl >> i) & 1;
        const double sq = bad ? 0.0 : sqrt(lam), isq = bad ? 0.0 : 1.0 / sqrt(lam);
        M[rr * K + i] = u[rr * K + i] * isq;
        B[i * K + rr] = sq * u[rr * K + i];
    }
}

// Column `col` of the [dim][K] block X <- Gaussian numbers from a SplitMix64
// counter stream (seed, alpha) with a Box-Muller step.
template <typename T, int K>
__global__ void fill_random_col(T *__restrict__ X, int col, uint64_t seed, int64_t dim)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < dim; a += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(2 * a + 1);
        auto mix = [](uint64_t v) {
            v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
            v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
            return v ^ (v >> 31);
        };
        const uint64_t r1 = mix(z), r2 = mix(z + 0x9E3779B97F4A7C15ull);
        const double u1 = ((r1 >> 11) + 1) * (1.0 / 9007199254740992.0), u2 = (r2 >> 11) * (1.0 / 9007199254740992.0);
        X[a * K + col] = (T)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
    }
}

struct LState {
    int k = 1, dt = 0, ncta = 304;
    int64_t dim = 0, bstride = 0;
    void *V = nullptr, *W = nullptr;      // basis blocks and work block
    double *partial = nullptr, *C = nullptr, *M = nullptr, *Bn = nullptr, *Ahist = nullptr, *Bhist = nullptr;
    int *flags = nullptr;
    int *err = nullptr;                   // device status word (bounded waits of the streamed kernels)
    bool padded = false;                  // V, W blocks readable up to the next 16 bytes past dim * K
    cudaStream_t s = 0;
};

// ---- streamed block products (the HBM-bound part of every Lanczos step)
//
// V_b^T W and W -= sum_b V_b C_b read the whole stored basis once per call.
// A CTA takes chunks of kRsCE consecutive elements (kRsCE / K rows) in turn;
// per chunk it streams the tile of W and then the matching tile of every
// block V_b through a ring of S shared-memory stages that one producer
// thread fills with TMA bulk copies (S x 8 KB in flight per CTA at FP32, no
// registers held by outstanding loads).  W is thus read once per call, not
// once per group of blocks.  Consumer thread (r, j), r < 256 / K, owns
// column j of the rows r + (256 / K) m, m < kRsRT, of each tile.
//
// Dot products: each thread sums its kRsRT rows (FP32 FMAs unless EXACT),
// the lanes of a warp with equal j are combined (the first two steps in
// FP32, so a plain FP32 sum never spans more than 4 kRsRT = 32 products;
// then double-float), the 8 warps in a fixed order, and the tile's K x K
// result is added to the CTA's double-float partial in global memory, which
// dots_reduce sums over CTAs in FP64 in a fixed order: deterministic.
// EXACT forms every product exactly (p + fma residual) in double-float, as
// the row-slot kernel does.  FP64 vectors use FP64 throughout.
// The update applies, per output element, the blocks in order and within a
// block i = 0..K-1, the order of blk_update, so both give identical W.
// Applicability: 16-byte aligned V, W and block stride (the TMA rule) and
// either dim * K * sizeof(T) a multiple of 16 or blocks padded to 16 bytes
// (the Lanczos driver's own buffers); anything else runs the row-slot
// kernels above.
constexpr int kRsCons = 256;     // consumer threads (8 warps) + one producer warp
constexpr int kRsCE = 2048;      // elements per tile
constexpr int kRsRT = 8;         // rows per consumer thread per tile = kRsCE / kRsCons
constexpr int kRsCEU = 4096;     // elements per tile of the update kernel

__device__ __forceinline__ float2 df_sum(float2 a, float2 b)
{
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float e = (a.x - (s - bb)) + (b.x - bb);
    const float t = e + a.y + b.y;
    const float hi = s + t;
    return make_float2(hi, t - (hi - s));
}

template <typename T>
struct RsRed;
template <>
struct RsRed<float> {   // double-float (hi, lo)
    using S = float2;
    static __device__ __forceinline__ S zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ S add(S a, S b) { return df_sum(a, b); }
    static __device__ __forceinline__ S shfl(S a, int o)
    {
        return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
    }
    static __device__ __forceinline__ double value(S a) { return (double)a.x + (double)a.y; }
};
template <>
struct RsRed<double> {
    using S = double;
    static __device__ __forceinline__ S zero() { return 0.0; }
    static __device__ __forceinline__ S add(S a, S b) { return a + b; }
    static __device__ __forceinline__ S shfl(S a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
    static __device__ __forceinline__ double value(S a) { return a; }
};

// Stage and phase of the tile sequence (S stages, used in turn).
template <int S>
struct RsRing {
    int s = 0;
    uint32_t ph = 0;   // parity of the current use of stage s
    int uses = 0;      // tiles so far
    __device__ __forceinline__ void next()
    {
        ++uses;
        if (++s == S) {
            s = 0;
            ph ^= 1u;
        }
    }
};

// Producer of both kernels: for each chunk of this CTA, the W tile then the
// tiles of blocks 0..nb-1 into the stages in turn.  Returns false on a wait
// timeout.
template <typename T, int S, int CE = kRsCE>
__device__ __forceinline__ bool rs_produce(const T *V, int64_t bstride, int nb, const T *W, int64_t nel, T *ring,
                                           uint32_t full0, uint32_t empty0)
{
    using namespace tma;
    const int64_t nch = (nel + CE - 1) / CE;
    RsRing<S> q;
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        const int64_t e0 = ch * CE;
        // a multiple of 16 bytes: exact unless the caller's blocks are padded
        const uint32_t bytes = (uint32_t)((min((int64_t)CE, nel - e0) * (int64_t)sizeof(T) + 15) / 16 * 16);
        for (int b = -1; b < nb; ++b, q.next()) {
            // stage s was used S tiles ago: wait until every consumer warp released it
            if (q.uses >= S && bar_wait(empty0 + 8u * q.s, q.ph ^ 1u)) {
                drain_ring(full0, S, q.uses);   // no copy left in flight at exit
                return false;
            }
            // order the consumers' reads of the stage (generic proxy, observed
            // through the empty barrier) before the bulk copy's writes (async
            // proxy); without it the copy can overwrite data still being read
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bar_expect_tx(full0 + 8u * q.s, bytes);
            bulk_copy(su32(ring + (size_t)q.s * CE), (b < 0 ? W : V + (int64_t)b * bstride) + e0, bytes,
                      full0 + 8u * q.s);
        }
    }
    return true;
}

// partial[cta][b][i][j] (RsRed<T>::S) = this CTA's share of sum_alpha V_b[alpha][i] W[alpha][j].
// Warps 0-7 consume tiles: thread (r, i), r < 256 / K, takes element i of
// rows r + (256 / K) m, m < kRsRT, with the W rows of those elements in
// registers for the whole chunk (one conflict-free scalar shared-memory read
// per V element).  Each warp sums its tile over its rows and lanes and hands
// the K x K result to warp 9 through a ring of SR staging slots; warp 9 adds
// the 8 warps' results in a fixed order to the CTA's running sums and, at the
// end, writes them out.  So no consumer waits on a CTA-wide barrier.  The
// running sums stay in shared memory when nb K^2 of them fit (acc_in_smem),
// else in `partial` itself.
constexpr int kRsSR = 4;   // staging slots of warp results
// FP32, K = 8: the consumer lanes hand over their raw sums (lane (rl, i), 8
// values j each) instead of reducing across lanes themselves; per warp the
// slot holds [i][j][rl] with an i-stride of 36 floats (conflict-free stores:
// bank 4 i + rl + 4 j), read back by the reducer as one 16-byte load per
// (warp, i, j).
constexpr int kRsLaneIS = 36;
constexpr int kRsLaneSR = 2;

template <typename T, int K, bool EXACT>
__host__ __device__ constexpr bool rs_lane_staging()
{
    return std::is_same<T, float>::value && !EXACT && K == 8;
}

template <typename T, int K, bool EXACT, int S>
__global__ void __launch_bounds__(kRsCons + 64, sizeof(T) == 4 ? 2 : 1)
    rs_dots(const T *__restrict__ V, int64_t bstride, int nb, const T *__restrict__ W, int64_t nel,
            typename RsRed<T>::S *__restrict__ partial, int acc_in_smem, const int *__restrict__ nb_iter, int *err)
{
    using namespace tma;
    using R = RsRed<T>;
    using Sv = typename R::S;
    constexpr int NR = kRsCons / K;
    constexpr int NCW = kRsCons / 32;   // consumer warps
    constexpr bool PACKED = std::is_same<T, float>::value && !EXACT && K >= 2;   // two-wide FP32 FMAs
    constexpr bool LANES = rs_lane_staging<T, K, EXACT>();
    constexpr int SR = LANES ? kRsLaneSR : kRsSR;
    constexpr int SLOT = LANES ? NCW * K * kRsLaneIS * 4 : NCW * K * K * (int)sizeof(Sv);   // bytes per staging slot
    if (nb_iter) nb = *nb_iter + 1;   // graph replay: blocks 0..n of iteration n
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);   // full[S], empty[S], pfull[SR], pempty[SR] (256 bytes)
    T *ring = reinterpret_cast<T *>(smem + 256);
    unsigned char *stage = reinterpret_cast<unsigned char *>(ring + (size_t)S * kRsCE);   // [SR][SLOT]
    Sv *red = reinterpret_cast<Sv *>(stage);
    Sv *cacc = acc_in_smem ? reinterpret_cast<Sv *>(stage + (size_t)SR * SLOT)
                           : partial + (int64_t)blockIdx.x * nb * K * K;   // [nb][K * K]
    const uint32_t full0 = su32(bars), empty0 = su32(bars + S);
    const uint32_t pfull0 = su32(bars + 2 * S), pempty0 = su32(bars + 2 * S + SR);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            bar_init(full0 + 8u * s, 1);
            bar_init(empty0 + 8u * s, NCW);
        }
        for (int s = 0; s < SR; ++s) {
            bar_init(pfull0 + 8u * s, NCW);
            bar_init(pempty0 + 8u * s, 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int64_t nch = (nel + kRsCE - 1) / kRsCE;
    if (warp == NCW) {   // producer
        if (lane == 0 && !rs_produce<T, S>(V, bstride, nb, W, nel, ring, full0, empty0)) atomicExch(err, BS_ETIMEOUT);
        return;
    }
    if (warp == NCW + 1) {   // reducer: the 8 warps' tile results, in warp order, into the running sums
        RsRing<SR> sr;
        bool bad = false, first = true;
        for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x, first = false) {
            for (int b = 0; b < nb; ++b, sr.next()) {
                if (!bad && __any_sync(0xffffffffu, bar_wait(pfull0 + 8u * sr.s, sr.ph))) {
                    bad = true;
                    if (lane == 0) atomicExch(err, BS_ETIMEOUT);
                }
                if constexpr (LANES) {
                    // per (warp, i, j): the 4 lanes' sums in FP32 (32 products), then warps in double-float
                    const float *sb = reinterpret_cast<const float *>(stage + (size_t)sr.s * SLOT);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int e = lane + 32 * h, ii = e / K, jj = e % K;
                        DF tot{0.f, 0.f};
#pragma unroll
                        for (int w2 = 0; w2 < NCW; ++w2) {
                            const float4 v4 = *reinterpret_cast<const float4 *>(sb + ((size_t)w2 * K + ii) * kRsLaneIS + jj * 4);
                            const float sw = (v4.x + v4.y) + (v4.z + v4.w);
                            if (w2 == 0) tot = DF{sw, 0.f};
                            else df_add(tot, sw);
                        }
                        const float2 t2 = make_float2(tot.hi, tot.lo);
                        Sv *p = cacc + (int64_t)b * K * K + e;
                        *p = first ? t2 : R::add(*p, t2);
                    }
                } else {
                    const Sv *rb = red + (size_t)sr.s * NCW * K * K;
                    for (int e = lane; e < K * K; e += 32) {
                        Sv tot = rb[e];
#pragma unroll
                        for (int w2 = 1; w2 < NCW; ++w2) tot = R::add(tot, rb[(size_t)w2 * K * K + e]);
                        Sv *p = cacc + (int64_t)b * K * K + e;
                        *p = first ? tot : R::add(*p, tot);
                    }
                }
                __syncwarp();
                if (lane == 0) bar_arrive(pempty0 + 8u * sr.s);
            }
        }
        __syncwarp();
        if (acc_in_smem) {
            for (int e = lane; e < nb * K * K; e += 32)
                partial[(int64_t)blockIdx.x * nb * K * K + e] = first ? R::zero() : cacc[e];
        } else if (first) {   // no chunk for this CTA: its partials are zero
            for (int e = lane; e < nb * K * K; e += 32) partial[(int64_t)blockIdx.x * nb * K * K + e] = R::zero();
        }
        return;
    }
    const int i = tid % K, r = tid / K;
    RsRing<S> q;
    RsRing<SR> sr;
    bool bad = false;
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        const int rows = (int)(min((int64_t)kRsCE, nel - ch * kRsCE) / K);
        T w[kRsRT][K];
        {
            if (!bad && __any_sync(0xffffffffu, bar_wait(full0 + 8u * q.s, q.ph))) {
                bad = true;
                if (lane == 0) atomicExch(err, BS_ETIMEOUT);
            }
            const T *tile = ring + (size_t)q.s * kRsCE;
#pragma unroll
            for (int m = 0; m < kRsRT; ++m) {
                const int a = r + NR * m;
                if (!bad && a < rows) {
                    ldrow<T, K>(tile + a * K, w[m]);
                } else {
#pragma unroll
                    for (int j = 0; j < K; ++j) w[m][j] = T(0);
                }
            }
            __syncwarp();
            if (lane == 0) bar_arrive(empty0 + 8u * q.s);
            q.next();
        }
        for (int b = 0; b < nb; ++b, q.next(), sr.next()) {
            if (!bad && __any_sync(0xffffffffu, bar_wait(full0 + 8u * q.s, q.ph))) {
                bad = true;
                if (lane == 0) atomicExch(err, BS_ETIMEOUT);
            }
            const T *tile = ring + (size_t)q.s * kRsCE;
            Sv sum[K];
            float2 acc[PACKED ? K / 2 : 1];
            if constexpr (PACKED) {
#pragma unroll
                for (int j = 0; j < K / 2; ++j) acc[j] = make_float2(0.f, 0.f);
                if (!bad) {
#pragma unroll
                    for (int m = 0; m < kRsRT; ++m) {
                        const int a = r + NR * m;
                        if (a < rows) {
                            const float v = tile[a * K + i];
                            const float2 v2 = make_float2(v, v);
#pragma unroll
                            for (int j = 0; j < K / 2; ++j)
                                acc[j] = __ffma2_rn(v2, make_float2(w[m][2 * j], w[m][2 * j + 1]), acc[j]);
                        }
                    }
                }
            }
            if constexpr (LANES) {
                // raw lane sums go to the reducer
            } else if constexpr (PACKED) {
                // the first two lane steps in FP32 (at most 4 kRsRT products per plain sum)
                const float2 one = make_float2(1.f, 1.f);
#pragma unroll
                for (int o = K; o < 32 && o <= 2 * K; o <<= 1)
#pragma unroll
                    for (int j = 0; j < K / 2; ++j) {
                        const float2 t2 = make_float2(__shfl_xor_sync(0xffffffffu, acc[j].x, o),
                                                      __shfl_xor_sync(0xffffffffu, acc[j].y, o));
                        acc[j] = __ffma2_rn(t2, one, acc[j]);
                    }
#pragma unroll
                for (int j = 0; j < K / 2; ++j) {
                    sum[2 * j] = make_float2(acc[j].x, 0.f);
                    sum[2 * j + 1] = make_float2(acc[j].y, 0.f);
                }
#pragma unroll
                for (int o = 4 * K; o < 32; o <<= 1)
#pragma unroll
                    for (int j = 0; j < K; ++j) sum[j] = R::add(sum[j], R::shfl(sum[j], o));
            } else if constexpr (std::is_same<T, float>::value && !EXACT) {   // K = 1
                float acc = 0.f;
                if (!bad) {
#pragma unroll
                    for (int m = 0; m < kRsRT; ++m) {
                        const int a = r + NR * m;
                        if (a < rows) acc = fmaf(tile[a], w[m][0], acc);
                    }
                }
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                sum[0] = make_float2(acc, 0.f);
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) sum[0] = R::add(sum[0], R::shfl(sum[0], o));
            } else {
                if constexpr (std::is_same<T, float>::value) {
                    DF acc[K];
#pragma unroll
                    for (int j = 0; j < K; ++j) acc[j] = DF{0.f, 0.f};
                    if (!bad) {
#pragma unroll
                        for (int m = 0; m < kRsRT; ++m) {
                            const int a = r + NR * m;
                            if (a < rows) {
                                const float v = tile[a * K + i];
#pragma unroll
                                for (int j = 0; j < K; ++j) df_add_prod(acc[j], v, w[m][j]);
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < K; ++j) sum[j] = make_float2(acc[j].hi, acc[j].lo);
                } else {
#pragma unroll
                    for (int j = 0; j < K; ++j) sum[j] = 0.0;
                    if (!bad) {
#pragma unroll
                        for (int m = 0; m < kRsRT; ++m) {
                            const int a = r + NR * m;
                            if (a < rows) {
                                const double v = (double)tile[a * K + i];
#pragma unroll
                                for (int j = 0; j < K; ++j) sum[j] = fma(v, (double)w[m][j], sum[j]);
                            }
                        }
                    }
                }
#pragma unroll
                for (int o = K; o < 32; o <<= 1)
#pragma unroll
                    for (int j = 0; j < K; ++j) sum[j] = R::add(sum[j], R::shfl(sum[j], o));
            }
            __syncwarp();
            if (lane == 0) bar_arrive(empty0 + 8u * q.s);
            // hand the warp's result to the reducer (staging slot free once it read it)
            if (!bad && sr.uses >= SR && __any_sync(0xffffffffu, bar_wait(pempty0 + 8u * sr.s, sr.ph ^ 1u))) {
                bad = true;
                if (lane == 0) atomicExch(err, BS_ETIMEOUT);
            }
            if constexpr (LANES) {
                float *sb = reinterpret_cast<float *>(stage + (size_t)sr.s * SLOT) + ((size_t)warp * K + i) * kRsLaneIS + lane / K;
#pragma unroll
                for (int j = 0; j < K / 2; ++j) {
                    sb[(2 * j) * 4] = acc[j].x;
                    sb[(2 * j + 1) * 4] = acc[j].y;
                }
            } else if (lane < K) {   // lane = i here: the warp's sums of row i
                Sv *rb = red + ((size_t)sr.s * NCW + warp) * K * K;
#pragma unroll
                for (int j = 0; j < K; ++j) rb[i * K + j] = sum[j];
            }
            __syncwarp();
            if (lane == 0) bar_arrive(pfull0 + 8u * sr.s);
        }
    }
}

// V_b^T W for FP32 blocks of K = 4 or 8 vectors with W held in shared memory
// (the Gram-Schmidt coefficients, plain products).  A CTA owns one contiguous
// range of rows and walks it in pieces of kRwWT tiles: the piece of W sits in
// kRwWT slots, each loaded once per piece by TMA, while the matching tiles of
// every block V_b stream through a ring of kRwS tiles.  A W slot is released
// when the last block's tile at that position has been consumed, so the next
// piece's W loads overlap the end of the current one.
// Consumer thread t owns the rows t, t + 384, ... of each tile and keeps all
// K x K plain FP32 sums of its rows in registers (packed FMAs, V elements
// duplicated into pairs).  For K = 8 a lane reads the two 16-byte halves of
// its rows in the order (lane >> 2) & 1, which makes the quarter-warp reads
// conflict-free; the sums are put back in order before they are combined.
// After at most kChunk = 16 products per sum (FL tiles of RPT rows: 8 rows at
// K = 8, 16 at K = 4) the warp combines its lanes' sums by a
// butterfly that leaves each lane with K^2 / 32 of the warp's K^2 sums (five
// FP32 addition levels), which the lane adds to its double-float sums.  At the
// end of a block's piece the 12 warps' sums are added in a fixed order into this
// CTA's partial for the block.  So a plain sum holds at most 16 products and
// 5 further roundings before it reaches double-float.  Deterministic: fixed
// orders throughout, and dots_reduce adds the CTAs' partials in a fixed
// order.  Needs the TMA rules of the kernel above.
constexpr int kRwCons = 384;    // consumer threads (12 warps) + one producer warp
constexpr int kRwTile = 24576;  // bytes per V or W tile slot
constexpr int kRwS = 4;         // V ring stages
constexpr int kRwWT = 4;        // W slots: tiles per piece

template <int K>
__host__ __device__ constexpr size_t rw_smem()
{
    return 256 + (size_t)(kRwWT + kRwS) * kRwTile + 2 * (size_t)(kRwCons / 32) * K * K * sizeof(float2);
}

// One butterfly step over the warp on x[0 .. N) of each lane: the lanes with
// bit O set keep the upper half of their values, the others the lower half,
// and each adds its partner's copy of the half it keeps (pairs of values at a
// time).  After it, x[0 .. N / 2) holds the kept half.
template <int N, int O>
__device__ __forceinline__ void rw_bfly_step(float *x, int lane)
{
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int p = 0; p < N / 2; p += 2) {
        const float k0 = up ? x[p + N / 2] : x[p], k1 = up ? x[p + 1 + N / 2] : x[p + 1];
        const float s0 = up ? x[p] : x[p + N / 2], s1 = up ? x[p + 1] : x[p + 1 + N / 2];
        const float2 r = make_float2(__shfl_xor_sync(0xffffffffu, s0, O), __shfl_xor_sync(0xffffffffu, s1, O));
        const float2 t = __fadd2_rn(make_float2(k0, k1), r);
        x[p] = t.x;
        x[p + 1] = t.y;
    }
}

template <int K>
__global__ void __launch_bounds__(kRwCons + 32, 1)
    rs_dots_w(const float *__restrict__ V, int64_t bstride, int nb, const float *__restrict__ W, int64_t dim,
              float2 *__restrict__ partial, const int *__restrict__ nb_iter, int *err)
{
    using namespace tma;
    static_assert(K == 4 || K == 8, "K = 4 or 8");
    constexpr int RB = K * 4;                // bytes per row
    constexpr int RPT = kRwTile / RB / kRwCons;   // rows per thread per tile
    constexpr int TR = RPT * kRwCons;             // rows per tile (at most kRwTile bytes)
    constexpr int PR = kRwWT * TR;                // rows per piece
    constexpr int FL = kChunk / RPT < kRwWT ? kChunk / RPT : kRwWT;   // tiles per plain FP32 sum
    constexpr int NCW = kRwCons / 32;
    constexpr int NL = K * K >= 32 ? K * K / 32 : 1;   // sums per lane after the butterfly
    static_assert(RPT >= 1 && RPT * FL <= kChunk && kRwWT % FL == 0, "plain sums of at most kChunk products");
    if (nb_iter) nb = *nb_iter + 1;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);   // full[kRwS], empty[kRwS], wfull[kRwWT], wempty[kRwWT]
    float *Wp = reinterpret_cast<float *>(smem + 256);
    float *ring = Wp + (size_t)kRwWT * (kRwTile / 4);
    float2 *red = reinterpret_cast<float2 *>(ring + (size_t)kRwS * (kRwTile / 4));   // [2][NCW][K * K]
    const uint32_t full0 = su32(bars), empty0 = su32(bars + kRwS);
    const uint32_t wfull0 = su32(bars + 2 * kRwS), wempty0 = su32(bars + 2 * kRwS + kRwWT);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kRwS; ++s) {
            bar_init(full0 + 8u * s, 1);
            bar_init(empty0 + 8u * s, NCW);
        }
        for (int s = 0; s < kRwWT; ++s) {
            bar_init(wfull0 + 8u * s, 1);
            bar_init(wempty0 + 8u * s, NCW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // this CTA's rows: a contiguous range
    const int64_t rpc = (dim + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rpc, r1 = min(dim, r0 + rpc);
    float2 *part = partial + (int64_t)blockIdx.x * nb * K * K;
    if (warp == NCW) {   // producer
        if (lane != 0) return;
        int64_t tiles = 0, wcopies = 0;
        int piece = 0;
        bool ok = true;
        for (int64_t p0 = r0; ok && p0 < r1; p0 += PR, ++piece) {
            const int64_t pr = min((int64_t)PR, r1 - p0);
            const int nt = (int)((pr + TR - 1) / TR);
            int s = (int)(tiles % kRwS);
            for (int b = 0; ok && b < nb; ++b)
                for (int t = 0; t < nt; ++t, ++tiles, s = s + 1 == kRwS ? 0 : s + 1) {
                    const uint32_t bytes = (uint32_t)(min((int64_t)TR, pr - (int64_t)t * TR) * RB);
                    if (b == 0) {   // W slot t: free once the previous piece's last block used it
                        if (piece > 0 && bar_wait(wempty0 + 8u * t, (uint32_t)(piece - 1) & 1u)) { ok = false; break; }
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        bar_expect_tx(wfull0 + 8u * t, bytes);
                        bulk_copy(su32(Wp + (size_t)t * (kRwTile / 4)), W + (p0 + (int64_t)t * TR) * K, bytes, wfull0 + 8u * t);
                        ++wcopies;
                    }
                    const int64_t use = tiles / kRwS;
                    if (use > 0 && bar_wait(empty0 + 8u * s, (uint32_t)(use - 1) & 1u)) { ok = false; break; }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bar_expect_tx(full0 + 8u * s, bytes);
                    bulk_copy(su32(ring + (size_t)s * (kRwTile / 4)), V + (int64_t)b * bstride + (p0 + (int64_t)t * TR) * K,
                              bytes, full0 + 8u * s);
                }
        }
        if (!ok) {   // no copy left in flight at exit
            atomicExch(err, BS_ETIMEOUT);
            drain_ring(full0, kRwS, tiles);
            drain_ring(wfull0, kRwWT, wcopies);
        }
        return;
    }
    // consumers: rows tid + kRwCons m of each tile; for K = 8 the halves in the order hf, 1 - hf
    // (conflict-free quarter-warp reads)
    const int hf = K == 8 ? (lane >> 2) & 1 : 0;
    const int o0 = 4 * hf, o1 = 4 - 4 * hf;
    float2 acc[K][K / 2];   // plain sums of the current rows: (i, 2q), (i, 2q + 1)
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int q = 0; q < K / 2; ++q) acc[i][q] = make_float2(0.f, 0.f);
    int s = 0;
    uint32_t ph = 0;   // stage and parity of the next tile
    int piece = 0, nred = 0;
    bool bad = false;
    for (int64_t p0 = r0; p0 < r1; p0 += PR, ++piece) {
        const int64_t pr = min((int64_t)PR, r1 - p0);
        const int nt = (int)((pr + TR - 1) / TR);
        for (int b = 0; b < nb; ++b, ++nred) {
            // this block's running partial, read now so that the load is done by the end of the piece
            float2 prev = make_float2(0.f, 0.f);
            if (piece > 0 && tid < K * K) prev = part[(int64_t)b * K * K + tid];
            DF d[NL];
#pragma unroll
            for (int u = 0; u < NL; ++u) d[u] = DF{0.f, 0.f};
            const int trl = (int)(pr - (int64_t)(nt - 1) * TR);   // rows of the piece's last tile
#pragma unroll
            for (int t = 0; t < kRwWT; ++t) {   // unrolled: slot addresses and barriers are constants
                if (t >= nt) break;
                if (b == 0 && !bad && __any_sync(0xffffffffu, bar_wait(wfull0 + 8u * t, (uint32_t)piece & 1u))) {
                    bad = true;
                    if (lane == 0) atomicExch(err, BS_ETIMEOUT);
                }
                if (!bad && __any_sync(0xffffffffu, bar_wait(full0 + 8u * s, ph))) {
                    bad = true;
                    if (lane == 0) atomicExch(err, BS_ETIMEOUT);
                }
                if (!bad) {
                    const int tr = t == nt - 1 ? trl : TR;
                    const float *tile = ring + (size_t)s * (kRwTile / 4);
                    const float *wt = Wp + (size_t)t * (kRwTile / 4);
#pragma unroll
                    for (int m = 0; m < RPT; ++m) {
                        const int a = tid + kRwCons * m;
                        const bool first = t % FL == 0 && m == 0;   // a plain sum starts: multiply, no add
                        if (a < tr) {
                            float v[K];
                            float2 w[K / 2];
                            const float4 va = *reinterpret_cast<const float4 *>(tile + a * K + o0);
                            const float4 wa = *reinterpret_cast<const float4 *>(wt + a * K + o0);
                            v[0] = va.x, v[1] = va.y, v[2] = va.z, v[3] = va.w;
                            w[0] = make_float2(wa.x, wa.y), w[1] = make_float2(wa.z, wa.w);
                            if constexpr (K == 8) {
                                const float4 vb = *reinterpret_cast<const float4 *>(tile + a * K + o1);
                                const float4 wb = *reinterpret_cast<const float4 *>(wt + a * K + o1);
                                v[4] = vb.x, v[5] = vb.y, v[6] = vb.z, v[7] = vb.w;
                                w[2] = make_float2(wb.x, wb.y), w[3] = make_float2(wb.z, wb.w);
                            }
#pragma unroll
                            for (int i = 0; i < K; ++i) {
                                const float2 vi = make_float2(v[i], v[i]);
#pragma unroll
                                for (int q = 0; q < K / 2; ++q)
                                    acc[i][q] = first ? __fmul2_rn(vi, w[q]) : __ffma2_rn(vi, w[q], acc[i][q]);
                            }
                        } else if (first) {
#pragma unroll
                            for (int i = 0; i < K; ++i)
#pragma unroll
                                for (int q = 0; q < K / 2; ++q) acc[i][q] = make_float2(0.f, 0.f);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    bar_arrive(empty0 + 8u * s);
                    if (b == nb - 1) bar_arrive(wempty0 + 8u * t);
                }
                if (++s == kRwS) {
                    s = 0;
                    ph ^= 1u;
                }
                if ((t + 1) % FL == 0 || t == nt - 1) {   // end of a plain sum: combine the warp's lanes
                    float *xs = &acc[0][0].x;   // K * K values, (i, j) row-major in register order
                    if constexpr (K == 8) {
                        // lanes L and L ^ 4 first.  A lane with hf = 1 holds value (i ^ 4, j ^ 4) at
                        // (i, j), i.e. index e ^ 36 at e, and its partner has the other hf, so
                        // keeping values 0..31 and adding the partner's values (e + 32) ^ 4 combines
                        // equal indices without selects.  Then offsets 16, 8, 2, 1; lane L ends with
                        // the indices base(L), base(L) + 1 (the swap of index bit 2 stays with hf).
#pragma unroll
                        for (int p = 0; p < 32; p += 2) {
                            const float2 r = make_float2(__shfl_xor_sync(0xffffffffu, xs[(p + 32) ^ 4], 4),
                                                         __shfl_xor_sync(0xffffffffu, xs[(p + 33) ^ 4], 4));
                            const float2 t2 = __fadd2_rn(make_float2(xs[p], xs[p + 1]), r);
                            xs[p] = t2.x;
                            xs[p + 1] = t2.y;
                        }
                        rw_bfly_step<32, 16>(xs, lane);
                        rw_bfly_step<16, 8>(xs, lane);
                        rw_bfly_step<8, 2>(xs, lane);
                        rw_bfly_step<4, 1>(xs, lane);
                    } else {   // offsets 16, 8, 4, 2, then 1 on the one value left: lanes L, L ^ 1 hold index L / 2
                        rw_bfly_step<16, 16>(xs, lane);
                        rw_bfly_step<8, 8>(xs, lane);
                        rw_bfly_step<4, 4>(xs, lane);
                        rw_bfly_step<2, 2>(xs, lane);
                        xs[0] += __shfl_xor_sync(0xffffffffu, xs[0], 1);
                    }
#pragma unroll
                    for (int u = 0; u < NL; ++u) df_add(d[u], xs[u]);
                }
            }
            // the warps in order; lane L holds sums base(L), base(L) + 1 (K = 8) or L / 2 (K = 4)
            float2 *rb = red + (size_t)(nred & 1) * NCW * K * K;
            if constexpr (K == 8) {
                const int b2 = (lane >> 2) & 1;
                const int base = 32 * b2 + 16 * ((lane >> 4) & 1) + 8 * ((lane >> 3) & 1) + 4 * (((lane >> 1) & 1) ^ b2) +
                                 2 * (lane & 1);
#pragma unroll
                for (int u = 0; u < NL; ++u) rb[(size_t)warp * K * K + base + u] = make_float2(d[u].hi, d[u].lo);
            } else {
                if ((lane & 1) == 0) rb[(size_t)warp * K * K + (lane >> 1)] = make_float2(d[0].hi, d[0].lo);
            }
            asm volatile("bar.sync 1, %0;" ::"n"(kRwCons) : "memory");   // the consumer warps only
            if (tid < K * K) {   // a fixed pairwise tree over the warps (depth 4, not a chain of NCW - 1)
                float2 t2[NCW];
#pragma unroll
                for (int w2 = 0; w2 < NCW; ++w2) t2[w2] = rb[(size_t)w2 * K * K + tid];
#pragma unroll
                for (int h = 1; h < NCW; h *= 2)
#pragma unroll
                    for (int w2 = 0; w2 + h < NCW; w2 += 2 * h) t2[w2] = df_sum(t2[w2], t2[w2 + h]);
                part[(int64_t)b * K * K + tid] = piece == 0 ? t2[0] : df_sum(prev, t2[0]);
            }
        }
    }
    if (r0 >= r1) {   // no rows for this CTA: its partials are zero
        for (int e = tid; e < nb * K * K; e += kRwCons) part[e] = make_float2(0.f, 0.f);
    }
}

// W[alpha][j] -= sum_b sum_i V_b[alpha][i] C[b][i][j]  (C: FP64, used in the vectors' precision).
// Tiles of kRsCEU elements: thread t owns the whole rows t + 256 m, m <
// kRsCEU / (256 K), of each chunk (its W values in registers), reads each of
// its V rows once (consecutive lanes, consecutive rows) and C_b as
// warp-uniform broadcasts, each C_b row serving all of its rows (the C reads
// bound shared memory at one row per thread).  FP32 pairs of
// columns go through two-wide FMAs, each component rounded as fmaf would.
template <typename T, int K, int S>
__global__ void __launch_bounds__(kRsCons + 32) rs_update(const T *__restrict__ V, int64_t bstride, int nb,
                                                          const double *__restrict__ C, T *__restrict__ W,
                                                          int64_t nel, const int *__restrict__ nb_iter,
                                                          const int *__restrict__ c_iter, int *err)
{
    using namespace tma;
    constexpr int RU = kRsCEU / K / kRsCons;   // rows per thread per tile
    constexpr bool PACKED = std::is_same<T, float>::value && K >= 2;
    if (nb_iter) nb = *nb_iter + 1;
    if (c_iter) C += (int64_t)(*c_iter) * K * K;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    T *ring = reinterpret_cast<T *>(smem + 128);
    T *Cs = ring + (size_t)S * kRsCEU;   // [nb][i][j]
    const uint32_t full0 = su32(bars), empty0 = su32(bars + S);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            bar_init(full0 + 8u * s, 1);
            bar_init(empty0 + 8u * s, kRsCons / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = tid; e < nb * K * K; e += blockDim.x) Cs[e] = (T)C[e];
    __syncthreads();
    if (warp == kRsCons / 32) {
        if (lane == 0 && !rs_produce<T, S, kRsCEU>(V, bstride, nb, W, nel, ring, full0, empty0)) atomicExch(err, BS_ETIMEOUT);
        return;
    }
    const int64_t nch = (nel + kRsCEU - 1) / kRsCEU;
    RsRing<S> q;
    bool bad = false;
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        const int64_t e0 = ch * kRsCEU;
        const int rows = (int)(min((int64_t)kRsCEU, nel - e0) / K);
        T w[RU][K];
        for (int b = -1; b < nb; ++b, q.next()) {
            if (!bad && __any_sync(0xffffffffu, bar_wait(full0 + 8u * q.s, q.ph))) {
                bad = true;
                if (lane == 0) atomicExch(err, BS_ETIMEOUT);
            }
            const T *tile = ring + (size_t)q.s * kRsCEU;
            if (b < 0) {
#pragma unroll
                for (int m = 0; m < RU; ++m) {
                    const int a = tid + kRsCons * m;
                    if (!bad && a < rows) {
                        ldrow<T, K>(tile + a * K, w[m]);
                    } else {
#pragma unroll
                        for (int j = 0; j < K; ++j) w[m][j] = T(0);
                    }
                }
            } else if (!bad) {
                T v[RU][K];
#pragma unroll
                for (int m = 0; m < RU; ++m) {
                    const int a = tid + kRsCons * m;
                    if (a < rows) {
                        ldrow<T, K>(tile + a * K, v[m]);
                    } else {
#pragma unroll
                        for (int ii = 0; ii < K; ++ii) v[m][ii] = T(0);
                    }
                }
                const T *cb = Cs + (size_t)b * K * K;
#pragma unroll
                for (int ii = 0; ii < K; ++ii) {
                    T ci[K];
                    ldrow<T, K>(cb + ii * K, ci);
#pragma unroll
                    for (int m = 0; m < RU; ++m) {
                        if constexpr (PACKED) {
                            const float2 nv2 = make_float2(-v[m][ii], -v[m][ii]);
#pragma unroll
                            for (int j = 0; j < K / 2; ++j) {
                                const float2 o2 = __ffma2_rn(nv2, make_float2(ci[2 * j], ci[2 * j + 1]),
                                                             make_float2(w[m][2 * j], w[m][2 * j + 1]));
                                w[m][2 * j] = o2.x;
                                w[m][2 * j + 1] = o2.y;
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < K; ++j) w[m][j] = fma(-v[m][ii], ci[j], w[m][j]);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) bar_arrive(empty0 + 8u * q.s);
        }
        if (!bad) {
#pragma unroll
            for (int m = 0; m < RU; ++m) {
                const int a = tid + kRsCons * m;
                if (a < rows) pst<T, K>(W + e0 + (int64_t)a * K, w[m]);
            }
        }
    }
}

template <typename T>
constexpr int rs_stages() { return sizeof(T) == 4 ? 6 : 4; }

template <typename T, int K>
bool rs_applies(const LState &L, const void *V, const void *W)
{
    return L.err && ((uintptr_t)V % 16 == 0) && ((uintptr_t)W % 16 == 0) &&
           ((L.bstride * (int64_t)sizeof(T)) % 16 == 0) && (L.padded || (L.dim * K * (int64_t)sizeof(T)) % 16 == 0);
}

// nb_iter / out_iter (device, may be null): take the block count n+1 or the
// output slot n from the iteration counter, for graph replay.  nb_max bounds
// the launch when the count comes from the device.
template <typename T, int K, bool EXACT = true>
void dots(LState &L, const T *V, int nb, const T *W, double *out, const int *nb_iter = nullptr,
          const int *out_iter = nullptr, int nb_max = 0)
{
    const int n = (nb_iter ? nb_max : nb) * K * K;
    if constexpr (!EXACT && std::is_same<T, float>::value && (K == 4 || K == 8)) {
        if (rs_applies<T, K>(L, V, W)) {
            constexpr size_t smem = rw_smem<K>();
            static unsigned long long attr = 0;   // per instantiation: devices already configured
            int dev = 0, nsm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            if (dev < 64 && !(attr >> dev & 1ull)) {
                cudaFuncSetAttribute(rs_dots_w<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                attr |= 1ull << dev;
            }
            const int g = std::min(nsm, L.ncta);   // one CTA per SM; the partials hold L.ncta
            rs_dots_w<K><<<g, kRwCons + 32, smem, L.s>>>(V, L.bstride, nb, W, L.dim, reinterpret_cast<float2 *>(L.partial),
                                                        nb_iter, L.err);
            reduce_parts<float2>(reinterpret_cast<const float2 *>(L.partial), g, n, nb * K * K, out, nb_iter, out_iter,
                                 K * K, L.s);
            return;
        }
    }
    if (rs_applies<T, K>(L, V, W)) {
        using Sv = typename RsRed<T>::S;
        constexpr int S = rs_stages<T>();
        const size_t acc = (size_t)(nb_iter ? nb_max : nb) * K * K * sizeof(Sv);
        constexpr bool LANES = rs_lane_staging<T, K, EXACT>();
        const size_t slots = LANES ? (size_t)kRsLaneSR * 8 * K * kRsLaneIS * 4 : (size_t)kRsSR * 8 * K * K * sizeof(Sv);
        const size_t fixed = 256 + (size_t)S * kRsCE * sizeof(T) + slots;
        const int acc_in_smem = fixed + acc <= 113 * 1024;
        const size_t smem = fixed + (acc_in_smem ? acc : 0);
        static unsigned long long attr = 0;   // per instantiation: devices already configured
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 64 && !(attr >> dev & 1ull)) {
            cudaFuncSetAttribute(rs_dots<T, K, EXACT, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, 113 * 1024);
            attr |= 1ull << dev;
        }
        rs_dots<T, K, EXACT, S><<<L.ncta, kRsCons + 64, smem, L.s>>>(V, L.bstride, nb, W, L.dim * K,
                                                                     reinterpret_cast<Sv *>(L.partial), acc_in_smem,
                                                                     nb_iter, L.err);
        reduce_parts<Sv>(reinterpret_cast<const Sv *>(L.partial), L.ncta, n, nb * K * K, out, nb_iter, out_iter, K * K,
                         L.s);
        return;
    }
    blk_dots<T, K, EXACT><<<L.ncta, kDotThreads, 0, L.s>>>(V, L.bstride, nb, W, L.dim, L.partial, nb_iter);
    reduce_parts<double>(L.partial, L.ncta, n, nb * K * K, out, nb_iter, out_iter, K * K, L.s);
}

template <typename T, int K>
void update(LState &L, const T *V, int nb, const double *C, T *W, const int *nb_iter = nullptr,
            const int *c_iter = nullptr, int nb_max = 0)
{
    const int nbm = nb_iter ? nb_max : nb;
    const size_t csm = (size_t)nbm * K * K * sizeof(T);
    constexpr int S = sizeof(T) == 4 ? 3 : 2;   // 16 KB (FP32) or 32 KB (FP64) tiles
    const size_t rsm = 128 + (size_t)S * kRsCEU * sizeof(T) + csm;
    if (rs_applies<T, K>(L, V, W) && rsm <= 112 * 1024) {
        static unsigned long long attr = 0;   // per instantiation: devices already configured
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 64 && !(attr >> dev & 1ull)) {
            cudaFuncSetAttribute(rs_update<T, K, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
            attr |= 1ull << dev;
        }
        rs_update<T, K, S><<<L.ncta, kRsCons + 32, rsm, L.s>>>(V, L.bstride, nb, C, W, L.dim * K, nb_iter, c_iter, L.err);
        return;
    }
    blk_update<T, K><<<L.ncta, 256, csm, L.s>>>(V, L.bstride, nb, C, W, L.dim, nb_iter, c_iter);
}

}  // namespace

template <typename T, int K>
static int lanczos_run(bs_ctx *c, const bs_lanczos_opts &o, const void *pivot, double *evals, double *evecs,
                       bs_lanczos_report *rep, const StrengthReq *sreq)
{
    LState L;
    L.k = K;
    L.dim = c->basis.dim;
    // block stride rounded up to 16 bytes: every block starts on a TMA
    // boundary, and the streamed kernels may copy up to the next 16 bytes
    L.bstride = (L.dim * K + (int64_t)(16 / sizeof(T)) - 1) / (int64_t)(16 / sizeof(T)) * (int64_t)(16 / sizeof(T));
    L.padded = true;
    L.s = (cudaStream_t)o.stream;
    int dev = 0;
    cudaGetDevice(&dev);
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    L.ncta = 2 * nsm;
    L.err = c->dev.err;
    int niter = std::max(1, o.niter);
    niter = (int)std::min<int64_t>(niter, std::max<int64_t>(1, L.dim / K));
    const size_t es = sizeof(T);
    std::vector<void *> owned;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
        owned.push_back(p);
        return p;
    };
    auto cleanup = [&]() {
        for (void *p : owned) cudaFree(p);
        owned.clear();
    };
    // thick restart: nthick / K blocks of Ritz vectors, formed in as many
    // scratch blocks past V_niter
    const int tb = o.nthick > 0 ? o.nthick / K : 0;
    const bool thick = tb > 0;
    if (thick && tb + 1 >= niter) { c->err = "lanczos: nthick / k + 1 must stay below niter (clamped to dim / k)"; return BS_EINVAL; }
    L.V = alloc((size_t)(niter + 1 + tb) * L.bstride * es);
    L.W = alloc((size_t)L.bstride * es);
    // targeted restart (Sec. "Targeted thick-restart Lanczos"): the operator is
    // (H - E_bar)^2, applied as two products with the shift in between
    const bool targeted = o.targeted != 0;
    T *W1 = targeted ? (T *)alloc((size_t)L.bstride * es) : nullptr;
    const T tshift = (T)(-o.target);
    auto apply_op = [&](const T *x, T *y) -> int {
        if (!targeted) return launch_hx(c, x, y, K, o.dtype, L.s, c->err);
        int r = launch_hx(c, x, W1, K, o.dtype, L.s, c->err);
        if (r) return r;
        vec_axpy<T><<<L.ncta, 256, 0, L.s>>>(W1, x, tshift, L.dim * K);
        if ((r = launch_hx(c, W1, y, K, o.dtype, L.s, c->err))) return r;
        vec_axpy<T><<<L.ncta, 256, 0, L.s>>>(y, W1, tshift, L.dim * K);
        return BS_OK;
    };
    double *Ct = (double *)alloc((size_t)std::max(tb, 1) * niter * K * K * sizeof(double));
    // dot scratch: (niter+1) blocks of K x K, or one 8 x 8 block for the refinement
    const size_t ndot = std::max<size_t>((size_t)(niter + 1) * K * K, 64);
    L.partial = (double *)alloc((size_t)L.ncta * ndot * sizeof(double));
    L.C = (double *)alloc(ndot * sizeof(double));
    L.M = (double *)alloc(K * K * sizeof(double));
    L.Bn = (double *)alloc(K * K * sizeof(double));
    L.Ahist = (double *)alloc((size_t)niter * K * K * sizeof(double));
    L.Bhist = (double *)alloc((size_t)niter * K * K * sizeof(double));
    L.flags = (int *)alloc(sizeof(int));
    for (void *p : owned)
        if (!p) { cleanup(); c->err = "lanczos: device allocation failed"; return BS_ENOMEM; }
    {
        cudaError_t e = cudaFuncSetAttribute(blk_update<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)std::min<size_t>((size_t)(niter + 1) * K * K * es, 227 * 1024));
        if (e != cudaSuccess) { cleanup(); c->err = std::string("lanczos: ") + cudaGetErrorString(e); return BS_ECUDA; }
        if ((size_t)(niter + 1) * K * K * es > 227 * 1024) { cleanup(); c->err = "lanczos: too many blocks for the reorthogonalization kernel"; return BS_EINVAL; }
    }
    T *V = (T *)L.V, *W = (T *)L.W;
    const double rel = 1e-24;
    cudaEvent_t ev[4];
    for (auto &e : ev) cudaEventCreate(&e);
    // every CUDA error of the call is caught here and reported with the
    // stage that met it, never left in the runtime's last-error state
    std::string cuda_fail;
    auto stage = [&](const char *where) {
        const cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess && cuda_fail.empty()) cuda_fail = std::string(where) + ": " + cudaGetErrorString(le);
        return cuda_fail.empty();
    };
    // event timings are diagnostics: an event that cannot be timed counts 0
    auto elapsed = [&](cudaEvent_t from, cudaEvent_t to) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, from, to) != cudaSuccess) {
            (void)cudaGetLastError();
            ms = 0.f;
        }
        return ms;
    };
    float ms_mv = 0.f, ms_or = 0.f;
    int breakdowns = 0, done = 0;
    std::vector<double> Ah((size_t)niter * K * K), Bh((size_t)niter * K * K);
    int rc = BS_OK;
    const auto t0 = std::chrono::steady_clock::now();
    const int passes = std::max(1, o.reorth_passes);

    // orthonormalize the pivot block (FP64 Gram, one reorthogonalization-free QR)
    cudaMemcpyAsync(W, pivot, (size_t)L.dim * K * es, cudaMemcpyDeviceToDevice, L.s);
    dots<T, K>(L, W, 1, W, L.C);
    // a strength pivot must be well conditioned (its overlaps go through
    // B_0): overlap eigenvalues below 1e-12 of the largest count as rank loss
    small_gram<<<1, 32, 0, L.s>>>(K, L.C, sreq ? 1e-12 : rel, L.M, L.Bn, L.flags, nullptr, nullptr);
    blk_scale<T, K><<<L.ncta, 256, 0, L.s>>>(W, L.M, V, L.dim, nullptr, 0, nullptr);
    // strength function: W_0 = V_0 B_0 with B_0 = Lambda^1/2 U^T of the pivot's
    // overlap matrix (Sec. "Block strength function"); the pivot must have full rank
    std::vector<double> B0((size_t)K * K);
    if (sreq) {
        int fl = 0;
        cudaMemcpyAsync(B0.data(), L.Bn, (size_t)K * K * sizeof(double), cudaMemcpyDeviceToHost, L.s);
        cudaMemcpyAsync(&fl, L.flags, sizeof(int), cudaMemcpyDeviceToHost, L.s);
        int src = BS_OK;
        if (cudaStreamSynchronize(L.s) != cudaSuccess) { c->err = "strength: pivot copy failed"; src = BS_ECUDA; }
        else if (fl) { c->err = "strength: the pivot block is rank deficient"; src = BS_EINVAL; }
        if (src != BS_OK) {
            for (auto &e : ev) cudaEventDestroy(e);
            cleanup();
            return src;
        }
    }

    // Graph mode: the whole block iteration (H X, alpha, reorthogonalization,
    // Gram eigen-decomposition, normalization) is captured once in a CUDA
    // graph whose kernels read the iteration number n from a device counter;
    // each iteration is one graph launch.  H X reads a fixed copy of V_n
    // (Xcur, written by the normalization of the previous iteration).
    T *Xcur = nullptr;
    int *d_iter = nullptr;
    cudaGraphExec_t gexec = nullptr;
    if (o.use_graph) {
        Xcur = (T *)alloc((size_t)L.bstride * es);
        d_iter = (int *)alloc(sizeof(int));
        if (!Xcur || !d_iter) { cleanup(); c->err = "lanczos: device allocation failed"; return BS_ENOMEM; }
        cudaMemcpyAsync(Xcur, V, (size_t)L.bstride * es, cudaMemcpyDeviceToDevice, L.s);
        cudaMemsetAsync(d_iter, 0, sizeof(int), L.s);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(L.s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaEventRecord(ev[0], L.s);
            rc = apply_op(Xcur, W);
            cudaEventRecord(ev[1], L.s);
            dots<T, K>(L, Xcur, 1, W, L.Ahist, nullptr, d_iter, 1);
            update<T, K>(L, Xcur, 1, L.Ahist, W, nullptr, d_iter, 1);
            for (int p = 0; p < passes; ++p) {
                dots<T, K, false>(L, V, 1, W, L.C, d_iter, nullptr, niter + 1);
                update<T, K>(L, V, 1, L.C, W, d_iter, nullptr, niter + 1);
            }
            dots<T, K>(L, W, 1, W, L.C);
            small_gram<<<1, 32, 0, L.s>>>(K, L.C, rel, L.M, L.Bhist, L.flags, L.Ahist, d_iter);
            blk_scale<T, K><<<L.ncta, 256, 0, L.s>>>(W, L.M, V, L.dim, d_iter, L.bstride, Xcur);
            iter_advance<<<1, 1, 0, L.s>>>(d_iter);
            cudaEventRecord(ev[2], L.s);
            e = cudaStreamEndCapture(L.s, &graph);
        }
        if (e == cudaSuccess && rc == BS_OK) e = cudaGraphInstantiate(&gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess || rc != BS_OK) {
            if (rc == BS_OK) { c->err = std::string("lanczos graph: ") + cudaGetErrorString(e); rc = BS_ECUDA; }
            for (auto &ee : ev) cudaEventDestroy(ee);
            cleanup();
            return rc;
        }
    }

    // Cycles: one without thick restart; with it, each cycle runs the block
    // iterations n0..niter-1 (n0 = 0, then nthick / K), diagonalizes T and,
    // unless done, restarts (Sec. "Thick-restart block Lanczos").
    int n0 = 0, restarts = 0, matvecs = 0;
    bool exhausted = false;
    std::vector<double> Eth, Rth;   // arrow of the restarted T: kept Ritz values, coupling [K][nthick]
    std::vector<double> wT, Z;
    const int nkeep = std::max(1, o.nkeep);
    int nT = 0, nv = 0;
    double resid_est = 0.0;
    for (;;) {
    for (int n = n0; n < niter && rc == BS_OK && !exhausted; ++n) {
            T *Vn = V + (int64_t)n * L.bstride;
            if (gexec) {
                cudaError_t e = cudaGraphLaunch(gexec, L.s);
                if (e != cudaSuccess) { c->err = std::string("lanczos graph launch: ") + cudaGetErrorString(e); rc = BS_ECUDA; break; }
            } else {
            cudaEventRecord(ev[0], L.s);
            if ((rc = apply_op(Vn, W))) break;
            cudaEventRecord(ev[1], L.s);
            // alpha first: A_n = V_n^T W, W -= V_n A_n
            double *An = L.Ahist + (size_t)n * K * K;
            dots<T, K>(L, Vn, 1, W, An);
            update<T, K>(L, Vn, 1, An, W);
            for (int p = 0; p < passes; ++p) {
                dots<T, K, false>(L, V, n + 1, W, L.C);
                update<T, K>(L, V, n + 1, L.C, W);
            }
            dots<T, K>(L, W, 1, W, L.C);
            small_gram<<<1, 32, 0, L.s>>>(K, L.C, rel, L.M, L.Bhist + (size_t)n * K * K, L.flags, An, nullptr);
            blk_scale<T, K><<<L.ncta, 256, 0, L.s>>>(W, L.M, V + (int64_t)(n + 1) * L.bstride, L.dim, nullptr, 0, nullptr);
            cudaEventRecord(ev[2], L.s);
            }
            int flags = 0;
            cudaError_t e = cudaMemcpyAsync(&flags, L.flags, sizeof(int), cudaMemcpyDeviceToHost, L.s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(L.s);
            if (e != cudaSuccess) { c->err = std::string("lanczos: ") + cudaGetErrorString(e); rc = BS_ECUDA; break; }
            ms_mv += elapsed(ev[0], ev[1]);
            ms_or += elapsed(ev[1], ev[2]);
            if (!stage("block iteration")) { rc = BS_ECUDA; break; }
            done = n + 1;
            if (flags && (n + 1 < niter || thick)) {
                // breakdown: flagged columns of V_{n+1} are zero; refill them with
                // random vectors, orthogonalize against V_0..V_n, renormalize the
                // block, and fold the change of basis into B_n
                ++breakdowns;
                T *Vn1 = V + (int64_t)(n + 1) * L.bstride;
                for (int i = 0; i < K; ++i)
                    if (flags >> i & 1)
                        fill_random_col<T, K><<<L.ncta, 256, 0, L.s>>>(Vn1, i, 0xB5297A4D3F84D5B5ull + 7919ull * (uint64_t)(n * K + i), L.dim);
                for (int p = 0; p < 2; ++p) {
                    dots<T, K, false>(L, V, n + 1, Vn1, L.C);
                    update<T, K>(L, V, n + 1, L.C, Vn1);
                }
                cudaMemcpyAsync(W, Vn1, (size_t)L.bstride * es, cudaMemcpyDeviceToDevice, L.s);
                dots<T, K>(L, W, 1, W, L.C);
                small_gram<<<1, 32, 0, L.s>>>(K, L.C, 1e-20, L.M, L.Bn, L.flags, nullptr, nullptr);
                blk_scale<T, K><<<L.ncta, 256, 0, L.s>>>(W, L.M, Vn1, L.dim, nullptr, 0, nullptr);
                // B_n <- G B_n with G = Bn (the Gram factor of the refilled block: W = Vnew G)
                std::vector<double> G(K * K), Bn(K * K), out(K * K, 0.0);
                int fl2 = 0;
                cudaMemcpyAsync(G.data(), L.Bn, K * K * sizeof(double), cudaMemcpyDeviceToHost, L.s);
                cudaMemcpyAsync(Bn.data(), L.Bhist + (size_t)n * K * K, K * K * sizeof(double), cudaMemcpyDeviceToHost, L.s);
                cudaMemcpyAsync(&fl2, L.flags, sizeof(int), cudaMemcpyDeviceToHost, L.s);
                cudaStreamSynchronize(L.s);
                if (fl2) { exhausted = true; break; }   // the Krylov space is exhausted
                for (int i = 0; i < K; ++i)
                    for (int j = 0; j < K; ++j)
                        for (int l = 0; l < K; ++l) out[i * K + j] += G[i * K + l] * Bn[l * K + j];
                cudaMemcpyAsync(L.Bhist + (size_t)n * K * K, out.data(), K * K * sizeof(double), cudaMemcpyHostToDevice, L.s);
                if (Xcur) cudaMemcpyAsync(Xcur, Vn1, (size_t)L.bstride * es, cudaMemcpyDeviceToDevice, L.s);
                cudaStreamSynchronize(L.s);
            }
        matvecs += targeted ? 2 : 1;
    }
    if (rc != BS_OK) break;
    cudaMemcpyAsync(Ah.data(), L.Ahist, (size_t)done * K * K * sizeof(double), cudaMemcpyDeviceToHost, L.s);
    cudaMemcpyAsync(Bh.data(), L.Bhist, (size_t)done * K * K * sizeof(double), cudaMemcpyDeviceToHost, L.s);
    if (cudaStreamSynchronize(L.s) != cudaSuccess) { rc = BS_ECUDA; c->err = "lanczos: copy failed"; break; }
    nT = done * K;
    std::vector<double> T_((size_t)nT * nT, 0.0);
    if (restarts > 0) {
        // arrow of the thick-restart matrix: E on the diagonal, r in the rows of block tb
        for (int m = 0; m < o.nthick; ++m) T_[(size_t)m * nT + m] = Eth[m];
        for (int i = 0; i < K; ++i)
            for (int m = 0; m < o.nthick; ++m) {
                const double r = Rth[(size_t)i * o.nthick + m];
                T_[(size_t)(tb * K + i) * nT + m] = r;
                T_[(size_t)m * nT + tb * K + i] = r;
            }
    }
    for (int n = n0; n < done; ++n)
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j) {
                T_[(size_t)(n * K + i) * nT + n * K + j] = Ah[(size_t)n * K * K + i * K + j];
                if (n + 1 < done) {
                    const double b = Bh[(size_t)n * K * K + i * K + j];   // B_n: row i of block n+1, column j of block n
                    T_[(size_t)((n + 1) * K + i) * nT + n * K + j] = b;
                    T_[(size_t)(n * K + j) * nT + (n + 1) * K + i] = b;
                }
            }
    const int nwant = std::max(nkeep, thick ? o.nthick : 0);
    const int nval = std::min(nT, std::max(nkeep + 5, nwant));
    nv = std::min(nwant, nT);
    wT.assign(std::max(nT, 1), 0.0);
    Z.assign((size_t)nT * std::max(nv, 1), 0.0);
    int bw = 0;
    if (restarts == 0) {
        // T is banded: B_n = Lambda^1/2 Q^T from the Gram eigendecomposition
        // is a full k x k block, so the half-bandwidth is up to 2k - 1 (read
        // off T).  Eigenvalues by bisection on inertia counts, eigenvectors by
        // inverse iteration, O(nT bw^2) each.
        for (int i = 0; i < nT; ++i)
            for (int j = 0; j < i - bw; ++j)
                if (T_[(size_t)i * nT + j] != 0.0) { bw = i - j; break; }
        if (!host_eigh_banded(nT, bw, T_.data(), nval, wT.data(), Z.data(), nv)) { rc = BS_EBREAKDOWN; c->err = "lanczos: eigensolver failed"; break; }
    } else if (!host_eigh(nT, T_.data(), wT.data(), Z.data(), nv)) {   // the arrow is not banded
        rc = BS_EBREAKDOWN; c->err = "lanczos: eigensolver failed"; break;
    }
    // convergence measure of the paper: the lowest nkeep+5 eigenvalues of
    // T now and one block iteration earlier
    if (rep) {
        const int nprev = (done - 1) * K, m = std::min(nkeep + 5, nprev);
        double delta = 0.0;
        if (m > 0) {
            std::vector<double> Tp((size_t)nprev * nprev), wp(std::max(nprev, 1));
            for (int i = 0; i < nprev; ++i)
                for (int j = 0; j < nprev; ++j) Tp[(size_t)i * nprev + j] = T_[(size_t)i * nT + j];
            std::vector<double> dummy(1);
            if (restarts == 0) host_eigh_banded(nprev, bw, Tp.data(), m, wp.data(), dummy.data(), 0);
            else host_eigh(nprev, Tp.data(), wp.data(), dummy.data(), 0);
            for (int i = 0; i < m; ++i) delta += std::fabs(wT[i] - wp[i]);
            delta /= std::sqrt((double)m);
        }
        rep->delta_conv = delta;
    }
    // |H psi_mu - E_mu psi_mu| = |B_last U[last block rows, mu]| for the Ritz
    // pairs of T (the component of H psi along the next Lanczos block)
    auto coupling = [&](int i, int m) {
        double r = 0.0;
        for (int j = 0; j < K; ++j)
            r += Bh[(size_t)(done - 1) * K * K + i * K + j] * Z[(size_t)((done - 1) * K + j) * nv + m];
        return r;
    };
    resid_est = 0.0;
    for (int m = 0; m < std::min(nkeep, nv); ++m) {
        double r2 = 0.0;
        for (int i = 0; i < K; ++i) r2 += coupling(i, m) * coupling(i, m);
        resid_est = std::max(resid_est, std::sqrt(r2));
    }
    if (sreq) {
        // every eigenpair of T; overlaps <w_i|E_r> = sum_j (B_0)_ji L_jr over the
        // first block's rows (T is dense-diagonalized: all vectors are needed)
        std::vector<double> wa((size_t)nT), za((size_t)nT * nT);
        if (!host_eigh(nT, T_.data(), wa.data(), za.data(), nT)) { rc = BS_EBREAKDOWN; c->err = "strength: eigensolver failed"; break; }
        for (int r = 0; r < sreq->n_out; ++r) {
            sreq->E[r] = r < nT ? wa[r] : NAN;
            for (int i = 0; i < K; ++i) {
                double ov = 0.0;
                for (int j = 0; j < K && r < nT; ++j) ov += B0[(size_t)j * K + i] * za[(size_t)j * nT + r];
                sreq->S[(size_t)i * sreq->n_out + r] = r < nT ? ov * ov : NAN;
            }
        }
    }
    if (!thick || exhausted || done < niter || restarts >= o.max_restarts || (o.tol > 0.0 && resid_est <= o.tol)) break;
    // restart: Y_j = sum_b V_b U[b rows, j cols] (j < tb) into the scratch
    // blocks past V_niter, then V_niter -> V_tb and Y -> V_0..V_(tb-1)
    cudaEventRecord(ev[0], L.s);
    {
        std::vector<double> Ch((size_t)tb * done * K * K);
        for (int jb = 0; jb < tb; ++jb)
            for (int b = 0; b < done; ++b)
                for (int i = 0; i < K; ++i)
                    for (int jj = 0; jj < K; ++jj)
                        Ch[(((size_t)jb * done + b) * K + i) * K + jj] = -Z[(size_t)(b * K + i) * nv + jb * K + jj];
        cudaMemcpyAsync(Ct, Ch.data(), Ch.size() * sizeof(double), cudaMemcpyHostToDevice, L.s);
        T *scratch = V + (int64_t)(niter + 1) * L.bstride;
        cudaMemsetAsync(scratch, 0, (size_t)tb * L.bstride * es, L.s);
        for (int jb = 0; jb < tb; ++jb)
            update<T, K>(L, V, done, Ct + (size_t)jb * done * K * K, scratch + (int64_t)jb * L.bstride);
        cudaMemcpyAsync(V + (int64_t)tb * L.bstride, V + (int64_t)done * L.bstride, (size_t)L.bstride * es,
                        cudaMemcpyDeviceToDevice, L.s);
        cudaMemcpyAsync(V, scratch, (size_t)tb * L.bstride * es, cudaMemcpyDeviceToDevice, L.s);
        if (gexec) {
            cudaMemcpyAsync(Xcur, V + (int64_t)tb * L.bstride, (size_t)L.bstride * es, cudaMemcpyDeviceToDevice, L.s);
            iter_set<<<1, 1, 0, L.s>>>(d_iter, tb);
        }
        Eth.assign(wT.begin(), wT.begin() + o.nthick);
        Rth.assign((size_t)K * o.nthick, 0.0);
        for (int i = 0; i < K; ++i)
            for (int m = 0; m < o.nthick; ++m) Rth[(size_t)i * o.nthick + m] = coupling(i, m);
        // Ch must outlive its (pageable, staged) copy
        cudaEventRecord(ev[3], L.s);
        if (cudaStreamSynchronize(L.s) != cudaSuccess) { rc = BS_ECUDA; c->err = "lanczos: restart failed"; break; }
    }
    ms_or += elapsed(ev[0], ev[3]);
    if (!stage("thick restart")) { rc = BS_ECUDA; break; }
    n0 = tb;
    ++restarts;
    }

    int nk = std::min(nkeep, nT);
    if (rc == BS_OK) {
        for (int i = 0; i < nk; ++i) evals[i] = wT[i];
        for (int i = nk; i < nkeep; ++i) evals[i] = NAN;
    }
    // Ritz vectors (FP64) and the FP64 refinement of the kept pairs, in groups
    // of at most 8 columns (the widest FP64 block product)
    if (rc == BS_OK && (evecs || o.refine)) {
        if (nk > 64) { nk = 64; }
        const int gmax = std::min(nk, 8);
        const int kref = gmax <= 1 ? 1 : gmax <= 2 ? 2 : gmax <= 4 ? 4 : 8;
        double *X = evecs;
        double *Xown = nullptr, *HX = nullptr, *Yd = nullptr, *R = nullptr;
        Yd = (double *)alloc((size_t)nT * kref * sizeof(double));
        Xown = (double *)alloc((size_t)L.dim * kref * sizeof(double));
        HX = (double *)alloc((size_t)L.dim * kref * sizeof(double));
        R = (double *)alloc(2 * 64 * sizeof(double));
        if (!Yd || !Xown || !HX || !R) { rc = BS_ENOMEM; c->err = "lanczos: allocation failed"; }
        for (int g0 = 0; rc == BS_OK && g0 < nk; g0 += kref) {
            const int ng = std::min(kref, nk - g0);
            std::vector<double> Yh((size_t)nT * ng);
            for (int r = 0; r < nT; ++r)
                for (int m = 0; m < ng; ++m) Yh[(size_t)r * ng + m] = Z[(size_t)r * nv + g0 + m];
            cudaMemcpyAsync(Yd, Yh.data(), Yh.size() * sizeof(double), cudaMemcpyHostToDevice, L.s);
            cudaMemsetAsync(Xown, 0, (size_t)L.dim * kref * sizeof(double), L.s);
            blk_combine<T, K><<<L.ncta, 256, 0, L.s>>>(V, L.bstride, done, Yd, ng, Xown, kref, L.dim);
            if (o.refine) {
                // FP64 H psi, Rayleigh quotients and residuals
                if ((rc = launch_hx(c, Xown, HX, kref, BS_F64, L.s, c->err)) != BS_OK) break;
                LState L2 = L;
                L2.bstride = L.dim * kref;
                L2.padded = false;
                std::vector<double> xx(kref * kref), xh(kref * kref), hh(kref * kref);
                auto dots64 = [&](const double *A, const double *Bm, double *out) {
                    switch (kref) {
                    case 1: dots<double, 1>(L2, A, 1, Bm, out); break;
                    case 2: dots<double, 2>(L2, A, 1, Bm, out); break;
                    case 4: dots<double, 4>(L2, A, 1, Bm, out); break;
                    default: dots<double, 8>(L2, A, 1, Bm, out); break;
                    }
                };
                dots64(Xown, Xown, L.C);
                cudaMemcpyAsync(xx.data(), L.C, kref * kref * sizeof(double), cudaMemcpyDeviceToHost, L.s);
                dots64(Xown, HX, L.C);
                cudaMemcpyAsync(xh.data(), L.C, kref * kref * sizeof(double), cudaMemcpyDeviceToHost, L.s);
                cudaStreamSynchronize(L.s);
                std::vector<double> e(kref, 0.0);
                for (int m = 0; m < ng; ++m) e[m] = xh[m * kref + m] / xx[m * kref + m];   // Rayleigh quotient
                cudaMemcpyAsync(R, e.data(), kref * sizeof(double), cudaMemcpyHostToDevice, L.s);
                resid_inplace<<<L.ncta, 256, 0, L.s>>>(HX, Xown, R, ng, kref, L.dim);
                dots64(HX, HX, L.C);
                cudaMemcpyAsync(hh.data(), L.C, kref * kref * sizeof(double), cudaMemcpyDeviceToHost, L.s);
                cudaStreamSynchronize(L.s);
                for (int m = 0; m < ng; ++m) {
                    evals[g0 + m] = e[m];
                    if (rep) rep->residual[g0 + m] = std::sqrt(std::max(hh[m * kref + m], 0.0) / xx[m * kref + m]);
                }
            }
            if (X) {
                // copy the group's columns to the caller's [dim][nkeep] buffer
                cudaMemcpy2DAsync(X + g0, (size_t)nkeep * sizeof(double), Xown, (size_t)kref * sizeof(double),
                                  (size_t)ng * sizeof(double), (size_t)L.dim, cudaMemcpyDeviceToDevice, L.s);
            }
            cudaStreamSynchronize(L.s);
        }
    }
    stage("Ritz vectors and refinement");
    for (auto &e : ev) cudaEventDestroy(e);
    if (gexec) cudaGraphExecDestroy(gexec);
    cleanup();
    if (!stage("release") && rc == BS_OK) rc = BS_ECUDA;
    if (rc == BS_ECUDA && !cuda_fail.empty()) c->err = "lanczos: " + cuda_fail;
    else if (rc == BS_OK && !cuda_fail.empty()) { rc = BS_ECUDA; c->err = "lanczos: " + cuda_fail; }
    const auto t1 = std::chrono::steady_clock::now();
    if (rep) {
        rep->iterations = done;
        rep->breakdowns = breakdowns;
        rep->ms_matvec = ms_mv;
        rep->ms_reorth = ms_or;
        rep->ms_total = std::chrono::duration<double, std::milli>(t1 - t0).count();
        rep->n_kept = nk;
        rep->restarts = restarts;
        rep->matvec_blocks = matvecs;
        rep->resid_est = resid_est;
    }
    return rc;
}

template <typename T, int K>
static int block_dots_run(bs_ctx *c, const void *V, int nb, const void *W, double *C, cudaStream_t s)
{
    LState L;
    L.dim = c->basis.dim;
    L.bstride = L.dim * K;
    L.s = s;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    L.ncta = 2 * nsm;
    L.err = c->dev.err;
    cudaError_t e = cudaMallocAsync((void **)&L.partial, (size_t)L.ncta * nb * K * K * sizeof(double), s);
    if (e != cudaSuccess) { c->err = std::string("block dots: ") + cudaGetErrorString(e); return BS_ENOMEM; }
    dots<T, K>(L, (const T *)V, nb, (const T *)W, C);
    cudaFreeAsync(L.partial, s);
    if ((e = cudaGetLastError()) != cudaSuccess) { c->err = std::string("block dots: ") + cudaGetErrorString(e); return BS_ECUDA; }
    return BS_OK;
}

template <typename T, int K>
static int block_update_run(bs_ctx *c, const void *V, int nb, const double *C, void *W, cudaStream_t s)
{
    LState L;
    L.dim = c->basis.dim;
    L.bstride = L.dim * K;
    L.s = s;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    L.ncta = 2 * nsm;
    L.err = c->dev.err;
    if ((size_t)nb * K * K * sizeof(T) > 227 * 1024) { c->err = "block update: nb * k * k coefficients exceed shared memory"; return BS_EINVAL; }
    cudaError_t e = cudaFuncSetAttribute(blk_update<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((size_t)nb * K * K * sizeof(T)));
    if (e != cudaSuccess) { c->err = std::string("block update: ") + cudaGetErrorString(e); return BS_ECUDA; }
    update<T, K>(L, (const T *)V, nb, C, (T *)W);
    if ((e = cudaGetLastError()) != cudaSuccess) { c->err = std::string("block update: ") + cudaGetErrorString(e); return BS_ECUDA; }
    return BS_OK;
}

int run_block_update(bs_ctx *c, const void *V, int nb, const double *C, void *W, int k, bs_dtype dt, void *stream)
{
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return BS_ECUDA; }
    cudaStream_t s = (cudaStream_t)stream;
    if (dt == BS_F64) {
        switch (k) {
        case 1: return block_update_run<double, 1>(c, V, nb, C, W, s);
        case 2: return block_update_run<double, 2>(c, V, nb, C, W, s);
        case 4: return block_update_run<double, 4>(c, V, nb, C, W, s);
        default: return block_update_run<double, 8>(c, V, nb, C, W, s);
        }
    }
    switch (k) {
    case 1: return block_update_run<float, 1>(c, V, nb, C, W, s);
    case 2: return block_update_run<float, 2>(c, V, nb, C, W, s);
    case 4: return block_update_run<float, 4>(c, V, nb, C, W, s);
    default: return block_update_run<float, 8>(c, V, nb, C, W, s);
    }
}

int run_block_dots(bs_ctx *c, const void *V, int nb, const void *W, int k, bs_dtype dt, double *C, void *stream)
{
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return BS_ECUDA; }
    cudaStream_t s = (cudaStream_t)stream;
    if (dt == BS_F64) {
        switch (k) {
        case 1: return block_dots_run<double, 1>(c, V, nb, W, C, s);
        case 2: return block_dots_run<double, 2>(c, V, nb, W, C, s);
        case 4: return block_dots_run<double, 4>(c, V, nb, W, C, s);
        default: return block_dots_run<double, 8>(c, V, nb, W, C, s);
        }
    }
    switch (k) {
    case 1: return block_dots_run<float, 1>(c, V, nb, W, C, s);
    case 2: return block_dots_run<float, 2>(c, V, nb, W, C, s);
    case 4: return block_dots_run<float, 4>(c, V, nb, W, C, s);
    default: return block_dots_run<float, 8>(c, V, nb, W, C, s);
    }
}

int run_lanczos(bs_ctx *c, const bs_lanczos_opts &o_in, const void *pivot, double *evals, double *evecs,
                bs_lanczos_report *rep, const StrengthReq *sreq)
{
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return BS_ECUDA; }
    bs_lanczos_opts o = o_in;
    cudaStream_t own = nullptr;
    if (o.use_graph && !o.stream) {   // capture needs a created stream
        if ((e = cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking)) != cudaSuccess) { c->err = cudaGetErrorString(e); return BS_ECUDA; }
        o.stream = own;
    }
    struct Own {
        cudaStream_t s;
        ~Own() { if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); } }
    } guard{own};
    // kernel workspace before any capture (a failure only disables that path)
    {
        std::string ignored;
        (void)prepare_hx(c, o.k, o.dtype, ignored);
    }
    if (o.dtype == BS_F64) {
        switch (o.k) {
        case 1: return lanczos_run<double, 1>(c, o, pivot, evals, evecs, rep, sreq);
        case 2: return lanczos_run<double, 2>(c, o, pivot, evals, evecs, rep, sreq);
        case 4: return lanczos_run<double, 4>(c, o, pivot, evals, evecs, rep, sreq);
        default: return lanczos_run<double, 8>(c, o, pivot, evals, evecs, rep, sreq);
        }
    }
    switch (o.k) {
    case 1: return lanczos_run<float, 1>(c, o, pivot, evals, evecs, rep, sreq);
    case 2: return lanczos_run<float, 2>(c, o, pivot, evals, evecs, rep, sreq);
    case 4: return lanczos_run<float, 4>(c, o, pivot, evals, evecs, rep, sreq);
    default: return lanczos_run<float, 8>(c, o, pivot, evals, evecs, rep, sreq);
    }
}

// ---------------------------------------------------------------------------
// Allocation-free block inner products.  The per-CTA partial sums live in a
// fixed device array that the module carries; its device address is looked
// up once per device and then reused by every call.
static __device__ __align__(256) double g_noalloc_partials[BS_BLOCK_DOTS_NOALLOC_MAX];

namespace {

std::mutex g_noalloc_mtx;
double *g_noalloc_ptr[64] = {};

// Device address of g_noalloc_partials on device `dev` (which must be
// current); looked up on the first call for that device.
int noalloc_scratch(int dev, double **out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mtx);
    if (dev < 0 || dev >= 64) return BS_EINVAL;
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return BS_ECUDA;
        g_noalloc_ptr[dev] = (double *)p;
    }
    *out = g_noalloc_ptr[dev];
    return BS_OK;
}

template <typename T, int K>
int noalloc_dots_run(const void *V, int nb, const void *W, int64_t dim, double *C, cudaStream_t s, double *scratch,
                     int nsm)
{
    const int64_t per = (int64_t)nb * K * K;
    // as many CTAs as the fixed array holds partial blocks for, at most 2 per SM
    const int ncta = (int)std::max<int64_t>(1, std::min<int64_t>(2 * (int64_t)nsm, BS_BLOCK_DOTS_NOALLOC_MAX / per));
    blk_dots<T, K><<<ncta, kDotThreads, 0, s>>>((const T *)V, dim * K, nb, (const T *)W, dim, scratch, nullptr);
    reduce_parts<double>(scratch, ncta, (int)per, (int)per, C, nullptr, nullptr, K * K, s);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ECUDA;
}

}  // namespace

}  // namespace bs

extern "C" int bs_block_dots_noalloc(const void *V, int nb, const void *W, int64_t dim, int k, bs_dtype dtype,
                                     double *C, void *stream)
{
    if (!V || !W || !C || nb < 1 || dim < 1) return BS_EINVAL;
    if (k != 1 && k != 2 && k != 4 && k != 8) return BS_EINVAL;
    if (dtype != BS_F64 && dtype != BS_F32) return BS_EINVAL;
    if ((int64_t)nb * k * k > BS_BLOCK_DOTS_NOALLOC_MAX) return BS_ENOMEM;
    // the row-slot kernel loads a basis state's k values as 16-byte vectors
    // once they span 16 bytes or more: refuse pointers it would fault on
    const uintptr_t elem = (uintptr_t)k * (dtype == BS_F64 ? 8u : 4u), need = elem < 16 ? elem : 16;
    if ((uintptr_t)V % need || (uintptr_t)W % need || (uintptr_t)C % 8) return BS_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BS_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return BS_ECUDA;
    double *scratch = nullptr;
    const int rc = bs::noalloc_scratch(dev, &scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == BS_F64) {
        switch (k) {
        case 1: return bs::noalloc_dots_run<double, 1>(V, nb, W, dim, C, s, scratch, nsm);
        case 2: return bs::noalloc_dots_run<double, 2>(V, nb, W, dim, C, s, scratch, nsm);
        case 4: return bs::noalloc_dots_run<double, 4>(V, nb, W, dim, C, s, scratch, nsm);
        default: return bs::noalloc_dots_run<double, 8>(V, nb, W, dim, C, s, scratch, nsm);
        }
    }
    switch (k) {
    case 1: return bs::noalloc_dots_run<float, 1>(V, nb, W, dim, C, s, scratch, nsm);
    case 2: return bs::noalloc_dots_run<float, 2>(V, nb, W, dim, C, s, scratch, nsm);
    case 4: return bs::noalloc_dots_run<float, 4>(V, nb, W, dim, C, s, scratch, nsm);
    default: return bs::noalloc_dots_run<float, 8>(V, nb, W, dim, C, s, scratch, nsm);
    }
}
