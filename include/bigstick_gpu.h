/*
 * bigstick_gpu.h -- C ABI of libbsgpu.so: the factorized, on-the-fly product
 * y = H x of the M-scheme shell-model Hamiltonian on one GB300 (sm_103a).
 *
 * The method is the one of the BIGSTICK manual (arXiv:1801.08432):
 *   - basis: proton and neutron Slater determinants as occupation bitstrings,
 *     grouped into sectors by (2M, parity); every proton SD of a sector is
 *     combined with every neutron SD of the conjugate sector (M_p + M_n = M),
 *     proton index outer, neutron index inner (Sec. "Factorization of the
 *     basis", Table al27, basis-file pseudocode "pstart + nstart");
 *   - Hamiltonian: Eq. (hamdef), single-particle energies plus isospin-coupled
 *     two-body matrix elements V_JT(ab,cd) between normalized states (Sec.
 *     "Interaction files", Eq. tbmedef), pp/nn from T=1 and pn from
 *     Eq. (xpndef);
 *   - application: proton-only and neutron-only jumps, the pn term as a proton
 *     one-body jump times a neutron one-body jump (Sec. "The Lanczos
 *     algorithm and computational cost", jump discussion around Table jumps);
 *   - Lanczos with full reorthogonalization (Sec. "Standard Lanczos
 *     algorithm") and block Lanczos (Sec. "Block Lanczos").
 *
 * Conventions shared by every call
 *   - Single-particle states: orbit after orbit in input order, 2m ascending
 *     inside an orbit.  A Slater determinant is a uint64 bitmask (bit s =
 *     state s occupied), so at most 64 states per species.
 *   - Sectors: (2M, parity) with 2M ascending and parity + before -; inside
 *     a sector, SDs sorted by bitmask ascending.  Blocks: proton sectors in
 *     order, each with its conjugate neutron sector; basis index =
 *     block offset + ip_local * |S_n| + jn_local.
 *   - Vectors (x, y, gy, gx, pivot, evecs) are DEVICE buffers laid out
 *     [dim][k], the k vectors of a block contiguous per basis state (the
 *     row-wise block layout of Sec. "Block Lanczos").  Element type is double
 *     for BS_F64 and float for BS_F32.  Buffers must be 16-byte aligned.
 *     The caller owns them; the library never frees or keeps them.
 *   - `stream` is a cudaStream_t (0 = legacy default stream).  Work is
 *     enqueued asynchronously; the call returns before the GPU finishes
 *     unless stated otherwise.
 *   - Every call returns BS_OK (0) or a negative code; on error the output
 *     buffers are unspecified and bs_last_error() holds a message.  No C++
 *     exception crosses this interface.  A context is not thread-safe.
 *   - Calls that apply H (bs_apply_H, bs_apply_H_host, bs_apply_H_backward,
 *     bs_lanczos, bs_strength) share device workspace the context owns (the
 *     partial vectors of the core-grouped kernels, the host entry point's
 *     staging buffers).  Issue them on one stream, or order them with
 *     events: two such calls running at the same time on the GPU race.
 *     bs_apply_H_host_async orders its own products among themselves.
 */
#ifndef BIGSTICK_GPU_H
#define BIGSTICK_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bs_ctx bs_ctx;

/* One orbit (n, l, 2j, w) of the single-particle space (Sec. "Single-particle
 * space"); l fixes the parity (-1)^l.  w is the orbit's truncation weight,
 * read only by bs_build_basis_trunc (a non-negative integer there). */
typedef struct { int n, l, twoj, w; } bs_orbit;

/* One isospin-coupled two-body matrix element V_JT(ab,cd) in MeV, labels
 * 1-based orbit indices, in any label order and any list order (Sec.
 * "Interaction files"). */
typedef struct { int a, b, c, d, J, T; double v; } bs_tbme;

typedef enum { BS_F64 = 0, BS_F32 = 1 } bs_dtype;

enum {
    BS_OK = 0,
    BS_EINVAL = -1,      /* bad argument: orbits, Z/N, 2M parity vs A, TBME label or selection rule, k, dtype */
    BS_ENOBASIS = -2,    /* no basis built yet */
    BS_ENOINT = -3,      /* no interaction loaded yet */
    BS_ENOMEM = -4,      /* device or host allocation failed, or a memory cap was exceeded */
    BS_ECUDA = -5,       /* a CUDA call failed */
    BS_EBREAKDOWN = -6,  /* Lanczos breakdown that could not be restarted */
    BS_ETIMEOUT = -7     /* a device-side wait ran out of its iteration budget */
};

/* Creates a context on CUDA device `cuda_device`.  *out receives the handle.
 * cuda_device = -1 makes a host-only context: basis, decoupling and jump
 * tables are built on the CPU and nothing is uploaded; every product call
 * then fails with BS_EINVAL.  Errors: BS_EINVAL (no such device), BS_ECUDA. */
int bs_create(bs_ctx **out, int cuda_device);

/* Frees every table and workspace of the context (device and host). */
void bs_destroy(bs_ctx *ctx);

/* Message of the last failed call on this context ("" if none).  The string
 * stays valid until the next call on the context. */
const char *bs_last_error(const bs_ctx *ctx);

/* Builds the M-scheme basis of Z valence protons and N valence neutrons with
 * total 2M = twoM and parity (+1 or -1) over the given orbits (Sec.
 * "Factorization of the basis").  Replaces any earlier basis and interaction.
 * The orbits' w are ignored (no truncation).
 * Errors: BS_EINVAL (n_orbits <= 0, 2j even or <= 0, more than 64 states,
 * Z or N negative or larger than the number of states, twoM of the wrong
 * parity for A = Z + N, parity not +-1, empty basis, a sector of more than
 * 65,535 SDs). */
int bs_build_basis(bs_ctx *ctx, const bs_orbit *orbits, int n_orbits,
                   int Z, int N, int twoM, int parity);

/* The same basis under the W truncation of Sec. "Truncation of the many-body
 * space": each orbit carries its weight w (>= 0), a Slater determinant's W is
 * the sum of w over its occupied states, W_min is the smallest Z-proton plus
 * N-neutron total (the lowest-w states filled), and only states with
 * W_p + W_n <= W_min + max_excite are kept (max_excite = -1: no truncation,
 * as bs_build_basis).  Sectors are keyed by (2M, parity, W), sorted by 2M,
 * then parity (+ before -), then W; a proton sector pairs with every
 * conjugate neutron sector whose W fits, in neutron-sector order, so it may
 * head several blocks (the basis-file loop: proton sector, its conjugate
 * neutron sectors, proton SDs, neutron SDs).  bs_export_basis gives the
 * blocks; bs_debug_table "p_sec_w" / "n_sec_w" the sectors' W.  On such a
 * basis the products run on the tiled kernel (like-particle moves that
 * change W come from other blocks), and bs_apply_H_backward and bs_density
 * return BS_EINVAL.  Errors: as bs_build_basis, and BS_EINVAL for a negative
 * w or max_excite < -1. */
int bs_build_basis_trunc(bs_ctx *ctx, const bs_orbit *orbits, int n_orbits,
                         int Z, int N, int twoM, int parity, int max_excite);

/* Sizes of the built basis.  Any pointer may be NULL.  Errors: BS_ENOBASIS. */
int bs_basis_info(bs_ctx *ctx, int64_t *dim, int *n_psec, int *n_nsec,
                  int *n_psd, int *n_nsd, int *n_blocks);

/* Copies the basis to caller-allocated HOST arrays (for bit-exact checks):
 * p_bits[n_psd], n_bits[n_nsd]; p_sec[4*n_psec], n_sec[4*n_nsec] as
 * (2M, parity 0=+ 1=-, start, count); blocks[3*n_blocks] as (proton sector,
 * neutron sector, offset).  Errors: BS_ENOBASIS. */
int bs_export_basis(bs_ctx *ctx, uint64_t *p_bits, uint64_t *n_bits,
                    int64_t *p_sec, int64_t *n_sec, int64_t *blocks);

/* Loads the interaction: spe[n_spe] single-particle energies, one per orbit,
 * used for protons and neutrons alike; tbme[n_tbme] isospin-coupled elements.
 * An empty TBME list is legal (SPE only).  Decouples them to M-scheme
 * elements in FP64 (Eq. hamdef with Clebsch-Gordan coefficients of Edmonds,
 * Eq. xpndef for pn), builds the jump tables and uploads FP64 and FP32 copies
 * of all coefficients.  May be called again to replace the interaction.
 * Errors: BS_ENOBASIS; BS_EINVAL (n_spe != n_orbits, a label out of range,
 * T not 0/1, J outside a pair's triangle, same-orbit pair with J+T even,
 * parity change, the same element given twice); BS_ENOMEM; BS_ECUDA. */
int bs_load_interaction(bs_ctx *ctx, const double *spe, int n_spe,
                        const bs_tbme *tbme, int n_tbme);

/* y = H x for a block of k vectors (k in 1, 2, 4, 8), on `stream`.
 * x, y: device, [dim][k], dtype elements, distinct (no aliasing).  BS_F64
 * computes in double; BS_F32 reads/writes float and accumulates in float
 * with coefficients rounded once from the FP64 decoupling.  y is fully
 * overwritten.  Deterministic: every element of y is owned by one thread and
 * summed in a fixed order.  Errors: BS_ENOBASIS, BS_ENOINT, BS_EINVAL, BS_ECUDA. */
int bs_apply_H(bs_ctx *ctx, const void *x, void *y, int k, bs_dtype dtype, void *stream);

/* The same product with HOST buffers x_host, y_host ([dim][k]); copies in,
 * applies, copies out on `stream` and synchronizes it before returning.
 * Uses device buffers the context owns (allocated on first use, reused).
 * Errors as bs_apply_H plus BS_ENOMEM. */
int bs_apply_H_host(bs_ctx *ctx, const void *x_host, void *y_host, int k,
                    bs_dtype dtype, void *stream);

/* The same product with HOST buffers, enqueued on `stream` without waiting:
 * x_host is copied into the context's staging slot `slot` (0 or 1), H is
 * applied, and the result is copied into y_host.  On the GPU, the copy in
 * waits until the slot's previous call has finished copying out, and the
 * product waits until the previous call's product (on any stream) has ended,
 * since products share the context's workspace.  A caller that alternates
 * two streams and the two slots therefore overlaps one call's copies with
 * the other's product.  x_host and y_host must be pinned (cudaHostAlloc or
 * cudaHostRegister) for the copies to run asynchronously.  The caller must
 * not read y_host or rewrite x_host until `stream` has been synchronized.
 * The staging buffers are allocated on first use and reused (2 x 2 blocks).
 * Errors as bs_apply_H_host; BS_EINVAL for a slot other than 0 or 1. */
int bs_apply_H_host_async(bs_ctx *ctx, const void *x_host, void *y_host, int k,
                          bs_dtype dtype, void *stream, int slot);

/* Adjoint of y = H(theta) x, theta = (spe[n_spe], tbme values in the order
 * they were loaded).  gx = H gy (H is symmetric; device, [dim][k], dtype),
 * and if gtheta != NULL (HOST, n_spe + n_tbme doubles):
 *   gtheta[t] += sum over the k columns of gy^T (dH/dtheta_t) x,
 * the derivative of the pairing gy . H x -- with x = gy = psi (normalized) it
 * is the Hellmann-Feynman derivative dE/dtheta_t, the paper's "diagonal"
 * two-body density X_J(ab,cd) = dE/dV_J(ab,cd) for a TBME slot.  H is linear
 * in theta, so the transition densities gy . x over all jumps (pp and nn per
 * jump, pn per pair of decoupled operators; GPU kernels, FP64 accumulation)
 * are contracted on the host with dW/dtheta, built once per label set by
 * decoupling unit interactions.  x, gy, gx: distinct except x may equal gy.
 * Synchronizes the stream when gtheta != NULL.  Errors: as bs_apply_H,
 * BS_ENOMEM. */
int bs_apply_H_backward(bs_ctx *ctx, const void *x, const void *gy, void *gx, double *gtheta, int k,
                        bs_dtype dtype, void *stream);

/* The update half of a block Gram-Schmidt pass (Sec. "Block Lanczos": the
 * reorthogonalization of bs_lanczos): W[alpha][j] -= sum_b sum_i
 * V_b[alpha][i] C[b][i][j] for b < nb, with V nb consecutive [dim][k] blocks,
 * W one [dim][k] block not overlapping V (device, dtype) and C nb*k*k FP64
 * coefficients (device, e.g. from bs_block_dots), used in the vectors'
 * precision; per element the blocks are applied in order and within a
 * block i = 0..k-1, each as one fused multiply-add.  nb*k*k coefficients
 * must fit shared memory (227 KB).  Runs on `stream`.  Errors: BS_ENOBASIS,
 * BS_ENOINT, BS_EINVAL (null pointer, nb < 1, overlap, too many
 * coefficients, k, dtype), BS_ECUDA. */
int bs_block_update(bs_ctx *ctx, const void *V, int nb, const double *C, void *W, int k, bs_dtype dtype,
                    void *stream);

/* Inner products of basis vectors with FP64-grade accumulation (overlaps of
 * wave functions; the alpha, Gram and reorthogonalization products of
 * bs_lanczos): for b < nb, C[b][i][j] = sum_alpha V_b[alpha][i] W[alpha][j],
 * where V holds nb consecutive [dim][k] blocks and W one [dim][k] block
 * (device, dtype).  C: device, nb*k*k doubles.  FP64 vectors use FP64 fused
 * multiply-adds; FP32 vectors sum exact products in double-float; the
 * per-CTA partial sums (2 x SMs x nb x k x k doubles, allocated and freed
 * stream-ordered by the call) are reduced in FP64 in a fixed order, so the
 * result is bit-reproducible.  Errors: BS_ENOBASIS, BS_ENOINT, BS_EINVAL,
 * BS_ENOMEM, BS_ECUDA. */
int bs_block_dots(bs_ctx *ctx, const void *V, int nb, const void *W, int k, bs_dtype dtype, double *C,
                  void *stream);

/* Capacity, in doubles, of the fixed device array behind
 * bs_block_dots_noalloc (2 MiB per device that loads the library). */
#define BS_BLOCK_DOTS_NOALLOC_MAX 262144

/* The products of bs_block_dots, C[b][i][j] = sum_alpha V_b[alpha][i]
 * W[alpha][j] (V: nb consecutive [dim][k] blocks, W: one [dim][k] block, C:
 * nb*k*k doubles, all device memory the caller owns), computed without
 * allocating anything: no cudaMalloc, no cudaFree, no allocating library
 * call, and no context is needed.  It is for callers that cannot allocate
 * device memory where they need an overlap -- an application whose caching
 * allocator already owns the GPU's memory (a cudaMalloc there can fail or
 * fragment it), or a latency-critical loop that must not enter the driver's
 * allocator, where cudaFree also waits for the whole device.  The paper has
 * no counterpart: this is a deployment variant of the inner products the
 * Lanczos driver uses.
 * The per-CTA partial sums go to a fixed file-scope device array of
 * BS_BLOCK_DOTS_NOALLOC_MAX doubles that every GPU loading the library holds
 * until the process exits.  The first call on a device (the current one)
 * looks up that array's device address; make that first call before any
 * stream capture.  Every call writes all the partials it reads, so nothing is
 * carried over from the previous call, but all calls share the one array:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialized by the caller.  It always runs the row-slot kernel
 * (FP64 fused multiply-adds for FP64 vectors; exact FP32 products summed in
 * double-float for FP32 vectors; per-CTA partials added in FP64 in a fixed
 * order, so repeated calls are bit-identical).  bs_block_dots streams
 * 16-byte-aligned blocks through another kernel whose summation order
 * differs, so the two entry points agree to rounding, not bit for bit.  Up to
 * 2 x SMs CTAs run while nb*k*k <= BS_BLOCK_DOTS_NOALLOC_MAX / (2 x SMs);
 * larger requests run on fewer CTAs (one at the maximum).  V and W must be
 * aligned to min(16, k x element size) bytes and C to 8 bytes.  Runs on
 * `stream` (a cudaStream_t) on the current device.  Errors: BS_EINVAL (null
 * pointer, misaligned pointer, nb < 1, dim < 1, k not in 1, 2, 4, 8, bad
 * dtype; nothing is launched); BS_ENOMEM (nb*k*k >
 * BS_BLOCK_DOTS_NOALLOC_MAX); BS_ECUDA. */
int bs_block_dots_noalloc(const void *V, int nb, const void *W, int64_t dim, int k, bs_dtype dtype, double *C,
                          void *stream);

/* Options of bs_lanczos. */
typedef struct {
    int k;              /* block size: 1 (standard Lanczos), 2, 4 or 8 */
    bs_dtype dtype;     /* precision of the stored Lanczos vectors and of H x */
    int niter;          /* block iterations; clamped to dim / k */
    int nkeep;          /* eigenvalues returned (lowest first) */
    int refine;         /* 1: FP64 H psi of the lowest min(nkeep, 64) Ritz vectors,
                           evals become FP64 Rayleigh quotients, residuals reported */
    int reorth_passes;  /* Gram-Schmidt passes against all stored blocks (2 = default) */
    int use_graph;      /* 1: capture one block iteration in a CUDA graph (kernels read the
                           iteration number from a device counter) and replay it */
    void *stream;       /* cudaStream_t the work runs on (not the legacy default stream
                           when use_graph = 1: capture needs a created stream) */
    int nthick;         /* thick restart (Sec. "Thick-restart block Lanczos"): Ritz vectors
                           kept per restart, a multiple of k with nthick / k + 1 < niter;
                           0 = no restart.  The method needs nthick > nkeep (the paper
                           suggests about 3 nkeep): pairs beyond nthick are discarded at
                           every restart and may not converge */
    int max_restarts;   /* restarts at most (ignored when nthick = 0) */
    double tol;         /* stop restarting once the residual estimate of each of the lowest
                           nkeep pairs is <= tol (0 = run all max_restarts restarts) */
    int targeted;       /* 1: interior levels (Sec. "Targeted thick-restart Lanczos"): the
                           iteration runs on (H - target)^2, two products H X per block
                           iteration, so the levels nearest target come first; needs
                           refine = 1 and nkeep <= 8 (evals are then FP64 Rayleigh quotients
                           of H, ordered as the levels of (H - target)^2, residuals of H) */
    double target;      /* E_bar of the targeted operator */
} bs_lanczos_opts;

/* What bs_lanczos did. */
typedef struct {
    int iterations;          /* block iterations done */
    int breakdowns;          /* Gram eigenvalues below 1e-24 of the largest, restarted with random columns */
    int n_kept;              /* pairs with Ritz vectors / refinement (<= 64) */
    double residual[64];     /* |H psi - E psi| / |psi| in FP64, per refined pair */
    double delta_conv;       /* sum_{i <= nkeep+5} |E_i(n) - E_i(n-1)| / sqrt(nkeep+5) over the last iteration */
    double ms_matvec;        /* GPU time in H x */
    double ms_reorth;        /* GPU time in alpha, reorthogonalization, Gram and normalization */
    double ms_total;         /* wall time of the call */
    int restarts;            /* thick restarts done */
    int matvec_blocks;       /* block products H X done (restarts included; two per block
                                iteration when targeted) */
    double resid_est;        /* max over the lowest nkeep pairs of |B_last U_last,mu|, the
                                Lanczos estimate of |H psi - E psi| from the last T */
} bs_lanczos_report;

/* Block Lanczos with full reorthogonalization (Sec. "Standard Lanczos
 * algorithm": alpha first, then orthogonalization against every earlier
 * vector; Sec. "Block Lanczos": A_n = V_n^T W, O = W'^T W' = U L U^T,
 * B_n = L^(1/2) U^T, V_(n+1) = W' U L^(-1/2)), all on the GPU.
 * pivot: device [dim][k] block in opts->dtype (any full-rank block; it is
 * orthonormalized).  evals: host array of nkeep doubles (lowest first).
 * evecs: device [dim][nkeep] FP64 Ritz vectors of the lowest min(nkeep, 64)
 * pairs, or NULL.  report may be NULL.  Inner products accumulate in
 * extended precision (FP64, or exact FP32 products summed in double-float);
 * T is diagonalized in FP64 on the host.
 * Thick restart (opts->nthick > 0): after niter block iterations the lowest
 * nthick Ritz vectors of T replace the first nthick / k stored blocks, the
 * last Lanczos block becomes the next pivot, and T restarts in the arrow form
 * of Sec. "Thick-restart Lanczos" (Ritz values on the diagonal, coupling
 * r = B_last U[last block rows, 1:nthick] to the pivot block), so storage
 * stays at niter + 1 blocks however many block products the run takes.
 * Allocates its workspace (about (niter + 2 + nthick / k) dim k elements)
 * for the call and frees it.  Synchronizes the stream.  Errors: BS_ENOBASIS, BS_ENOINT, BS_EINVAL (k, dtype, niter,
 * nkeep, nthick, max_restarts, tol), BS_ENOMEM, BS_ECUDA, BS_EBREAKDOWN
 * (eigensolver failure). */
int bs_lanczos(bs_ctx *ctx, const bs_lanczos_opts *opts, const void *pivot, double *evals, double *evecs,
               bs_lanczos_report *report);

/* Strength function (Sec. "Generating strength function distributions",
 * Sec. "Block strength function"): block Lanczos from the caller's pivot
 * block W_0 (device [dim][k] in opts->dtype, any norm, full rank), which is
 * orthonormalized as V_0 = W_0 U Lambda^(-1/2) with O = W_0^T W_0 =
 * U Lambda U^T, so W_0 = V_0 B_0, B_0 = Lambda^(1/2) U^T.  After
 * opts->niter block iterations T = L E L^T is diagonalized (dense, FP64,
 * host) and, for the lowest n_out eigenvalues E_r of T, energies[r] = E_r
 * and strengths[i * n_out + r] = |<w_i|E_r>|^2 = (sum_j (B_0)_ji L_jr)^2
 * (HOST arrays of n_out and k * n_out doubles; entries past the dimension
 * of T, when the Krylov space is exhausted early, are NaN).  Summed over
 * all r, the strengths of column i give |w_i|^2, and sum_r E_r^p S_ir =
 * <w_i|H^p|w_i> for p < 2 niter.  opts->refine, nkeep and max_restarts are
 * ignored; opts->nthick must be 0.  Errors: as bs_lanczos, and BS_EINVAL for
 * a rank-deficient pivot block (an overlap eigenvalue below 1e-12 of the
 * largest) or n_out < 1. */
int bs_strength(bs_ctx *ctx, const bs_lanczos_opts *opts, const void *pivot, int n_out, double *energies,
                double *strengths, bs_lanczos_report *report);

/* One-body transition densities (Sec. "One-body density matrices and
 * occupations", the M-scheme matrix elements under the reduced densities):
 *   rho[((t * ns + i) * ns + l) * k * k + f * k + j] = <F_f| a+_i a_l |X_j>
 * for species t (0 protons, 1 neutrons), single-particle states i, l
 * (numbered orbit-major, 2m ascending; ns states) and the k columns of F and
 * X, two FP64 device blocks [dim][k] on this context's basis.  Only pairs
 * with 2m_i = 2m_l and equal parity can connect two states of one basis;
 * every other entry is 0.  rho: HOST array of 2 ns^2 k^2 doubles.  The
 * diagonal sums to the particle numbers times <F_f|X_j>.  Accumulated in
 * FP64 with atomics (last bits may vary between runs).  Synchronizes the
 * stream; allocates and frees a small work area.  Errors: BS_ENOBASIS,
 * BS_ENOINT (the jump tables come with the interaction), BS_EINVAL (k not
 * 1, 2, 4 or 8, null pointer), BS_ENOMEM, BS_ECUDA. */
int bs_density(bs_ctx *ctx, const double *F, const double *X, int k, double *rho, void *stream);

/* Measurement aid: the measured on-chip ceiling of the H x kernels' inner
 * step.  Every multiply-add of the product gathers one k-float element of a
 * source vector at an index read from a list and applies it to one or more
 * destination rows.  This times that step alone: one CTA of 576 threads per
 * SM walks a list of 8,192 seeded random indices, gathers the element at
 * each (where = 0: from a 96 KB table in shared memory; 1: from a 64 MB table
 * in global memory, L2-resident) and applies it to `rows` (1, 2 or 4)
 * accumulator rows with packed FP32 FMAs.  *gflops = 2 x multiply-adds / s
 * (k = 4 or 8).  Uses the context's device; allocates and frees ~64 MB;
 * synchronizes the stream.  Errors: BS_EINVAL, BS_ENOMEM, BS_ECUDA. */
int bs_gather_ceiling(bs_ctx *ctx, int where, int k, int rows, double *gflops, void *stream);

/* Test aid for the failure path of the bounded waits: launches one warp on
 * `stream` that waits on a shared-memory mbarrier nothing arrives at, through
 * the same bounded wait as the TMA kernels but giving up after `limit` tries
 * (1 .. 4,194,304, the kernels' own limit).  No copy is issued, so none is in
 * flight when it gives up.  The expiry is recorded in the context's status
 * word as a product kernel records it, so the next bs_sync_status returns
 * BS_ETIMEOUT (and clears it); the context stays usable.  Errors:
 * BS_ENOBASIS, BS_ENOINT (the status word comes with the interaction),
 * BS_EINVAL (limit), BS_ECUDA. */
int bs_debug_wait_expiry(bs_ctx *ctx, int limit, void *stream);

/* Test aid: all eigenvalues (ascending, w[n]) and the eigenvectors of the
 * lowest nvec (columns of Z, n x nvec row-major) of the symmetric n x n
 * matrix A (row-major, HOST), by the host FP64 solver bs_lanczos uses for T.
 * Errors: BS_EINVAL, BS_EBREAKDOWN. */
int bs_debug_eigh(int n, const double *A, double *w, double *Z, int nvec);

/* Test aid: the lowest nval eigenvalues (ascending, w[nval]) and the
 * eigenvectors of the lowest nvec <= nval (Z, n x nvec row-major) of the
 * symmetric n x n matrix A (row-major, HOST) whose entries vanish beyond
 * bandwidth bw, by the banded solver bs_lanczos uses for the block-tridiagonal
 * T (bisection on inertia counts, inverse iteration).  Errors: BS_EINVAL,
 * BS_EBREAKDOWN. */
int bs_debug_eigh_banded(int n, int bw, const double *A, int nval, double *w, double *Z, int nvec);

/* Chooses the H x kernel.  1 = the tiled kernel (one CTA per destination
 * row and 128-column tile, operands read through L1); 2..5 = variants
 * (threads per CTA, shared-memory budget) of the row kernel (one CTA per
 * destination proton row, the row accumulated in shared memory, source rows
 * staged by double-buffered TMA bulk copies); 6..10 = variants (consumer
 * warps, columns per thread, ring depth, shared-memory budget) of the
 * pipelined kernel (a producer warp fills a ring of shared-memory slots by
 * TMA, consumer warps keep their columns' sums in registers; needs k values
 * of 16 bytes or more per basis state); 11..20 = the core-grouped path for
 * FP32 with k = 4 or 8: a persistent kernel computes the pn term per
 * (Z-1)-proton core (up to four destination rows per staged source row) into
 * Z partial vectors (11, 13, 15, 16: 18 consumer warps with one 32-column
 * slice each; 12, 14: 9 warps with two slices each, a long and a short list;
 * 15, 16: as 13 with the whole 227 KB of shared memory and three or four
 * neutron-list buffers; 17, 18, 19: 227 KB, two list buffers; 20: 227 KB,
 * three list buffers); in 11, 12, 17
 * the pipelined kernel computes the like-particle terms into one more (17:
 * the first pipelined variant that fits, for neutron sectors wider than 576
 * columns); in 13..16 and 18..20 a second persistent kernel computes the pp
 * two-body term per
 * (Z-2)-proton core into C(Z,2) more and a row-tile kernel (4 rows per CTA,
 * 2 in 19 and 20, column tiles of 576 for wider sectors; 18: the first pipelined
 * variant that fits) the nn term and the proton single-particle energies
 * into one more; a last kernel
 * sums the partial vectors in a fixed order (workspace: up to
 * (Z + C(Z,2) + 1) x dim x k floats, allocated on first use, or by
 * bs_lanczos before it captures a graph; a first call inside a stream
 * capture without it falls back to the pipelined kernel).  A mode that does not fit
 * the basis falls back to the tiled kernel.  0 (default) = the mode bs_autotune picked
 * for the call's (k, dtype), else mode 13 where it applies (FP32, k = 4, 8),
 * else the first pipelined variant, else the first row variant.  All modes give the same result up to summation order.
 * Errors: BS_EINVAL. */
int bs_set_kernel(bs_ctx *ctx, int mode);

/* Number of selectable H x kernel modes (1..BS_KERNEL_MODES). */
#define BS_KERNEL_MODES 20

/* Times every kernel mode 1..BS_KERNEL_MODES for (k, dtype) on `stream` on
 * scratch vectors it allocates and frees (2 x dim x k elements), and records
 * the fastest for mode 0; *mode_out (may be NULL) receives it, ms_out (may be
 * NULL, else BS_KERNEL_MODES floats) the mean milliseconds per product of each
 * mode.
 * Synchronizes `stream`.  Errors: as bs_apply_H, BS_ENOMEM. */
int bs_autotune(bs_ctx *ctx, int k, bs_dtype dtype, void *stream, int *mode_out, float *ms_out);

/* Records `mode` (1..BS_KERNEL_MODES) as the autotuned mode for (k, dtype),
 * as bs_autotune would after timing, so that a tuning measured once (for
 * example by a previous process on the same GPU and basis) is replayed
 * without re-timing; calls with mode 0 then take it.  No device work.
 * Errors: BS_EINVAL (k not 1, 2, 4, 8; unknown dtype; mode out of range). */
int bs_set_tuned(bs_ctx *ctx, int k, bs_dtype dtype, int mode);

/* Synchronizes `stream` and reads the context's device status word: returns
 * BS_ETIMEOUT (and clears the word) if a kernel's bounded wait on an
 * mbarrier expired since the last check, else BS_OK.  Kernels that hit such
 * an expiry leave their output rows unwritten.  Errors: BS_ECUDA. */
int bs_sync_status(bs_ctx *ctx, void *stream);

/* Most products bs_time_kernel records. */
#define BS_TIME_MAX 4096

/* Kernel timing: records a pair of CUDA events, on the product's stream,
 * around the dominant kernel of each of the next n (<= BS_TIME_MAX) products
 * y = H x (the pn kernel in the core-grouped modes 11..20, else the one
 * kernel); n = 0 stops.  Discards earlier records.  Errors: BS_EINVAL,
 * BS_ECUDA. */
int bs_time_kernel(bs_ctx *ctx, int n);

/* Waits for the recorded events and writes the elapsed milliseconds of each
 * recorded launch to ms (may be NULL; else room for the count), the count to
 * *n.  Errors: BS_EINVAL, BS_ECUDA. */
int bs_kernel_times(bs_ctx *ctx, float *ms, int *n);

/* Test aid: copies a host-side table of the built interaction by name
 * ("pp_ptr", "pp_src", "pp_coef", "nn_*", "p1_ptr", "p1_ent", "p1_cls",
 * "n1_*", "wpn", "links", "ops", "op_lists", "stats", the pipelined and
 * core-grouped kernels' tables "pe_*", "ww", "ww_off", "core_units",
 * "core_src", "wc", "pp_units", "pps_row", "pps_w", "pdiag") into `out` (HOST,
 * caller-allocated; NULL to query the size).  *nbytes receives the size in
 * bytes.  Works on host-only contexts (bs_create with cuda_device = -1),
 * so the host builders can be checked on a machine without a GPU.
 * Errors: BS_ENOINT, BS_EINVAL (unknown name). */
int bs_debug_table(bs_ctx *ctx, const char *name, void *out, int64_t *nbytes);

#ifdef __cplusplus
}
#endif

#endif /* BIGSTICK_GPU_H */
