/*
 * ftlm.h -- C ABI of libftlm, a GB300 (sm_103a) implementation of the hot path of
 * the finite-temperature Lanczos method (FTLM) for spin-1/2 Heisenberg clusters
 * (Ghassemi Tabrizi & Kuehne, "GPU-accelerated finite-temperature Lanczos method
 * for spin Hamiltonians", arXiv 2605.26261).
 *
 * The path has three nested parts:
 *   H.v      the matrix-free action of H = sum_b J_b S_i . S_j (Eq. 1, with a
 *            coupling per bond) on one total-S^z sector, evaluated row by row as a
 *            gather (Eq. 12-14); the state-to-index map is either the compressed
 *            lookup table (CLT, Eq. 18-20, Algorithm 2) or combinatorial ranking
 *            (CR, Eq. 15-17, Algorithm 1).
 *   Lanczos  the three-term recurrence without reorthogonalization around it,
 *            with the dot product and norm fused into the H.v launches, followed
 *            by the small tridiagonal eigenproblem (Sec. 2, FTLM paragraph).
 *   FTLM     the stochastic trace estimator over random start vectors and S^z
 *            sectors, giving E(T), C(T) and chi(T) (Eq. 2-9).
 *
 * Conventions for every call:
 *   - Pointers named *_dev are device pointers (cudaMalloc'd or from a caching
 *     allocator) owned by the caller; other pointers are host memory.  Device
 *     pointers of vectors must be 16-byte aligned (32-byte for blocks whose rows
 *     are 32 bytes or more, see ftlm_hv_block).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is queued
 *     on it asynchronously; outputs are valid once the stream reaches that point.
 *   - Every call returns an ftlm_status; nothing aborts, throws or exits.  On a
 *     failure ftlm_last_error() returns a message for the calling host thread.
 *     FTLM_ECUDA means a CUDA runtime call failed (the message names it).
 *   - No call spins on the device: there is no device-side wait to time out.
 *   - Sector basis order: labels n = sum_k a_k 2^k with a_k = m_k + 1/2 (bit k = 1
 *     means site k is up, Eq. 11) in increasing order; sector index = position
 *     in that order.  A sector is fixed by its up-spin count K = N/2 + S^z
 *     (Eq. 17), passed as two_sz = 2 S^z = 2K - N.
 *   - dtype selects the storage and gather type of vectors: FTLM_F32 or FTLM_F64.
 *     Dot products, norms, the tridiagonal eigenproblem and the thermodynamic
 *     sums are FP64 in both cases.
 */
#ifndef FTLM_H
#define FTLM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FTLM_OK = 0,
    FTLM_EINVAL = 1,       /* an argument is out of range or inconsistent          */
    FTLM_ENOMEM = 2,       /* device allocation failed / workspace too small       */
    FTLM_EUNSUPPORTED = 3, /* valid request outside what the library implements    */
    FTLM_ECUDA = 4,        /* a CUDA runtime call failed                           */
    FTLM_ETIMEOUT = 5,     /* reserved: a bounded device wait expired              */
    FTLM_ENOCONV = 6       /* a tridiagonal eigenproblem did not converge          */
} ftlm_status;

typedef enum {
    FTLM_RANK_AUTO = 0, /* CLT if N <= 32, D < 2^20 and its tables fit in 1/4 of device memory, else CR */
    FTLM_RANK_CLT = 1,  /* compressed lookup table: basis array + {M_b, C_b} (Eq. 18-21) */
    FTLM_RANK_CR = 2    /* combinatorial ranking (Eq. 15-17), digit blocks via tables   */
} ftlm_rank_mode;

typedef enum { FTLM_F64 = 0, FTLM_F32 = 1 } ftlm_dtype;

typedef enum { FTLM_VEC_GAUSS = 0, FTLM_VEC_RADEMACHER = 1 } ftlm_vec_dist;

typedef struct ftlm_basis ftlm_basis; /* one (cluster, N, S^z) sector; opaque */

#define FTLM_MAX_SITES 36
#define FTLM_MAX_BONDS 256
#define FTLM_MAX_LANCZOS 1024
#define FTLM_MAX_SECTORS 64

/* ---------------------------------------------------------------- sectors ---
 * ftlm_basis_create -- set up one S^z sector of the cluster (step a1).
 *   N          sites, 1 <= N <= FTLM_MAX_SITES.
 *   two_sz     2 S^z; |two_sz| <= N and two_sz = N (mod 2).
 *   n_bonds    0 <= n_bonds <= FTLM_MAX_BONDS; bond b couples sites bi[b] != bj[b]
 *              (0 <= bi, bj < N) with J[b] (host arrays); an unordered pair may
 *              appear only once.  H = sum_b J[b] S_bi . S_bj (Eq. 1 with J per bond).
 *   mode       rank strategy.  CLT needs N <= 32 and stores the sorted basis
 *              (4 D bytes) and the CLT (8 ceil(2^N/32) bytes, Eq. 21); CR stores
 *              only small digit-block tables (Eq. 15-16) and needs D < 2^32.
 *   stream     tables are built on it; create returns after that work has
 *              completed on `stream` (no other stream is waited for), so the basis
 *              is usable at once on any stream.
 *   out        receives the handle; the library owns the device tables it holds:
 *              one block from a per-device stream-ordered memory pool, so creating
 *              and releasing sectors does not synchronize the device.
 * Errors: EINVAL (ranges, duplicate pair, i == j), EUNSUPPORTED (CLT with N > 32,
 * D >= 2^32), ENOMEM, ECUDA.
 */
ftlm_status ftlm_basis_create(int N, int two_sz, int n_bonds, const int *bi, const int *bj,
                              const double *J, ftlm_rank_mode mode, void *stream,
                              ftlm_basis **out);

/* ftlm_basis_create_spin -- the sector of total S^z = two_sz / 2 for local spin
 * s = two_s / 2 (Sec. 2: labels with base-d digits a_k = m_k + s, d = 2s + 1,
 * Eq. 11; digit sum A = N s + S^z, Eq. 17; H.v rows of Eq. 12 with the ladder
 * coefficients of Eq. 13-14 for general s).
 *   two_s = 1 is ftlm_basis_create with FTLM_RANK_AUTO.  For 2 <= two_s <= 7 the
 *   rank is Algorithm 1 in base d with digit blocks (mode FTLM_RANK_CR): N <= 16,
 *   d^(N - L) <= 2^27 high labels (L low digits with d^L <= 2^14), D < 2^32.
 *   two_sz must have the parity of N two_s.  Bond arguments, stream and ownership
 *   as for ftlm_basis_create.  The handle works with every entry point that takes
 *   a basis (ftlm_basis_labels returns base-d labels sum_k a_k d^k; ftlm_basis_clt
 *   is EUNSUPPORTED); ftlm_basis_updates is N_nz of Eq. 10.  Chain keys of
 *   ftlm_lanczos use (N | two_s << 8, A) in place of (N, K).
 * Errors: EINVAL (ranges, parity, duplicate pair, i == j), EUNSUPPORTED (two_s > 7,
 * N > 16, table or dimension limits), ENOMEM, ECUDA. */
ftlm_status ftlm_basis_create_spin(int N, int two_s, int two_sz, int n_bonds, const int *bi, const int *bj,
                                   const double *J, void *stream, ftlm_basis **out);

/* ftlm_basis_create_sectors -- n sectors (2 S^z = two_sz[k], 1 <= n <= 64) of one
 * cluster, as n calls of ftlm_basis_create (two_s = 1, with `mode`) or
 * ftlm_basis_create_spin (two_s > 1, mode ignored), with at most one wait for
 * `stream`: wait != 0 returns once every table is built; wait = 0 returns once
 * their builds are queued on `stream`, and the caller orders every use of the
 * tables on other streams after that point (an event) -- a request loop that keeps
 * the device busy then never blocks on table builds.  The host-side queries
 * (ftlm_basis_dim, _bytes, _mode, _updates) answer at once either way.  out
 * receives n handles, each released by ftlm_basis_destroy(_async).  On any error
 * nothing is kept (every out[k] = NULL, tables freed in the order of `stream`) and
 * the first error is returned. */
ftlm_status ftlm_basis_create_sectors(int N, int two_s, int n, const int *two_sz, int n_bonds, const int *bi,
                                      const int *bj, const double *J, ftlm_rank_mode mode, int wait, void *stream,
                                      ftlm_basis **out);

/* Release the handle and its device tables.  Waits until the device has finished
 * all queued work first (any stream may still read the tables).  NULL is ignored. */
void ftlm_basis_destroy(ftlm_basis *basis);

/* Release the handle at once and return its device tables to the pool in the order
 * of `stream`, without waiting: every kernel that reads the tables must already be
 * queued on `stream`, or be ordered before this point of `stream` by the caller
 * (cudaStreamWaitEvent).  For request loops that retire jobs while others run.
 * NULL is ignored (FTLM_OK).  ECUDA if the release cannot be queued (the handle is
 * freed regardless). */
ftlm_status ftlm_basis_destroy_async(ftlm_basis *basis, void *stream);

/* ftlm_basis_set_schedule -- how the Lanczos H.v launches of this sector walk the
 * rows (CR rank mode at s = 1/2; other sectors ignore it).  Eq. 12 is evaluated
 * row by row in either case; only the order of the work and the launches differ.
 *   FTLM_HV_ONE_WALK  one launch over the rows in sector (label) order.
 *   FTLM_HV_SPLIT     two launches: the rows near label order (tiles of 32
 *                     low-block ranks x 4 high patterns) with the bonds that
 *                     touch the low digit block, then the rows in the transposed
 *                     order (low-block rank fixed per lane, high patterns in turn)
 *                     with the bonds inside the high block, which adds its terms
 *                     to the first launch's output and finishes alpha_j.  A bond
 *                     inside the high block moves a row by thi[h ^ m] - thi[h],
 *                     far beyond L2 for the top sites in label order, but within
 *                     the same 32 columns in the transposed order.
 *   FTLM_HV_AUTO      (default) SPLIT when one block of B vectors of the call
 *                     holds at least 256 MiB (FP32 rows of 32 bytes or more:
 *                     blocks of 8 or 16), 768 MiB (other FP32 blocks) or 1 GiB
 *                     (FP64) and at least
 *                     16 bonds lie inside the high block, else ONE_WALK (the
 *                     crossover measured on GB300; the split moves two row
 *                     streams per step, the one walk misses L2 on long jumps).
 *   rows_per_tile: high patterns per tile of the transposed walk, 1..32, or 0 for
 *   the default (8).  SPLIT needs 1..64 bonds inside the high block (the N - L
 *   highest sites, L = min(N, 14)); otherwise the sector runs one walk.  Results
 *   agree with ONE_WALK up to the summation order of each row (FP rounding).
 *   Not thread-safe against Lanczos calls on the same basis.  EINVAL for a bad
 *   schedule or rows_per_tile. */
typedef enum { FTLM_HV_AUTO = 0, FTLM_HV_ONE_WALK = 1, FTLM_HV_SPLIT = 2 } ftlm_hv_schedule;
ftlm_status ftlm_basis_set_schedule(ftlm_basis *basis, ftlm_hv_schedule schedule, int rows_per_tile);

/* The walks (FTLM_HV_ONE_WALK or FTLM_HV_SPLIT) that Lanczos calls on this basis
 * with blocks of B vectors of dtype use under its current schedule.  EINVAL for a
 * bad B or dtype. */
ftlm_status ftlm_basis_hv_schedule(const ftlm_basis *basis, int B, ftlm_dtype dtype, ftlm_hv_schedule *used);

/* Sector dimension D = C(N, K). */
ftlm_status ftlm_basis_dim(const ftlm_basis *basis, uint64_t *dim);

/* Device bytes held by the basis tables (for admission by free memory). */
ftlm_status ftlm_basis_bytes(const ftlm_basis *basis, uint64_t *table_bytes);

/* Rank mode actually in use (AUTO resolved). */
ftlm_status ftlm_basis_mode(const ftlm_basis *basis, ftlm_rank_mode *mode);

/* Matrix-element updates applied by one H.v on one vector: D diagonal terms plus
 * every off-diagonal ladder term, D + 2 sum_b C(N-2, K-1) (Eq. 10 at s = 1/2). */
ftlm_status ftlm_basis_updates(const ftlm_basis *basis, uint64_t *updates);

/* Sector labels of indices first .. first+count-1 into labels_dev (uint64[count]);
 * CLT reads the stored basis array, CR unranks (the inverse map of Sec. 2).
 * EINVAL when first + count > D. */
ftlm_status ftlm_basis_labels(const ftlm_basis *basis, uint64_t first, uint64_t count,
                              uint64_t *labels_dev, void *stream);

/* Sector index of each label (uint64[count]) into index_dev (int64[count]), -1 for
 * a label outside the sector or >= 2^N; uses the basis' own rank strategy. */
ftlm_status ftlm_basis_rank(const ftlm_basis *basis, uint64_t count, const uint64_t *labels_dev,
                            int64_t *index_dev, void *stream);

/* CLT arrays of Eq. 18 (CLT mode only, else EUNSUPPORTED): mask_dev and prefix_dev
 * receive ceil(2^N/32) uint32 each (occupancy masks M_b and prefix counts C_b). */
ftlm_status ftlm_basis_clt(const ftlm_basis *basis, uint32_t *mask_dev, uint32_t *prefix_dev,
                           void *stream);

/* -------------------------------------------------------------------- H.v ---
 * ftlm_hv -- y = H x on the sector (step a3; Eq. 12 with Eq. 13-14 at s = 1/2):
 *   y[t] = (sum_b J_b m_i m_j) x[t] + sum_{b antiparallel in n_t} (J_b / 2) x[rank(n_t with
 *          spins i, j exchanged)];
 * for a general-spin basis (ftlm_basis_create_spin) the two ladder terms of every
 * bond with the coefficients of Eq. 13 and Eq. 14.
 * x_dev, y_dev: D elements of dtype (float or double), contiguous; x and y must not
 * overlap.  One thread per row, no atomics.  No scratch memory.
 */
ftlm_status ftlm_hv(const ftlm_basis *basis, ftlm_dtype dtype, const void *x_dev, void *y_dev,
                    void *stream);

/* ftlm_hv_block -- Y = H X for a block of B vectors stored interleaved: entry
 * (t, r) of vector r at X[t * B + r] (B in {1, 4, 8, 16}; x_dev, y_dev hold D * B
 * elements of dtype, 32-byte aligned when a row of B entries is 32 bytes or
 * more, else 16-byte aligned; EINVAL otherwise).  Each row's rank work is shared
 * by the B vectors (the batched scheme of Sec. 3.4); column r of Y is
 * bit-identical to ftlm_hv on column r of X.  EINVAL for another B. */
ftlm_status ftlm_hv_block(const ftlm_basis *basis, ftlm_dtype dtype, int B, const void *x_dev,
                          void *y_dev, void *stream);

/* ---------------------------------------------------------------- Lanczos ---
 * Workspace bytes ftlm_lanczos / ftlm_lanczos_from need for R chains of at most M
 * steps: two blocks of D x B_w elements of dtype plus O(R M) coefficients, and for
 * CR spin-1/2 sectors ceil(D / 32) x B_w doubles of per-tile dot-product sums; B_w
 * is the widest block of chains the call runs at once (chains go in blocks of 16,
 * 8 or 4 interleaved vectors, up to the width of ftlm_lanczos_set_block -- by
 * default 8 in FP32 and 4 in FP64 -- then single chains).  EINVAL for R < 1 or M
 * outside 1..FTLM_MAX_LANCZOS. */
ftlm_status ftlm_lanczos_workspace_bytes(const ftlm_basis *basis, int R, int M, ftlm_dtype dtype,
                                         uint64_t *bytes);

/* ftlm_lanczos_set_block -- widest block of chains that later ftlm_lanczos,
 * ftlm_lanczos_from and ftlm_lanczos_workspace_bytes calls use: 1 (every chain
 * on its own, the plain one-vector path), 4, 8 or 16; 0 restores the default
 * (FTLM_BLOCK from the environment, else 8 in FP32 and 4 in FP64).  Process-wide;
 * size workspaces after setting it.  EINVAL for another width. */
ftlm_status ftlm_lanczos_set_block(int width);

/* ftlm_lanczos -- R Lanczos chains (steps a2, a4, a5) on one sector.
 *   Chain r starts from a counter-based random vector keyed by (seed, N, K, r):
 *     u(c)  = F(key + (c+1) G), c-th output of splitmix64 from state key,
 *             G = 0x9E3779B97F4A7C15, F the splitmix64 output function;
 *     key   = F(F(seed + G) + (N << 48 | K << 32 | r) + G);
 *     GAUSS:      x_t = sqrt(-2 ln U1) cos(2 pi U2), U1 = ((u(2t) >> 11) + 1) 2^-53,
 *                 U2 = (u(2t+1) >> 11) 2^-53;
 *     RADEMACHER: x_t = -1 if the top bit of u(t) is set, else +1;
 *   normalized in FP64, then rounded to dtype.
 *   Recurrence (Paige's ordering, no reorthogonalization), for j = 1 .. min(M, D):
 *     y = H q_j - beta_{j-1} q_{j-1};  alpha_j = <q_j, y>;  w = y - alpha_j q_j;
 *     beta_j = ||w||;  q_{j+1} = w / beta_j.
 *   The chain stops after step j (m_eff = j) when beta_j <= tau = 100 u (3/4)
 *   sum_b |J_b| (u = 2^-53 for F64, 2^-24 for F32).
 *   Ritz step (FP64 on the device): theta_k, w_k = s_{k,1}^2 of the m_eff x m_eff
 *   tridiagonal T, ascending in theta.
 *   Chains run in blocks (see ftlm_lanczos_workspace_bytes) through ftlm_hv_block's
 *   kernel; every chain's arithmetic is its own, so a chain's result does not
 *   depend on the other chains of its block, up to the summation order of the
 *   dot products.  Every sum runs in a fixed order for a given sector, block width
 *   and device, so repeated calls give bit-identical outputs (CR launches hand out
 *   row tiles dynamically, but each tile's sums have a slot of their own).
 * Outputs (device, row r of chain r, each row M long, entries >= m_eff zero):
 *   theta_dev, weight_dev: double[R*M];  m_eff_dev: int[R];
 *   alpha_dev, beta_dev: double[R*M] or NULL (Lanczos coefficients; beta row r
 *   holds beta_1 .. beta_{m_eff-1}).
 * work_dev: caller-owned scratch of at least ftlm_lanczos_workspace_bytes() bytes,
 *   256-byte aligned; its contents are overwritten.  ENOMEM when too small.
 * The call only queues work on `stream`; it allocates nothing.
 */
ftlm_status ftlm_lanczos(const ftlm_basis *basis, int R, int M, uint64_t seed,
                         ftlm_vec_dist dist, ftlm_dtype dtype, void *work_dev, uint64_t work_bytes,
                         double *theta_dev, double *weight_dev, int *m_eff_dev, double *alpha_dev,
                         double *beta_dev, void *stream);

/* ftlm_lanczos_from -- as ftlm_lanczos, but chain r starts from the caller's vector
 * start_dev + r*D (double[R*D], need not be normalized; a zero vector gives
 * m_eff = 0).  Used for exact-trace runs (unit vectors) and for feeding identical
 * start vectors to another implementation. */
ftlm_status ftlm_lanczos_from(const ftlm_basis *basis, int R, int M, const double *start_dev,
                              ftlm_dtype dtype, void *work_dev, uint64_t work_bytes,
                              double *theta_dev, double *weight_dev, int *m_eff_dev,
                              double *alpha_dev, double *beta_dev, void *stream);

/* ftlm_lanczos_noalloc -- ftlm_lanczos without a caller workspace and without any
 * device allocation.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc at all, or not at the time of the call, e.g.
 * a host application that owns every device allocation and forbids new ones after
 * start-up, or a caller that must not risk the implicit device synchronization
 * that cudaMalloc/cudaFree can cause.
 *   Scratch: a file-scope __device__ array of FTLM_NOALLOC_SCRATCH_BYTES inside the
 *   library.  Every GPU that loads the library holds it until the process exits.
 *   The first call on a device looks up the array's device address on the current
 *   device (cudaGetSymbolAddress) and caches it with the id of the current
 *   context; make that first call before any stream capture.  A device reset
 *   (cudaDeviceReset) loads the library's device code again at a new address: the
 *   next call sees the new context and looks the address up again, so after a
 *   reset, too, the first call should come before any stream capture.
 *   Limit: the call is accepted when ftlm_lanczos_workspace_bytes() for the same
 *   (basis, R, M, dtype) is at most FTLM_NOALLOC_SCRATCH_BYTES (the exact test),
 *   else FTLM_EUNSUPPORTED.  That workspace is about 2 B_w D s + D B_w / 4 bytes
 *   plus O(R M) coefficients, with s = 8 (FP64) or 4 (FP32) bytes and B_w the widest
 *   block of chains of the call: the largest of 16, 8, 4 not above both R and the
 *   block width of ftlm_lanczos_set_block (default 4 in FP64, 8 in FP32), else 1.
 *   With the 32 MiB array that admits about D <= 2.0 million (R < 4) and 0.5
 *   million (R >= 4) in FP64; 4.0 million (R < 4), 1.0 million (4 <= R < 8) and
 *   0.5 million (R >= 8) in FP32.
 *   Sharing: all calls on a device use the same array and it keeps the previous
 *   call's contents; each call clears what must start at zero.  Calls whose work
 *   overlaps on the GPU (different streams, or different host threads) race on the
 *   array; serialize them.
 *   Arguments and outputs as for ftlm_lanczos.  Allocates nothing: no cudaMalloc,
 *   cudaFree or allocating library routine. */
#define FTLM_NOALLOC_SCRATCH_BYTES (32ull << 20)
ftlm_status ftlm_lanczos_noalloc(const ftlm_basis *basis, int R, int M, uint64_t seed,
                                 ftlm_vec_dist dist, ftlm_dtype dtype, double *theta_dev,
                                 double *weight_dev, int *m_eff_dev, double *alpha_dev,
                                 double *beta_dev, void *stream);

/* ------------------------------------------------------------- batches ---
 * Many sectors (of one or many clusters) in one go: the batched form of
 * ftlm_lanczos for workloads of many small sectors, where one launch sequence
 * per sector would be launch-bound.
 *
 * ftlm_batch_item: chains r = 0 .. R-1 of `basis`, keyed as chains
 *   first_chain + r under `seed` (the start-vector definition of ftlm_lanczos);
 *   outputs theta_dev, weight_dev (double[R*M]) and m_eff_dev (int[R]) as for
 *   ftlm_lanczos.  The basis and the outputs must outlive every run of the batch.
 * ftlm_batch_create -- plan a batch: sectors with D <= 32768 are cut into units
 *   of `block` chains (block = 1, 4, 8 or 16; 0 = 16 for FP32, 8 for FP64) that one
 *   persistent kernel runs, one CTA per unit at a time, each unit's chains entirely
 *   inside its CTA (vectors in a per-CTA workspace slot, CTA-local reductions).
 *   Larger spin-1/2 sectors with N <= 32, and every general-spin sector, are cut
 *   into units of `block` chains that advance together, all units of a wave per
 *   launch (two launches per Lanczos step: H.v with alpha, update with beta;
 *   per-unit reductions over tiles of 2048 rows for H.v, handed out in order from
 *   a counter, and 16384 rows for the update; waves of at most FTLM_MS_WAVE_MB =
 *   256 MB of vectors) on a stream forked from the caller's.  Spin-1/2 sectors
 *   with N > 32 run the launch sequence of ftlm_lanczos with blocks of up to
 *   `block` chains, spread over up to `streams` side streams (1..8; 0 =
 *   FTLM_BATCH_STREAMS or 4).  Uploads the plan's descriptors on
 *   `stream` (one block from the library's device memory pool, owned by the
 *   batch) and returns when they are in place.  EINVAL for an empty batch or bad
 *   items.
 * ftlm_batch_workspace_bytes -- scratch the plan needs (per-CTA vector slots,
 *   O(chains M) coefficients, the vectors of the largest wave, one sector
 *   workspace per side stream).
 * ftlm_batch_run -- queue the batch on `stream`: memsets, kernel launches and
 *   event records/waits only, so a run can be captured into a CUDA graph (the side
 *   streams join the capture) and replayed.  Results match ftlm_lanczos on each
 *   item up to the summation order of the dot products; a chain's results do not
 *   depend on the other items of the batch nor on the side-stream assignment.  ENOMEM when the workspace is too small.  Runs of one
 *   batch must not overlap.
 * ftlm_batch_destroy -- waits for the device to finish queued work, then releases.
 * ftlm_batch_destroy_async -- releases without waiting; the descriptors return to
 *   the pool in the order of `stream`, which every run of the batch must precede.
 */
typedef struct {
    const ftlm_basis *basis;
    int R;
    int first_chain;
    uint64_t seed;
    double *theta_dev;
    double *weight_dev;
    int *m_eff_dev;
} ftlm_batch_item;

typedef struct ftlm_batch ftlm_batch;

ftlm_status ftlm_batch_create(int n_items, const ftlm_batch_item *items, int M, ftlm_vec_dist dist,
                              ftlm_dtype dtype, int block, int streams, void *stream, ftlm_batch **out);
ftlm_status ftlm_batch_workspace_bytes(const ftlm_batch *batch, uint64_t *bytes);
ftlm_status ftlm_batch_run(const ftlm_batch *batch, void *work_dev, uint64_t work_bytes, void *stream);
void ftlm_batch_destroy(ftlm_batch *batch);
ftlm_status ftlm_batch_destroy_async(ftlm_batch *batch, void *stream);

/* Batch plans with explicit tile sizes.  ftlm_batch_plan: block and streams as for
 * ftlm_batch_create; tile_rows = rows per H.v tile and stream_rows = rows per tile
 * of the start/update kernels of the multi-sector path (multiples of 256 up to
 * 2^20; 0: 2048 and 16384).  ftlm_batch_create_plan plans with them (results agree
 * with other plans up to the summation order of the per-tile sums).
 * ftlm_batch_autotune_plan times candidate plans on the items (each candidate: one
 * untimed and one timed run, as ftlm_batch_autotune) by coordinate search -- block
 * width in {4, 8, 16} (and side streams in {1, 2, 4, 8} when an item runs on
 * them), then tile_rows in {1024, 2048, 4096} and stream_rows in {8192, 16384,
 * 32768} when an item runs on the multi-sector path -- and returns the fastest in
 * *best; the first max_tried candidates and their times go to tried / ms_out,
 * *n_tried = candidates timed.  Blocks the host; overwrites the items' outputs. */
typedef struct {
    int block;
    int streams;
    int tile_rows;
    int stream_rows;
} ftlm_batch_plan;
ftlm_status ftlm_batch_create_plan(int n_items, const ftlm_batch_item *items, int M, ftlm_vec_dist dist,
                                   ftlm_dtype dtype, const ftlm_batch_plan *plan, void *stream, ftlm_batch **out);
ftlm_status ftlm_batch_autotune_plan(int n_items, const ftlm_batch_item *items, int M, ftlm_vec_dist dist,
                                     ftlm_dtype dtype, void *stream, ftlm_batch_plan *best, ftlm_batch_plan *tried,
                                     float *ms_out, int max_tried, int *n_tried);

/* ftlm_batch_autotune -- pick the block width and side-stream count of a batch by
 * timing it: for block in {4, 8, 16} and (when some item runs on the side
 * streams) streams in {1, 2, 4, 8}, plan the batch, run it once untimed and once
 * between CUDA events on `stream`, and return the fastest pair in *block_out,
 * *streams_out (streams 1 when no item uses them).  ms_out, if
 * not NULL, receives the timed runs (float[12], index 4 * (0, 1, 2 for block 4, 8,
 * 16) + (0..3 for streams 1, 2, 4, 8); entries not tried are left alone).  Blocks
 * the host until the runs finish.  The items' outputs are overwritten.  Workspaces
 * come from the library's pool and are released before return.  Tune on a
 * representative subset of a large job: each candidate runs the whole list twice.
 * Errors as ftlm_batch_create and ftlm_batch_run. */
ftlm_status ftlm_batch_autotune(int n_items, const ftlm_batch_item *items, int M, ftlm_vec_dist dist,
                                ftlm_dtype dtype, void *stream, int *block_out, int *streams_out,
                                float *ms_out);

/* ------------------------------------------------------- continuous flow ---
 * A request loop's chain-level continuous batching: the chains of many sectors
 * advance together, one multi-sector H.v launch per rank kind and one update
 * launch per Lanczos step, and sectors join and leave at step boundaries.  A
 * sector added while others are at step 40 runs its step 1 in the next launch; a
 * sector that reaches its last step gets its Ritz step and its device memory
 * serves the next one.  Each sector's chains are cut into units of `block`
 * chains with the tiles and per-unit reductions of the batch's multi-sector path,
 * so a sector's results are bit-identical alone, in any mix and whenever it was
 * added (and equal to its ftlm_batch results when the batch runs it on the
 * multi-sector path).
 * ftlm_flow_create -- dtype, block (1, 4, 8, 16), M steps, start-vector dist as for
 *   ftlm_batch_create; max_units: units the flow holds at once.  work_dev
 *   (256-byte aligned, work_bytes, caller-owned) holds 2 max_units block M doubles
 *   of coefficient rows and the units' regions (ftlm_flow_unit_bytes each); the
 *   library allocates the unit descriptors and tile maps from its pool on
 *   `stream`, pinned host staging buffers, the wave streams and the Ritz stream.  Spin-1/2 sectors with N <= 32 and general-spin
 *   sectors.
 * ftlm_flow_add -- queue the R chains of item (as an ftlm_batch_item: chains keyed
 *   first_chain + r under seed; outputs theta, weight, m_eff as for ftlm_lanczos,
 *   written when the sector finishes).  *ticket identifies it.  Admitted at the next
 *   step.  FTLM_ENOMEM when its units do not fit in the free workspace or the
 *   max_units limit right now (nothing is queued: add it again later).
 * ftlm_flow_step -- queue up to `steps` Lanczos steps of every admitted unit on
 *   `stream` (start vectors for the newly admitted ones first).  The units are
 *   visited in waves of consecutive units (admission order) of at most 256 MB of
 *   vectors, each wave running its steps before the next one on its stream starts
 *   (so that a wave's vectors stay in L2 between its steps).  The waves are spread
 *   over the flow's wave streams (least loaded first), which start after the work
 *   queued on `stream` and which `stream` waits for at the end of the call: the
 *   launches of different waves overlap (one wave's gathers with another's row
 *   streams, and launch tails).  The Ritz step of every sector
 *   that finished in the call runs in one launch on the flow's own stream after
 *   the call's work on `stream`, overlapping the next call's steps.  Every flow
 *   call that queues work must use the same stream (or calls ordered by the
 *   caller).
 * ftlm_flow_done -- up to max tickets of sectors whose Ritz step has been queued,
 *   in finishing order; each ticket is returned once.
 * ftlm_flow_set_streams -- wave streams of later step calls, 1 .. 4 (default 4;
 *   1: every wave on `stream`).  Results do not depend on it.  EINVAL otherwise.
 * ftlm_flow_wait_outputs -- makes `stream` wait until the outputs of every sector
 *   finished so far are written (an event wait, no host block).  Call it before
 *   reading the outputs of tickets from ftlm_flow_done on `stream`.
 * ftlm_flow_status -- units and sectors in the flow, free workspace bytes.
 * ftlm_flow_unit_bytes -- workspace bytes of one unit of `block` chains of basis.
 * ftlm_flow_destroy -- waits for the device, then releases. */
typedef struct ftlm_flow ftlm_flow;
ftlm_status ftlm_flow_create(ftlm_dtype dtype, int block, int M, ftlm_vec_dist dist, int max_units, void *work_dev,
                             uint64_t work_bytes, void *stream, ftlm_flow **out);
ftlm_status ftlm_flow_unit_bytes(const ftlm_basis *basis, ftlm_dtype dtype, int block, uint64_t *bytes);
ftlm_status ftlm_flow_add(ftlm_flow *flow, const ftlm_batch_item *item, int *ticket);
ftlm_status ftlm_flow_step(ftlm_flow *flow, int steps, void *stream);
ftlm_status ftlm_flow_done(ftlm_flow *flow, int *tickets, int max, int *n);
ftlm_status ftlm_flow_wait_outputs(ftlm_flow *flow, void *stream);
ftlm_status ftlm_flow_set_streams(ftlm_flow *flow, int n);
ftlm_status ftlm_flow_status(const ftlm_flow *flow, int *units, int *sectors, uint64_t *free_bytes);
void ftlm_flow_destroy(ftlm_flow *flow);

/* ftlm_ritz -- the Ritz step alone (a5): for each of n chains, the eigenvalues theta
 * and first-component weights w = s_{k,1}^2 of the tridiagonal matrix with diagonal
 * alpha_dev[c*M .. c*M+m-1] and off-diagonal beta_dev[c*M .. c*M+m-2], m = m_dev[c]
 * (0 <= m <= M).  Implicit symmetric QR with Wilkinson shifts in FP64, one thread
 * per chain (up to 32 chains per CTA); outputs ascending, zero past m.  EINVAL for
 * n < 0 or M outside 1..FTLM_MAX_LANCZOS. */
ftlm_status ftlm_ritz(int n, int M, const double *alpha_dev, const double *beta_dev,
                      const int *m_dev, double *theta_dev, double *weight_dev, void *stream);

/* Non-convergence of the tridiagonal eigenproblems.  The implicit QR of the Ritz
 * step (ftlm_ritz, ftlm_lanczos*, ftlm_batch_run) and of the T^(1) spectra of
 * ftlm_ghosts stops after a sweep limit (default 64 m sweeps for an m x m matrix;
 * the Wilkinson shift converges in a few sweeps per eigenvalue).  A chain that
 * reaches the limit gets NaN in its theta and weight rows (ftlm_ghosts: NaN ell,
 * no ghost flags), so its NaN propagates into ftlm_thermo's observables, and the
 * device counts it.  Those calls only queue work, so they cannot return the
 * failure themselves:
 * ftlm_ritz_status -- waits for `stream`, then returns the number of problems on
 *   the current device that did not converge since the previous ftlm_ritz_status
 *   (work of other streams counts once it has run) in *unconverged (may be NULL),
 *   clears the count, and returns FTLM_ENOCONV when it is not zero.
 * ftlm_ritz_set_max_sweeps -- process-wide sweep limit per problem for later
 *   launches, 0 restores the default (for tests of this path).  EINVAL for < 0. */
ftlm_status ftlm_ritz_status(void *stream, uint64_t *unconverged);
ftlm_status ftlm_ritz_set_max_sweeps(int sweeps);

/* ------------------------------------------------------------------ thermo ---
 * ftlm_thermo -- FTLM observables on a temperature grid (step a6, Eq. 6-9).
 *   n_sectors computed sectors (1..FTLM_MAX_SECTORS); sector s has 2 S^z =
 *   two_sz[s], dimension dims[s], R chains with Ritz data theta[s], weight[s]
 *   (device double[R*M], from ftlm_lanczos) and m_eff[s] (device int[R]).  Host
 *   arrays of device pointers.
 *   mirror_neg != 0: each sector with S^z > 0 also stands for -S^z (identical
 *   spectra, Sec. 2 Model paragraph).  Zeeman term -h S^z shifts sector energies
 *   by -h S^z.  g: gyromagnetic factor.
 *   Z = sum_sectors (D/R) sum_r sum_k w e^{-beta(E - E0)}, E0 the lowest Ritz
 *   energy (the shift cancels in every ratio); E = <H>, C = beta^2 Var(H),
 *   chi = g^2 beta <(S^z)^2> at h = 0 (Eq. 9), g^2 beta Var(S^z) otherwise;
 *   mag = <S^z>.  k_B = 1.
 *   T_dev: double[nT] > 0; E_dev, C_dev, chi_dev: double[nT]; mag_dev may be NULL.
 */
ftlm_status ftlm_thermo(int n_sectors, const int *two_sz, const uint64_t *dims, int R, int M,
                        const double *const *theta, const double *const *weight,
                        const int *const *m_eff, int mirror_neg, double g, double h, int nT,
                        const double *T_dev, double *E_dev, double *C_dev, double *chi_dev,
                        double *mag_dev, void *stream);

/* ftlm_partition -- the shifted partition function of the FTLM estimate on a T grid
 * (Eq. 7 with every exponent shifted by E0, the lowest Ritz energy of the data):
 *   Z_dev[t] = sum over sectors (and mirror images), chains and Ritz pairs of
 *              (D / R) w_k exp(-(theta_k - h S^z - E0) / T[t]),   E0_dev[t] = E0,
 * i.e. Z_eff = Tr exp(-beta (H - E0)) of Sec. 3.1, for sigma_theo = O / sqrt(Z_eff).
 * Arguments as ftlm_thermo (E0_dev may be NULL). */
ftlm_status ftlm_partition(int n_sectors, const int *two_sz, const uint64_t *dims, int R, int M,
                           const double *const *theta, const double *const *weight, const int *const *m_eff,
                           int mirror_neg, double h, int nT, const double *T_dev, double *Z_dev, double *E0_dev,
                           void *stream);

/* ------------------------------------------------------- FP32 diagnostics ---
 * ftlm_ghosts -- Cullum-Willoughby ghost test (Sec. 3.2, Eq. 25) for n chains.
 *   Inputs per chain c: alpha_dev/beta_dev rows of length M (as for ftlm_ritz),
 *   m_dev[c], and its Ritz values theta_dev (ascending) and weights weight_dev
 *   (the outputs of ftlm_ritz or ftlm_lanczos).
 *   With T^(1) the tridiagonal matrix without its first row and column (eigen-
 *   values theta^(1)_j, FP64 implicit QR), for k < m:
 *     ell_dev[c*M+k]     l_k = min_j |theta_k - theta^(1)_j|   (+inf when m = 1)
 *     flags_dev[c*M+k]   1 when l_k < tau = c_tau * u * (theta_max - theta_min)
 *     cluster_dev[c*M+k] index of the first member of theta_k's cluster: ascending
 *                        Ritz values closer than tau belong to one cluster
 *     cweight_dev[c*M+k] total weight of that cluster
 *   and count_dev[c] = number of ghosts; entries k >= m are 0 (cluster -1).  The
 *   paper takes u = the FP32 unit roundoff for FP32 and FP64 runs alike, c_tau of
 *   order one.  EINVAL for n < 0, M outside 1..FTLM_MAX_LANCZOS, negative c_tau
 *   or u, or NULL pointers. */
ftlm_status ftlm_ghosts(int n, int M, const double *alpha_dev, const double *beta_dev, const int *m_dev,
                        const double *theta_dev, const double *weight_dev, double c_tau, double u, double *ell_dev,
                        int *cluster_dev, double *cweight_dev, int *flags_dev, int *count_dev, void *stream);

/* ftlm_sigma_emp -- Eq. 22 over N_s independent FTLM estimates: obs_dev holds
 * ns rows of nT values (row s = the observable on the T grid from seed s);
 * mean_dev[t] (may be NULL) = the average, sigma_dev[t] = sqrt(sum_s (O_s - mean)^2
 * / ns) with the 1/N_s of Eq. 22.  EINVAL for ns < 1. */
ftlm_status ftlm_sigma_emp(int ns, int nT, const double *obs_dev, double *mean_dev, double *sigma_dev,
                           void *stream);

/* ftlm_launch_count -- kernels the library has queued in this process so far (every
 * launch of every entry point, on any stream; a launch captured into a CUDA graph
 * counts once, at capture, not at each replay). */
ftlm_status ftlm_launch_count(uint64_t *count);

/* ------------------------------------------------------------- diagnostics ---
 * Kernel timing: while enabled, CUDA events are recorded on the launch stream
 * around every H.v launch (ftlm_hv, ftlm_hv_block and the Lanczos H.v step) and
 * every Lanczos vector-update launch.  ftlm_profile_read waits for those events,
 * returns launch counts, the number of vectors the H.v launches applied H to (a
 * block launch counts B), and summed device milliseconds since the last read, and
 * clears them.  Any output pointer may be NULL.  Process-wide; thread-safe. */
ftlm_status ftlm_profile_enable(int on);
ftlm_status ftlm_profile_read(uint64_t *hv_launches, uint64_t *hv_vectors, double *hv_ms,
                              uint64_t *update_launches, double *update_ms);

/* ftlm_probe_read_bandwidth -- read rate of this device for the rooflines of the
 * H.v kernels: reads buf_dev (bytes, 32-byte aligned; its first multiple of 32
 * bytes) `reps` times in one launch, 32 bytes per thread and load, after one
 * untimed pass, and returns GB/s of the timed launch (CUDA events on `stream`;
 * waits for them).  A buffer that fits in L2 (129 MB on GB300) gives the L2 read
 * rate that bounds the gathers of an L2-resident H.v; a buffer of several GB the
 * DRAM read rate.  The buffer's contents are only read.  EINVAL for bad arguments. */
ftlm_status ftlm_probe_read_bandwidth(const void *buf_dev, uint64_t bytes, int reps, void *stream, double *gbps);

/* ftlm_probe_gather_bandwidth -- read rate of this device for the access patterns
 * of the H.v gathers: every 32-byte row of buf_dev (bytes, 32-byte aligned; whole
 * blocks of `run` rows) is read once per pass, `reps` passes in one launch after an
 * untimed pass, in an order scrambled by blocks of `run` consecutive rows -- run = 1:
 * every thread a row of its own (the scattered low-block gathers), run = 32: every
 * warp one contiguous run of 32 rows, 1 KB (the gathers of the transposed walk).
 * Returns GB/s of the timed launch (CUDA events on `stream`; waits for them).  No
 * counterpart in the paper: a measurement tool for the rooflines.  EINVAL for bad
 * arguments (run other than 1 or 32, a buffer smaller than one block). */
ftlm_status ftlm_probe_gather_bandwidth(const void *buf_dev, uint64_t bytes, int run, int reps, void *stream,
                                        double *gbps);

const char *ftlm_status_string(ftlm_status status);
const char *ftlm_last_error(void); /* message of the last failure on this host thread */

#ifdef __cplusplus
}
#endif

#endif /* FTLM_H */
