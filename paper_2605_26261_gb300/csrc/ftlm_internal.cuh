// Internal declarations shared by the libftlm translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "ftlm.h"

namespace ftlm {

// Low digit block of the combinatorial rank: the L lowest label bits (L <= 14).
constexpr int kLoBitsMax = 14;
// Coarse row index: one high-block pattern per 2^kHsShift rows narrows the inverse
// map's search to the few blocks between two consecutive entries.
constexpr int kHsShift = 8;
// Threads per block of the row-parallel kernels.
constexpr int kRowThreads = 256;
// Upper bound on resident blocks per SM the reduction partials are sized for.
constexpr int kMaxBlocksPerSm = 8;

// Bonds are processed in chunks of kBondChunk: a chunk first computes every rank,
// then issues every gather, then accumulates, so each thread keeps kBondChunk
// independent loads in flight.  Ranges are padded to whole chunks with dummy
// bonds (mask 0: never antiparallel, coupling 0).
constexpr int kBondChunk = 8;
constexpr int kMaxBondSlots = FTLM_MAX_BONDS + 2 * kBondChunk;

// Bond list as the kernels see it.  Each slot is one 16-byte entry
// {mlo, mhi, J/2 (float, or the two halves of a double)} in device memory; a block
// stages the list into shared memory once and every lane of a warp then reads the
// same entry (a broadcast), so no per-bond constant-bank load is issued.
//   CR:  [0, n_lo) both sites in the low digit block (mlo = their bits),
//        [n_lo, n_lo + n_hi) both sites in the high block (mhi = their bits >> L),
//        [n_lo + n_hi, nb) any bond (full two-bit mask = mlo | mhi << 32).
//        n_lo and n_hi are whole chunks; bonds left over go to the last range.
//   CLT: [0, nb) in the caller's order, full mask in mlo (N <= 32).
struct BondList {
    int nb;    // slots in use, a multiple of kBondChunk
    int n_lo;
    int n_hi;
    int pad;
    double jsum4;  // sum_b J_b / 4 : the diagonal when every bond is parallel
    const uint4 *slots_f32;  // J/2 as float in .z
    const uint4 *slots_f64;  // J/2 as double in .z (low word), .w (high word)
};

// Scalars of one Lanczos chain, kept on the device between launches.  The stored
// vector u_j is un-normalized: q_j = u_j / s_cur.
struct ChainState {
    double s_cur;      // s_j   (norm of the start vector, then beta_{j-1})
    double s_prev;     // s_{j-1}
    double beta_prev;  // beta_{j-1} (0 at j = 1)
    double alpha;      // alpha_j of the step in flight
    int m_eff;         // steps completed when the chain ended
    int stopped;       // set once beta_j <= tau (or a zero start vector)
    int pad[2];
};

// Block widths: chains run in blocks of B vectors stored interleaved, element
// (t, r) of a block at t * B + r, so one rank computation serves B vectors and a
// gather moves B contiguous values.
constexpr int kMaxBlock = 16;

// Device-side tables of one sector, in the form the kernels take them.
struct SectorTables {
    uint32_t D;          // sector dimension (< 2^32)
    int N, K, L;         // sites, up spins, low-block bits
    uint32_t lomask;     // (1 << L) - 1
    uint32_t H;          // 2^(N - L): high-block patterns
    const uint32_t *thi; // [H]  number of sector labels below h * 2^L
    const uint16_t *tlo; // [2^L] rank of a low pattern among patterns of its popcount
    const uint16_t *ulo; // [2^L] patterns grouped by popcount, ascending (inverse of tlo)
    const uint32_t *uoff; // [kLoBitsMax + 2] start of popcount group c in ulo
    const uint32_t *hs;   // [(D-1) >> kHsShift + 2] high pattern of row min(k << kHsShift, D-1)
    const uint32_t *basis;  // CLT mode: sorted labels [D]
    const uint2 *clt;       // CLT mode: {M_b, C_b} per 32-label block
};

// Split Lanczos H.v (CR, spin 1/2).  Rows t = (h, l) are stored in label order:
// high pattern h major, low pattern l minor.  A bond with both sites in the high
// block maps row (h, l) to (h ^ m, l), a jump of thi[h ^ m] - thi[h] rows that for
// the top sites spans a large part of the sector, so in a walk over the rows in
// label order those gathers miss L2.  The split runs two walks per Lanczos step:
//   walk A  rows near label order (blocks of 32 low ranks x a few high patterns,
//           see LoWalk), bonds with a site in the low block (lo-lo and cross
//           bonds: their jumps stay near the row);
//   walk B  the transposed order -- a warp fixes 32 consecutive low ranks r_lo
//           (one per lane) and steps through the high patterns h of the matching
//           popcount -- with the high-high bonds, whose sources (h ^ m, r_lo) lie
//           in the same 32 columns: every gather is one contiguous run of 32 rows,
//           and the columns' vector data (32 x C(N - L, K - q) rows) stays in L2.
// Walk B adds its terms to walk A's output in place and finishes the Lanczos
// epilogue.  HiWalk describes walk B's tiles: tile (g, c, r) = columns
// 32c .. 32c + 31 of low popcount group g, high patterns rh r .. rh r + rh - 1 of
// group K - q; tiles of a group are numbered column-major (all h of one column
// chunk before the next), so the warps of a launch share one chunk's data.
constexpr int kMaxHiBonds = 64;
constexpr int kMaxHighBits = FTLM_MAX_SITES - kLoBitsMax;
constexpr int kMaxHiGroups = kLoBitsMax + 1;
struct HiWalk {
    int ngroups;                      // low popcount groups with a non-empty high group
    int nbonds;                       // high-high bonds, <= kMaxHiBonds
    int rh;                           // high patterns per tile
    uint32_t ntiles;
    double jsum4;                     // sum of J_b / 4 over the high-high bonds
    uint32_t tile0[kMaxHiGroups + 1]; // first tile of each group (tile0[ngroups] = ntiles)
    uint32_t nl[kMaxHiGroups];        // low ranks (columns) of the group, C(L, q)
    uint32_t nh[kMaxHiGroups];        // high patterns of the group, C(N - L, K - q)
    uint32_t hoff[kMaxHiGroups];      // start of the group's high patterns in uhi
    uint32_t nr[kMaxHiGroups];        // tiles per column chunk, ceil(nh / rh)
    const uint32_t *uhi;              // high patterns grouped by popcount, ascending
    const uint4 *bonds;               // {m >> L, J/2 as float, J/2 as double (lo, hi)}
};

// Walk A of the split in blocks (walka.cu).  A tile is 32 consecutive low ranks
// r_lo (one column per lane) of low popcount group q and a run of up to kLoRun high
// patterns h of popcount K - q (consecutive in uhi).  A lo-lo bond leaves h alone
// and its source (h, l ^ m) sits at thi[h] + tlo[l ^ m]: whether it is antiparallel
// and the rank tlo[l ^ m] depend on the lane's column only, so one lookup serves
// every h of the run.  A cross bond (low site i, high site j) flips one bit of each
// half: source thi[h ^ 2^(j-L)] + tlo[l ^ 2^i], the high term uniform over the
// warp.  Tiles are listed in the order of their runs' first high pattern (all
// popcount classes interleaved, chunks of a run consecutive), i.e. rows near label
// order: the rows of every h of the runs in flight, which the lo-lo gathers read,
// and the neighbouring h ^ 2^(j-L) of the cross bonds stay in L2.  Table entry:
// (position of the run's first h in uhi) << 7 | column chunk.
constexpr int kLoRun = 4;
struct LoWalk {
    uint32_t ntiles;
    int n_ll, n_cr;                   // lo-lo and cross bond slots (each a multiple of 4)
    int nb;                           // n_ll + n_cr
    double jsum4;                     // sum of J_b / 4 over the lo-lo and cross bonds
    uint32_t hend[kMaxHighBits + 2];  // end of popcount class p in uhi
    const uint32_t *tiles;            // [ntiles] (uhi position << 7) | chunk
    const uint32_t *uhi;
    const uint4 *slots_f32;           // lo-lo {m_lo, 0, J/2}, then cross {2^i, 2^(j-L), J/2}
    const uint4 *slots_f64;
};

// General local spin s = two_s / 2 >= 1 (spin.cu): labels n = sum_k a_k d^k with
// base-d digits a_k = m_k + s, d = two_s + 1 (Eq. 11).  The digit-block tables of
// SectorTables are used with base d: thi over the d^(N-L) high labels, tlo/ulo
// over the d^L low labels grouped by digit sum (uoff: start of each group).
struct SpinDev {
    uint32_t d, two_s, A, nb;   // digit base, 2s, sector digit sum (Eq. 17), bonds
    uint64_t magic;             // division by d: q = (n * magic) >> shift, n < 2^29
    uint32_t shift;
    uint32_t n_ll, n_hh;        // bonds [0, n_ll) low-low, [n_ll, n_ll + n_hh) high-high, then cross
    uint32_t pad;
    const uint4 *slots;         // per bond {i | j << 8 | hi_i << 16 | hi_j << 17, d^i', d^j', 0}
                                // (d^k' = power of the site within its digit block)
    const float *jf;            // J_b
    const double *jd;
    const float *upf;           // up[a] = sqrt(s(s+1) - m(m+1)), m = a - s, a = 0 .. 2s-1
    const double *upd;
};

}  // namespace ftlm

struct ftlm_basis {
    int N, K, two_sz;       // K: digit sum of the sector (up spins at s = 1/2)
    int two_s;              // 2s: 1 for spin 1/2, >= 2 for the general-spin path
    int key_n;              // N argument of the chain keys: N, or N | two_s << 8 for s > 1/2
    uint64_t D;
    ftlm_rank_mode mode;
    int L;
    uint64_t H;
    uint64_t nblocks;  // CLT blocks ceil(2^N / 32)
    uint64_t updates;
    uint64_t table_bytes;
    double tau64, tau32;
    int device, num_sms;
    ftlm::BondList bonds_cr;
    ftlm::BondList bonds_clt;
    double jsum4_a;                // split H.v, walk A: sum of J_b / 4 over its lo-lo and cross bonds
    int n_hi_bonds;                // high-high bonds (walk B of the split H.v)
    double jsum4_hi;               // their sum of J_b / 4
    void *block;        // one pooled device allocation holding every table below
    uint4 *bond_slots;  // device: cr f32, cr f64, clt f32, clt f64, walk-A f32, walk-A f64
                        // (LoWalk layout), walk-B bonds (kMaxBondSlots each)
    uint32_t *uhi;      // CR: high patterns grouped by popcount, ascending (walk B)
    uint32_t *lo_tiles; // CR: walk A tile table of the split H.v (LoWalk), or null
    uint32_t n_lo_tiles;
    int n_ll_a, n_cr_a; // walk A bond slots: lo-lo, cross (multiples of 4)
    ftlm_hv_schedule hv_schedule;  // Lanczos H.v walks (ftlm_basis_set_schedule)
    int walk_rh;        // high patterns per walk-B tile (0: the default)
    uint32_t uhi_off[ftlm::kMaxHighBits + 2];  // start of popcount group p in uhi
    uint32_t ulo_off[ftlm::kLoBitsMax + 2];
    uint32_t *thi;
    uint16_t *tlo;
    uint16_t *ulo;
    uint32_t *uoff;
    uint32_t *hs;
    uint64_t n_hs;
    uint32_t *basis;
    uint2 *clt;
    ftlm::SpinDev spin;     // two_s >= 2 only

    ftlm::SectorTables tables() const;
};

namespace ftlm {

// ---- error reporting (api.cu) --------------------------------------------
ftlm_status fail(ftlm_status s, const std::string &msg);
ftlm_status cuda_fail(cudaError_t e, const char *what);
#define FTLM_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return ftlm::cuda_fail(e_, #call); \
    } while (0)

// ---- device memory for tables and descriptors (api.cu) ----------------------
// A stream-ordered pool per device: creating and releasing sector tables and batch
// descriptors then neither synchronizes the device nor returns memory to the
// driver at every release (the pool keeps up to kPoolKeepBytes cached).
constexpr uint64_t kPoolKeepBytes = 4ull << 30;
cudaError_t table_pool(int device, cudaMemPool_t *pool);
// Host-to-device copy of a small host image on `stream` through pinned staging
// (the host buffer may be reused when it returns); images above 256 KB go through
// pageable memory.
cudaError_t upload_async(void *dst, const void *src, size_t bytes, cudaStream_t stream);

// ---- launch count (api.cu): every kernel the library queues calls this once ----
void note_launch();

// ---- per-kernel launch configuration (api.cu) -------------------------------
// Resident CTAs per SM of `kern` at `threads` threads and `smem` bytes of dynamic
// shared memory (at least 1), computed once per (kernel, threads, smem) and cached
// (thread-safe).  With set_smem_attr the kernel's dynamic shared memory limit is
// raised to `smem` first.
cudaError_t kernel_occupancy(const void *kern, int threads, size_t smem, bool set_smem_attr, int *occ);

// ---- kernel timing (api.cu) ----------------------------------------------
enum ProfileKind { kProfHv = 0, kProfUpdate = 1 };
// Returns an opaque token (or nullptr when profiling is off) for a launch about to
// be queued on `stream` that processes `vectors` vectors; profile_end records the
// stop event.
void *profile_begin(int kind, cudaStream_t stream, int vectors = 1);
void profile_end(void *token, cudaStream_t stream);

// ---- launch helpers --------------------------------------------------------
// Blocks for a persistent row-parallel kernel: min(rows / threads, SMs * occupancy).
int row_grid(const ftlm_basis *b, uint64_t rows, int occupancy_blocks_per_sm);
int max_row_grid(const ftlm_basis *b);

// Lanczos epilogue of the H.v launch (hv.cu), for a block of B chains.
struct LanczosHv {
    ChainState *st;        // [B]
    double *partials;      // [grid * B]
    unsigned int *counter; // blocks finished in the current launch (zero between launches)
    double *alpha_out;     // alpha_j of chain r goes to alpha_out[r * alpha_stride]
    int alpha_stride;
    int j;
    double *tile_part;     // [hv_lanczos_tiles() * B]: per-tile sums of a dynamic tile order
};
// General-spin counterparts (spin.cu) of the H.v launch and the label/rank kernels.
ftlm_status launch_hv_spin(const ftlm_basis *b, ftlm_dtype dtype, int B, const void *x, void *y,
                           const LanczosHv *epi, cudaStream_t stream);
ftlm_status launch_spin_labels(const ftlm_basis *b, uint64_t first, uint64_t count, uint64_t *out,
                               cudaStream_t stream);
ftlm_status launch_spin_rank(const ftlm_basis *b, uint64_t count, const uint64_t *labels, int64_t *out,
                             cudaStream_t stream);
// Coarse row index of a basis whose thi table is in place (basis.cu).
void launch_hs_fill(const ftlm_basis *b, cudaStream_t stream);

// y = H x for a block of B interleaved vectors (B in {1, 4, 8, 16}); with epi, the
// Lanczos epilogue (y overwrites the u_{j-1} block in place).
ftlm_status launch_hv(const ftlm_basis *b, ftlm_dtype dtype, int B, const void *x, void *y,
                      const LanczosHv *epi, cudaStream_t stream);
bool valid_block(int B);
// FTLM_RANK_AUTO picks CR for sectors of at least this many rows.
constexpr uint64_t kAutoCrRows = 1ull << 20;
// Upper bound on the tiles of a Lanczos H.v launch of B vectors that takes its tiles
// in dynamic order and leaves alpha_j as per-tile sums in LanczosHv::tile_part (CR
// rank mode, one walk or split); 0 when the launch finishes alpha_j itself.
uint32_t hv_lanczos_tiles(const ftlm_basis *b, int B);

// ---- split Lanczos H.v (basis.cu, walkb.cu, hv.cu) -------------------------
// Walk B's tile layout for rh high patterns per tile (1 <= rh <= 32); false when
// the sector has no split (not CR spin 1/2, no high block, no high-high bond, or
// more than kMaxHiBonds of them).
bool build_hi_walk(const ftlm_basis *b, int rh, HiWalk *w);
struct EpiDev;
// Walk B of a split Lanczos step (the epilogue's alpha as per-tile sums).
ftlm_status launch_walk_b(const ftlm_basis *b, const HiWalk &w, ftlm_dtype dtype, int B, const void *x, void *y,
                          const EpiDev &ep, cudaStream_t stream);
// Walk A's tile layout (false when the sector has no walk A tile table).
bool build_lo_walk(const ftlm_basis *b, LoWalk *w);
// Walk A of a split Lanczos step in blocks (no alpha; walk B finishes the rows).
ftlm_status launch_walk_a(const ftlm_basis *b, const LoWalk &w, ftlm_dtype dtype, int B, const void *x, void *y,
                          const EpiDev &ep, cudaStream_t stream);

// Lanczos chains of one sector (lanczos.cu): chain r is keyed as chain chain0 + r.
ftlm_status lanczos_run(const ftlm_basis *b, int R, int M, int chain0, uint64_t seed, int dist, const double *src,
                        ftlm_dtype dtype, void *work, uint64_t work_bytes, double *theta, double *weight,
                        int *m_eff, double *alpha_dev, double *beta_dev, cudaStream_t stream, int bmax = 0);
// bmax: widest block of chains (0: the process-wide setting).
uint64_t lanczos_workspace(const ftlm_basis *b, int R, int M, ftlm_dtype dtype, int bmax = 0);
// Sweep limit of the tridiagonal QR (ftlm_ritz_set_max_sweeps; 0: 64 n), and the
// per-device counts of problems that did not converge (read and cleared).
int ritz_max_sweeps();
ftlm_status ritz_unconverged_take(cudaStream_t stream, uint64_t *count);
ftlm_status ghost_unconverged_take(cudaStream_t stream, uint64_t *count);
// Sector creation (ftlm_basis_create, ftlm_basis_create_spin); wait: return once
// the tables are built on `stream`, else once their build is queued.
ftlm_status basis_create_half(int N, int two_sz, int n_bonds, const int *bi, const int *bj, const double *J,
                              ftlm_rank_mode mode, cudaStream_t stream, bool wait, ftlm_basis **out);
ftlm_status basis_create_spin(int N, int two_s, int two_sz, int n_bonds, const int *bi, const int *bj,
                              const double *J, cudaStream_t stream, bool wait, ftlm_basis **out);
// Ritz step of n chains (alpha/beta rows of length M, m_eff per chain).
ftlm_status launch_ritz(int n, int M, const double *alpha, const double *beta, const int *mv, double *theta,
                        double *weight, cudaStream_t stream);
// Chain c of an indirect Ritz launch: its coefficient row of alpha/beta/m_eff and
// where its M Ritz values, M weights and chain length go.
struct RitzRow {
    double *theta, *weight;
    int *m_eff;
    uint32_t row, pad;
};
ftlm_status launch_ritz_rows(int n, int M, const double *alpha, const double *beta, const int *mv,
                             const RitzRow *rows, cudaStream_t stream);

}  // namespace ftlm
