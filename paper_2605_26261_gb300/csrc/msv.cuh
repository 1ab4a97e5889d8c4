// Descriptors of the multi-sector Lanczos path (msv.cu), planned by ftlm_batch.
#pragma once

#include "ftlm_internal.cuh"

namespace ftlm {

// Default rows per H.v tile (a multiple of kRowThreads); a plan may choose others
// (ftlm_batch_create_plan, ftlm_batch_autotune_plan).
constexpr uint32_t kMsTileRows = 2048;
// Default rows per tile of the streaming kernels (start vectors, update): eight H.v
// tiles.  The update's work per row is a few loads, so larger tiles amortize the
// per-tile reduction (measured on the 256-cluster step: update 3.7 / 2.0 / 1.5 / 1.1
// s per step at 1024 / 2048 / 4096 / 8192 rows with one FP64 tree per chain; with
// the transposed trees 1.35 / 1.18 / 1.67 s at 8192 / 16384 / 32768 rows; H.v best
// at 2048).
constexpr uint32_t kMsStreamRows = 8 * kMsTileRows;

// One block of B chains of one sector.  Offsets are into the run's workspace.
struct MsUnit {
    SectorTables s;
    BondList bl;
    uint64_t off_v0, off_v1;  // the two vector blocks, D x B each
    uint64_t off_st;          // ChainState[kMaxBlock], then the unit's reduction counter
    uint64_t off_part;        // per-tile partial sums [n_tiles][B]
    uint64_t seed;
    double tau;
    uint32_t tile0, n_tiles;  // the unit's H.v tiles within its wave
    uint32_t stile0, n_stiles;  // the unit's tiles of the streaming kernels
    uint32_t tile_rows;       // rows per H.v tile (a multiple of kRowThreads)
    uint32_t stream_rows;     // rows per tile of the streaming kernels
    uint32_t chain_base;      // chain 0 of the unit in the batch's alpha/beta/meff arrays
    int key_n, K, chain0;     // chain keys: chain r is keyed (seed, key_n, K, chain0 + r)
    int nact;                 // chains of the unit (<= B); the other columns stay zero
    int m_max;
    int j0;                   // step launches of the unit run as Lanczos step j - j0 (0 in a batch; a
                              // continuous flow starts units at later launches)
    SpinDev spin;             // general-spin units (kMsSpin)
};

// Rank kinds of a wave (one kernel instantiation each).
enum MsKind { kMsCr = 0, kMsClt = 1, kMsSpin = 2 };

// Units run together (one rank kind), their tiles numbered 0 .. n_tiles-1.
struct MsWave {
    uint32_t unit0, n_units;  // units [unit0, unit0 + n_units) of the plan
    uint32_t tile_off;        // offset of the wave's tile->unit map in the plan's map
    uint32_t n_tiles;
    uint32_t stile_off;       // the same for the tiles of the streaming kernels
    uint32_t n_stiles;
    int m_max;                // longest chain length of the wave
    int kind;                 // MsKind
};

// Queue one wave: start vectors, m_max steps of (H.v + alpha, update + beta), and
// the chain lengths into meff.  units and tile_unit point at the wave's own entries.
ftlm_status ms_run_wave(const MsWave &w, ftlm_dtype dtype, int B, const MsUnit *units, const uint32_t *tile_unit,
                        const uint32_t *stile_unit, int M, int dist, char *ws, double *alpha, double *beta,
                        int *meff, int num_sms, cudaStream_t stream);

// Vector bytes per wave of the multi-sector path (FTLM_MS_WAVE_MB, default 256 MB;
// batch.cu), used by batches and by the continuous flow.
uint64_t ms_wave_bytes();

// Single launches of a continuous flow (flow.cu): reset + start vectors of the
// units with j0 == jstart; the H.v + alpha launch of one rank kind (its units and
// tile map); the update + beta launch over every unit of the flow.  j is the flow's
// launch counter; a unit runs Lanczos step j - j0 and skips launches outside
// 1 .. m_max.
ftlm_status ms_flow_start(ftlm_dtype dtype, int B, const MsUnit *units, uint32_t n_units, const uint32_t *stile_unit,
                          uint32_t n_stiles, int jstart, int dist, char *ws, int num_sms, cudaStream_t stream);
ftlm_status ms_flow_hv(ftlm_dtype dtype, int B, int kind, const MsUnit *units, const uint32_t *tile_unit,
                       uint32_t n_tiles, int j, int M, double *alpha, char *ws, int num_sms, cudaStream_t stream);
ftlm_status ms_flow_update(ftlm_dtype dtype, int B, const MsUnit *units, const uint32_t *stile_unit, uint32_t n_stiles,
                           int j, int M, double *beta, char *ws, int num_sms, cudaStream_t stream);

}  // namespace ftlm
