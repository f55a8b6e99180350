// jefi_internal.h -- structures shared by the libjefi host code and its kernels.
//
// Device data layout (all owned by one problem handle):
//
//   ring      [cell][Hp][8]  FP32 or FP64, Hp = P + M + 4.  Cells are in brick
//             order: brick b = (bz*nby + by)*nbx + bx covers the 4x4x4 source
//             cells (4bx+i, 4by+j, 4bz+k); cell = b*64 + (k*16 + j*4 + i).
//             Grid extents are padded up to whole bricks with cells whose
//             channels stay zero.  The ring's period P is the history length
//             H rounded up to a multiple of 4: slice n lives in slot n mod P
//             (slots of slices older than the last H are never read); slots
//             [P, P+M) mirror slots [0, M) so that any M consecutive slots are
//             one contiguous TMA box; slots P+M .. P+M+3 are permanently zero
//             (slot P+M stands for sources before slice 0).  M = 0 unless the
//             staged kernel is used, and a multiple of 4.
//             Channels: c*rho, Jx, Jy, Jz, drho/dt, dJx/dt/c, dJy/dt/c, dJz/dt/c.
//             With these, per pair
//               E' += D (ch0/R^3 + ch4/R^2) - ch5..7/R   ->  E = (k_e dV / c) E'
//               B  += (ch1..3/R^3 + ch5..7/R^2) x D      ->  B = k_b dV B
//             which is Eqs. E-1 and B-1 with the constants factored out.
//   obs_xyz   [n_slots][3] FP64 observation points in tile order (256 per
//             tile); padding slots repeat a real point.
//   obs_scr   [6][n_slots] int32 per-axis source-index ranges [lo, hi] of
//             the screening box of each observation point (FP64 decision).
//   tab32     [n_t][K] float4 {hi, lo, phys_slot (int bits), 0} per candidate
//             slot k = k0 + i: S32 in (lo, hi] proves slot k exactly.
//   theta     [n_t][theta_stride(K)]: K+1 FP64 exact thresholds (slot(S) >=
//             k0+i iff S <= theta[i]), then the same thresholds as FP32 pairs
//             (hi, lo), hi + lo = theta[i] to 2^-48 relative, bit-copied into
//             the next K+1 doubles (the double-float check of undecided pairs).
//   partials  [n_t][n_split][6][n_slots] FP64 per-split sums.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace jefi {

constexpr int kTileThreads = 256;   // observation points per tile (one per thread)
constexpr int kBrick = 4;           // source brick edge (cells)
constexpr int kBrickCells = 64;
constexpr int kZeroPadSlots = 4;    // the zero line after the P + M ring slots

#ifdef __CUDACC__
#define JEFI_HD __host__ __device__
#else
#define JEFI_HD
#endif

// Doubles per evaluation time in a threshold table (see SumParams::theta).
JEFI_HD constexpr size_t theta_stride(int K) { return 2 * (size_t)(K + 1); }

// Staged FP32 kernel: compiled band heights (slots per staged cell), the
// cells per stage of each, and whether its rows are copied with the 32-byte
// swizzle (bands of 32 slots and more, whose rows spread over many
// shared-memory banks).  Swizzled stage buffers start on a 256-byte boundary
// (the swizzle's period); the dynamic shared memory gets kStagedAlignPad
// extra bytes for that.
constexpr int kStagedBands[6] = {16, 24, 32, 48, 64, 96};
constexpr int kStagedMaxBand = 96;
constexpr int kStagedAlignPad = 256;
JEFI_HD constexpr bool staged_swizzled(int band) { return band >= 32; }
JEFI_HD constexpr int staged_stage_cells(int band) { return band <= 24 ? 64 : (band <= 48 ? 32 : 16); }
constexpr int kTileBoxFloats = 12;  // per tile: box lo xyz, hi xyz, O xyz, rho_lo, rho_hi, 0
constexpr int kStagedCtrlBytes = 128 + 2 * 256;   // control block after the stage buffers (with 256 stage bands)

struct TimeParams {
    float A;            // fp32(T/dt - k0): candidate index ~ floor(A - R/(c dt))
    float Ag;           // A + g, g >= |error of the FP32 candidate|: floor(Ag - R K) in {n-k0, n-k0+1}
    int32_t oldest_rel; // oldest resident slot - k0 (clamped to int32)
    float A_lo;         // fp32(T/dt - k0 - A): A + A_lo carries T/dt - k0 to ~2^-48 (interpolation weights)
    int64_t k0;         // table origin slot
    double A64;         // T/dt - k0 in FP64 (interpolation weight of the FP64 kernel)
    int32_t k0_mod;     // k0 mod P (the ring's period), in [0, P): physical rows without 64-bit division
    int32_t pad;
};

constexpr int kTabGuard = 32;       // guard entries on each side of the staged kernel's table

struct SumParams {
    // source geometry
    int32_t nbx, nby, nbz, n_bricks;
    int32_t npx, npy, npz;          // padded grid extents (4 * nb)
    double lo[3], d[3];             // source lattice, FP64
    int32_t org[3];                 // first cell of the source grid in its lattice: cell i of
                                    // axis a is centred at lo[a] + (org[a] + i + 0.5) d[a]
    float d32[3];
    // observation tiles
    int32_t n_slots;                // padded observation count
    int32_t n_tiles;
    const double* obs_xyz;
    const int32_t* obs_scr;
    // history ring
    const void* ring;
    int32_t Hp;                     // slots per cell including the mirror and the zero line
    int32_t zero_slot;              // == P + M
    // per-time tables
    const float4* tab32;
    const double* theta;
    const TimeParams* times;
    int32_t n_t;
    int32_t K;                      // candidate slots per time
    float K32;                      // fp32(1 / (c dt))
    // work split
    int32_t n_split;
    int32_t bricks_per_split;
    int32_t split_merge;            // staged kernel: consecutive splits one work item sums (>= 1);
                                    // each split's partials are written as if it were an item of its own
    // outputs
    double* partials;
    unsigned long long* fallbacks;  // pairs whose slot was recomputed in FP64
    int32_t* debug_slots;           // NULL, or [n_slots][n_cells] logical slot per pair
    int32_t* status;                // device error word (0 = ok, else a jefi_status)
    // staged kernel only
    const float2* tab2;             // [n_t][K + 2 kTabGuard] {T_hi, T_lo} per candidate slot
    const float* tile_box;          // [n_tiles][kTileBoxFloats]: min xyz, max xyz of (x_o - anchor) and
                                    // O - anchor (O the source grid's centre), fp32; the range
                                    // [rho_lo, rho_hi] of |x_o - O| over the tile, fp32 outward
                                    // (rho_lo < 0: the kernel uses the box alone)
    int32_t n_src_axis[3];          // real source cells per axis
    int32_t nfull[3];               // whole bricks per axis (bricks past them hold padding cells)
    int32_t H;                      // ring period P (physical slot of slice n is n mod P)
    int32_t comp;                   // FP32: compensated (Kahan) per-thread sums
    // direct-gather kernel, per candidate slot k' (the staged kernel's candidate
    // rule, slots read from global memory): [n_t][K + 2 kTabGuard] {T_lo, physical
    // slots of k' (low 16 bits) and k'-1 (high 16 bits)}, and T_hi in tabh
    const float2* tabg;
    const float* tabh;
    int32_t exact;                  // lattice geometry: T_hi == T_lo, no pair undecided
    // second-order retarded time: sources interpolated between slots n and n+1
    int32_t interp;
    float K32_lo;                   // fp32(1/(c dt) - K32)
    // Double-float check of undecided pairs (FP32 kernels): per slot the
    // point's coordinates as FP32 pairs (x hi, x lo, y hi, y lo, z hi, z lo),
    // per padded cell of each axis its centre as an FP32 pair (x cells, then
    // y, then z), and the bound B = df_b1 R + df_b2 S on |S_df - S64|.
    const float* obs_hl;
    const float2* cc_hl;
    float df_b1, df_b2;
    int32_t pad_yz;                 // the grid ends inside its last bricks along y or z
    double K64;                     // 1 / (c dt)
};

// Persistent batched launches: problem i owns items [item_start[i], item_start[i+1]),
// item = (time, split, tile) in that order of significance.
struct BatchArgs {
    const SumParams* params;        // [n] device
    const int32_t* item_start;      // [n+1] device
    int32_t n;
    int32_t n_items;
    unsigned int* counter;          // device, zero at launch
};

struct PushParams {
    int32_t nx, ny, nz;
    int32_t nbx, nby;
    int64_t n_src;
    // the slice arrays cover a larger grid of fnx x fny x ... cells; this
    // handle's cell (i, j, k) is their cell (ox + i, oy + j, oz + k)
    int32_t fnx, fny;
    int32_t ox, oy, oz;
    int32_t Hp;
    int32_t slot;                   // physical slot to write
    int32_t supplied;
    int32_t fp64;
    int32_t mirror_slot;            // also write the slice here (the ring's mirror copy), or -1
    double c, inv_c, dt;
    const double* rho;
    const double* J;
    const double* drho;
    const double* dJ;
    double* prev;                   // [n_src][4] previous slice (backward differences)
    void* ring;
    // central differences: also rewrite the derivative channels of slice n-1
    // as (f[n] - f[n-2]) / (2 dt)
    int32_t central;
    int32_t prev_slot;              // physical slot of slice n-1, or -1 (n = 0)
    int32_t prev_mirror_slot;       // its mirror copy, or -1
    double* prev2;                  // [n_src][4] slice n-2
};

struct ReduceParams {
    int32_t n_obs, n_slots, n_split, n_t;
    const int32_t* inv_perm;        // [n_obs] observation index -> tile slot
    const double* partials;
    double e_scale, b_scale;
    double* E;                      // [n_t][n_obs][3]
    double* B;
};

constexpr int kMaxBatchMaps = 224;  // tensor maps per staged batched launch (kernel-parameter space)

#ifdef CUDA_VERSION
struct StagedBatchArgs {
    const SumParams* params;
    const int32_t* item_start;
    int32_t n;
    int32_t n_items;
    unsigned int* counter;
    CUtensorMap maps[kMaxBatchMaps];
};
cudaError_t launch_sum_f32_staged_batch(const StagedBatchArgs& a, int band, bool exact, size_t smem,
                                        int grid, cudaStream_t s);
#endif

struct ReduceItem {
    const int32_t* inv_perm;
    const double* partials;         // this item's [n_split][6][n_slots]
    int32_t n_obs, n_slots, n_split, pad;
    double e_scale, b_scale;
    double* E;
    double* B;
};

cudaError_t launch_sum_f32_batch(const BatchArgs& a, bool compensated, size_t smem, int grid, cudaStream_t s);
cudaError_t launch_sum_f64_batch(const BatchArgs& a, size_t smem, int grid, cudaStream_t s);
cudaError_t launch_reduce_batch(const ReduceItem* items, const int64_t* out_start, int n, int64_t total,
                                cudaStream_t s);

struct StagedConfig {
    int32_t band;                   // slot rows staged per cell (a compiled variant)
    bool exact;                     // FP32 squared distances are exact (lattice geometry)
    bool compensated;
    const void* tensor_map;         // CUtensorMap over the FP32 ring
};

// Rank-ordered FP64 sum of the fields of several S-O pairs over the same points.
constexpr int kMaxSumParts = 64;
struct SumPartsParams {
    int32_t n_parts;
    int64_t n;                      // doubles per field array (3 per point)
    const double* E_parts[kMaxSumParts];
    const double* B_parts[kMaxSumParts];
    double* E;
    double* B;
};
cudaError_t launch_sum_parts(const SumPartsParams& p, cudaStream_t s);

cudaError_t launch_push(const PushParams& p, cudaStream_t s);
cudaError_t launch_wait_timeout_probe(int32_t* status, uint64_t limit_ns, cudaStream_t s);
cudaError_t launch_sum_f32_staged(const SumParams& p, const StagedConfig& c, cudaStream_t s);
size_t staged_smem_bytes(const SumParams& p, int band, bool batched);
size_t staged_buffer_bytes(int band);   // one stage buffer: cells per stage x band x 32 bytes
bool staged_band_supported(int band);
#ifdef CUDA_VERSION
#define JEFI_DECLARE_STAGED_BAND(BAND)                                                                  \
    cudaError_t staged_launch_##BAND(const SumParams& p, const StagedConfig& c, cudaStream_t s);          \
    cudaError_t staged_launch_batch_##BAND(const StagedBatchArgs& a, bool exact, size_t smem, int grid,  \
                                           cudaStream_t s);
JEFI_DECLARE_STAGED_BAND(16)
JEFI_DECLARE_STAGED_BAND(24)
JEFI_DECLARE_STAGED_BAND(32)
JEFI_DECLARE_STAGED_BAND(48)
JEFI_DECLARE_STAGED_BAND(64)
JEFI_DECLARE_STAGED_BAND(96)
#undef JEFI_DECLARE_STAGED_BAND
#endif
cudaError_t launch_sum_f32(const SumParams& p, bool compensated, cudaStream_t s);
cudaError_t launch_sum_f64(const SumParams& p, cudaStream_t s);
cudaError_t launch_reduce(const ReduceParams& p, cudaStream_t s);
size_t sum_smem_bytes(const SumParams& p);

}  // namespace jefi
