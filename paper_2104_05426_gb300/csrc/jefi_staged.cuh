// jefi_staged.cuh -- FP32 retarded direct sum (Eqs. E-1, B-1, tr-1) with the
// history band of every source stage staged in shared memory by TMA.
// Templates shared by the translation units that instantiate the compiled
// band heights (jefi_staged.cu: 16, 24; jefi_staged_b32_48.cu; jefi_staged_b64_96.cu).
//
// One CTA = one tile of 256 observation points x a contiguous range of source
// bricks.  A brick (4x4x4 cells) is processed in stages of kCells cells (the
// whole brick for narrow bands; 32 or 16 cells, i.e. two z slabs or one, for
// wide bands so that two stage buffers of two CTAs fit one SM).  For each
// stage one thread computes the band of slots [lo, lo + BAND) that any pair
// of the tile and the stage's cells can retard into, and one
// cp.async.bulk.tensor copies the stage's cells x BAND slots x 8 channels of
// the ring into a shared-memory buffer (two buffers: the next stage's copy
// overlaps the current stage's arithmetic; completion through an mbarrier,
// waits bounded in time).
//
// Shared-memory layout of a stage buffer: [cell][slot][8 channels] FP32,
// 32 bytes per (cell, slot) row.  Bands of 32 rows and more are copied with
// the tensor map's 32-byte swizzle: in every other group of four rows the
// two 16-byte halves of each row trade places (address bit 4 XOR bit 7), so
// the first halves of any eight consecutive rows fall on eight different
// groups of banks.  The lanes of a quarter-warp read one cell at nearby
// slots; in the dense layout rows four apart share banks.
//
// Slot selection per pair, exact with respect to the FP64 rule of Eq. tr-1:
//   k' = floor(A + g - R32/(c dt)), g bounding the FP32 error of the
//   candidate, so that k' is n or n+1; one threshold entry (T_hi, T_lo) of
//   Theta_k' (largest S64 whose slot is >= k') decides: S32 > T_lo -> n = k'-1,
//   S32 <= T_hi -> n = k'.  On exact-lattice geometry S32 == S64 and
//   T_hi == T_lo == Theta_k' rounded down, so every pair is decided without a
//   branch.  Otherwise the rare pairs between T_hi and T_lo contribute nothing
//   in the unrolled loop and are redone after the stage with their slot
//   recomputed in FP64.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "jefi_device.cuh"
#include "jefi_internal.h"

namespace jefi {
namespace staged {
using namespace dev;

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // a bounded wait gives up after 2 s
constexpr int kStatusTimeout = 6;                    // JEFI_ETIMEOUT
constexpr int kStatusInternal = 7;                   // JEFI_EINTERNAL
constexpr int kBandSkip = -32768;                    // a stage whose band did not fit: skipped (fits int16)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity; false if it has not completed
// after limit_ns.
static __device__ __noinline__ bool mbar_wait_bounded(uint32_t a, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1; it != 0; ++it) {
        if (mbar_try_wait(a, parity)) return true;
        if ((it & 63u) == 0 && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// ~0u if a > b, else 0 (false for NaN operands)
__device__ __forceinline__ uint32_t gt_mask(float a, float b) {
    uint32_t r;
    asm("set.gt.u32.f32 %0, %1, %2;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
        : "memory");
}

// Byte offset of a dense [cell][slot][8] offset inside a 256-byte aligned
// buffer written with the 32-byte swizzle: bit 4 XOR bit 7.
__device__ __forceinline__ uint32_t swz32(uint32_t off) { return off ^ ((off >> 3) & 0x10u); }

template <int BAND>
struct Layout {
    static constexpr bool kSwz = staged_swizzled(BAND);
    static constexpr int kCells = staged_stage_cells(BAND);   // cells per stage
    static constexpr int kParts = kBrickCells / kCells;         // stages per brick
    static constexpr int kSlabs = kCells / 16;                  // 4x4-cell z slabs per stage
    static constexpr uint32_t kRowBytes = 32;                   // 8 FP32 channels
    static constexpr uint32_t kCellBytes = BAND * kRowBytes;
    static constexpr uint32_t kBufBytes = kCells * kCellBytes;
    static constexpr uint32_t kCtrl = 2 * kBufBytes;            // mbarriers, band origins, item
    static constexpr uint32_t kTileBox = kCtrl + 64;            // the item's tile box (kTileBoxFloats)
    static constexpr uint32_t kBands = kCtrl + 128;             // bands of 256 upcoming stages (int16)
    static constexpr uint32_t kTab = kCtrl + kStagedCtrlBytes;  // float2 table
    // control words of the non-lattice fall-back (one item): offset of the
    // FP64 geometry (the tile's points, then the cell centres of x, y, z),
    // the cell counts of x and y, and the pairs redone
    static constexpr uint32_t kGeo = kCtrl + 48;
    static_assert(kBufBytes % kStagedAlignPad == 0, "stage buffers keep the alignment of the swizzle");
};

// The staged region of dynamic shared memory.  Swizzled bands start it at
// the first 256-byte boundary (the 32-byte swizzle pattern follows address
// bits 4 and 7 and repeats every 256 bytes; the launch adds kStagedAlignPad
// bytes for it); dense bands use the
// array itself (a TMA destination needs 128 bytes), so their offsets stay
// compile-time relative to it.
template <int BAND>
__device__ __forceinline__ unsigned char* staged_base() {
    extern __shared__ __align__(1024) unsigned char smem[];
    if constexpr (staged_swizzled(BAND)) {
        const uint32_t pad = (0u - smem_u32(smem)) & (kStagedAlignPad - 1);
        return smem + pad;
    } else {
        return smem;
    }
}

// Shared-memory offset of the FP64 geometry of one item: after the float2
// table, the FP64 thresholds and the float brick offsets.
__host__ __device__ __forceinline__ uint32_t staged_geometry_offset(uint32_t tab, int K, int nb_sum) {
    const uint32_t d = tab + (uint32_t)(K + 2 * kTabGuard) * 8u + (uint32_t)(K + 1) * 8u;
    return (d + (uint32_t)nb_sum * 4u + 7u) & ~7u;
}

// Exact slot of one undecided pair from the FP64 geometry in shared memory
// (written by the item's preamble).  A call of its own, so
// the FP64 search does not weigh on the registers of the stage loop.
template <int BAND>
__device__ __noinline__ int staged_slot_fp64(int ix, int iy, int iz, const double* s_th, int K, int guess) {
    using L = Layout<BAND>;
    unsigned char* sb = staged_base<BAND>();
    const uint32_t* g = reinterpret_cast<const uint32_t*>(sb + L::kGeo);
    const double* s_xo = reinterpret_cast<const double*>(sb + g[0]) + 3 * threadIdx.x;
    const double* s_cc = reinterpret_cast<const double*>(sb + g[0]) + 3 * kTileThreads;
    return slot_fp64_stored(s_xo, s_cc[ix], s_cc[g[1] + iy], s_cc[g[1] + g[2] + iz], s_th, K, guess);
}

// Both staged kernels initialise the two mbarriers once per CTA.
template <int BAND>
__device__ __forceinline__ void staged_init_barriers() {
    using L = Layout<BAND>;
    if (threadIdx.x == 0) {
        uint64_t* s_mbar = reinterpret_cast<uint64_t*>(staged_base<BAND>() + L::kCtrl);
        mbar_init(smem_u32(&s_mbar[0]), 1);
        mbar_init(smem_u32(&s_mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// Non-lattice geometry of one item (before the item's first barrier): the
// tile's FP64 points and the FP64 cell centres of each axis, for the exact
// slot of the pairs the FP32 rule leaves undecided; zeroes the item's count.
template <int BAND>
__device__ __noinline__ void staged_fill_geometry(const double* txyz, int K, int nb_sum, int npx, int npy, int npz,
                                                  double lox, double loy, double loz, double dx_, double dy_,
                                                  double dz_, const int32_t* org) {
    using L = Layout<BAND>;
    unsigned char* sb = staged_base<BAND>();
    const int tid = threadIdx.x;
    const uint32_t geo = staged_geometry_offset(L::kTab, K, nb_sum);
    double* s_xo = reinterpret_cast<double*>(sb + geo);
    double* s_cc = s_xo + 3 * kTileThreads;
    for (int i = tid; i < npx; i += kTileThreads) s_cc[i] = cell_center(lox, dx_, org[0] + i);
    for (int i = tid; i < npy; i += kTileThreads) s_cc[npx + i] = cell_center(loy, dy_, org[1] + i);
    for (int i = tid; i < npz; i += kTileThreads) s_cc[npx + npy + i] = cell_center(loz, dz_, org[2] + i);
    for (int a = 0; a < 3; ++a) s_xo[3 * tid + a] = txyz[3 * tid + a];
    if (tid == 0) {
        uint32_t* g = reinterpret_cast<uint32_t*>(sb + L::kGeo);
        g[0] = geo;
        g[1] = (uint32_t)npx;
        g[2] = (uint32_t)npy;
        g[3] = 0u;
    }
}

// Both 16-byte halves of the row at dense offset `off` of a stage buffer.
template <int BAND>
__device__ __forceinline__ void load_row(const unsigned char* bufp, uint32_t off, float4& v0, float4& v1) {
    if constexpr (Layout<BAND>::kSwz) {
        const uint32_t a = swz32(off);
        v0 = *reinterpret_cast<const float4*>(bufp + a);
        v1 = *reinterpret_cast<const float4*>(bufp + (a ^ 16u));
    } else {
        v0 = *reinterpret_cast<const float4*>(bufp + off);
        v1 = *reinterpret_cast<const float4*>(bufp + off + 16u);
    }
}

struct FixSums {
    float v[6];   // E', B contributions
};

// Pairs of a full stage whose slot the FP32 rule left undecided (non-lattice
// geometry): the exact slot by the double-float check (slot_double_float),
// else by the FP64 rule, then the pair from the stage's buffer.  A call of
// its own (rare), so its registers do not weigh on the stage loop, with few
// arguments: everything the item does not vary comes from the parameters'
// copy in shared memory (`sp`), so that the stage loop keeps no extra values
// alive for the call.  `mask` holds brick cell indices; the stage's cells
// start at cell0; buf_off is the stage buffer's offset in the staged region.
// GEO: the FP64 geometry of the pair in shared memory and the count there
// (the single-problem kernel); otherwise the point from global memory, the
// centre computed, and the count the caller's.
template <int BAND, bool DEBUG, bool INTERP, bool GEO>
__device__ __noinline__ FixSums staged_fixup(uint64_t mask, uint32_t buf_off, int cell0, int band_rel, float Px,
                                             float Py, float Pz, int bx, int by, int bz, int b, int slot, int ti,
                                             const SumParams* sp) {
    using L = Layout<BAND>;
    unsigned char* const sb = staged_base<BAND>();
    const unsigned char* bufp = sb + buf_off;
    const int K = sp->K;
    const double* s_th = reinterpret_cast<const double*>(sb + L::kTab + (size_t)(K + 2 * kTabGuard) * sizeof(float2));
    const TimeParams tp = sp->times[ti];
    const float K32 = sp->K32, K32_lo = sp->K32_lo;
    const float d32x = sp->d32[0], d32y = sp->d32[1], d32z = sp->d32[2];
    const float* xo_hl = sp->obs_hl + (size_t)6 * slot;
    const float2* cc_hl = sp->cc_hl;
    const float2* th_hl = reinterpret_cast<const float2*>(sp->theta + (size_t)ti * theta_stride(K) + (K + 1));
    const int npx = sp->npx, npy = sp->npy;
    const size_t n_cells = (size_t)sp->n_bricks * kBrickCells;
    // every undecided pair counts, whichever check decides it
    if (GEO) atomicAdd(reinterpret_cast<uint32_t*>(sb + L::kGeo) + 3, (uint32_t)__popcll(mask));
    float pe[3] = {0.f, 0.f, 0.f}, pb[3] = {0.f, 0.f, 0.f};
    while (mask) {
        const int cl = __ffsll((long long)mask) - 1;
        mask &= mask - 1;
        const int i = cl & 3, j = (cl >> 2) & 3, k = cl >> 4;
        const float dx = fmaf(-(float)i, d32x, Px);
        const float dy = fmaf(-(float)j, d32y, Py);
        const float dz = fmaf(-(float)k, d32z, Pz);
        const float S = __fadd_rn(__fmul_rn(dx, dx), __fadd_rn(__fmul_rn(dy, dy), __fmul_rn(dz, dz)));
        const float ri = rsqrt_ftz(S);
        const uint32_t bits = __float_as_uint(__fadd_rd(fmaf(-(S * ri), K32, tp.Ag), kMagic));
        const int guess = (int)(bits - kMagicBits);
        const int ix = kBrick * bx + i, iy = kBrick * by + j, iz = kBrick * bz + k;
        int idx = slot_double_float(xo_hl, cc_hl[ix], cc_hl[npx + iy], cc_hl[npx + npy + iz], th_hl, K, guess,
                                    S * ri, sp->df_b1, sp->df_b2);
        if (idx < 0) {
            if constexpr (GEO) {
                idx = staged_slot_fp64<BAND>(ix, iy, iz, s_th, K, guess);
            } else {
                idx = slot_fallback_f32(sp->obs_xyz, slot, sp->lo[0], sp->lo[1], sp->lo[2], sp->d[0], sp->d[1],
                                        sp->d[2], sp->org[0] + ix, sp->org[1] + iy, sp->org[2] + iz, s_th, K, guess,
                                        nullptr);
            }
        }
        int row = idx - band_rel;
        if (row < 0 || row >= BAND) {
            atomicExch(sp->status, kStatusInternal);
            row = row < 0 ? 0 : BAND - 1;
        }
        if (DEBUG) sp->debug_slots[(size_t)slot * n_cells + (size_t)b * kBrickCells + cl] = (int)(tp.k0 + idx);
        const uint32_t off = (uint32_t)(cl - cell0) * L::kCellBytes + (uint32_t)row * L::kRowBytes;
        float4 v0, v1;
        load_row<BAND>(bufp, off, v0, v1);
        if (INTERP) {
            float4 u0, u1;
            load_row<BAND>(bufp, off + L::kRowBytes, u0, u1);
            lerp8(v0, v1, u0, u1, interp_weight(S, ri, (float)idx, tp.A, tp.A_lo, K32, K32_lo));
        }
        pair_f32(dx, dy, dz, ri, v0, v1, pe, pb);
    }
    return FixSums{{pe[0], pe[1], pe[2], pb[0], pb[1], pb[2]}};
}

// Capacity of a thread's queue of undecided pairs (non-lattice geometry).
constexpr int kFixQueue = 16;

// Pairs whose slot the FP32 rule left undecided (non-lattice geometry): the
// exact slot by the double-float check (slot_double_float), else by the FP64
// rule, then the pair from the ring in global memory.  The stage loop queues
// a thread's undecided pairs (`fq`, nf entries of (brick << 6) | cell) and
// the warp redoes them together once per split, or when a queue would
// overflow (then with the current stage's `mask`, cells of brick mb): one
// pass of this call for many stages, with many lanes busy, where a call per
// stage had one lane busy and held the other warps at the stage barrier.
// A call of its own (rare), so its registers do not weigh on the stage loop;
// what the item does not vary it reads from the parameters (`sp`).  The
// FP64 geometry of the item is in shared memory and the pairs are counted
// there.  (oox, ooy, ooz): the point's offset from the tile's anchor.
template <int BAND, bool DEBUG, bool INTERP>
__device__ __noinline__ FixSums staged_fix_deferred(const uint32_t* fq, int nf, uint64_t mask, int mb, float oox,
                                                    float ooy, float ooz, int slot, int ti, const SumParams* sp) {
    using L = Layout<BAND>;
    unsigned char* const sb = staged_base<BAND>();
    const int K = sp->K;
    const double* s_th = reinterpret_cast<const double*>(sb + L::kTab + (size_t)(K + 2 * kTabGuard) * sizeof(float2));
    const float* s_D = reinterpret_cast<const float*>(s_th + K + 1);
    const TimeParams tp = sp->times[ti];
    const float K32 = sp->K32, K32_lo = sp->K32_lo;
    const float d32x = sp->d32[0], d32y = sp->d32[1], d32z = sp->d32[2];
    const float* xo_hl = sp->obs_hl + (size_t)6 * slot;
    const float2* cc_hl = sp->cc_hl;
    const float2* th_hl = reinterpret_cast<const float2*>(sp->theta + (size_t)ti * theta_stride(K) + (K + 1));
    const int npx = sp->npx, npy = sp->npy, nbx = sp->nbx, nby = sp->nby;
    const int Hp = sp->Hp, P = sp->H, zero_slot = sp->zero_slot;
    const float4* ring = reinterpret_cast<const float4*>(sp->ring);
    const size_t n_cells = (size_t)sp->n_bricks * kBrickCells;
    // every undecided pair counts, whichever check decides it
    atomicAdd(reinterpret_cast<uint32_t*>(sb + L::kGeo) + 3, (uint32_t)(nf + __popcll(mask)));
    // physical ring row of slot k0 + n (the zero line for slots before slice 0)
    auto phys = [&](int n) -> int {
        if (tp.k0 + n < 0) return zero_slot;
        int r = tp.k0_mod + n;
        while (r >= P) r -= P;
        while (r < 0) r += P;
        return r;
    };
    float pe[3] = {0.f, 0.f, 0.f}, pb[3] = {0.f, 0.f, 0.f};
    for (int e = 0;; ++e) {
        int b, cl;
        if (e < nf) {
            const uint32_t q = fq[e];
            b = (int)(q >> 6);
            cl = (int)(q & 63u);
        } else if (mask) {
            b = mb;
            cl = __ffsll((long long)mask) - 1;
            mask &= mask - 1;
        } else {
            break;
        }
        const int bx = b % nbx, r_ = b / nbx, by = r_ % nby, bz = r_ / nby;
        const int i = cl & 3, j = (cl >> 2) & 3, k = cl >> 4;
        // the stage loop's operations, so the same S and candidate
        const float Px = oox + s_D[bx];
        const float Py = ooy + s_D[nbx + by];
        const float Pz = ooz + s_D[nbx + nby + bz];
        const float dx = fmaf(-(float)i, d32x, Px);
        const float dy = fmaf(-(float)j, d32y, Py);
        const float dz = fmaf(-(float)k, d32z, Pz);
        const float S = __fadd_rn(__fmul_rn(dx, dx), __fadd_rn(__fmul_rn(dy, dy), __fmul_rn(dz, dz)));
        const float ri = rsqrt_ftz(S);
        const uint32_t bits = __float_as_uint(__fadd_rd(fmaf(-(S * ri), K32, tp.Ag), kMagic));
        const int guess = (int)(bits - kMagicBits);
        const int ix = kBrick * bx + i, iy = kBrick * by + j, iz = kBrick * bz + k;
        int idx = slot_double_float(xo_hl, cc_hl[ix], cc_hl[npx + iy], cc_hl[npx + npy + iz], th_hl, K, guess,
                                    S * ri, sp->df_b1, sp->df_b2);
        if (idx < 0) idx = staged_slot_fp64<BAND>(ix, iy, iz, s_th, K, guess);
        if (DEBUG) sp->debug_slots[(size_t)slot * n_cells + (size_t)b * kBrickCells + cl] = (int)(tp.k0 + idx);
        const size_t cell = (size_t)b * kBrickCells + cl;
        int ps = phys(idx);
        if (cell >= n_cells || ps < 0 || ps >= Hp) {   // never, for a consistent handle
            atomicExch(sp->status, kStatusInternal);
            continue;
        }
        const float4* q = ring + (cell * Hp + ps) * 2;
        float4 v0 = __ldg(q), v1 = __ldg(q + 1);
        if (INTERP) {   // slot n+1
            ps = phys(idx + 1);
            if (ps < 0 || ps >= Hp) {
                atomicExch(sp->status, kStatusInternal);
                continue;
            }
            const float4* u = ring + (cell * Hp + ps) * 2;
            lerp8(v0, v1, __ldg(u), __ldg(u + 1), interp_weight(S, ri, (float)idx, tp.A, tp.A_lo, K32, K32_lo));
        }
        pair_f32(dx, dy, dz, ri, v0, v1, pe, pb);
    }
    return FixSums{{pe[0], pe[1], pe[2], pb[0], pb[1], pb[2]}};
}

// One work item: observation tile `tile` x source splits [group split_merge,
// (group + 1) split_merge) at time index `ti` of problem p.  g_it counts the CTA's stages across items (it
// selects the buffer and the mbarrier phase).  Returns false if a copy did
// not complete in time (the caller stops).  PAD: the source grid ends inside
// its last bricks along y or z; their padding rows and slabs are skipped
// (zero channels: no sum changes).  GEO: undecided pairs take their
// FP64 geometry from shared memory and are counted there (the single-problem
// kernel); otherwise from global memory (the batched kernel).
template <int BAND, bool EXACT, bool DEBUG, bool INTERP, bool GEO, bool PAD>
__device__ __forceinline__ bool staged_item(const CUtensorMap* tmap_ptr, const SumParams& p, const SumParams* sp,
                                            const int comp, const int tile, const int group, const int ti,
                                            uint32_t& g_it) {
    using L = Layout<BAND>;
    unsigned char* const sb = staged_base<BAND>();
    const int K = p.K;
    const int KT = K + 2 * kTabGuard;
    uint64_t* s_mbar = reinterpret_cast<uint64_t*>(sb + L::kCtrl);
    int* s_band = reinterpret_cast<int*>(sb + L::kCtrl + 16);
    float2* s_tab = reinterpret_cast<float2*>(sb + L::kTab);
    double* s_th = reinterpret_cast<double*>(sb + L::kTab + (size_t)KT * sizeof(float2));
    float* s_D = reinterpret_cast<float*>(s_th + K + 1);
    float* s_tb = reinterpret_cast<float*>(sb + L::kTileBox);

    const int tid = threadIdx.x;
    if (tid < kTileBoxFloats) s_tb[tid] = p.tile_box[(size_t)tile * kTileBoxFloats + tid];

    const float2* g_tab = p.tab2 + (size_t)ti * KT;
    for (int i = tid; i < KT; i += kTileThreads) s_tab[i] = g_tab[i];
    const double* g_th = p.theta + (size_t)ti * theta_stride(K);
    for (int i = tid; i <= K; i += kTileThreads) s_th[i] = g_th[i];
    const double* txyz = p.obs_xyz + (size_t)tile * kTileThreads * 3;
    if constexpr (!EXACT && GEO)
        staged_fill_geometry<BAND>(txyz, K, p.nbx + p.nby + p.nbz, p.npx, p.npy, p.npz, p.lo[0], p.lo[1], p.lo[2],
                                   p.d[0], p.d[1], p.d[2], p.org);
    const double cox = txyz[0], coy = txyz[1], coz = txyz[2];
    const int nbxy = p.nbx + p.nby;
    for (int i = tid; i < nbxy + p.nbz; i += kTileThreads) {
        const int a = i < p.nbx ? 0 : (i < nbxy ? 1 : 2);
        const int b = a == 0 ? i : (a == 1 ? i - p.nbx : i - nbxy);
        const double co = a == 0 ? cox : (a == 1 ? coy : coz);
        s_D[i] = __double2float_rn(__dsub_rn(co, cell_center(p.lo[a], p.d[a], p.org[a] + kBrick * b)));
    }
    __syncthreads();

    ThreadCtx ctx;
    ctx.slot = tile * kTileThreads + tid;
    const double xo = txyz[3 * tid + 0], yo = txyz[3 * tid + 1], zo = txyz[3 * tid + 2];
    const float oox = __double2float_rn(__dsub_rn(xo, cox));
    const float ooy = __double2float_rn(__dsub_rn(yo, coy));
    const float ooz = __double2float_rn(__dsub_rn(zo, coz));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ctx.rlo[a] = p.obs_scr[(2 * a) * p.n_slots + ctx.slot];
        ctx.rhi[a] = p.obs_scr[(2 * a + 1) * p.n_slots + ctx.slot];
    }
    const TimeParams tp = p.times[ti];
    const float K32 = p.K32;
    const float Ag = tp.Ag;
    const float A = tp.A, A_lo = tp.A_lo, K32_lo = p.K32_lo;   // interpolation weights only
    const float d32x = p.d32[0], d32y = p.d32[1], d32z = p.d32[2];
    const size_t n_cells = (size_t)p.n_bricks * kBrickCells;
    const uint32_t mbar_u32[2] = {smem_u32(&s_mbar[0]), smem_u32(&s_mbar[1])};
    const uint32_t buf_u32[2] = {smem_u32(sb), smem_u32(sb + L::kBufBytes)};

    float se[3] = {0.f, 0.f, 0.f}, sbv[3] = {0.f, 0.f, 0.f};
    float ce[3] = {0.f, 0.f, 0.f}, cbv[3] = {0.f, 0.f, 0.f};
    // pairs whose slot was recomputed in FP64 through global memory, counted
    // per thread and added once per warp (not one atomic per pair)
    uint32_t n_fb = 0;
    // undecided pairs (non-lattice geometry) of the current split, queued
    // until the split ends: (brick << 6) | cell
    static_assert(EXACT || GEO, "non-lattice items keep their FP64 geometry in shared memory");
    uint32_t fq[(EXACT || BAND > 24) ? 1 : kFixQueue];
    int nf = 0;
    // The item covers splits [split_lo, split_hi) (p.split_merge per item);
    // each split's bricks are summed and its partials written as an item of
    // its own would: the result does not depend on how many splits an item
    // merges, while the preamble and the pipeline's first copy are paid once.
    const int split_lo = group * p.split_merge;
    const int split_hi = min(split_lo + p.split_merge, p.n_split);
    const int b_begin = split_lo * p.bricks_per_split;
    const int b_end = min(split_hi * p.bricks_per_split, p.n_bricks);
    auto write_split = [&](int sp) {
        double* out = p.partials + ((size_t)ti * p.n_split + sp) * 6 * p.n_slots + ctx.slot;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            out[(size_t)a * p.n_slots] = comp ? (double)se[a] - (double)ce[a] : (double)se[a];
            out[(size_t)(3 + a) * p.n_slots] = comp ? (double)sbv[a] - (double)cbv[a] : (double)sbv[a];
        }
    };
    const uint32_t n_stages = b_end > b_begin ? (uint32_t)(b_end - b_begin) * L::kParts : 0u;
    const uint32_t tbase = L::kTab + (uint32_t)(kTabGuard - kMagicBits) * 8u;

    // Slot band of (this tile, item stage g): bounds every pair distance two
    // ways and keeps the tighter: the boxes of the tile and of the stage's
    // cells, and the shell [rho_lo, rho_hi] of the tile's distances from the
    // point O (the source grid's centre) widened by the stage's farthest
    // distance from O.  kBandSkip (and the status word set) for a band that
    // does not fit the buffer (never, if the creation-time bound holds): its
    // stage is skipped, so no pair reads past the buffer.
    auto stage_band = [&](uint32_t g) -> int {
        const int b = b_begin + (int)(g / L::kParts);
        const int q = (int)(g % L::kParts);
        const int bx_ = b % p.nbx, r_ = b / p.nbx, by_ = r_ % p.nby, bz_ = r_ / p.nby;
        const float* tb = s_tb;
        const float cb[3] = {-s_D[bx_], -s_D[p.nbx + by_], -s_D[nbxy + bz_]};
        const float dd[3] = {d32x, d32y, d32z};
        const float c_lo[3] = {0.f, 0.f, (float)(q * L::kSlabs)};
        const float c_hi[3] = {3.f, 3.f, (float)(q * L::kSlabs + L::kSlabs - 1)};
        float mn2 = 0.f, mx2 = 0.f, span = 0.f, od2 = 0.f, ospan = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // source cells of the stage span [s_lo, s_hi] (anchor-relative);
            // pair offsets D = x_o - x_s span [box_lo - s_hi, box_hi - s_lo]
            const float s_lo = fmaf(c_lo[a], dd[a], cb[a]);
            const float s_hi = fmaf(c_hi[a], dd[a], cb[a]);
            const float lo = tb[a] - s_hi;
            const float hi = tb[3 + a] - s_lo;
            const float mn = lo > 0.f ? lo : (hi < 0.f ? -hi : 0.f);
            const float mx = fmaxf(fabsf(lo), fabsf(hi));
            mn2 = fmaf(mn, mn, mn2);
            mx2 = fmaf(mx, mx, mx2);
            span += fabsf(cb[a]) + fabsf(tb[a]) + fabsf(tb[3 + a]) + 3.f * dd[a];
            const float od = fmaxf(fabsf(s_lo - tb[6 + a]), fabsf(s_hi - tb[6 + a]));
            od2 = fmaf(od, od, od2);
            ospan += fabsf(tb[6 + a]) + fabsf(s_lo) + fabsf(s_hi);
        }
        const float slack = 1e-5f * span;
        float rmin = fmaxf(sqrtf(mn2) * (1.f - 1e-5f) - slack, 0.f);
        float rmax = sqrtf(mx2) * (1.f + 1e-5f) + slack;
        if (tb[9] >= 0.f) {   // tiles whose shell can be tighter than their box (the host decides)
            const float odist = sqrtf(od2) * (1.f + 1e-5f) + 1e-5f * ospan;
            const float oslack = 1e-5f * (tb[10] + odist);
            rmin = fmaxf(rmin, tb[9] - odist - oslack);
            rmax = fminf(rmax, tb[10] + odist + oslack);
        }
        const int hi_rel = (int)floorf(tp.A - rmin * K32) + 2;
        const int lo_rel = (int)floorf(tp.A - rmax * K32) - 2;
        const int band_rel = max(lo_rel, tp.oldest_rel);
        if (hi_rel - band_rel + 1 > BAND) {
            atomicExch(p.status, kStatusInternal);
            return kBandSkip;
        }
        return band_rel;
    };
    // The bands of 256 stages at a time, one per thread: the copy issue on
    // one thread then only reads its stage's band (the other warps do not
    // wait at the stage barrier for that thread's arithmetic).
    int16_t* s_bands = reinterpret_cast<int16_t*>(sb + L::kBands);   // bands relative to k0 fit 16 bits
    auto fill_bands = [&](uint32_t g0) {
        const uint32_t g = g0 + (uint32_t)tid;
        if (g < n_stages) s_bands[tid] = (int16_t)stage_band(g);
    };
    // Producer (thread 0): TMA copy of item stage g into buffer bufi.
    auto issue = [&](uint32_t g, int bufi) {
        const int band_rel = s_bands[g & (kTileThreads - 1)];
        s_band[bufi] = band_rel;
        const int b = b_begin + (int)(g / L::kParts);
        const int q = (int)(g % L::kParts);
        int y0 = 0;   // a skipped stage still copies (rows 0..) to keep the phases in step
        if (band_rel != kBandSkip) {
            const long long band_abs = tp.k0 + band_rel;
            if (band_abs >= 0) {
                // (k0 mod P + band_rel) mod P, band_rel being small: no 64-bit division
                y0 = tp.k0_mod + band_rel;
                while (y0 >= p.H) y0 -= p.H;
                while (y0 < 0) y0 += p.H;
            } else {
                y0 = band_abs < -(1ll << 30) ? -(1 << 30) : (int)band_abs;   // rows < 0 read as zero
            }
        }
        // the buffer was last read through the generic proxy: order those
        // reads before the async-proxy write
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(mbar_u32[bufi], L::kBufBytes);
        tma_load_3d(buf_u32[bufi], tmap_ptr, 0, y0, b * kBrickCells + q * L::kCells, mbar_u32[bufi]);
    };

    if (n_stages > 0) {
        fill_bands(0);
        __syncthreads();
        if (tid == 0) issue(0, g_it & 1);
    }
    int64_t aborted_at = -1;
    // brick coordinates of b, advanced incrementally (no division per brick)
    int bx = 0, by = 0, bz = 0;
    if (b_begin < b_end) {
        bx = b_begin % p.nbx;
        const int rest = b_begin / p.nbx;
        by = rest % p.nby;
        bz = rest / p.nby;
    }
    for (int b = b_begin; b < b_end && aborted_at < 0; ++b) {
        const bool near = (ctx.rlo[0] <= kBrick * bx + 3) & (ctx.rhi[0] >= kBrick * bx) &
                          (ctx.rlo[1] <= kBrick * by + 3) & (ctx.rhi[1] >= kBrick * by) &
                          (ctx.rlo[2] <= kBrick * bz + 3) & (ctx.rhi[2] >= kBrick * bz);
        // Bricks with a screened pair take the checked path.  Padding cells
        // (past the grid's last cell) take the fast one: their channels are
        // zero in every slot, their distances are unscreened and bounded away
        // from zero like every padded pair (creation checks it), and their
        // slots fall in the stage's band (computed from the padded box).
        const bool fast = !__any_sync(kFull, near);
        const float Px = oox + s_D[bx];
        const float Py = ooy + s_D[p.nbx + by];
        const float Pz = ooz + s_D[nbxy + bz];
        // the brick's sum over its stages (compensated once per brick)
        float pe[3] = {0.f, 0.f, 0.f}, pb[3] = {0.f, 0.f, 0.f};
        // brick b ends its split (whose partials are written after it)
        const bool split_last = (b + 1) % p.bricks_per_split == 0 || b + 1 == b_end;
        // One stage: q-th group of kCells cells of brick b.  False if its copy
        // did not complete in time (the item then stops).
        auto stage = [&](const int q) -> bool {
            const uint32_t g = (uint32_t)(b - b_begin) * L::kParts + (uint32_t)q;   // stage of the item
            const uint32_t it = g_it + g;
            const int buf = it & 1;
            // the next stage's copy goes into the other buffer, whose last
            // readers passed the barrier at the end of the previous stage
            if (tid == 0 && g + 1 < n_stages) issue(g + 1, buf ^ 1);
            const bool ready = mbar_wait_bounded(mbar_u32[buf], (it >> 1) & 1);
            const int band_rel = s_band[buf];
            if (ready && band_rel != kBandSkip) {
                const int cell0 = q * L::kCells;
                const unsigned char* bufp = sb + (uint32_t)buf * L::kBufBytes;
                uint64_t mask = 0;   // undecided pairs of the stage (non-lattice geometry)
                if (fast) {
                    // Per-axis offsets and squares of the brick's 4 columns; the
                    // z slabs are a rolled loop (keeps the hot body small), the
                    // 16 cells of a slab are unrolled.
                    float ddx[4], ddy[4], sqx[4], sqy[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        ddx[i] = fmaf(-(float)i, d32x, Px);
                        ddy[i] = fmaf(-(float)i, d32y, Py);
                        sqx[i] = __fmul_rn(ddx[i], ddx[i]);
                        sqy[i] = __fmul_rn(ddy[i], ddy[i]);
                    }
                    // offset of row n (relative to k0) of the stage's first cell,
                    // (n - band_rel) * 32 with n carried in the magic bits: from
                    // the buffer's start for swizzled rows (the swizzle acts on
                    // it), from the shared array's for dense rows (one 32-bit
                    // address per pair, the buffer folded in here)
                    const unsigned char* const rows = L::kSwz ? bufp : sb;
                    const uint32_t gbase = (L::kSwz ? 0u : (uint32_t)buf * L::kBufBytes) -
                                           (uint32_t)(kMagicBits + band_rel) * L::kRowBytes;
                    // operands of the candidates of two cells at once (packed FP32
                    // with the scalar roundings: the same bits as one cell at a time)
                    const float2 nK2 = make_float2(-K32, -K32), Ag2 = make_float2(Ag, Ag);
                    const float2 magic2 = make_float2(kMagic, kMagic);
                    // E' = sum D q - sum (dJ/c) r^-1 and B = sum V x D: the
                    // products with D in scalars (no operand pair to build per
                    // pair), the dJ-terms of y and z packed and subtracted per
                    // stage (no negated pair per pair)
                    // (the floor-rule lattice kernel keeps two sets, for even and
                    // odd cells: shorter dependency chains, measured 0.5 % faster
                    // there, 1.7 % slower on the non-lattice kernels and 4 % on
                    // the interpolating one)
                    constexpr int kAcc = (EXACT && !INTERP) ? 2 : 1;
                    float acc_ex2[kAcc], acc_ey2[kAcc], acc_ez2[kAcc], acc_bz2[kAcc];
                    float2 acc_jyz2[kAcc], acc_bxy2[kAcc];
#pragma unroll
                    for (int a = 0; a < kAcc; ++a) {
                        acc_ex2[a] = acc_ey2[a] = acc_ez2[a] = acc_bz2[a] = 0.f;
                        acc_jyz2[a] = acc_bxy2[a] = make_float2(0.f, 0.f);
                    }
                    // slabs and rows past the grid's last cell (PAD) hold only
                    // padding: skipped
                    const int k_end =
                        PAD ? min(max(p.n_src_axis[2] - kBrick * bz - q * L::kSlabs, 0), L::kSlabs) : L::kSlabs;
                    const int j_end = PAD ? p.n_src_axis[1] - kBrick * by : 4;
#pragma unroll 1
                    for (int kk = 0; kk < k_end; ++kk) {
                        const int k = q * L::kSlabs + kk;
                        const float dz = fmaf(-(float)k, d32z, Pz);
                        const float sqz = __fmul_rn(dz, dz);
                        const uint32_t gk = gbase + (uint32_t)(kk * 16) * L::kCellBytes;
                        uint32_t m16 = 0;           // undecided cells of this slab (non-lattice geometry)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            if (PAD && j >= j_end) break;
                            const float syz = __fadd_rn(sqy[j], sqz);
                            const float2 syz2 = make_float2(syz, syz);
                            float2 S2, R2, B2;   // S, r^-1 and candidate bits of cells i, i+1
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int c16 = j * 4 + i;
                                float S, ri;
                                uint32_t bits;
                                if constexpr (EXACT || BAND <= 24) {
                                    // two cells' candidates at once (the lattice kernels and
                                    // the narrow bands: measured faster there; the wide
                                    // non-lattice kernels spill with it),
                                    // S*r^-1*(-K) + A + g rounded as fmaf(-(S*ri), K, Ag)
                                    if ((i & 1) == 0) {
                                        S2 = __fadd2_rn(make_float2(sqx[i], sqx[i + 1]), syz2);
                                        R2 = make_float2(rsqrt_ftz(S2.x), rsqrt_ftz(S2.y));
                                        B2 = __fadd2_rd(__ffma2_rn(__fmul2_rn(S2, R2), nK2, Ag2), magic2);
                                    }
                                    S = (i & 1) ? S2.y : S2.x;
                                    ri = (i & 1) ? R2.y : R2.x;
                                    bits = __float_as_uint((i & 1) ? B2.y : B2.x);
                                } else {
                                    // one cell at a time
                                    S = __fadd_rn(sqx[i], syz);
                                    ri = rsqrt_ftz(S);
                                    bits = __float_as_uint(__fadd_rd(fmaf(-(S * ri), K32, Ag), kMagic));
                                }
                                // row of candidate k' (bits), moved down one row when S is
                                // past the threshold: lower = 0 or ~0u
                                uint32_t lower;
                                if (EXACT) {
                                    // T_hi == T_lo: one 32-bit threshold decides
                                    const float th = *reinterpret_cast<const float*>(sb + (tbase + 4u + bits * 8u));
                                    lower = gt_mask(S, th);
                                } else {
                                    const float2 th = *reinterpret_cast<const float2*>(sb + (tbase + bits * 8u));
                                    lower = gt_mask(S, th.y);
                                    if (!(S <= th.x) && lower == 0u) {   // undecided: redo after the stage
                                        m16 |= 1u << c16;   // c16 is a constant of the unrolled body
                                        ri = 0.f;
                                    }
                                }
                                if (DEBUG) {
                                    p.debug_slots[(size_t)ctx.slot * n_cells + (size_t)b * kBrickCells + k * 16 +
                                                  c16] = (int)(tp.k0 + (int)(bits + lower - kMagicBits));
                                }
                                const uint32_t row_hi = gk + bits * L::kRowBytes;
                                // (a select of the row, not a multiply by the mask: 0.6 %
                                // faster on the lattice kernel, 2 % on the dipole's; the
                                // interpolating kernels keep the product, which spills
                                // less there)
                                const uint32_t row = INTERP ? row_hi + lower * L::kRowBytes
                                                            : (lower ? row_hi - L::kRowBytes : row_hi);
                                const uint32_t off = row + (uint32_t)c16 * L::kCellBytes;
                                float4 v0, v1;
                                load_row<BAND>(rows, off, v0, v1);
                                if (INTERP) {   // slot n+1 is the next row of the same cell
                                    float4 u0, u1;
                                    load_row<BAND>(rows, off + L::kRowBytes, u0, u1);
                                    const float nrel = __uint_as_float(bits + lower) - kMagic;
                                    lerp8(v0, v1, u0, u1, interp_weight(S, ri, nrel, A, A_lo, K32, K32_lo));
                                }
                                // Eqs. E-1/B-1 with packed pairs, r^-2 factored out:
                                //   (q, Vx) = ((drho, dJx/c) + (c rho, Jx) r^-1) r^-2,  q the D-term of E
                                //   (Vy, Vz) = ((dJy, dJz)/c + (Jy, Jz) r^-1) r^-2
                                const float2 ri2 = make_float2(ri, ri);
                                const float2 r2 = __fmul2_rn(ri2, ri2);
                                const float2 qvx = __fmul2_rn(__ffma2_rn(make_float2(v0.x, v0.y), ri2,
                                                                         make_float2(v1.x, v1.y)), r2);
                                const float2 vyz = __fmul2_rn(__ffma2_rn(make_float2(v0.z, v0.w), ri2,
                                                                         make_float2(v1.z, v1.w)), r2);
                                const float qq = qvx.x, vx = qvx.y;
                                const int ia = kAcc == 2 ? (i & 1) : 0;
                                float& acc_ex = acc_ex2[ia];
                                float& acc_ey = acc_ey2[ia];
                                float& acc_ez = acc_ez2[ia];
                                float& acc_bz = acc_bz2[ia];
                                float2& acc_jyz = acc_jyz2[ia];
                                float2& acc_bxy = acc_bxy2[ia];
                                // E' += D q - (dJ/c) r^-1
                                acc_ex = fmaf(ddx[i], qq, acc_ex);
                                acc_ex = fmaf(-v1.y, ri, acc_ex);
                                acc_ey = fmaf(ddy[j], qq, acc_ey);
                                acc_ez = fmaf(dz, qq, acc_ez);
                                acc_jyz = __ffma2_rn(make_float2(v1.z, v1.w), ri2, acc_jyz);
                                // B += V x D
                                acc_bxy.x = fmaf(vyz.x, dz, acc_bxy.x);              // Vy dz
                                acc_bxy.y = fmaf(vyz.y, ddx[i], acc_bxy.y);          // Vz dx
                                acc_bxy.x = fmaf(-vyz.y, ddy[j], acc_bxy.x);         // - Vz dy
                                acc_bxy.y = fmaf(-vx, dz, acc_bxy.y);                // - Vx dz
                                acc_bz = fmaf(vx, ddy[j], acc_bz);
                                acc_bz = fmaf(-vyz.x, ddx[i], acc_bz);
                            }
                        }
                        if (!EXACT) mask |= (uint64_t)m16 << (k * 16);
                    }
                    if constexpr (kAcc == 2) {
                        pe[0] += acc_ex2[0] + acc_ex2[1];
                        pe[1] += (acc_ey2[0] + acc_ey2[1]) - (acc_jyz2[0].x + acc_jyz2[1].x);
                        pe[2] += (acc_ez2[0] + acc_ez2[1]) - (acc_jyz2[0].y + acc_jyz2[1].y);
                        pb[0] += acc_bxy2[0].x + acc_bxy2[1].x;
                        pb[1] += acc_bxy2[0].y + acc_bxy2[1].y;
                        pb[2] += acc_bz2[0] + acc_bz2[1];
                    } else {
                        pe[0] += acc_ex2[0];
                        pe[1] += acc_ey2[0] - acc_jyz2[0].x;
                        pe[2] += acc_ez2[0] - acc_jyz2[0].y;
                        pb[0] += acc_bxy2[0].x;
                        pb[1] += acc_bxy2[0].y;
                        pb[2] += acc_bz2[0];
                    }
                } else {
                    // Bricks with screened pairs: rolled loop with per-pair checks
                    // and clamped indices.
                    for (int cl = cell0; cl < cell0 + L::kCells; ++cl) {
                        const int i = cl & 3, j = (cl >> 2) & 3, k = cl >> 4;
                        const int ix = kBrick * bx + i, iy = kBrick * by + j, iz = kBrick * bz + k;
                        const bool real = (ix < p.n_src_axis[0]) & (iy < p.n_src_axis[1]) & (iz < p.n_src_axis[2]);
                        const bool scr = (ix >= ctx.rlo[0]) & (ix <= ctx.rhi[0]) & (iy >= ctx.rlo[1]) &
                                         (iy <= ctx.rhi[1]) & (iz >= ctx.rlo[2]) & (iz <= ctx.rhi[2]);
                        const bool use = real & !scr;
                        const float dx = fmaf(-(float)i, d32x, Px);
                        const float dy = fmaf(-(float)j, d32y, Py);
                        const float dz = fmaf(-(float)k, d32z, Pz);
                        const float S = __fadd_rn(__fmul_rn(dx, dx),
                                                  __fadd_rn(__fmul_rn(dy, dy), __fmul_rn(dz, dz)));
                        float ri = rsqrt_ftz(S);
                        const uint32_t bits = __float_as_uint(__fadd_rd(fmaf(-(S * ri), K32, Ag), kMagic));
                        const uint32_t tix = min(bits - (uint32_t)kMagicBits + (uint32_t)kTabGuard, (uint32_t)(KT - 1));
                        const float2 th = s_tab[tix];
                        const bool lower = S > th.y;
                        int idx = (int)tix - kTabGuard - (lower ? 1 : 0);
                        if (use && !(S <= th.x) && !lower) {
                            if constexpr (EXACT || !GEO) {
                                idx = slot_fallback_f32(p.obs_xyz, ctx.slot, p.lo[0], p.lo[1], p.lo[2], p.d[0],
                                                        p.d[1], p.d[2], p.org[0] + ix, p.org[1] + iy, p.org[2] + iz,
                                                        s_th, K, idx, nullptr);
                                if constexpr (!EXACT) ++n_fb;
                            } else {
                                atomicAdd(reinterpret_cast<uint32_t*>(sb + L::kGeo) + 3, 1u);
                                idx = staged_slot_fp64<BAND>(ix, iy, iz, s_th, K, idx);
                            }
                        }
                        int row = idx - band_rel;
                        if (!use) {
                            ri = 0.f;
                            row = 0;
                        } else if (row < 0 || row >= BAND - (INTERP ? 1 : 0)) {
                            atomicExch(p.status, kStatusInternal);
                            row = row < 0 ? 0 : BAND - 1 - (INTERP ? 1 : 0);
                        }
                        if (DEBUG) {
                            p.debug_slots[(size_t)ctx.slot * n_cells + (size_t)b * kBrickCells + cl] =
                                scr ? INT32_MIN : (int)(tp.k0 + idx);
                        }
                        const uint32_t off = (uint32_t)(cl - cell0) * L::kCellBytes + (uint32_t)row * L::kRowBytes;
                        float4 v0, v1;
                        load_row<BAND>(bufp, off, v0, v1);
                        if (INTERP) {   // row + 1 < BAND: the band covers slot n+1 of every pair
                            float4 u0, u1;
                            load_row<BAND>(bufp, off + L::kRowBytes, u0, u1);
                            lerp8(v0, v1, u0, u1, interp_weight(S, ri, (float)idx, A, A_lo, K32, K32_lo));
                        }
                        pair_f32(dx, dy, dz, ri, v0, v1, pe, pb);
                    }
                }
                if constexpr (!EXACT && BAND > 24) {
                    // wide bands: the stage's undecided pairs now, from the
                    // stage buffer (a queue made their batched item spill)
                    if (__any_sync(kFull, mask != 0ull)) {
                        const FixSums f = staged_fixup<BAND, DEBUG, INTERP, GEO>(
                            mask, (uint32_t)buf * L::kBufBytes, cell0, band_rel, Px, Py, Pz, bx, by, bz, b,
                            ctx.slot, ti, sp);
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            pe[a] += f.v[a];
                            pb[a] += f.v[3 + a];
                        }
                    }
                } else if constexpr (!EXACT) {
                    // Undecided pairs join the thread's queue.  The warp redoes
                    // the queued pairs (and this stage's) when a queue would
                    // overflow and at the split's last stage, so that they join
                    // their own split's sums; one call site keeps the stage
                    // loop's registers as they were.
                    const bool last = split_last && q == L::kParts - 1;
                    if (__any_sync(kFull, nf + __popcll(mask) > kFixQueue || (last && (nf > 0 || mask != 0ull)))) {
                        const FixSums f = staged_fix_deferred<BAND, DEBUG, INTERP>(fq, nf, mask, b, oox, ooy, ooz,
                                                                                   ctx.slot, ti, sp);
                        nf = 0;
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            pe[a] += f.v[a];
                            pb[a] += f.v[3 + a];
                        }
                    } else {
                        while (mask) {
                            const int cl = __ffsll((long long)mask) - 1;
                            mask &= mask - 1;
                            fq[nf++] = ((uint32_t)b << 6) | (uint32_t)cl;
                        }
                    }
                }
            }
            // the next 256 bands, before the stage that issues the first of them
            if (((g + 2) & (kTileThreads - 1)) == 0 && g + 2 < n_stages) fill_bands(g + 2);
            // every thread is done with this buffer (and s_bands is complete)
            // before the next copy is issued
            if (__syncthreads_or(!ready)) {
                aborted_at = (int64_t)g;
                return false;
            }
            return true;
        };
        if constexpr (L::kParts == 1) {
            stage(0);                      // whole-brick stages: q is the constant 0
        } else {
#pragma unroll 1
            for (int q = 0; q < L::kParts; ++q)
                if (!stage(q)) break;
        }
        if (aborted_at < 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (comp) {
                    kahan_add(se[a], ce[a], pe[a]);
                    kahan_add(sbv[a], cbv[a], pb[a]);
                } else {
                    se[a] += pe[a];
                    sbv[a] += pb[a];
                }
            }
        }
        if (++bx == p.nbx) {
            bx = 0;
            if (++by == p.nby) { by = 0; ++bz; }
        }
        if (split_last) {
            // the split of brick b is complete (its queued pairs were redone
            // in its last stage): its partial sums
            write_split(b / p.bricks_per_split);
#pragma unroll
            for (int a = 0; a < 3; ++a) se[a] = sbv[a] = ce[a] = cbv[a] = 0.f;
        }
    }
    if (aborted_at >= 0) {
        // a copy did not complete in time: report, then wait (bounded) for
        // the copies still in flight (this stage's, and the next one's if it
        // was issued) before the shared memory goes away
        if (tid == 0) {
            const uint32_t it = g_it + (uint32_t)aborted_at;
            atomicExch(p.status, kStatusTimeout);
            mbar_wait_bounded(mbar_u32[it & 1], (it >> 1) & 1);
            if ((uint32_t)aborted_at + 1 < n_stages) mbar_wait_bounded(mbar_u32[(it + 1) & 1], ((it + 1) >> 1) & 1);
        }
        __syncthreads();
    }
    g_it += n_stages;
    if constexpr (!EXACT) {   // exact lattices decide every pair in FP32
        const uint32_t w = __reduce_add_sync(kFull, n_fb);
        if ((tid & 31) == 0 && w) atomicAdd(p.fallbacks, (unsigned long long)w);
    }
    if constexpr (!EXACT && GEO) {
        // every thread passed the loop's last barrier: the item's count is complete
        const uint32_t n = reinterpret_cast<const uint32_t*>(sb + L::kGeo)[3];
        if (tid == 0 && n) atomicAdd(p.fallbacks, (unsigned long long)n);
    }

    // a split without bricks still gets its (zero) partials; after a copy
    // timed out the status word reports the item as failed
    for (int sp = split_lo; sp < split_hi; ++sp)
        if (sp * p.bricks_per_split >= b_end) write_split(sp);
    return aborted_at < 0;
}

template <int BAND, bool EXACT, bool DEBUG, bool INTERP, bool PAD>
__global__ void __launch_bounds__(kTileThreads, 2)
    sum_f32_staged_kernel(const __grid_constant__ CUtensorMap tmap, const SumParams p) {
    // the parameters the fix-up of undecided pairs reads (the stage loop
    // reads its own from the constant bank)
    __shared__ SumParams s_par;
    if (!EXACT && threadIdx.x == 0) s_par = p;
    staged_init_barriers<BAND>();
    uint32_t g_it = 0;
    staged_item<BAND, EXACT, DEBUG, INTERP, true, PAD>(&tmap, p, &s_par, p.comp, blockIdx.x, blockIdx.y,
                                                       blockIdx.z, g_it);
}

// One item of the batched kernel as a call of its own: the item body gets
// the register budget of the single-problem kernel instead of sharing it
// with the queue loop (the call happens once per item, thousands of pairs).
// Non-lattice items take the FP64 geometry of undecided pairs from shared
// memory, as the single-problem kernel does.
template <int BAND, bool EXACT, bool INTERP>
__device__ __noinline__ bool staged_batch_item(const CUtensorMap* map, const SumParams& p, int tile, int group,
                                               int ti, uint32_t& g_it) {
    return staged_item<BAND, EXACT, false, INTERP, !EXACT, true>(map, p, &p, p.comp, tile, group, ti, g_it);
}

// Persistent batched kernel: CTAs take (problem, time, split group, tile) items
// from a queue until it is empty; each item runs the same code as the
// single-problem kernel, so a problem's result does not depend on the batch.
template <int BAND, bool EXACT>
__global__ void __launch_bounds__(kTileThreads, 2) sum_f32_staged_batch(const __grid_constant__ StagedBatchArgs a) {
    using L = Layout<BAND>;
    int* s_item = reinterpret_cast<int*>(staged_base<BAND>() + L::kCtrl + 32);
    __shared__ SumParams s_par;
    staged_init_barriers<BAND>();
    uint32_t g_it = 0;
    for (;;) {
        if (threadIdx.x == 0) *s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int item = *s_item;
        __syncthreads();
        if (item >= a.n_items) break;
        int lo = 0, hi = a.n - 1;                 // problem: last start <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.item_start[mid] <= item) lo = mid; else hi = mid - 1;
        }
        // The item's parameters go to shared memory: read through a dynamic
        // index into global memory, their loop invariants would be held in
        // registers (the single-problem kernel reads them from the constant
        // bank) and the batched kernel would spill.
        {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(&a.params[lo]);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&s_par);
            for (int w = threadIdx.x; w < (int)(sizeof(SumParams) / 4); w += kTileThreads) dst[w] = src[w];
        }
        __syncthreads();
        const SumParams& p = s_par;
        const int local = item - a.item_start[lo];
        const int n_groups = (p.n_split + p.split_merge - 1) / p.split_merge;
        const int per_t = p.n_tiles * n_groups;
        const int ti = local / per_t;
        const int r = local - ti * per_t;
        const int group = r / p.n_tiles;
        const int tile = r - group * p.n_tiles;
        // the retarded-time rule is a property of the problem (uniform per item)
        const bool ok = p.interp ? staged_batch_item<BAND, EXACT, true>(&a.maps[lo], p, tile, group, ti, g_it)
                                 : staged_batch_item<BAND, EXACT, false>(&a.maps[lo], p, tile, group, ti, g_it);
        if (!ok) break;
    }
}

template <int BAND, bool EXACT, bool DEBUG, bool INTERP = false>
cudaError_t launch_variant(const SumParams& p, const StagedConfig& c, cudaStream_t s) {
    const dim3 grid(p.n_tiles, (p.n_split + p.split_merge - 1) / p.split_merge, p.n_t);
    const size_t smem = staged_smem_bytes(p, BAND, false);
    // The padding skip changes the stage loop's code: measured, bands of 32
    // rows and more run faster in that form whether or not the grid pads,
    // the 16- and 24-row kernels ~5 % slower unless it does (the heavy-ion
    // and dipole grids do not).  The slot-recording kernels never skip.
    auto k = sum_f32_staged_kernel<BAND, EXACT, DEBUG, INTERP, false>;
    if constexpr (!DEBUG) {
        if (BAND >= 32 || p.pad_yz) k = sum_f32_staged_kernel<BAND, EXACT, DEBUG, INTERP, true>;
    }
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const CUtensorMap* tm = static_cast<const CUtensorMap*>(c.tensor_map);
    k<<<grid, kTileThreads, smem, s>>>(*tm, p);
    return cudaGetLastError();
}

template <int BAND, bool EXACT>
cudaError_t launch_batch_variant(const StagedBatchArgs& a, size_t smem, int grid, cudaStream_t s) {
    auto k = sum_f32_staged_batch<BAND, EXACT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kTileThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// Single-problem launch of one compiled band height.
template <int BAND>
cudaError_t launch_band(const SumParams& p, const StagedConfig& c, cudaStream_t s) {
    const bool dbg = p.debug_slots != nullptr;
    // the slot of every pair is the same with and without interpolation, so
    // the slot-recording kernels exist only in the floor-rule form
    if (!dbg && p.interp)
        return c.exact ? launch_variant<BAND, true, false, true>(p, c, s) : launch_variant<BAND, false, false, true>(p, c, s);
    if (c.exact) return dbg ? launch_variant<BAND, true, true>(p, c, s) : launch_variant<BAND, true, false>(p, c, s);
    return dbg ? launch_variant<BAND, false, true>(p, c, s) : launch_variant<BAND, false, false>(p, c, s);
}

// Batched launch of one compiled band height.
template <int BAND>
cudaError_t launch_batch_band(const StagedBatchArgs& a, bool exact, size_t smem, int grid, cudaStream_t s) {
    return exact ? launch_batch_variant<BAND, true>(a, smem, grid, s) : launch_batch_variant<BAND, false>(a, smem, grid, s);
}

}  // namespace staged
}  // namespace jefi

// Defines the launchers of one compiled band height (declared in
// jefi_internal.h): staged_launch_<BAND> and staged_launch_batch_<BAND>.
#define JEFI_STAGED_BAND_LAUNCHERS(BAND)                                                                   \
    cudaError_t staged_launch_##BAND(const SumParams& p, const StagedConfig& c, cudaStream_t s) {            \
        return staged::launch_band<BAND>(p, c, s);                                                         \
    }                                                                                                      \
    cudaError_t staged_launch_batch_##BAND(const StagedBatchArgs& a, bool exact, size_t smem, int grid,     \
                                           cudaStream_t s) {                                               \
        return staged::launch_batch_band<BAND>(a, exact, smem, grid, s);                                   \
    }
