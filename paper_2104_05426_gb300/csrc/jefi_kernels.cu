// jefi_kernels.cu -- sm_103a kernels of libjefi.
//
//   push_kernel      one source slice -> ring slot (brick order, 8 channels),
//                    backward differences of Eq. E-1 formed in FP64
//   sum_f32_kernel   retarded direct sum of Eqs. E-1/B-1 (FP32 arithmetic,
//                    optional Kahan compensation per thread, FP64 partials)
//   sum_f64_kernel   the same sum in FP64
//   reduce_kernel    deterministic FP64 sum over source splits, scaling,
//                    scatter to input order
//
// Work decomposition of the sums: one CTA = one tile of 256 observation
// points (one per thread; a warp holds a compact 4x4x2 block for grids) x
// one contiguous range of source bricks.  All threads of a warp visit the
// same source cell at the same time, so the ring gathers of a warp hit a few
// neighbouring slots of one cell.  The retarded slot of every pair is exact
// (Eq. tr-1 in FP64): the FP64 kernel compares its exact squared distance
// with exact thresholds, the FP32 kernel proves its slot with error-bounded
// thresholds and recomputes the rare undecided pairs in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "jefi_device.cuh"
#include "jefi_internal.h"

namespace jefi {

using namespace dev;

// ============================================================================ FP32
// Shared memory: tabg[KT] float2 | tabh[KT] float (padded to 16 B) | tab32[K] float4 | theta[K+1] double |
// D[nbx+nby+nbz] float, KT = K + 2 guard

struct Fix6 {
    float v[6];   // E', B contributions
};

// Pairs of a far brick whose slot the FP32 rule left undecided: exact slot
// by the double-float check (slot_double_float), else in FP64, then the pair
// as usual.  A call of its own (rare), so that its registers do not weigh on
// the brick loop.  th_hl: this time's thresholds as FP32 pairs.
template <bool DEBUG, bool INTERP>
__device__ __noinline__ Fix6 direct_fixup(const SumParams& p, uint64_t mask, int slot, int b, int bx, int by, int bz,
                                          float Px, float Py, float Pz, const float4* cbase, const float4* s_tab,
                                          const double* s_th, int64_t k0, float A, float A_lo,
                                          const float2* th_hl) {
    float pe[3] = {0.f, 0.f, 0.f}, pb[3] = {0.f, 0.f, 0.f};
    const int K = p.K, Hp = p.Hp;
    const float K32 = p.K32, K32_lo = p.K32_lo;
    const size_t n_cells = (size_t)p.n_bricks * kBrickCells;
    while (mask) {
        const int cl = __ffsll((long long)mask) - 1;
        mask &= mask - 1;
        const int i = cl & 3, j = (cl >> 2) & 3, k = cl >> 4;
        const float dx = fmaf(-(float)i, p.d32[0], Px);
        const float dy = fmaf(-(float)j, p.d32[1], Py);
        const float dz = fmaf(-(float)k, p.d32[2], Pz);
        const float S = __fadd_rn(__fmul_rn(dx, dx), __fadd_rn(__fmul_rn(dy, dy), __fmul_rn(dz, dz)));
        const float ri = rsqrt_ftz(S);
        const unsigned cand = candidate_index(S, ri, K32, A, K);
        const int ix = kBrick * bx + i, iy = kBrick * by + j, iz = kBrick * bz + k;
        int idx = slot_double_float(p.obs_hl + (size_t)6 * slot, p.cc_hl[ix], p.cc_hl[p.npx + iy],
                                    p.cc_hl[p.npx + p.npy + iz], th_hl, K, (int)cand, S * ri, p.df_b1, p.df_b2);
        if (idx < 0)
            idx = slot_fallback_f32(p.obs_xyz, slot, p.lo[0], p.lo[1], p.lo[2], p.d[0], p.d[1], p.d[2],
                                    p.org[0] + ix, p.org[1] + iy, p.org[2] + iz, s_th, K, (int)cand, nullptr);
        if (DEBUG) p.debug_slots[(size_t)slot * n_cells + (size_t)b * kBrickCells + cl] = (int)(k0 + idx);
        const float4* q = cbase + (cl * Hp + __float_as_int(s_tab[idx].z)) * 2;
        float4 v0 = __ldg(q), v1 = __ldg(q + 1);
        if (INTERP) {
            const float4* q1 = cbase + (cl * Hp + __float_as_int(s_tab[idx + 1].z)) * 2;
            lerp8(v0, v1, __ldg(q1), __ldg(q1 + 1), interp_weight(S, ri, (float)idx, A, A_lo, K32, K32_lo));
        }
        pair_f32(dx, dy, dz, ri, v0, v1, pe, pb);
    }
    return Fix6{{pe[0], pe[1], pe[2], pb[0], pb[1], pb[2]}};
}

template <bool COMP, bool DEBUG, bool INTERP>
__device__ __forceinline__ void direct_f32_item(const SumParams& p, const int tile, const int split,
                                                const int ti) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = p.K;
    const int KT = K + 2 * kTabGuard;
    const uint32_t tabh_off = (uint32_t)KT * 8u;                       // byte offsets in smem
    const uint32_t tab_off = (tabh_off + (uint32_t)KT * 4u + 15u) & ~15u;
    float2* s_tabg = reinterpret_cast<float2*>(smem);
    float* s_tabh = reinterpret_cast<float*>(smem + tabh_off);
    float4* s_tab = reinterpret_cast<float4*>(smem + tab_off);
    double* s_th = reinterpret_cast<double*>(s_tab + K);
    float* s_D = reinterpret_cast<float*>(s_th + K + 1);
    const int tid = threadIdx.x;

    const float4* g_tab = p.tab32 + (size_t)ti * K;
    const double* g_th = p.theta + (size_t)ti * theta_stride(K);
    const float2* g_tabg = p.tabg + (size_t)ti * KT;
    const float* g_tabh = p.tabh + (size_t)ti * KT;
    for (int i = tid; i < KT; i += kTileThreads) {
        s_tabg[i] = g_tabg[i];
        s_tabh[i] = g_tabh[i];
    }
    for (int i = tid; i < K; i += kTileThreads) s_tab[i] = g_tab[i];
    for (int i = tid; i <= K; i += kTileThreads) s_th[i] = g_th[i];
    // s_tabg[bits - kMagicBits + kTabGuard] sits at byte smem + tgbase + 8 bits, s_tabh[...] at
    // smem + thbase + 4 bits (offsets mod 2^32)
    const uint32_t tgbase = (uint32_t)(kTabGuard - kMagicBits) * 8u;
    const uint32_t thbase = tabh_off + (uint32_t)(kTabGuard - kMagicBits) * 4u;
    const bool exact = p.exact != 0;

    // Anchor: the tile's first point.  D[b] = fp32(anchor - centre of the
    // brick's first cell) per axis, so that P = (x_o - anchor) + D is small
    // and well rounded for every pair of a brick.
    const double* txyz = p.obs_xyz + (size_t)tile * kTileThreads * 3;
    const double cox = txyz[0], coy = txyz[1], coz = txyz[2];
    const int nbxy = p.nbx + p.nby;
    for (int i = tid; i < nbxy + p.nbz; i += kTileThreads) {
        int a = i < p.nbx ? 0 : (i < nbxy ? 1 : 2);
        int b = a == 0 ? i : (a == 1 ? i - p.nbx : i - nbxy);
        double co = a == 0 ? cox : (a == 1 ? coy : coz);
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
    const float A = tp.A;
    const float K32 = p.K32;
    const float A_lo = tp.A_lo, K32_lo = p.K32_lo;   // interpolation weights only
    const float Ag = tp.Ag;
    const float d32x = p.d32[0], d32y = p.d32[1], d32z = p.d32[2];
    const int Hp = p.Hp;
    const float4* ring = reinterpret_cast<const float4*>(p.ring);
    const size_t n_cells = (size_t)p.n_bricks * kBrickCells;

    float se[3] = {0.f, 0.f, 0.f}, sb[3] = {0.f, 0.f, 0.f};
    float ce[3] = {0.f, 0.f, 0.f}, cb[3] = {0.f, 0.f, 0.f};
    // pairs whose slot was recomputed in FP64, counted per thread and added
    // once per warp (not one atomic per pair)
    uint32_t n_fb = 0;

    const int b_begin = split * p.bricks_per_split;
    const int b_end = min(b_begin + p.bricks_per_split, p.n_bricks);
    for (int b = b_begin; b < b_end; ++b) {
        const int bx = b % p.nbx;
        const int rest = b / p.nbx;
        const int by = rest % p.nby;
        const int bz = rest / p.nby;
        const float Px = oox + s_D[bx];
        const float Py = ooy + s_D[p.nbx + by];
        const float Pz = ooz + s_D[nbxy + bz];
        const float4* cbase = ring + (size_t)b * kBrickCells * Hp * 2;
        float pe[3] = {0.f, 0.f, 0.f}, pb[3] = {0.f, 0.f, 0.f};

        const bool near = (ctx.rlo[0] <= kBrick * bx + 3) & (ctx.rhi[0] >= kBrick * bx) &
                          (ctx.rlo[1] <= kBrick * by + 3) & (ctx.rhi[1] >= kBrick * by) &
                          (ctx.rlo[2] <= kBrick * bz + 3) & (ctx.rhi[2] >= kBrick * bz);
        if (__any_sync(kFull, near)) {
            // Bricks that may hold screened pairs: rolled loop with the
            // per-pair screening test (rare: only bricks next to the tile).
            for (int cl = 0; cl < kBrickCells; ++cl) {
                const int i = cl & 3, j = (cl >> 2) & 3, k = cl >> 4;
                const int ix = kBrick * bx + i, iy = kBrick * by + j, iz = kBrick * bz + k;
                const float dx = fmaf(-(float)i, d32x, Px);
                const float dy = fmaf(-(float)j, d32y, Py);
                const float dz = fmaf(-(float)k, d32z, Pz);
                const float S = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)),
                                          __fmul_rn(dz, dz));
                const bool scr = (ix >= ctx.rlo[0]) & (ix <= ctx.rhi[0]) & (iy >= ctx.rlo[1]) &
                                 (iy <= ctx.rhi[1]) & (iz >= ctx.rlo[2]) & (iz <= ctx.rhi[2]);
                float ri = rsqrt_ftz(S);
                unsigned idx = candidate_index(S, ri, K32, A, K);
                float4 e = s_tab[idx];
                bool ok = scr | ((S <= e.x) & (S > e.y));
                if (__any_sync(kFull, !ok)) {
                    if (!ok) {
                        idx = slot_fallback_f32(p.obs_xyz, ctx.slot, p.lo[0], p.lo[1], p.lo[2],
                                                p.d[0], p.d[1], p.d[2], p.org[0] + ix, p.org[1] + iy,
                                                p.org[2] + iz, s_th, K, (int)idx, nullptr);
                        ++n_fb;
                        e = s_tab[idx];
                    }
                }
                const int ps = scr ? p.zero_slot : __float_as_int(e.z);
                if (scr) ri = 0.f;
                if (DEBUG) {
                    p.debug_slots[(size_t)ctx.slot * n_cells + (size_t)b * kBrickCells + cl] =
                        scr ? INT32_MIN : (int)(tp.k0 + idx);
                }
                const float4* q = cbase + (cl * Hp + ps) * 2;
                float4 v0 = __ldg(q), v1 = __ldg(q + 1);
                if (INTERP) {   // slot n+1: the next candidate's physical slot
                    const int ps1 = scr ? p.zero_slot : __float_as_int(s_tab[idx + 1].z);
                    const float4* q1 = cbase + (cl * Hp + ps1) * 2;
                    lerp8(v0, v1, __ldg(q1), __ldg(q1 + 1),
                          interp_weight(S, ri, (float)(int)idx, A, A_lo, K32, K32_lo));
                }
                pair_f32(dx, dy, dz, ri, v0, v1, pe, pb);
            }
        } else {
            // Far bricks: the staged kernel's slot rule (candidate k' from
            // A + g, one threshold decides k' or k'-1) with the slot's row
            // read from global memory; no branch per pair, so the gathers of
            // a slab can all be in flight together.  The z slabs are a rolled
            // loop, the 16 cells of a slab are unrolled.
            float ddx[4], ddy[4], sqx[4], sqy[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ddx[i] = fmaf(-(float)i, d32x, Px);
                ddy[i] = fmaf(-(float)i, d32y, Py);
                sqx[i] = __fmul_rn(ddx[i], ddx[i]);
                sqy[i] = __fmul_rn(ddy[i], ddy[i]);
            }
            uint64_t mask = 0;          // undecided pairs (non-lattice geometry), redone below
            float2 acc_eyz = make_float2(0.f, 0.f), acc_bxy = make_float2(0.f, 0.f);
            float acc_ex = 0.f, acc_bz = 0.f;
#pragma unroll 1
            for (int k = 0; k < 4; ++k) {
                const float dz = fmaf(-(float)k, d32z, Pz);
                const float sqz = __fmul_rn(dz, dz);
                const float4* ck = cbase + (size_t)(k * 16) * Hp * 2;
                float2 dyz[4], dzx[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    dyz[i] = make_float2(ddy[i], dz);
                    dzx[i] = make_float2(dz, ddx[i]);
                }
                uint32_t m16 = 0;           // undecided cells of this slab
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float syz = __fadd_rn(sqy[j], sqz);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int c16 = j * 4 + i;
                        const float S = __fadd_rn(sqx[i], syz);
                        float ri = rsqrt_ftz(S);
                        const uint32_t bits = __float_as_uint(__fadd_rd(fmaf(-(S * ri), K32, Ag), kMagic));
                        const float2 e = *reinterpret_cast<const float2*>(smem + (tgbase + bits * 8u));
                        const bool lower = S > e.x;
                        if (!exact) {   // T_hi < S <= T_lo: undecided, redone after the brick
                            const float th_hi = *reinterpret_cast<const float*>(smem + (thbase + bits * 4u));
                            if (!(S <= th_hi) && !lower) {
                                m16 |= 1u << c16;   // c16 is a constant of the unrolled body
                                ri = 0.f;
                            }
                        }
                        const uint32_t pk = __float_as_uint(e.y);
                        const int ps = (int)(lower ? (pk >> 16) : (pk & 0xFFFFu));
                        if (DEBUG) {
                            p.debug_slots[(size_t)ctx.slot * n_cells + (size_t)b * kBrickCells + k * 16 + c16] =
                                (int)(tp.k0 + (int)(bits - kMagicBits) - (lower ? 1 : 0));
                        }
                        const float4* q = ck + (c16 * Hp + ps) * 2;
                        float4 v0, v1;
                        ldg_row8(q, v0, v1);
                        if (INTERP) {   // slot n+1: k' when n = k'-1, else k'+1
                            const uint32_t pk1 = *reinterpret_cast<const uint32_t*>(smem + (tgbase + bits * 8u + 12u));
                            const float4* q1 = ck + (c16 * Hp + (int)(lower ? (pk & 0xFFFFu) : (pk1 & 0xFFFFu))) * 2;
                            const float nrel = __uint_as_float(bits - (lower ? 1u : 0u)) - kMagic;
                            float4 u0, u1;
                            ldg_row8(q1, u0, u1);
                            lerp8(v0, v1, u0, u1, interp_weight(S, ri, nrel, A, A_lo, K32, K32_lo));
                        }
                        // Eqs. E-1/B-1, packed, r^-2 factored out (as in the staged kernel)
                        const float2 ri2 = make_float2(ri, ri);
                        const float2 r2 = __fmul2_rn(ri2, ri2);
                        const float2 qvx = __fmul2_rn(__ffma2_rn(make_float2(v0.x, v0.y), ri2,
                                                                 make_float2(v1.x, v1.y)), r2);
                        const float2 vyz = __fmul2_rn(__ffma2_rn(make_float2(v0.z, v0.w), ri2,
                                                                 make_float2(v1.z, v1.w)), r2);
                        const float qq = qvx.x, vx = qvx.y;
                        acc_ex = fmaf(ddx[i], qq, acc_ex);
                        acc_ex = fmaf(-v1.y, ri, acc_ex);
                        acc_eyz = __ffma2_rn(dyz[j], make_float2(qq, qq), acc_eyz);
                        acc_eyz = __ffma2_rn(make_float2(-v1.z, -v1.w), ri2, acc_eyz);
                        acc_bxy = __ffma2_rn(vyz, dzx[i], acc_bxy);
                        acc_bxy.x = fmaf(-vyz.y, ddy[j], acc_bxy.x);
                        acc_bxy.y = fmaf(-vx, dz, acc_bxy.y);
                        acc_bz = fmaf(vx, ddy[j], acc_bz);
                        acc_bz = fmaf(-vyz.x, ddx[i], acc_bz);
                    }
                }
                if (!exact) mask |= (uint64_t)m16 << (k * 16);
            }
            pe[0] += acc_ex;
            pe[1] += acc_eyz.x;
            pe[2] += acc_eyz.y;
            pb[0] += acc_bxy.x;
            pb[1] += acc_bxy.y;
            pb[2] += acc_bz;
            if (__any_sync(kFull, mask != 0ull)) {
                n_fb += (uint32_t)__popcll(mask);
                const Fix6 f = direct_fixup<DEBUG, INTERP>(
                    p, mask, ctx.slot, b, bx, by, bz, Px, Py, Pz, cbase, s_tab, s_th, tp.k0, A, A_lo,
                    reinterpret_cast<const float2*>(p.theta + (size_t)ti * theta_stride(K) + (K + 1)));
                pe[0] += f.v[0];
                pe[1] += f.v[1];
                pe[2] += f.v[2];
                pb[0] += f.v[3];
                pb[1] += f.v[4];
                pb[2] += f.v[5];
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (COMP) {
                kahan_add(se[a], ce[a], pe[a]);
                kahan_add(sb[a], cb[a], pb[a]);
            } else {
                se[a] += pe[a];
                sb[a] += pb[a];
            }
        }
    }

    {
        const uint32_t w = __reduce_add_sync(kFull, n_fb);
        if ((tid & 31) == 0 && w) atomicAdd(p.fallbacks, (unsigned long long)w);
    }
    double* out = p.partials + ((size_t)ti * p.n_split + split) * 6 * p.n_slots + ctx.slot;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // s - c: the Kahan compensation holds the negated lost low part
        out[(size_t)a * p.n_slots] = COMP ? (double)se[a] - (double)ce[a] : (double)se[a];
        out[(size_t)(3 + a) * p.n_slots] = COMP ? (double)sb[a] - (double)cb[a] : (double)sb[a];
    }
}

template <bool COMP, bool DEBUG, bool INTERP>
__global__ void __launch_bounds__(kTileThreads, 2) sum_f32_kernel(const SumParams p) {
    direct_f32_item<COMP, DEBUG, INTERP>(p, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Take the next item of a persistent batched launch; false when the queue is empty.
__device__ __forceinline__ bool next_item(const BatchArgs& a, int* s_item, int* pr, int* tile, int* split, int* ti) {
    if (threadIdx.x == 0) *s_item = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int item = *s_item;
    __syncthreads();
    if (item >= a.n_items) return false;
    int lo = 0, hi = a.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.item_start[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const SumParams& p = a.params[lo];
    const int local = item - a.item_start[lo];
    const int per_t = p.n_tiles * p.n_split;
    *pr = lo;
    *ti = local / per_t;
    const int r = local - *ti * per_t;
    *split = r / p.n_tiles;
    *tile = r - *split * p.n_tiles;
    return true;
}

// One item of the batched direct-gather kernel as a call of its own (the
// item body keeps the single-problem kernel's register budget).
template <bool COMP, bool INTERP>
__device__ __noinline__ void direct_batch_item(const SumParams& p, int tile, int split, int ti) {
    direct_f32_item<COMP, false, INTERP>(p, tile, split, ti);
}

template <bool COMP>
__global__ void __launch_bounds__(kTileThreads, 2) sum_f32_batch(const BatchArgs a) {
    __shared__ int s_item;
    __shared__ SumParams s_par;
    int pr, tile, split, ti;
    while (next_item(a, &s_item, &pr, &tile, &split, &ti)) {
        // The item's parameters go to shared memory (every thread passed the
        // queue's barriers, so none still reads the previous item's): read
        // through a dynamic index into global memory, their loop invariants
        // would be held in registers and spilled.
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&a.params[pr]);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&s_par);
        for (int w = threadIdx.x; w < (int)(sizeof(SumParams) / 4); w += kTileThreads) dst[w] = src[w];
        __syncthreads();
        if (s_par.interp)     // the retarded-time rule is a property of the problem (uniform per item)
            direct_batch_item<COMP, true>(s_par, tile, split, ti);
        else
            direct_batch_item<COMP, false>(s_par, tile, split, ti);
    }
}

// ============================================================================ FP64
// Shared memory: tab32[K] float4 | theta[K+1] double | xs[npx] ys[npy] zs[npz] double
__device__ __forceinline__ void pair_f64(double dx, double dy, double dz, double ri,
                                         const double2& a0, const double2& a1, const double2& a2,
                                         const double2& a3, double (&pe)[3], double (&pb)[3]) {
    // a0 = (c rho, Jx), a1 = (Jy, Jz), a2 = (drho, dJx/c), a3 = (dJy/c, dJz/c)
    const double r2 = ri * ri;
    const double r3 = r2 * ri;
    const double q = fma(a2.x, r2, a0.x * r3);
    pe[0] = fma(dx, q, pe[0]);
    pe[1] = fma(dy, q, pe[1]);
    pe[2] = fma(dz, q, pe[2]);
    pe[0] = fma(-a2.y, ri, pe[0]);
    pe[1] = fma(-a3.x, ri, pe[1]);
    pe[2] = fma(-a3.y, ri, pe[2]);
    const double vx = fma(a2.y, r2, a0.y * r3);
    const double vy = fma(a3.x, r2, a1.x * r3);
    const double vz = fma(a3.y, r2, a1.y * r3);
    pb[0] = fma(vy, dz, pb[0]);
    pb[1] = fma(vz, dx, pb[1]);
    pb[2] = fma(vx, dy, pb[2]);
    pb[0] = fma(-vz, dy, pb[0]);
    pb[1] = fma(-vx, dz, pb[1]);
    pb[2] = fma(-vy, dx, pb[2]);
}

// Second-order retarded time: the channels of slot n moved toward those of
// slot n+1 by the weight w = u - n, u = (T - R/c)/dt (Eq. tr-1 without the floor).
__device__ __forceinline__ double2 lerp2(const double2& a, const double2& b, double w) {
    return make_double2(fma(w, b.x - a.x, a.x), fma(w, b.y - a.y, a.y));
}

template <bool DEBUG, bool INTERP>
__device__ __forceinline__ void f64_item(const SumParams& p, const int tile, const int split, const int ti) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = p.K;
    float4* s_tab = reinterpret_cast<float4*>(smem);
    double* s_th = reinterpret_cast<double*>(s_tab + K);
    double* s_xs = s_th + K + 1;
    double* s_ys = s_xs + p.npx;
    double* s_zs = s_ys + p.npy;

    const int tid = threadIdx.x;
    const float4* g_tab = p.tab32 + (size_t)ti * K;
    const double* g_th = p.theta + (size_t)ti * theta_stride(K);
    for (int i = tid; i < K; i += kTileThreads) s_tab[i] = g_tab[i];
    for (int i = tid; i <= K; i += kTileThreads) s_th[i] = g_th[i];
    for (int i = tid; i < p.npx; i += kTileThreads) s_xs[i] = cell_center(p.lo[0], p.d[0], p.org[0] + i);
    for (int i = tid; i < p.npy; i += kTileThreads) s_ys[i] = cell_center(p.lo[1], p.d[1], p.org[1] + i);
    for (int i = tid; i < p.npz; i += kTileThreads) s_zs[i] = cell_center(p.lo[2], p.d[2], p.org[2] + i);
    __syncthreads();

    ThreadCtx ctx;
    ctx.slot = tile * kTileThreads + tid;
    const double xo = p.obs_xyz[3 * ctx.slot + 0];
    const double yo = p.obs_xyz[3 * ctx.slot + 1];
    const double zo = p.obs_xyz[3 * ctx.slot + 2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ctx.rlo[a] = p.obs_scr[(2 * a) * p.n_slots + ctx.slot];
        ctx.rhi[a] = p.obs_scr[(2 * a + 1) * p.n_slots + ctx.slot];
    }
    const TimeParams tp = p.times[ti];
    const float A = tp.A;
    const float K32 = p.K32;
    const int Hp = p.Hp;
    const double2* ring = reinterpret_cast<const double2*>(p.ring);
    const size_t n_cells = (size_t)p.n_bricks * kBrickCells;

    double se[3] = {0, 0, 0}, sb[3] = {0, 0, 0};
    const int b_begin = split * p.bricks_per_split;
    const int b_end = min(b_begin + p.bricks_per_split, p.n_bricks);
    for (int b = b_begin; b < b_end; ++b) {
        const int bx = b % p.nbx;
        const int rest = b / p.nbx;
        const int by = rest % p.nby;
        const int bz = rest / p.nby;
        double ddx[4], ddy[4], ddz[4], sqx[4], sqy[4], sqz[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ddx[i] = __dsub_rn(xo, s_xs[kBrick * bx + i]);
            ddy[i] = __dsub_rn(yo, s_ys[kBrick * by + i]);
            ddz[i] = __dsub_rn(zo, s_zs[kBrick * bz + i]);
            sqx[i] = __dmul_rn(ddx[i], ddx[i]);
            sqy[i] = __dmul_rn(ddy[i], ddy[i]);
            sqz[i] = __dmul_rn(ddz[i], ddz[i]);
        }
        double sxy[16];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) sxy[j * 4 + i] = __dadd_rn(sqx[i], sqy[j]);
        const bool near = (ctx.rlo[0] <= kBrick * bx + 3) & (ctx.rhi[0] >= kBrick * bx) &
                          (ctx.rlo[1] <= kBrick * by + 3) & (ctx.rhi[1] >= kBrick * by) &
                          (ctx.rlo[2] <= kBrick * bz + 3) & (ctx.rhi[2] >= kBrick * bz);
        const bool any_near = __any_sync(kFull, near);
        const double2* cbase = ring + (size_t)b * kBrickCells * Hp * 4;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int cl = k * 16 + j * 4 + i;
                    const double S = __dadd_rn(sxy[j * 4 + i], sqz[k]);
                    bool scr = false;
                    if (any_near) {
                        const int ix = kBrick * bx + i, iy = kBrick * by + j, iz = kBrick * bz + k;
                        scr = (ix >= ctx.rlo[0]) & (ix <= ctx.rhi[0]) & (iy >= ctx.rlo[1]) &
                              (iy <= ctx.rhi[1]) & (iz >= ctx.rlo[2]) & (iz <= ctx.rhi[2]);
                    }
                    const float Sf = __double2float_rn(S);
                    int it = (int)candidate_index(Sf, rsqrtf(Sf), K32, A, K);
                    if (!scr) {
                        if (!((S <= s_th[it]) & (S > s_th[it + 1]))) it = theta_search(s_th, K, it, S);
                    }
                    const int ps = scr ? p.zero_slot : __float_as_int(s_tab[it].z);
                    if (DEBUG) {
                        p.debug_slots[(size_t)ctx.slot * n_cells + (size_t)b * kBrickCells + cl] =
                            scr ? INT32_MIN : (int)(tp.k0 + it);
                    }
                    const double ri = scr ? 0.0 : rsqrt(S);
                    const double2* q = cbase + (cl * Hp + ps) * 4;
                    double2 a0 = __ldg(q), a1 = __ldg(q + 1), a2 = __ldg(q + 2), a3 = __ldg(q + 3);
                    if (INTERP) {
                        const int ps1 = scr ? p.zero_slot : __float_as_int(s_tab[it + 1].z);
                        const double2* q1 = cbase + (cl * Hp + ps1) * 4;
                        // w = (T/dt - k0) - R/(c dt) - (n - k0), R = S / sqrt(S)
                        const double w = fma(-(S * ri), p.K64, tp.A64) - (double)it;
                        a0 = lerp2(a0, __ldg(q1), w);
                        a1 = lerp2(a1, __ldg(q1 + 1), w);
                        a2 = lerp2(a2, __ldg(q1 + 2), w);
                        a3 = lerp2(a3, __ldg(q1 + 3), w);
                    }
                    pair_f64(ddx[i], ddy[j], ddz[k], ri, a0, a1, a2, a3, se, sb);
                }
            }
        }
    }
    double* out = p.partials + ((size_t)ti * p.n_split + split) * 6 * p.n_slots + ctx.slot;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        out[(size_t)a * p.n_slots] = se[a];
        out[(size_t)(3 + a) * p.n_slots] = sb[a];
    }
}

template <bool DEBUG, bool INTERP>
__global__ void __launch_bounds__(kTileThreads, 1) sum_f64_kernel(const SumParams p) {
    f64_item<DEBUG, INTERP>(p, blockIdx.x, blockIdx.y, blockIdx.z);
}

__global__ void __launch_bounds__(kTileThreads, 1) sum_f64_batch(const BatchArgs a) {
    __shared__ int s_item;
    int pr, tile, split, ti;
    while (next_item(a, &s_item, &pr, &tile, &split, &ti)) {
        if (a.params[pr].interp)
            f64_item<false, true>(a.params[pr], tile, split, ti);
        else
            f64_item<false, false>(a.params[pr], tile, split, ti);
    }
}

// ============================================================================ push
__global__ void push_kernel(const PushParams p) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= p.n_src) return;
    const int ix = (int)(g % p.nx);
    const int64_t r = g / p.nx;
    const int iy = (int)(r % p.ny);
    const int iz = (int)(r / p.ny);
    const int64_t brick = ((int64_t)(iz >> 2) * p.nby + (iy >> 2)) * p.nbx + (ix >> 2);
    const int64_t cell = brick * kBrickCells + ((iz & 3) * 16 + (iy & 3) * 4 + (ix & 3));
    // the same cell in the caller's slice arrays (a region of a larger grid, or the grid itself)
    const int64_t gs = ((int64_t)(p.oz + iz) * p.fny + (p.oy + iy)) * p.fnx + (p.ox + ix);

    const double rho = p.rho[gs];
    const double j0 = p.J[3 * gs + 0], j1 = p.J[3 * gs + 1], j2 = p.J[3 * gs + 2];
    if (p.central && p.prev_slot >= 0) {
        // slice n-1 now has both neighbours: its derivative channels become
        // the central difference (f[n] - f[n-2]) / (2 dt), f[-1] = 0
        double* p2 = p.prev2 + 4 * g;
        const double two_dt = __dmul_rn(2.0, p.dt);
        const double cd[4] = {__ddiv_rn(__dsub_rn(rho, p2[0]), two_dt),
                              __ddiv_rn(__ddiv_rn(__dsub_rn(j0, p2[1]), two_dt), p.c),
                              __ddiv_rn(__ddiv_rn(__dsub_rn(j1, p2[2]), two_dt), p.c),
                              __ddiv_rn(__ddiv_rn(__dsub_rn(j2, p2[3]), two_dt), p.c)};
        const int n_cp = p.prev_mirror_slot >= 0 ? 2 : 1;
        for (int copy = 0; copy < n_cp; ++copy) {
            const int slot = copy == 0 ? p.prev_slot : p.prev_mirror_slot;
            const size_t off = ((size_t)cell * p.Hp + slot) * 8 + 4;
            if (p.fp64) {
                double2* dst = reinterpret_cast<double2*>(static_cast<double*>(p.ring) + off);
                dst[0] = make_double2(cd[0], cd[1]);
                dst[1] = make_double2(cd[2], cd[3]);
            } else {
                float4* dst = reinterpret_cast<float4*>(static_cast<float*>(p.ring) + off);
                dst[0] = make_float4(__double2float_rn(cd[0]), __double2float_rn(cd[1]),
                                     __double2float_rn(cd[2]), __double2float_rn(cd[3]));
            }
        }
    }
    if (p.central) {
        // slice n-1 (still in prev, updated below) becomes slice n-2
        double* p2 = p.prev2 + 4 * g;
        const double* pv = p.prev + 4 * g;
        p2[0] = pv[0];
        p2[1] = pv[1];
        p2[2] = pv[2];
        p2[3] = pv[3];
    }
    double dr, dj0, dj1, dj2;
    if (p.supplied) {
        dr = p.drho[gs];
        dj0 = p.dJ[3 * gs + 0];
        dj1 = p.dJ[3 * gs + 1];
        dj2 = p.dJ[3 * gs + 2];
    } else {
        // backward difference (f[n] - f[n-1]) / dt, Eq. E-1
        double* pv = p.prev + 4 * g;
        dr = __ddiv_rn(__dsub_rn(rho, pv[0]), p.dt);
        dj0 = __ddiv_rn(__dsub_rn(j0, pv[1]), p.dt);
        dj1 = __ddiv_rn(__dsub_rn(j1, pv[2]), p.dt);
        dj2 = __ddiv_rn(__dsub_rn(j2, pv[3]), p.dt);
        pv[0] = rho;
        pv[1] = j0;
        pv[2] = j1;
        pv[3] = j2;
    }
    const double ch[8] = {__dmul_rn(p.c, rho), j0, j1, j2, dr, __ddiv_rn(dj0, p.c),
                          __ddiv_rn(dj1, p.c), __ddiv_rn(dj2, p.c)};
    const int n_copies = p.mirror_slot >= 0 ? 2 : 1;
    for (int copy = 0; copy < n_copies; ++copy) {
        const int slot = copy == 0 ? p.slot : p.mirror_slot;
        const size_t off = ((size_t)cell * p.Hp + slot) * 8;
        if (p.fp64) {
            double2* dst = reinterpret_cast<double2*>(static_cast<double*>(p.ring) + off);
            dst[0] = make_double2(ch[0], ch[1]);
            dst[1] = make_double2(ch[2], ch[3]);
            dst[2] = make_double2(ch[4], ch[5]);
            dst[3] = make_double2(ch[6], ch[7]);
        } else {
            float4* dst = reinterpret_cast<float4*>(static_cast<float*>(p.ring) + off);
            dst[0] = make_float4(__double2float_rn(ch[0]), __double2float_rn(ch[1]),
                                 __double2float_rn(ch[2]), __double2float_rn(ch[3]));
            dst[1] = make_float4(__double2float_rn(ch[4]), __double2float_rn(ch[5]),
                                 __double2float_rn(ch[6]), __double2float_rn(ch[7]));
        }
    }
}

// ============================================================================ reduce
__global__ void reduce_kernel(const ReduceParams p) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)p.n_t * p.n_obs;
    if (gid >= total) return;
    const int ti = (int)(gid / p.n_obs);
    const int o = (int)(gid % p.n_obs);
    const int slot = p.inv_perm[o];
    const double* base = p.partials + (size_t)ti * p.n_split * 6 * p.n_slots + slot;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int s = 0; s < p.n_split; ++s) {
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += base[((size_t)s * 6 + c) * p.n_slots];
    }
    double* E = p.E + (size_t)gid * 3;
    double* B = p.B + (size_t)gid * 3;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        E[a] = acc[a] * p.e_scale;
        B[a] = acc[3 + a] * p.b_scale;
    }
}

// Batched reduction: output point `gid` of the concatenation of all items.
__global__ void reduce_batch_kernel(const ReduceItem* items, const int64_t* out_start, int n, int64_t total) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (out_start[mid] <= gid) lo = mid; else hi = mid - 1;
    }
    const ReduceItem it = items[lo];
    const int o = (int)(gid - out_start[lo]);
    const double* base = it.partials + it.inv_perm[o];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int s = 0; s < it.n_split; ++s) {
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += base[((size_t)s * 6 + c) * it.n_slots];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        it.E[(size_t)o * 3 + a] = acc[a] * it.e_scale;
        it.B[(size_t)o * 3 + a] = acc[3 + a] * it.b_scale;
    }
}

// ============================================================================ S-O sums
// E = sum over parts k = 0, 1, ... of E_parts[k], in that order (FP64): the
// fields of S-O pairs that share their observation points (paper Sec. 2.2,
// Fig. 2), summed in the same order whatever the number of ranks.
__global__ void sum_parts_kernel(const SumPartsParams p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    double e = 0.0, b = 0.0;
    for (int k = 0; k < p.n_parts; ++k) {
        e += p.E_parts[k][i];
        b += p.B_parts[k][i];
    }
    p.E[i] = e;
    p.B[i] = b;
}

// ============================================================================ launchers
cudaError_t launch_sum_parts(const SumPartsParams& p, cudaStream_t s) {
    if (p.n == 0) return cudaSuccess;
    sum_parts_kernel<<<(unsigned)((p.n + 255) / 256), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_sum_f32_batch(const BatchArgs& a, bool compensated, size_t smem, int grid, cudaStream_t s) {
    void (*k)(BatchArgs) = compensated ? sum_f32_batch<true> : sum_f32_batch<false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kTileThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sum_f64_batch(const BatchArgs& a, size_t smem, int grid, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(sum_f64_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sum_f64_batch<<<grid, kTileThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reduce_batch(const ReduceItem* items, const int64_t* out_start, int n, int64_t total,
                                cudaStream_t s) {
    if (total == 0) return cudaSuccess;
    reduce_batch_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(items, out_start, n, total);
    return cudaGetLastError();
}

size_t sum_smem_bytes(const SumParams& p) {
    size_t b = (size_t)p.K * sizeof(float4) + (size_t)(p.K + 1) * sizeof(double);
    if (p.tabg) b += ((size_t)(p.K + 2 * kTabGuard) * 12 + 15) & ~(size_t)15;
    return b + (size_t)(p.npx + p.npy + p.npz) * sizeof(double);
}

cudaError_t launch_sum_f32(const SumParams& p, bool compensated, cudaStream_t s) {
    const dim3 grid(p.n_tiles, p.n_split, p.n_t);
    const size_t smem = sum_smem_bytes(p);
    void (*k)(SumParams);
    if (p.debug_slots)
        k = compensated ? sum_f32_kernel<true, true, false> : sum_f32_kernel<false, true, false>;
    else if (p.interp)
        k = compensated ? sum_f32_kernel<true, false, true> : sum_f32_kernel<false, false, true>;
    else
        k = compensated ? sum_f32_kernel<true, false, false> : sum_f32_kernel<false, false, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kTileThreads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_sum_f64(const SumParams& p, cudaStream_t s) {
    const dim3 grid(p.n_tiles, p.n_split, p.n_t);
    const size_t smem = sum_smem_bytes(p);
    void (*k)(SumParams) = p.debug_slots ? sum_f64_kernel<true, false>
                           : (p.interp ? sum_f64_kernel<false, true> : sum_f64_kernel<false, false>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kTileThreads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_push(const PushParams& p, cudaStream_t s) {
    if (p.n_src == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (p.n_src + threads - 1) / threads;
    push_kernel<<<(unsigned)blocks, threads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const ReduceParams& p, cudaStream_t s) {
    const int64_t total = (int64_t)p.n_t * p.n_obs;
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    reduce_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace jefi
