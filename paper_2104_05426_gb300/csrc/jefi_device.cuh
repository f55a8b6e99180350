// jefi_device.cuh -- device helpers shared by the libjefi kernels: the exact
// FP64 cell-centre and squared-distance rules, the threshold search, the FP32
// slot candidate, compensated addition and the per-pair FP32 accumulation of
// Eqs. E-1 and B-1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace jefi {
namespace dev {

static constexpr unsigned kFull = 0xffffffffu;
static constexpr float kMagic = 12582912.0f;      // 1.5 * 2^23: rd(u + M) has floor(u) in its low bits
static constexpr int kMagicBits = 0x4B400000;

// Cell centre x_i = lo + (i + 0.5) d, product then sum, each rounded.
static __device__ __forceinline__ double cell_center(double lo, double d, int i) {
    return __dadd_rn(lo, __dmul_rn(__dadd_rn((double)i, 0.5), d));
}

// Spec squared distance (Dx*Dx + Dy*Dy) + Dz*Dz, every operation rounded.
static __device__ __forceinline__ double spec_s64(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Table index whose threshold interval (theta[i+1], theta[i]] holds S.
// Thresholds are non-increasing; the exact slot always lies strictly
// inside the table, so both walks stop there.
static __device__ __forceinline__ int theta_search(const double* th, int K, int i, double S) {
    i = i < 0 ? 0 : (i > K - 1 ? K - 1 : i);
    while (i > 0 && S > th[i]) --i;
    while (i < K - 1 && S <= th[i + 1]) ++i;
    return i;
}

// Exact slot of one pair from scratch in FP64 (the rare undecided case of
// the FP32 kernel).  Returns the table index.
static __device__ __noinline__ int slot_fallback_f32(const double* obs_xyz, int slot, double lox,
                                              double loy, double loz, double dx_, double dy_,
                                              double dz_, int ix, int iy, int iz,
                                              const double* th, int K, int guess,
                                              unsigned long long* counter) {
    const double xo = obs_xyz[3 * slot + 0];
    const double yo = obs_xyz[3 * slot + 1];
    const double zo = obs_xyz[3 * slot + 2];
    const double S = spec_s64(__dsub_rn(xo, cell_center(lox, dx_, ix)),
                              __dsub_rn(yo, cell_center(loy, dy_, iy)),
                              __dsub_rn(zo, cell_center(loz, dz_, iz)));
    if (counter) atomicAdd(counter, 1ull);
    return theta_search(th, K, guess, S);
}

// Exact slot of one pair in FP64 from the point and the source cell centre
// (each an FP64 value the spec computes: the point as given, the centre by
// cell_center), stored in shared memory by the caller: the spec's squared
// distance and the threshold search, with no global load.
static __device__ __forceinline__ int slot_fp64_stored(const double* xo, double cx, double cy, double cz,
                                                       const double* th, int K, int guess) {
    const double S = spec_s64(__dsub_rn(xo[0], cx), __dsub_rn(xo[1], cy), __dsub_rn(xo[2], cz));
    return theta_search(th, K, guess, S);
}

// a + b as s + e exactly (Knuth's two-sum; no operation may be contracted).
static __device__ __forceinline__ void two_sum_f32(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Exact slot of an undecided pair without FP64 arithmetic, where it is
// clearly inside one slot (a cheap pre-check before the FP64 rule: FP64
// instructions run at 1/64 of the FP32 rate on this GPU).
//
// The squared distance is formed in double-float arithmetic from the point
// and the cell centre split into FP32 pairs (hi = nearest float, lo = nearest
// float to the remainder; both within 2^-48 of the FP64 value), every
// difference by two-sum, every square as hi^2 (exact, by fma) + 2 hi lo.  On
// creation the host bounds |S_df - S64| <= B = b1 R + b2 S (S64 the FP64
// rule's squared distance; R a distance within 1e-5 of the pair's).  With
// the thresholds as FP32 pairs too, slot i (theta[i+1] < S64 <= theta[i]) is
// certain when S_df - theta[i] <= -B and S_df - theta[i+1] > B.  Only the
// candidate g (the FP32 rule's k') and g - 1 are tried: the exact slot is one
// of them.  Returns the table index, or -1 if the pair is within B of a
// threshold (an exact tie of the FP64 rule, typically): the caller then
// takes the FP64 rule.
static __device__ __forceinline__ int slot_double_float(const float* xo_hl, float2 cx, float2 cy, float2 cz,
                                                        const float2* th_hl, int K, int g, float R, float b1,
                                                        float b2) {
    if (g < 1 || g > K - 1) return -1;
    const float2 c[3] = {cx, cy, cz};
    float ph[3], pl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float s, e;
        two_sum_f32(xo_hl[2 * a], -c[a].x, s, e);
        float dh, dl;
        two_sum_f32(s, __fadd_rn(e, __fsub_rn(xo_hl[2 * a + 1], c[a].y)), dh, dl);
        ph[a] = __fmul_rn(dh, dh);
        pl[a] = fmaf(__fmul_rn(2.f, dh), dl, fmaf(dh, dh, -ph[a]));
    }
    float s1, e1, s2, e2;
    two_sum_f32(ph[0], ph[1], s1, e1);
    two_sum_f32(s1, ph[2], s2, e2);
    const float lo = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(pl[0], pl[1]), pl[2]));
    const float Sh = __fadd_rn(s2, lo);
    const float Sl = __fsub_rn(lo, __fsub_rn(Sh, s2));
    const float B = fmaf(b1, R, __fmul_rn(b2, Sh));
    auto diff = [&](int i) {   // S_df - theta[i]
        const float2 t = th_hl[i];
        return __fadd_rn(__fsub_rn(Sh, t.x), __fsub_rn(Sl, t.y));
    };
    const float d0 = diff(g);
    if (d0 <= -B && diff(g + 1) > B) return g;
    if (d0 > B && diff(g - 1) <= -B) return g - 1;
    return -1;
}

static __device__ __forceinline__ unsigned candidate_index(float S, float ri, float K32, float A, int K) {
    const float R = S * ri;
    const float u = fmaf(-R, K32, A);
    const int bits = __float_as_int(__fadd_rd(u, kMagic));
    const unsigned idx = (unsigned)(bits - kMagicBits);
    return min(idx, (unsigned)(K - 1));
}

// 1/sqrt(x) by rsqrt.approx.ftz.f32.  For normal x it returns what rsqrtf
// returns; it leaves out rsqrtf's rescaling of subnormal inputs.  The FP32
// kernels only see S >= 1e-30 (jefi_create rejects FP32 problems with closer
// unscreened pairs) or S = 0 on screened pairs, whose result is discarded.
static __device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// One ring row (8 FP32 channels, 32 bytes, 32-byte aligned) in a single
// 256-bit global load through the read-only path: half the L1 requests of
// two 128-bit loads, and each sector is touched once.
static __device__ __forceinline__ void ldg_row8(const float4* q, float4& v0, float4& v1) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v0.x), "=f"(v0.y), "=f"(v0.z), "=f"(v0.w), "=f"(v1.x), "=f"(v1.y), "=f"(v1.z), "=f"(v1.w)
        : "l"(q));
}

static __device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Accumulate one pair (FP32).  v0 = (c rho, J), v1 = (drho, dJ/c).
static __device__ __forceinline__ void pair_f32(float dx, float dy, float dz, float ri, const float4& v0,
                                         const float4& v1, float (&pe)[3], float (&pb)[3]) {
    const float r2 = ri * ri;
    const float r3 = r2 * ri;
    const float q = fmaf(v1.x, r2, v0.x * r3);
    pe[0] = fmaf(dx, q, pe[0]);
    pe[1] = fmaf(dy, q, pe[1]);
    pe[2] = fmaf(dz, q, pe[2]);
    pe[0] = fmaf(-v1.y, ri, pe[0]);
    pe[1] = fmaf(-v1.z, ri, pe[1]);
    pe[2] = fmaf(-v1.w, ri, pe[2]);
    const float vx = fmaf(v1.y, r2, v0.y * r3);
    const float vy = fmaf(v1.z, r2, v0.z * r3);
    const float vz = fmaf(v1.w, r2, v0.w * r3);
    pb[0] = fmaf(vy, dz, pb[0]);
    pb[1] = fmaf(vz, dx, pb[1]);
    pb[2] = fmaf(vx, dy, pb[2]);
    pb[0] = fmaf(-vz, dy, pb[0]);
    pb[1] = fmaf(-vx, dz, pb[1]);
    pb[2] = fmaf(-vy, dx, pb[2]);
}

// Second-order retarded time: weight w = u - n of slot n+1, u = (T/dt - k0)
// - R/(c dt) (Eq. tr-1 without the floor), n relative to k0.  A + A_lo and
// K + K_lo carry T/dt - k0 and 1/(c dt) beyond FP32 and R gets one Newton
// correction, so the weight's error is a few roundings of numbers of order
// one rather than a rounding of u itself (a bias shared by every pair).
static __device__ __forceinline__ float interp_weight(float S, float ri, float nrel, float A, float A_lo, float K,
                                               float K_lo) {
    float R = S * ri;
    R = fmaf(0.5f * fmaf(-R, R, S), ri, R);
    const float t1 = fmaf(-R, K, A - nrel);   // A - nrel is exact
    const float t2 = fmaf(-R, K_lo, A_lo);
    return t1 + t2;
}

// (1 - w) a + w b for the 8 channels, packed.
static __device__ __forceinline__ void lerp8(float4& v0, float4& v1, const float4& u0, const float4& u1, float w) {
    const float2 w2 = make_float2(w, w), nw2 = make_float2(-w, -w);
    auto l = [&](float a0, float a1, float b0, float b1) {
        return __ffma2_rn(w2, make_float2(b0, b1), __ffma2_rn(nw2, make_float2(a0, a1), make_float2(a0, a1)));
    };
    const float2 p0 = l(v0.x, v0.y, u0.x, u0.y), p1 = l(v0.z, v0.w, u0.z, u0.w);
    const float2 p2 = l(v1.x, v1.y, u1.x, u1.y), p3 = l(v1.z, v1.w, u1.z, u1.w);
    v0 = make_float4(p0.x, p0.y, p1.x, p1.y);
    v1 = make_float4(p2.x, p2.y, p3.x, p3.y);
}

struct ThreadCtx {
    int slot;
    int rlo[3], rhi[3];   // screening index ranges
};

}  // namespace dev

}  // namespace jefi
