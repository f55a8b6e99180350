// jefi_host.cpp -- host side of libjefi: problem set-up, exact slot tables,
// validity checks and the C ABI declared in include/jefi.h.
//
// Built with -ffp-contract=off: the FP64 slot rule below must round every
// operation exactly as written (no fused multiply-add).
#include "jefi.h"

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "jefi_internal.h"

using namespace jefi;

namespace {

constexpr int kTimeChunk = 8;      // evaluation times per sum launch (base handles)
constexpr int kViewTimeChunk = 2;  // views keep scratch for fewer times
constexpr int kTablePad = 3;       // candidate-table margin on each side (slots)
constexpr double kSafety = 2.0;    // factor on the FP32 squared-distance error bound
constexpr int kMaxEventPairs = 4096;

// ---------------------------------------------------------------- exact FP64 rules
// Cell centre lo + (i + 0.5) d (product, then sum).
inline double center(double lo, double d, int64_t i) {
    double off = ((double)i + 0.5) * d;
    return lo + off;
}

// Retarded slot of Eq. tr-1 from the squared distance S; T = t - t0.
inline int64_t slot_of(double S, double T, double c, double dt) {
    double R = std::sqrt(S);
    double q = R / c;
    double u = (T - q) / dt;
    double f = std::floor(u);
    if (!(f > -4e18)) return INT64_MIN / 2;   // far past (or NaN): below any table
    if (!(f < 4e18)) return INT64_MAX / 2;
    return (int64_t)f;
}

inline double sq_sum(double sx, double sy, double sz) {
    double sxy = sx + sy;
    return sxy + sz;
}

// Largest S >= 0 with slot_of(S) >= k; -1 if none, +inf if every S.
double threshold(int64_t k, double T, double c, double dt) {
    if (slot_of(0.0, T, c, dt) < k) return -1.0;
    if (slot_of(DBL_MAX, T, c, dt) >= k) return INFINITY;
    auto bits = [](double x) { int64_t b; std::memcpy(&b, &x, 8); return b; };
    auto from = [](int64_t b) { double x; std::memcpy(&x, &b, 8); return x; };
    int64_t lo = 0, hi = bits(DBL_MAX);  // slot(lo) >= k, slot(hi) < k
    // narrow the bracket around the analytic boundary ((T - k dt) c)^2
    double g = (T - (double)k * dt) * c;
    if (g > 0 && std::isfinite(g * g)) {
        double s = g * g;
        for (double w = 1e-12; w < 1.0; w *= 1e3) {
            double a = s * (1.0 - w), b = s * (1.0 + w);
            if (!std::isfinite(b)) break;
            if (slot_of(a, T, c, dt) >= k && slot_of(b, T, c, dt) < k) {
                lo = bits(a);
                hi = bits(b);
                break;
            }
        }
    }
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (slot_of(from(mid), T, c, dt) >= k)
            lo = mid;
        else
            hi = mid;
    }
    return from(lo);
}

float round_down_f32(double x) {
    if (std::isnan(x)) return -INFINITY;
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, -INFINITY);
    return f;
}

float round_up_f32(double x) {
    if (std::isnan(x)) return INFINITY;
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}

struct AxisInfo {
    double far_sq, near_sq, near_out_sq;  // extremes of fl(D^2) along one axis
    int32_t rlo, rhi;                      // screening index range (rlo > rhi: empty)
};

// Per-axis extremes of one observation coordinate against source centres
// j in [0, nlim) (monotone: D(j) = xo - x_j is non-increasing in j).
AxisInfo axis_info(double xo, double lo, double d, int64_t org, int64_t nlim, int64_t npad, double delta) {
    AxisInfo r;
    auto D = [&](int64_t j) { return xo - center(lo, d, org + j); };
    // screening range over the padded index space [0, npad)
    int64_t a = 0, b = npad;  // first j with D(j) <= delta
    while (a < b) {
        int64_t m = (a + b) / 2;
        if (D(m) <= delta) b = m; else a = m + 1;
    }
    int64_t first = a;
    a = -1;
    b = npad - 1;  // last j with D(j) >= -delta
    while (a < b) {
        int64_t m = b - (b - a) / 2;
        if (D(m) >= -delta) a = m; else b = m - 1;
    }
    int64_t last = a;
    if (first <= last) {
        r.rlo = (int32_t)first;
        r.rhi = (int32_t)last;
    } else {
        r.rlo = INT32_MAX;
        r.rhi = INT32_MIN;
    }
    auto sq = [&](int64_t j) { double v = D(j); return v * v; };
    r.far_sq = std::max(sq(0), sq(nlim - 1));
    // nearest centre: first j with D(j) <= 0 and its left neighbour
    a = 0;
    b = nlim;
    while (a < b) {
        int64_t m = (a + b) / 2;
        if (D(m) <= 0) b = m; else a = m + 1;
    }
    r.near_sq = INFINITY;
    for (int64_t j = a - 1; j <= a; ++j)
        if (j >= 0 && j < nlim) r.near_sq = std::min(r.near_sq, sq(j));
    if (first > last) {
        r.near_out_sq = r.near_sq;
    } else {
        // nearest real index on each side of the screening range (the range
        // may lie partly or wholly outside [0, nlim))
        r.near_out_sq = INFINITY;
        const int64_t left = std::min(first - 1, nlim - 1);
        const int64_t right = std::max<int64_t>(last + 1, 0);
        if (left >= 0) r.near_out_sq = std::min(r.near_out_sq, sq(left));
        if (right < nlim) r.near_out_sq = std::min(r.near_out_sq, sq(right));
    }
    return r;
}

struct Extremes {
    double s_min = INFINITY;  // over unscreened pairs
    double s_max = -INFINITY;
};

void fold(Extremes& e, const AxisInfo (&ax)[3]) {
    double smax = sq_sum(ax[0].far_sq, ax[1].far_sq, ax[2].far_sq);
    double s0 = sq_sum(ax[0].near_out_sq, ax[1].near_sq, ax[2].near_sq);
    double s1 = sq_sum(ax[0].near_sq, ax[1].near_out_sq, ax[2].near_sq);
    double s2 = sq_sum(ax[0].near_sq, ax[1].near_sq, ax[2].near_out_sq);
    e.s_min = std::min(e.s_min, std::min(s0, std::min(s1, s2)));
    e.s_max = std::max(e.s_max, smax);
}

// Morton key of a point quantised to 21 bits per axis inside [lo, hi].
constexpr uint64_t kFnvBasis = 1469598103934665603ull;

// FNV-1a hash of n bytes, continuing from h.
uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

uint64_t morton(const double* p, const double* lo, const double* hi) {
    uint64_t key = 0;
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        double span = hi[a] - lo[a];
        double f = span > 0 ? (p[a] - lo[a]) / span : 0.0;
        f = std::min(std::max(f, 0.0), 1.0);
        q[a] = (uint32_t)(f * 2097151.0);
    }
    for (int bit = 20; bit >= 0; --bit)
        for (int a = 2; a >= 0; --a) key = (key << 1) | ((q[a] >> bit) & 1u);
    return key;
}

bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

// True when every observation coordinate, every (padded) source centre and the
// source spacing are integer multiples of one power of two q, small enough that
// the FP32 kernel's squared-distance chain (anchor offsets, brick offsets,
// differences, squares and their sums) is exact: then S32 == S64 for every pair.
bool exact_lattice(const std::vector<double>& obs_xyz, const jefi_grid& src, const int32_t* org, const int64_t* npad) {
    std::vector<double> vals(obs_xyz);
    double lo[3], hi[3], olo[3] = {INFINITY, INFINITY, INFINITY}, ohi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (size_t i = 0; i < obs_xyz.size(); ++i) {
        olo[i % 3] = std::min(olo[i % 3], obs_xyz[i]);
        ohi[i % 3] = std::max(ohi[i % 3], obs_xyz[i]);
    }
    for (int a = 0; a < 3; ++a) {
        vals.push_back(src.d[a]);
        for (int64_t j = 0; j < npad[a]; ++j) vals.push_back(center(src.lo[a], src.d[a], org[a] + j));
        lo[a] = center(src.lo[a], src.d[a], org[a]);
        hi[a] = center(src.lo[a], src.d[a], org[a] + npad[a] - 1);
    }
    int e = -40;
    for (; e <= 60; ++e) {
        bool ok = true;
        for (double v : vals) {
            const double w = std::ldexp(v, e);
            if (w != std::floor(w) || std::fabs(w) >= 1048576.0) { ok = false; break; }
        }
        if (ok) break;
    }
    if (e > 60) return false;
    // largest |D| along any axis, in units of q; three squares must fit 24 bits
    double m = 0;
    for (int a = 0; a < 3; ++a)
        m = std::max(m, std::max(std::fabs(ohi[a] - lo[a]), std::fabs(hi[a] - olo[a])));
    const double M = std::ldexp(m, e);
    return 3.0 * M * M < 16777216.0;
}

}  // namespace

// ============================================================================ handle
namespace {

// Centre O of the source grid, the farthest (brick-padded) cell centre from
// it, and the diagonal of one brick's cell centres: the source-side terms of
// the staged kernel's band bounds.
void source_shell(const jefi_grid& src, const int32_t* org, const int64_t* npad, double* O, double* r_src,
                  double* db) {
    double r2 = 0, d2 = 0;
    for (int a = 0; a < 3; ++a) {
        O[a] = src.lo[a] + (org[a] + 0.5 * src.n[a]) * src.d[a];
        const double far = std::max(std::fabs(center(src.lo[a], src.d[a], org[a]) - O[a]),
                                    std::fabs(center(src.lo[a], src.d[a], org[a] + npad[a] - 1) - O[a]));
        r2 += far * far;
        d2 += 9.0 * src.d[a] * src.d[a];
    }
    *r_src = std::sqrt(r2);
    *db = std::sqrt(d2);
}

// Widest pair-distance range over the tiles of `order` (256 entries per
// tile, -1 = padding): per tile the tighter of the box bound (the tile box's
// diagonal plus a brick's) and the shell bound (the range of the tile's
// distances from O plus twice the farthest source cell from O).
double tiles_extent(const std::vector<int64_t>& order, const double* pts, const double* O, double r_src, double db) {
    double ext_max = 0;
    for (size_t t0 = 0; t0 < order.size(); t0 += kTileThreads) {
        double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
        double rho_lo = INFINITY, rho_hi = 0;
        for (size_t s = t0; s < t0 + kTileThreads && s < order.size(); ++s) {
            if (order[s] < 0) continue;
            const double* x = pts + 3 * order[s];
            double r2 = 0;
            for (int a = 0; a < 3; ++a) {
                mn[a] = std::min(mn[a], x[a]);
                mx[a] = std::max(mx[a], x[a]);
                r2 += (x[a] - O[a]) * (x[a] - O[a]);
            }
            rho_lo = std::min(rho_lo, std::sqrt(r2));
            rho_hi = std::max(rho_hi, std::sqrt(r2));
        }
        if (!(rho_hi >= rho_lo)) continue;
        double d2 = 0;
        for (int a = 0; a < 3; ++a) d2 += (mx[a] - mn[a]) * (mx[a] - mn[a]);
        ext_max = std::max(ext_max, std::min(std::sqrt(d2) + db, (rho_hi - rho_lo) + 2 * r_src));
    }
    return ext_max;
}

// Tile shapes of observation grids (points per tile along x, y, z; each a
// whole number of 4x4x2-point warps, 256 points): index 1..8, 0 = chosen at
// creation.  A tile's warps are laid out x fastest, then y, then z.
constexpr int kTileShapes[9][3] = {{0, 0, 0}, {8, 8, 4}, {16, 4, 4}, {4, 8, 8}, {8, 4, 8},
                                   {4, 16, 4}, {16, 8, 2}, {8, 16, 2}, {4, 4, 16}};
constexpr int kNumTileShapes = 8;   // box shapes; JEFI_TILE_PACKED (9) is the packed tiling
constexpr int kTilePacked = 9;

// The widest pair-distance range over the tiles of shape s of an observation
// grid, from each tile's box alone (the box of a tile's points is known from
// its index ranges): the box bound as in tiles_extent, the shell bound with
// the box's nearest and farthest distances from O (never narrower than the
// points').  O(tiles): this only ranks the shapes.
double grid_tiles_extent(const jefi_grid& g, int s, const double* O, double r_src, double db) {
    const int64_t n[3] = {g.n[0], g.n[1], g.n[2]};
    int64_t t[3];
    for (int a = 0; a < 3; ++a) t[a] = (n[a] + kTileShapes[s][a] - 1) / kTileShapes[s][a];
    double ext_max = 0;
    for (int64_t tz = 0; tz < t[2]; ++tz)
        for (int64_t ty = 0; ty < t[1]; ++ty)
            for (int64_t tx = 0; tx < t[0]; ++tx) {
                const int64_t ti[3] = {tx, ty, tz};
                double d2 = 0, near2 = 0, far2 = 0;
                for (int a = 0; a < 3; ++a) {
                    const int64_t i0 = ti[a] * kTileShapes[s][a];
                    const int64_t i1 = std::min(i0 + kTileShapes[s][a], n[a]) - 1;
                    const double lo = center(g.lo[a], g.d[a], i0), hi = center(g.lo[a], g.d[a], i1);
                    d2 += (hi - lo) * (hi - lo);
                    const double nr = O[a] < lo ? lo - O[a] : (O[a] > hi ? O[a] - hi : 0.0);
                    const double fr = std::max(std::fabs(lo - O[a]), std::fabs(hi - O[a]));
                    near2 += nr * nr;
                    far2 += fr * fr;
                }
                ext_max = std::max(ext_max, std::min(std::sqrt(d2) + db,
                                                     std::sqrt(far2) - std::sqrt(near2) + 2 * r_src));
            }
    return ext_max;
}

// Observation order of a gx x gy x gz grid in tiles of shape s: tile slot ->
// point index (x fastest), -1 for padding.
void grid_tile_order(int64_t gx, int64_t gy, int64_t gz, int s, std::vector<int64_t>& order) {
    const int sx = kTileShapes[s][0], sy = kTileShapes[s][1], sz = kTileShapes[s][2];
    const int wx = sx / 4, wy = sy / 4;
    const int64_t tx = (gx + sx - 1) / sx, ty = (gy + sy - 1) / sy, tz = (gz + sz - 1) / sz;
    order.assign((size_t)(tx * ty * tz) * kTileThreads, -1);
    for (int64_t tile = 0; tile < tx * ty * tz; ++tile) {
        const int64_t bx = tile % tx, by = (tile / tx) % ty, bz = tile / (tx * ty);
        for (int tid = 0; tid < kTileThreads; ++tid) {
            const int w = tid >> 5, l = tid & 31;
            const int64_t i = sx * bx + 4 * (w % wx) + (l & 3);
            const int64_t j = sy * by + 4 * ((w / wx) % wy) + ((l >> 2) & 3);
            const int64_t k = sz * bz + 2 * (w / (wx * wy)) + (l >> 4);
            if (i < gx && j < gy && k < gz) order[tile * kTileThreads + tid] = (k * gy + j) * gx + i;
        }
    }
}

// Packed tiling of an observation grid (JEFI_TILE_PACKED): the grid cut
// into warp blocks of 4x4x2 points (every block holds at least one point),
// the blocks in Morton order of their block coordinates, eight consecutive
// blocks per tile (the last tile may hold fewer).  On grids whose sides are
// not multiples of a box shape this leaves far fewer padding lanes (which do
// a point's arithmetic too) than box tiles, at the price of less regular
// tiles where the Morton order turns.
void packed_tile_order(int64_t gx, int64_t gy, int64_t gz, std::vector<int64_t>& order) {
    const int64_t nbx = (gx + 3) / 4, nby = (gy + 3) / 4, nbz = (gz + 1) / 2;
    std::vector<std::pair<uint64_t, int64_t>> keys;
    keys.reserve((size_t)(nbx * nby * nbz));
    for (int64_t k = 0; k < nbz; ++k)
        for (int64_t j = 0; j < nby; ++j)
            for (int64_t i = 0; i < nbx; ++i) {
                const uint64_t q[3] = {(uint64_t)i, (uint64_t)j, (uint64_t)k};
                uint64_t key = 0;
                for (int bit = 20; bit >= 0; --bit)
                    for (int a = 2; a >= 0; --a) key = (key << 1) | ((q[a] >> bit) & 1u);
                keys.push_back({key, (k * nby + j) * nbx + i});
            }
    std::sort(keys.begin(), keys.end());
    const int64_t n_tiles = ((int64_t)keys.size() + 7) / 8;
    order.assign((size_t)n_tiles * kTileThreads, -1);
    for (size_t w = 0; w < keys.size(); ++w) {
        const int64_t b = keys[w].second;
        const int64_t bi = b % nbx, bj = (b / nbx) % nby, bk = b / (nbx * nby);
        for (int l = 0; l < 32; ++l) {
            const int64_t i = 4 * bi + (l & 3), j = 4 * bj + ((l >> 2) & 3), k = 2 * bk + (l >> 4);
            if (i < gx && j < gy && k < gz) order[w * 32 + l] = (k * gy + j) * gx + i;
        }
    }
}

// Relative time per (tile, brick) of the FP32 sum at a staged band height
// (0: the direct-gather kernel), measured on GB300 on wide-band problems;
// only ranks tilings of one problem against each other.
double band_cost(int band) {
    switch (band) {
        case 16: case 24: return 1.0;
        case 32: return 1.2;
        case 48: return 1.3;
        case 64: return 1.5;
        case 96: return 1.8;
        default: return 3.0;
    }
}

// The staged band height a widest pair-distance range `ext` needs (0 if
// none fits, or none within `max_band`).
int band_for_extent(double ext, double Kd, int max_band) {
    const double need = std::ceil(ext * Kd * (1 + 1e-4) + 1e-3) + 7;
    for (int b : kStagedBands)
        if (need <= b) return b <= max_band ? b : 0;
    return 0;
}

}  // namespace

struct jefi_problem {
    jefi_params prm{};
    jefi_grid src{};
    bool fp64 = false;
    int32_t nbx = 0, nby = 0, nbz = 0, n_bricks = 0, npx = 0, npy = 0, npz = 0;
    int64_t n_src = 0, n_obs = 0;
    int32_t n_slots = 0, n_tiles = 0;
    int32_t H = 0, Hp = 0;
    int32_t P = 0;                   // ring period: H rounded up to a multiple of 4
    int32_t org[3] = {0, 0, 0};      // first source cell in the source lattice (jefi_params.src_origin)
    int32_t tile_shape = 0;          // observation-grid tile shape (kTileShapes index; 0: point list)
    uint64_t obs_sig = 0;            // hash of the observation points in tile order (tune cache key)
    double screen[3] = {0, 0, 0};
    int64_t n_latest = -1;
    int32_t n_split = 1, bricks_per_split = 0;
    int32_t n_split_max = 1;         // splits the partials buffer was sized for (creation)
    int32_t K = 0;                 // candidate-table length per time
    // exact squared-distance extremes over unscreened pairs
    Extremes real, pad;
    bool any_pairs = false;
    // FP32 error model: |S32 - S64| <= err_rel*S + err_lin*sqrt(S) + err_abs
    double err_rel = 0, err_lin = 0, err_abs = 0;
    // host tables
    std::vector<int32_t> inv_perm;   // observation -> tile slot
    std::vector<int32_t> slot_obs;   // tile slot -> observation (-1: padding)
    // device memory
    void* ring = nullptr;
    double* obs_xyz = nullptr;
    float* obs_hl = nullptr;         // FP32: per slot the point as FP32 pairs (x hi, x lo, y hi, ...)
    float2* cc_hl = nullptr;         // FP32: padded cell centres per axis as FP32 pairs (x, y, z)
    float df_b1 = 0.f, df_b2 = 0.f;  // FP32: bound on |S_df - S64| (slot_double_float)
    std::vector<float> h_obs_hl;
    std::vector<float2> h_cc_hl;
    int32_t* obs_scr = nullptr;
    int32_t* d_inv_perm = nullptr;
    double* prev = nullptr;
    double* prev2 = nullptr;         // slice n-2 (central differences only)
    double* stage_in = nullptr;      // host pushes: rho, J, drho, dJ
    // second-order retarded time (JEFI_FLAG_INTERP); central: the ring's
    // derivative channels hold central differences, written one slice late
    bool interp = false, central = false;
    int32_t time_chunk = kTimeChunk; // evaluation times per launch (scratch slots)
    double* partials = nullptr;      // [time_chunk][n_split][6][n_slots]
    double* out_stage = nullptr;     // host outputs: E, B for time_chunk times
    float4* tab32 = nullptr;
    double* theta = nullptr;
    TimeParams* times = nullptr;
    unsigned long long* fallbacks = nullptr;
    std::vector<std::pair<void*, size_t>> allocs;
    int64_t device_bytes = 0;
    // host staging for the per-eval tables
    std::vector<float4> h_tab;
    std::vector<double> h_theta;
    std::vector<TimeParams> h_times;
    // staged FP32 kernel (0 = direct-gather kernel)
    int32_t band = 0;
    int32_t band0 = 0;               // the staged band chosen at creation (0: none)
    int32_t band_alt = 0;            // the next wider compiled band the ring's mirror allows (0: none)
    int32_t tmap_band = 0;           // the band the tensor map was encoded for
    int32_t mirror = 0;              // M: mirrored ring slots
    bool exact = false;              // lattice geometry: S32 == S64
    double g_bias = 0;               // bound on the FP32 candidate error (slots)
    float* tile_box = nullptr;
    float2* tab2 = nullptr;
    std::vector<float2> h_tab2;
    float2* tabg = nullptr;          // direct-gather kernel: T_lo and packed slots per candidate
    float* tabh = nullptr;           // direct-gather kernel: T_hi per candidate
    std::vector<float2> h_tabg;
    std::vector<float> h_tabh;
    alignas(64) CUtensorMap tmap;
    int32_t* status = nullptr;
    // observation views share a base handle's ring and pushes
    jefi_problem* base = nullptr;
    int32_t n_views = 0;
    int32_t n_plans = 0;             // live batch plans holding this handle
    // completion of the latest work enqueued on this handle's memory (any stream)
    cudaEvent_t last_use = nullptr;
    // statistics
    int64_t launches = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending, ev_free;
    int64_t sum_launches = 0;
    double sum_ms = 0;
};

namespace {

// A named NVTX range around one C-ABI call (profiler timelines, ncu --nvtx
// filters); a no-op unless a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

#define JEFI_CUDA(x)                                     \
    do {                                                 \
        cudaError_t _e = (x);                            \
        if (_e != cudaSuccess) return JEFI_ECUDA;        \
    } while (0)

void* dev_alloc(jefi_problem* h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (h->prm.alloc) {
        p = h->prm.alloc(bytes, h->prm.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        h->allocs.emplace_back(p, bytes);
        h->device_bytes += (int64_t)bytes;
    }
    return p;
}

void release_all(jefi_problem* h) {
    for (auto& a : h->allocs) {
        if (h->prm.free)
            h->prm.free(a.first, h->prm.alloc_ctx);
        else
            cudaFree(a.first);
    }
    h->allocs.clear();
    if (h->last_use) cudaEventDestroy(h->last_use);
    h->last_use = nullptr;
    for (auto& e : h->ev_pending) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    for (auto& e : h->ev_free) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    h->ev_pending.clear();
    h->ev_free.clear();
}

// Device and host tables of the direct-gather kernel; false if out of memory.
bool alloc_direct_tables(jefi_problem* h) {
    if (h->tabg) return true;
    const size_t n = (size_t)h->time_chunk * (h->K + 2 * kTabGuard);
    float2* g = (float2*)dev_alloc(h, sizeof(float2) * n);
    float* t = g ? (float*)dev_alloc(h, sizeof(float) * n) : nullptr;
    if (!g || !t) return false;
    h->tabg = g;
    h->tabh = t;
    h->h_tabg.resize(n);
    h->h_tabh.resize(n);
    return true;
}

// SM count of the current device (the work split targets whole waves of
// CTAs).  Without a device the query fails and 1 is returned: such a
// creation fails at its first device call anyway.
int current_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n < 1) {
        cudaGetLastError();
        return 1;
    }
    return n;
}

// CTAs of a staged sum kernel resident at once: two per SM while two
// fit the SM's shared memory (228 KB, 1 KB of it reserved per CTA).
int64_t staged_resident_ctas(size_t smem_bytes) {
    const int64_t per_sm = std::min<int64_t>(2, (int64_t)(233472 / (smem_bytes + 1024)));
    return std::max<int64_t>(1, per_sm) * current_sm_count();
}

// Consecutive source splits one staged work item sums in a single-problem
// launch of `units` (tile, time) pairs.  Items of equal work run in waves of
// the resident CTAs; the merge is the one with the least predicted time:
// waves x (bricks per item + a preamble of about half a brick's work).  The
// partials are those of one item per split whatever the value, so it changes
// the cost of a launch (its items' preambles and first copies, its last
// wave), never its result.  Only the least merge of each item count is a
// candidate (a larger one with as many items costs more), so the search
// takes O(sqrt(n_split)) steps.  `cost`, if given, receives the prediction.
int32_t split_merge_for(int64_t units, int32_t n_split, int32_t bricks_per_split, int64_t resident,
                        double* cost = nullptr) {
    const int64_t n = std::max(n_split, 1);
    const int64_t r = std::max<int64_t>(resident, 1);
    double best = 0.0;
    int32_t best_m = 1;
    for (int64_t m = 1; m <= n;) {
        const int64_t q = (n + m - 1) / m;   // items per (tile, time)
        const int64_t waves = (units * q + r - 1) / r;
        const double c = (double)waves * ((double)m * bricks_per_split + 0.5);
        if (m == 1 || c < best) {
            best = c;
            best_m = (int32_t)m;
        }
        if (q == 1) break;
        m = (n + q - 2) / (q - 1);   // least merge with fewer items
    }
    if (cost) *cost = best;
    return best_m;
}

// Source splits of a staged handle with n_tiles tiles over n_bricks bricks,
// at most ns_max: the count whose launches of 1, 2, 4, ... time_chunk
// evaluation times fill their waves best (split_merge_for's prediction over
// the ideal units x bricks / resident), the fewest splits among equals.
// Whole waves of equal items matter most where the units are few: a view of
// 128 tiles over 4096 bricks (at most 10 splits) at one time runs 3 waves of
// 7 splits, 98 % full, where 10 splits ran as 2 groups of 5 in one wave 84 %
// full.
int64_t split_count_for(int64_t n_tiles, int64_t n_bricks, int64_t ns_max, int32_t time_chunk,
                        int64_t resident) {
    const int64_t nb = std::max<int64_t>(n_bricks, 1);
    const int64_t nt = std::max<int64_t>(n_tiles, 1);
    ns_max = std::max<int64_t>(1, std::min(ns_max, nb));
    double best = 0.0;
    int64_t best_ns = 1;
    for (int64_t ns = 1; ns <= ns_max; ++ns) {
        const int64_t bps = (nb + ns - 1) / ns;
        if ((nb + bps - 1) / bps != ns) continue;   // the same splits as a smaller count
        double score = 0.0;
        int n_launch = 0;
        for (int32_t t = 1;; t = std::min(2 * t, time_chunk)) {
            double c = 0.0;
            split_merge_for(nt * t, (int32_t)ns, (int32_t)bps, resident, &c);
            score += c / ((double)(nt * t) * (double)nb / (double)std::max<int64_t>(resident, 1));
            ++n_launch;
            if (t >= time_chunk) break;
        }
        score /= n_launch;
        if (ns == 1 || score < best - 1e-9) {
            best = score;
            best_ns = ns;
        }
    }
    return best_ns;
}

// Record that work on h's memory was enqueued on stream s (jefi_destroy waits for it).
int mark_use(jefi_problem* h, cudaStream_t s) {
    if (!h->last_use) JEFI_CUDA(cudaEventCreateWithFlags(&h->last_use, cudaEventDisableTiming));
    JEFI_CUDA(cudaEventRecord(h->last_use, s));
    return JEFI_OK;
}

int64_t phys_slot(const jefi_problem* h, int64_t k) {
    if (k < 0 || k > h->n_latest || k < h->n_latest - h->H + 1) return h->P + h->mirror;  // zero slot
    return k % h->P;
}

// Slices past a pair's slot n that an evaluation reads: 0 (floor rule),
// 1 (interpolation), 2 (interpolation of central differences).
int64_t slices_ahead(const jefi_problem* h) { return h->interp ? (h->central ? 2 : 1) : 0; }

// Range of slots [n_lo, n_hi] needed at time t by real unscreened pairs.
void needed_range(const jefi_problem* h, double T, int64_t* n_lo, int64_t* n_hi) {
    *n_lo = slot_of(h->real.s_max, T, h->prm.c, h->prm.dt);
    *n_hi = slot_of(h->real.s_min, T, h->prm.c, h->prm.dt);
}

int check_time(const jefi_problem* h, double t) {
    if (!std::isfinite(t)) return JEFI_EINVAL;
    if (!h->any_pairs) return JEFI_OK;
    const double T = t - h->prm.t0;
    const double c = h->prm.c, dt = h->prm.dt;
    // |u| must stay well inside int64 and the FP32 candidate range
    const double umax = (std::fabs(T) + std::sqrt(h->pad.s_max) / c) / dt;
    if (!(umax < 1e15)) return JEFI_EUNSUPPORTED;
    int64_t lo, hi;
    needed_range(h, T, &lo, &hi);
    // interpolation also reads slice n+1, and n+2 through a central difference
    const int64_t ahead = slices_ahead(h);
    if (hi + (h->interp ? 1 : 0) < 0) return JEFI_OK;   // all sources still in the future
    if (hi + ahead > h->n_latest) return JEFI_ENOTYET;
    const int64_t oldest = h->n_latest - h->H + 1;
    if (std::max<int64_t>(lo, 0) < oldest) return JEFI_EEVICTED;
    return JEFI_OK;
}

// Build the candidate tables of one evaluation time into slot ti of the staging arrays.
void build_tables(jefi_problem* h, int ti, double t) {
    const double T = t - h->prm.t0;
    const double c = h->prm.c, dt = h->prm.dt;
    const int64_t n_lo = slot_of(h->pad.s_max, T, c, dt);
    const int64_t k0 = n_lo - kTablePad;
    const int K = h->K;
    double* th = h->h_theta.data() + (size_t)ti * theta_stride(K);
    for (int i = 0; i <= K; ++i) th[i] = threshold(k0 + i, T, c, dt);
    // the same thresholds as FP32 pairs: hi = the nearest float, lo = the
    // nearest float to the (exact) remainder
    float2* thl = reinterpret_cast<float2*>(th + K + 1);
    for (int i = 0; i <= K; ++i) {
        const double v = th[i];
        if (!std::isfinite(v)) {
            thl[i] = make_float2((float)v, 0.f);
        } else {
            const float hi = (float)v;
            thl[i] = make_float2(hi, std::isfinite(hi) ? (float)(v - (double)hi) : 0.f);
        }
    }
    float4* tab = h->h_tab.data() + (size_t)ti * K;
    auto err = [&](double S) { return h->err_rel * S + h->err_lin * std::sqrt(S) + h->err_abs; };
    for (int i = 0; i < K; ++i) {
        const double hi_t = th[i], lo_t = th[i + 1];
        float hi, lo;
        if (hi_t < 0) hi = -INFINITY;
        else if (std::isinf(hi_t)) hi = INFINITY;
        else hi = round_down_f32(hi_t - err(hi_t));
        if (lo_t < 0) lo = -INFINITY;
        else if (std::isinf(lo_t)) lo = INFINITY;
        else lo = round_up_f32(lo_t + err(lo_t));
        int32_t ps = (int32_t)phys_slot(h, k0 + i);
        float psf;
        std::memcpy(&psf, &ps, 4);
        tab[i] = make_float4(hi, lo, psf, 0.f);
    }
    if (h->band > 0) {
        // staged kernel: (T_hi, T_lo) of Theta_k for k = k0 - guard ... k0 + K + guard - 1
        const int KT = K + 2 * kTabGuard;
        float2* t2 = h->h_tab2.data() + (size_t)ti * KT;
        for (int e = 0; e < KT; ++e) {
            const int i = e - kTabGuard;
            if (i < 0 || i >= K) {
                t2[e] = make_float2(-INFINITY, INFINITY);   // never reached; undecided if it were
                continue;
            }
            const double th_k = th[i];
            float thi, tlo;
            if (th_k < 0) thi = tlo = -INFINITY;
            else if (std::isinf(th_k)) thi = tlo = INFINITY;
            else if (h->exact) thi = tlo = round_down_f32(th_k);
            else {
                thi = round_down_f32(th_k - err(th_k));
                tlo = round_up_f32(th_k + err(th_k));
            }
            t2[e] = make_float2(thi, tlo);
        }
    }
    if (h->tabg && h->band == 0) {
        // direct-gather kernel: (T_hi, T_lo) of Theta_k' and the physical slots of k', k'-1
        const int KT = K + 2 * kTabGuard;
        float2* tg = h->h_tabg.data() + (size_t)ti * KT;
        float* th_hi = h->h_tabh.data() + (size_t)ti * KT;
        auto slot_pair = [&](int64_t k) {   // physical slots of k (low half) and k-1 (high half)
            const uint32_t pk = (uint32_t)phys_slot(h, k), pm = (uint32_t)phys_slot(h, k - 1);
            const uint32_t packed = (pk & 0xFFFFu) | (pm << 16);
            float f;
            std::memcpy(&f, &packed, 4);
            return f;
        };
        for (int e = 0; e < KT; ++e) {
            const int i = e - kTabGuard;
            const float zw = slot_pair(k0 + i);
            if (i < 0 || i >= K) {
                tg[e] = make_float2(INFINITY, zw);   // never reached; undecided if it were
                th_hi[e] = -INFINITY;
                continue;
            }
            const double th_k = th[i];
            float thi, tlo;
            if (th_k < 0) thi = tlo = -INFINITY;
            else if (std::isinf(th_k)) thi = tlo = INFINITY;
            else if (h->exact) thi = tlo = round_down_f32(th_k);
            else {
                thi = round_down_f32(th_k - err(th_k));
                tlo = round_up_f32(th_k + err(th_k));
            }
            tg[e] = make_float2(tlo, zw);
            th_hi[e] = thi;
        }
    }
    TimeParams tp;
    const double A = T / dt - (double)k0;
    tp.A = (float)A;
    const double w_max = std::sqrt(h->pad.s_max) / (c * dt);
    tp.Ag = (float)(A + h->g_bias + 8 * std::ldexp(1.0, -53) * (std::fabs(T / dt) + w_max + 1));
    // Before the ring wraps, pairs may need slots < 0 (sources not yet on):
    // the band may then start below 0 and read zeros there.  Once slices have
    // been evicted, no valid pair needs a slot older than the oldest resident.
    const int64_t oldest = h->n_latest - h->H + 1;
    const int64_t oldest_rel = oldest > 0 ? oldest - k0 : (int64_t)(INT32_MIN / 2);
    tp.oldest_rel = (int32_t)std::max<int64_t>(std::min<int64_t>(oldest_rel, INT32_MAX / 2), INT32_MIN / 2);
    tp.A_lo = (float)(A - (double)tp.A);
    tp.k0 = k0;
    tp.k0_mod = (int32_t)(((k0 % h->P) + h->P) % h->P);
    tp.pad = 0;
    tp.A64 = A;
    h->h_times[ti] = tp;
}

// TMA descriptor over the FP32 ring [cells][Hp][8]: box = 8 channels x band
// slots x the stage's cells.  Wide bands use the 32-byte swizzle, whose span
// is the box's inner extent (one 32-byte row), so the box lands densely.
// Before any launch the box is checked against the stage buffer it lands
// in: the bytes it writes must equal the buffer's size (the kernel waits for
// exactly that many) and a swizzled box's inner extent must be the full
// 32-byte swizzle span.  JEFI_EINTERNAL otherwise.
int make_tensor_map(jefi_problem* h) {
    const bool swz = staged_swizzled(h->band);
    const cuuint32_t box_inner = 8;                                 // floats: one row
    const cuuint32_t box_rows = (cuuint32_t)h->band;
    const cuuint32_t box_cells = (cuuint32_t)staged_stage_cells(h->band);
    const size_t landed = (size_t)box_inner * sizeof(float) * box_rows * box_cells;
    if (landed != staged_buffer_bytes(h->band) || (swz && box_inner * sizeof(float) != 32) || box_rows > 256 ||
        box_cells > 256)
        return JEFI_EINTERNAL;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || fn == nullptr || q != cudaDriverEntryPointSuccess)
        return JEFI_ECUDA;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const cuuint64_t dims[3] = {box_inner, (cuuint64_t)h->Hp, (cuuint64_t)h->n_bricks * kBrickCells};
    const cuuint64_t strides[2] = {box_inner * sizeof(float), (cuuint64_t)h->Hp * 8 * sizeof(float)};
    const cuuint32_t box[3] = {box_inner, box_rows, box_cells};
    const cuuint32_t elem[3] = {1, 1, 1};
    const CUresult r = encode(&h->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->ring, dims, strides, box, elem,
                              CU_TENSOR_MAP_INTERLEAVE_NONE,
                              swz ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return JEFI_ECUDA;
    h->tmap_band = h->band;
    return JEFI_OK;
}

// Switch h's FP32 sum kernel: 0 = the direct gather, else a staged band
// (the creation band or the wider alternative), re-encoding the tensor map
// for a band it was not encoded for.
int set_band(jefi_problem* h, int32_t b) {
    const int32_t old = h->band;
    h->band = b;
    if (b > 0 && b != h->tmap_band) {
        const int rc = make_tensor_map(h);
        if (rc != JEFI_OK) {
            h->band = old;
            return rc;
        }
    }
    return JEFI_OK;
}

// Kernel parameters of handle h for n_t evaluation times whose tables sit in
// table slots [slot0, slot0 + n_t) of the handle's device buffers.
SumParams make_params(const jefi_problem* h, int n_t, int slot0, int32_t* debug_slots) {
    const int K = h->K;
    SumParams p{};
    p.nbx = h->nbx; p.nby = h->nby; p.nbz = h->nbz; p.n_bricks = h->n_bricks;
    for (int a = 0; a < 3; ++a) p.org[a] = h->org[a];
    p.npx = h->npx; p.npy = h->npy; p.npz = h->npz;
    for (int a = 0; a < 3; ++a) {
        p.lo[a] = h->src.lo[a];
        p.d[a] = h->src.d[a];
        p.d32[a] = (float)h->src.d[a];
    }
    p.n_slots = h->n_slots;
    p.n_tiles = h->n_tiles;
    p.obs_xyz = h->obs_xyz;
    p.obs_hl = h->obs_hl;
    p.cc_hl = h->cc_hl;
    p.df_b1 = h->df_b1;
    p.df_b2 = h->df_b2;
    p.pad_yz = (h->src.n[1] % kBrick != 0 || h->src.n[2] % kBrick != 0) ? 1 : 0;
    p.obs_scr = h->obs_scr;
    p.ring = h->ring;
    p.Hp = h->Hp;
    p.zero_slot = h->P + h->mirror;
    p.H = h->P;
    p.status = h->status;
    p.tab2 = h->tab2 ? h->tab2 + (size_t)slot0 * (K + 2 * kTabGuard) : nullptr;
    p.tabg = h->tabg ? h->tabg + (size_t)slot0 * (K + 2 * kTabGuard) : nullptr;
    p.tabh = h->tabh ? h->tabh + (size_t)slot0 * (K + 2 * kTabGuard) : nullptr;
    p.exact = h->exact ? 1 : 0;
    p.tile_box = h->tile_box;
    for (int a = 0; a < 3; ++a) {
        p.n_src_axis[a] = h->src.n[a];
        p.nfull[a] = h->src.n[a] / kBrick;
    }
    p.tab32 = h->tab32 + (size_t)slot0 * K;
    p.theta = h->theta + (size_t)slot0 * theta_stride(K);
    p.times = h->times + slot0;
    p.n_t = n_t;
    p.K = K;
    p.K32 = (float)(1.0 / (h->prm.c * h->prm.dt));
    p.K64 = 1.0 / (h->prm.c * h->prm.dt);
    p.K32_lo = (float)(p.K64 - (double)p.K32);
    p.interp = h->interp ? 1 : 0;
    p.n_split = h->n_split;
    p.bricks_per_split = h->bricks_per_split;
    p.split_merge = 1;
    p.partials = h->partials + (size_t)slot0 * h->n_split * 6 * h->n_slots;
    p.fallbacks = h->fallbacks;
    p.debug_slots = debug_slots;
    p.comp = h->prm.precision == JEFI_FP32_COMP ? 1 : 0;
    return p;
}

// Upload the tables built in host slots [0, n_t) to the device.
int upload_tables(jefi_problem* h, int n_t, cudaStream_t s) {
    const int K = h->K;
    JEFI_CUDA(cudaMemcpyAsync(h->tab32, h->h_tab.data(), sizeof(float4) * K * n_t,
                              cudaMemcpyHostToDevice, s));
    JEFI_CUDA(cudaMemcpyAsync(h->theta, h->h_theta.data(), sizeof(double) * theta_stride(K) * n_t,
                              cudaMemcpyHostToDevice, s));
    JEFI_CUDA(cudaMemcpyAsync(h->times, h->h_times.data(), sizeof(TimeParams) * n_t,
                              cudaMemcpyHostToDevice, s));
    if (h->band > 0)
        JEFI_CUDA(cudaMemcpyAsync(h->tab2, h->h_tab2.data(),
                                  sizeof(float2) * (K + 2 * kTabGuard) * n_t, cudaMemcpyHostToDevice, s));
    if (h->tabg && h->band == 0) {
        JEFI_CUDA(cudaMemcpyAsync(h->tabg, h->h_tabg.data(),
                                  sizeof(float2) * (K + 2 * kTabGuard) * n_t, cudaMemcpyHostToDevice, s));
        JEFI_CUDA(cudaMemcpyAsync(h->tabh, h->h_tabh.data(),
                                  sizeof(float) * (K + 2 * kTabGuard) * n_t, cudaMemcpyHostToDevice, s));
    }
    return JEFI_OK;
}

int launch_chunk(jefi_problem* h, int n_t, const double* t, double* E, double* B, cudaStream_t s,
                 int32_t* debug_slots) {
    for (int i = 0; i < n_t; ++i) build_tables(h, i, t[i]);
    {
        const int rc = upload_tables(h, n_t, s);
        if (rc != JEFI_OK) return rc;
    }
    SumParams p = make_params(h, n_t, 0, debug_slots);
    if (h->band == 0 && sum_smem_bytes(p) > 200 * 1024) return JEFI_EUNSUPPORTED;
    if (h->band > 0)
        p.split_merge = split_merge_for((int64_t)h->n_tiles * n_t, h->n_split, h->bricks_per_split,
                                        staged_resident_ctas(staged_smem_bytes(p, h->band, false)));

    const bool timed = (h->prm.flags & JEFI_FLAG_STATS) != 0 && !debug_slots;
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (timed && (int)h->ev_pending.size() < kMaxEventPairs) {
        if (!h->ev_free.empty()) {
            ev = h->ev_free.back();
            h->ev_free.pop_back();
        } else {
            JEFI_CUDA(cudaEventCreate(&ev.first));
            JEFI_CUDA(cudaEventCreate(&ev.second));
        }
        JEFI_CUDA(cudaEventRecord(ev.first, s));
    }
    cudaError_t e;
    if (h->fp64) {
        e = launch_sum_f64(p, s);
    } else if (h->band > 0) {
        StagedConfig sc;
        sc.band = h->band;
        sc.exact = h->exact;
        sc.compensated = h->prm.precision == JEFI_FP32_COMP;
        sc.tensor_map = &h->tmap;
        e = launch_sum_f32_staged(p, sc, s);
    } else {
        e = launch_sum_f32(p, h->prm.precision == JEFI_FP32_COMP, s);
    }
    if (e != cudaSuccess) return JEFI_ECUDA;
    h->launches++;
    if (ev.first) {
        JEFI_CUDA(cudaEventRecord(ev.second, s));
        h->ev_pending.push_back(ev);
    }
    if (debug_slots) return JEFI_OK;
    ReduceParams r{};
    r.n_obs = (int32_t)h->n_obs;
    r.n_slots = h->n_slots;
    r.n_split = h->n_split;
    r.n_t = n_t;
    r.inv_perm = h->d_inv_perm;
    r.partials = h->partials;
    r.e_scale = h->prm.k_e * (h->src.d[0] * h->src.d[1] * h->src.d[2]) / h->prm.c;
    r.b_scale = h->prm.k_b * (h->src.d[0] * h->src.d[1] * h->src.d[2]);
    r.E = E;
    r.B = B;
    JEFI_CUDA(launch_reduce(r, s));
    h->launches++;
    return JEFI_OK;
}

// ---------------------------------------------------------------- batched launches
// Device memory for the metadata of batched launches, one arena per device.
// A batch waits (on its stream) for the previous batch that used the arena
// before overwriting it.
struct BatchArena {
    std::mutex lock;
    void* dev = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    int n_sm = 0;
};
std::mutex g_arena_lock;
std::map<std::pair<int, cudaStream_t>, BatchArena*> g_arenas;   // per (device, stream)

BatchArena& arena_for(int dev, cudaStream_t s) {
    std::lock_guard<std::mutex> guard(g_arena_lock);
    BatchArena*& a = g_arenas[{dev, s}];
    if (!a) a = new BatchArena();
    return *a;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int arena_reserve(BatchArena& a, size_t bytes) {
    if (!a.done) {
        JEFI_CUDA(cudaEventCreateWithFlags(&a.done, cudaEventDisableTiming));
        int dev = 0;
        JEFI_CUDA(cudaGetDevice(&dev));
        JEFI_CUDA(cudaDeviceGetAttribute(&a.n_sm, cudaDevAttrMultiProcessorCount, dev));
    }
    if (a.cap >= bytes) return JEFI_OK;
    if (a.dev) {
        JEFI_CUDA(cudaEventSynchronize(a.done));
        cudaFree(a.dev);
        a.dev = nullptr;
        a.cap = 0;
    }
    const size_t cap = std::max<size_t>(bytes, 1 << 20);
    if (cudaMalloc(&a.dev, cap) != cudaSuccess) {
        cudaGetLastError();
        a.dev = nullptr;
        return JEFI_ENOMEM;
    }
    a.cap = cap;
    return JEFI_OK;
}

// ---------------------------------------------------------------- batch layout
// Shared by jefi_eval_batch and batch plans: the problems of a batch grouped
// by kernel variant (one persistent launch per group), their reduction
// items, and the byte layout of the launch metadata.
struct BatchGroup {
    int kind;           // 0 FP64, 1 FP32 direct, 2 FP32 staged
    int comp, band;
    bool exact;
    std::vector<int> members;
};

struct BatchLayout {
    std::vector<BatchGroup> groups;
    std::vector<ReduceItem> ritems;
    std::vector<int64_t> rstart;
    std::vector<int> zero_entries;      // entries with points but no pairs: zero fields
    // per group [params | item_start | counter], then [reduce items | starts]
    std::vector<size_t> off_params, off_start, off_counter;
    size_t off_ritems = 0, off_rstart = 0, bytes = 0;
    // filled by batch_fill
    std::vector<int> n_items;
    std::vector<size_t> smem;
};

// Group entries i (handle hs[i], scratch slot occ[i], outputs E[i], B[i]) and
// lay out the metadata from byte 0, 256-byte aligned.
void batch_layout(jefi_problem* const* hs, const int* occ, double* const* E, double* const* B, int n,
                  BatchLayout* L) {
    L->groups.clear();
    L->ritems.clear();
    L->rstart.assign(1, 0);
    L->zero_entries.clear();
    for (int i = 0; i < n; ++i) {
        jefi_problem* h = hs[i];
        if (h->n_obs == 0) continue;
        if (!h->any_pairs) {
            L->zero_entries.push_back(i);
            continue;
        }
        BatchGroup key{h->fp64 ? 0 : (h->band > 0 ? 2 : 1), h->prm.precision == JEFI_FP32_COMP ? 1 : 0, h->band,
                       h->exact, {}};
        if (key.kind != 1) key.comp = 0;
        if (key.kind != 2) { key.band = 0; key.exact = false; }
        BatchGroup* g = nullptr;
        for (auto& x : L->groups)
            if (x.kind == key.kind && x.comp == key.comp && x.band == key.band && x.exact == key.exact &&
                (x.kind != 2 || (int)x.members.size() < kMaxBatchMaps))
                g = &x;
        if (!g) {
            L->groups.push_back(key);
            g = &L->groups.back();
        }
        g->members.push_back(i);
        ReduceItem r{};
        r.inv_perm = h->d_inv_perm;
        r.partials = h->partials + (size_t)occ[i] * h->n_split * 6 * h->n_slots;
        r.n_obs = (int32_t)h->n_obs;
        r.n_slots = h->n_slots;
        r.n_split = h->n_split;
        r.e_scale = h->prm.k_e * (h->src.d[0] * h->src.d[1] * h->src.d[2]) / h->prm.c;
        r.b_scale = h->prm.k_b * (h->src.d[0] * h->src.d[1] * h->src.d[2]);
        r.E = E[i];
        r.B = B[i];
        L->ritems.push_back(r);
        L->rstart.push_back(L->rstart.back() + h->n_obs);
    }
    const size_t ng = L->groups.size();
    L->off_params.resize(ng);
    L->off_start.resize(ng);
    L->off_counter.resize(ng);
    size_t bytes = 0;
    for (size_t g = 0; g < ng; ++g) {
        L->off_params[g] = bytes;
        bytes = align256(bytes + sizeof(SumParams) * L->groups[g].members.size());
        L->off_start[g] = bytes;
        bytes = align256(bytes + sizeof(int32_t) * (L->groups[g].members.size() + 1));
        L->off_counter[g] = bytes;
        bytes = align256(bytes + sizeof(unsigned int));
    }
    L->off_ritems = bytes;
    bytes = align256(bytes + sizeof(ReduceItem) * L->ritems.size());
    L->off_rstart = bytes;
    bytes = align256(bytes + sizeof(int64_t) * L->rstart.size());
    L->bytes = bytes;
}

// Write the metadata into the host image `host` (zeroed by the caller, so
// the queue counters start at zero): kernel parameters of every member
// (params(i) gives entry i's), work-item starts, reduction items; record
// per group its item count and shared memory.  JEFI_EUNSUPPORTED if a
// group needs more shared memory than a block may have.
template <class Params>
int batch_fill(BatchLayout* L, unsigned char* host, Params&& params) {
    const size_t ng = L->groups.size();
    L->n_items.assign(ng, 0);
    L->smem.assign(ng, 0);
    for (size_t g = 0; g < ng; ++g) {
        BatchGroup& G = L->groups[g];
        SumParams* prm = reinterpret_cast<SumParams*>(host + L->off_params[g]);
        int32_t* start = reinterpret_cast<int32_t*>(host + L->off_start[g]);
        const size_t nm = G.members.size();
        std::vector<SumParams> par(nm);
        for (size_t m = 0; m < nm; ++m) {
            par[m] = params(G.members[m]);
            L->smem[g] = std::max(L->smem[g], G.kind == 2 ? staged_smem_bytes(par[m], G.band, true)
                                                            : sum_smem_bytes(par[m]));
        }
        if (G.kind == 2) {
            // Staged items merge a member's splits up to about an equal share
            // of the group's work (4 waves of the resident CTAs; never finer
            // than the member's own splits), and the members are queued by
            // item work, largest first: the queue's last items, which set the
            // launch's tail, are its smallest.  Neither changes a result
            // (each split's partials are written as one item per split would).
            int64_t work = 0;   // (tile, brick) units of the group
            for (size_t m = 0; m < nm; ++m) work += (int64_t)par[m].n_tiles * par[m].n_bricks;
            const int64_t per_item = std::max<int64_t>(1, work / (4 * staged_resident_ctas(L->smem[g])));
            std::vector<int64_t> item_work(nm);
            for (size_t m = 0; m < nm; ++m) {
                const int64_t bps = std::max<int32_t>(par[m].bricks_per_split, 1);
                par[m].split_merge = (int32_t)std::max<int64_t>(
                    1, std::min<int64_t>((per_item + bps / 2) / bps, par[m].n_split));
                item_work[m] = std::min<int64_t>((int64_t)par[m].split_merge * bps, par[m].n_bricks);
            }
            std::vector<size_t> order(nm);
            for (size_t m = 0; m < nm; ++m) order[m] = m;
            std::stable_sort(order.begin(), order.end(),
                             [&](size_t x, size_t y) { return item_work[x] > item_work[y]; });
            std::vector<int> members(nm);
            std::vector<SumParams> sorted(nm);
            for (size_t m = 0; m < nm; ++m) {
                members[m] = G.members[order[m]];
                sorted[m] = par[order[m]];
            }
            G.members.swap(members);
            par.swap(sorted);
        }
        int32_t acc = 0;
        for (size_t m = 0; m < nm; ++m) {
            prm[m] = par[m];
            if (G.kind != 2) prm[m].split_merge = 1;
            start[m] = acc;
            acc += prm[m].n_tiles * ((prm[m].n_split + prm[m].split_merge - 1) / prm[m].split_merge);
        }
        start[G.members.size()] = acc;
        L->n_items[g] = acc;
        if (L->smem[g] > 220 * 1024) return JEFI_EUNSUPPORTED;
    }
    if (!L->ritems.empty())
        std::memcpy(host + L->off_ritems, L->ritems.data(), sizeof(ReduceItem) * L->ritems.size());
    std::memcpy(host + L->off_rstart, L->rstart.data(), sizeof(int64_t) * L->rstart.size());
    return JEFI_OK;
}

// Persistent launch of group g on stream s, reading the metadata at device address d.
cudaError_t batch_launch_group(const BatchLayout& L, size_t g, jefi_problem* const* hs, unsigned char* d,
                               int n_sm, cudaStream_t s) {
    const BatchGroup& G = L.groups[g];
    // persistent CTAs on a work queue: two per SM for the FP32 kernels (CTAs
    // beyond what the shared memory lets the SM hold start later, find the
    // queue empty and exit), one for the FP64 kernel (its register budget)
    const int per_sm = G.kind == 0 ? 1 : 2;
    const int grid = std::max(1, std::min(L.n_items[g], per_sm * n_sm));
    if (G.kind == 2) {
        StagedBatchArgs a;
        std::memset(&a, 0, sizeof(a));
        a.params = reinterpret_cast<const SumParams*>(d + L.off_params[g]);
        a.item_start = reinterpret_cast<const int32_t*>(d + L.off_start[g]);
        a.n = (int32_t)G.members.size();
        a.n_items = L.n_items[g];
        a.counter = reinterpret_cast<unsigned int*>(d + L.off_counter[g]);
        for (size_t m = 0; m < G.members.size(); ++m) a.maps[m] = hs[G.members[m]]->tmap;
        return launch_sum_f32_staged_batch(a, G.band, G.exact, L.smem[g], grid, s);
    }
    BatchArgs a;
    a.params = reinterpret_cast<const SumParams*>(d + L.off_params[g]);
    a.item_start = reinterpret_cast<const int32_t*>(d + L.off_start[g]);
    a.n = (int32_t)G.members.size();
    a.n_items = L.n_items[g];
    a.counter = reinterpret_cast<unsigned int*>(d + L.off_counter[g]);
    return G.kind == 0 ? launch_sum_f64_batch(a, L.smem[g], grid, s)
                       : launch_sum_f32_batch(a, G.comp != 0, L.smem[g], grid, s);
}

cudaError_t batch_launch_reduce(const BatchLayout& L, unsigned char* d, cudaStream_t s) {
    return launch_reduce_batch(reinterpret_cast<const ReduceItem*>(d + L.off_ritems),
                               reinterpret_cast<const int64_t*>(d + L.off_rstart), (int)L.ritems.size(),
                               L.rstart.back(), s);
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

void jefi_default_params(jefi_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->c = 1.0;
    p->k_e = 1.0;
    p->k_b = 1.0;
    p->dt = 1.0;
    p->t0 = 0.0;
    p->history_slots = 64;
    p->precision = JEFI_FP32_COMP;
    p->deriv = JEFI_DERIV_BACKWARD;
    p->screen[0] = p->screen[1] = p->screen[2] = -1.0;
}

const char* jefi_strerror(int code) {
    switch (code) {
        case JEFI_OK: return "ok";
        case JEFI_EINVAL: return "invalid argument";
        case JEFI_ENOMEM: return "out of memory";
        case JEFI_ENOTYET: return "evaluation time needs a slice that has not been pushed";
        case JEFI_EEVICTED: return "evaluation time needs a slice that was evicted from the ring";
        case JEFI_ECUDA: return "CUDA runtime error";
        case JEFI_ETIMEOUT: return "bounded device wait expired";
        case JEFI_EINTERNAL: return "internal consistency check failed";
        case JEFI_EUNSUPPORTED: return "request outside what this library supports";
        default: return "unknown jefi status";
    }
}

void jefi_host_pair_slots(int64_t n, const double* xo, const double* xs, double t, double t0,
                          double c, double dt, int64_t* out) {
    const double T = t - t0;
    for (int64_t k = 0; k < n; ++k) {
        double dx = xo[3 * k] - xs[3 * k];
        double dy = xo[3 * k + 1] - xs[3 * k + 1];
        double dz = xo[3 * k + 2] - xs[3 * k + 2];
        out[k] = slot_of(sq_sum(dx * dx, dy * dy, dz * dz), T, c, dt);
    }
}

int jefi_host_split_plan(int64_t n_tiles, int64_t n_bricks, int64_t max_splits, int32_t times_per_launch,
                         int64_t resident_ctas, int32_t* n_split, int32_t* bricks_per_split, int32_t* merge) {
    if (n_tiles < 1 || n_bricks < 1 || max_splits < 1 || times_per_launch < 1 || resident_ctas < 1 || !n_split ||
        !bricks_per_split || !merge || n_bricks > INT32_MAX)
        return JEFI_EINVAL;
    const int64_t ns = split_count_for(n_tiles, n_bricks, max_splits, times_per_launch, resident_ctas);
    const int64_t bps = (n_bricks + ns - 1) / ns;
    *n_split = (int32_t)((n_bricks + bps - 1) / bps);
    *bricks_per_split = (int32_t)bps;
    *merge = split_merge_for(n_tiles, *n_split, *bricks_per_split, resident_ctas);
    return JEFI_OK;
}

static int create_impl(const jefi_grid* src, const jefi_grid* obs_grid, const double* obs_points,
                       int64_t n_obs_in, const jefi_params* p, void* stream, jefi_problem* base,
                       jefi_handle* out) {
    if (!src || !p || !out) return JEFI_EINVAL;
    *out = nullptr;
    if (!(p->c > 0) || !std::isfinite(p->c) || !(p->dt > 0) || !std::isfinite(p->dt) ||
        !std::isfinite(p->t0) || !std::isfinite(p->k_e) || !std::isfinite(p->k_b) ||
        p->history_slots < 1 || p->precision < 0 || p->precision > 2 || p->deriv < 0 ||
        p->deriv > 1 || (p->alloc == nullptr) != (p->free == nullptr))
        return JEFI_EINVAL;
    for (int a = 0; a < 3; ++a) {
        if (src->n[a] < 0 || !(src->d[a] > 0) || !std::isfinite(src->d[a]) ||
            !std::isfinite(src->lo[a]) || !std::isfinite(p->screen[a]) || p->src_origin[a] < 0 ||
            p->tile_shape < 0 || p->tile_shape > kTilePacked ||
            (int64_t)p->src_origin[a] + src->n[a] + 4 > ((int64_t)1 << 30))
            return JEFI_EINVAL;
    }
    int64_t n_obs = 0;
    if (obs_grid) {
        for (int a = 0; a < 3; ++a)
            if (obs_grid->n[a] < 0 || !(obs_grid->d[a] > 0) || !std::isfinite(obs_grid->d[a]) ||
                !std::isfinite(obs_grid->lo[a]))
                return JEFI_EINVAL;
        n_obs = (int64_t)obs_grid->n[0] * obs_grid->n[1] * obs_grid->n[2];
    } else {
        if (n_obs_in < 0 || (n_obs_in > 0 && !obs_points)) return JEFI_EINVAL;
        n_obs = n_obs_in;
        for (int64_t i = 0; i < n_obs; ++i)
            if (!finite3(obs_points + 3 * i)) return JEFI_EINVAL;
    }
    if (n_obs > (int64_t)1 << 28 || p->history_slots > (1 << 28)) return JEFI_EUNSUPPORTED;

    jefi_problem* h = new (std::nothrow) jefi_problem();
    if (!h) return JEFI_ENOMEM;
    h->base = base;
    h->time_chunk = base ? kViewTimeChunk : kTimeChunk;
    h->prm = *p;
    h->src = *src;
    h->fp64 = p->precision == JEFI_FP64;
    h->interp = (p->flags & JEFI_FLAG_INTERP) != 0;
    h->central = h->interp && p->deriv == JEFI_DERIV_BACKWARD;
    h->H = p->history_slots;
    for (int a = 0; a < 3; ++a) h->org[a] = p->src_origin[a];
    h->P = (h->H + 3) / 4 * 4;
    for (int a = 0; a < 3; ++a) h->screen[a] = p->screen[a] < 0 ? src->d[a] / 2 : p->screen[a];
    h->n_src = (int64_t)src->n[0] * src->n[1] * src->n[2];
    h->n_obs = n_obs;
    h->nbx = (src->n[0] + 3) / 4;
    h->nby = (src->n[1] + 3) / 4;
    h->nbz = (src->n[2] + 3) / 4;
    h->npx = 4 * h->nbx;
    h->npy = 4 * h->nby;
    h->npz = 4 * h->nbz;
    const int64_t n_bricks = (int64_t)h->nbx * h->nby * h->nbz;
    const int64_t n_cells = n_bricks * kBrickCells;
    if (n_bricks > INT32_MAX / 2 || (double)n_cells * (h->P + kStagedMaxBand + 4.0) > 4e11) {
        delete h;
        return JEFI_EUNSUPPORTED;
    }
    h->n_bricks = (int32_t)n_bricks;

    // ---------------------------------------------------------------- observation tiles
    std::vector<double> pts((size_t)n_obs * 3);
    std::vector<int64_t> order;  // tile slot -> observation index (-1 padding)
    if (obs_grid) {
        const int gx = obs_grid->n[0], gy = obs_grid->n[1], gz = obs_grid->n[2];
        for (int64_t o = 0; o < n_obs; ++o) {
            const int64_t i = o % gx, j = (o / gx) % gy, k = o / ((int64_t)gx * gy);
            pts[3 * o + 0] = center(obs_grid->lo[0], obs_grid->d[0], i);
            pts[3 * o + 1] = center(obs_grid->lo[1], obs_grid->d[1], j);
            pts[3 * o + 2] = center(obs_grid->lo[2], obs_grid->d[2], k);
        }
        if (n_obs > 0) {
            int shape = p->tile_shape > 0 ? p->tile_shape : 1;
            if (p->tile_shape == 0 && !h->fp64 && h->n_src > 0) {
                // The tiling with the least predicted time: its tiles times the
                // relative cost of the band height its widest tile needs (box
                // shapes from their boxes, the packed tiling from its points);
                // on equal cost the narrower widest tile, then the first.
                // FP32 handles choose alike whichever kernel they start on, so
                // a handle switched between kernels equals one created on the
                // other (same tiles, same sums)
                const int64_t np3[3] = {h->npx, h->npy, h->npz};
                double O[3], r_src, db;
                source_shell(*src, h->org, np3, O, &r_src, &db);
                const double Kd = 1.0 / (p->c * p->dt);
                const int max_band = base ? base->mirror : kStagedMaxBand;
                double best_cost = INFINITY, best_ext = INFINITY;
                auto consider = [&](int s_, int64_t tiles, double e) {
                    const double cost = (double)tiles * band_cost(band_for_extent(e, Kd, max_band));
                    const bool tie = std::fabs(cost - best_cost) <= 1e-9 * cost;
                    if ((!tie && cost < best_cost) || (tie && e < best_ext * (1 - 1e-9))) {
                        best_cost = cost;
                        best_ext = e;
                        shape = s_;
                        return true;
                    }
                    return false;
                };
                for (int s_ = 1; s_ <= kNumTileShapes; ++s_) {
                    int64_t tiles = 1;
                    for (int a = 0; a < 3; ++a) tiles *= (obs_grid->n[a] + kTileShapes[s_][a] - 1) / kTileShapes[s_][a];
                    consider(s_, tiles, grid_tiles_extent(*obs_grid, s_, O, r_src, db));
                }
                std::vector<int64_t> packed;
                packed_tile_order(gx, gy, gz, packed);
                if (consider(kTilePacked, (int64_t)(packed.size() / kTileThreads),
                             tiles_extent(packed, pts.data(), O, r_src, db)))
                    order.swap(packed);
            }
            h->tile_shape = shape;
            if (shape != kTilePacked)
                grid_tile_order(gx, gy, gz, shape, order);
            else if (order.empty())
                packed_tile_order(gx, gy, gz, order);
        }
    } else {
        std::memcpy(pts.data(), obs_points, sizeof(double) * 3 * (size_t)n_obs);
        if (n_obs > 0) {
            double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int64_t o = 0; o < n_obs; ++o)
                for (int a = 0; a < 3; ++a) {
                    lo[a] = std::min(lo[a], pts[3 * o + a]);
                    hi[a] = std::max(hi[a], pts[3 * o + a]);
                }
            std::vector<std::pair<uint64_t, int64_t>> keys((size_t)n_obs);
            for (int64_t o = 0; o < n_obs; ++o) keys[o] = {morton(&pts[3 * o], lo, hi), o};
            std::sort(keys.begin(), keys.end());
            const int64_t n_tiles = (n_obs + kTileThreads - 1) / kTileThreads;
            order.assign((size_t)n_tiles * kTileThreads, -1);
            for (int64_t o = 0; o < n_obs; ++o) order[o] = keys[o].second;
            if (!h->fp64 && h->n_src > 0) {
                // Points far from the sources (shells, distant detectors) have
                // narrow slot bands when a tile holds points at similar
                // distances from the source grid, whatever its box: take the
                // radial order (Morton order among equal distances) when it
                // narrows the widest tile's distance range clearly.
                const int64_t np3[3] = {h->npx, h->npy, h->npz};
                double O[3], r_src, db;
                source_shell(*src, h->org, np3, O, &r_src, &db);
                std::vector<std::pair<double, uint64_t>> rk((size_t)n_obs);
                for (int64_t o = 0; o < n_obs; ++o) {
                    double r2 = 0;
                    for (int a = 0; a < 3; ++a) r2 += (pts[3 * o + a] - O[a]) * (pts[3 * o + a] - O[a]);
                    rk[o] = {std::sqrt(r2), (uint64_t)o};
                }
                std::vector<int64_t> by_r((size_t)n_obs);
                for (int64_t o = 0; o < n_obs; ++o) by_r[o] = o;
                std::vector<uint64_t> mkey((size_t)n_obs);
                for (int64_t o = 0; o < n_obs; ++o) mkey[o] = morton(&pts[3 * o], lo, hi);
                std::sort(by_r.begin(), by_r.end(), [&](int64_t a, int64_t b) {
                    return rk[a].first != rk[b].first ? rk[a].first < rk[b].first : mkey[a] < mkey[b];
                });
                std::vector<int64_t> radial((size_t)n_tiles * kTileThreads, -1);
                for (int64_t o = 0; o < n_obs; ++o) radial[o] = by_r[o];
                const double e_m = tiles_extent(order, pts.data(), O, r_src, db);
                const double e_r = tiles_extent(radial, pts.data(), O, r_src, db);
                if (e_r < 0.75 * e_m) order.swap(radial);
            }
        }
    }
    // Anchor of each tile (its slot 0, from which the FP32 kernels form their
    // offsets): on non-lattice geometry the point nearest the centre of the
    // tile's box, which halves the largest anchor offset and with it the
    // FP32 squared-distance error bound (fewer undecided pairs).  Lattices
    // keep their order: every offset is exact there, from any anchor.
    if (!h->fp64 && h->n_src > 0 && n_obs > 0) {
        const int64_t np3[3] = {h->npx, h->npy, h->npz};
        if (!exact_lattice(pts, *src, h->org, np3)) {
            for (size_t t0 = 0; t0 < order.size(); t0 += kTileThreads) {
                double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
                for (size_t q = t0; q < t0 + kTileThreads; ++q) {
                    if (order[q] < 0) continue;
                    for (int a = 0; a < 3; ++a) {
                        lo[a] = std::min(lo[a], pts[3 * order[q] + a]);
                        hi[a] = std::max(hi[a], pts[3 * order[q] + a]);
                    }
                }
                size_t best = t0;
                double best_d = INFINITY;
                for (size_t q = t0; q < t0 + kTileThreads; ++q) {
                    if (order[q] < 0) continue;
                    double dm = 0;
                    for (int a = 0; a < 3; ++a)
                        dm = std::max(dm, std::fabs(pts[3 * order[q] + a] - 0.5 * (lo[a] + hi[a])));
                    if (dm < best_d) {
                        best_d = dm;
                        best = q;
                    }
                }
                std::swap(order[t0], order[best]);
            }
        }
    }
    h->n_slots = (int32_t)order.size();
    h->n_tiles = h->n_slots / kTileThreads;
    h->slot_obs.resize(order.size());
    h->inv_perm.resize((size_t)n_obs);
    std::vector<double> slot_xyz((size_t)h->n_slots * 3);
    std::vector<int32_t> scr((size_t)6 * h->n_slots);
    double O[3] = {0, 0, 0}, Xmax = 0;
    const int64_t npad_axis[3] = {h->npx, h->npy, h->npz};
    for (int a = 0; a < 3; ++a) {
        Xmax = std::max(Xmax, std::fabs(src->lo[a]));
        Xmax = std::max(Xmax, std::fabs(center(src->lo[a], src->d[a], h->org[a] + npad_axis[a])));
    }
    for (int64_t tile = 0; tile < h->n_tiles; ++tile) {
        // padding slots repeat the last real point of their tile (or the first)
        int64_t fill = -1;
        for (int tid = 0; tid < kTileThreads; ++tid)
            if (order[tile * kTileThreads + tid] >= 0) fill = order[tile * kTileThreads + tid];
        for (int tid = 0; tid < kTileThreads; ++tid) {
            const int64_t s = tile * kTileThreads + tid;
            const int64_t o = order[s];
            h->slot_obs[s] = (int32_t)o;
            if (o >= 0) h->inv_perm[o] = (int32_t)s;
            const int64_t src_o = o >= 0 ? o : fill;
            for (int a = 0; a < 3; ++a) slot_xyz[3 * s + a] = pts[3 * src_o + a];
        }
        // the anchor of the FP32 kernel is the tile's first slot
        for (int tid = 0; tid < kTileThreads; ++tid) {
            const int64_t s = tile * kTileThreads + tid;
            for (int a = 0; a < 3; ++a) {
                O[a] = std::max(O[a], std::fabs(slot_xyz[3 * s + a] - slot_xyz[3 * tile * kTileThreads + a]));
                Xmax = std::max(Xmax, std::fabs(slot_xyz[3 * s + a]));
            }
        }
    }

    h->obs_sig = fnv1a(kFnvBasis, slot_xyz.data(), sizeof(double) * slot_xyz.size());

    // Double-float copies of the geometry for the FP32 kernels' check of
    // undecided pairs, and its bound.  Every coordinate splits as hi + lo
    // within 2^-48 of its FP64 value; with X the largest coordinate, each
    // double-float difference is within 8 X 2^-48 of the exact one, which
    // moves the squared distance by at most 2 sqrt(3) R 8 X 2^-48; the
    // squares, sums and the comparison add at most 2^-42.3 S, the FP64
    // rule's own roundings 5 S 2^-53 and the thresholds' split 2^-48 S.
    // Four times that: B = 2^-41 X R + 2^-40 S.
    if (!h->fp64) {
        auto split = [](double v) {
            const float hi = (float)v;
            return make_float2(hi, (float)(v - (double)hi));
        };
        h->h_obs_hl.resize((size_t)6 * h->n_slots);
        for (size_t q = 0; q < (size_t)h->n_slots * 3; ++q) {
            const float2 v = split(slot_xyz[q]);
            h->h_obs_hl[2 * q] = v.x;
            h->h_obs_hl[2 * q + 1] = v.y;
        }
        h->h_cc_hl.clear();
        for (int a = 0; a < 3; ++a)
            for (int64_t i = 0; i < npad_axis[a]; ++i)
                h->h_cc_hl.push_back(split(center(src->lo[a], src->d[a], h->org[a] + i)));
        h->df_b1 = (float)(std::ldexp(1.0, -41) * Xmax);
        h->df_b2 = (float)std::ldexp(1.0, -40);
    }

    // ---------------------------------------------------------------- screening and extremes
    const int64_t nlim[3] = {src->n[0], src->n[1], src->n[2]};
    const int64_t npad[3] = {h->npx, h->npy, h->npz};
    if (h->n_src > 0) {
        // Per-axis results depend on one coordinate only; observation grids
        // repeat each coordinate many times, so memoise them per axis.
        std::map<double, std::pair<AxisInfo, AxisInfo>> memo[3];
        for (int64_t s = 0; s < h->n_slots; ++s) {
            AxisInfo real_ax[3], pad_ax[3];
            for (int a = 0; a < 3; ++a) {
                const double x = slot_xyz[3 * s + a];
                auto it = obs_grid ? memo[a].find(x) : memo[a].end();
                if (it != memo[a].end()) {
                    pad_ax[a] = it->second.first;
                    real_ax[a] = it->second.second;
                } else {
                    pad_ax[a] = axis_info(x, src->lo[a], src->d[a], h->org[a], npad[a], npad[a], h->screen[a]);
                    real_ax[a] = axis_info(x, src->lo[a], src->d[a], h->org[a], nlim[a], npad[a], h->screen[a]);
                    if (obs_grid) memo[a][x] = {pad_ax[a], real_ax[a]};
                }
                scr[(2 * a) * h->n_slots + s] = pad_ax[a].rlo;
                scr[(2 * a + 1) * h->n_slots + s] = pad_ax[a].rhi;
            }
            fold(h->pad, pad_ax);
            if (h->slot_obs[s] >= 0) fold(h->real, real_ax);
        }
    }
    h->any_pairs = h->n_src > 0 && n_obs > 0 && std::isfinite(h->real.s_min);
    if (h->any_pairs && !h->fp64 && !(h->pad.s_min > 1e-30)) {
        delete h;
        return JEFI_EUNSUPPORTED;  // unscreened pairs closer than FP32 can square
    }

    // ---------------------------------------------------------------- FP32 error model
    h->exact = exact_lattice(slot_xyz, *src, h->org, npad);
    if (h->exact) {
        h->err_rel = h->err_lin = h->err_abs = 0.0;   // S32 == S64 exactly
    } else {
        const double u = std::ldexp(1.0, -24);
        double G2 = 0;
        for (int a = 0; a < 3; ++a) {
            const double G = u * (2 * O[a] + 12 * src->d[a]) + 4 * std::ldexp(1.0, -53) * Xmax;
            G2 += G * G;
        }
        const double G = std::sqrt(G2) * (1 + 1e-6);
        h->err_rel = kSafety * (9.1 * u + 1e-15);
        h->err_lin = kSafety * 2 * G;
        h->err_abs = kSafety * G * G;
    }

    // ---------------------------------------------------------------- table size, splits
    if (h->any_pairs) {
        const double span = (std::sqrt(h->pad.s_max) - std::sqrt(h->pad.s_min)) / (p->c * p->dt);
        const double K = std::ceil(span) + 4 + 2 * kTablePad;
        if (!(K < 8192)) {
            delete h;
            return JEFI_EUNSUPPORTED;
        }
        h->K = (int32_t)K;
    } else {
        h->K = 1;
    }
    {
        // Source splits: at most twice the count that gives eight waves of
        // (tile, split) items of two CTAs per SM at one evaluation time (four
        // for views), at most one per brick, and partials of at most 256 MB
        // (32 MB for views, many of which are cached under a serving
        // budget); within that, the count whose launches fill their waves
        // (split_count_for; a launch can still merge them, split_merge_for).
        const int64_t resident = 2 * (int64_t)current_sm_count();
        const int64_t target = (base ? 4 : 8) * resident;
        int64_t ns = std::max<int64_t>(1, (target + h->n_tiles - 1) / std::max<int32_t>(h->n_tiles, 1));
        ns = std::min<int64_t>(2 * ns, std::max<int32_t>(h->n_bricks, 1));
        const int64_t split_bytes = (int64_t)h->time_chunk * 6 * 8 * std::max<int32_t>(h->n_slots, 1);
        const int64_t cap = base ? ((int64_t)32 << 20) : ((int64_t)256 << 20);
        ns = std::max<int64_t>(1, std::min<int64_t>(ns, cap / split_bytes));
        ns = split_count_for(h->n_tiles, h->n_bricks, ns, h->time_chunk, resident);
        h->bricks_per_split = (int32_t)((h->n_bricks + ns - 1) / ns);
        if (h->bricks_per_split < 1) h->bricks_per_split = 1;
        h->n_split = (int32_t)((h->n_bricks + h->bricks_per_split - 1) / h->bricks_per_split);
        if (h->n_split < 1) h->n_split = 1;
        h->n_split_max = h->n_split;
    }

    // ---------------------------------------------------------------- FP32 candidate bias
    // g bounds |floor argument in FP32 - FP64 rule| (slots), without the |T/dt|
    // term that each evaluation adds: floor(A + g - R K) is then n or n+1 and
    // one threshold decides (both FP32 sum kernels).
    if (!h->fp64 && h->any_pairs) {
        const double Kd = 1.0 / (p->c * p->dt);
        const double u = std::ldexp(1.0, -24);
        const double eps_rsqrt = std::ldexp(1.0, -22);   // measured max 2^-22.93 over all normals
        const double eps_S = h->exact ? 0.0
                                      : h->err_rel + h->err_lin / std::sqrt(h->pad.s_min) + h->err_abs / h->pad.s_min;
        const double w_max = std::sqrt(h->pad.s_max) * Kd;
        const double A_max = h->K + 2.0;
        h->g_bias = 2.0 * (u * (2 * A_max + 2) + w_max * (eps_S / 2 + eps_rsqrt + 4 * u) +
                           u * (A_max + w_max + 2));
        if (!(2 * (h->g_bias + 1e-3) < 1.0)) {
            delete h;
            return JEFI_EUNSUPPORTED;   // FP32 cannot place the candidate within one slot: use FP64
        }
    }

    // ---------------------------------------------------------------- staged FP32 kernel
    // The TMA-staged kernel needs every (tile, stage) slot band to fit one of
    // the compiled band heights, and a candidate bias g with 2g < 1.  Per
    // tile the kernel bounds the pair distances two ways and keeps the
    // tighter: the tile's box against the stage's box, and the shell
    // [rho_lo, rho_hi] of the tile's distances from O (the source grid's
    // centre) widened by the farthest source cell from O (only where the
    // shell can be the tighter bound: rho_lo < 0 marks the others).  The host
    // takes the widest band over tiles of the same bounds (plus one spare
    // slot).
    std::vector<float> tile_box((size_t)h->n_tiles * kTileBoxFloats);
    if (!h->fp64 && h->any_pairs && !(p->flags & JEFI_FLAG_DIRECT_GATHER)) {
        double O[3], r_src, db;
        source_shell(*src, h->org, npad, O, &r_src, &db);
        double ext_max = 0;
        for (int64_t tile = 0; tile < h->n_tiles; ++tile) {
            double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
            double rho_lo = INFINITY, rho_hi = 0;
            const double* anchor = &slot_xyz[3 * tile * kTileThreads];
            for (int tid = 0; tid < kTileThreads; ++tid) {
                const double* x = &slot_xyz[3 * (tile * kTileThreads + tid)];
                double r2 = 0;
                for (int a = 0; a < 3; ++a) {
                    mn[a] = std::min(mn[a], x[a] - anchor[a]);
                    mx[a] = std::max(mx[a], x[a] - anchor[a]);
                    r2 += (x[a] - O[a]) * (x[a] - O[a]);
                }
                rho_lo = std::min(rho_lo, std::sqrt(r2));
                rho_hi = std::max(rho_hi, std::sqrt(r2));
            }
            double d2 = 0;
            float* tb = &tile_box[tile * kTileBoxFloats];
            for (int a = 0; a < 3; ++a) {
                tb[a] = round_down_f32(mn[a]);
                tb[3 + a] = round_up_f32(mx[a]);
                tb[6 + a] = (float)(O[a] - anchor[a]);
                d2 += (mx[a] - mn[a]) * (mx[a] - mn[a]);
            }
            // widest distance range of any pair of this tile: box bound or shell bound
            const double ext_box = std::sqrt(d2) + db;
            const double ext_shell = (rho_hi - rho_lo) + 2 * r_src;
            ext_max = std::max(ext_max, std::min(ext_box, ext_shell));
            // the kernel tries the shell only where it can beat the box (it
            // costs the producing thread a few more operations per stage)
            const bool shell = ext_shell < ext_box;
            tb[9] = shell ? round_down_f32(rho_lo * (1 - 1e-12)) : -1.f;
            tb[10] = round_up_f32(rho_hi * (1 + 1e-12));
            tb[11] = 0.f;
        }
        const double Kd = 1.0 / (p->c * p->dt);
        const double need = std::ceil(ext_max * Kd * (1 + 1e-4) + 1e-3) + 7;
        int band = 0;
        for (int b : kStagedBands)
            if (need <= b) { band = b; break; }
        if (base && band > base->mirror) band = 0;      // a view fits the base ring's mirror
        if (band > 0) {
            SumParams probe{};
            probe.K = h->K;
            probe.nbx = h->nbx;
            probe.nby = h->nby;
            probe.nbz = h->nbz;
            probe.npx = (int)npad[0];
            probe.npy = (int)npad[1];
            probe.npz = (int)npad[2];
            probe.exact = h->exact ? 1 : 0;
            if (staged_smem_bytes(probe, band, false) <= 220 * 1024) h->band = band;
            // the next compiled height: a wider band with other stages (cells,
            // swizzle) that the tuner may time against this one
            for (int b : kStagedBands)
                if (h->band > 0 && b > h->band && !(base && b > base->mirror) &&
                    staged_smem_bytes(probe, b, false) <= 220 * 1024) {
                    h->band_alt = b;
                    break;
                }
        }
    }
    if (base) {
        h->mirror = base->mirror;
    } else if (!h->fp64 && (p->flags & JEFI_FLAG_SHARED_RING)) {
        h->mirror = kStagedMaxBand;                      // room for the widest staged band of any view
    } else {
        h->mirror = std::max(h->band, h->band_alt);
    }
    h->Hp = h->P + h->mirror + kZeroPadSlots;
    h->band0 = h->band;
    if (!h->fp64 && h->any_pairs && h->band == 0 && h->Hp > 65536) {
        delete h;   // the direct-gather kernel packs two physical slots in 16 bits each
        return JEFI_EUNSUPPORTED;
    }

    // ---------------------------------------------------------------- device buffers
    cudaStream_t s = (cudaStream_t)stream;
    const size_t esz = h->fp64 ? sizeof(double) : sizeof(float);
    const size_t ring_bytes = (size_t)n_cells * h->Hp * 8 * esz;
    h->ring = base ? base->ring : dev_alloc(h, ring_bytes);
    h->obs_xyz = (double*)dev_alloc(h, sizeof(double) * slot_xyz.size());
    h->obs_scr = (int32_t*)dev_alloc(h, sizeof(int32_t) * scr.size());
    h->d_inv_perm = (int32_t*)dev_alloc(h, sizeof(int32_t) * std::max<size_t>(1, h->inv_perm.size()));
    h->prev = base ? base->prev : (double*)dev_alloc(h, sizeof(double) * 4 * std::max<int64_t>(1, h->n_src));
    if (h->central)
        h->prev2 = base ? base->prev2 : (double*)dev_alloc(h, sizeof(double) * 4 * std::max<int64_t>(1, h->n_src));
    h->stage_in = base ? base->stage_in : (double*)dev_alloc(h, sizeof(double) * 8 * std::max<int64_t>(1, h->n_src));
    h->partials = (double*)dev_alloc(h, sizeof(double) * h->time_chunk * h->n_split * 6 * std::max<int32_t>(1, h->n_slots));
    h->out_stage = (double*)dev_alloc(h, sizeof(double) * h->time_chunk * 6 * std::max<int64_t>(1, n_obs));
    h->tab32 = (float4*)dev_alloc(h, sizeof(float4) * h->time_chunk * h->K);
    h->theta = (double*)dev_alloc(h, sizeof(double) * h->time_chunk * theta_stride(h->K));
    h->times = (TimeParams*)dev_alloc(h, sizeof(TimeParams) * h->time_chunk);
    h->fallbacks = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long));
    h->status = (int32_t*)dev_alloc(h, sizeof(int32_t));
    if (!h->fp64) {
        h->obs_hl = (float*)dev_alloc(h, sizeof(float) * h->h_obs_hl.size());
        h->cc_hl = (float2*)dev_alloc(h, sizeof(float2) * h->h_cc_hl.size());
        if (!h->obs_hl || !h->cc_hl) h->status = nullptr;
    }
    if (!h->fp64 && h->any_pairs && h->band == 0 && !alloc_direct_tables(h)) h->status = nullptr;
    if (h->band > 0) {
        h->tile_box = (float*)dev_alloc(h, sizeof(float) * tile_box.size());
        h->tab2 = (float2*)dev_alloc(h, sizeof(float2) * h->time_chunk * (h->K + 2 * kTabGuard));
        if (!h->tile_box || !h->tab2) h->status = nullptr;
        h->h_tab2.resize((size_t)h->time_chunk * (h->K + 2 * kTabGuard));
    }
    if (!h->ring || !h->obs_xyz || !h->obs_scr || !h->d_inv_perm || !h->prev || !h->stage_in ||
        !h->partials || !h->out_stage || !h->tab32 || !h->theta || !h->times || !h->fallbacks ||
        !h->status) {
        release_all(h);
        delete h;
        return JEFI_ENOMEM;
    }
    h->h_tab.resize((size_t)h->time_chunk * h->K);
    h->h_theta.resize((size_t)h->time_chunk * theta_stride(h->K));
    h->h_times.resize(h->time_chunk);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess && !base) e = cudaMemsetAsync(h->ring, 0, ring_bytes, s);
    if (e == cudaSuccess && !base)
        e = cudaMemsetAsync(h->prev, 0, sizeof(double) * 4 * std::max<int64_t>(1, h->n_src), s);
    if (e == cudaSuccess && !base && h->prev2)   // a view shares its base's difference state
        e = cudaMemsetAsync(h->prev2, 0, sizeof(double) * 4 * std::max<int64_t>(1, h->n_src), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->fallbacks, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess && h->band > 0)
        e = cudaMemcpyAsync(h->tile_box, tile_box.data(), sizeof(float) * tile_box.size(), cudaMemcpyHostToDevice, s);
    int tmap_rc = JEFI_OK;
    if (e == cudaSuccess && h->band > 0) {
        tmap_rc = make_tensor_map(h);
        if (tmap_rc != JEFI_OK) e = cudaErrorInvalidValue;
    }
    if (e == cudaSuccess && !slot_xyz.empty())
        e = cudaMemcpyAsync(h->obs_xyz, slot_xyz.data(), sizeof(double) * slot_xyz.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !scr.empty())
        e = cudaMemcpyAsync(h->obs_scr, scr.data(), sizeof(int32_t) * scr.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && h->obs_hl && !h->h_obs_hl.empty())
        e = cudaMemcpyAsync(h->obs_hl, h->h_obs_hl.data(), sizeof(float) * h->h_obs_hl.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && h->cc_hl && !h->h_cc_hl.empty())
        e = cudaMemcpyAsync(h->cc_hl, h->h_cc_hl.data(), sizeof(float2) * h->h_cc_hl.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !h->inv_perm.empty())
        e = cudaMemcpyAsync(h->d_inv_perm, h->inv_perm.data(), sizeof(int32_t) * h->inv_perm.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);   // copies already enqueued finish before the memory is released
        cudaGetLastError();
        release_all(h);
        delete h;
        return tmap_rc != JEFI_OK ? tmap_rc : JEFI_ECUDA;
    }
    if (base) {
        base->n_views++;
        h->n_latest = base->n_latest;
    }
    *out = h;
    return JEFI_OK;
}

int jefi_create(const jefi_grid* src, const jefi_grid* obs_grid, const double* obs_points,
                int64_t n_obs, const jefi_params* p, void* stream, jefi_handle* out) {
    NvtxRange nvtx_range("jefi_create");
    return create_impl(src, obs_grid, obs_points, n_obs, p, stream, nullptr, out);
}

int jefi_create_view(jefi_handle base, const jefi_grid* obs_grid, const double* obs_points,
                     int64_t n_obs, void* stream, jefi_handle* out) {
    NvtxRange nvtx_range("jefi_create_view");
    if (!base || !out) return JEFI_EINVAL;
    if (base->base) return JEFI_EINVAL;                  // views of views are not supported
    return create_impl(&base->src, obs_grid, obs_points, n_obs, &base->prm, stream, base, out);
}

// Push one slice whose arrays cover full_n cells (x fastest); the handle's
// cell (i, j, k) is their cell offset + (i, j, k).
static int push_impl(jefi_handle h, const double* rho, const double* J, const double* drho, const double* dJ,
                     const int32_t* full_n, const int32_t* offset, int on_device, void* stream) {
    if (!h || h->base) return JEFI_EINVAL;               // views read the base's history
    const bool supplied = h->prm.deriv == JEFI_DERIV_SUPPLIED;
    if (h->n_src > 0 && (!rho || !J)) return JEFI_EINVAL;
    if (supplied != (drho != nullptr) || supplied != (dJ != nullptr)) return JEFI_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (offset[a] < 0 || full_n[a] < 0 || (int64_t)offset[a] + h->src.n[a] > full_n[a]) return JEFI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = h->n_src;
    const bool region = full_n[0] != h->src.n[0] || full_n[1] != h->src.n[1] || full_n[2] != h->src.n[2];
    const double *r = rho, *j = J, *dr = drho, *dj = dJ;
    int32_t fnx = full_n[0], fny = full_n[1], ox = offset[0], oy = offset[1], oz = offset[2];
    if (!on_device && n > 0) {
        // host slices: the handle's cells (gathered from a region first) go
        // to the staging buffer, then the push reads them as a whole grid
        std::vector<double> gather;
        const double *hr = rho, *hj = J, *hdr = drho, *hdj = dJ;
        if (region) {
            const int nx = h->src.n[0], ny = h->src.n[1], nz = h->src.n[2];
            gather.resize((size_t)n * (supplied ? 8 : 4));
            double* gr = gather.data();
            double* gj = gr + n;
            for (int k = 0; k < nz; ++k)
                for (int jj = 0; jj < ny; ++jj)
                    for (int i = 0; i < nx; ++i) {
                        const int64_t g = ((int64_t)k * ny + jj) * nx + i;
                        const int64_t f = ((int64_t)(oz + k) * fny + (oy + jj)) * fnx + (ox + i);
                        gr[g] = rho[f];
                        for (int a = 0; a < 3; ++a) gj[3 * g + a] = J[3 * f + a];
                        if (supplied) {
                            gr[4 * n + g] = drho[f];
                            for (int a = 0; a < 3; ++a) gr[5 * n + 3 * g + a] = dJ[3 * f + a];
                        }
                    }
            hr = gr;
            hj = gj;
            hdr = supplied ? gr + 4 * n : nullptr;
            hdj = supplied ? gr + 5 * n : nullptr;
            fnx = nx;
            fny = ny;
            ox = oy = oz = 0;
        }
        double* st = h->stage_in;
        JEFI_CUDA(cudaMemcpyAsync(st, hr, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        JEFI_CUDA(cudaMemcpyAsync(st + n, hj, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
        r = st;
        j = st + n;
        if (supplied) {
            JEFI_CUDA(cudaMemcpyAsync(st + 4 * n, hdr, sizeof(double) * n, cudaMemcpyHostToDevice, s));
            JEFI_CUDA(cudaMemcpyAsync(st + 5 * n, hdj, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
            dr = st + 4 * n;
            dj = st + 5 * n;
        }
        // the gathered copy must outlive the (pageable) copies above
        if (region) JEFI_CUDA(cudaStreamSynchronize(s));
    }
    const int64_t next = h->n_latest + 1;
    PushParams p{};
    p.nx = h->src.n[0];
    p.ny = h->src.n[1];
    p.nz = h->src.n[2];
    p.nbx = h->nbx;
    p.nby = h->nby;
    p.n_src = n;
    p.fnx = fnx;
    p.fny = fny;
    p.ox = ox;
    p.oy = oy;
    p.oz = oz;
    p.Hp = h->Hp;
    p.slot = (int32_t)(next % h->P);
    p.mirror_slot = p.slot < h->mirror ? p.slot + h->P : -1;
    p.supplied = supplied;
    p.fp64 = h->fp64;
    p.c = h->prm.c;
    p.inv_c = 1.0 / h->prm.c;
    p.dt = h->prm.dt;
    p.rho = r;
    p.J = j;
    p.drho = dr;
    p.dJ = dj;
    p.prev = h->prev;
    p.ring = h->ring;
    p.central = h->central ? 1 : 0;
    p.prev2 = h->prev2;
    p.prev_slot = -1;
    p.prev_mirror_slot = -1;
    if (h->central && next >= 1) {
        p.prev_slot = (int32_t)((next - 1) % h->P);
        p.prev_mirror_slot = p.prev_slot < h->mirror ? p.prev_slot + h->P : -1;
    }
    JEFI_CUDA(launch_push(p, s));
    if (n > 0) h->launches++;
    h->n_latest = next;
    return mark_use(h, s);
}

int jefi_push_sources(jefi_handle h, const double* rho, const double* J, const double* drho,
                      const double* dJ, int on_device, void* stream) {
    NvtxRange nvtx_range("jefi_push_sources");
    if (!h) return JEFI_EINVAL;
    const int32_t zero[3] = {0, 0, 0};
    return push_impl(h, rho, J, drho, dJ, h->src.n, zero, on_device, stream);
}

int jefi_push_sources_region(jefi_handle h, const double* rho, const double* J, const double* drho,
                             const double* dJ, const int32_t* full_n, const int32_t* offset, int on_device,
                             void* stream) {
    NvtxRange nvtx_range("jefi_push_sources_region");
    if (!h || !full_n || !offset) return JEFI_EINVAL;
    return push_impl(h, rho, J, drho, dJ, full_n, offset, on_device, stream);
}

static void sync_view(jefi_problem* h) {
    if (h && h->base) h->n_latest = h->base->n_latest;
}

static int eval_impl(jefi_handle h, int32_t n_t, const double* t, double* E, double* B,
                     int on_device, void* stream) {
    NvtxRange nvtx_range("jefi_eval_fields");
    if (!h || n_t < 0 || (n_t > 0 && !t)) return JEFI_EINVAL;
    sync_view(h);
    if (n_t == 0 || h->n_obs == 0) return JEFI_OK;
    if (!E || !B) return JEFI_EINVAL;
    for (int i = 0; i < n_t; ++i) {
        const int rc = check_time(h, t[i]);
        if (rc != JEFI_OK) return rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t per_t = (size_t)h->n_obs * 3;
    for (int base = 0; base < n_t; base += h->time_chunk) {
        const int m = std::min(h->time_chunk, n_t - base);
        double* Ed = on_device ? E + base * per_t : h->out_stage;
        double* Bd = on_device ? B + base * per_t : h->out_stage + h->time_chunk * per_t;
        if (!h->any_pairs) {
            JEFI_CUDA(cudaMemsetAsync(Ed, 0, sizeof(double) * per_t * m, s));
            JEFI_CUDA(cudaMemsetAsync(Bd, 0, sizeof(double) * per_t * m, s));
        } else {
            const int rc = launch_chunk(h, m, t + base, Ed, Bd, s, nullptr);
            if (rc != JEFI_OK) return rc;
        }
        if (!on_device) {
            JEFI_CUDA(cudaMemcpyAsync(E + base * per_t, Ed, sizeof(double) * per_t * m, cudaMemcpyDeviceToHost, s));
            JEFI_CUDA(cudaMemcpyAsync(B + base * per_t, Bd, sizeof(double) * per_t * m, cudaMemcpyDeviceToHost, s));
            int32_t st = 0;
            JEFI_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost, s));
            JEFI_CUDA(cudaStreamSynchronize(s));
            if (st != 0) return st;
        }
    }
    return mark_use(h, s);
}

int jefi_eval_fields(jefi_handle h, double t, double* E, double* B, int on_device, void* stream) {
    return eval_impl(h, 1, &t, E, B, on_device, stream);
}

int jefi_eval_fields_multi(jefi_handle h, int32_t n_t, const double* t, double* E, double* B,
                           int on_device, void* stream) {
    return eval_impl(h, n_t, t, E, B, on_device, stream);
}

int jefi_eval_batch(const jefi_handle* hs, const double* t, double* const* E, double* const* B, int32_t n,
                    void* stream) {
    NvtxRange nvtx_range("jefi_eval_batch");
    if (n < 0 || (n > 0 && (!hs || !t || !E || !B))) return JEFI_EINVAL;
    if (n == 0) return JEFI_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> occ(n);
    std::map<jefi_problem*, int> count;
    for (int i = 0; i < n; ++i) {
        jefi_problem* h = hs[i];
        if (!h) return JEFI_EINVAL;
        sync_view(h);
        if (h->n_obs > 0 && (!E[i] || !B[i])) return JEFI_EINVAL;
        const int rc = check_time(h, t[i]);
        if (rc != JEFI_OK) return rc;
        occ[i] = count[h]++;
        if (occ[i] >= h->time_chunk) return JEFI_EUNSUPPORTED;   // scratch slots per handle
    }
    for (int i = 0; i < n; ++i)
        if (hs[i]->any_pairs && hs[i]->n_obs > 0) build_tables(hs[i], occ[i], t[i]);
    for (auto& kv : count)
        if (kv.first->any_pairs && kv.first->n_obs > 0) {
            const int rc = upload_tables(kv.first, kv.second, s);
            if (rc != JEFI_OK) return rc;
        }

    // One persistent launch per kernel variant, then one reduction.
    BatchLayout L;
    batch_layout(hs, occ.data(), E, B, n, &L);
    for (int i : L.zero_entries) {
        JEFI_CUDA(cudaMemsetAsync(E[i], 0, sizeof(double) * 3 * hs[i]->n_obs, s));
        JEFI_CUDA(cudaMemsetAsync(B[i], 0, sizeof(double) * 3 * hs[i]->n_obs, s));
    }
    if (L.groups.empty()) return JEFI_OK;

    int dev = 0;
    JEFI_CUDA(cudaGetDevice(&dev));
    BatchArena& arena = arena_for(dev, s);
    std::lock_guard<std::mutex> guard(arena.lock);
    {
        const int rc = arena_reserve(arena, L.bytes);
        if (rc != JEFI_OK) return rc;
    }
    std::vector<unsigned char> host(L.bytes, 0);
    {
        const int rc = batch_fill(&L, host.data(), [&](int i) { return make_params(hs[i], 1, occ[i], nullptr); });
        if (rc != JEFI_OK) return rc;
    }
    unsigned char* d = static_cast<unsigned char*>(arena.dev);
    JEFI_CUDA(cudaStreamWaitEvent(s, arena.done, 0));
    JEFI_CUDA(cudaMemcpyAsync(d, host.data(), L.bytes, cudaMemcpyHostToDevice, s));
    for (size_t g = 0; g < L.groups.size(); ++g)
        if (batch_launch_group(L, g, hs, d, arena.n_sm, s) != cudaSuccess) return JEFI_ECUDA;
    JEFI_CUDA(batch_launch_reduce(L, d, s));
    JEFI_CUDA(cudaEventRecord(arena.done, s));
    for (int i = 0; i < n; ++i) {
        const int rc = mark_use(hs[i], s);
        if (rc != JEFI_OK) return rc;
    }
    return JEFI_OK;
}

int jefi_debug_slots(jefi_handle h, double t, int32_t* slots, void* stream) {
    if (!h || !slots) return JEFI_EINVAL;
    sync_view(h);
    const int rc = check_time(h, t);
    if (rc != JEFI_OK) return rc;
    if (h->n_obs == 0 || h->n_src == 0) return JEFI_OK;
    const int64_t n_cells = (int64_t)h->n_bricks * kBrickCells;
    const int64_t total = (int64_t)h->n_slots * n_cells;
    if (total > ((int64_t)1 << 30)) return JEFI_EUNSUPPORTED;
    if (!h->any_pairs) {
        for (int64_t i = 0; i < h->n_obs * h->n_src; ++i) slots[i] = INT32_MIN;
        return JEFI_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int32_t* d = nullptr;
    JEFI_CUDA(cudaMalloc(&d, sizeof(int32_t) * total));
    std::vector<int32_t> host((size_t)total);
    int r = launch_chunk(h, 1, &t, nullptr, nullptr, s, d);
    if (r == JEFI_OK) {
        cudaError_t e = cudaMemcpyAsync(host.data(), d, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) r = JEFI_ECUDA;
    }
    cudaFree(d);
    if (r != JEFI_OK) return r;
    const int nx = h->src.n[0], ny = h->src.n[1];
    for (int64_t o = 0; o < h->n_obs; ++o) {
        const int64_t slot = h->inv_perm[o];
        for (int64_t g = 0; g < h->n_src; ++g) {
            const int64_t ix = g % nx, iy = (g / nx) % ny, iz = g / ((int64_t)nx * ny);
            const int64_t brick = ((iz >> 2) * h->nby + (iy >> 2)) * h->nbx + (ix >> 2);
            const int64_t cell = brick * kBrickCells + ((iz & 3) * 16 + (iy & 3) * 4 + (ix & 3));
            slots[o * h->n_src + g] = host[(size_t)(slot * n_cells + cell)];
        }
    }
    return JEFI_OK;
}

int jefi_debug_wait_timeout(double limit_s, void* stream) {
    if (!(limit_s > 0) || !(limit_s <= 10.0)) return JEFI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t* d = nullptr;
    JEFI_CUDA(cudaMalloc(&d, sizeof(int32_t)));
    int32_t st = -1;
    cudaError_t e = cudaMemsetAsync(d, 0xff, sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_wait_timeout_probe(d, (uint64_t)(limit_s * 1e9), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, d, sizeof(st), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return JEFI_ECUDA;
    return st;
}

namespace {

// Can the direct-gather kernel run handle h?
bool direct_possible(jefi_problem* h) {
    if (h->Hp > 65536) return false;   // two physical slots packed in 16 bits each
    if (!alloc_direct_tables(h)) return false;
    return sum_smem_bytes(make_params(h, 1, 0, nullptr)) <= 200 * 1024;
}

// Device time of one evaluation of h at t into the handle's staging buffer,
// after one untimed evaluation, in ms.  Returns JEFI_OK or an error code.
int time_eval(jefi_problem* h, double t, cudaStream_t s, float* ms) {
    const size_t per_t = (size_t)h->n_obs * 3;
    double* E = h->out_stage;
    double* B = h->out_stage + h->time_chunk * per_t;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int rc = JEFI_OK;
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) rc = JEFI_ECUDA;
    if (rc == JEFI_OK) rc = launch_chunk(h, 1, &t, E, B, s, nullptr);
    if (rc == JEFI_OK && cudaEventRecord(ev[0], s) != cudaSuccess) rc = JEFI_ECUDA;
    if (rc == JEFI_OK) rc = launch_chunk(h, 1, &t, E, B, s, nullptr);
    if (rc == JEFI_OK && (cudaEventRecord(ev[1], s) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
                          cudaEventElapsedTime(ms, ev[0], ev[1]) != cudaSuccess))
        rc = JEFI_ECUDA;
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (rc == JEFI_ECUDA) cudaGetLastError();
    return rc;
}

}  // namespace

int jefi_select_kernel(jefi_handle h, int32_t mode, double t, int32_t* staged_band, void* stream) {
    NvtxRange nvtx_range("jefi_select_kernel");
    if (!h || h->fp64 || mode < JEFI_KERNEL_MEASURE || mode > JEFI_KERNEL_STAGED) return JEFI_EINVAL;
    sync_view(h);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = JEFI_OK;
    if (mode == JEFI_KERNEL_STAGED) {
        if (h->band0 == 0) rc = JEFI_EUNSUPPORTED;
        else rc = set_band(h, h->band0);
    } else if (mode == JEFI_KERNEL_DIRECT) {
        if (h->band != 0 && h->any_pairs) {
            if (direct_possible(h)) h->band = 0;
            else rc = JEFI_EUNSUPPORTED;
        }
    } else {
        rc = check_time(h, t);
        if (rc == JEFI_OK && h->band0 != 0 && h->any_pairs && h->n_obs > 0) {
            // candidates: the creation band, the wider compiled band, the direct gather
            int32_t cand[3];
            int nc = 0;
            cand[nc++] = h->band0;
            if (h->band_alt > 0) cand[nc++] = h->band_alt;
            if (direct_possible(h)) cand[nc++] = 0;
            const int32_t keep = h->band;
            int32_t best = keep;
            float best_ms = INFINITY;
            for (int c = 0; c < nc && nc > 1 && rc == JEFI_OK; ++c) {
                float ms = 0.f;
                rc = set_band(h, cand[c]);
                if (rc == JEFI_OK) rc = time_eval(h, t, s, &ms);
                if (rc == JEFI_OK && ms < best_ms) {
                    best_ms = ms;
                    best = cand[c];
                }
            }
            const int rb = set_band(h, rc != JEFI_OK ? keep : best);
            if (rc == JEFI_OK) rc = rb;
            if (rc == JEFI_OK && nc > 1) {
                int32_t st = 0;
                JEFI_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost, s));
                JEFI_CUDA(cudaStreamSynchronize(s));
                if (st != 0) rc = st;
            }
            const int mu = mark_use(h, s);
            if (rc == JEFI_OK) rc = mu;
        }
    }
    if (staged_band) *staged_band = h->band;
    return rc;
}

int jefi_valid_window(jefi_handle h, double* t_lo, double* t_hi) {
    if (!h || !t_lo || !t_hi) return JEFI_EINVAL;
    sync_view(h);
    if (h->n_latest < 0) return JEFI_ENOTYET;
    if (!h->any_pairs) {
        *t_lo = -INFINITY;
        *t_hi = INFINITY;
        return JEFI_OK;
    }
    const double c = h->prm.c, dt = h->prm.dt, t0 = h->prm.t0;
    const double rmin = std::sqrt(h->real.s_min), rmax = std::sqrt(h->real.s_max);
    const int64_t ahead = slices_ahead(h);
    auto ok_hi = [&](double t) { return slot_of(h->real.s_min, t - t0, c, dt) + ahead <= h->n_latest; };
    // monotone in t: the farthest pair's slot has not yet fallen out of the ring
    auto ok_lo = [&](double t) {
        const int64_t oldest = h->n_latest - h->H + 1;
        return slot_of(h->real.s_max, t - t0, c, dt) >= oldest;
    };
    // t_hi: largest t with ok_hi, found from the estimate by exact stepping/bisection
    auto refine = [&](double guess, auto pred, bool want_max) {
        double a = guess, b = guess;
        double step = std::max(std::fabs(guess) * 1e-12, 1e-300);
        if (want_max) {
            while (!pred(a)) { a -= step; step *= 2; }
            step = std::max(std::fabs(guess) * 1e-12, 1e-300);
            while (pred(b)) { b += step; step *= 2; }
        } else {
            while (!pred(b)) { b += step; step *= 2; }
            step = std::max(std::fabs(guess) * 1e-12, 1e-300);
            while (pred(a)) { a -= step; step *= 2; }
        }
        // invariant: want_max: pred(a) && !pred(b); else: !pred(a) && pred(b)
        for (int it = 0; it < 200; ++it) {
            double m = a + (b - a) / 2;
            if (m == a || m == b) break;
            if (pred(m) == want_max) a = m; else b = m;
        }
        return want_max ? a : b;
    };
    *t_hi = refine(t0 + (double)(h->n_latest + 1 - ahead) * dt + rmin / c, ok_hi, true);
    if (h->n_latest - h->H + 1 <= 0) {
        *t_lo = -INFINITY;
    } else {
        *t_lo = refine(t0 + (double)(h->n_latest - h->H + 1) * dt + rmax / c, ok_lo, false);
    }
    if (*t_lo > *t_hi) return JEFI_ENOTYET;
    return JEFI_OK;
}

int jefi_get_info(jefi_handle h, jefi_info* out) {
    if (!h || !out) return JEFI_EINVAL;
    sync_view(h);
    for (auto& ev : h->ev_pending) {
        float ms = 0;
        JEFI_CUDA(cudaEventSynchronize(ev.second));
        JEFI_CUDA(cudaEventElapsedTime(&ms, ev.first, ev.second));
        h->sum_ms += ms;
        h->sum_launches++;
        h->ev_free.push_back(ev);
    }
    h->ev_pending.clear();
    unsigned long long fb = 0;
    JEFI_CUDA(cudaMemcpy(&fb, h->fallbacks, sizeof(fb), cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    out->n_src = h->n_src;
    out->n_obs = h->n_obs;
    out->n_latest = h->n_latest;
    out->pairs_per_eval = h->n_src * h->n_obs;
    out->device_bytes = h->device_bytes;
    out->kernel_launches = h->launches;
    out->slot_fallbacks = (int64_t)fb;
    out->sum_launches = h->sum_launches;
    out->sum_ms_total = h->sum_ms;
    out->n_split = h->n_split;
    out->precision = h->prm.precision;
    int32_t st = 0;
    JEFI_CUDA(cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost));
    out->device_status = st;
    out->staged_band = h->band;
    out->tile_shape = h->tile_shape;
    return JEFI_OK;
}

int jefi_reset_stats(jefi_handle h) {
    if (!h) return JEFI_EINVAL;
    jefi_info tmp;
    int rc = jefi_get_info(h, &tmp);
    if (rc != JEFI_OK) return rc;
    h->sum_ms = 0;
    h->sum_launches = 0;
    JEFI_CUDA(cudaMemset(h->fallbacks, 0, sizeof(unsigned long long)));
    return mark_use(h, 0);
}

// ---------------------------------------------------------------- checkpoint / resume
namespace {

constexpr char kCkpMagic[8] = {'J', 'E', 'F', 'I', 'C', 'K', 'P', '1'};
constexpr uint32_t kCkpVersion = 2;    // 2: the ring image holds the P = 4 ceil(H/4) slots of the period

struct CkpHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int32_t src_n[3];
    int32_t H;
    int32_t src_origin[3];
    int32_t pad0;
    double src_lo[3], src_d[3];
    double c, dt, t0;
    int32_t precision, deriv, interp, esz;
    int64_t n_latest;
    int64_t n_cells;                 // brick-padded cells
    int64_t n_src;
    int64_t ring_bytes;              // slots 0..P-1 of every cell (P: the ring's period)
    int64_t state_bytes;             // previous slice (and the one before, central differences)
};

int64_t ckp_ring_bytes(const jefi_problem* h) {
    return (int64_t)h->n_bricks * kBrickCells * h->P * 8 * (h->fp64 ? 8 : 4);
}

int64_t ckp_state_bytes(const jefi_problem* h) {
    return h->n_src * 4 * (int64_t)sizeof(double) * (h->central ? 2 : 1);
}

CkpHeader ckp_header(const jefi_problem* h) {
    CkpHeader c{};
    std::memcpy(c.magic, kCkpMagic, 8);
    c.version = kCkpVersion;
    c.header_bytes = sizeof(CkpHeader);
    for (int a = 0; a < 3; ++a) {
        c.src_n[a] = h->src.n[a];
        c.src_origin[a] = h->org[a];
        c.src_lo[a] = h->src.lo[a];
        c.src_d[a] = h->src.d[a];
    }
    c.H = h->H;
    c.c = h->prm.c;
    c.dt = h->prm.dt;
    c.t0 = h->prm.t0;
    c.precision = h->fp64 ? JEFI_FP64 : JEFI_FP32;   // FP32 and FP32_COMP share the ring format
    c.deriv = h->prm.deriv;
    c.interp = h->interp ? 1 : 0;
    c.esz = h->fp64 ? 8 : 4;
    c.n_latest = h->n_latest;
    c.n_cells = (int64_t)h->n_bricks * kBrickCells;
    c.n_src = h->n_src;
    c.ring_bytes = ckp_ring_bytes(h);
    c.state_bytes = ckp_state_bytes(h);
    return c;
}

}  // namespace

int jefi_checkpoint_bytes(jefi_handle h, size_t* bytes) {
    if (!h || !bytes || h->base) return JEFI_EINVAL;
    *bytes = sizeof(CkpHeader) + (size_t)ckp_ring_bytes(h) + (size_t)ckp_state_bytes(h);
    return JEFI_OK;
}

int jefi_checkpoint(jefi_handle h, void* dst, size_t bytes, void* stream) {
    size_t need = 0;
    const int rc = jefi_checkpoint_bytes(h, &need);
    if (rc != JEFI_OK) return rc;
    if (!dst || bytes < need) return JEFI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const CkpHeader hdr = ckp_header(h);
    unsigned char* out = static_cast<unsigned char*>(dst);
    std::memcpy(out, &hdr, sizeof(hdr));
    unsigned char* ring_out = out + sizeof(hdr);
    const size_t row = (size_t)8 * hdr.esz;
    if (hdr.ring_bytes > 0)
        JEFI_CUDA(cudaMemcpy2DAsync(ring_out, (size_t)h->P * row, h->ring, (size_t)h->Hp * row, (size_t)h->P * row,
                                    (size_t)hdr.n_cells, cudaMemcpyDeviceToHost, s));
    unsigned char* st = ring_out + hdr.ring_bytes;
    const size_t one = (size_t)h->n_src * 4 * sizeof(double);
    if (one > 0) {
        JEFI_CUDA(cudaMemcpyAsync(st, h->prev, one, cudaMemcpyDeviceToHost, s));
        if (h->central) JEFI_CUDA(cudaMemcpyAsync(st + one, h->prev2, one, cudaMemcpyDeviceToHost, s));
    }
    JEFI_CUDA(cudaStreamSynchronize(s));
    return JEFI_OK;
}

int jefi_restore(jefi_handle h, const void* src, size_t bytes, void* stream) {
    size_t need = 0;
    const int rc = jefi_checkpoint_bytes(h, &need);
    if (rc != JEFI_OK) return rc;
    if (!src || bytes < need) return JEFI_EINVAL;
    CkpHeader in;
    std::memcpy(&in, src, sizeof(in));
    const CkpHeader want = ckp_header(h);
    bool same = std::memcmp(in.magic, kCkpMagic, 8) == 0 && in.version == kCkpVersion &&
                in.header_bytes == sizeof(CkpHeader) && in.H == want.H && in.precision == want.precision &&
                in.deriv == want.deriv && in.interp == want.interp && in.esz == want.esz &&
                in.n_cells == want.n_cells && in.n_src == want.n_src && in.ring_bytes == want.ring_bytes &&
                in.state_bytes == want.state_bytes && in.c == want.c && in.dt == want.dt && in.t0 == want.t0 &&
                in.n_latest >= -1 && in.n_latest < ((int64_t)1 << 52);
    for (int a = 0; a < 3; ++a)
        same = same && in.src_n[a] == want.src_n[a] && in.src_lo[a] == want.src_lo[a] &&
               in.src_d[a] == want.src_d[a] && in.src_origin[a] == want.src_origin[a];
    if (!same) return JEFI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned char* ring_in = static_cast<const unsigned char*>(src) + sizeof(CkpHeader);
    const size_t row = (size_t)8 * in.esz;
    if (in.ring_bytes > 0) {
        JEFI_CUDA(cudaMemcpy2DAsync(h->ring, (size_t)h->Hp * row, ring_in, (size_t)h->P * row, (size_t)h->P * row,
                                    (size_t)in.n_cells, cudaMemcpyHostToDevice, s));
        // this handle's mirror rows: slot P + k repeats slot k, k < min(M, P)
        const int m = std::min(h->mirror, h->P);
        if (m > 0)
            JEFI_CUDA(cudaMemcpy2DAsync(static_cast<unsigned char*>(h->ring) + (size_t)h->P * row, (size_t)h->Hp * row,
                                        h->ring, (size_t)h->Hp * row, (size_t)m * row, (size_t)in.n_cells,
                                        cudaMemcpyDeviceToDevice, s));
    }
    const unsigned char* st = ring_in + in.ring_bytes;
    const size_t one = (size_t)h->n_src * 4 * sizeof(double);
    if (one > 0) {
        JEFI_CUDA(cudaMemcpyAsync(h->prev, st, one, cudaMemcpyHostToDevice, s));
        if (h->central) JEFI_CUDA(cudaMemcpyAsync(h->prev2, st + one, one, cudaMemcpyHostToDevice, s));
    }
    JEFI_CUDA(cudaStreamSynchronize(s));
    h->n_latest = in.n_latest;
    return JEFI_OK;
}

// ---------------------------------------------------------------- batch plans
// A fixed batch recorded as CUDA graphs.  The plan's buffer holds what
// jefi_eval_batch puts in its arena (kernel parameters, work-item starts,
// queue counters, reduction items) plus every entry's slot tables, so one
// host-to-device copy per launch refreshes all of it; the kernel parameters
// point at the plan's copy of the tables instead of the handles' own.
}  // extern "C"

struct jefi_batch_plan_s {
    std::vector<jefi_problem*> hs;
    std::vector<double*> E, B;
    std::vector<int> occ;                     // scratch slot of entry i in its handle
    std::vector<int32_t> cap_band, cap_split, cap_bps;   // handle configuration the graphs were recorded with
    struct Tables {                           // byte offsets in the buffer; 0 = absent
        size_t tab32 = 0, theta = 0, times = 0, tab2 = 0, tabg = 0, tabh = 0;
    };
    std::vector<Tables> tabs;                 // per entry; tab32 == 0: nothing to copy
    size_t bytes = 0;
    void* dev = nullptr;
    unsigned char* pinned[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr};
    bool pending[2] = {false, false};
    int next = 0;
    int n_sm = 0;
    bool built = false;
    bool concurrent = true;                   // kernel variants as parallel graph branches
};

namespace {

// Wait for every launch of the plan still in flight (they read its pinned buffers).
int plan_wait(jefi_batch_plan_s* p) {
    for (int j = 0; j < 2; ++j)
        if (p->pending[j]) {
            JEFI_CUDA(cudaEventSynchronize(p->done[j]));
            p->pending[j] = false;
        }
    return JEFI_OK;
}

void plan_release_graphs(jefi_batch_plan_s* p) {
    for (int j = 0; j < 2; ++j) {
        if (p->exec[j]) cudaGraphExecDestroy(p->exec[j]);
        p->exec[j] = nullptr;
        if (p->pinned[j]) cudaFreeHost(p->pinned[j]);
        p->pinned[j] = nullptr;
    }
    if (p->dev) cudaFree(p->dev);
    p->dev = nullptr;
    p->bytes = 0;
    p->built = false;
}

bool plan_stale(const jefi_batch_plan_s* p) {
    if (!p->built) return true;
    for (size_t i = 0; i < p->hs.size(); ++i)
        if (p->hs[i]->band != p->cap_band[i] || p->hs[i]->n_split != p->cap_split[i] ||
            p->hs[i]->bricks_per_split != p->cap_bps[i])
            return true;
    return false;
}

// Record the plan's graphs for the handles' current kernels and splits.
// Earlier launches must have finished (plan_wait).
int plan_build(jefi_batch_plan_s* p) {
    plan_release_graphs(p);
    const int n = (int)p->hs.size();
    BatchLayout L;
    batch_layout(p->hs.data(), p->occ.data(), p->E.data(), p->B.data(), n, &L);
    p->tabs.assign(n, jefi_batch_plan_s::Tables{});
    p->cap_band.resize(n);
    p->cap_split.resize(n);
    p->cap_bps.resize(n);
    for (int i = 0; i < n; ++i) {
        p->cap_band[i] = p->hs[i]->band;
        p->cap_split[i] = p->hs[i]->n_split;
        p->cap_bps[i] = p->hs[i]->bricks_per_split;
    }
    // Every entry's slot tables follow the launch metadata.
    size_t bytes = L.bytes;
    for (const auto& grp : L.groups)
        for (int i : grp.members) {
            const jefi_problem* h = p->hs[i];
            const size_t KT = (size_t)h->K + 2 * kTabGuard;
            auto& tb = p->tabs[i];
            tb.tab32 = bytes;
            bytes = align256(bytes + sizeof(float4) * h->K);
            tb.theta = bytes;
            bytes = align256(bytes + sizeof(double) * theta_stride(h->K));
            tb.times = bytes;
            bytes = align256(bytes + sizeof(TimeParams));
            if (h->band > 0) {
                tb.tab2 = bytes;
                bytes = align256(bytes + sizeof(float2) * KT);
            } else if (h->tabg) {
                tb.tabg = bytes;
                bytes = align256(bytes + sizeof(float2) * KT);
                tb.tabh = bytes;
                bytes = align256(bytes + sizeof(float) * KT);
            }
        }
    if (L.groups.empty() && L.zero_entries.empty()) {   // nothing on the device
        p->built = true;
        return JEFI_OK;
    }
    bytes = std::max<size_t>(bytes, 256);
    if (cudaMalloc(&p->dev, bytes) != cudaSuccess) {
        cudaGetLastError();
        p->dev = nullptr;
        return JEFI_ENOMEM;
    }
    p->bytes = bytes;
    for (int j = 0; j < 2; ++j) {
        if (cudaHostAlloc((void**)&p->pinned[j], bytes, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            p->pinned[j] = nullptr;
            plan_release_graphs(p);
            return JEFI_ENOMEM;
        }
        std::memset(p->pinned[j], 0, bytes);    // queue counters start at zero on every launch
    }

    // Launch metadata, with every entry's kernel parameters pointing at the
    // plan's copy of its tables.
    unsigned char* d = static_cast<unsigned char*>(p->dev);
    const int frc = batch_fill(&L, p->pinned[0], [&](int i) {
        const auto& tb = p->tabs[i];
        SumParams q = make_params(p->hs[i], 1, p->occ[i], nullptr);
        q.tab32 = reinterpret_cast<const float4*>(d + tb.tab32);
        q.theta = reinterpret_cast<const double*>(d + tb.theta);
        q.times = reinterpret_cast<const TimeParams*>(d + tb.times);
        q.tab2 = tb.tab2 ? reinterpret_cast<const float2*>(d + tb.tab2) : nullptr;
        q.tabg = tb.tabg ? reinterpret_cast<const float2*>(d + tb.tabg) : nullptr;
        q.tabh = tb.tabh ? reinterpret_cast<const float*>(d + tb.tabh) : nullptr;
        return q;
    });
    if (frc != JEFI_OK) {
        plan_release_graphs(p);
        return frc;
    }
    std::memcpy(p->pinned[1], p->pinned[0], bytes);

    // Record: [zero fields] -> copy -> one persistent launch per group -> reduction.
    // Concurrent: the groups' launches are parallel branches between the copy
    // and the reduction (their items are independent), so the device can
    // start one variant's items while another's last items finish.
    const size_t ng = L.groups.size();
    const bool fork = p->concurrent && ng > 1;
    cudaStream_t cs = nullptr;
    std::vector<cudaStream_t> side(fork ? ng : 0, nullptr);
    std::vector<cudaEvent_t> evs(fork ? ng + 1 : 0, nullptr);
    int rc = JEFI_OK;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) rc = JEFI_ECUDA;
    for (auto& x : side)
        if (rc == JEFI_OK && cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) rc = JEFI_ECUDA;
    for (auto& x : evs)
        if (rc == JEFI_OK && cudaEventCreateWithFlags(&x, cudaEventDisableTiming) != cudaSuccess) rc = JEFI_ECUDA;
    for (int j = 0; j < 2 && rc == JEFI_OK; ++j) {
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            rc = JEFI_ECUDA;
            break;
        }
        cudaError_t e = cudaSuccess;
        for (int i : L.zero_entries) {
            const size_t fb = sizeof(double) * 3 * p->hs[i]->n_obs;
            if (e == cudaSuccess) e = cudaMemsetAsync(p->E[i], 0, fb, cs);
            if (e == cudaSuccess) e = cudaMemsetAsync(p->B[i], 0, fb, cs);
        }
        if (e == cudaSuccess && ng > 0) e = cudaMemcpyAsync(d, p->pinned[j], bytes, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess && fork) e = cudaEventRecord(evs[ng], cs);
        for (size_t g = 0; g < ng && e == cudaSuccess; ++g) {
            const cudaStream_t gs = fork ? side[g] : cs;
            if (fork) e = cudaStreamWaitEvent(gs, evs[ng], 0);
            if (e == cudaSuccess) e = batch_launch_group(L, g, p->hs.data(), d, p->n_sm, gs);
            if (e == cudaSuccess && fork) e = cudaEventRecord(evs[g], gs);
            if (e == cudaSuccess && fork) e = cudaStreamWaitEvent(cs, evs[g], 0);
        }
        if (e == cudaSuccess && ng > 0) e = batch_launch_reduce(L, d, cs);
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = ee;
        if (e == cudaSuccess && graph) e = cudaGraphInstantiate(&p->exec[j], graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess || !p->exec[j]) {
            cudaGetLastError();
            rc = JEFI_ECUDA;
        }
    }
    if (cs) cudaStreamDestroy(cs);
    for (auto x : side)
        if (x) cudaStreamDestroy(x);
    for (auto x : evs)
        if (x) cudaEventDestroy(x);
    if (rc != JEFI_OK) {
        plan_release_graphs(p);
        return rc;
    }
    p->built = true;
    return JEFI_OK;
}

// Every entry's time must be in its window; graphs recorded for the
// handles' current configuration.
int plan_check(jefi_batch_plan_s* p, const double* t) {
    for (size_t i = 0; i < p->hs.size(); ++i) {
        sync_view(p->hs[i]);
        const int rc = check_time(p->hs[i], t[i]);
        if (rc != JEFI_OK) return rc;
    }
    if (plan_stale(p)) {
        int rc = plan_wait(p);
        if (rc == JEFI_OK) rc = plan_build(p);
        if (rc != JEFI_OK) return rc;
    }
    return JEFI_OK;
}

// Slot tables of every entry at its time into pinned copy j (after the
// launch that last read that copy has finished).
int plan_prepare(jefi_batch_plan_s* p, int j, const double* t) {
    if (p->pending[j]) {
        JEFI_CUDA(cudaEventSynchronize(p->done[j]));
        p->pending[j] = false;
    }
    if (!p->pinned[j]) return JEFI_OK;
    unsigned char* host = p->pinned[j];
    for (size_t i = 0; i < p->hs.size(); ++i) {
        const auto& tb = p->tabs[i];
        if (!tb.tab32) continue;
        jefi_problem* h = p->hs[i];
        const int o = p->occ[i];
        const size_t K = (size_t)h->K, KT = K + 2 * kTabGuard;
        build_tables(h, o, t[i]);
        std::memcpy(host + tb.tab32, h->h_tab.data() + o * K, sizeof(float4) * K);
        std::memcpy(host + tb.theta, h->h_theta.data() + o * theta_stride((int)K), sizeof(double) * theta_stride((int)K));
        std::memcpy(host + tb.times, &h->h_times[o], sizeof(TimeParams));
        if (tb.tab2) std::memcpy(host + tb.tab2, h->h_tab2.data() + o * KT, sizeof(float2) * KT);
        if (tb.tabg) {
            std::memcpy(host + tb.tabg, h->h_tabg.data() + o * KT, sizeof(float2) * KT);
            std::memcpy(host + tb.tabh, h->h_tabh.data() + o * KT, sizeof(float) * KT);
        }
    }
    return JEFI_OK;
}

int plan_submit(jefi_batch_plan_s* p, int j, cudaStream_t s) {
    if (p->exec[j]) {
        JEFI_CUDA(cudaGraphLaunch(p->exec[j], s));
        JEFI_CUDA(cudaEventRecord(p->done[j], s));
        p->pending[j] = true;
    }
    for (jefi_problem* h : p->hs) {
        const int rc = mark_use(h, s);
        if (rc != JEFI_OK) return rc;
    }
    return JEFI_OK;
}

// Split the source bricks of h into about `want` parts (at most the count
// its partial sums were sized for at creation).
void set_splits(jefi_problem* h, int64_t want) {
    want = std::max<int64_t>(1, std::min<int64_t>(want, h->n_split_max));
    const int64_t nb = std::max<int32_t>(h->n_bricks, 1);
    h->bricks_per_split = (int32_t)std::max<int64_t>(1, (nb + want - 1) / want);
    h->n_split = (int32_t)std::max<int64_t>(1, (nb + h->bricks_per_split - 1) / h->bricks_per_split);
}

// Device time of one launch of the plan at t, after one untimed launch, in ms.
int plan_time(jefi_batch_plan_s* p, const double* t, cudaStream_t s, double* ms) {
    int rc = plan_wait(p);
    if (rc == JEFI_OK && plan_stale(p)) rc = plan_build(p);
    if (rc != JEFI_OK) return rc;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) rc = JEFI_ECUDA;
    if (rc == JEFI_OK) rc = plan_prepare(p, 0, t);
    if (rc == JEFI_OK) rc = plan_submit(p, 0, s);
    if (rc == JEFI_OK) rc = plan_prepare(p, 1, t);
    if (rc == JEFI_OK && cudaEventRecord(ev[0], s) != cudaSuccess) rc = JEFI_ECUDA;
    if (rc == JEFI_OK) rc = plan_submit(p, 1, s);
    float f = 0.f;
    if (rc == JEFI_OK && (cudaEventRecord(ev[1], s) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
                          cudaEventElapsedTime(&f, ev[0], ev[1]) != cudaSuccess))
        rc = JEFI_ECUDA;
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (rc == JEFI_ECUDA) cudaGetLastError();
    p->next = 0;
    *ms = f;
    return rc;
}

}  // namespace

extern "C" {

int jefi_batch_plan_create(const jefi_handle* hs, double* const* E, double* const* B, int32_t n,
                           jefi_batch_plan* out) {
    NvtxRange nvtx_range("jefi_batch_plan_create");
    if (!out || n < 0 || (n > 0 && (!hs || !E || !B))) return JEFI_EINVAL;
    *out = nullptr;
    std::map<jefi_problem*, int> count;
    std::vector<int> occ(n);
    for (int i = 0; i < n; ++i) {
        jefi_problem* h = hs[i];
        if (!h) return JEFI_EINVAL;
        if (h->n_obs > 0 && (!E[i] || !B[i])) return JEFI_EINVAL;
        occ[i] = count[h]++;
        if (occ[i] >= h->time_chunk) return JEFI_EUNSUPPORTED;   // scratch slots per handle
    }
    jefi_batch_plan_s* p = new (std::nothrow) jefi_batch_plan_s();
    if (!p) return JEFI_ENOMEM;
    p->hs.assign(hs, hs + n);
    p->E.assign(E, E + n);
    p->B.assign(B, B + n);
    p->occ = occ;
    int dev = 0;
    int rc = JEFI_OK;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->done[1], cudaEventDisableTiming) != cudaSuccess)
        rc = JEFI_ECUDA;
    for (int i = 0; i < n && rc == JEFI_OK; ++i) sync_view(p->hs[i]);
    if (rc == JEFI_OK) rc = plan_build(p);
    if (rc != JEFI_OK) {
        cudaGetLastError();
        plan_release_graphs(p);
        for (cudaEvent_t e : p->done)
            if (e) cudaEventDestroy(e);
        delete p;
        return rc;
    }
    for (auto& kv : count) kv.first->n_plans++;
    *out = p;
    return JEFI_OK;
}

int jefi_batch_plan_launch(jefi_batch_plan p, const double* t, void* stream) {
    NvtxRange nvtx_range("jefi_batch_plan_launch");
    if (!p || (!t && !p->hs.empty())) return JEFI_EINVAL;
    if (p->hs.empty()) return JEFI_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = plan_check(p, t);
    const int j = p->next;
    if (rc == JEFI_OK) rc = plan_prepare(p, j, t);
    if (rc == JEFI_OK) rc = plan_submit(p, j, s);
    if (rc == JEFI_OK) p->next ^= 1;
    return rc;
}

// ---------------------------------------------------------------- tune cache
// What decides a handle's kernels' work, hashed: the tune cache's key part.
static uint64_t handle_signature(const jefi_problem* h) {
    uint64_t s = kFnvBasis;
    s = fnv1a(s, &h->src, sizeof(h->src));
    s = fnv1a(s, h->org, sizeof(h->org));
    s = fnv1a(s, &h->obs_sig, sizeof(h->obs_sig));
    const int32_t ints[11] = {h->H, h->prm.precision, h->prm.deriv, (int32_t)(h->prm.flags & ~JEFI_FLAG_STATS),
                              h->interp ? 1 : 0, h->band0, h->band_alt, h->n_split_max, h->tile_shape,
                              h->base ? 1 : 0, h->mirror};
    s = fnv1a(s, ints, sizeof(ints));
    const double dbl[3] = {h->prm.dt, h->prm.c, h->prm.t0};
    return fnv1a(s, dbl, sizeof(dbl));
}

static uint64_t plan_signature(const jefi_batch_plan_s* p, int n_sm) {
    uint64_t s = fnv1a(kFnvBasis, &n_sm, sizeof(n_sm));
    for (const jefi_problem* h : p->hs) {
        const uint64_t hs = handle_signature(h);
        s = fnv1a(s, &hs, sizeof(hs));
    }
    return s;
}

struct TuneChoice {
    int concurrent = 1, divisor = 0;
    std::vector<int32_t> bands;     // per distinct handle, in order of first appearance
};

// The last line of the cache file with this key; false on a miss (or no file).
static bool tune_cache_find(const char* path, uint64_t key, size_t u, TuneChoice* out) {
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[65536];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        unsigned long long k = 0;
        int conc = 0, div = 0, n = 0, pos = 0;
        if (std::sscanf(line, "jefi-tune-1 %llx %d %d %d%n", &k, &conc, &div, &n, &pos) != 4 || k != key ||
            n != (int)u)
            continue;
        TuneChoice c;
        c.concurrent = conc;
        c.divisor = div;
        const char* q = line + pos;
        bool ok = true;
        for (int i = 0; i < n && ok; ++i) {
            int b = 0, used = 0;
            ok = std::sscanf(q, "%d%n", &b, &used) == 1;
            q += used;
            c.bands.push_back(b);
        }
        if (ok) {
            *out = c;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

static void tune_cache_store(const char* path, uint64_t key, const TuneChoice& c) {
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "jefi-tune-1 %016llx %d %d %d", (unsigned long long)key, c.concurrent, c.divisor,
                 (int)c.bands.size());
    for (int32_t b : c.bands) std::fprintf(f, " %d", b);
    std::fprintf(f, "\n");
    std::fclose(f);
}

int jefi_batch_plan_tune(jefi_batch_plan p, const double* t, void* stream, jefi_tune_report* report) {
    NvtxRange nvtx_range("jefi_batch_plan_tune");
    if (!p || (!t && !p->hs.empty())) return JEFI_EINVAL;
    jefi_tune_report rep{};
    rep.split_divisor = 1;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = plan_check(p, t);
    if (rc != JEFI_OK) return rc;
    // distinct handles with pairs, in order of first appearance, and one time each
    std::vector<jefi_problem*> uniq;
    std::vector<double> t_of;
    for (size_t i = 0; i < p->hs.size(); ++i) {
        jefi_problem* h = p->hs[i];
        if (!h->any_pairs || h->n_obs == 0 || std::find(uniq.begin(), uniq.end(), h) != uniq.end()) continue;
        uniq.push_back(h);
        t_of.push_back(t[i]);
    }
    const size_t u = uniq.size();
    std::vector<int32_t> band_in(u), split_in(u), bps_in(u), band_meas(u);
    for (size_t k = 0; k < u; ++k) {
        band_in[k] = uniq[k]->band;
        split_in[k] = uniq[k]->n_split;
        bps_in[k] = uniq[k]->bricks_per_split;
    }
    auto restore = [&]() {
        for (size_t k = 0; k < u; ++k) {
            set_band(uniq[k], band_in[k]);
            uniq[k]->n_split = split_in[k];
            uniq[k]->bricks_per_split = bps_in[k];
        }
    };
    double ms = 0;
    // a choice stored for this plan's geometry: applied and timed once
    const char* cache_path = std::getenv("JEFI_TUNE_CACHE");
    const uint64_t cache_key = plan_signature(p, p->n_sm);
    TuneChoice hit;
    if (cache_path && cache_path[0] && tune_cache_find(cache_path, cache_key, u, &hit)) {
        bool ok = true;
        for (size_t k = 0; k < u && ok; ++k) {
            const int32_t b = hit.bands[k];
            jefi_problem* h = uniq[k];
            ok = b == h->band || (!h->fp64 && ((b > 0 && (b == h->band0 || b == h->band_alt)) ||
                                                (b == 0 && h->band0 > 0 && direct_possible(h))));
        }
        ok = ok && (hit.divisor == 0 || hit.divisor == 1 || hit.divisor == 2 || hit.divisor == 4 || hit.divisor == 8);
        if (ok) {
            p->concurrent = hit.concurrent != 0;
            p->built = false;
            for (size_t k = 0; k < u && rc == JEFI_OK; ++k) {
                rc = set_band(uniq[k], hit.bands[k]);
                if (hit.divisor > 0) set_splits(uniq[k], (uniq[k]->n_split_max + hit.divisor - 1) / hit.divisor);
            }
            if (rc == JEFI_OK) rc = plan_wait(p);
            if (rc == JEFI_OK && plan_stale(p)) rc = plan_build(p);
            if (rc == JEFI_OK) rc = plan_time(p, t, s, &ms);
            if (rc != JEFI_OK) {
                restore();
                return rc;
            }
            rep.candidates = 1;
            rep.ms_initial = rep.ms_tuned = ms;
            rep.split_divisor = hit.divisor;
            rep.concurrent_groups = p->concurrent ? 1 : 0;
            rep.from_cache = 1;
            for (size_t k = 0; k < u; ++k) {
                if (uniq[k]->band != band_in[k]) rep.measured_kernels = 1;
                if (uniq[k]->band > 0 && uniq[k]->band == uniq[k]->band_alt) rep.widened_bands++;
            }
            for (jefi_problem* h : p->hs)
                if (!h->fp64 && h->band > 0 && h->any_pairs && h->n_obs > 0) rep.staged_problems++;
            if (report) *report = rep;
            return JEFI_OK;
        }
    }
    rc = plan_time(p, t, s, &ms);
    if (rc != JEFI_OK) return rc;
    rep.candidates = 1;
    rep.ms_initial = ms;
    double best_ms = ms;
    int best_pol = 0, best_div = 0;   // best_div 0: splits as they were

    // Kernel variants in parallel graph branches or one after another: kept
    // for the remaining candidates.
    p->concurrent = !p->concurrent;
    p->built = false;
    rc = plan_time(p, t, s, &ms);
    if (rc != JEFI_OK) {
        p->concurrent = !p->concurrent;
        p->built = false;
        return rc;
    }
    rep.candidates++;
    if (ms < best_ms) {
        best_ms = ms;
    } else {
        p->concurrent = !p->concurrent;
        p->built = false;
    }

    // Kernel choice measured per FP32 handle that has both kernels.
    bool differs = false;
    for (size_t k = 0; k < u && rc == JEFI_OK; ++k) {
        jefi_problem* h = uniq[k];
        band_meas[k] = h->band;
        if (h->fp64 || h->band0 == 0) continue;
        int32_t b = h->band;
        rc = jefi_select_kernel(h, JEFI_KERNEL_MEASURE, t_of[k], &b, stream);
        band_meas[k] = b;
        set_band(h, band_in[k]);
        differs = differs || b != band_in[k];
    }
    const int divs[4] = {1, 2, 4, 8};
    for (int pol = 0; pol < 2 && rc == JEFI_OK; ++pol) {
        if (pol == 1 && !differs) break;
        std::vector<std::vector<int32_t>> seen;
        if (pol == 0) seen.push_back(split_in);
        for (int dv : divs) {
            for (size_t k = 0; k < u; ++k) {
                set_band(uniq[k], pol ? band_meas[k] : band_in[k]);
                set_splits(uniq[k], (uniq[k]->n_split_max + dv - 1) / dv);
            }
            std::vector<int32_t> cur(u);
            for (size_t k = 0; k < u; ++k) cur[k] = uniq[k]->n_split;
            if (std::find(seen.begin(), seen.end(), cur) != seen.end()) continue;
            seen.push_back(cur);
            rc = plan_time(p, t, s, &ms);
            if (rc != JEFI_OK) break;
            rep.candidates++;
            if (ms < best_ms) {
                best_ms = ms;
                best_pol = pol;
                best_div = dv;
            }
        }
    }
    restore();
    if (rc != JEFI_OK) return rc;
    for (size_t k = 0; k < u; ++k) {
        if (best_pol == 1) set_band(uniq[k], band_meas[k]);
        if (best_div > 0) set_splits(uniq[k], (uniq[k]->n_split_max + best_div - 1) / best_div);
    }
    rc = plan_wait(p);
    if (rc == JEFI_OK && plan_stale(p)) rc = plan_build(p);
    if (rc != JEFI_OK) return rc;
    rep.split_divisor = best_div > 0 ? best_div : 0;
    rep.measured_kernels = best_pol;
    rep.concurrent_groups = p->concurrent ? 1 : 0;
    rep.ms_tuned = best_ms;
    for (jefi_problem* h : p->hs)
        if (!h->fp64 && h->band > 0 && h->any_pairs && h->n_obs > 0) {
            rep.staged_problems++;
            if (h->band == h->band_alt) rep.widened_bands++;
        }
    if (cache_path && cache_path[0]) {
        TuneChoice c;
        c.concurrent = p->concurrent ? 1 : 0;
        c.divisor = rep.split_divisor;
        for (size_t k = 0; k < u; ++k) c.bands.push_back(uniq[k]->band);
        tune_cache_store(cache_path, cache_key, c);
    }
    if (report) *report = rep;
    return JEFI_OK;
}

int jefi_batch_plan_destroy(jefi_batch_plan p) {
    if (!p) return JEFI_EINVAL;
    plan_wait(p);
    plan_release_graphs(p);
    for (cudaEvent_t e : p->done)
        if (e) cudaEventDestroy(e);
    std::map<jefi_problem*, int> seen;
    for (jefi_problem* h : p->hs)
        if (seen[h]++ == 0) h->n_plans--;
    delete p;
    return JEFI_OK;
}

// ---------------------------------------------------------------- S-O decomposition
int jefi_so_partition(const jefi_grid* src, const int32_t* parts, jefi_grid* sub, int32_t* origin) {
    if (!src || !parts || !sub || !origin) return JEFI_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (parts[a] < 1 || parts[a] > 4096 || src->n[a] < 0) return JEFI_EINVAL;
    // per axis: part k holds bricks [k nb / p, (k + 1) nb / p) of the nb = ceil(n / 4)
    // bricks, i.e. cells [4 b0, min(4 b1, n))
    std::vector<int32_t> first[3], count[3];
    for (int a = 0; a < 3; ++a) {
        const int64_t nb = (src->n[a] + 3) / 4, p = parts[a];
        for (int64_t k = 0; k < p; ++k) {
            const int64_t b0 = k * nb / p, b1 = (k + 1) * nb / p;
            const int64_t c0 = std::min<int64_t>(4 * b0, src->n[a]), c1 = std::min<int64_t>(4 * b1, src->n[a]);
            first[a].push_back((int32_t)c0);
            count[a].push_back((int32_t)(c1 - c0));
        }
    }
    int64_t k = 0;
    for (int kz = 0; kz < parts[2]; ++kz)
        for (int ky = 0; ky < parts[1]; ++ky)
            for (int kx = 0; kx < parts[0]; ++kx, ++k) {
                const int idx[3] = {kx, ky, kz};
                for (int a = 0; a < 3; ++a) {
                    sub[k].n[a] = count[a][idx[a]];
                    sub[k].lo[a] = src->lo[a];
                    sub[k].d[a] = src->d[a];
                    origin[3 * k + a] = first[a][idx[a]];
                }
            }
    return JEFI_OK;
}

int jefi_sum_fields(int32_t n_parts, const double* const* E_parts, const double* const* B_parts, int64_t n_obs,
                    double* E, double* B, void* stream) {
    NvtxRange nvtx_range("jefi_sum_fields");
    if (n_parts < 1 || n_parts > kMaxSumParts || !E_parts || !B_parts || n_obs < 0 || (n_obs > 0 && (!E || !B)))
        return JEFI_EINVAL;
    SumPartsParams p{};
    p.n_parts = n_parts;
    p.n = n_obs * 3;
    for (int k = 0; k < n_parts; ++k) {
        if (n_obs > 0 && (!E_parts[k] || !B_parts[k])) return JEFI_EINVAL;
        p.E_parts[k] = E_parts[k];
        p.B_parts[k] = B_parts[k];
    }
    p.E = E;
    p.B = B;
    JEFI_CUDA(launch_sum_parts(p, (cudaStream_t)stream));
    return JEFI_OK;
}

int jefi_destroy(jefi_handle h) {
    if (!h) return JEFI_EINVAL;
    if (h->n_views > 0) return JEFI_EINVAL;              // destroy the views first
    if (h->n_plans > 0) return JEFI_EINVAL;              // destroy the batch plans first
    // the handle's own work only: other streams and handles keep running
    if (h->last_use) cudaEventSynchronize(h->last_use);
    if (h->base) h->base->n_views--;
    release_all(h);
    delete h;
    return JEFI_OK;
}

}  // extern "C"
