// jefi_noalloc.cu -- jefi_eval_fields_noalloc: a one-shot FP64 evaluation
// that allocates no device memory.
//
// Some callers cannot allocate device memory when they need fields: a host
// application that hands all device memory to its own pool allocator and
// forbids outside cudaMalloc calls, or a time-critical loop where cudaMalloc /
// cudaFree would synchronise the device.  This entry point serves them.  The
// caller passes every input and output as device buffers; the only working
// memory is the file-scope array below, which each GPU that loads the library
// holds until the process exits.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress, which also loads this
// module on the device, and the device's SM count; make that first call
// before any stream capture begins.  Each call returns after its kernels have
// finished on the caller's stream (it reads the status word back).
// Every call shares the array and it keeps the last call's contents; the call
// clears what must start at zero.  Calls that overlap on the GPU (different
// streams or host threads) race on the array and must be serialised by the
// caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "jefi.h"
#include "jefi_device.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kBrickEdge = 4;
constexpr int kCellsPerBrick = 64;
constexpr size_t kHeaderBytes = 256;          // status word, rest unused
constexpr int kMaxAxisCells = 6144;           // total padded cells over the three axes (48 KB)
constexpr int kMaxDevices = 64;

}  // namespace

// Working memory of jefi_eval_fields_noalloc: [status | partial sums].
static __device__ __align__(256) unsigned char g_noalloc_scratch[JEFI_NOALLOC_SCRATCH_BYTES];

namespace {

struct NoallocParams {
    int32_t nx, ny, nz, nbx, nby, nbz, n_bricks;
    int32_t n_slots, n_split, bricks_per_split;
    int64_t n_src, n_obs, n_slices;
    double lo[3], d[3], screen[3];
    double T, c, dt;
    const double* obs;
    const double* rho;
    const double* J;
    double* partials;     // [n_split][6][n_slots]
    int32_t* status;
};

// Variant of the FP64 sum kernel that reads the caller's plain FP64 history
// (slice-major, cells x fastest) instead of the library's ring, forms the
// backward difference of Eq. E-1 on the fly and evaluates the slot of
// Eq. tr-1 with the FP64 operations as written.
__global__ void __launch_bounds__(kThreads, 1) noalloc_sum_f64(const NoallocParams p) {
    extern __shared__ double s_axis[];
    const int npx = kBrickEdge * p.nbx, npy = kBrickEdge * p.nby, npz = kBrickEdge * p.nbz;
    double* s_x = s_axis;
    double* s_y = s_x + npx;
    double* s_z = s_y + npy;
    for (int i = threadIdx.x; i < npx; i += kThreads) s_x[i] = jefi::dev::cell_center(p.lo[0], p.d[0], i);
    for (int i = threadIdx.x; i < npy; i += kThreads) s_y[i] = jefi::dev::cell_center(p.lo[1], p.d[1], i);
    for (int i = threadIdx.x; i < npz; i += kThreads) s_z[i] = jefi::dev::cell_center(p.lo[2], p.d[2], i);
    __syncthreads();

    const int slot = blockIdx.x * kThreads + threadIdx.x;
    const int64_t o = slot < p.n_obs ? slot : p.n_obs - 1;   // padding threads repeat a point
    const double xo = p.obs[3 * o + 0], yo = p.obs[3 * o + 1], zo = p.obs[3 * o + 2];
    double se[3] = {0, 0, 0}, sb[3] = {0, 0, 0};
    const int b_begin = blockIdx.y * p.bricks_per_split;
    const int b_end = min(b_begin + p.bricks_per_split, p.n_bricks);
    const int64_t Ns = p.n_src;
    for (int b = b_begin; b < b_end; ++b) {
        const int bx = b % p.nbx;
        const int rest = b / p.nbx;
        const int by = rest % p.nby;
        const int bz = rest / p.nby;
        for (int cl = 0; cl < kCellsPerBrick; ++cl) {
            const int ix = kBrickEdge * bx + (cl & 3);
            const int iy = kBrickEdge * by + ((cl >> 2) & 3);
            const int iz = kBrickEdge * bz + (cl >> 4);
            if (ix >= p.nx || iy >= p.ny || iz >= p.nz) continue;
            const double dx = __dsub_rn(xo, s_x[ix]);
            const double dy = __dsub_rn(yo, s_y[iy]);
            const double dz = __dsub_rn(zo, s_z[iz]);
            if (fabs(dx) <= p.screen[0] && fabs(dy) <= p.screen[1] && fabs(dz) <= p.screen[2]) continue;
            const double S = jefi::dev::spec_s64(dx, dy, dz);
            const double u = __ddiv_rn(__dsub_rn(p.T, __ddiv_rn(__dsqrt_rn(S), p.c)), p.dt);
            if (!(u >= 0.0)) continue;                      // slot < 0: no source yet
            if (u >= (double)p.n_slices) {                  // needs a slice not given
                atomicExch(p.status, (int)JEFI_ENOTYET);
                continue;
            }
            const int64_t n = (int64_t)floor(u);
            const int64_t cell = ((int64_t)iz * p.ny + iy) * p.nx + ix;
            const double r = p.rho[n * Ns + cell];
            const double* Jn = p.J + 3 * (n * Ns + cell);
            const int64_t prev = n >= 1 ? (n - 1) * Ns + cell : -1;   // slice n-1, or none
            const double rp = prev >= 0 ? p.rho[prev] : 0.0;
            double dj[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                dj[a] = __ddiv_rn(__dsub_rn(Jn[a], prev >= 0 ? p.J[3 * prev + a] : 0.0), p.dt);
            const double dr = __ddiv_rn(__dsub_rn(r, rp), p.dt);
            // channels c*rho, J, drho, dJ/c as the ring stores them
            const double ch0 = __dmul_rn(p.c, r);
            const double g0 = __ddiv_rn(dj[0], p.c), g1 = __ddiv_rn(dj[1], p.c), g2 = __ddiv_rn(dj[2], p.c);
            const double ri = rsqrt(S);
            const double r2 = ri * ri;
            const double r3 = r2 * ri;
            const double q = fma(dr, r2, ch0 * r3);
            se[0] = fma(dx, q, se[0]);
            se[1] = fma(dy, q, se[1]);
            se[2] = fma(dz, q, se[2]);
            se[0] = fma(-g0, ri, se[0]);
            se[1] = fma(-g1, ri, se[1]);
            se[2] = fma(-g2, ri, se[2]);
            const double vx = fma(g0, r2, Jn[0] * r3);
            const double vy = fma(g1, r2, Jn[1] * r3);
            const double vz = fma(g2, r2, Jn[2] * r3);
            sb[0] = fma(vy, dz, sb[0]);
            sb[1] = fma(vz, dx, sb[1]);
            sb[2] = fma(vx, dy, sb[2]);
            sb[0] = fma(-vz, dy, sb[0]);
            sb[1] = fma(-vx, dz, sb[1]);
            sb[2] = fma(-vy, dx, sb[2]);
        }
    }
    double* out = p.partials + (size_t)blockIdx.y * 6 * p.n_slots + slot;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        out[(size_t)a * p.n_slots] = se[a];
        out[(size_t)(3 + a) * p.n_slots] = sb[a];
    }
}

// Sum the splits in order, scale, write E and B in the caller's point order.
__global__ void noalloc_reduce(const double* partials, int64_t n_obs, int n_slots, int n_split,
                               double e_scale, double b_scale, double* E, double* B) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_obs) return;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int s = 0; s < n_split; ++s) {
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += partials[((size_t)s * 6 + c) * n_slots + o];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        E[3 * o + a] = acc[a] * e_scale;
        B[3 * o + a] = acc[3 + a] * b_scale;
    }
}

std::mutex g_setup_lock;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

// Device address of the scratch array on the current device and the
// device's SM count (set-up on first use).
int scratch_on_current_device(unsigned char** out, int* n_sm) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return JEFI_ECUDA;
    std::lock_guard<std::mutex> guard(g_setup_lock);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        int sms = 0;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
            cudaGetLastError();
            return JEFI_ECUDA;
        }
        g_sm_count[dev] = sms;
        g_scratch_ptr[dev] = static_cast<unsigned char*>(ptr);
    }
    *out = g_scratch_ptr[dev];
    *n_sm = g_sm_count[dev];
    return JEFI_OK;
}

}  // namespace

extern "C" int jefi_eval_fields_noalloc(const jefi_grid* src, const double* obs, int64_t n_obs,
                                        const double* rho, const double* J, int64_t n_slices,
                                        const jefi_params* prm, double t, double* E, double* B,
                                        void* stream) {
    if (!src || !prm || n_obs < 0 || n_slices < 0) return JEFI_EINVAL;
    if (!(prm->c > 0) || !std::isfinite(prm->c) || !(prm->dt > 0) || !std::isfinite(prm->dt) ||
        !std::isfinite(prm->t0) || !std::isfinite(prm->k_e) || !std::isfinite(prm->k_b) || !std::isfinite(t))
        return JEFI_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (src->n[a] < 0 || !(src->d[a] > 0) || !std::isfinite(src->d[a]) || !std::isfinite(src->lo[a]) ||
            !std::isfinite(prm->screen[a]))
            return JEFI_EINVAL;
    if (n_obs == 0) return JEFI_OK;
    if (!obs || !E || !B) return JEFI_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n_src = (int64_t)src->n[0] * src->n[1] * src->n[2];
    if (n_src == 0 || n_slices == 0) {                 // no sources: zero fields
        if (cudaMemsetAsync(E, 0, sizeof(double) * 3 * n_obs, s) != cudaSuccess ||
            cudaMemsetAsync(B, 0, sizeof(double) * 3 * n_obs, s) != cudaSuccess)
            return JEFI_ECUDA;
        return cudaStreamSynchronize(s) == cudaSuccess ? JEFI_OK : JEFI_ECUDA;
    }
    if (!rho || !J) return JEFI_EINVAL;

    NoallocParams p{};
    p.nx = src->n[0];
    p.ny = src->n[1];
    p.nz = src->n[2];
    p.nbx = (p.nx + 3) / 4;
    p.nby = (p.ny + 3) / 4;
    p.nbz = (p.nz + 3) / 4;
    const int64_t n_bricks = (int64_t)p.nbx * p.nby * p.nbz;
    const int64_t axis_cells = 4LL * (p.nbx + p.nby + p.nbz);
    if (axis_cells > kMaxAxisCells || n_bricks > INT32_MAX) return JEFI_EUNSUPPORTED;
    p.n_bricks = (int32_t)n_bricks;
    const int64_t n_tiles = (n_obs + kThreads - 1) / kThreads;
    const int64_t n_slots = n_tiles * kThreads;
    // Capacity: the partial sums [n_split][6][n_slots] FP64 must fit the array.
    const int64_t cap = (int64_t)(JEFI_NOALLOC_SCRATCH_BYTES - kHeaderBytes) / (int64_t)(6 * sizeof(double));
    if (n_slots > cap) return JEFI_EUNSUPPORTED;       // more points than the array can hold
    unsigned char* scratch = nullptr;
    int n_sm = 0;
    int rc = scratch_on_current_device(&scratch, &n_sm);
    if (rc != JEFI_OK) return rc;
    // two CTAs per SM over tiles x source splits
    int64_t n_split = std::max<int64_t>(1, (2 * (int64_t)n_sm + n_tiles - 1) / n_tiles);
    n_split = std::min<int64_t>(n_split, std::min<int64_t>(n_bricks, cap / n_slots));
    p.bricks_per_split = (int32_t)((n_bricks + n_split - 1) / n_split);
    p.n_split = (int32_t)((n_bricks + p.bricks_per_split - 1) / p.bricks_per_split);
    p.n_slots = (int32_t)n_slots;
    p.n_src = n_src;
    p.n_obs = n_obs;
    p.n_slices = n_slices;
    for (int a = 0; a < 3; ++a) {
        p.lo[a] = src->lo[a];
        p.d[a] = src->d[a];
        p.screen[a] = prm->screen[a] < 0 ? src->d[a] / 2 : prm->screen[a];
    }
    p.T = t - prm->t0;
    p.c = prm->c;
    p.dt = prm->dt;
    p.obs = obs;
    p.rho = rho;
    p.J = J;

    p.status = reinterpret_cast<int32_t*>(scratch);
    p.partials = reinterpret_cast<double*>(scratch + kHeaderBytes);

    // the status word must start at zero; every partial sum is overwritten
    if (cudaMemsetAsync(p.status, 0, sizeof(int32_t), s) != cudaSuccess) return JEFI_ECUDA;
    const dim3 grid((unsigned)n_tiles, (unsigned)p.n_split);
    noalloc_sum_f64<<<grid, kThreads, sizeof(double) * axis_cells, s>>>(p);
    if (cudaGetLastError() != cudaSuccess) return JEFI_ECUDA;
    const double dV = src->d[0] * src->d[1] * src->d[2];
    noalloc_reduce<<<(unsigned)((n_obs + 255) / 256), 256, 0, s>>>(
        p.partials, n_obs, p.n_slots, p.n_split, prm->k_e * dV / prm->c, prm->k_b * dV, E, B);
    if (cudaGetLastError() != cudaSuccess) return JEFI_ECUDA;
    int32_t status = 0;
    if (cudaMemcpyAsync(&status, p.status, sizeof(status), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return JEFI_ECUDA;
    return status;
}
