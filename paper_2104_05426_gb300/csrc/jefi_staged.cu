// jefi_staged.cu -- the TMA-staged FP32 sum: launches of the narrow band
// heights (16 and 24 slots, whole-brick stages, dense rows), the dispatch
// over every compiled height, and the bounded-wait diagnostic.  The kernels
// themselves are the templates of jefi_staged.cuh; the wide heights are
// compiled in jefi_staged_b32_48.cu and jefi_staged_b64_96.cu.
#include "jefi_staged.cuh"

namespace jefi {

JEFI_STAGED_BAND_LAUNCHERS(16)
JEFI_STAGED_BAND_LAUNCHERS(24)

namespace staged {

// Diagnostic: wait on an mbarrier that nothing arrives at, with the same
// bounded wait as the staged kernel, and report the outcome in *status.
__global__ void wait_timeout_probe(int32_t* status, uint64_t limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(smem_u32(&bar), 0, limit_ns);
    if (threadIdx.x == 0) *status = ok ? 0 : kStatusTimeout;
}

}  // namespace staged

cudaError_t launch_wait_timeout_probe(int32_t* status, uint64_t limit_ns, cudaStream_t s) {
    staged::wait_timeout_probe<<<1, 32, 0, s>>>(status, limit_ns);
    return cudaGetLastError();
}

bool staged_band_supported(int band) {
    for (int b : kStagedBands)
        if (b == band) return true;
    return false;
}

size_t staged_buffer_bytes(int band) { return (size_t)staged_stage_cells(band) * band * 32; }

size_t staged_smem_bytes(const SumParams& p, int band, bool batched) {
    // alignment pad, two stage buffers, mbarriers / band origins / item / tile box
    const size_t tab = 2 * staged_buffer_bytes(band) + kStagedCtrlBytes;
    const int nb_sum = p.nbx + p.nby + p.nbz;
    size_t b = tab + (size_t)(p.K + 2 * kTabGuard) * sizeof(float2);
    b += (size_t)(p.K + 1) * sizeof(double);
    b += (size_t)nb_sum * sizeof(float);
    // non-lattice geometry: FP64 points of the tile and cell centres, for the
    // fall-back (single and batched kernels alike)
    (void)batched;
    if (!p.exact)
        b = staged::staged_geometry_offset((uint32_t)tab, p.K, nb_sum) +
            (size_t)(3 * kTileThreads + p.npx + p.npy + p.npz) * 8;
    return (staged_swizzled(band) ? kStagedAlignPad : 0) + b;
}

cudaError_t launch_sum_f32_staged(const SumParams& p, const StagedConfig& c, cudaStream_t s) {
    switch (c.band) {
        case 16: return staged_launch_16(p, c, s);
        case 24: return staged_launch_24(p, c, s);
        case 32: return staged_launch_32(p, c, s);
        case 48: return staged_launch_48(p, c, s);
        case 64: return staged_launch_64(p, c, s);
        case 96: return staged_launch_96(p, c, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sum_f32_staged_batch(const StagedBatchArgs& a, int band, bool exact, size_t smem,
                                        int grid, cudaStream_t s) {
    switch (band) {
        case 16: return staged_launch_batch_16(a, exact, smem, grid, s);
        case 24: return staged_launch_batch_24(a, exact, smem, grid, s);
        case 32: return staged_launch_batch_32(a, exact, smem, grid, s);
        case 48: return staged_launch_batch_48(a, exact, smem, grid, s);
        case 64: return staged_launch_batch_64(a, exact, smem, grid, s);
        case 96: return staged_launch_batch_96(a, exact, smem, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace jefi
