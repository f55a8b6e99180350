// jefi_staged_b64_96.cu -- the TMA-staged FP32 sum compiled for bands of 64
// and 96 slots (stages of one z slab, rows copied with the 32-byte swizzle);
// the kernels are the templates of jefi_staged.cuh.
#include "jefi_staged.cuh"

namespace jefi {
JEFI_STAGED_BAND_LAUNCHERS(64)
JEFI_STAGED_BAND_LAUNCHERS(96)
}  // namespace jefi
