// jefi_staged_b32_48.cu -- the TMA-staged FP32 sum compiled for bands of 32
// and 48 slots (stages of two z slabs, rows copied with the 32-byte swizzle);
// the kernels are the templates of jefi_staged.cuh.
#include "jefi_staged.cuh"

namespace jefi {
JEFI_STAGED_BAND_LAUNCHERS(32)
JEFI_STAGED_BAND_LAUNCHERS(48)
}  // namespace jefi
