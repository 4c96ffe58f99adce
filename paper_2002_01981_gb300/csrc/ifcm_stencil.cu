// Dispatch of the stencil kernel over (c, particles per work item, membership
// layout), used by the run loops.  The kernel is in stencil_kernel.cuh; its
// instantiations are compiled in ifcm_stencil_{planar,np2,bf16,bf16_np2,f32p,
// f32p_np2}.cu so that they build in parallel.
#include "launch.h"

namespace pifcm {

#define PIFCM_STENCIL_FAMILY(name)                                                   \
  size_t smem_bytes_##name(int c);                                                   \
  int blocks_per_sm_##name(int c);                                                   \
  cudaError_t launch_stencil_##name(int c, const StencilArgs& a, int grid, cudaStream_t s);
PIFCM_STENCIL_FAMILY(planar_np1)
PIFCM_STENCIL_FAMILY(planar_np2)
PIFCM_STENCIL_FAMILY(bf16_np1)
PIFCM_STENCIL_FAMILY(bf16_np2)
PIFCM_STENCIL_FAMILY(f32p_np1)
PIFCM_STENCIL_FAMILY(f32p_np2)
#undef PIFCM_STENCIL_FAMILY

bool stencil_np_supported(int c, int np) {
  if (c < 2 || c > kMaxC) return false;
  return np == 1 || (np == 2 && c <= 5);
}

int stencil_default_np(int c) { return c <= 5 ? 2 : 1; }

long long pair_unit_words(int c, int np, int P) {
  return np == 2 ? static_cast<long long>((P + 1) / 2) * c
                 : static_cast<long long>(P) * ((c + 1) / 2);
}

#define PIFCM_STENCIL_PICK(fn, ...)                                              \
  if (layout == UL_BF16) return np == 2 ? fn##_bf16_np2(__VA_ARGS__) : fn##_bf16_np1(__VA_ARGS__); \
  if (layout == UL_F32P) return np == 2 ? fn##_f32p_np2(__VA_ARGS__) : fn##_f32p_np1(__VA_ARGS__); \
  return np == 2 ? fn##_planar_np2(__VA_ARGS__) : fn##_planar_np1(__VA_ARGS__);

size_t stencil_smem_bytes(int c, int np, int layout) { PIFCM_STENCIL_PICK(smem_bytes, c) }

int stencil_blocks_per_sm(int c, int np, int layout) { PIFCM_STENCIL_PICK(blocks_per_sm, c) }

cudaError_t launch_stencil(int c, int np, int layout, const StencilArgs& a, int grid,
                           cudaStream_t s) {
  if (!stencil_np_supported(c, np)) return cudaErrorInvalidValue;
  PIFCM_STENCIL_PICK(launch_stencil, c, a, grid, s)
}
#undef PIFCM_STENCIL_PICK

}  // namespace pifcm
