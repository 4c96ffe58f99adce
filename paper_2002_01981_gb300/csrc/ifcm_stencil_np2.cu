// The stencil kernel with two particles per work item (c <= 4): the pair
// shares the x tile and every g of the neighbourhood, and its sums are the
// two lanes of each packed FP32x2 register.  FP32 memberships here; the bf16
// pair-word form of the same kernel is in ifcm_stencil_bf16_np2.cu.
#include "stencil_kernel.cuh"

namespace pifcm {

// Defined in ifcm_stencil_bf16_np2.cu.
cudaError_t launch_stencil_bf16_np2(int c, const StencilArgs& a, int grid, cudaStream_t s);
int blocks_per_sm_bf16_np2(int c);
size_t smem_bytes_bf16_np2(int c);

size_t smem_bytes_np2(int c, bool bf16) {
  if (bf16) return smem_bytes_bf16_np2(c);
  switch (c) {
    case 2: return smem_total<2, 2, false>();
    case 3: return smem_total<3, 2, false>();
    default: return smem_total<4, 2, false>();
  }
}

int blocks_per_sm_np2(int c, bool bf16) {
  if (bf16) return blocks_per_sm_bf16_np2(c);
  switch (c) {
    case 2: return blocks_per_sm_c<2, 2, false>();
    case 3: return blocks_per_sm_c<3, 2, false>();
    default: return blocks_per_sm_c<4, 2, false>();
  }
}

cudaError_t launch_stencil_np2(int c, bool bf16, const StencilArgs& a, int grid, cudaStream_t s) {
  if (bf16) return launch_stencil_bf16_np2(c, a, grid, s);
  switch (c) {
    case 2: return launch_c<2, 2, false>(a, grid, s);
    case 3: return launch_c<3, 2, false>(a, grid, s);
    case 4: return launch_c<4, 2, false>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pifcm
