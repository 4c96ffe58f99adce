// The stencil kernel with FP32 planar memberships and two particles per work
// item (c <= 5): the pair shares the x tile and every g of the neighbourhood,
// and its sums are the two lanes of each packed FP32x2 register.
#include "stencil_kernel.cuh"

namespace pifcm {

size_t smem_bytes_planar_np2(int c) {
  switch (c) {
    case 2: return smem_total<2, 2, UL_PLANAR>();
    case 3: return smem_total<3, 2, UL_PLANAR>();
    case 4: return smem_total<4, 2, UL_PLANAR>();
    default: return smem_total<5, 2, UL_PLANAR>();
  }
}

int blocks_per_sm_planar_np2(int c) {
  switch (c) {
    case 2: return blocks_per_sm_c<2, 2, UL_PLANAR>();
    case 3: return blocks_per_sm_c<3, 2, UL_PLANAR>();
    case 4: return blocks_per_sm_c<4, 2, UL_PLANAR>();
    default: return blocks_per_sm_c<5, 2, UL_PLANAR>();
  }
}

cudaError_t launch_stencil_planar_np2(int c, const StencilArgs& a, int grid, cudaStream_t s) {
  switch (c) {
    case 2: return launch_c<2, 2, UL_PLANAR>(a, grid, s);
    case 3: return launch_c<3, 2, UL_PLANAR>(a, grid, s);
    case 4: return launch_c<4, 2, UL_PLANAR>(a, grid, s);
    case 5: return launch_c<5, 2, UL_PLANAR>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pifcm
