// The stencil kernel with two particles per work item (c <= 4): the pair
// shares the x tile and every g of the neighbourhood, and its sums are the
// two lanes of each packed FP32x2 register.  Compiled apart from the
// one-particle form so that the two build in parallel.
#include "stencil_kernel.cuh"

namespace pifcm {

size_t smem_bytes_np2(int c) {
  switch (c) {
    case 2: return smem_total<2, 2>();
    case 3: return smem_total<3, 2>();
    default: return smem_total<4, 2>();
  }
}

int blocks_per_sm_np2(int c) {
  switch (c) {
    case 2: return blocks_per_sm_c<2, 2>();
    case 3: return blocks_per_sm_c<3, 2>();
    default: return blocks_per_sm_c<4, 2>();
  }
}

cudaError_t launch_stencil_np2(int c, const StencilArgs& a, int grid, cudaStream_t s) {
  switch (c) {
    case 2: return launch_c<2, 2>(a, grid, s);
    case 3: return launch_c<3, 2>(a, grid, s);
    case 4: return launch_c<4, 2>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pifcm
