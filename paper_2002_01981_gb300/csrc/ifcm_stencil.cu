// The stencil kernel with one particle per work item (every c), and the
// dispatch over (c, particles per item) used by the run loops.  The kernel
// itself is in stencil_kernel.cuh; two particles per item (c <= 4) are
// compiled in ifcm_stencil_np2.cu.
#include "stencil_kernel.cuh"

namespace pifcm {

// Defined in ifcm_stencil_np2.cu.
cudaError_t launch_stencil_np2(int c, const StencilArgs& a, int grid, cudaStream_t s);
int blocks_per_sm_np2(int c);
size_t smem_bytes_np2(int c);

bool stencil_np_supported(int c, int np) {
  if (c < 2 || c > kMaxC) return false;
  return np == 1 || (np == 2 && c <= 4);
}

int stencil_default_np(int c) { return c <= 4 ? 2 : 1; }

size_t stencil_smem_bytes(int c, int np) {
  if (np == 2) return smem_bytes_np2(c);
  switch (c) {
    case 2: return smem_total<2, 1>();
    case 3: return smem_total<3, 1>();
    case 4: return smem_total<4, 1>();
    case 5: return smem_total<5, 1>();
    case 6: return smem_total<6, 1>();
    case 7: return smem_total<7, 1>();
    default: return smem_total<8, 1>();
  }
}

int stencil_blocks_per_sm(int c, int np) {
  if (np == 2) return blocks_per_sm_np2(c);
  switch (c) {
    case 2: return blocks_per_sm_c<2, 1>();
    case 3: return blocks_per_sm_c<3, 1>();
    case 4: return blocks_per_sm_c<4, 1>();
    case 5: return blocks_per_sm_c<5, 1>();
    case 6: return blocks_per_sm_c<6, 1>();
    case 7: return blocks_per_sm_c<7, 1>();
    default: return blocks_per_sm_c<8, 1>();
  }
}

cudaError_t launch_stencil(int c, int np, const StencilArgs& a, int grid, cudaStream_t s) {
  if (!stencil_np_supported(c, np)) return cudaErrorInvalidValue;
  if (np == 2) return launch_stencil_np2(c, a, grid, s);
  switch (c) {
    case 2: return launch_c<2, 1>(a, grid, s);
    case 3: return launch_c<3, 1>(a, grid, s);
    case 4: return launch_c<4, 1>(a, grid, s);
    case 5: return launch_c<5, 1>(a, grid, s);
    case 6: return launch_c<6, 1>(a, grid, s);
    case 7: return launch_c<7, 1>(a, grid, s);
    case 8: return launch_c<8, 1>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pifcm
