// The stencil kernel with one particle per work item and FP32 memberships
// (every c), and the dispatch over (c, particles per item, membership type)
// used by the run loops.  The kernel itself is in stencil_kernel.cuh; the
// other instantiations are compiled in ifcm_stencil_np2.cu (FP32, two
// particles per item), ifcm_stencil_bf16.cu and ifcm_stencil_bf16_np2.cu
// (bf16 pair words), so that they build in parallel.
#include "stencil_kernel.cuh"

namespace pifcm {

// Defined in the other stencil translation units.
cudaError_t launch_stencil_np2(int c, bool bf16, const StencilArgs& a, int grid, cudaStream_t s);
int blocks_per_sm_np2(int c, bool bf16);
size_t smem_bytes_np2(int c, bool bf16);
cudaError_t launch_stencil_bf16_np1(int c, const StencilArgs& a, int grid, cudaStream_t s);
int blocks_per_sm_bf16_np1(int c);
size_t smem_bytes_bf16_np1(int c);

bool stencil_np_supported(int c, int np) {
  if (c < 2 || c > kMaxC) return false;
  return np == 1 || (np == 2 && c <= 4);
}

int stencil_default_np(int c) { return c <= 4 ? 2 : 1; }

long long bf16_unit_words(int c, int np, int P) {
  return np == 2 ? static_cast<long long>((P + 1) / 2) * c
                 : static_cast<long long>(P) * ((c + 1) / 2);
}

size_t stencil_smem_bytes(int c, int np, bool bf16) {
  if (np == 2) return smem_bytes_np2(c, bf16);
  if (bf16) return smem_bytes_bf16_np1(c);
  switch (c) {
    case 2: return smem_total<2, 1, false>();
    case 3: return smem_total<3, 1, false>();
    case 4: return smem_total<4, 1, false>();
    case 5: return smem_total<5, 1, false>();
    case 6: return smem_total<6, 1, false>();
    case 7: return smem_total<7, 1, false>();
    default: return smem_total<8, 1, false>();
  }
}

int stencil_blocks_per_sm(int c, int np, bool bf16) {
  if (np == 2) return blocks_per_sm_np2(c, bf16);
  if (bf16) return blocks_per_sm_bf16_np1(c);
  switch (c) {
    case 2: return blocks_per_sm_c<2, 1, false>();
    case 3: return blocks_per_sm_c<3, 1, false>();
    case 4: return blocks_per_sm_c<4, 1, false>();
    case 5: return blocks_per_sm_c<5, 1, false>();
    case 6: return blocks_per_sm_c<6, 1, false>();
    case 7: return blocks_per_sm_c<7, 1, false>();
    default: return blocks_per_sm_c<8, 1, false>();
  }
}

cudaError_t launch_stencil(int c, int np, bool bf16, const StencilArgs& a, int grid,
                           cudaStream_t s) {
  if (!stencil_np_supported(c, np)) return cudaErrorInvalidValue;
  if (np == 2) return launch_stencil_np2(c, bf16, a, grid, s);
  if (bf16) return launch_stencil_bf16_np1(c, a, grid, s);
  switch (c) {
    case 2: return launch_c<2, 1, false>(a, grid, s);
    case 3: return launch_c<3, 1, false>(a, grid, s);
    case 4: return launch_c<4, 1, false>(a, grid, s);
    case 5: return launch_c<5, 1, false>(a, grid, s);
    case 6: return launch_c<6, 1, false>(a, grid, s);
    case 7: return launch_c<7, 1, false>(a, grid, s);
    case 8: return launch_c<8, 1, false>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pifcm
