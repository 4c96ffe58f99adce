// The stencil kernel over float2 pair words with one particle per work item
// (every c): word (particle p, pair k) holds clusters 2k and 2k+1 of p, loaded
// and stored as one 64-bit access.  The FP32 layout of batched runs.
// Iterations that read Eq 2's memberships (every one after the first) with
// m = 2 run the 3D volumes through stencil3d_kernel and the 2D images
// through stencil2d_kernel.
#include "stencil2d.cuh"

namespace pifcm {

namespace {
template <int C>
cudaError_t launch_np1(const StencilArgs& a, int grid, cudaStream_t s) {
  if (!stencil_lean(UL_F32P, 1, a.m_is_2, a.sum_one)) return launch_c<C, 1, UL_F32P>(a, grid, s);
  bool deep = false, flat = false;
  for (int v = 0; v < a.n_vol; ++v) (a.vol[v].nz == 1 ? flat : deep) = true;
  if (deep) {
    const cudaError_t e = launch3d_c<C, 1>(a, grid, s);
    if (e != cudaSuccess || !flat) return e;
  }
  return launch2d_c<C, 1, UL_F32P>(a, grid, s);
}
}  // namespace

size_t smem_bytes_f32p_np1(int c) {
  switch (c) {
    case 2: return smem_total<2, 1, UL_F32P>();
    case 3: return smem_total<3, 1, UL_F32P>();
    case 4: return smem_total<4, 1, UL_F32P>();
    case 5: return smem_total<5, 1, UL_F32P>();
    case 6: return smem_total<6, 1, UL_F32P>();
    case 7: return smem_total<7, 1, UL_F32P>();
    default: return smem_total<8, 1, UL_F32P>();
  }
}

int blocks_per_sm_f32p_np1(int c) {
  switch (c) {
    case 2: return blocks_per_sm_c<2, 1, UL_F32P>();
    case 3: return blocks_per_sm_c<3, 1, UL_F32P>();
    case 4: return blocks_per_sm_c<4, 1, UL_F32P>();
    case 5: return blocks_per_sm_c<5, 1, UL_F32P>();
    case 6: return blocks_per_sm_c<6, 1, UL_F32P>();
    case 7: return blocks_per_sm_c<7, 1, UL_F32P>();
    default: return blocks_per_sm_c<8, 1, UL_F32P>();
  }
}

cudaError_t launch_stencil_f32p_np1(int c, const StencilArgs& a, int grid, cudaStream_t s) {
  switch (c) {
    case 2: return launch_np1<2>(a, grid, s);
    case 3: return launch_np1<3>(a, grid, s);
    case 4: return launch_np1<4>(a, grid, s);
    case 5: return launch_np1<5>(a, grid, s);
    case 6: return launch_np1<6>(a, grid, s);
    case 7: return launch_np1<7>(a, grid, s);
    case 8: return launch_np1<8>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pifcm
