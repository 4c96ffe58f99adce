// The stencil kernel over bf16 pair words with two particles per work item
// (c <= 5): word (pair k, cluster j) holds cluster j of particles 2k and
// 2k+1, the two lanes of the packed FP32x2 sums.
#include "stencil2d.cuh"

namespace pifcm {

namespace {
template <int C>
cudaError_t launch_np2_bf16(const StencilArgs& a, int grid, cudaStream_t s) {
  if (!stencil_lean(UL_BF16, 2, a.m_is_2, a.sum_one)) return launch_c<C, 2, UL_BF16>(a, grid, s);
  bool deep = false, flat = false;
  for (int v = 0; v < a.n_vol; ++v) (a.vol[v].nz == 1 ? flat : deep) = true;
  if (deep) {
    const cudaError_t e = launch3d_c<C, 2, UL_BF16>(a, grid, s);
    if (e != cudaSuccess || !flat) return e;
  }
  return launch2d_c<C, 2, UL_BF16>(a, grid, s);
}
}  // namespace

size_t smem_bytes_bf16_np2(int c) {
  switch (c) {
    case 2: return smem_total<2, 2, UL_BF16>();
    case 3: return smem_total<3, 2, UL_BF16>();
    case 4: return smem_total<4, 2, UL_BF16>();
    default: return smem_total<5, 2, UL_BF16>();
  }
}

int blocks_per_sm_bf16_np2(int c) {
  switch (c) {
    case 2: return blocks_per_sm_c<2, 2, UL_BF16>();
    case 3: return blocks_per_sm_c<3, 2, UL_BF16>();
    case 4: return blocks_per_sm_c<4, 2, UL_BF16>();
    default: return blocks_per_sm_c<5, 2, UL_BF16>();
  }
}

cudaError_t launch_stencil_bf16_np2(int c, const StencilArgs& a, int grid, cudaStream_t s) {
  switch (c) {
    case 2: return launch_np2_bf16<2>(a, grid, s);
    case 3: return launch_np2_bf16<3>(a, grid, s);
    case 4: return launch_np2_bf16<4>(a, grid, s);
    case 5: return launch_np2_bf16<5>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pifcm
