// The plain IFCM iteration for one particle with the first neighbourhood
// shell (V = 1): one thread per voxel, neighbours read straight from global
// memory -- the shape of the paper's Algorithm 2 steps 6-8.  It is the plain
// comparison form (ifcm_fit_plain) and the FCM start (stencil off).  It sits
// in a translation unit of its own so that its code generation does not
// depend on the other kernels.
#include "ifcm_math.cuh"
#include "launch.h"

namespace pifcm {

namespace {

constexpr int PT = 256;   // threads per block (plain_blocks() assumes it)

template <int C>
__global__ void __launch_bounds__(PT) plain_kernel(const PlainArgs a) {
  __shared__ float s_red[PT / 32][2 * C + 2];
  if (!a.active[0]) return;
  const long long nvox = static_cast<long long>(a.nx) * a.ny * a.nz;
  const size_t plane = static_cast<size_t>(a.nz) * a.ny * a.pitch;
  MethodConsts k;
  if (a.lam_xi) {
    k.lam = static_cast<float>(a.lam_xi[0]);
    k.xi = static_cast<float>(a.lam_xi[1]);
  } else {
    k.lam = a.lam;
    k.xi = a.xi;
  }
  k.dist_floor = a.dist_floor;
  k.m = a.m;
  k.inv_m1 = a.inv_m1;
  k.m_is_2 = a.m_is_2;
  float cc[C];
#pragma unroll
  for (int j = 0; j < C; ++j) cc[j] = static_cast<float>(a.centres[j]);
  const bool stencil = a.stencil && (k.lam != 0.0f || k.xi != 0.0f);

  float s0[C], s1[C], Js = 0.0f, dm = 0.0f;
#pragma unroll
  for (int j = 0; j < C; ++j) s0[j] = s1[j] = 0.0f;

  const long long first = static_cast<long long>(blockIdx.x) * PT * a.vpt;
  for (int r = 0; r < a.vpt; ++r) {
    const long long i = first + static_cast<long long>(r) * PT + threadIdx.x;
    if (i >= nvox) break;
    const int X = static_cast<int>(i % a.nx);
    const long long yz = i / a.nx;
    const int Y = static_cast<int>(yz % a.ny);
    const int Z = static_cast<int>(yz / a.ny);
    const size_t off = (static_cast<size_t>(Z) * a.ny + Y) * a.pitch + X;
    const float xc = a.x[off];
    float uc[C];
#pragma unroll
    for (int j = 0; j < C; ++j) uc[j] = a.u_src ? a.u_src[j * plane + off] : 1.0f / C;
    float H[C], F[C];
#pragma unroll
    for (int j = 0; j < C; ++j) H[j] = F[j] = 0.0f;
    if (stencil) {
      float G = 0.0f, Q = 0.0f;
      int cnt = 0;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0 && dz == 0) continue;
            const int kx = X + dx, ky = Y + dy, kz = Z + dz;
            if (kx < 0 || kx >= a.nx || ky < 0 || ky >= a.ny || kz < 0 || kz >= a.nz) continue;
            const size_t ko = (static_cast<size_t>(kz) * a.ny + ky) * a.pitch + kx;
            const float g = fabsf(xc - a.x[ko]);                       // Eq 6
            const float q2 = static_cast<float>(dx * dx + dy * dy + dz * dz);   // Eq 8
#pragma unroll
            for (int j = 0; j < C; ++j) {
              const float uk = a.u_src ? a.u_src[j * plane + ko] : 1.0f / C;
              H[j] = fmaf(uk, g, H[j]);
              F[j] = fmaf(uk * uk, q2, F[j]);
            }
            G += g;
            Q += q2;
            ++cnt;
          }
      if (cnt > 0) {
        const float invQ = __frcp_rn(Q);
#pragma unroll
        for (int j = 0; j < C; ++j) F[j] *= invQ;
        if (G > 0.0f) {
          const float invG = __frcp_rn(G);
#pragma unroll
          for (int j = 0; j < C; ++j) H[j] *= invG;
        } else if (a.u_src) {
          flat_neighbourhood_mean<C>(a.u_src, X, Y, Z, a.nx, a.ny, a.nz, a.pitch, H);
        } else {
#pragma unroll
          for (int j = 0; j < C; ++j) H[j] = 1.0f / C;
        }
      }
    }
    float u[C], um[C], Jv;
    voxel_update<C>(H, F, xc, cc, k, u, um, Jv);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      if (IFCM_CHECK(static_cast<long long>((j + 1) * plane) <= a.dst_elems, a.status, 43))
        a.u_dst[j * plane + off] = u[j];
      s0[j] += um[j];
      s1[j] = fmaf(um[j], xc, s1[j]);
      dm = fmaxf(dm, fabsf(u[j] - uc[j]));
    }
    Js += Jv;
  }

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const float v0 = warp_sum(s0[j]);
    const float v1 = warp_sum(s1[j]);
    if (lane == 0) {
      s_red[warp][j] = v0;
      s_red[warp][C + j] = v1;
    }
  }
  const float vj = warp_sum(Js);
  const float vm = warp_max(dm);
  if (lane == 0) {
    s_red[warp][2 * C] = vj;
    s_red[warp][2 * C + 1] = vm;
  }
  __syncthreads();
  if (!IFCM_CHECK(static_cast<long long>(blockIdx.x) < a.n_records, a.status, 44)) {
  } else if (threadIdx.x < 2 * C + 1) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < PT / 32; ++w) sum += static_cast<double>(s_red[w][threadIdx.x]);
    a.partials[static_cast<size_t>(blockIdx.x) * (2 * C + 1) + threadIdx.x] = sum;
  } else if (threadIdx.x == 2 * C + 1) {
    float mm = 0.0f;
#pragma unroll
    for (int w = 0; w < PT / 32; ++w) mm = fmaxf(mm, s_red[w][2 * C + 1]);
    a.dmax[blockIdx.x] = mm;
  }
}

}  // namespace

cudaError_t launch_plain_v1(int c, const PlainArgs& a, int blocks, cudaStream_t s) {
  switch (c) {
    case 2: plain_kernel<2><<<blocks, PT, 0, s>>>(a); break;
    case 3: plain_kernel<3><<<blocks, PT, 0, s>>>(a); break;
    case 4: plain_kernel<4><<<blocks, PT, 0, s>>>(a); break;
    case 5: plain_kernel<5><<<blocks, PT, 0, s>>>(a); break;
    case 6: plain_kernel<6><<<blocks, PT, 0, s>>>(a); break;
    case 7: plain_kernel<7><<<blocks, PT, 0, s>>>(a); break;
    case 8: plain_kernel<8><<<blocks, PT, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pifcm
