// Whole IFCM runs of small volumes held in shared memory: one CTA per
// (volume, particle) of a batch keeps x, U^t and U^{t+1} of its volume in
// shared memory and runs every iteration of the particle's run (Eqs 1-10,
// reading R5) inside one launch, the centre sums of Eq 3 and the objective
// of Eq 1 reduced in the CTA after each iteration and the stop rule taken
// there.  The particles of a batch are independent runs, so no iteration needs
// a grid-wide step: a batch is one launch instead of two per iteration
// (stencil + reduce), which on images of a few thousand voxels removes the
// fixed cost of each launch -- the shape of Algorithm 2's step function for a
// swarm, with the loop of its steps 6-10 on the device.
//
// The per-voxel arithmetic is that of the plain kernel (plain_kernel.cu):
// g_ik = |x_i - x_k| (Eq 6), q^2 = dx^2 + dy^2 + dz^2 (Eq 8, reading R1),
// H and F as the normalised sums of Eqs 5 and 7 over the in-volume neighbours
// (reading R4), the plain mean of u_kj where every g_ik is 0 (reading R3),
// then Eq 4 (clamped, floored: reading R2) and Eq 2 in voxel_update.  Sums:
// FP32 within a thread (a few voxels) and a warp, then FP64 (or
// Neumaier-compensated FP32) across the warps in a fixed order.
#include "ifcm_math.cuh"
#include "launch.h"

namespace pifcm {

namespace {

constexpr int RT3 = kResidentThreads;
constexpr int NW = RT3 / 32;

template <int C>
struct ResShared {
  float red[NW][2 * C + 2];           // per-warp FP32 shares: S0, S1, J, max|du|
  double S[2 * C + 1];                // the iteration's sums (Eqs 1, 3)
  float dm;                           // the iteration's max|du|
  double cen[C];                      // C^t
  float cenf[C];
  float lam, xi;
  int vi, p, stop;
};

// The in-volume neighbour mean of cluster memberships from shared memory
// (H where every g_ik = 0, reading R3).  Rare path.
template <int C>
__device__ __noinline__ void res_flat_mean(const float* __restrict__ su, int N, int X, int Y,
                                           int Z, int nx, int ny, int nz, float (&H)[C]) {
  float s[C];
#pragma unroll
  for (int j = 0; j < C; ++j) s[j] = 0.0f;
  int n = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (dx == 0 && dy == 0 && dz == 0) continue;
        const int kx = X + dx, ky = Y + dy, kz = Z + dz;
        if (kx < 0 || kx >= nx || ky < 0 || ky >= ny || kz < 0 || kz >= nz) continue;
        const int k = (kz * ny + ky) * nx + kx;
#pragma unroll
        for (int j = 0; j < C; ++j) s[j] += su[j * N + k];
        ++n;
      }
  const float inv = n > 0 ? 1.0f / static_cast<float>(n) : 0.0f;
#pragma unroll
  for (int j = 0; j < C; ++j) H[j] = s[j] * inv;
}

template <int C>
__global__ void __launch_bounds__(RT3, 1) resident_kernel(const __grid_constant__ ResidentArgs a) {
  extern __shared__ __align__(16) float res_smem[];
  __shared__ ResShared<C> sh;
  constexpr int NV = 2 * C + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gp = blockIdx.x;                 // particle of the launch

  if (tid == 0) {
    int vi = 0;
    while (vi + 1 < a.n_vol && a.vol[vi + 1].pbase <= gp) ++vi;
    sh.vi = vi;
    sh.p = gp - a.vol[vi].pbase;
    const ResidentVol& rv = a.vol[vi];
    sh.lam = rv.lam_xi ? static_cast<float>(rv.lam_xi[2 * sh.p]) : 0.0f;
    sh.xi = rv.lam_xi ? static_cast<float>(rv.lam_xi[2 * sh.p + 1]) : 0.0f;
    sh.stop = 0;
  }
  __syncthreads();
  const ResidentVol& rv = a.vol[sh.vi];
  const int nx = rv.nx, ny = rv.ny, nz = rv.nz, pitch = rv.pitch;
  const int N = nx * ny * nz;
  const size_t gplane = static_cast<size_t>(nz) * ny * pitch;
  if (tid < C) {
    const double c = rv.c0 ? rv.c0[tid] : (tid + 0.5) / C;
    sh.cen[tid] = c;
    sh.cenf[tid] = static_cast<float>(c);
  }
  float* sx = res_smem;                      // x_i          [N]
  float* su = res_smem + N;                  // U^t          [C][N]
  float* sv = res_smem + N + C * N;          // U^{t+1}      [C][N]

  // load x and the shared start into shared memory (compact [z][y][x])
  for (int i = tid; i < N; i += RT3) {
    const int X = i % nx, YZ = i / nx;
    const size_t off = static_cast<size_t>(YZ) * pitch + X;
    sx[i] = rv.x[off];
#pragma unroll
    for (int j = 0; j < C; ++j) su[j * N + i] = rv.u0 ? rv.u0[j * gplane + off] : 1.0f / C;
  }
  __syncthreads();

  MethodConsts k;
  k.lam = sh.lam;
  k.xi = sh.xi;
  k.dist_floor = a.dist_floor;
  k.m = a.m;
  k.inv_m1 = a.inv_m1;
  k.m_is_2 = a.m_is_2;
  const bool stencil = a.stencil && (k.lam != 0.0f || k.xi != 0.0f);
  int it = 0;
  double J = 0.0;
  while (it < a.max_iter) {
    float cc[C];
#pragma unroll
    for (int j = 0; j < C; ++j) cc[j] = sh.cenf[j];
    float s0[C], s1[C], Js = 0.0f, dm = 0.0f;
#pragma unroll
    for (int j = 0; j < C; ++j) s0[j] = s1[j] = 0.0f;
    for (int i = tid; i < N; i += RT3) {
      const int X = i % nx, YZ = i / nx;
      const int Y = YZ % ny, Z = YZ / ny;
      const float xc = sx[i];
      float H[C], F[C];
#pragma unroll
      for (int j = 0; j < C; ++j) H[j] = F[j] = 0.0f;
      if (stencil) {
        float G = 0.0f, Q = 0.0f;
        int cnt = 0;
        // neighbour kk at squared distance q2 (Eqs 6 and 8); u_k^2 is
        // rounded before the q2 term (__fmul_rn is never contracted), so a
        // constant q2 gives the sums of a variable one
        auto add = [&](int kk, float q2) {
          const float g = fabsf(xc - sx[kk]);
#pragma unroll
          for (int j = 0; j < C; ++j) {
            const float uk = su[j * N + kk];
            H[j] = fmaf(uk, g, H[j]);
            F[j] = fmaf(__fmul_rn(uk, uk), q2, F[j]);
          }
          G += g;
          Q += q2;
          ++cnt;
        };
        if (nz == 1) {
          // an image: the 8 in-plane neighbours, in the order of the 3D loop
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
              if (dx == 0 && dy == 0) continue;
              const int kx = X + dx, ky = Y + dy;
              if (kx < 0 || kx >= nx || ky < 0 || ky >= ny) continue;
              add(ky * nx + kx, static_cast<float>(dx * dx + dy * dy));
            }
        } else {
          for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                const int kx = X + dx, ky = Y + dy, kz = Z + dz;
                if (kx < 0 || kx >= nx || ky < 0 || ky >= ny || kz < 0 || kz >= nz) continue;
                add((kz * ny + ky) * nx + kx, static_cast<float>(dx * dx + dy * dy + dz * dz));
              }
        }
        if (cnt > 0) {
          const float invQ = __frcp_rn(Q);
#pragma unroll
          for (int j = 0; j < C; ++j) F[j] *= invQ;
          if (G > 0.0f) {
            const float invG = __frcp_rn(G);
#pragma unroll
            for (int j = 0; j < C; ++j) H[j] *= invG;
          } else {
            res_flat_mean<C>(su, N, X, Y, Z, nx, ny, nz, H);
          }
        }
      }
      float u[C], um[C], Jv;
      voxel_update<C>(H, F, xc, cc, k, u, um, Jv);
#pragma unroll
      for (int j = 0; j < C; ++j) {
        dm = fmaxf(dm, fabsf(u[j] - su[j * N + i]));
        sv[j * N + i] = u[j];
        s0[j] += um[j];
        s1[j] = fmaf(um[j], xc, s1[j]);
      }
      Js += Jv;
    }
    // the iteration's sums: FP32 in the thread and the warp, then across the
    // warps in a fixed order
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const float v0 = warp_sum(s0[j]);
      const float v1 = warp_sum(s1[j]);
      if (lane == 0) {
        sh.red[warp][j] = v0;
        sh.red[warp][C + j] = v1;
      }
    }
    {
      const float vj = warp_sum(Js);
      const float vm = warp_max(dm);
      if (lane == 0) {
        sh.red[warp][2 * C] = vj;
        sh.red[warp][2 * C + 1] = vm;
      }
    }
    __syncthreads();
    // one warp per value: lane w holds warp w's share
    for (int v = warp; v < NV + 1; v += NW) {
      if (v == NV) {
        float m = lane < NW ? sh.red[lane][v] : 0.0f;
        m = warp_max(m);
        if (lane == 0) sh.dm = m;
      } else if (a.reduce == IFCM_REDUCE_FP64) {
        double s = lane < NW ? static_cast<double>(sh.red[lane][v]) : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sh.S[v] = s;
      } else if (lane == 0) {   // compensated FP32 (Neumaier) across the warps
        float s = 0.0f, comp = 0.0f;
        for (int w = 0; w < NW; ++w) neumaier_add(s, comp, sh.red[w][v]);
        sh.S[v] = static_cast<double>(__fadd_rn(s, comp));
      }
    }
    __syncthreads();
    ++it;
    if (tid < C) {                                                     // Eq 3
      if (a.reduce == IFCM_REDUCE_FP64) {
        if (sh.S[tid] > 0.0) sh.cen[tid] = sh.S[C + tid] / sh.S[tid];
      } else {
        const float S0 = static_cast<float>(sh.S[tid]), S1 = static_cast<float>(sh.S[C + tid]);
        if (S0 > 0.0f) sh.cen[tid] = static_cast<double>(__fdiv_rn(S1, S0));
      }
      sh.cenf[tid] = static_cast<float>(sh.cen[tid]);
    }
    J = sh.S[2 * C];                                                   // Eq 1
    const bool stop = !(static_cast<double>(sh.dm) >= a.eps) || it >= a.max_iter;
    {   // U^{t+1} becomes U^t
      float* t = su;
      su = sv;
      sv = t;
    }
    __syncthreads();
    if (stop) break;
  }

  // outputs: the run state and the volume's results at the last iteration
  if (tid == 0) {
    const int p = sh.p;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      a.st.centres[static_cast<size_t>(gp) * C + j] = sh.cen[j];
      if (rv.c_out) rv.c_out[static_cast<size_t>(p) * C + j] = sh.cen[j];
    }
    a.st.J[gp] = J;
    a.st.iters[gp] = it;
    a.st.active[gp] = 0;
    if (rv.fitness) rv.fitness[p] = J;
    if (rv.iters_out) rv.iters_out[p] = it;
    atomicAdd(a.st.updates, static_cast<unsigned long long>(N) * it);
  }
  if (rv.u_final && sh.p == 0) {
    for (int i = tid; i < N; i += RT3) {
      const int X = i % nx, YZ = i / nx;
      const size_t off = static_cast<size_t>(YZ) * pitch + X;
#pragma unroll
      for (int j = 0; j < C; ++j) rv.u_final[j * gplane + off] = su[j * N + i];
    }
  }
}

}  // namespace

size_t resident_smem_bytes(int c, long long nvox) {
  return static_cast<size_t>(1 + 2 * c) * static_cast<size_t>(nvox) * sizeof(float);
}

cudaError_t launch_resident(int c, const ResidentArgs& a, int P_total, long long max_nvox,
                            cudaStream_t s) {
  const size_t smem = resident_smem_bytes(c, max_nvox);
  if (smem > kResidentSmemBytes) return cudaErrorInvalidValue;
  switch (c) {
#define PIFCM_RES_CASE(CC)                                                                 \
  case CC: {                                                                               \
    cudaError_t e = cudaFuncSetAttribute(resident_kernel<CC>,                              \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                         static_cast<int>(kResidentSmemBytes));            \
    if (e != cudaSuccess) return e;                                                        \
    resident_kernel<CC><<<P_total, RT3, smem, s>>>(a);                                     \
    break;                                                                                 \
  }
    PIFCM_RES_CASE(2)
    PIFCM_RES_CASE(3)
    PIFCM_RES_CASE(4)
    PIFCM_RES_CASE(5)
    PIFCM_RES_CASE(6)
    PIFCM_RES_CASE(7)
    PIFCM_RES_CASE(8)
#undef PIFCM_RES_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pifcm
