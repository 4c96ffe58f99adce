// Per-voxel tail of one IFCM iteration, shared by the stencil kernel and the
// plain (one thread per voxel) kernel.
//
// Given the neighbourhood terms H_ij and F_ij of a voxel (Eqs 5 and 7), its
// intensity x_i and the centres C^t, compute the modified distance of Eq 4
// (with reading R2: the factor 1 - lambda H - xi F is clamped at 0 and d^2 is
// floored), the new memberships of Eq 2, u^m for the centre sums of Eq 3, and
// the voxel's share of the objective of Eq 1.
#pragma once

#include "common.cuh"

namespace pifcm {

struct MethodConsts {
  float lam, xi;        // (lambda, xi) of the run
  float dist_floor;     // floor of d^2
  float m;              // fuzzifier
  float inv_m1;         // 1 / (m - 1)
  int m_is_2;           // fast path: u_j = (1/d2_j) / sum_k (1/d2_k)
};

template <int C>
__device__ __forceinline__ void voxel_update(const float (&H)[C], const float (&F)[C], float xc,
                                             const float (&cc)[C], const MethodConsts& k,
                                             float (&u)[C], float (&um)[C], float& Jv) {
  float d2[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const float fac = fmaxf(1.0f - k.lam * H[j] - k.xi * F[j], 0.0f);   // Eq 4
    const float dd = xc - cc[j];
    d2[j] = fmaxf(dd * dd * fac, k.dist_floor);
  }
  if (k.m_is_2) {
    // m = 2: u_j = (1/d2_j) / S with S = sum_k 1/d2_k (Eq 2); then
    // sum_j u_j^2 d2_j = 1/S exactly in real arithmetic (Eq 1 share).
    float r[C];
    float S = 0.0f;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      r[j] = __frcp_rn(d2[j]);
      S += r[j];
    }
    const float invS = __frcp_rn(S);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      u[j] = r[j] * invS;
      um[j] = u[j] * u[j];
    }
    Jv = invS;
  } else {
    // general m: u_j = d2_j^(-1/(m-1)) / sum_k d2_k^(-1/(m-1))  (Eq 2)
    float a[C];
    float S = 0.0f;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      a[j] = exp2f(-k.inv_m1 * log2f(d2[j]));
      S += a[j];
    }
    const float invS = __frcp_rn(S);
    Jv = 0.0f;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      u[j] = a[j] * invS;
      um[j] = exp2f(k.m * log2f(u[j]));
      Jv += um[j] * d2[j];
    }
  }
}

// Hardware reciprocal (rcp.approx, at most 1 ulp off for normal inputs).
__device__ __forceinline__ float fast_rcp(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// In-volume neighbour count and sum of q^2 = dx^2 + dy^2 + dz^2 (Eq 8,
// reading R1) over the 3x3x3 box around (X, Y, Z), excluding the voxel itself
// and every position outside the volume (reading R4).  With a_* in-volume
// neighbours along an axis and n_* = 1 + a_*, the box holds n_x n_y n_z voxels
// and sum q^2 = a_x n_y n_z + a_y n_x n_z + a_z n_x n_y.
__device__ __forceinline__ void box_counts(int X, int Y, int Z, int nx, int ny, int nz, int& cnt,
                                           float& Q) {
  const int ax = (X > 0) + (X < nx - 1);
  const int ay = (Y > 0) + (Y < ny - 1);
  const int az = (Z > 0) + (Z < nz - 1);
  const int nX = 1 + ax, nY = 1 + ay, nZ = 1 + az;
  cnt = nX * nY * nZ - 1;
  Q = static_cast<float>(ax * nY * nZ + ay * nX * nZ + az * nX * nY);
}

// Mean of u_kj over the in-volume neighbours of (X, Y, Z), read from global
// memory: the H term of Eq 5 where every g_ik is 0 (reading R3).  Rare path.
template <int C>
__device__ __noinline__ void flat_neighbourhood_mean(const float* __restrict__ u, int X, int Y,
                                                     int Z, int nx, int ny, int nz, int pitch,
                                                     float (&H)[C]) {
  const size_t plane = static_cast<size_t>(nz) * ny * pitch;
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
        const size_t off = (static_cast<size_t>(kz) * ny + ky) * pitch + kx;
#pragma unroll
        for (int j = 0; j < C; ++j) s[j] += u[j * plane + off];
        ++n;
      }
  const float inv = n > 0 ? 1.0f / static_cast<float>(n) : 0.0f;
#pragma unroll
  for (int j = 0; j < C; ++j) H[j] = s[j] * inv;
}

// The same mean over bf16 pair words (two memberships per 32-bit word, low
// half first): with pair_particles, word plane j holds cluster j of a particle
// pair and `lane` picks the particle; otherwise word plane j/2 holds clusters
// 2(j/2) and 2(j/2)+1 of one particle.
template <int C>
__device__ __noinline__ void flat_neighbourhood_mean_bf16(const uint32_t* __restrict__ u,
                                                          bool pair_particles, int lane, int X,
                                                          int Y, int Z, int nx, int ny, int nz,
                                                          int pitch, float (&H)[C]) {
  const size_t plane = static_cast<size_t>(nz) * ny * pitch;
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
        const size_t off = (static_cast<size_t>(kz) * ny + ky) * pitch + kx;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const int wp = pair_particles ? j : j >> 1;
          const int hi = pair_particles ? lane : (j & 1);
          const uint32_t w = u[wp * plane + off];
          s[j] += __uint_as_float(hi ? (w & 0xffff0000u) : (w << 16));
        }
        ++n;
      }
  const float inv = n > 0 ? 1.0f / static_cast<float>(n) : 0.0f;
#pragma unroll
  for (int j = 0; j < C; ++j) H[j] = s[j] * inv;
}

// The same mean over float2 pair words (pairing as for the bf16 words above).
template <int C>
__device__ __noinline__ void flat_neighbourhood_mean_f32p(const float2* __restrict__ u,
                                                          bool pair_particles, int lane, int X,
                                                          int Y, int Z, int nx, int ny, int nz,
                                                          int pitch, float (&H)[C]) {
  const size_t plane = static_cast<size_t>(nz) * ny * pitch;
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
        const size_t off = (static_cast<size_t>(kz) * ny + ky) * pitch + kx;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const int wp = pair_particles ? j : j >> 1;
          const int hi = pair_particles ? lane : (j & 1);
          const float2 w = u[wp * plane + off];
          s[j] += hi ? w.y : w.x;
        }
        ++n;
      }
  const float inv = n > 0 ? 1.0f / static_cast<float>(n) : 0.0f;
#pragma unroll
  for (int j = 0; j < C; ++j) H[j] = s[j] * inv;
}

// Compensated (Neumaier) FP32 summation step: sum + comp carries the running
// total with the rounding error of every addition kept in comp.
__device__ __forceinline__ void neumaier_add(float& sum, float& comp, float v) {
  const float t = __fadd_rn(sum, v);
  if (fabsf(sum) >= fabsf(v))
    comp = __fadd_rn(comp, __fadd_rn(__fsub_rn(sum, t), v));
  else
    comp = __fadd_rn(comp, __fadd_rn(__fsub_rn(v, t), sum));
  sum = t;
}

}  // namespace pifcm
