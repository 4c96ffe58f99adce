// Reverse pass of K unrolled IFCM iterations: dJ^{K-1}/d(lambda, xi).
//
// The forward pass (the stencil kernel, one particle) keeps every U^t and a
// trace of C^{t+1}, S0^{t+1} = sum_i u^m and J^t.  Going back over iteration
// t, with u_bar the adjoint of U^{t+1} and c_bar that of C^{t+1}:
//
//   point kernel, per voxel i (recomputing H, F, d^2 and u' of Eqs 5-8, 4, 2
//   from U^t exactly as the forward did):
//     w_bar  = J_bar d2 + c_bar_j (x_i - c^{t+1}_j) / S0_j     (Eqs 1, 3)
//     u_tot  = u_bar + m u^(m-1) w_bar
//     d2_bar = J_bar u^m - p (u_tot - sum_k u_tot_k u_k) u / d2,  p = 1/(m-1)  (Eq 2)
//     f_bar  = d2_bar D, where neither clamp of reading R2 is active  (Eq 4)
//     lambda_bar += -f_bar H, xi_bar += -f_bar F, c_bar^t_j += -2 d2_bar fac (x_i - c^t_j)
//     A_ij = -lambda f_bar / G_i (/ n_i where G_i = 0, reading R3),
//     B_ij = -xi f_bar / Q_i, e_i = 1 where G_i = 0
//   gather kernel, per voxel k (the transposed stencils of Eqs 5 and 7; the
//   neighbourhood is symmetric, g_ik = g_ki, q^2_ik = q^2_ki):
//     u_bar^t_kj = sum_{i in NB(k)} A_ij (g_ik + e_i) + 2 u_kj sum_i B_ij q^2_ik
//     (where G_i = 0 every g_ik is 0, so g_ik + e_i is the weight 1 of the mean)
//   reduce kernel: the per-block partial sums of lambda_bar, xi_bar and c_bar^t
//   in FP64 in a fixed order.
//
// The point kernel marches 32 x 8 column tiles along z with a three-plane
// shared-memory ring (one-voxel halo, the next plane fetched into registers
// while the current one is computed); the gather kernel reads global memory.
// FP32 arithmetic; per-block partials are FP32 within a warp and FP64 across
// warps.
#include <math_constants.h>

#include "ifcm_math.cuh"
#include "launch.h"

namespace pifcm {

namespace {

// Tiles: 32 x 8 columns per block (one thread per column), marched along z
// over chunks of AZ planes.  Each step keeps three planes (z - 1, z, z + 1) of
// the needed channels with a one-voxel halo in a shared-memory ring; a plane
// is loaded cooperatively with coalesced row reads.  Positions outside the
// volume are filled so that they contribute nothing without masks: the
// volume x with NaN (g = max(|x_i - x_k|, 0) turns it into 0), every other
// channel with 0.
constexpr int ATX = 32, ATY = 8, AT = ATX * ATY;
// z-chunks of 32 planes: 8-plane chunks re-read 25 % more halo planes and make
// 4x the partial records (128^3, K = 20: 9.07 -> 8.00 ms per gradient)
constexpr int AZ = 32;
constexpr int HX = ATX + 2, HY = ATY + 2, HP = HX * HY;   // halo plane cells

__device__ __forceinline__ float gdist_nan0(float a, float b) {
  float r;
  asm("max.f32 %0, %1, 0f00000000;" : "=f"(r) : "f"(fabsf(a - b)));
  return r;
}

struct TileGeo {
  int x0, y0, z0, z1;
};

__device__ __forceinline__ TileGeo tile_of(const AdjointArgs& a) {
  const int tx = (a.nx + ATX - 1) / ATX, ty = (a.ny + ATY - 1) / ATY;
  int b = blockIdx.x;
  const int bx = b % tx;
  b /= tx;
  const int by = b % ty;
  const int bz = b / ty;
  TileGeo t;
  t.x0 = bx * ATX;
  t.y0 = by * ATY;
  t.z0 = bz * AZ;
  t.z1 = min(t.z0 + AZ, a.nz);
  return t;
}

// Plane z of NCH channels, gathered into registers: element i = threadIdx.x +
// k AT of the [NCH][HP] plane.  Channel 0 is the volume x (NaN outside),
// channels 1.. come from src[ch - 1] (0 outside).  The loads are issued here
// and consumed later (store_plane), so their latency overlaps the stencil.
template <int NCH>
struct PlaneRegs {
  static constexpr int K = (NCH * HP + AT - 1) / AT;
  float v[K];
};

template <int NCH>
__device__ __forceinline__ void fetch_plane(const AdjointArgs& a, const TileGeo& t, int z,
                                            const float* const (&src)[NCH - 1],
                                            PlaneRegs<NCH>& r) {
  const bool zin = z >= 0 && z < a.nz;
#pragma unroll
  for (int k = 0; k < PlaneRegs<NCH>::K; ++k) {
    const int i = threadIdx.x + k * AT;
    float v = 0.0f;
    if (i < NCH * HP) {
      const int ch = i / HP, cell = i - ch * HP;
      const int cy = cell / HX, cx = cell - cy * HX;
      const int X = t.x0 - 1 + cx, Y = t.y0 - 1 + cy;
      v = ch == 0 ? __int_as_float(0x7fc00000) : 0.0f;
      if (zin && X >= 0 && X < a.nx && Y >= 0 && Y < a.ny) {
        const size_t off = (static_cast<size_t>(z) * a.ny + Y) * a.pitch + X;
        v = ch == 0 ? a.x[off] : src[ch - 1][off];
      }
    }
    r.v[k] = v;
  }
}

template <int NCH>
__device__ __forceinline__ void store_plane(const PlaneRegs<NCH>& r, float* dst) {
#pragma unroll
  for (int k = 0; k < PlaneRegs<NCH>::K; ++k) {
    const int i = threadIdx.x + k * AT;
    if (i < NCH * HP) dst[i] = r.v[k];
  }
}

template <int C>
__global__ void __launch_bounds__(AT) adjoint_point_kernel(const AdjointArgs a) {
  extern __shared__ float ring[];                   // [3][1 + C][HP]
  __shared__ float s_red[AT / 32][2 + C];
  constexpr int NCH = 1 + C;
  const TileGeo t = tile_of(a);
  const size_t plane = static_cast<size_t>(a.nz) * a.ny * a.pitch;
  const float* srcs[NCH - 1];
#pragma unroll
  for (int j = 0; j < C; ++j) srcs[j] = a.u + j * plane;
  const float lam = static_cast<float>(a.lam_xi[0]), xi = static_cast<float>(a.lam_xi[1]);
  float ct[C], cn[C], cb[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    ct[j] = static_cast<float>(a.c_t[j]);
    cn[j] = static_cast<float>(a.c_next[j]);
    // c_bar_j / S0_j of Eq 3's derivative
    cb[j] = a.cbar_next ? static_cast<float>(a.cbar_next[j] / a.s0_next[j]) : 0.0f;
  }
  const float Jb = a.J_bar;
  const float p = a.m_is_2 ? 1.0f : a.inv_m1;
  float lb = 0.0f, xb = 0.0f, cbt[C];
#pragma unroll
  for (int j = 0; j < C; ++j) cbt[j] = 0.0f;

  const int tx = threadIdx.x % ATX, ty = threadIdx.x / ATX;
  const int X = t.x0 + tx, Y = t.y0 + ty;
  const bool col_ok = X < a.nx && Y < a.ny;
  // ring slot of plane z: z mod 3; planes z0 - 1 and z0 first, then plane
  // Z + 1 is fetched before plane Z is computed and stored after it
  PlaneRegs<NCH> pr;
  fetch_plane<NCH>(a, t, t.z0 - 1, srcs, pr);
  store_plane<NCH>(pr, ring + ((t.z0 + 2) % 3) * NCH * HP);
  fetch_plane<NCH>(a, t, t.z0, srcs, pr);
  store_plane<NCH>(pr, ring + (t.z0 % 3) * NCH * HP);
  fetch_plane<NCH>(a, t, t.z0 + 1, srcs, pr);
  store_plane<NCH>(pr, ring + ((t.z0 + 1) % 3) * NCH * HP);
  __syncthreads();
  for (int Z = t.z0; Z < t.z1; ++Z) {
    if (Z + 1 < t.z1) fetch_plane<NCH>(a, t, Z + 2, srcs, pr);
    if (col_ok) {
      const float* pm = ring + (Z % 3) * NCH * HP;
      const int cc = (ty + 1) * HX + tx + 1;
      const float xc = pm[cc];
      float H[C], F[C], S[C], G = 0.0f;
#pragma unroll
      for (int j = 0; j < C; ++j) H[j] = F[j] = S[j] = 0.0f;
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) {
        const float* pl = ring + ((Z + dz + 3) % 3) * NCH * HP;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0 && dz == 0) continue;
            const int o = cc + dy * HX + dx;
            const float g = gdist_nan0(xc, pl[o]);
            const float q2 = static_cast<float>(dx * dx + dy * dy + dz * dz);
#pragma unroll
            for (int j = 0; j < C; ++j) {
              const float uk = pl[(1 + j) * HP + o];
              H[j] = fmaf(uk, g, H[j]);
              F[j] = fmaf(uk * uk, q2, F[j]);
              S[j] += uk;
            }
            G += g;
          }
      }
      int n;
      float Q;
      box_counts(X, Y, Z, a.nx, a.ny, a.nz, n, Q);
      if (n > 0) {
        const float invQ = __frcp_rn(Q);
#pragma unroll
        for (int j = 0; j < C; ++j) F[j] *= invQ;
        if (G > 0.0f) {
          const float invG = __frcp_rn(G);
#pragma unroll
          for (int j = 0; j < C; ++j) H[j] *= invG;
        } else {                                 // reading R3: plain mean
          const float inv = __frcp_rn(static_cast<float>(n));
#pragma unroll
          for (int j = 0; j < C; ++j) H[j] = S[j] * inv;
        }
      }
      const size_t off = (static_cast<size_t>(Z) * a.ny + Y) * a.pitch + X;
      // Eq 4 (reading R2) and Eq 2
      float D[C], f[C], fac[C], P[C], d2[C], u[C];
      float Ssum = 0.0f;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const float dd = xc - ct[j];
        D[j] = dd * dd;
        f[j] = 1.0f - lam * H[j] - xi * F[j];
        fac[j] = fmaxf(f[j], 0.0f);
        P[j] = D[j] * fac[j];
        d2[j] = fmaxf(P[j], a.dist_floor);
        u[j] = a.m_is_2 ? __frcp_rn(d2[j]) : exp2f(-a.inv_m1 * log2f(d2[j]));
        Ssum += u[j];
      }
      const float invS = __frcp_rn(Ssum);
#pragma unroll
      for (int j = 0; j < C; ++j) u[j] *= invS;
      // adjoints
      float ut[C], um[C];
      float dot = 0.0f;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const float um1 = a.m_is_2 ? u[j] : exp2f((a.m - 1.0f) * log2f(u[j]));   // u^(m-1)
        um[j] = um1 * u[j];                                                      // u^m
        const float wb = Jb * d2[j] + cb[j] * (xc - cn[j]);
        const float ub = a.ubar_next ? a.ubar_next[j * plane + off] : 0.0f;
        ut[j] = ub + a.m * um1 * wb;
        dot = fmaf(ut[j], u[j], dot);
      }
      const float invG = G > 0.0f ? __frcp_rn(G)
                                  : (n > 0 ? __frcp_rn(static_cast<float>(n)) : 0.0f);
      const float invQ = n > 0 ? __frcp_rn(Q) : 0.0f;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const float d2b = Jb * um[j] - p * (ut[j] - dot) * u[j] / d2[j];
        const float Pb = P[j] > a.dist_floor ? d2b : 0.0f;
        const float fb = f[j] > 0.0f ? Pb * D[j] : 0.0f;
        lb = fmaf(-fb, H[j], lb);
        xb = fmaf(-fb, F[j], xb);
        cbt[j] = fmaf(-2.0f * Pb * fac[j], xc - ct[j], cbt[j]);
        a.A[j * plane + off] = -lam * fb * invG;
        a.B[j * plane + off] = -xi * fb * invQ;
      }
      a.e[off] = (n > 0 && G == 0.0f) ? 1.0f : 0.0f;
    }
    __syncthreads();                     // slot (Z - 1) mod 3 is free
    if (Z + 1 < t.z1) {
      store_plane<NCH>(pr, ring + ((Z + 2) % 3) * NCH * HP);
      __syncthreads();
    }
  }

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float v0 = warp_sum(lb), v1 = warp_sum(xb);
  if (lane == 0) {
    s_red[warp][0] = v0;
    s_red[warp][1] = v1;
  }
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const float v = warp_sum(cbt[j]);
    if (lane == 0) s_red[warp][2 + j] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2 + C) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < AT / 32; ++w) sum += static_cast<double>(s_red[w][threadIdx.x]);
    a.partials[static_cast<size_t>(blockIdx.x) * (2 + C) + threadIdx.x] = sum;
  }
}

// The transposed stencil reads its 26 neighbours' coefficients straight from
// global memory (L1 / L2), one thread per voxel: with little arithmetic per
// voxel and 2c + 2 channels, staging planes in shared memory measured slower.
template <int C>
__global__ void __launch_bounds__(AT) adjoint_gather_kernel(const AdjointArgs a) {
  const long long nvox = static_cast<long long>(a.nx) * a.ny * a.nz;
  const size_t plane = static_cast<size_t>(a.nz) * a.ny * a.pitch;
  for (long long k = blockIdx.x * static_cast<long long>(AT) + threadIdx.x; k < nvox;
       k += static_cast<long long>(gridDim.x) * AT) {
    const int X = static_cast<int>(k % a.nx);
    const long long yz = k / a.nx;
    const int Y = static_cast<int>(yz % a.ny);
    const int Z = static_cast<int>(yz / a.ny);
    const size_t off = (static_cast<size_t>(Z) * a.ny + Y) * a.pitch + X;
    const float xk = a.x[off];
    float sh[C], sf[C];
#pragma unroll
    for (int j = 0; j < C; ++j) sh[j] = sf[j] = 0.0f;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (dx == 0 && dy == 0 && dz == 0) continue;
          const int ix = X + dx, iy = Y + dy, iz = Z + dz;
          if (ix < 0 || ix >= a.nx || iy < 0 || iy >= a.ny || iz < 0 || iz >= a.nz) continue;
          const size_t io = (static_cast<size_t>(iz) * a.ny + iy) * a.pitch + ix;
          const float wgt = fabsf(xk - a.x[io]) + a.e[io];
          const float q2 = static_cast<float>(dx * dx + dy * dy + dz * dz);
#pragma unroll
          for (int j = 0; j < C; ++j) {
            sh[j] = fmaf(a.A[j * plane + io], wgt, sh[j]);
            sf[j] = fmaf(a.B[j * plane + io], q2, sf[j]);
          }
        }
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const float uk = a.u[j * plane + off];
      a.ubar_out[j * plane + off] = fmaf(2.0f * uk, sf[j], sh[j]);
    }
  }
}

// grad[0..1] += the blocks' lambda_bar, xi_bar; cbar_out = sum of c_bar^t.
template <int C>
__global__ void adjoint_reduce_kernel(const double* partials, int blocks, double* grad,
                                      double* cbar_out) {
  constexpr int NV = 2 + C;
  const int v = threadIdx.x;
  if (v >= NV) return;
  double s = 0.0;
  for (int b = 0; b < blocks; ++b) s += partials[static_cast<size_t>(b) * NV + v];
  if (v < 2) grad[v] += s;
  else cbar_out[v - 2] = s;
}

// The polish loop's bookkeeping.  mode 0: best = (lambda, xi, +inf).
// mode 1: keep the best point seen, then one projected, normalised descent
// step (lambda, xi) <- clip((lambda, xi) - alpha g / |g|, 0, 1).  mode 2: keep
// the best point seen and return it in lam_xi.
__global__ void polish_step_kernel(double* lam_xi, const double* grad, const double* J,
                                   double* best, double alpha, int mode) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (mode == 0) {
    best[0] = lam_xi[0];
    best[1] = lam_xi[1];
    best[2] = CUDART_INF;
    return;
  }
  if (J[0] < best[2]) {
    best[0] = lam_xi[0];
    best[1] = lam_xi[1];
    best[2] = J[0];
  }
  if (mode == 2) {
    lam_xi[0] = best[0];
    lam_xi[1] = best[1];
    return;
  }
  const double g0 = grad[0], g1 = grad[1];
  const double nrm = sqrt(g0 * g0 + g1 * g1);
  if (nrm > 0.0) {
    lam_xi[0] = fmin(fmax(lam_xi[0] - alpha * g0 / nrm, 0.0), 1.0);
    lam_xi[1] = fmin(fmax(lam_xi[1] - alpha * g1 / nrm, 0.0), 1.0);
  }
}

#define PIFCM_ADJ_DISPATCH(c, CALL)  \
  switch (c) {                        \
    case 2: { constexpr int C = 2; CALL; } \
    case 3: { constexpr int C = 3; CALL; } \
    case 4: { constexpr int C = 4; CALL; } \
    case 5: { constexpr int C = 5; CALL; } \
    case 6: { constexpr int C = 6; CALL; } \
    case 7: { constexpr int C = 7; CALL; } \
    case 8: { constexpr int C = 8; CALL; } \
    default: return cudaErrorInvalidValue; \
  }

}  // namespace

int adjoint_blocks(int nx, int ny, int nz) {
  return ((nx + ATX - 1) / ATX) * ((ny + ATY - 1) / ATY) * ((nz + AZ - 1) / AZ);
}

template <int C>
cudaError_t launch_point_c(const AdjointArgs& a, int blocks, cudaStream_t s) {
  const int smem = 3 * (1 + C) * HP * static_cast<int>(sizeof(float));
  cudaError_t e = cudaFuncSetAttribute(adjoint_point_kernel<C>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  adjoint_point_kernel<C><<<blocks, AT, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_point(int c, const AdjointArgs& a, int blocks, cudaStream_t s) {
  PIFCM_ADJ_DISPATCH(c, return launch_point_c<C>(a, blocks, s));
}

cudaError_t launch_adjoint_gather(int c, const AdjointArgs& a, cudaStream_t s) {
  long long b = (static_cast<long long>(a.nx) * a.ny * a.nz + AT - 1) / AT;
  if (b > 152LL * 8) b = 152LL * 8;                 // grid-stride beyond 8 blocks per SM
  const int blocks = b < 1 ? 1 : static_cast<int>(b);
  PIFCM_ADJ_DISPATCH(c, (adjoint_gather_kernel<C><<<blocks, AT, 0, s>>>(a));
                     return cudaGetLastError());
}

cudaError_t launch_adjoint_reduce(int c, const double* partials, int blocks, double* grad,
                                  double* cbar_out, cudaStream_t s) {
  PIFCM_ADJ_DISPATCH(c, (adjoint_reduce_kernel<C><<<1, 32, 0, s>>>(partials, blocks, grad,
                                                                 cbar_out));
                     return cudaGetLastError());
}

cudaError_t launch_polish_step(double* lam_xi, const double* grad, const double* J, double* best,
                               double alpha, int mode, cudaStream_t s) {
  polish_step_kernel<<<1, 32, 0, s>>>(lam_xi, grad, J, best, alpha, mode);
  return cudaGetLastError();
}

}  // namespace pifcm
