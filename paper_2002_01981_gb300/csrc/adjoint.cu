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
// One thread per voxel, neighbours read from global memory (L1 / L2), FP32
// arithmetic, per-block partials FP32 within a warp and FP64 across warps.
#include <math_constants.h>

#include "ifcm_math.cuh"
#include "launch.h"

namespace pifcm {

namespace {

constexpr int AT = 256;   // threads per block

// H, F of Eqs 5 and 7 from U^t at voxel (X, Y, Z), with G = sum g, Q = sum q^2
// and the in-volume neighbour count n.
template <int C>
__device__ __forceinline__ void neighbour_terms(const AdjointArgs& a, int X, int Y, int Z,
                                                float xc, size_t plane, float (&H)[C],
                                                float (&F)[C], float& G, float& Q, int& n) {
#pragma unroll
  for (int j = 0; j < C; ++j) H[j] = F[j] = 0.0f;
  G = 0.0f;
  Q = 0.0f;
  n = 0;
  float S[C];
#pragma unroll
  for (int j = 0; j < C; ++j) S[j] = 0.0f;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (dx == 0 && dy == 0 && dz == 0) continue;
        const int kx = X + dx, ky = Y + dy, kz = Z + dz;
        if (kx < 0 || kx >= a.nx || ky < 0 || ky >= a.ny || kz < 0 || kz >= a.nz) continue;
        const size_t ko = (static_cast<size_t>(kz) * a.ny + ky) * a.pitch + kx;
        const float g = fabsf(xc - a.x[ko]);
        const float q2 = static_cast<float>(dx * dx + dy * dy + dz * dz);
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const float uk = a.u[j * plane + ko];
          H[j] = fmaf(uk, g, H[j]);
          F[j] = fmaf(uk * uk, q2, F[j]);
          S[j] += uk;
        }
        G += g;
        Q += q2;
        ++n;
      }
  if (n == 0) return;                          // no neighbours: H = F = 0
  const float invQ = __frcp_rn(Q);
#pragma unroll
  for (int j = 0; j < C; ++j) F[j] *= invQ;
  if (G > 0.0f) {
    const float invG = __frcp_rn(G);
#pragma unroll
    for (int j = 0; j < C; ++j) H[j] *= invG;
  } else {                                     // reading R3: plain mean
    const float inv = __frcp_rn(static_cast<float>(n));
#pragma unroll
    for (int j = 0; j < C; ++j) H[j] = S[j] * inv;
  }
}

template <int C>
__global__ void __launch_bounds__(AT) adjoint_point_kernel(const AdjointArgs a) {
  __shared__ float s_red[AT / 32][2 + C];
  const long long nvox = static_cast<long long>(a.nx) * a.ny * a.nz;
  const size_t plane = static_cast<size_t>(a.nz) * a.ny * a.pitch;
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

  for (long long i = blockIdx.x * static_cast<long long>(AT) + threadIdx.x; i < nvox;
       i += static_cast<long long>(gridDim.x) * AT) {
    const int X = static_cast<int>(i % a.nx);
    const long long yz = i / a.nx;
    const int Y = static_cast<int>(yz % a.ny);
    const int Z = static_cast<int>(yz / a.ny);
    const size_t off = (static_cast<size_t>(Z) * a.ny + Y) * a.pitch + X;
    const float xc = a.x[off];
    float H[C], F[C], G, Q;
    int n;
    neighbour_terms<C>(a, X, Y, Z, xc, plane, H, F, G, Q, n);
    // Eq 4 (reading R2) and Eq 2
    float D[C], f[C], fac[C], P[C], d2[C], u[C];
    float S = 0.0f;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const float dd = xc - ct[j];
      D[j] = dd * dd;
      f[j] = 1.0f - lam * H[j] - xi * F[j];
      fac[j] = fmaxf(f[j], 0.0f);
      P[j] = D[j] * fac[j];
      d2[j] = fmaxf(P[j], a.dist_floor);
      u[j] = a.m_is_2 ? __frcp_rn(d2[j]) : exp2f(-a.inv_m1 * log2f(d2[j]));
      S += u[j];
    }
    const float invS = __frcp_rn(S);
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
    const float invG = G > 0.0f ? __frcp_rn(G) : (n > 0 ? __frcp_rn(static_cast<float>(n)) : 0.0f);
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

int adjoint_blocks(long long nvox) {
  long long b = (nvox + AT - 1) / AT;
  const long long cap = 152LL * 8;
  if (b > cap) b = cap;
  return b < 1 ? 1 : static_cast<int>(b);
}

cudaError_t launch_adjoint_point(int c, const AdjointArgs& a, int blocks, cudaStream_t s) {
  PIFCM_ADJ_DISPATCH(c, (adjoint_point_kernel<C><<<blocks, AT, 0, s>>>(a));
                     return cudaGetLastError());
}

cudaError_t launch_adjoint_gather(int c, const AdjointArgs& a, int blocks, cudaStream_t s) {
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
