// Auxiliary kernels of the 3DPIFCM path: min-max normalisation (Algorithm 2
// step 1), the particle swarm (Algorithm 1 steps 3 and 5-8) with its
// Philox4x32-10 draws, best-particle selection (step 11), the copy-out of a
// run's final memberships, and the result block.
#include <math_constants.h>

#include <cuda_bf16.h>

#include "launch.h"

namespace pifcm {

namespace {

// ------------------------------------------------ Algorithm 2 step 1
constexpr int NT = 256;

__global__ void __launch_bounds__(NT) minmax_kernel(const float* __restrict__ v, int nx, int ny,
                                                    int nz, int pitch, float* pmin, float* pmax,
                                                    int32_t* pbad) {
  __shared__ float smin[NT], smax[NT];
  __shared__ int sbad[NT];
  float lo = CUDART_INF_F, hi = -CUDART_INF_F;
  int bad = 0;
  const long long rows = static_cast<long long>(ny) * nz;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const float* row = v + r * pitch;
    for (int x = threadIdx.x; x < nx; x += NT) {
      const float e = row[x];
      if (!isfinite(e)) bad = 1;
      lo = fminf(lo, e);
      hi = fmaxf(hi, e);
    }
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  sbad[threadIdx.x] = bad;
  __syncthreads();
  for (int h = NT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + h]);
      smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + h]);
      sbad[threadIdx.x] |= sbad[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pmin[blockIdx.x] = smin[0];
    pmax[blockIdx.x] = smax[0];
    pbad[blockIdx.x] = sbad[0];
  }
}

__global__ void __launch_bounds__(NT) scale_kernel(const float* v, float* x, int nx, int ny,
                                                   int nz, int pitch, const float* pmin,
                                                   const float* pmax, const int32_t* pbad,
                                                   int nparts, DevStatus* st) {
  __shared__ float smin[NT], smax[NT];
  __shared__ int sbad[NT];
  float lo = CUDART_INF_F, hi = -CUDART_INF_F;
  int bad = 0;
  for (int i = threadIdx.x; i < nparts; i += NT) {
    lo = fminf(lo, pmin[i]);
    hi = fmaxf(hi, pmax[i]);
    bad |= pbad[i];
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  sbad[threadIdx.x] = bad;
  __syncthreads();
  for (int h = NT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + h]);
      smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + h]);
      sbad[threadIdx.x] |= sbad[threadIdx.x + h];
    }
    __syncthreads();
  }
  const float mn = smin[0], mxv = smax[0];
  if (sbad[0] || !(mxv > mn)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(st, IFCM_ERR_INVALID, 2);
    return;
  }
  const float range = mxv - mn;
  const long long rows = static_cast<long long>(ny) * nz;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const float* in = v + r * pitch;
    float* out = x + r * pitch;
    for (int e = threadIdx.x; e < nx; e += NT) out[e] = __fdiv_rn(in[e] - mn, range);
  }
}

// ------------------------------------------------------- run copy-out
// dst <- the buffer holding U after `iters` iterations (odd: a, even: b).
__global__ void select_copy_kernel(const float4* a, const float4* b, const int32_t* iters,
                                   float4* dst, long long n4) {
  const float4* src = ((*iters) & 1) ? a : b;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n4;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    dst[i] = src[i];
}

// ------------------------------------------------ bf16 pair-word buffers
__device__ __forceinline__ uint32_t bf16_pair(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);   // lo in the low half
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Shared start as pair words: np = 2 -> word plane j = (u_j, u_j) (both
// particles of every pair start from it); np = 1 -> word plane k =
// (u_2k, u_2k+1), with 0 in the high half past the last cluster.  W is a
// bf16x2 word (uint32_t) or a float2 word.
__device__ __forceinline__ void put_pair(uint32_t* out, long long i, float lo, float hi) {
  out[i] = bf16_pair(lo, hi);
}
__device__ __forceinline__ void put_pair(float2* out, long long i, float lo, float hi) {
  out[i] = make_float2(lo, hi);
}
__device__ __forceinline__ float lane_of(uint32_t w, bool hi) {
  return __uint_as_float(hi ? (w & 0xffff0000u) : (w << 16));
}
__device__ __forceinline__ float lane_of(float2 w, bool hi) { return hi ? w.y : w.x; }

template <class W>
__global__ void pack_start_kernel(const float* u0, W* out, int c, int np, long long plane) {
  const int planes = np == 2 ? c : (c + 1) / 2;
  const long long n = static_cast<long long>(planes) * plane;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long k = i / plane, v = i - k * plane;
    if (np == 2) {
      const float u = u0[k * plane + v];
      put_pair(out, i, u, u);
    } else {
      const float lo = u0[(2 * k) * plane + v];
      const float hi = 2 * k + 1 < c ? u0[(2 * k + 1) * plane + v] : 0.0f;
      put_pair(out, i, lo, hi);
    }
  }
}

// Particle 0's memberships (unit 0, low lane for np = 2) as FP32 planes.
template <class W>
__global__ void unpack_select_kernel(const W* a, const W* b, const int32_t* iters, float* dst,
                                     int c, int np, long long plane) {
  const W* src = ((*iters) & 1) ? a : b;
  const long long n = static_cast<long long>(c) * plane;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long j = i / plane, v = i - j * plane;
    const W w = np == 2 ? src[j * plane + v] : src[(j >> 1) * plane + v];
    dst[i] = lane_of(w, np == 2 ? false : (j & 1));
  }
}

// 1/G of every voxel of a 3D volume (G = sum over the in-volume neighbours of
// |x_i - x_k|, Eqs 5-6; reading R4), summed in FP64 and rounded once; a G
// below FP32's range is stored as the largest float.  A flat neighbourhood
// (G = 0, reading R3) is stored as -1/(n g0), n its in-volume neighbours:
// stencil3d_kernel weighs every neighbour of such a voxel with g0 =
// |(x_i + 2) - x_k| = |(x_i + 2) - x_i| in FP32 (the same for all of them),
// which turns H into the plain mean of the neighbours' memberships.
__global__ void gsum_kernel(const float* __restrict__ x, int nx, int ny, int nz, int pitch,
                            float* __restrict__ out) {
  const long long n = static_cast<long long>(nx) * ny * nz;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int X = static_cast<int>(i % nx);
    const long long r = i / nx;
    const int Y = static_cast<int>(r % ny), Z = static_cast<int>(r / ny);
    const float xi = x[(static_cast<long long>(Z) * ny + Y) * pitch + X];
    double G = 0.0;
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int kx = X + dx, ky = Y + dy, kz = Z + dz;
          if ((dx == 0 && dy == 0 && dz == 0) || kx < 0 || kx >= nx || ky < 0 || ky >= ny ||
              kz < 0 || kz >= nz)
            continue;
          G += fabs(static_cast<double>(xi) -
                    static_cast<double>(x[(static_cast<long long>(kz) * ny + ky) * pitch + kx]));
          ++cnt;
        }
    float s;
    if (G > 0.0) s = static_cast<float>(fmin(1.0 / G, 3.4028234663852886e38));
    else if (cnt > 0) {
      const float g0 = fabsf(__fsub_rn(__fadd_rn(xi, 2.0f), xi));
      s = static_cast<float>(-1.0 / (static_cast<double>(cnt) * g0));
    } else {
      s = 0.0f;
    }
    out[(static_cast<long long>(Z) * ny + Y) * pitch + X] = s;
  }
}

__global__ void fill_kernel(float* dst, float value, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    dst[i] = value;
}

// -------------------------------------------- Philox4x32-10 (SC'11 s3.2)
struct U4 {
  uint32_t v[4];
};

__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c.v[0]), lo0 = M0 * c.v[0];
    const uint32_t hi1 = __umulhi(M1, c.v[2]), lo1 = M1 * c.v[2];
    U4 n;
    n.v[0] = hi1 ^ c.v[1] ^ k0;
    n.v[1] = lo1;
    n.v[2] = hi0 ^ c.v[3] ^ k1;
    n.v[3] = lo0;
    c = n;
  }
  return c;
}

// U[0,1) double from (generation, particle, dimension, stream) under `seed`.
__device__ __forceinline__ double swarm_uniform(uint64_t seed, uint32_t gen, uint32_t particle,
                                                uint32_t dim, uint32_t stream) {
  U4 c;
  c.v[0] = gen;
  c.v[1] = particle;
  c.v[2] = dim;
  c.v[3] = stream;
  const U4 r = philox10(c, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  const double hi = static_cast<double>(r.v[0] >> 5);
  const double lo = static_cast<double>(r.v[1] >> 6);
  return __dmul_rn(__dadd_rn(__dmul_rn(hi, 67108864.0), lo), 1.0 / 9007199254740992.0);
}

constexpr uint32_t kInitX = 0, kInitV = 1, kP1 = 2, kP2 = 3;

__global__ void pso_init_kernel(pso_state s) {
  const int i = threadIdx.x;
  if (i < s.P) {
    for (int d = 0; d < 2; ++d) {
      const double x = swarm_uniform(s.seed, 0, i, d, kInitX);
      const double u = swarm_uniform(s.seed, 0, i, d, kInitV);
      s.x[2 * i + d] = x;
      s.pbest_x[2 * i + d] = x;
      s.v[2 * i + d] = __dmul_rn(s.vmax, __dsub_rn(__dmul_rn(2.0, u), 1.0));
    }
    s.pbest_f[i] = CUDART_INF;
  }
  if (i == 0) *s.gen = 0;
}

// Algorithm 1 steps 5-8 for one generation; one thread per particle.
__global__ void pso_step_kernel(pso_state s, const double* fitness) {
  __shared__ double sf[kMaxP];
  const int i = threadIdx.x;
  const uint32_t gen = static_cast<uint32_t>(*s.gen);
  if (i < s.P) {
    const double f = fitness[i];
    if (f < s.pbest_f[i]) {                      // step 5 (strict)
      s.pbest_f[i] = f;
      s.pbest_x[2 * i] = s.x[2 * i];
      s.pbest_x[2 * i + 1] = s.x[2 * i + 1];
    }
    sf[i] = s.pbest_f[i];
  }
  __syncthreads();
  if (i < s.P) {
    int best = -1;                               // step 6: ring neighbours
    for (int o = -s.radius; o <= s.radius; ++o) {
      int k = (i + o) % s.P;
      if (k < 0) k += s.P;
      if (best < 0 || sf[k] < sf[best] || (sf[k] == sf[best] && k < best)) best = k;
    }
    for (int d = 0; d < 2; ++d) {                // steps 7-8
      const double p1 = swarm_uniform(s.seed, gen, i, d, kP1);
      const double p2 = swarm_uniform(s.seed, gen, i, d, kP2);
      const double x = s.x[2 * i + d];
      const double a = __dmul_rn(p1, __dsub_rn(s.pbest_x[2 * i + d], x));
      const double b = __dmul_rn(p2, __dsub_rn(s.pbest_x[2 * best + d], x));
      double v = __dadd_rn(__dadd_rn(s.v[2 * i + d], a), b);
      v = fmin(fmax(v, -s.vmax), s.vmax);
      s.v[2 * i + d] = v;
      s.x[2 * i + d] = fmin(fmax(__dadd_rn(x, v), 0.0), 1.0);
    }
  }
  __syncthreads();
  if (i == 0) *s.gen = static_cast<int32_t>(gen + 1);
}

// Best personal best (lowest fitness, ties to the lowest index).
__global__ void pso_best_kernel(const double* pbest_x, const double* pbest_f, int P,
                                double* lam_xi, int32_t* best) {
  if (threadIdx.x != 0) return;
  int b = 0;
  for (int i = 1; i < P; ++i)
    if (pbest_f[i] < pbest_f[b]) b = i;
  lam_xi[0] = pbest_x[2 * b];
  lam_xi[1] = pbest_x[2 * b + 1];
  if (best) *best = b;
}

__global__ void result_kernel(int c, const double* centres, const double* lam_xi,
                              const double* J, const double* pbest_f, int P,
                              const int32_t* iters_final, const int32_t* iters_init,
                              const unsigned long long* updates, const int32_t* best,
                              const DevStatus* status, pifcm_result* out) {
  if (threadIdx.x != 0) return;
  for (int j = 0; j < 8; ++j) out->centres[j] = j < c ? centres[j] : 0.0;
  out->lambda = lam_xi[0];
  out->xi = lam_xi[1];
  out->J = J[0];
  double bf = CUDART_INF;
  for (int i = 0; i < P; ++i) bf = fmin(bf, pbest_f[i]);
  out->best_fitness = bf;
  out->updates = static_cast<int64_t>(*updates);
  out->iters_final = *iters_final;
  out->iters_init = *iters_init;
  out->status = status->status;
  out->best_particle = best ? *best : 0;
}

}  // namespace

cudaError_t launch_minmax(const float* v, int nx, int ny, int nz, int pitch, float* pmin,
                          float* pmax, int32_t* pbad, int blocks, cudaStream_t s) {
  minmax_kernel<<<blocks, NT, 0, s>>>(v, nx, ny, nz, pitch, pmin, pmax, pbad);
  return cudaGetLastError();
}

cudaError_t launch_scale(const float* v, float* x, int nx, int ny, int nz, int pitch,
                         const float* pmin, const float* pmax, const int32_t* pbad, int nparts,
                         DevStatus* st, cudaStream_t s) {
  scale_kernel<<<nparts, NT, 0, s>>>(v, x, nx, ny, nz, pitch, pmin, pmax, pbad, nparts, st);
  return cudaGetLastError();
}

cudaError_t launch_select_copy(const float* a, const float* b, const int32_t* iters,
                               float* dst, long long n, cudaStream_t s) {
  const long long n4 = n / 4;
  long long blocks = (n4 + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  select_copy_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(
      reinterpret_cast<const float4*>(a), reinterpret_cast<const float4*>(b), iters,
      reinterpret_cast<float4*>(dst), n4);
  return cudaGetLastError();
}

cudaError_t launch_pack_start(const float* u0, void* out, int c, int np, int layout,
                              long long plane, cudaStream_t s) {
  const long long n = static_cast<long long>(np == 2 ? c : (c + 1) / 2) * plane;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  if (layout == UL_BF16)
    pack_start_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(
        u0, static_cast<uint32_t*>(out), c, np, plane);
  else
    pack_start_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(
        u0, static_cast<float2*>(out), c, np, plane);
  return cudaGetLastError();
}

cudaError_t launch_unpack_select(const void* a, const void* b, const int32_t* iters, float* dst,
                                 int c, int np, int layout, long long plane, cudaStream_t s) {
  const long long n = static_cast<long long>(c) * plane;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  if (layout == UL_BF16)
    unpack_select_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(
        static_cast<const uint32_t*>(a), static_cast<const uint32_t*>(b), iters, dst, c, np,
        plane);
  else
    unpack_select_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(
        static_cast<const float2*>(a), static_cast<const float2*>(b), iters, dst, c, np, plane);
  return cudaGetLastError();
}

cudaError_t launch_fill(float* dst, float value, long long n, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  fill_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(dst, value, n);
  return cudaGetLastError();
}

cudaError_t launch_gsum(const float* x, int nx, int ny, int nz, int pitch, float* s_out,
                        cudaStream_t s) {
  const long long n = static_cast<long long>(nx) * ny * nz;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  gsum_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(x, nx, ny, nz, pitch, s_out);
  return cudaGetLastError();
}

cudaError_t launch_pso_init(const pso_state& st, cudaStream_t s) {
  pso_init_kernel<<<1, kMaxP, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_pso_step(const pso_state& st, const double* fitness, cudaStream_t s) {
  pso_step_kernel<<<1, kMaxP, 0, s>>>(st, fitness);
  return cudaGetLastError();
}

cudaError_t launch_pso_best(const double* pbest_x, const double* pbest_f, int P,
                            double* lam_xi, int32_t* best, cudaStream_t s) {
  pso_best_kernel<<<1, 32, 0, s>>>(pbest_x, pbest_f, P, lam_xi, best);
  return cudaGetLastError();
}

cudaError_t launch_result(int c, const double* centres, const double* lam_xi, const double* J,
                          const double* pbest_f, int P, const int32_t* iters_final,
                          const int32_t* iters_init, const unsigned long long* updates,
                          const int32_t* best, const DevStatus* status, pifcm_result* out,
                          cudaStream_t s) {
  result_kernel<<<1, 32, 0, s>>>(c, centres, lam_xi, J, pbest_f, P, iters_final, iters_init,
                                 updates, best, status, out);
  return cudaGetLastError();
}

}  // namespace pifcm
