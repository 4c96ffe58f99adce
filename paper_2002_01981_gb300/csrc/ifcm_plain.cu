// The plain IFCM iteration with V > 1 shells (one thread per voxel,
// neighbours read straight from global memory), the per-particle reduction
// that finalises every iteration (Eq 3 centres, Eq 1 objective, stop rule),
// the run-state initialisation, and the dispatch of the plain iteration (the
// V = 1 kernel is in plain_kernel.cu).
#include "ifcm_math.cuh"
#include "launch.h"

namespace pifcm {

namespace {

constexpr int PT = 256;   // threads per block of the plain kernel

// Mean of u_kj over the in-volume voxels of the shell at Chebyshev distance r
// around (X, Y, Z): the shell's H term where all its g_ik are 0 (reading R3).
template <int C>
__device__ __noinline__ void shell_mean(const float* __restrict__ u, int X, int Y, int Z, int r,
                                        int nx, int ny, int nz, int pitch, float (&Hr)[C]) {
  const size_t plane = static_cast<size_t>(nz) * ny * pitch;
  float s[C];
#pragma unroll
  for (int j = 0; j < C; ++j) s[j] = 0.0f;
  int n = 0;
  for (int dz = -r; dz <= r; ++dz)
    for (int dy = -r; dy <= r; ++dy) {
      const bool face = (dz == -r || dz == r || dy == -r || dy == r);
      for (int dx = -r; dx <= r; dx += face ? 1 : 2 * r) {
        const int kx = X + dx, ky = Y + dy, kz = Z + dz;
        if (kx < 0 || kx >= nx || ky < 0 || ky >= ny || kz < 0 || kz >= nz) continue;
        const size_t ko = (static_cast<size_t>(kz) * ny + ky) * pitch + kx;
#pragma unroll
        for (int j = 0; j < C; ++j) s[j] += u[j * plane + ko];
        ++n;
      }
    }
  const float inv = n > 0 ? 1.0f / static_cast<float>(n) : 0.0f;
#pragma unroll
  for (int j = 0; j < C; ++j) Hr[j] = s[j] * inv;
}

// H and F of Eqs 5 and 7 with V shells (reading R17: shell r is the surface
// of the cube of Chebyshev radius r), weighted by W_r of Eq 10 and
// renormalised over the shells that hold an in-volume voxel.
template <int C>
__device__ void shell_terms(const PlainArgs& a, const ShellArgs& sh, const float* __restrict__ u,
                            int X, int Y, int Z, float xc, float (&H)[C], float (&F)[C]) {
  const size_t plane = static_cast<size_t>(a.nz) * a.ny * a.pitch;
  float wsum = 0.0f;
#pragma unroll
  for (int j = 0; j < C; ++j) H[j] = F[j] = 0.0f;
  for (int r = 1; r <= sh.V; ++r) {
    float hr[C], fr[C], G = 0.0f, Q = 0.0f;
    int n = 0;
#pragma unroll
    for (int j = 0; j < C; ++j) hr[j] = fr[j] = 0.0f;
    for (int dz = -r; dz <= r; ++dz)
      for (int dy = -r; dy <= r; ++dy) {
        const bool face = (dz == -r || dz == r || dy == -r || dy == r);
        for (int dx = -r; dx <= r; dx += face ? 1 : 2 * r) {
          const int kx = X + dx, ky = Y + dy, kz = Z + dz;
          if (kx < 0 || kx >= a.nx || ky < 0 || ky >= a.ny || kz < 0 || kz >= a.nz) continue;
          const size_t ko = (static_cast<size_t>(kz) * a.ny + ky) * a.pitch + kx;
          const float g = fabsf(xc - a.x[ko]);                                // Eq 6
          const float q2 = static_cast<float>(dx * dx + dy * dy + dz * dz);   // Eq 8
#pragma unroll
          for (int j = 0; j < C; ++j) {
            const float uk = u ? u[j * plane + ko] : 1.0f / C;
            hr[j] = fmaf(uk, g, hr[j]);
            fr[j] = fmaf(uk * uk, q2, fr[j]);
          }
          G += g;
          Q += q2;
          ++n;
        }
      }
    if (n == 0) continue;                      // empty shell: dropped
    if (G > 0.0f) {
      const float invG = __frcp_rn(G);
#pragma unroll
      for (int j = 0; j < C; ++j) hr[j] *= invG;
    } else if (u) {
      shell_mean<C>(u, X, Y, Z, r, a.nx, a.ny, a.nz, a.pitch, hr);
    } else {
#pragma unroll
      for (int j = 0; j < C; ++j) hr[j] = 1.0f / C;
    }
    const float invQ = __frcp_rn(Q), w = sh.W[r - 1];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      H[j] = fmaf(w, hr[j], H[j]);
      F[j] = fmaf(w, fr[j] * invQ, F[j]);
    }
    wsum += w;
  }
  if (wsum > 0.0f) {
    const float inv = __frcp_rn(wsum);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      H[j] *= inv;
      F[j] *= inv;
    }
  }
}

// The plain iteration with V > 1 shells (Eq 10, reading R17) for P
// particles at once (grid y = particle).  The V = 1, one-particle kernel
// (plain_kernel.cu) is the paper-shaped form and the FCM start; it is
// compiled apart so that its code stays that of the plain form alone.
template <int C>
__global__ void __launch_bounds__(PT) plain_shell_kernel(const PlainArgs a, const ShellArgs sh) {
  __shared__ float s_red[PT / 32][2 * C + 2];
  const int pid = blockIdx.y;                  // particle of the launch
  if (!a.active[pid]) return;
  const long long nvox = static_cast<long long>(a.nx) * a.ny * a.nz;
  const size_t plane = static_cast<size_t>(a.nz) * a.ny * a.pitch;
  // the particle's U^t and U^{t+1}; a.u_src == NULL (u = 1/c) is tested on the
  // kernel parameter itself so that the test stays uniform and out of the loops
  const long long soff = pid * sh.src_pstride, doff = pid * sh.dst_pstride;
  MethodConsts k;
  if (a.lam_xi) {
    k.lam = static_cast<float>(a.lam_xi[2 * pid]);
    k.xi = static_cast<float>(a.lam_xi[2 * pid + 1]);
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
  for (int j = 0; j < C; ++j) cc[j] = static_cast<float>(a.centres[pid * C + j]);
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
    for (int j = 0; j < C; ++j) uc[j] = a.u_src ? a.u_src[soff + j * plane + off] : 1.0f / C;
    float H[C], F[C];
#pragma unroll
    for (int j = 0; j < C; ++j) H[j] = F[j] = 0.0f;
    if (stencil) {
      shell_terms<C>(a, sh, a.u_src ? a.u_src + soff : nullptr, X, Y, Z, xc, H, F);
    }
    float u[C], um[C], Jv;
    voxel_update<C>(H, F, xc, cc, k, u, um, Jv);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      if (IFCM_CHECK(doff + static_cast<long long>((j + 1) * plane) <= a.dst_elems, a.status, 41))
        a.u_dst[doff + j * plane + off] = u[j];
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
  const size_t rec = static_cast<size_t>(pid) * sh.n_rec + blockIdx.x;
  if (!IFCM_CHECK(static_cast<long long>(rec) < a.n_records, a.status, 42)) {
  } else if (threadIdx.x < 2 * C + 1) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < PT / 32; ++w) sum += static_cast<double>(s_red[w][threadIdx.x]);
    a.partials[rec * (2 * C + 1) + threadIdx.x] = sum;
  } else if (threadIdx.x == 2 * C + 1) {
    float mm = 0.0f;
#pragma unroll
    for (int w = 0; w < PT / 32; ++w) mm = fmaxf(mm, s_red[w][2 * C + 1]);
    a.dmax[rec] = mm;
  }
}

// One block per particle: FP64 sum of the particle's partial records in a
// fixed order (so the result does not depend on scheduling), then Eq 3
// centres, the Eq 1 objective, and the stop rule of the run.
constexpr int RT = 256;

// Per-particle finalisation with compensated FP32 sums instead of FP64: each
// thread sums its records with Neumaier's method, the (sum, compensation)
// pairs are combined pairwise in shared memory, and Eqs 3 and 1 are taken in
// FP32 from sum + compensation.  max|du| and the stop rule are as in FP64.
// s_hi, s_lo: NV x RT floats each; s_mx: RT floats (the FP64 path's shared
// arrays, reused).
template <int C>
__device__ __noinline__ void reduce_comp32(const ReduceArgs& a, const ReduceVol& rv, int gp,
                                           int p, const double* rec, long long first,
                                           float (*s_hi)[RT], float (*s_lo)[RT], float* s_mx) {
  constexpr int NV = 2 * C + 1;
  float hi[NV], lo[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) hi[v] = lo[v] = 0.0f;
  float mx = 0.0f;
  for (int r = threadIdx.x; r < rv.n_rec; r += RT) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
      neumaier_add(hi[v], lo[v], static_cast<float>(rec[static_cast<size_t>(r) * NV + v]));
    mx = fmaxf(mx, a.dmax[first + r]);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    s_hi[v][threadIdx.x] = hi[v];
    s_lo[v][threadIdx.x] = lo[v];
  }
  s_mx[threadIdx.x] = mx;
  __syncthreads();
  for (int h = RT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float sh = s_hi[v][threadIdx.x], sl = s_lo[v][threadIdx.x];
        neumaier_add(sh, sl, s_hi[v][threadIdx.x + h]);
        s_hi[v][threadIdx.x] = sh;
        s_lo[v][threadIdx.x] = __fadd_rn(sl, s_lo[v][threadIdx.x + h]);
      }
      s_mx[threadIdx.x] = fmaxf(s_mx[threadIdx.x], s_mx[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* cen = a.st.centres + static_cast<size_t>(gp) * C;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const float S0 = __fadd_rn(s_hi[j][0], s_lo[j][0]);
      const float S1 = __fadd_rn(s_hi[C + j][0], s_lo[C + j][0]);
      if (S0 > 0.0f) cen[j] = static_cast<double>(__fdiv_rn(S1, S0));   // Eq 3
      if (rv.c_out) rv.c_out[static_cast<size_t>(p) * C + j] = cen[j];
    }
    const double J = static_cast<double>(__fadd_rn(s_hi[2 * C][0], s_lo[2 * C][0]));  // Eq 1
    a.st.J[gp] = J;
    const int it = a.st.iters[gp] + 1;
    a.st.iters[gp] = it;
    if (rv.trace && it <= a.max_iter) {
      double* tr = rv.trace + (static_cast<size_t>(p) * a.max_iter + (it - 1)) * (2 * C + 1);
#pragma unroll
      for (int j = 0; j < C; ++j) {
        tr[j] = cen[j];
        tr[C + j] = static_cast<double>(__fadd_rn(s_hi[j][0], s_lo[j][0]));
      }
      tr[2 * C] = J;
    }
    if (rv.fitness) rv.fitness[p] = J;
    if (rv.iters_out) rv.iters_out[p] = it;
    const double delta = static_cast<double>(s_mx[0]);
    if (!(delta >= a.eps) || it >= a.max_iter) a.st.active[gp] = 0;
    atomicAdd(a.st.updates, static_cast<unsigned long long>(rv.nvox));
  }
}

template <int C>
__global__ void __launch_bounds__(RT) reduce_kernel(const ReduceArgs a) {
  constexpr int NV = 2 * C + 1;
  __shared__ double s_sum[NV][RT];
  __shared__ float s_max[RT];
  const int gp = blockIdx.x;                 // particle of the launch
  // launched as a dependent of the stencil launch before it
  grid_dep_trigger();
  grid_dep_wait();
  if (!a.st.active[gp]) return;
  int vi = 0;
  while (vi + 1 < a.n_vol && a.vol[vi + 1].pbase <= gp) ++vi;
  const ReduceVol& rv = a.vol[vi];
  const int p = gp - rv.pbase;               // the volume's particle
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  float mx = 0.0f;
  const long long first = rv.rec_base + static_cast<long long>(p) * rv.n_rec;
  if (!IFCM_CHECK(first >= 0 && first + rv.n_rec <= a.n_records, a.status, 40)) return;
  const double* rec = a.partials + first * NV;
  if (a.reduce == IFCM_REDUCE_COMP32) {
    float(*fs)[RT] = reinterpret_cast<float(*)[RT]>(&s_sum[0][0]);
    reduce_comp32<C>(a, rv, gp, p, rec, first, fs, fs + NV, s_max);
    return;
  }
  for (int r = threadIdx.x; r < rv.n_rec; r += RT) {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] += rec[static_cast<size_t>(r) * NV + v];
    mx = fmaxf(mx, a.dmax[first + r]);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) s_sum[v][threadIdx.x] = acc[v];
  s_max[threadIdx.x] = mx;
  __syncthreads();
  for (int h = RT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
#pragma unroll
      for (int v = 0; v < NV; ++v) s_sum[v][threadIdx.x] += s_sum[v][threadIdx.x + h];
      s_max[threadIdx.x] = fmaxf(s_max[threadIdx.x], s_max[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* cen = a.st.centres + static_cast<size_t>(gp) * C;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const double S0 = s_sum[j][0], S1 = s_sum[C + j][0];
      if (S0 > 0.0) cen[j] = S1 / S0;                        // Eq 3
      if (rv.c_out) rv.c_out[static_cast<size_t>(p) * C + j] = cen[j];
    }
    const double J = s_sum[2 * C][0];                       // Eq 1
    a.st.J[gp] = J;
    const int it = a.st.iters[gp] + 1;
    a.st.iters[gp] = it;
    if (rv.trace && it <= a.max_iter) {    // C^{t+1}, S0^{t+1}, J^t for the reverse pass
      double* tr = rv.trace + (static_cast<size_t>(p) * a.max_iter + (it - 1)) * (2 * C + 1);
#pragma unroll
      for (int j = 0; j < C; ++j) {
        tr[j] = cen[j];
        tr[C + j] = s_sum[j][0];
      }
      tr[2 * C] = J;
    }
    if (rv.fitness) rv.fitness[p] = J;
    if (rv.iters_out) rv.iters_out[p] = it;
    const double delta = static_cast<double>(s_max[0]);
    if (!(delta >= a.eps) || it >= a.max_iter) a.st.active[gp] = 0;
    atomicAdd(a.st.updates, static_cast<unsigned long long>(rv.nvox));
  }
}

template <int C>
__global__ void run_init_kernel(int P, const double* c0, RunState st, double* J_clear) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
#pragma unroll
  for (int j = 0; j < C; ++j)
    st.centres[static_cast<size_t>(p) * C + j] = c0 ? c0[j] : (j + 0.5) / C;
  st.active[p] = 1;
  st.iters[p] = 0;
  st.J[p] = 0.0;
  if (J_clear) J_clear[p] = 0.0;
}

#define PIFCM_DISPATCH_C(c, CALL)  \
  switch (c) {                     \
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

// Defined in plain_kernel.cu.
cudaError_t launch_plain_v1(int c, const PlainArgs& a, int blocks, cudaStream_t s);

int plain_blocks(long long nvox, int vpt) {
  const long long per = static_cast<long long>(PT) * vpt;
  return static_cast<int>((nvox + per - 1) / per);
}

cudaError_t launch_plain(int c, const PlainArgs& a, const ShellArgs& sh, int blocks,
                         cudaStream_t s) {
  if (sh.P < 1 || sh.V < 1 || sh.V > kMaxV) return cudaErrorInvalidValue;
  if (sh.V > 1 && a.stencil) {
    const dim3 grid(blocks, sh.P);
    PIFCM_DISPATCH_C(c, (plain_shell_kernel<C><<<grid, PT, 0, s>>>(a, sh));
                     return cudaGetLastError());
  }
  if (sh.P != 1) return cudaErrorInvalidValue;    // V = 1 batches run the stencil kernel
  return launch_plain_v1(c, a, blocks, s);
}

cudaError_t launch_reduce(int c, const ReduceArgs& a, cudaStream_t s) {
  PIFCM_DISPATCH_C(c, return launch_dependent(reduce_kernel<C>, dim3(a.P_total), dim3(RT), 0, s, a));
}

cudaError_t launch_run_init(int c, int P, const double* c0, RunState st, double* J_clear,
                            cudaStream_t s) {
  const int b = (P + 127) / 128;
  PIFCM_DISPATCH_C(c, (run_init_kernel<C><<<b, 128, 0, s>>>(P, c0, st, J_clear));
                   return cudaGetLastError());
}

}  // namespace pifcm
