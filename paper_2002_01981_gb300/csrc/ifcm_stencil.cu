// Batched IFCM iteration: the neighbourhood stencil of Eqs 5-9 fused with the
// distance (Eq 4), membership (Eq 2), objective (Eq 1) and centre sums (Eq 3),
// for every active particle of a batch, in one persistent launch.
//
// Work item = (particle, TX x TY column tile, z-chunk of tz planes).  A CTA
// walks its items' planes in order; for each plane one thread issues two TMA
// tile loads (the normalised volume x and the c membership planes U^t of the
// particle, each with a one-voxel halo in y and an aligned four-voxel margin in
// x) into a ring of shared-memory stages completed by mbarriers.  Thread (tx,
// ty) owns column (x0 + tx, y0 + ty) and keeps three centres of that column in
// registers: the plane just loaded contributes to the centre below it
// (dz = +1), to its own centre (dz = 0) and to the centre above (dz = -1), so
// every plane is read from shared memory once.  Neighbours outside the volume
// are excluded (reading R4): TMA fills them with zero memberships and the
// per-neighbour weight g is masked in edge tiles.  Once a centre has seen its
// three planes it is finalised: H = sum u g / sum g, F = sum u^2 q^2 / sum q^2
// (q^2 = dx^2+dy^2+dz^2, reading R1), then Eqs 4, 2, 1, 3.  U^{t+1} is written
// straight from registers; per-item sums of u^m, u^m x, the J share and
// max|du| go to a partial record, reduced per particle in FP64 by the reduce
// kernel.
#include <cstdio>

#include "ifcm_math.cuh"
#include "launch.h"

namespace pifcm {

namespace {

constexpr int TX = kTX, TY = kTY, NT = kThreads;
constexpr int BX = TX + 8;          // x box: 4-voxel aligned margins (TMA x must be 16-B aligned)
constexpr int BY = TY + 2;          // y box: one-voxel halo
constexpr int PLANE = BX * BY;      // floats in one channel of a stage
constexpr int NSTAGE = 4;
constexpr int XBYTES = ((PLANE * 4 + 127) / 128) * 128;

template <int C>
__host__ __device__ constexpr int stage_bytes() {
  return ((XBYTES + C * PLANE * 4 + 127) / 128) * 128;
}
template <int C>
__host__ __device__ constexpr uint32_t stage_tx_bytes() {
  return static_cast<uint32_t>((1 + C) * PLANE * 4);
}

struct Item {
  int p, tile, x0, y0, z0, z1, pzb, pze;
};

__device__ __forceinline__ Item decode_item(const StencilArgs& a, const int* act, long long w) {
  Item it;
  const int ap = static_cast<int>(w / a.n_tiles);
  it.tile = static_cast<int>(w - static_cast<long long>(ap) * a.n_tiles);
  it.p = act[ap];
  const int per_z = a.tiles_x * a.tiles_y;
  const int zc = it.tile / per_z;
  const int rem = it.tile - zc * per_z;
  const int ty = rem / a.tiles_x;
  const int tx = rem - ty * a.tiles_x;
  it.x0 = tx * TX;
  it.y0 = ty * TY;
  it.z0 = zc * a.tz;
  it.z1 = min(it.z0 + a.tz, a.nz);
  it.pzb = max(it.z0 - 1, 0);
  it.pze = min(it.z1, a.nz - 1);
  return it;
}

// Accumulators of one centre voxel of the thread's column.
template <int C>
struct Slot {
  float G;        // sum_k g_ik (Eq 5 denominator)
  float H[C];     // sum_k u_kj g_ik (Eq 5 numerator)
  float F[C];     // sum_k u_kj^2 q^2_ik (Eq 7 numerator)
  float xc;       // x_i
  float uc[C];    // u^t_ij (for max|du|)
  __device__ __forceinline__ void clear() {
    G = 0.0f;
#pragma unroll
    for (int j = 0; j < C; ++j) H[j] = F[j] = 0.0f;
  }
};

// Contributions of one loaded plane to the three centres of the column.
// EDGE: mask neighbours outside the volume in x/y.  Z3: the volume has more
// than one plane (otherwise only the in-plane 8-neighbourhood exists).
template <int C, bool EDGE, bool Z3>
__device__ __forceinline__ void accumulate_plane(const float* __restrict__ xs,
                                                 const float* __restrict__ us, int tx, int ty,
                                                 const float (&mx)[3], const float (&my)[3],
                                                 Slot<C>& lo, Slot<C>& mid, Slot<C>& hi) {
  float A[C], B[C];   // sum_k w and sum_k (dx^2+dy^2) w over the 3x3 window, w = u^2
#pragma unroll
  for (int j = 0; j < C; ++j) A[j] = B[j] = 0.0f;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int off = (ty + 1 + dy) * BX + (tx + 4 + dx);
      const float xk = xs[off];
      float uk[C];
#pragma unroll
      for (int j = 0; j < C; ++j) uk[j] = us[j * PLANE + off];
      const bool self = (dx == 0 && dy == 0);
      float mk = 1.0f;
      if (EDGE) mk = mx[dx + 1] * my[dy + 1];
      if (Z3) {
        float gl = fabsf(lo.xc - xk), gh = fabsf(hi.xc - xk);
        if (EDGE) { gl *= mk; gh *= mk; }
        lo.G += gl;
        hi.G += gh;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          lo.H[j] = fmaf(uk[j], gl, lo.H[j]);
          hi.H[j] = fmaf(uk[j], gh, hi.H[j]);
        }
      }
      if (!self) {
        float gm = fabsf(mid.xc - xk);
        if (EDGE) gm *= mk;
        mid.G += gm;
#pragma unroll
        for (int j = 0; j < C; ++j) mid.H[j] = fmaf(uk[j], gm, mid.H[j]);
      }
      const int q2 = (dx * dx + dy * dy);   // folded after unrolling
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const float wk = uk[j] * uk[j];
        A[j] += wk;
        if (q2 == 1) B[j] += wk;
        if (q2 == 2) B[j] = fmaf(2.0f, wk, B[j]);
      }
    }
  }
  // planes above / below: q^2 = 1 + dx^2 + dy^2; same plane: q^2 = dx^2 + dy^2
#pragma unroll
  for (int j = 0; j < C; ++j) {
    if (Z3) {
      const float ab = A[j] + B[j];
      lo.F[j] += ab;
      hi.F[j] += ab;
    }
    mid.F[j] += B[j];
  }
}

template <int C>
struct Sums {
  float s0[C], s1[C], J, dm;
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int j = 0; j < C; ++j) s0[j] = s1[j] = 0.0f;
    J = dm = 0.0f;
  }
};

template <int C>
__device__ __forceinline__ void finalize_centre(const Slot<C>& sl, int X, int Y, int z,
                                                const StencilArgs& a, int p,
                                                const float (&cc)[C], const MethodConsts& k,
                                                Sums<C>& acc) {
  int cnt;
  float Q;
  box_counts(X, Y, z, a.nx, a.ny, a.nz, cnt, Q);
  float H[C], F[C];
  if (cnt == 0) {
#pragma unroll
    for (int j = 0; j < C; ++j) H[j] = F[j] = 0.0f;
  } else {
    const float invQ = __frcp_rn(Q);
#pragma unroll
    for (int j = 0; j < C; ++j) F[j] = sl.F[j] * invQ;
    if (sl.G > 0.0f) {
      const float invG = __frcp_rn(sl.G);
#pragma unroll
      for (int j = 0; j < C; ++j) H[j] = sl.H[j] * invG;
    } else {
      flat_neighbourhood_mean<C>(a.u_src + static_cast<long long>(p) * a.src_pstride, X, Y, z,
                                 a.nx, a.ny, a.nz, a.pitch, H);
    }
  }
  float u[C], um[C], Jv;
  voxel_update<C>(H, F, sl.xc, cc, k, u, um, Jv);
  const size_t plane = static_cast<size_t>(a.nz) * a.ny * a.pitch;
  float* dst = a.u_dst + static_cast<size_t>(p) * C * plane +
               (static_cast<size_t>(z) * a.ny + Y) * a.pitch + X;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    dst[j * plane] = u[j];
    acc.s0[j] += um[j];
    acc.s1[j] = fmaf(um[j], sl.xc, acc.s1[j]);
    acc.dm = fmaxf(acc.dm, fabsf(u[j] - sl.uc[j]));
  }
  acc.J += Jv;
}

template <int C>
__global__ void __launch_bounds__(NT, 2)
    stencil_kernel(const __grid_constant__ CUtensorMap tm_x,
                   const __grid_constant__ CUtensorMap tm_u, const StencilArgs a) {
  extern __shared__ unsigned char dsmem_raw[];
  __shared__ __align__(8) uint64_t full[NSTAGE];
  __shared__ int s_act[kMaxP];
  __shared__ int s_nact;
  __shared__ float s_red[NT / 32][2 * C + 2];

  unsigned char* dsmem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsmem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int tid = threadIdx.x;
  const int tx = tid & 31, ty = tid >> 5;

  if (tid == 0) {
    int n = 0;
    for (int p = 0; p < a.P; ++p)
      if (a.active[p]) s_act[n++] = p;
    s_nact = n;
    for (int s = 0; s < NSTAGE; ++s) mbar_init(&full[s], 1);
    fence_mbarrier_init();
    prefetch_tensormap(&tm_x);
    prefetch_tensormap(&tm_u);
  }
  __syncthreads();
  const long long n_items = static_cast<long long>(s_nact) * a.n_tiles;
  if (static_cast<long long>(blockIdx.x) >= n_items) return;

  auto xs_of = [&](int s) { return reinterpret_cast<float*>(dsmem + s * stage_bytes<C>()); };
  auto us_of = [&](int s) {
    return reinterpret_cast<float*>(dsmem + s * stage_bytes<C>() + XBYTES);
  };

  // Producer cursor (used by thread 0 only): next plane to issue.
  long long pw = blockIdx.x;
  int pk = 0;
  long long issued = 0;
  auto issue_next = [&]() {
    if (pw >= n_items) return;
    const Item it = decode_item(a, s_act, pw);
    const int s = static_cast<int>(issued % NSTAGE);
    mbar_arrive_expect_tx(&full[s], stage_tx_bytes<C>());
    const int pz = it.pzb + pk;
    tma_load_3d(xs_of(s), &tm_x, &full[s], it.x0 - 4, it.y0 - 1, pz);
    tma_load_4d(us_of(s), &tm_u, &full[s], it.x0 - 4, it.y0 - 1, pz, it.p * a.src_cstride);
    ++issued;
    if (++pk > it.pze - it.pzb) {
      pk = 0;
      pw += gridDim.x;
    }
  };
  if (tid == 0)
    for (int i = 0; i < NSTAGE - 1; ++i) issue_next();

  MethodConsts k;
  k.dist_floor = a.dist_floor;
  k.m = a.m;
  k.inv_m1 = a.inv_m1;
  k.m_is_2 = a.m_is_2;
  const bool z3 = a.nz > 1;
  long long q = 0;   // consumer plane counter
  bool timed_out = false;

  for (long long w = blockIdx.x; w < n_items; w += gridDim.x) {
    const Item it = decode_item(a, s_act, w);
    const int X = it.x0 + tx, Y = it.y0 + ty;
    const bool col_ok = (X < a.nx) && (Y < a.ny);
    const bool edge = (it.x0 == 0) || (it.x0 + TX >= a.nx) || (it.y0 == 0) ||
                      (it.y0 + TY >= a.ny);
    const float mx[3] = {X > 0 ? 1.0f : 0.0f, 1.0f, X < a.nx - 1 ? 1.0f : 0.0f};
    const float my[3] = {Y > 0 ? 1.0f : 0.0f, 1.0f, Y < a.ny - 1 ? 1.0f : 0.0f};
    k.lam = static_cast<float>(a.lam_xi[2 * it.p]);
    k.xi = static_cast<float>(a.lam_xi[2 * it.p + 1]);
    float cc[C];
#pragma unroll
    for (int j = 0; j < C; ++j) cc[j] = static_cast<float>(a.centres[it.p * C + j]);

    Slot<C> lo, mid, hi;
    lo.clear();
    mid.clear();
    hi.clear();
    lo.xc = mid.xc = hi.xc = 0.0f;
#pragma unroll
    for (int j = 0; j < C; ++j) lo.uc[j] = mid.uc[j] = hi.uc[j] = 0.0f;
    Sums<C> acc;
    acc.clear();

    const int np = it.pze - it.pzb + 1;
    for (int kk = 0; kk < np; ++kk, ++q) {
      if (__syncthreads_or(timed_out)) goto abort;
      if (tid == 0) {
        fence_proxy_async_smem();
        issue_next();
      }
      const int s = static_cast<int>(q % NSTAGE);
      if (!mbar_wait_bounded(&full[s], static_cast<uint32_t>((q / NSTAGE) & 1))) {
        timed_out = true;
        continue;
      }
      const int pz = it.pzb + kk;
      const float* xs = xs_of(s);
      const float* us = us_of(s);
      const int coff = (ty + 1) * BX + tx + 4;
      mid.xc = xs[coff];
#pragma unroll
      for (int j = 0; j < C; ++j) mid.uc[j] = us[j * PLANE + coff];
      if (kk + 1 < np) {   // centre above: its x comes from the next plane (already issued)
        const int s1 = static_cast<int>((q + 1) % NSTAGE);
        if (!mbar_wait_bounded(&full[s1], static_cast<uint32_t>(((q + 1) / NSTAGE) & 1))) {
          timed_out = true;
          continue;
        }
        hi.xc = xs_of(s1)[coff];
      } else {
        hi.xc = 0.0f;
      }
      if (z3) {
        if (edge) accumulate_plane<C, true, true>(xs, us, tx, ty, mx, my, lo, mid, hi);
        else accumulate_plane<C, false, true>(xs, us, tx, ty, mx, my, lo, mid, hi);
      } else {
        if (edge) accumulate_plane<C, true, false>(xs, us, tx, ty, mx, my, lo, mid, hi);
        else accumulate_plane<C, false, false>(xs, us, tx, ty, mx, my, lo, mid, hi);
      }
      if (col_ok) {
        if (pz - 1 >= it.z0 && pz - 1 < it.z1)
          finalize_centre<C>(lo, X, Y, pz - 1, a, it.p, cc, k, acc);
        if (pz == a.nz - 1 && pz >= it.z0 && pz < it.z1)
          finalize_centre<C>(mid, X, Y, pz, a, it.p, cc, k, acc);
      }
      lo = mid;
      mid = hi;
      hi.clear();
    }

    // Item partial sums: FP32 within a thread and a warp, FP64 across warps.
    {
      const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const float v0 = warp_sum(acc.s0[j]);
        const float v1 = warp_sum(acc.s1[j]);
        if (lane == 0) {
          s_red[warp][j] = v0;
          s_red[warp][C + j] = v1;
        }
      }
      const float vj = warp_sum(acc.J);
      const float vm = warp_max(acc.dm);
      if (lane == 0) {
        s_red[warp][2 * C] = vj;
        s_red[warp][2 * C + 1] = vm;
      }
      __syncthreads();
      const size_t rec = static_cast<size_t>(it.p) * a.n_tiles + it.tile;
      if (tid < 2 * C + 1) {
        double sum = 0.0;
#pragma unroll
        for (int wv = 0; wv < NT / 32; ++wv) sum += static_cast<double>(s_red[wv][tid]);
        a.partials[rec * (2 * C + 1) + tid] = sum;
      } else if (tid == 2 * C + 1) {
        float mm = 0.0f;
#pragma unroll
        for (int wv = 0; wv < NT / 32; ++wv) mm = fmaxf(mm, s_red[wv][2 * C + 1]);
        a.dmax[rec] = mm;
      }
    }
  }
  return;

abort:
  // A bounded wait ran out: record it, give the copies already issued a
  // bounded chance to land, and leave.
  if (tid == 0) {
    set_status(a.status, IFCM_ERR_TIMEOUT, 1);
    for (long long r = q; r < issued; ++r)
      (void)mbar_wait_bounded(&full[r % NSTAGE], static_cast<uint32_t>((r / NSTAGE) & 1), 1u << 16);
  }
}

template <int C>
cudaError_t launch_c(const CUtensorMap& tm_x, const CUtensorMap& tm_u, const StencilArgs& a,
                     int grid, cudaStream_t s) {
  const int smem = NSTAGE * stage_bytes<C>() + 128;
  static bool configured = false;   // per process; attribute is per function
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(stencil_kernel<C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  stencil_kernel<C><<<grid, NT, smem, s>>>(tm_x, tm_u, a);
  return cudaGetLastError();
}

template <int C>
int blocks_per_sm_c() {
  const int smem = NSTAGE * stage_bytes<C>() + 128;
  cudaFuncSetAttribute(stencil_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stencil_kernel<C>, NT, smem) !=
      cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

}  // namespace

size_t stencil_smem_bytes(int c) {
  switch (c) {
    case 2: return NSTAGE * stage_bytes<2>() + 128;
    case 3: return NSTAGE * stage_bytes<3>() + 128;
    case 4: return NSTAGE * stage_bytes<4>() + 128;
    case 5: return NSTAGE * stage_bytes<5>() + 128;
    case 6: return NSTAGE * stage_bytes<6>() + 128;
    case 7: return NSTAGE * stage_bytes<7>() + 128;
    default: return NSTAGE * stage_bytes<8>() + 128;
  }
}

int stencil_blocks_per_sm(int c) {
  switch (c) {
    case 2: return blocks_per_sm_c<2>();
    case 3: return blocks_per_sm_c<3>();
    case 4: return blocks_per_sm_c<4>();
    case 5: return blocks_per_sm_c<5>();
    case 6: return blocks_per_sm_c<6>();
    case 7: return blocks_per_sm_c<7>();
    default: return blocks_per_sm_c<8>();
  }
}

cudaError_t launch_stencil(int c, const CUtensorMap& tm_x, const CUtensorMap& tm_u,
                           const StencilArgs& a, int grid, cudaStream_t s) {
  switch (c) {
    case 2: return launch_c<2>(tm_x, tm_u, a, grid, s);
    case 3: return launch_c<3>(tm_x, tm_u, a, grid, s);
    case 4: return launch_c<4>(tm_x, tm_u, a, grid, s);
    case 5: return launch_c<5>(tm_x, tm_u, a, grid, s);
    case 6: return launch_c<6>(tm_x, tm_u, a, grid, s);
    case 7: return launch_c<7>(tm_x, tm_u, a, grid, s);
    case 8: return launch_c<8>(tm_x, tm_u, a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pifcm
