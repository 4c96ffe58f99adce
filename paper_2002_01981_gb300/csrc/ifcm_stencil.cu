// Batched IFCM iteration: the neighbourhood stencil of Eqs 5-9 fused with the
// distance (Eq 4), membership (Eq 2), objective (Eq 1) and centre sums (Eq 3),
// for every active particle of a batch, in one persistent launch.
//
// Work item = (group of NP particles, TX x TY column tile, z-chunk of tz
// planes).  Warp 8 of each CTA is the producer: one lane walks the CTA's items
// plane by plane and, for each plane, issues TMA tile loads of the normalised
// volume x and of the c membership planes U^t of each particle of the group
// (one-voxel halo in y, aligned four-voxel margins in x) into a ring of
// shared-memory stages, gated by "full" (transaction bytes) and "empty"
// (one arrival per consumer warp) mbarriers.  Warps 0-7 are consumers: thread
// (tx, ty) owns column (x0 + tx, y0 + ty) and keeps three centres of the column
// in registers.  The plane being consumed contributes to the centre below it
// (dz = +1), its own centre (dz = 0) and the centre above (dz = -1); the three
// register sets rotate roles from plane to plane (the loop is unrolled by
// three), so nothing is copied.  A plane's stage is released only after the
// next plane has been consumed, because the centre it holds is finalised then:
// H = sum u g / sum g, F = sum u^2 q^2 / sum q^2 (q^2 = dx^2+dy^2+dz^2,
// reading R1), Eqs 4 and 2, U^{t+1} written from registers, and the centre's
// shares of sum u^m, sum u^m x, J and max|du|.
//
// Neighbours outside the volume are excluded (reading R4) without masks:
// the volume's tensor map fills positions outside the volume with NaN and
// g = max(|x_i - x_k|, 0) turns them into 0 (max ignores a NaN operand),
// while the membership tensor maps fill them with 0.  Out-of-range planes are
// never loaded.  The NP particles of a group share the x tile, every g_ik and
// sum_k g_ik.  Per item and particle, the sums go to a partial record (FP32
// within a thread and a warp, FP64 across warps) that the reduce kernel sums
// per particle in FP64.
#include "ifcm_math.cuh"
#include "launch.h"

namespace pifcm {

namespace {

constexpr int TX = kTX, TY = kTY;
constexpr int NCW = 8;                 // consumer warps
constexpr int NCT = NCW * 32;          // consumer threads (one per column of the tile)
constexpr int NT = NCT + 32;           // + one producer warp
constexpr int BX = TX + 8;             // x box: 4-voxel aligned margins (TMA x must be 16-B aligned)
constexpr int BY = TY + 2;             // y box: one-voxel halo
constexpr int PLANE = BX * BY;         // floats in one channel of a stage
#ifndef PIFCM_STENCIL_STAGES
#define PIFCM_STENCIL_STAGES 5
#endif
constexpr int NSTAGE = PIFCM_STENCIL_STAGES;   // ring depth (>= 4: prev, current, next + 1 in flight)
static_assert(NSTAGE >= 4, "the consumers hold three stages at a time");
constexpr int XBYTES = ((PLANE * 4 + 127) / 128) * 128;
constexpr int CBAR = 1;                // named barrier id of the consumer warps

// Build-time tuning: CTAs per SM the register budget targets, and particles
// per work item for c <= 4 (c > 4 always uses one).
#ifndef PIFCM_STENCIL_MIN_BLOCKS
#define PIFCM_STENCIL_MIN_BLOCKS 1
#endif
#ifndef PIFCM_STENCIL_NP_SMALL_C
#define PIFCM_STENCIL_NP_SMALL_C 2
#endif

// One particle's c membership planes in a stage, padded so that every TMA
// destination starts on a 128-byte boundary.
template <int C>
__host__ __device__ constexpr int ubytes() {
  return ((C * PLANE * 4 + 127) / 128) * 128;
}
template <int C>
__host__ __device__ constexpr int ufloats() {
  return ubytes<C>() / 4;
}
template <int C, int NP>
__host__ __device__ constexpr int stage_bytes() {
  return XBYTES + NP * ubytes<C>();
}
static_assert(XBYTES % 128 == 0 && ubytes<3>() % 128 == 0 && ubytes<5>() % 128 == 0 &&
                  ubytes<7>() % 128 == 0,
              "TMA shared-memory destinations must start on 128-byte boundaries");
template <int C, int NP>
__host__ __device__ constexpr uint32_t stage_tx_bytes() {
  return static_cast<uint32_t>((1 + NP * C) * PLANE * 4);
}
template <int C, int NP>
__host__ __device__ constexpr int smem_total() {
  return NSTAGE * stage_bytes<C, NP>() + 128;
}

__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync %0, %1;" ::"n"(CBAR), "n"(NCT) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// g = |a - b|, and 0 when b is the NaN that marks a position outside the volume.
__device__ __forceinline__ float gdist(float a, float b) {
  float r;
  asm("max.f32 %0, %1, 0f00000000;" : "=f"(r) : "f"(fabsf(a - b)));
  return r;
}

struct Item {
  int p0, p1;          // particles of the group (p1 = p0 when the group has one)
  bool two;            // p1 is a distinct particle
  int tile, x0, y0, z0, z1, pzb, pze;
};

template <int NP>
__device__ __forceinline__ Item decode_item(const StencilArgs& a, const int* act, int nact,
                                            int w) {
  Item it;
  const int g = w / a.n_tiles;
  it.tile = w - g * a.n_tiles;
  it.p0 = act[g * NP];
  it.two = (NP == 2) && (g * NP + 1 < nact);
  it.p1 = it.two ? act[g * NP + 1] : it.p0;
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

// Accumulators of one centre voxel of the column, for NP particles.
template <int C, int NP>
struct Slot {
  float G;            // sum_k g_ik (shared by the particles)
  float H[NP][C];     // sum_k u_kj g_ik
  float F[NP][C];     // sum_k u_kj^2 q^2_ik
  __device__ __forceinline__ void clear() {
    G = 0.0f;
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
      for (int j = 0; j < C; ++j) H[p][j] = F[p][j] = 0.0f;
  }
};

template <int C, int NP>
struct Sums {
  float s0[NP][C], s1[NP][C], J[NP], dm[NP];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
      for (int j = 0; j < C; ++j) s0[p][j] = s1[p][j] = 0.0f;
      J[p] = dm[p] = 0.0f;
    }
  }
};

// Contributions of one plane (x in xs, memberships of particle p at us + p *
// ufloats<C>()) to the centres below (lo), in (mid) and above (hi) it.
template <int C, int NP, bool Z3>
__device__ __forceinline__ void accumulate_plane(const float* __restrict__ xs,
                                                 const float* __restrict__ us, int cidx,
                                                 float x_lo, float x_mid, float x_hi,
                                                 Slot<C, NP>& lo, Slot<C, NP>& mid,
                                                 Slot<C, NP>& hi) {
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int off = cidx + dy * BX + dx;
      const float xk = xs[off];
      const bool self = (dx == 0 && dy == 0);
      const int q2 = dx * dx + dy * dy;          // folded after unrolling
      const float qm = static_cast<float>(q2);    // weight in the same plane
      const float qa = static_cast<float>(q2 + 1);  // weight in the planes above / below
      float gl = 0.0f, gh = 0.0f, gm = 0.0f;
      if (Z3) {
        gl = gdist(x_lo, xk);
        gh = gdist(x_hi, xk);
        lo.G += gl;
        hi.G += gh;
      }
      if (!self) {
        gm = gdist(x_mid, xk);
        mid.G += gm;
      }
#pragma unroll
      for (int p = 0; p < NP; ++p) {
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const float uk = us[p * ufloats<C>() + j * PLANE + off];
          const float wk = uk * uk;
          if (Z3) {
            lo.H[p][j] = fmaf(uk, gl, lo.H[p][j]);
            hi.H[p][j] = fmaf(uk, gh, hi.H[p][j]);
            lo.F[p][j] = fmaf(qa, wk, lo.F[p][j]);
            hi.F[p][j] = fmaf(qa, wk, hi.F[p][j]);
          }
          if (!self) {
            mid.H[p][j] = fmaf(uk, gm, mid.H[p][j]);
            mid.F[p][j] = fmaf(qm, wk, mid.F[p][j]);
          }
        }
      }
    }
  }
}

// Per-item constants of one consumer thread.
template <int C, int NP>
struct Ctx {
  int X, Y;
  bool col_ok, col_interior;
  int col_off;                 // Y * pitch + X
  float lam[NP], xi[NP], cc[NP][C];
  float* dst[NP];              // particle's U^{t+1} base
};

// Finalise one centre (its u^t is read from its plane's stage at cus).
template <int C, int NP>
__device__ __forceinline__ void finalize_centre(const Slot<C, NP>& sl, const float* cus,
                                                int cidx, float xc, int z, bool interior,
                                                const StencilArgs& a, const Item& it,
                                                const Ctx<C, NP>& cx, const MethodConsts& k,
                                                Sums<C, NP>& acc) {
  float invQ;
  int cnt = 1;
  if (interior) {
    invQ = a.nz > 1 ? (1.0f / 54.0f) : (1.0f / 12.0f);
  } else {
    float Q;
    box_counts(cx.X, cx.Y, z, a.nx, a.ny, a.nz, cnt, Q);
    invQ = cnt > 0 ? __frcp_rn(Q) : 0.0f;
  }
  const bool normal_g = sl.G >= 1.0e-30f;
  const float invG = normal_g ? fast_rcp(sl.G) : 0.0f;
  const int plane = a.nz * a.ny * a.pitch;              // < 2^31 / c (host-checked)
  const int voff = z * (a.ny * a.pitch) + cx.col_off;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    if (p == 1 && !it.two) break;
    float H[C], F[C];
    if (cnt == 0) {
#pragma unroll
      for (int j = 0; j < C; ++j) H[j] = F[j] = 0.0f;
    } else {
#pragma unroll
      for (int j = 0; j < C; ++j) F[j] = sl.F[p][j] * invQ;
      if (normal_g) {
#pragma unroll
        for (int j = 0; j < C; ++j) H[j] = sl.H[p][j] * invG;
      } else if (sl.G > 0.0f) {
        const float r = __frcp_rn(sl.G);
#pragma unroll
        for (int j = 0; j < C; ++j) H[j] = sl.H[p][j] * r;
      } else {
        const int pid = p == 0 ? it.p0 : it.p1;
        flat_neighbourhood_mean<C>(a.u_src + static_cast<long long>(pid) * a.src_pstride, cx.X,
                                   cx.Y, z, a.nx, a.ny, a.nz, a.pitch, H);
      }
    }
    MethodConsts kp = k;
    kp.lam = cx.lam[p];
    kp.xi = cx.xi[p];
    float u[C], um[C], Jv;
    voxel_update_fast<C>(H, F, xc, cx.cc[p], kp, u, um, Jv);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      cx.dst[p][j * plane + voff] = u[j];
      acc.s0[p][j] += um[j];
      acc.s1[p][j] = fmaf(um[j], xc, acc.s1[p][j]);
      acc.dm[p] = fmaxf(acc.dm[p], fabsf(u[j] - cus[p * ufloats<C>() + j * PLANE + cidx]));
    }
    acc.J[p] += Jv;
  }
}

template <int C, int NP>
__global__ void __launch_bounds__(NT, PIFCM_STENCIL_MIN_BLOCKS)
    stencil_kernel(const __grid_constant__ CUtensorMap tm_x,
                   const __grid_constant__ CUtensorMap tm_u, const StencilArgs a) {
  extern __shared__ unsigned char dsmem_raw[];
  __shared__ __align__(8) uint64_t full[NSTAGE];
  __shared__ __align__(8) uint64_t empty[NSTAGE];
  __shared__ int s_act[kMaxP];
  __shared__ int s_nact;
  __shared__ int s_abort;
  __shared__ float s_red[NCW][NP * (2 * C + 2)];

  unsigned char* dsmem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsmem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    int n = 0;
    for (int p = 0; p < a.P; ++p)
      if (a.active[p]) s_act[n++] = p;
    s_nact = n;
    s_abort = 0;
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    fence_mbarrier_init();
  }
  __syncthreads();
  const int nact = s_nact;
  const int groups = (nact + NP - 1) / NP;
  const int n_items = groups * a.n_tiles;
  if (static_cast<int>(blockIdx.x) >= n_items) return;

  auto xs_of = [&](int s) { return reinterpret_cast<float*>(dsmem + s * stage_bytes<C, NP>()); };
  auto us_of = [&](int s) {
    return reinterpret_cast<float*>(dsmem + s * stage_bytes<C, NP>() + XBYTES);
  };

  // ------------------------------------------------------------ producer
  if (warp == NCW) {
    if (lane == 0) {
      prefetch_tensormap(&tm_x);
      prefetch_tensormap(&tm_u);
      int q = 0;
      for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
        const Item it = decode_item<NP>(a, s_act, nact, w);
        for (int pz = it.pzb; pz <= it.pze; ++pz, ++q) {
          const int s = q % NSTAGE;
          if (q >= NSTAGE &&
              !mbar_wait_bounded(&empty[s], static_cast<uint32_t>(((q / NSTAGE) - 1) & 1))) {
            atomicExch(&s_abort, 1);
            set_status(a.status, IFCM_ERR_TIMEOUT, 3);
            return;
          }
          if (*reinterpret_cast<volatile int*>(&s_abort)) return;
          mbar_arrive_expect_tx(&full[s], stage_tx_bytes<C, NP>());
          tma_load_3d(xs_of(s), &tm_x, &full[s], it.x0 - 4, it.y0 - 1, pz);
          tma_load_4d(us_of(s), &tm_u, &full[s], it.x0 - 4, it.y0 - 1, pz,
                      it.p0 * a.src_cstride);
          if (NP == 2)
            tma_load_4d(us_of(s) + ufloats<C>(), &tm_u, &full[s], it.x0 - 4, it.y0 - 1, pz,
                        it.p1 * a.src_cstride);
        }
      }
    }
    return;
  }

  // ------------------------------------------------------------ consumers
  const int tx = tid & 31, ty = tid >> 5;
  const int cidx = (ty + 1) * BX + tx + 4;     // the column's position in a stage plane
  MethodConsts k;
  k.dist_floor = a.dist_floor;
  k.m = a.m;
  k.inv_m1 = a.inv_m1;
  k.m_is_2 = a.m_is_2;
  const bool z3 = a.nz > 1;
  const int plane = a.nz * a.ny * a.pitch;
  int q = 0;

  // Waits for plane qq's stage (bounded; after a timeout every wait is skipped
  // so that all consumer threads still reach the same barriers).
  auto wait_full = [&](int qq) -> bool {
    if (*reinterpret_cast<volatile int*>(&s_abort)) return false;
    if (!mbar_wait_bounded(&full[qq % NSTAGE], static_cast<uint32_t>((qq / NSTAGE) & 1))) {
      atomicExch(&s_abort, 1);
      set_status(a.status, IFCM_ERR_TIMEOUT, 4);
      return false;
    }
    return true;
  };
  auto release = [&](int qq) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[qq % NSTAGE]);
  };

  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const Item it = decode_item<NP>(a, s_act, nact, w);
    Ctx<C, NP> cx;
    cx.X = it.x0 + tx;
    cx.Y = it.y0 + ty;
    cx.col_ok = (cx.X < a.nx) && (cx.Y < a.ny);
    cx.col_interior = cx.X > 0 && cx.X < a.nx - 1 && cx.Y > 0 && cx.Y < a.ny - 1;
    cx.col_off = cx.Y * a.pitch + cx.X;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int pid = p == 0 ? it.p0 : it.p1;
      cx.lam[p] = static_cast<float>(a.lam_xi[2 * pid]);
      cx.xi[p] = static_cast<float>(a.lam_xi[2 * pid + 1]);
#pragma unroll
      for (int j = 0; j < C; ++j) cx.cc[p][j] = static_cast<float>(a.centres[pid * C + j]);
      cx.dst[p] = a.u_dst + static_cast<size_t>(pid) * C * plane;
    }
    Slot<C, NP> s0, s1, s2;
    s0.clear();
    s1.clear();
    s2.clear();
    Sums<C, NP> acc;
    acc.clear();
    const int np = it.pze - it.pzb + 1;
    const int q0 = q;

    // One plane step with roles (lo, mid, hi).
    auto step = [&](int kk, Slot<C, NP>& lo, Slot<C, NP>& mid, Slot<C, NP>& hi) {
      const int qq = q0 + kk;
      const int pz = it.pzb + kk;
      const bool has_next = kk + 1 < np;
      const bool ok = wait_full(qq) && (!has_next || wait_full(qq + 1));
      if (ok) {
        const float* xs = xs_of(qq % NSTAGE);
        const float* us = us_of(qq % NSTAGE);
        const float x_mid = xs[cidx];
        const float x_lo = kk > 0 ? xs_of((qq + NSTAGE - 1) % NSTAGE)[cidx] : 0.0f;
        const float x_hi = has_next ? xs_of((qq + 1) % NSTAGE)[cidx] : 0.0f;
        if (z3)
          accumulate_plane<C, NP, true>(xs, us, cidx, x_lo, x_mid, x_hi, lo, mid, hi);
        else
          accumulate_plane<C, NP, false>(xs, us, cidx, x_lo, x_mid, x_hi, lo, mid, hi);
        if (cx.col_ok) {
          if (pz - 1 >= it.z0 && pz - 1 < it.z1)   // the centre below is complete
            finalize_centre<C, NP>(lo, us_of((qq + NSTAGE - 1) % NSTAGE), cidx, x_lo, pz - 1,
                                   cx.col_interior && pz - 1 > 0 && pz - 1 < a.nz - 1, a, it,
                                   cx, k, acc);
          if (pz == a.nz - 1 && pz >= it.z0 && pz < it.z1)   // last plane of the volume
            finalize_centre<C, NP>(mid, us, cidx, x_mid, pz, cx.col_interior && !z3, a, it,
                                   cx, k, acc);
        }
      }
      if (kk > 0) release(qq - 1);         // the plane below is no longer needed
      if (kk + 1 == np) release(qq);       // last plane of the item
      lo.clear();                          // becomes the next step's "hi"
    };

    for (int kk = 0; kk < np; kk += 3) {
      step(kk, s0, s1, s2);
      if (kk + 1 < np) step(kk + 1, s1, s2, s0);
      if (kk + 2 < np) step(kk + 2, s2, s0, s1);
    }
    q = q0 + np;

    // Item partial sums: FP32 within a thread and a warp, FP64 across warps.
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const float v0 = warp_sum(acc.s0[p][j]);
        const float v1 = warp_sum(acc.s1[p][j]);
        if (lane == 0) {
          s_red[warp][p * (2 * C + 2) + j] = v0;
          s_red[warp][p * (2 * C + 2) + C + j] = v1;
        }
      }
      const float vj = warp_sum(acc.J[p]);
      const float vm = warp_max(acc.dm[p]);
      if (lane == 0) {
        s_red[warp][p * (2 * C + 2) + 2 * C] = vj;
        s_red[warp][p * (2 * C + 2) + 2 * C + 1] = vm;
      }
    }
    consumer_sync();
    if (tid < NP * (2 * C + 2)) {
      const int p = tid / (2 * C + 2), v = tid - p * (2 * C + 2);
      if (p == 0 || it.two) {
        const int pid = p == 0 ? it.p0 : it.p1;
        const size_t rec = static_cast<size_t>(pid) * a.n_tiles + it.tile;
        if (v < 2 * C + 1) {
          double sum = 0.0;
#pragma unroll
          for (int wv = 0; wv < NCW; ++wv) sum += static_cast<double>(s_red[wv][tid]);
          a.partials[rec * (2 * C + 1) + v] = sum;
        } else {
          float mm = 0.0f;
#pragma unroll
          for (int wv = 0; wv < NCW; ++wv) mm = fmaxf(mm, s_red[wv][tid]);
          a.dmax[rec] = mm;
        }
      }
    }
    consumer_sync();
  }
}

template <int C, int NP>
cudaError_t launch_c(const CUtensorMap& tm_x, const CUtensorMap& tm_u, const StencilArgs& a,
                     int grid, cudaStream_t s) {
  constexpr int smem = smem_total<C, NP>();
  cudaError_t e = cudaFuncSetAttribute(stencil_kernel<C, NP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  stencil_kernel<C, NP><<<grid, NT, smem, s>>>(tm_x, tm_u, a);
  return cudaGetLastError();
}

template <int C, int NP>
int blocks_per_sm_c() {
  constexpr int smem = smem_total<C, NP>();
  cudaFuncSetAttribute(stencil_kernel<C, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       smem);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stencil_kernel<C, NP>, NT, smem) !=
      cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

// Particles per item: PIFCM_STENCIL_NP_SMALL_C for c <= 4, one above.
template <int C>
constexpr int np_for() {
  return C <= 4 ? PIFCM_STENCIL_NP_SMALL_C : 1;
}

}  // namespace

int stencil_particles_per_item(int c) { return c <= 4 ? PIFCM_STENCIL_NP_SMALL_C : 1; }

size_t stencil_smem_bytes(int c) {
  switch (c) {
    case 2: return smem_total<2, np_for<2>()>();
    case 3: return smem_total<3, np_for<3>()>();
    case 4: return smem_total<4, np_for<4>()>();
    case 5: return smem_total<5, np_for<5>()>();
    case 6: return smem_total<6, np_for<6>()>();
    case 7: return smem_total<7, np_for<7>()>();
    default: return smem_total<8, np_for<8>()>();
  }
}

int stencil_blocks_per_sm(int c) {
  switch (c) {
    case 2: return blocks_per_sm_c<2, np_for<2>()>();
    case 3: return blocks_per_sm_c<3, np_for<3>()>();
    case 4: return blocks_per_sm_c<4, np_for<4>()>();
    case 5: return blocks_per_sm_c<5, np_for<5>()>();
    case 6: return blocks_per_sm_c<6, np_for<6>()>();
    case 7: return blocks_per_sm_c<7, np_for<7>()>();
    default: return blocks_per_sm_c<8, np_for<8>()>();
  }
}

cudaError_t launch_stencil(int c, const CUtensorMap& tm_x, const CUtensorMap& tm_u,
                           const StencilArgs& a, int grid, cudaStream_t s) {
  switch (c) {
    case 2: return launch_c<2, np_for<2>()>(tm_x, tm_u, a, grid, s);
    case 3: return launch_c<3, np_for<3>()>(tm_x, tm_u, a, grid, s);
    case 4: return launch_c<4, np_for<4>()>(tm_x, tm_u, a, grid, s);
    case 5: return launch_c<5, np_for<5>()>(tm_x, tm_u, a, grid, s);
    case 6: return launch_c<6, np_for<6>()>(tm_x, tm_u, a, grid, s);
    case 7: return launch_c<7, np_for<7>()>(tm_x, tm_u, a, grid, s);
    case 8: return launch_c<8, np_for<8>()>(tm_x, tm_u, a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pifcm
