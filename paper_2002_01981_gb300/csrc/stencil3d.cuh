// Batched IFCM iteration over 3D volumes, FP32 memberships in float2 pair
// words, m = 2: the neighbourhood stencil of Eqs 5-9 fused with Eq 4
// (distance), Eq 2 (membership), Eq 1 (objective) and the centre sums of Eq 3.
// This is the form of the batched fitness evaluation (Algorithm 1 step 4) that
// carries almost all of a run's time.  A pair word holds cluster j of the
// item's two particles (NP = 2, c <= 5) or clusters 2k, 2k+1 of its one
// particle (NP = 1, any c).  Every other case (2D images, m != 2, planar or
// bf16 memberships, the first iteration from a caller's start) runs
// stencil_kernel (stencil_kernel.cuh).
//
// Work decomposition, ring and producer are those of stencil_kernel: items of
// (pair-word unit, 32 x TY column tile, z-chunk), a TMA producer warp
// feeding an 8-stage ring of planes, one consumer thread per column marching
// up z.  What differs is the consumer's plane step, written for the fewest
// instructions per update:
//
// - G_i = sum_k g_ik does not change between iterations (x is fixed), so it is
//   computed once per volume (gsum_kernel, in FP64) and stored as s_i = 1/G_i.
// - Neighbours outside the volume need no mask or max: the volume's tensor
//   map fills them with x = 0 and the membership maps with u = 0, so their
//   products u_kj g_ik vanish (reading R4), and G excludes them.  g_ik =
//   |x_i - x_k| costs one FADD, the absolute value being an operand modifier
//   of the packed FMA that uses it.
// - A flat neighbourhood (G_i = 0, reading R3) is stored as s_i = -1/(n_i g0)
//   with n_i its in-volume neighbours, and its centre value in the g_ik is
//   x_i + 2: every in-volume neighbour then has the same weight g0 = |(x_i +
//   2) - x_i|, which turns H into the plain mean, with no branch.
// - Memberships of one voxel sum to one (Eq 2), so sum_j H_ij = 1 and the last
//   cluster's H is 1 - sum_{j<c-1} H_ij: its 26 neighbour products are not
//   formed, wherever that saves a whole pair word (NP = 2, or NP = 1 with c
//   odd, whose last word holds cluster c - 1 and a padding lane).  U^t always
//   comes from Eq 2 here (iteration 0, which reads the caller's start, runs
//   stencil_kernel).
// - F needs no per-centre accumulation across planes beyond one float2 per
//   pair word: each plane's window sums W0 (centre), S1 (faces), S2 (corners) of
//   u^2 give A = W0 + 2 S1 + 3 S2 (weight 1 + dx^2 + dy^2, to the centres
//   above and below) and V = S1 + 2 S2 (weight dx^2 + dy^2, to the centre in
//   the plane).
// - No warp votes or branches in the plane step: out-of-volume lanes of an
//   overhanging tile compute on (on x = 0) but their stores are
//   predicated off and their sums are zeroed once per item; the z-face
//   centres differ only in 1/Q, a step argument.
// - The four centre slots change roles, not values: the steady-state loop is
//   unrolled four planes deep (slot roles rotate statically), with a short
//   generic step (slot values rotated) for the first and last planes of an
//   item.
// - Shared-memory reads are plain LDS with immediate offsets from one base
//   per stage (the stage pointers keep the shared address space).
#pragma once

#include "stencil_kernel.cuh"

namespace pifcm {

namespace {

constexpr int SBYTES = ((TX * TY * 4 + 127) / 128) * 128;   // 1/G of the tile's centres

// Pair words per voxel (K), H sums kept (KH), and whether the last cluster's H
// is taken by complement (COMPL) and the last word's high lane is padding (PAD).
// With bf16 words the memberships of a voxel sum to one only up to their
// rounding, so no cluster's H is taken by complement there.
template <int C, int NP, int UL>
struct S3 {
  static constexpr int K = Pairs<C, NP>::K;
  static constexpr bool PAD = NP == 1 && (C & 1);
  static constexpr bool COMPL = UL == UL_F32P && (NP == 2 || PAD);
  static constexpr int KH = COMPL ? K - 1 : K;
};

// A pair word in a stage: float2, or a bf16 pair unpacked exactly.
template <int UL>
struct Word3 {
  using T = float2;
  static __device__ __forceinline__ float2 get(const T* p, int i) { return p[i]; }
};
template <>
struct Word3<UL_BF16> {
  using T = uint32_t;
  static __device__ __forceinline__ float2 get(const T* p, int i) { return unpack_bf16x2(p[i]); }
};

template <int C, int NP, int UL>
__host__ __device__ constexpr int s3_stage_bytes() {
  return XBYTES + SBYTES + ublock_bytes<C, NP, UL>();
}
template <int C, int NP, int UL>
__host__ __device__ constexpr uint32_t s3_tx_bytes() {
  return static_cast<uint32_t>(PLANE * 4 + TX * TY * 4 +
                               S3<C, NP, UL>::K * PLANE * word_bytes(UL));
}
template <int C, int NP, int UL>
__host__ __device__ constexpr int s3_smem_total() {
  return NSTAGE * s3_stage_bytes<C, NP, UL>() + 128;
}
static_assert(NSTAGE == 8, "stage indices are taken modulo 8 with a mask");
static_assert(SBYTES % 128 == 0, "TMA destinations start on 128-byte boundaries");
// every shared-memory read of a column stays inside its stage plane: the
// column's centre (ty + 1) BX + tx + 4 plus neighbour offsets of -BX - 1 ...
// BX + 1, for tx < TX and ty < TY
static_assert(BX + 4 - BX - 1 >= 0 && TY * BX + TX - 1 + 4 + BX + 1 < PLANE,
              "stencil reads stay inside the stage plane");

// One centre of the column: its sums over the planes read so far, one float2
// per pair word.
template <int C, int NP, int UL>
struct Slot3 {
  static constexpr int K = S3<C, NP, UL>::K, KH = S3<C, NP, UL>::KH;
  float2 H[KH];                      // sum_k u_kj g_ik (the last cluster's by complement)
  float2 F[K];                       // sum_k u_kj^2 q^2_ik
  float x;                           // x_i
  float s;                           // 1/G_i, or -1/(n_i g0) for a flat neighbourhood
  float xg;                          // x_i in g_ik: x_i, or x_i + 2 for a flat neighbourhood
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int q = 0; q < KH; ++q) H[q] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < K; ++q) F[q] = make_float2(0.0f, 0.0f);
    x = s = xg = 0.0f;
  }
};

// Constants of an item, paired like the sums.
template <int C, int NP, int UL>
struct Fin3 {
  float2 ncc[S3<C, NP, UL>::K];          // -c_j, paired like the sums (0 in a padding lane)
  float2 nlam;                       // -lambda of the lanes' particles
  float2 one_nlam;                   // 1 - lambda
  float floor;                       // dist_floor
};

// A thread's shares of the item's sums; with one particle, J and max|du| are
// in the low lane.
template <int C, int NP, int UL>
struct Acc3 {
  static constexpr int K = S3<C, NP, UL>::K;
  float2 s0[K], s1[K];               // sum u^m, sum u^m x
  float2 J, dm;                      // J, max|du|
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int q = 0; q < K; ++q) s0[q] = s1[q] = make_float2(0.0f, 0.0f);
    J = dm = make_float2(0.0f, 0.0f);
  }
};

// Finalise centre d: Eqs 5 and 7 folded into the factor of Eq 4 (1/G from s,
// -xi/Q given as nx, the last cluster's H by complement), Eq 4 with reading R2,
// Eq 2 for m = 2, the U^{t+1} store and the centre's shares of Eqs 1 and 3
// and of max|du|.  ud: the centre's U^t in its stage (pair words at its
// column); dst: its U^{t+1} word of pair 0.  With bf16 words U^{t+1} is
// rounded to nearest even when stored and max|du| compares stored values;
// Eqs 1 and 3 take the FP32 u' that was rounded.  MASK: the centre's shares
// are weighed by keep (1, or 0 for a lane outside the image).
template <int C, int NP, int UL, bool MASK = false>
__device__ __forceinline__ void fin3(const Slot3<C, NP, UL>& d,
                                     const typename Word3<UL>::T* __restrict__ ud, float2 nx,
                                     const Fin3<C, NP, UL>& fc, Acc3<C, NP, UL>& acc,
                                     typename Word3<UL>::T* __restrict__ dst, int plane, bool st,
                                     float keep = 1.0f) {
  constexpr int K = S3<C, NP, UL>::K, KH = S3<C, NP, UL>::KH;
  const float ig = fabsf(d.s);
  // f_j = 1 - lambda H_j - xi F_j with H_j = Hs_j / G and F_j = Fs_j / Q,
  // taking -lambda / G and -xi / Q once per centre
  const float2 nl = __fmul2_rn(fc.nlam, dup2(ig));
  float2 fq[K];
#pragma unroll
  for (int q = 0; q < KH; ++q) fq[q] = __ffma2_rn(nx, d.F[q], __ffma2_rn(nl, d.H[q], dup2(1.0f)));
  if (S3<C, NP, UL>::COMPL) {
    // the last cluster: 1 - lambda (1 - sum_{j<c-1} H_j) - xi F, with the
    // other clusters' sums of its particle (per lane for NP = 2; both lanes
    // of every other word for NP = 1, whose last word's high lane is padding)
    float2 hs = d.H[0];
#pragma unroll
    for (int q = 1; q < KH; ++q) hs = __fadd2_rn(hs, d.H[q]);
    if (NP == 1) hs = dup2(hs.x + hs.y);
    fq[K - 1] = __ffma2_rn(nx, d.F[K - 1], __ffma2_rn(__fmul2_rn(nl, dup2(-1.0f)), hs,
                                                      fc.one_nlam));
  }
  // Eq 4 (reading R2): max(D max(f, 0), floor) = max(D f, floor) for D >= 0
  float2 r[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const float2 dd = __fadd2_rn(dup2(d.x), fc.ncc[q]);
    const float2 d2 = max2(__fmul2_rn(__fmul2_rn(dd, dd), fq[q]), fc.floor);
    r[q] = make_float2(fast_rcp(d2.x), fast_rcp(d2.y));
  }
  if (S3<C, NP, UL>::PAD) r[K - 1].y = 0.0f;     // the padding lane is no cluster
  // Eq 2 with m = 2: u_j = (1/d2_j) / S, S = sum_k 1/d2_k; Eq 1 share = 1/S
  float2 S = r[0];
#pragma unroll
  for (int q = 1; q < K; ++q) S = __fadd2_rn(S, r[q]);
  float2 inv;
  if (NP == 2) {
    inv = make_float2(fast_rcp(S.x), fast_rcp(S.y));
    acc.J = MASK ? __ffma2_rn(inv, dup2(keep), acc.J) : __fadd2_rn(acc.J, inv);
  } else {
    inv = dup2(fast_rcp(S.x + S.y));
    acc.J.x = MASK ? fmaf(inv.x, keep, acc.J.x) : acc.J.x + inv.x;
  }
  const float2 x2 = dup2(d.x);
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const float2 u = __fmul2_rn(r[q], inv);
    const float2 um = MASK ? __fmul2_rn(__fmul2_rn(u, u), dup2(keep)) : __fmul2_rn(u, u);
    acc.s0[q] = __fadd2_rn(acc.s0[q], um);
    acc.s1[q] = __ffma2_rn(um, x2, acc.s1[q]);
    float2 e;                                                      // u' - u
    if constexpr (UL == UL_BF16) {
      const uint32_t w = pack_bf16x2(u);
      if (st) __stcg(reinterpret_cast<unsigned int*>(&dst[q * plane]), w);
      e = __ffma2_rn(unpack_bf16x2(ud[q * PLANE]), dup2(-1.0f), unpack_bf16x2(w));
    } else {
      if (st) __stcg(&dst[q * plane], u);
      e = __ffma2_rn(ud[q * PLANE], dup2(-1.0f), u);
    }
    if (MASK) e = __fmul2_rn(e, dup2(keep));
    if (NP == 2) {
      acc.dm.x = fmaxf(acc.dm.x, fabsf(e.x));
      acc.dm.y = fmaxf(acc.dm.y, fabsf(e.y));
    } else {
      acc.dm.x = fmaxf(acc.dm.x, fmaxf(fabsf(e.x), fabsf(e.y)));
    }
  }
}

// Plane pz of the column: finalise centre pz - 2 (slot d, when FIN), add
// plane pz to centres pz - 1 (l), pz (m) and pz + 1 (h, whose sums start
// here; its x and s come from stage pz + 1).  xs / us: stage pz at the
// column; xn / sn: stage pz + 1 at the column; ud: stage pz - 2 at the column.
template <int C, int NP, int UL, bool FIN>
__device__ __forceinline__ void step3(const float* __restrict__ xs,
                                      const typename Word3<UL>::T* __restrict__ us,
                                      const float* __restrict__ xn, const float* __restrict__ sn,
                                      const typename Word3<UL>::T* __restrict__ ud,
                                      Slot3<C, NP, UL>& d, Slot3<C, NP, UL>& l,
                                      Slot3<C, NP, UL>& m, Slot3<C, NP, UL>& h, float2 nx,
                                      const Fin3<C, NP, UL>& fc, Acc3<C, NP, UL>& acc,
                                      typename Word3<UL>::T* __restrict__ dst, int plane,
                                      bool st) {
  constexpr int K = S3<C, NP, UL>::K, KH = S3<C, NP, UL>::KH;
  h.x = xn[0];
  h.s = sn[0];
  h.xg = h.s < 0.0f ? h.x + 2.0f : h.x;
  if (FIN) fin3<C, NP, UL>(d, ud, nx, fc, acc, dst, plane, st);
  float2 W0[K], S1[K], S2[K];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int off = dy * BX + dx;
      const bool self = dx == 0 && dy == 0;
      const bool first = dx == -1 && dy == -1;
      const int q2 = dx * dx + dy * dy;
      const bool first_face = dy == -1 && dx == 0, first_corner = first;
      const float xk = xs[off];
      // g to the centres below and above: one packed difference with two
      // particles per item (measured 0.6 % and 3.7 % faster at c = 4 and 5),
      // two scalar ones with one (0.4 % faster at c = 6)
      float gl, gh;
      if constexpr (NP == 2) {
        const float2 glh = __fadd2_rn(make_float2(l.xg, h.xg), dup2(-xk));
        gl = fabsf(glh.x);
        gh = fabsf(glh.y);
      } else {
        gl = fabsf(l.xg - xk);
        gh = fabsf(h.xg - xk);
      }
      const float gm = self ? 0.0f : fabsf(m.xg - xk);
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const float2 uk = Word3<UL>::get(us, q * PLANE + off);
        if (q < KH) {
          l.H[q] = __ffma2_rn(uk, dup2(gl), l.H[q]);
          h.H[q] = first ? __fmul2_rn(uk, dup2(gh)) : __ffma2_rn(uk, dup2(gh), h.H[q]);
          if (!self) m.H[q] = __ffma2_rn(uk, dup2(gm), m.H[q]);
        }
        if (self) W0[q] = __fmul2_rn(uk, uk);
        else if (q2 == 1) S1[q] = first_face ? __fmul2_rn(uk, uk) : __ffma2_rn(uk, uk, S1[q]);
        else S2[q] = first_corner ? __fmul2_rn(uk, uk) : __ffma2_rn(uk, uk, S2[q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const float2 V = __ffma2_rn(dup2(2.0f), S2[q], S1[q]);                          // S1 + 2 S2
    const float2 A = __ffma2_rn(dup2(3.0f), S2[q], __ffma2_rn(dup2(2.0f), S1[q], W0[q]));
    l.F[q] = __fadd2_rn(l.F[q], A);
    m.F[q] = __fadd2_rn(m.F[q], V);
    h.F[q] = A;
  }
}

template <int C, int NP, int UL>
__global__ void __launch_bounds__(NT, 1) stencil3d_kernel(const __grid_constant__ StencilArgs a) {
  constexpr int K = S3<C, NP, UL>::K;
  using WT = typename Word3<UL>::T;
  extern __shared__ unsigned char dsmem_raw[];
  __shared__ __align__(8) uint64_t full[NSTAGE];
  __shared__ uint32_t lastq[NSTAGE];    // the last plane loaded into each stage
  __shared__ __align__(8) uint64_t empty[NSTAGE];
  __shared__ ItemTable tab;
  __shared__ int s_abort;
  __shared__ float s_red[NCW][NP * (2 * C + 2)];
  __shared__ ItemConst<C, NP> s_ic;
  // launched as a dependent of the stream's previous kernel: let the next
  // kernel be scheduled, and touch no memory before this one has finished
  grid_dep_trigger();
  grid_dep_wait();

  // 128-byte aligned start by pointer arithmetic, so that the compiler keeps
  // the shared address space of every stage pointer
  unsigned char* dsmem = dsmem_raw + ((128u - (smem_addr(dsmem_raw) & 127u)) & 127u);
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  constexpr int SB = s3_stage_bytes<C, NP, UL>();
  const uint64_t wait_ns = a.wait_ns ? a.wait_ns : kWaitLimitNs;

  // Active units of every volume (pairs (2k, 2k+1) active while either runs,
  // or particles), compacted one volume per warp (ballots).
  for (int v = warp; v < a.n_vol; v += NT / 32) {
    const VolDesc& vd = a.vol[v];
    const int units = vd.nz == 1 ? 0 : NP == 2 ? (vd.P + 1) / 2 : vd.P;
    int n = 0;
    for (int base = 0; base < units; base += 32) {
      const int p = base + lane;
      const bool on =
          p < units &&
          (NP == 2 ? (a.active[vd.pbase + 2 * p] != 0 ||
                      (2 * p + 1 < vd.P && a.active[vd.pbase + 2 * p + 1] != 0))
                   : a.active[vd.pbase + p] != 0);
      const unsigned msk = __ballot_sync(0xffffffffu, on);
      const int ia = vd.pbase + n + __popc(msk & ((1u << lane) - 1u));
      if (on && IFCM_CHECK(ia >= 0 && ia < kMaxBatchParticles, a.status, 30))
        tab.act[ia] = static_cast<short>(p);
      n += __popc(msk);
    }
    if (lane == 0) {
      tab.vfirst[v] = vd.pbase;
      tab.vnact[v] = n;
    }
  }
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      lastq[s] = 0xffffffffu;
      mbar_init(&empty[s], NCW);
    }
    fence_mbarrier_init();
  }
  __syncthreads();
  if (tid == 0) {
    int items = 0;
    for (int v = 0; v < a.n_vol; ++v) {
      tab.vitem[v] = items;
      items += tab.vnact[v] * a.vol[v].n_tiles;
    }
    tab.vitem[a.n_vol] = items;
  }
  __syncthreads();
  const int n_items = tab.vitem[a.n_vol];
  if (static_cast<int>(blockIdx.x) >= n_items) return;

  // One plane of an item into its ring stage (plane qq of the CTA's sequence).
  auto load_plane = [&](uint32_t qq, const Item& it, int pz) {
    const VolDesc& vd = a.vol[it.v];
    const uint32_t s = qq & (NSTAGE - 1);
    if (!IFCM_CHECK(pz >= 0 && pz < vd.nz && it.unit * vd.src_cstride + K <= vd.src_planes,
                    a.status, 31))
      return;
    unsigned char* st = dsmem + s * SB;
    lastq[s] = qq;
    mbar_arrive_expect_tx(&full[s], s3_tx_bytes<C, NP, UL>());
    tma_load_3d(st, &a.tm_x[it.v], &full[s], it.x0 - 4, it.y0 - 1, pz);
    tma_load_3d(st + XBYTES, &a.tm_s[it.v], &full[s], it.x0, it.y0, pz);
    tma_load_4d(st + XBYTES + SBYTES, &a.tm_u[it.v], &full[s], it.x0 - 4, it.y0 - 1, pz,
                it.unit * vd.src_cstride);
  };


  // ------------------------------------------------------------ producer
  if (warp == NCW) {
    if (lane == 0) {
      uint32_t q = 0;
      bool go = true;
      for (int w = blockIdx.x; go && w < n_items; w += gridDim.x) {
        const Item it = decode_item<NP, UL>(a, tab, w);
        for (int pz = it.pzb; pz <= it.pze; ++pz, ++q) {
          const uint32_t s = q & (NSTAGE - 1);
          if (q >= NSTAGE && !mbar_wait_bounded(&empty[s], ((q / NSTAGE) - 1) & 1, wait_ns)) {
            atomicExch(&s_abort, 1);
            set_status(a.status, IFCM_ERR_TIMEOUT, 5);
            go = false;
            break;
          }
          if (*reinterpret_cast<volatile int*>(&s_abort)) {
            go = false;
            break;
          }
          load_plane(q, it, pz);
        }
      }
    }
  } else {

  // ------------------------------------------------------------ consumers
  const int tx = tid & 31, ty = tid >> 5;
  const int cidx = (ty + 1) * BX + tx + 4;     // the column in a stage plane
  const int sidx = ty * TX + tx;               // the column in a stage's 1/G tile
  uint32_t q = 0;

  auto xs_at = [&](uint32_t qq) {
    return reinterpret_cast<const float*>(dsmem + (qq & (NSTAGE - 1)) * SB) + cidx;
  };
  auto ss_at = [&](uint32_t qq) {
    return reinterpret_cast<const float*>(dsmem + (qq & (NSTAGE - 1)) * SB + XBYTES) + sidx;
  };
  auto us_at = [&](uint32_t qq) {
    return reinterpret_cast<const WT*>(dsmem + (qq & (NSTAGE - 1)) * SB + XBYTES + SBYTES) + cidx;
  };
  auto wait_full = [&](uint32_t qq) -> bool {
    if (*reinterpret_cast<volatile int*>(&s_abort)) return false;
    const bool landed = mbar_wait_bounded(&full[qq & (NSTAGE - 1)], (qq / NSTAGE) & 1, wait_ns);
    if (!landed) {
      atomicExch(&s_abort, 1);
      set_status(a.status, IFCM_ERR_TIMEOUT, 6);
      return false;
    }
    return true;
  };

  // stage qq is free once every consumer warp released it
  auto release = [&](uint32_t qq) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[qq & (NSTAGE - 1)]);
  };

  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const Item it = decode_item<NP, UL>(a, tab, w);
    const VolDesc& vd = a.vol[it.v];
    const uint32_t q0 = q;
    const int plane = vd.nz * vd.ny * vd.pitch;
    const int np = it.pze - it.pzb + 1;
    const Ctx cx = column_ctx(it.x0 + tx, it.y0 + ty, vd);
    if (tid == 0) {
      float lam[2], xi[2], cc[2][C];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int pid = (p == 0 || NP == 1) ? it.p0 : it.p1;
        lam[p] = static_cast<float>(vd.lam_xi[2 * pid]);
        xi[p] = static_cast<float>(vd.lam_xi[2 * pid + 1]);
#pragma unroll
        for (int j = 0; j < C; ++j)
          cc[p][j] = static_cast<float>(a.centres[(vd.pbase + pid) * C + j]);
      }
      s_ic.dst[0] = vd.u_dst + static_cast<size_t>(it.unit) * K * plane * (word_bytes(UL) / 4);
      s_ic.nlam = make_float2(-lam[0], -lam[1]);
      s_ic.nxi = make_float2(-xi[0], -xi[1]);
#pragma unroll
      for (int q = 0; q < K; ++q)
        s_ic.ncc[q] = NP == 2 ? make_float2(-cc[0][q], -cc[1][q])
                              : make_float2(-cc[0][2 * q],
                                            2 * q + 1 < C ? -cc[0][2 * q + 1] : 0.0f);
    }
    consumer_sync();
    Acc3<C, NP, UL> acc;
    acc.clear();

    {
      float iqz;   // 1/Q of the column's centres on a z face
      {
        int cnt;
        float Q;
        box_counts(cx.X, cx.Y, 0, vd.nx, vd.ny, vd.nz, cnt, Q);
        iqz = cnt > 0 ? __frcp_rn(Q) : 0.0f;
      }
      Fin3<C, NP, UL> fc;
#pragma unroll
      for (int q = 0; q < K; ++q) fc.ncc[q] = s_ic.ncc[q];
      fc.nlam = s_ic.nlam;
      fc.one_nlam = __fadd2_rn(dup2(1.0f), s_ic.nlam);
      fc.floor = a.dist_floor;
      // -xi/Q of the column's centres off and on the z faces (Eq 7's 1/Q
      // folded into Eq 4's factor)
      const float2 nxc = __fmul2_rn(s_ic.nxi, dup2(cx.invQ_col));
      const float2 nxz = __fmul2_rn(s_ic.nxi, dup2(iqz));
      // stores of the column (the item's centres lie in [z0, z1) of the volume)
      const long long unit_end =
          (static_cast<long long>(it.unit) + 1) * K * plane * (word_bytes(UL) / 4);
      const bool st = cx.col_ok && IFCM_CHECK(it.z0 >= 0 && it.z1 <= vd.nz &&
                                                  unit_end <= vd.dst_elems,
                                              a.status, 32);
      WT* const col_dst = reinterpret_cast<WT*>(s_ic.dst[0]) + cx.col_off;
      const int zstride = vd.ny * vd.pitch;

      Slot3<C, NP, UL> s0, s1, s2, s3;
      // the first step whose delayed finalisation is a centre of the item
      const int kf = it.z0 - it.pzb + 2;
      // the generic step covers the steps before the first interior-z centre
      const int kh = kf + (it.z0 == 0 ? 1 : 0);
      bool ok = wait_full(q0) && (np < 2 || wait_full(q0 + 1));
      // centre pzb (slot m of the first step) starts with no sums; centre
      // pzb - 1 (slot l) is never finalised
      s1.clear();
      s2.clear();
      if (ok) {
        s2.x = xs_at(q0)[0];
        s2.s = ss_at(q0)[0];
        s2.xg = s2.s < 0.0f ? s2.x + 2.0f : s2.x;
      }

      // One plane with slot values rotated afterwards (first and last planes
      // of the item): the finalisation only from step kf on, the z-face 1/Q
      // for centre 0, no wait past the item's last plane.
      auto generic = [&](int kk) {
        const uint32_t qq = q0 + kk;
        const bool need2 = kk + 2 < np;
        const bool landed2 = !need2 || mbar_test_wait(&full[(qq + 2) & (NSTAGE - 1)],
                                                      ((qq + 2) / NSTAGE) & 1);
        const int zd = it.pzb + kk - 2;
        if (ok) {
          const float2 nx = zd == 0 ? nxz : nxc;
          WT* dst = col_dst + static_cast<long long>(zd) * zstride;
          if (kk >= kf)
            step3<C, NP, UL, true>(xs_at(qq), us_at(qq), xs_at(qq + 1), ss_at(qq + 1),
                                   us_at(qq + 6), s0, s1, s2, s3, nx, fc, acc, dst, plane, st);
          else
            step3<C, NP, UL, false>(xs_at(qq), us_at(qq), xs_at(qq + 1), ss_at(qq + 1),
                                    us_at(qq + 6), s0, s1, s2, s3, nx, fc, acc, dst, plane, st);
        }
        if (!landed2) ok = ok && wait_full(qq + 2);
        if (kk >= 2) release(qq - 2);
        s0 = s1;
        s1 = s2;
        s2 = s3;
      };

      int kk = 0;
      for (; kk < kh && kk < np; ++kk) generic(kk);
      // steady state: four planes per pass, slots in static rotation; every
      // step has its finalisation, an interior-z centre, and two stages ahead
      for (; ok && kk + 4 <= np - 2; kk += 4) {
        const uint32_t qq = q0 + kk;
        WT* dst = col_dst + static_cast<long long>(it.pzb + kk - 2) * zstride;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const uint32_t qr = qq + r;
          const bool landed2 =
              mbar_test_wait(&full[(qr + 2) & (NSTAGE - 1)], ((qr + 2) / NSTAGE) & 1);
          Slot3<C, NP, UL>& d = r == 0 ? s0 : r == 1 ? s1 : r == 2 ? s2 : s3;
          Slot3<C, NP, UL>& l = r == 0 ? s1 : r == 1 ? s2 : r == 2 ? s3 : s0;
          Slot3<C, NP, UL>& m = r == 0 ? s2 : r == 1 ? s3 : r == 2 ? s0 : s1;
          Slot3<C, NP, UL>& h = r == 0 ? s3 : r == 1 ? s0 : r == 2 ? s1 : s2;
          step3<C, NP, UL, true>(xs_at(qr), us_at(qr), xs_at(qr + 1), ss_at(qr + 1),
                                 us_at(qr + 6), d, l, m, h, nxc, fc, acc, dst + r * zstride, plane,
                                 st);
          if (!landed2) ok = ok && wait_full(qr + 2);
          release(qr - 2);
        }
      }
      for (; kk < np; ++kk) generic(kk);

      // After the last plane: s0 = centre pze - 1 (complete), s1 = centre pze
      // (complete only when pze is the top plane of the volume).
      const uint32_t ql = q0 + np - 1;
      const bool live = ok && !*reinterpret_cast<volatile int*>(&s_abort);
      const int zl = it.pze - 1;
      if (live && np >= 2 && zl >= it.z0 && zl < it.z1)
        fin3<C, NP, UL>(s0, us_at(ql - 1), zl == 0 ? nxz : nxc, fc, acc,
                        col_dst + static_cast<long long>(zl) * zstride, plane, st);
      if (live && it.pze == vd.nz - 1 && it.pze >= it.z0 && it.pze < it.z1)
        fin3<C, NP, UL>(s1, us_at(ql), nxz, fc, acc,
                        col_dst + static_cast<long long>(it.pze) * zstride, plane, st);
      if (np >= 2) release(ql - 1);
      release(ql);
    }
    q = q0 + np;
    if (!cx.col_ok) acc.clear();      // lanes outside the volume computed on garbage

    // Item partial sums: FP32 within a thread and a warp, FP64 across warps.
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
      for (int j = 0; j < C; ++j) {
        // cluster j of particle p: lane p of word j (NP = 2), lane j % 2 of word j / 2
        const bool hi = NP == 2 ? p == 1 : (j & 1);
        const int q = NP == 2 ? j : j >> 1;
        const float v0 = warp_sum(hi ? acc.s0[q].y : acc.s0[q].x);
        const float v1 = warp_sum(hi ? acc.s1[q].y : acc.s1[q].x);
        if (lane == 0) {
          s_red[warp][p * (2 * C + 2) + j] = v0;
          s_red[warp][p * (2 * C + 2) + C + j] = v1;
        }
      }
      const float vj = warp_sum(p == 0 ? acc.J.x : acc.J.y);
      const float vm = warp_max(p == 0 ? acc.dm.x : acc.dm.y);
      if (lane == 0) {
        s_red[warp][p * (2 * C + 2) + 2 * C] = vj;
        s_red[warp][p * (2 * C + 2) + 2 * C + 1] = vm;
      }
    }
    consumer_sync();
    if (tid < NP * (2 * C + 2)) {
      const int p = tid / (2 * C + 2), v = tid - p * (2 * C + 2);
      if (p == 0 ? it.on0 : it.two) {
        const int pid = p == 0 ? it.p0 : it.p1;
        const long long rec = vd.rec_base + static_cast<long long>(pid) * vd.n_tiles + it.tile;
        if (!IFCM_CHECK(rec >= 0 && rec < a.n_records, a.status, 33)) {
        } else if (v < 2 * C + 1) {
          if (a.reduce == IFCM_REDUCE_FP64) {
            double sum = 0.0;
#pragma unroll
            for (int wv = 0; wv < NCW; ++wv) sum += static_cast<double>(s_red[wv][tid]);
            a.partials[rec * (2 * C + 1) + v] = sum;
          } else {
            float sum = 0.0f, comp = 0.0f;
#pragma unroll
            for (int wv = 0; wv < NCW; ++wv) neumaier_add(sum, comp, s_red[wv][tid]);
            a.partials[rec * (2 * C + 1) + v] = static_cast<double>(__fadd_rn(sum, comp));
          }
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

  }   // consumers

  // After a timeout the consumers skipped their waits: before the CTA exits,
  // wait (bounded) for the copies still landing in its shared memory.  No
  // load is issued after the abort, so each stage has at most one.
  __syncthreads();
  if (tid == 0 && *reinterpret_cast<volatile int*>(&s_abort)) {
    for (int s = 0; s < NSTAGE; ++s)
      if (lastq[s] != 0xffffffffu) mbar_wait_bounded(&full[s], (lastq[s] / NSTAGE) & 1);
  }
}

// One launch of the 3D pair-word kernel (it takes the 3D volumes of `a`).
template <int C, int NP, int UL = UL_F32P>
cudaError_t launch3d_c(const StencilArgs& a, int grid, cudaStream_t s) {
  constexpr int smem = s3_smem_total<C, NP, UL>();
  cudaError_t e = cudaFuncSetAttribute(stencil3d_kernel<C, NP, UL>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return launch_dependent(stencil3d_kernel<C, NP, UL>, dim3(grid), dim3(NT), smem, s, a);
}

}  // namespace
}  // namespace pifcm
