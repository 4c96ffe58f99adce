// Batched IFCM iteration over 2D images, pair-word memberships, m = 2: the
// 8-neighbour stencil of Eqs 5-9 fused with Eq 4 (distance), Eq 2
// (membership), Eq 1 (objective) and the centre sums of Eq 3 -- the lean
// plane step of stencil3d_kernel (stencil3d.cuh) for images, which the paper's
// own experiments use (Table 7: n x n slices).
//
// Work items are those of stencil_kernel's 2D form: (pair-word unit, 32-column
// strip, run of TY-row tiles down the image); the TMA producer warp loads one
// tile per ring stage, with a one-row halo and aligned four-column margins,
// plus the tile's 1/G.  A tile's centres are complete once its stage is read
// (the 8-neighbourhood lies in the image plane), so a consumer thread keeps
// two centres: the tile's, whose H and F it sums in this step, and the
// previous tile's, which it finalises in the same step so that Eqs 4 and 2
// overlap the stencil.  As in 3D:
// - 1/G per pixel comes from gsum_kernel (once per image), and a flat
//   neighbourhood (reading R3) weighs every in-image neighbour alike through
//   the centre value x_i + 2;
// - pixels outside the image read x = 0 and u = 0 (zero-filled maps), so they
//   add nothing to H and F without a mask (reading R4);
// - with float2 words the last cluster's H is 1 - sum of the others (U^t from
//   Eq 2); bf16 words form every H;
// - F = S1 + 2 S2 from the window sums of u^2 over the four edge neighbours
//   (q^2 = 1) and the four corners (q^2 = 2);
// - Eq 4's factor folded: 1 + (-lambda/G) Hs_j + (-xi/Q) Fs_j.
// Lanes outside the image (the strip's overhang, the last tile's rows below
// the image) compute on zeros; their stores are predicated off and their
// shares weighed by 0.
#pragma once

#include "stencil3d.cuh"

namespace pifcm {

namespace {

// The tile's centre of the column: its sums over the 8 neighbours (KH H
// words, K F words) and its x, 1/G and x in g, as in 3D.
template <int C, int NP, int UL>
__device__ __forceinline__ void stencil2d_step(const float* __restrict__ xs,
                                               const float* __restrict__ ss,
                                               const typename Word3<UL>::T* __restrict__ us,
                                               Slot3<C, NP, UL>& m) {
  constexpr int K = S3<C, NP, UL>::K, KH = S3<C, NP, UL>::KH;
  m.x = xs[0];
  m.s = ss[0];
  m.xg = m.s < 0.0f ? m.x + 2.0f : m.x;
  float2 S1[K], S2[K];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      if (dx == 0 && dy == 0) continue;
      const int off = dy * BX + dx;
      const bool first = dx == -1 && dy == -1;
      const bool face = dx == 0 || dy == 0;
      const bool first_face = dy == -1 && dx == 0;
      const float g = fabsf(m.xg - xs[off]);
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const float2 uk = Word3<UL>::get(us, q * PLANE + off);
        if (q < KH) m.H[q] = first ? __fmul2_rn(uk, dup2(g)) : __ffma2_rn(uk, dup2(g), m.H[q]);
        if (face) S1[q] = first_face ? __fmul2_rn(uk, uk) : __ffma2_rn(uk, uk, S1[q]);
        else S2[q] = first ? __fmul2_rn(uk, uk) : __ffma2_rn(uk, uk, S2[q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < K; ++q) m.F[q] = __ffma2_rn(dup2(2.0f), S2[q], S1[q]);   // S1 + 2 S2
}

template <int C, int NP, int UL>
__global__ void __launch_bounds__(NT, 1) stencil2d_kernel(const __grid_constant__ StencilArgs a) {
  constexpr int K = S3<C, NP, UL>::K;
  using WT = typename Word3<UL>::T;
  extern __shared__ unsigned char dsmem_raw[];
  __shared__ __align__(8) uint64_t full[NSTAGE];
  __shared__ uint32_t lastq[NSTAGE];    // the last tile loaded into each stage
  __shared__ __align__(8) uint64_t empty[NSTAGE];
  __shared__ ItemTable tab;
  __shared__ int s_abort;
  __shared__ float s_red[NCW][NP * (2 * C + 2)];
  __shared__ ItemConst<C, NP> s_ic;
  // launched as a dependent of the stream's previous kernel: let the next
  // kernel be scheduled, and touch no memory before this one has finished
  grid_dep_trigger();
  grid_dep_wait();

  unsigned char* dsmem = dsmem_raw + ((128u - (smem_addr(dsmem_raw) & 127u)) & 127u);
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  constexpr int SB = s3_stage_bytes<C, NP, UL>();
  const uint64_t wait_ns = a.wait_ns ? a.wait_ns : kWaitLimitNs;

  // Active units of every image (pairs (2k, 2k+1) active while either runs,
  // or particles), compacted one volume per warp; 3D volumes get no items.
  for (int v = warp; v < a.n_vol; v += NT / 32) {
    const VolDesc& vd = a.vol[v];
    const int units = vd.nz != 1 ? 0 : NP == 2 ? (vd.P + 1) / 2 : vd.P;
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
      if (on && IFCM_CHECK(ia >= 0 && ia < kMaxBatchParticles, a.status, 34))
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

  // Tile pz of an item's strip into its ring stage (tile qq of the CTA's
  // sequence): x and U^t with a one-row halo, 1/G of the tile's pixels.
  auto load_tile = [&](uint32_t qq, const Item& it, int pz) {
    const VolDesc& vd = a.vol[it.v];
    const uint32_t s = qq & (NSTAGE - 1);
    if (!IFCM_CHECK(pz >= 0 && pz < (vd.ny + TY - 1) / TY &&
                        it.unit * vd.src_cstride + K <= vd.src_planes,
                    a.status, 35))
      return;
    unsigned char* st = dsmem + s * SB;
    lastq[s] = qq;
    mbar_arrive_expect_tx(&full[s], s3_tx_bytes<C, NP, UL>());
    tma_load_3d(st, &a.tm_x[it.v], &full[s], it.x0 - 4, pz * TY - 1, 0);
    tma_load_3d(st + XBYTES, &a.tm_s[it.v], &full[s], it.x0, pz * TY, 0);
    tma_load_4d(st + XBYTES + SBYTES, &a.tm_u[it.v], &full[s], it.x0 - 4, pz * TY - 1, 0,
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
            set_status(a.status, IFCM_ERR_TIMEOUT, 7);
            go = false;
            break;
          }
          if (*reinterpret_cast<volatile int*>(&s_abort)) {
            go = false;
            break;
          }
          load_tile(q, it, pz);
        }
      }
    }
  } else {

  // ------------------------------------------------------------ consumers
  const int tx = tid & 31, ty = tid >> 5;
  const int cidx = (ty + 1) * BX + tx + 4;     // the pixel in a stage plane
  const int sidx = ty * TX + tx;               // the pixel in a stage's 1/G tile
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
      set_status(a.status, IFCM_ERR_TIMEOUT, 8);
      return false;
    }
    return true;
  };
  auto release = [&](uint32_t qq) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[qq & (NSTAGE - 1)]);
  };

  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const Item it = decode_item<NP, UL>(a, tab, w);
    const VolDesc& vd = a.vol[it.v];
    const uint32_t q0 = q;
    const int plane = vd.ny * vd.pitch;
    const int np = it.pze - it.pzb + 1;
    const int X = it.x0 + tx;
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
      Fin3<C, NP, UL> fc;
#pragma unroll
      for (int q = 0; q < K; ++q) fc.ncc[q] = s_ic.ncc[q];
      fc.nlam = s_ic.nlam;
      fc.one_nlam = __fadd2_rn(dup2(1.0f), s_ic.nlam);
      fc.floor = a.dist_floor;
      const float2 nxi = s_ic.nxi;
      const long long unit_end =
          (static_cast<long long>(it.unit) + 1) * K * plane * (word_bytes(UL) / 4);
      const bool unit_ok = IFCM_CHECK(unit_end <= vd.dst_elems, a.status, 36);
      WT* const unit_dst = reinterpret_cast<WT*>(s_ic.dst[0]);

      // the centre of step kk: its pixel, whether it lies in the image, and
      // -xi/Q from its in-image neighbours (Eq 8, reading R4)
      auto centre_of = [&](int kk, float& keep, float2& nxq, WT*& dst) {
        const int Y = (it.pzb + kk) * TY + ty;
        const bool in = X < vd.nx && Y < vd.ny;
        int cnt;
        float Q;
        box_counts(X, Y, 0, vd.nx, vd.ny, 1, cnt, Q);
        keep = in ? 1.0f : 0.0f;
        nxq = __fmul2_rn(nxi, dup2(cnt > 0 ? __frcp_rn(Q) : 0.0f));
        dst = unit_dst + (in ? static_cast<long long>(Y) * vd.pitch + X : 0);
        return in && unit_ok;
      };

      Slot3<C, NP, UL> sd, sm;
      float keep_d = 0.0f;
      float2 nx_d = make_float2(0.0f, 0.0f);
      WT* dst_d = unit_dst;
      bool st_d = false;
      bool ok = wait_full(q0);
      for (int kk = 0; kk < np; ++kk) {
        const uint32_t qq = q0 + kk;
        const bool has_next = kk + 1 < np;
        const bool landed1 =
            !has_next || mbar_test_wait(&full[(qq + 1) & (NSTAGE - 1)], ((qq + 1) / NSTAGE) & 1);
        float keep_m;
        float2 nx_m;
        WT* dst_m;
        const bool st_m = centre_of(kk, keep_m, nx_m, dst_m);
        if (ok) {
          if (kk >= 1)
            fin3<C, NP, UL, true>(sd, us_at(qq - 1), nx_d, fc, acc, dst_d, plane, st_d, keep_d);
          stencil2d_step<C, NP, UL>(xs_at(qq), ss_at(qq), us_at(qq), sm);
        }
        if (!landed1) ok = ok && wait_full(qq + 1);
        if (kk >= 1) release(qq - 1);
        sd = sm;
        keep_d = keep_m;
        nx_d = nx_m;
        dst_d = dst_m;
        st_d = st_m;
      }
      const uint32_t ql = q0 + np - 1;
      if (ok && !*reinterpret_cast<volatile int*>(&s_abort))
        fin3<C, NP, UL, true>(sd, us_at(ql), nx_d, fc, acc, dst_d, plane, st_d, keep_d);
      release(ql);
    }
    q = q0 + np;

    // Item partial sums: FP32 within a thread and a warp, FP64 across warps.
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const bool hi = NP == 2 ? p == 1 : (j & 1);
        const int qw = NP == 2 ? j : j >> 1;
        const float v0 = warp_sum(hi ? acc.s0[qw].y : acc.s0[qw].x);
        const float v1 = warp_sum(hi ? acc.s1[qw].y : acc.s1[qw].x);
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
        if (!IFCM_CHECK(rec >= 0 && rec < a.n_records, a.status, 37)) {
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
  // wait (bounded) for the copies still landing in its shared memory.
  __syncthreads();
  if (tid == 0 && *reinterpret_cast<volatile int*>(&s_abort)) {
    for (int s = 0; s < NSTAGE; ++s)
      if (lastq[s] != 0xffffffffu) mbar_wait_bounded(&full[s], (lastq[s] / NSTAGE) & 1);
  }
}

// One launch of the 2D pair-word kernel (it takes the 2D images of `a`).
template <int C, int NP, int UL = UL_F32P>
cudaError_t launch2d_c(const StencilArgs& a, int grid, cudaStream_t s) {
  constexpr int smem = s3_smem_total<C, NP, UL>();
  cudaError_t e = cudaFuncSetAttribute(stencil2d_kernel<C, NP, UL>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return launch_dependent(stencil2d_kernel<C, NP, UL>, dim3(grid), dim3(NT), smem, s, a);
}

}  // namespace
}  // namespace pifcm
