// Batched IFCM iteration: the neighbourhood stencil of Eqs 5-9 fused with the
// distance (Eq 4), membership (Eq 2), objective (Eq 1) and centre sums (Eq 3),
// for every active particle of a batch, in one persistent launch.
//
// Work item = (group of NP particles, TX x TY column tile, z-chunk of tz
// planes); in a 2D image (group, column of tiles, run of tz tiles down the
// image), the tiles taking the place of the planes.  The last warp of each CTA
// (warp TY) is the producer: one lane walks the CTA's items plane by plane
// and, for each plane, issues TMA tile loads of the normalised volume x and of
// the c membership planes U^t of each particle of the group (one-voxel halo in
// y, aligned four-voxel margins in x) into a ring of shared-memory stages,
// gated by "full" (transaction bytes) and "empty" (one arrival per consumer
// warp) mbarriers.  Warps 0 .. TY-1 are consumers: thread (tx, ty) owns column
// (x0 + tx, y0 + ty) and keeps four centres of the column in registers.  The
// plane being consumed contributes to the centre below it (dz = +1), its own
// centre (dz = 0) and the centre above (dz = -1); the centre two planes below,
// completed by the previous plane, is finalised in the same step so that its
// long dependency chain overlaps the stencil arithmetic.  The per-centre sums
// are float2 pairs (the two particles of an item, or two clusters) updated
// with packed FP32x2 instructions.  A plane's stage is released once the
// centre it holds has been finalised:
// H = sum u g / sum g, F = sum u^2 q^2 / sum q^2 (q^2 = dx^2+dy^2+dz^2,
// reading R1), Eqs 4 and 2, U^{t+1} written from registers, and the centre's
// shares of sum u^m, sum u^m x, J and max|du|.
//
// Keeping the consumers' plane step free of stalls and branches decides the
// speed, since the kernel is bound by instruction issue and latency:
// - each stage's full barrier is tested once, without blocking, a plane
//   before the stage is needed; a blocking (bounded) wait follows only when
//   the stage had not landed by then;
// - the finalisation takes a branch-free form whenever every lane of the
//   warp allows it (a 3D centre off the z faces, sum g >= 1e-30, m = 2; Q of
//   the column computed once per item; lanes outside the volume masked), so
//   that it and the plane's stencil form one basic block the compiler can
//   interleave.  Every other centre takes the general form, with the same
//   arithmetic;
// - U^{t+1} goes out through explicit global stores, which the compiler can
//   move shared-memory loads across.
//
// Neighbours outside the volume are excluded (reading R4) without masks:
// the volume's tensor map fills positions outside the volume with NaN and
// g = max(|x_i - x_k|, 0) turns them into 0 (max ignores a NaN operand),
// while the membership tensor maps fill them with 0.  Out-of-range planes are
// never loaded.  The NP particles of a group share the x tile, every g_ik and
// sum_k g_ik.  Per item and particle, the sums go to a partial record (FP32
// within a thread and a warp, FP64 across warps) that the reduce kernel sums
// per particle in FP64.
//
// Membership layouts (template parameter UL): UL_PLANAR stores each particle's
// c FP32 planes; the pair-word layouts UL_BF16 and UL_F32P store one word per
// (voxel, pair) -- bf16x2 (4 bytes) or float2 (8 bytes) -- as described next.
//
// BF16 memberships (UL = UL_BF16): U^t and U^{t+1} are stored as bf16 pairs, one
// 32-bit word per (voxel, pair): the two particles of a fixed pair (2k, 2k+1)
// for the same cluster when NP = 2, or clusters (2k, 2k+1) of one particle
// when NP = 1 -- the same pairing as the packed FP32x2 sums, low half first.
// The TMA tiles therefore still move 4-byte elements (a pair plane has the
// shape of an FP32 plane), one shared-memory load yields a whole pair, and
// one 32-bit store writes one.  All arithmetic stays FP32: a word is unpacked
// exactly (bf16 -> f32 is a shift) and u' is rounded to nearest even once,
// when it is stored.  max|du| compares the stored (rounded) values; the sums of
// Eqs 1 and 3 use the FP32 u' that the rounding was applied to.  UL_F32P is
// the same pairing with float2 words: one 64-bit shared-memory load per pair
// and no unpacking, one 64-bit store per pair, bit-identical arithmetic to
// UL_PLANAR.
#pragma once

#include <cuda_bf16.h>

#include "ifcm_math.cuh"
#include "launch.h"

namespace pifcm {

namespace {

constexpr int TX = kTX, TY = kTY;
constexpr int NCW = TY;                // consumer warps, one per row of the tile
constexpr int NCT = NCW * 32;          // consumer threads (one per column of the tile)
constexpr int NT = NCT + 32;           // + one producer warp
constexpr int BX = TX + 8;             // x box: 4-voxel margins (TMA x must be 16-B aligned)
constexpr int BY = TY + 2;             // y box: one-voxel halo
constexpr int PLANE = BX * BY;         // floats in one channel of a stage
#ifndef PIFCM_STENCIL_STAGES
#define PIFCM_STENCIL_STAGES 8
#endif
constexpr int NSTAGE = PIFCM_STENCIL_STAGES;   // ring depth
static_assert(NSTAGE >= 6,
              "the consumers hold five stages at a time (pz-2 .. pz+1, and pz+2 tested)");
constexpr int XBYTES = ((PLANE * 4 + 127) / 128) * 128;
constexpr int CBAR = 1;                // named barrier id of the consumer warps

// Build-time tuning: CTAs per SM the register budget targets.
#ifndef PIFCM_STENCIL_MIN_BLOCKS
#define PIFCM_STENCIL_MIN_BLOCKS 1
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
// Pairs per voxel: with two particles per item, pair k is cluster k of both;
// with one, pair k is clusters 2k and 2k+1.
template <int C, int NP>
struct Pairs {
  static constexpr int K = NP == 2 ? C : (C + 1) / 2;
};
__host__ __device__ constexpr bool paired(int ul) { return ul != UL_PLANAR; }
__host__ __device__ constexpr int word_bytes(int ul) { return ul == UL_BF16 ? 4 : 8; }
// Bytes of a stage's membership block (every TMA destination 128-B aligned):
// c FP32 planes per particle, or one word plane per pair.
template <int C, int NP, int UL>
__host__ __device__ constexpr int ublock_bytes() {
  return paired(UL) ? ((Pairs<C, NP>::K * PLANE * word_bytes(UL) + 127) / 128) * 128
                    : NP * ubytes<C>();
}
template <int C, int NP, int UL>
__host__ __device__ constexpr int stage_bytes() {
  return XBYTES + ublock_bytes<C, NP, UL>();
}
static_assert(XBYTES % 128 == 0 && ubytes<3>() % 128 == 0 && ubytes<5>() % 128 == 0 &&
                  ubytes<7>() % 128 == 0,
              "TMA shared-memory destinations must start on 128-byte boundaries");
template <int C, int NP, int UL>
__host__ __device__ constexpr uint32_t stage_tx_bytes() {
  return static_cast<uint32_t>(PLANE * 4 + (paired(UL) ? Pairs<C, NP>::K * PLANE * word_bytes(UL)
                                                        : NP * C * PLANE * 4));
}
template <int C, int NP, int UL>
__host__ __device__ constexpr int smem_total() {
  return NSTAGE * stage_bytes<C, NP, UL>() + 128;
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
  int v;               // volume
  int p0, p1;          // the volume's particles of the group (p1 = p0 when the group has one)
  bool on0;            // p0 is running (its partial record is written)
  bool two;            // p1 is a distinct, running particle
  int unit;            // pair words: the pair (NP = 2) or particle (NP = 1) whose words are loaded
  int tile, x0, y0, z0, z1, pzb, pze;
};

// Work items of a launch, numbered volume by volume: the active units of
// volume v (act[vfirst[v] ...], vnact[v] of them) in groups, times the
// volume's tiles; vitem[v] is the volume's first item.  A unit is a particle,
// grouped NP at a time; with BF16 pairs of particles (NP = 2) it is a fixed
// pair (2k, 2k+1), active while either runs, one per group.
struct ItemTable {
  short act[kMaxBatchParticles];
  int vfirst[kMaxVols], vnact[kMaxVols], vitem[kMaxVols + 1];
};

// Units of a group: NP particles (planar), one unit (pair or particle) with pair words.
template <int NP, int UL>
__host__ __device__ constexpr int group_units() {
  return paired(UL) ? 1 : NP;
}

template <int NP, int UL>
__device__ __forceinline__ Item decode_item(const StencilArgs& a, const ItemTable& tab, int w) {
  Item it;
  int v = 0;
  while (v + 1 < a.n_vol && tab.vitem[v + 1] <= w) ++v;
  const VolDesc& vd = a.vol[v];
  it.v = v;
  const int wl = w - tab.vitem[v];
  const int g = wl / vd.n_tiles;
  it.tile = wl - g * vd.n_tiles;
  const short* act = tab.act + tab.vfirst[v];
  if (paired(UL) && NP == 2) {
    const int u = act[g];
    const bool has1 = 2 * u + 1 < vd.P;
    it.unit = u;
    it.p0 = 2 * u;
    it.p1 = has1 ? 2 * u + 1 : 2 * u;
    it.on0 = a.active[vd.pbase + it.p0] != 0;
    it.two = has1 && a.active[vd.pbase + it.p1] != 0;
  } else {
    it.p0 = act[g * NP];
    it.on0 = true;
    it.two = (NP == 2) && (g * NP + 1 < tab.vnact[v]);
    it.p1 = it.two ? act[g * NP + 1] : it.p0;
    it.unit = it.p0;
  }
  const int per_z = vd.tiles_x * vd.tiles_y;
  const int zc = it.tile / per_z;
  const int rem = it.tile - zc * per_z;
  const int ty = rem / vd.tiles_x;
  const int tx = rem - ty * vd.tiles_x;
  it.x0 = tx * TX;
  it.y0 = ty * TY;
  it.z0 = zc * vd.tz;
  if (vd.nz == 1) {   // 2D: steps z0 .. z1 - 1 are tiles down the image, tile z at rows TY z ..
    it.z1 = min(it.z0 + vd.tz, (vd.ny + TY - 1) / TY);
    it.pzb = it.z0;
    it.pze = it.z1 - 1;
  } else {
    it.z1 = min(it.z0 + vd.tz, vd.nz);
    it.pzb = max(it.z0 - 1, 0);
    it.pze = min(it.z1, vd.nz - 1);
  }
  return it;
}

// The per-centre sums are kept as float2 pairs and updated with packed FP32x2
// instructions (half the issue slots of scalar FP32).  With two particles per
// item, pair k holds cluster k of particle 0 and of particle 1; with one, pair
// k holds clusters 2k and 2k+1 (the second half of the last pair is unused
// when c is odd).

// A bf16 pair word as two exact floats (low half first).
__device__ __forceinline__ float2 unpack_bf16x2(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// Two floats rounded to nearest even into one bf16 pair word (x in the low half).
__device__ __forceinline__ uint32_t pack_bf16x2(float2 v) {
  const __nv_bfloat162 h = __float22bfloat162_rn(v);
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <int C, int NP, int UL>
__device__ __forceinline__ float2 load_pair(const float* __restrict__ us, int k, int off) {
  if (UL == UL_BF16) return unpack_bf16x2(reinterpret_cast<const uint32_t*>(us)[k * PLANE + off]);
  if (UL == UL_F32P) return reinterpret_cast<const float2*>(us)[k * PLANE + off];
  if (NP == 2) return make_float2(us[k * PLANE + off], us[ufloats<C>() + k * PLANE + off]);
  const float lo = us[(2 * k) * PLANE + off];
  const float hi = (2 * k + 1 < C) ? us[(2 * k + 1) * PLANE + off] : 0.0f;
  return make_float2(lo, hi);
}

// Component of (particle p, cluster j) in an array of pairs.
template <int C, int NP>
__device__ __forceinline__ float pick(const float2 (&v)[Pairs<C, NP>::K], int p, int j) {
  if (NP == 2) return p == 0 ? v[j].x : v[j].y;
  return (j & 1) ? v[j >> 1].y : v[j >> 1].x;
}

__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// Accumulators of one centre voxel of the column, for NP particles.
template <int C, int NP>
struct Slot {
  static constexpr int K = Pairs<C, NP>::K;
  float G;            // sum_k g_ik (shared by the particles)
  float2 H[K];        // sum_k u_kj g_ik
  float2 F[K];        // sum_k u_kj^2 q^2_ik
  __device__ __forceinline__ void clear() {
    G = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) H[k] = F[k] = make_float2(0.0f, 0.0f);
  }
};

// A thread's shares of the item's sums: sum u^m and sum u^m x (paired like the
// slots), J and max|du| per particle.
template <int C, int NP>
struct Sums {
  static constexpr int K = Pairs<C, NP>::K;
  float2 s0[K], s1[K];
  float J[NP], dm[NP];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int k = 0; k < K; ++k) s0[k] = s1[k] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int p = 0; p < NP; ++p) J[p] = dm[p] = 0.0f;
  }
};

// Constants of the item being processed, shared by the consumer threads.
template <int C, int NP>
struct ItemConst {
  float2 ncc[Pairs<C, NP>::K];   // minus the centres C^t, paired like the slots
  float2 nlam, nxi;              // minus lambda and xi of the pair's particles
  float* dst[NP];                // each particle's U^{t+1}
};

// Contributions of one plane (x in xs, memberships of particle p at us + p *
// ufloats<C>()) to the centres below (lo), in (mid) and above (hi) it.  F uses
// the plane's window sums of w = u^2 over the centre (W0), the four face
// neighbours (S1, dx^2 + dy^2 = 1) and the four corners (S2, = 2), each
// square fused into its sum: the planes above and below weigh q^2 =
// 1 + dx^2 + dy^2, i.e. W0 + 2 S1 + 3 S2; the same plane dx^2 + dy^2, i.e.
// S1 + 2 S2.
template <int C, int NP, int UL, bool Z3>
__device__ __forceinline__ void accumulate_plane(const float* __restrict__ xs,
                                                 const float* __restrict__ us, int cidx,
                                                 float x_lo, float x_mid, float x_hi,
                                                 Slot<C, NP>& lo, Slot<C, NP>& mid,
                                                 Slot<C, NP>& hi) {
  constexpr int K = Pairs<C, NP>::K;
  float2 W0[K], S1[K], S2[K];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int off = cidx + dy * BX + dx;
      const float xk = xs[off];
      const bool self = (dx == 0 && dy == 0);
      const int q2 = dx * dx + dy * dy;          // folded after unrolling
      const bool first_face = (dy == -1 && dx == 0), first_corner = (dy == -1 && dx == -1);
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
      const float2 gl2 = dup2(gl), gh2 = dup2(gh), gm2 = dup2(gm);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float2 uk = load_pair<C, NP, UL>(us, k, off);
        if (Z3) {
          lo.H[k] = __ffma2_rn(uk, gl2, lo.H[k]);
          hi.H[k] = __ffma2_rn(uk, gh2, hi.H[k]);
        }
        if (!self) mid.H[k] = __ffma2_rn(uk, gm2, mid.H[k]);
        if (self) W0[k] = __fmul2_rn(uk, uk);
        else if (q2 == 1) S1[k] = first_face ? __fmul2_rn(uk, uk) : __ffma2_rn(uk, uk, S1[k]);
        else S2[k] = first_corner ? __fmul2_rn(uk, uk) : __ffma2_rn(uk, uk, S2[k]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float2 B = __ffma2_rn(dup2(2.0f), S2[k], S1[k]);           // S1 + 2 S2
    if (Z3) {
      const float2 ab = __fadd2_rn(__fadd2_rn(W0[k], S1[k]), __fadd2_rn(S2[k], B));
      lo.F[k] = __fadd2_rn(lo.F[k], ab);
      hi.F[k] = __fadd2_rn(hi.F[k], ab);
    }
    mid.F[k] = __fadd2_rn(mid.F[k], B);
  }
}

// Per-item position of one consumer thread's column.
struct Ctx {
  int X, Y;
  bool col_ok, col_interior;
  int col_off;                 // Y * pitch + X
  float invQ_col;              // 1 / Q of the column's centres off the z faces (Eq 8)
};

// The position of a consumer thread's column (X, Y) in a volume; Q of its
// centres off the z faces (3D) or of its one centre (2D) comes from the
// in-volume neighbour count, 54 or 12 in the interior (Eq 8, reading R4).
__device__ __forceinline__ Ctx column_ctx(int X, int Y, const VolDesc& vd) {
  Ctx cx;
  cx.X = X;
  cx.Y = Y;
  cx.col_ok = (X < vd.nx) && (Y < vd.ny);
  cx.col_interior = X > 0 && X < vd.nx - 1 && Y > 0 && Y < vd.ny - 1;
  cx.col_off = Y * vd.pitch + X;
  const bool z3 = vd.nz > 1;
  if (cx.col_interior) {
    cx.invQ_col = z3 ? (1.0f / 54.0f) : (1.0f / 12.0f);
  } else {
    int cnt;
    float Q;
    box_counts(X, Y, z3 ? 1 : 0, vd.nx, vd.ny, z3 ? 3 : 1, cnt, Q);
    cx.invQ_col = cnt > 0 ? __frcp_rn(Q) : 0.0f;
  }
  return cx;
}

__device__ __forceinline__ float2 max2(float2 v, float lo) {
  return make_float2(fmaxf(v.x, lo), fmaxf(v.y, lo));
}

// H and F of a centre in the general case (Eqs 5-8): Q from the in-volume
// neighbours when the centre is on a face, and the small or zero sum_k g_ik
// cases of readings R2 and R3.
template <int C, int NP, int UL>
__device__ __forceinline__ void neighbour_terms(const Slot<C, NP>& sl, int z, bool interior,
                                                const VolDesc& a, const Item& it, const Ctx& cx,
                                                float2 (&H)[Pairs<C, NP>::K],
                                                float2 (&F)[Pairs<C, NP>::K]) {
  constexpr int K = Pairs<C, NP>::K;
  float invQ;
  int cnt = 1;
  if (interior) {
    invQ = a.nz > 1 ? (1.0f / 54.0f) : (1.0f / 12.0f);
  } else {
    float Q;
    box_counts(cx.X, cx.Y, z, a.nx, a.ny, a.nz, cnt, Q);
    invQ = cnt > 0 ? __frcp_rn(Q) : 0.0f;
  }
  if (cnt == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) H[q] = F[q] = make_float2(0.0f, 0.0f);
  } else {
    const float2 iq = dup2(invQ);
#pragma unroll
    for (int q = 0; q < K; ++q) F[q] = __fmul2_rn(sl.F[q], iq);
    if (sl.G >= 1.0e-30f) {
      const float2 ig = dup2(fast_rcp(sl.G));
#pragma unroll
      for (int q = 0; q < K; ++q) H[q] = __fmul2_rn(sl.H[q], ig);
    } else if (sl.G > 0.0f) {
      const float2 ig = dup2(__frcp_rn(sl.G));
#pragma unroll
      for (int q = 0; q < K; ++q) H[q] = __fmul2_rn(sl.H[q], ig);
    } else {   // every neighbour equals x_i: plain mean of u_kj (reading R3)
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const int pid = p == 0 ? it.p0 : it.p1;
        float Hm[C];
        if (UL == UL_BF16)
          flat_neighbourhood_mean_bf16<C>(
              reinterpret_cast<const uint32_t*>(a.u_src) +
                  static_cast<long long>(it.unit) * a.src_pstride,
              NP == 2, p, cx.X, cx.Y, z, a.nx, a.ny, a.nz, a.pitch, Hm);
        else if (UL == UL_F32P)
          flat_neighbourhood_mean_f32p<C>(
              reinterpret_cast<const float2*>(a.u_src) +
                  static_cast<long long>(it.unit) * a.src_pstride,
              NP == 2, p, cx.X, cx.Y, z, a.nx, a.ny, a.nz, a.pitch, Hm);
        else
          flat_neighbourhood_mean<C>(a.u_src + static_cast<long long>(pid) * a.src_pstride,
                                     cx.X, cx.Y, z, a.nx, a.ny, a.nz, a.pitch, Hm);
#pragma unroll
        for (int j = 0; j < C; ++j) {
          if (NP == 2) {
            if (p == 0) H[j].x = Hm[j];
            else H[j].y = Hm[j];
          } else if (j & 1) {
            H[j >> 1].y = Hm[j];
          } else {
            H[j >> 1].x = Hm[j];
            if (j == C - 1) H[j >> 1].y = 0.0f;
          }
        }
      }
    }
  }
}

// Finalise one centre (its u^t is read from its plane's stage at cus): H and F
// (Eqs 5, 7), then Eq 4 (clamped factor, floored d^2, reading R2), Eq 2, and
// the centre's shares of Eqs 1 and 3, in packed pairs.  FAST is the common
// case, taken only when the caller has checked it for every lane of the warp:
// a centre of a 3D volume off its z faces (Q depends on the column alone and
// was computed once per item), sum_k g_ik >= 1e-30 and m = 2.
// It has no branch, so that the compiler can schedule it in one basic block
// with the next plane's stencil; its arithmetic is the general path's.  With
// MASK, lanes whose column lies outside the volume (live = false) compute on
// but store nothing and add nothing to the sums.
template <int C, int NP, int UL, bool FAST, bool MASK = false>
__device__ __forceinline__ void finalize_centre(const Slot<C, NP>& sl, const float* cus,
                                                int cidx, float xc, int z, bool interior,
                                                const VolDesc& a, const Item& it,
                                                const ItemConst<C, NP>& ic, const Ctx& cx,
                                                const MethodConsts& k, Sums<C, NP>& acc,
                                                bool live = true) {
  constexpr int K = Pairs<C, NP>::K;
  // the stores of this centre: its plane and its unit's (or particle's)
  // U^{t+1} planes inside the destination buffer
  const long long plane_l = static_cast<long long>(a.nz) * a.ny * a.pitch;
  const long long unit_end =
      paired(UL) ? (static_cast<long long>(it.unit) + 1) * K * plane_l * (word_bytes(UL) / 4)
                 : (static_cast<long long>(it.two ? max(it.p0, it.p1) : it.p0) + 1) * C * plane_l;
  const bool keep = (!MASK || live) &&
                    IFCM_CHECK(z >= 0 && z < a.nz && unit_end <= a.dst_elems, a.status, 22);
  if (MASK) xc = keep ? xc : 0.0f;    // x is NaN outside the volume
  float2 H[K], F[K];
  if (FAST) {
    const float2 iq = dup2(cx.invQ_col);
    const float2 ig = dup2(fast_rcp(sl.G));
#pragma unroll
    for (int q = 0; q < K; ++q) {
      F[q] = __fmul2_rn(sl.F[q], iq);
      H[q] = __fmul2_rn(sl.H[q], ig);
    }
  } else {
    neighbour_terms<C, NP, UL>(sl, z, interior, a, it, cx, H, F);
  }
  // Eq 4 with reading R2: d2 = max(D max(f, 0), floor) = max(D f, floor) for
  // D >= 0 and floor > 0, so the factor needs no clamp of its own
  const float2 one2 = dup2(1.0f), xc2 = dup2(xc);
  float2 d2[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const float2 f = __ffma2_rn(ic.nxi, F[q], __ffma2_rn(ic.nlam, H[q], one2));
    const float2 dd = __fadd2_rn(xc2, ic.ncc[q]);
    d2[q] = max2(__fmul2_rn(__fmul2_rn(dd, dd), f), k.dist_floor);
  }
  // Eq 2
  float2 u[K], um[K];
  if (FAST || k.m_is_2) {
    float2 r[K];
#pragma unroll
    for (int q = 0; q < K; ++q) r[q] = make_float2(fast_rcp(d2[q].x), fast_rcp(d2[q].y));
    float2 inv;
    if (NP == 2) {
      float2 S = r[0];
#pragma unroll
      for (int q = 1; q < K; ++q) S = __fadd2_rn(S, r[q]);
      inv = make_float2(fast_rcp(S.x), fast_rcp(S.y));
      acc.J[0] += keep ? inv.x : 0.0f;         // sum_j u_j^2 d2_j = 1/S
      acc.J[NP - 1] += keep ? inv.y : 0.0f;
    } else {
      float S = 0.0f;
#pragma unroll
      for (int q = 0; q < K; ++q) S += (2 * q + 1 < C) ? r[q].x + r[q].y : r[q].x;
      inv = dup2(fast_rcp(S));
      acc.J[0] += keep ? inv.x : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      u[q] = __fmul2_rn(r[q], inv);
      um[q] = __fmul2_rn(u[q], u[q]);
      if (MASK) um[q] = keep ? um[q] : make_float2(0.0f, 0.0f);
    }
  } else {
    float Sp[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) Sp[p] = 0.0f;
    float av[NP][C];
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
      for (int j = 0; j < C; ++j) {
        av[p][j] = exp2f(-k.inv_m1 * log2f(pick<C, NP>(d2, p, j)));
        Sp[p] += av[p][j];
      }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float invS = fast_rcp(Sp[p]);
      float Jv = 0.0f;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const float uj = av[p][j] * invS;
        const float umj = exp2f(k.m * log2f(uj));
        Jv += umj * pick<C, NP>(d2, p, j);
        if (NP == 2) {
          if (p == 0) { u[j].x = uj; um[j].x = umj; }
          else { u[j].y = uj; um[j].y = umj; }
        } else if (j & 1) {
          u[j >> 1].y = uj; um[j >> 1].y = umj;
        } else {
          u[j >> 1].x = uj; um[j >> 1].x = umj;
          if (j == C - 1) { u[j >> 1].y = 0.0f; um[j >> 1].y = 0.0f; }
        }
      }
      acc.J[p] += Jv;
    }
  }
  // Eq 3 shares, max|du|, and the store of U^{t+1}
#pragma unroll
  for (int q = 0; q < K; ++q) {
    acc.s0[q] = __fadd2_rn(acc.s0[q], um[q]);
    acc.s1[q] = __ffma2_rn(um[q], xc2, acc.s1[q]);
  }
  const int plane = a.nz * a.ny * a.pitch;              // c * plane < 2^31 (host-checked)
  const int voff = z * (a.ny * a.pitch) + cx.col_off;
  if (UL == UL_F32P) {
    // one float2 word per pair (padding lane as for bf16 below)
    float2* dst = reinterpret_cast<float2*>(ic.dst[0]);
    const float2* cw = reinterpret_cast<const float2*>(cus);
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const bool pad_hi = NP == 1 && 2 * q + 1 >= C;
      const float2 uq = pad_hi ? make_float2(u[q].x, 0.0f) : u[q];
      if (keep) __stcg(&dst[q * plane + voff], uq);
      const float2 e = __ffma2_rn(cw[q * PLANE + cidx], dup2(-1.0f), uq);   // u' - u
      const float e0 = keep ? fabsf(e.x) : 0.0f, e1 = keep ? fabsf(e.y) : 0.0f;
      if (NP == 2) {
        acc.dm[0] = fmaxf(acc.dm[0], e0);
        acc.dm[NP - 1] = fmaxf(acc.dm[NP - 1], e1);
      } else {
        acc.dm[0] = fmaxf(acc.dm[0], pad_hi ? e0 : fmaxf(e0, e1));
      }
    }
    return;
  }
  if (UL == UL_BF16) {
    // one rounded pair word per pair; max|du| between stored values
    // (with one particle and an odd c, the high half of the last word is
    // padding: stored as 0 and left out of max|du|)
    uint32_t* dst = reinterpret_cast<uint32_t*>(ic.dst[0]);
    const uint32_t* cw = reinterpret_cast<const uint32_t*>(cus);
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const bool pad_hi = NP == 1 && 2 * q + 1 >= C;
      const float2 uq = pad_hi ? make_float2(u[q].x, 0.0f) : u[q];
      const uint32_t w = pack_bf16x2(uq);
      if (keep) __stcg(&dst[q * plane + voff], w);
      const float2 e = __ffma2_rn(unpack_bf16x2(cw[q * PLANE + cidx]), dup2(-1.0f),
                                  unpack_bf16x2(w));                       // u' - u
      const float e0 = keep ? fabsf(e.x) : 0.0f, e1 = keep ? fabsf(e.y) : 0.0f;
      if (NP == 2) {
        acc.dm[0] = fmaxf(acc.dm[0], e0);
        acc.dm[NP - 1] = fmaxf(acc.dm[NP - 1], e1);
      } else {
        acc.dm[0] = fmaxf(acc.dm[0], pad_hi ? e0 : fmaxf(e0, e1));
      }
    }
    return;
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    if (p == 1 && !it.two) break;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const float uj = pick<C, NP>(u, p, j);
      if (keep) __stcg(&ic.dst[p][j * plane + voff], uj);
      const float ej = fabsf(uj - cus[p * ufloats<C>() + j * PLANE + cidx]);
      acc.dm[p] = fmaxf(acc.dm[p], keep ? ej : 0.0f);
    }
  }
}

// FLAT selects the volumes a launch of this instantiation works on: the 2D
// images (FLAT) or the 3D volumes; the other kind gets no items.  The two
// plane loops are compiled apart so that neither shapes the other's code.
template <int C, int NP, int UL, bool FLAT>
__global__ void __launch_bounds__(NT, PIFCM_STENCIL_MIN_BLOCKS)
    stencil_kernel(const __grid_constant__ StencilArgs a) {
  extern __shared__ unsigned char dsmem_raw[];
  __shared__ __align__(8) uint64_t full[NSTAGE];
  __shared__ __align__(8) uint64_t empty[NSTAGE];
  __shared__ int lastq[NSTAGE];         // the last plane loaded into each stage
  __shared__ ItemTable tab;
  __shared__ int s_abort;
  __shared__ float s_red[NCW][NP * (2 * C + 2)];
  __shared__ ItemConst<C, NP> s_ic;
  // launched as a dependent of the stream's previous kernel: let the next
  // kernel be scheduled, and touch no memory before this one has finished
  grid_dep_trigger();
  grid_dep_wait();

  unsigned char* dsmem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsmem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const uint64_t wait_ns = a.wait_ns ? a.wait_ns : kWaitLimitNs;

  // Active units of every volume, compacted one volume per warp (ballots).
  constexpr bool kPairUnits = paired(UL) && NP == 2;
  for (int v = warp; v < a.n_vol; v += NT / 32) {
    const VolDesc& vd = a.vol[v];
    const int units = (vd.nz == 1) != FLAT ? 0 : kPairUnits ? (vd.P + 1) / 2 : vd.P;
    int n = 0;
    for (int base = 0; base < units; base += 32) {
      const int p = base + lane;
      bool on;
      if (kPairUnits)
        on = p < units && (a.active[vd.pbase + 2 * p] != 0 ||
                           (2 * p + 1 < vd.P && a.active[vd.pbase + 2 * p + 1] != 0));
      else
        on = p < units && a.active[vd.pbase + p] != 0;
      const unsigned m = __ballot_sync(0xffffffffu, on);
      const int ia = vd.pbase + n + __popc(m & ((1u << lane) - 1u));
      if (on && IFCM_CHECK(ia >= 0 && ia < kMaxBatchParticles, a.status, 20))
        tab.act[ia] = static_cast<short>(p);
      n += __popc(m);
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
      mbar_init(&empty[s], NCW);
      lastq[s] = -1;
    }
    fence_mbarrier_init();
  }
  __syncthreads();
  if (tid == 0) {
    int items = 0;
    for (int v = 0; v < a.n_vol; ++v) {
      tab.vitem[v] = items;
      constexpr int GU = group_units<NP, UL>();
      items += ((tab.vnact[v] + GU - 1) / GU) * a.vol[v].n_tiles;
    }
    tab.vitem[a.n_vol] = items;
  }
  __syncthreads();
  const int n_items = tab.vitem[a.n_vol];
  if (static_cast<int>(blockIdx.x) >= n_items) return;

  auto xs_of = [&](int s) {
    return reinterpret_cast<float*>(dsmem + s * stage_bytes<C, NP, UL>());
  };
  auto us_of = [&](int s) {
    return reinterpret_cast<float*>(dsmem + s * stage_bytes<C, NP, UL>() + XBYTES);
  };

  // ------------------------------------------------------------ producer
  // (after a timeout it stops loading and joins the CTA's final drain)
  if (warp == NCW) {
    if (lane == 0) {
      int q = 0;
      bool go = true;
      for (int w = blockIdx.x; go && w < n_items; w += gridDim.x) {
        const Item it = decode_item<NP, UL>(a, tab, w);
        const VolDesc& vd = a.vol[it.v];
        const CUtensorMap* mx = &a.tm_x[it.v];
        const CUtensorMap* mu = &a.tm_u[it.v];
        for (int pz = it.pzb; pz <= it.pze; ++pz, ++q) {
          const int s = q % NSTAGE;
          if (q >= NSTAGE &&
              !mbar_wait_bounded(&empty[s], static_cast<uint32_t>(((q / NSTAGE) - 1) & 1),
                                 wait_ns)) {
            atomicExch(&s_abort, 1);
            set_status(a.status, IFCM_ERR_TIMEOUT, 3);
            go = false;
            break;
          }
          if (*reinterpret_cast<volatile int*>(&s_abort)) {
            go = false;
            break;
          }
          {
            const int unit = paired(UL) ? it.unit : it.p0;
            const int K = paired(UL) ? Pairs<C, NP>::K : C;
            const int last = (NP == 2 && !paired(UL)) ? it.p1 : unit;
            const int ext = FLAT ? (vd.ny + TY - 1) / TY : vd.nz;
            if (!IFCM_CHECK(pz >= 0 && pz < ext && unit * vd.src_cstride + K <= vd.src_planes &&
                                last * vd.src_cstride + K <= vd.src_planes,
                            a.status, 21)) {
              go = false;
              break;
            }
          }
          lastq[s] = q;
          // a plane of the tile's column, or in 2D the tile of step pz
          const int ty0 = FLAT ? pz * TY : it.y0;
          const int tz0 = FLAT ? 0 : pz;
          mbar_arrive_expect_tx(&full[s], stage_tx_bytes<C, NP, UL>());
          tma_load_3d(xs_of(s), mx, &full[s], it.x0 - 4, ty0 - 1, tz0);
          tma_load_4d(us_of(s), mu, &full[s], it.x0 - 4, ty0 - 1, tz0,
                      (paired(UL) ? it.unit : it.p0) * vd.src_cstride);
          if (NP == 2 && !paired(UL))
            tma_load_4d(us_of(s) + ufloats<C>(), mu, &full[s], it.x0 - 4, ty0 - 1, tz0,
                        it.p1 * vd.src_cstride);
        }
      }
    }
  } else {

  // ------------------------------------------------------------ consumers
  const int tx = tid & 31, ty = tid >> 5;
  const int cidx = (ty + 1) * BX + tx + 4;     // the column's position in a stage plane
  MethodConsts k;
  k.dist_floor = a.dist_floor;
  k.m = a.m;
  k.inv_m1 = a.inv_m1;
  k.m_is_2 = a.m_is_2;
  int q = 0;

  // Waits for plane qq's stage (bounded; after a timeout every wait is skipped
  // so that all consumer threads still reach the same barriers).
  auto wait_full = [&](int qq) -> bool {
    if (*reinterpret_cast<volatile int*>(&s_abort)) return false;
    if (!mbar_wait_bounded(&full[qq % NSTAGE], static_cast<uint32_t>((qq / NSTAGE) & 1),
                           wait_ns)) {
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
    const Item it = decode_item<NP, UL>(a, tab, w);
    const VolDesc& vd = a.vol[it.v];
    const int plane = vd.nz * vd.ny * vd.pitch;
    // the thread's column (in 2D: its column in the item's first tile)
    const Ctx cx = column_ctx(it.x0 + tx, it.y0 + ty, vd);
    const bool warp_all_live = __all_sync(0xffffffffu, cx.col_ok);
    const bool warp_any_live = __any_sync(0xffffffffu, cx.col_ok);
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
        if (p < NP)
          s_ic.dst[p] = paired(UL) ? vd.u_dst + static_cast<size_t>(it.unit) *
                                                   Pairs<C, NP>::K * plane *
                                                   (word_bytes(UL) / 4)
                                   : vd.u_dst + static_cast<size_t>(pid) * C * plane;
      }
      s_ic.nlam = make_float2(-lam[0], -lam[1]);
      s_ic.nxi = make_float2(-xi[0], -xi[1]);
#pragma unroll
      for (int qk = 0; qk < Pairs<C, NP>::K; ++qk) {
        if (NP == 2) s_ic.ncc[qk] = make_float2(-cc[0][qk], -cc[1][qk]);
        else s_ic.ncc[qk] = make_float2(-cc[0][2 * qk], 2 * qk + 1 < C ? -cc[0][2 * qk + 1] : 0.0f);
      }
    }
    consumer_sync();
    Slot<C, NP> sd, sl, sm, sh;
    sd.clear();
    sl.clear();
    sm.clear();
    sh.clear();
    Sums<C, NP> acc;
    acc.clear();
    const int np = it.pze - it.pzb + 1;
    const int q0 = q;

    if (FLAT) {
      // 2D: the item's steps are tiles down the image, one per stage, each
      // with its own one-row halo.  A tile's centres are complete once its
      // stage is read (8-neighbourhood in the plane); each is finalised during
      // the next step, in the same basic block as that step's stencil, with
      // the branch-free form when the whole warp allows it (as in 3D).  Slot
      // sm takes the step's sums, sd holds the previous step's centre, whose
      // column is cp.
      bool ok = wait_full(q0);
      Ctx cp = cx;
      for (int kk = 0; kk < np; ++kk) {
        const int qq = q0 + kk;
        const bool has_next = kk + 1 < np;
        const bool landed1 =
            !has_next || mbar_test_wait(&full[(qq + 1) % NSTAGE],
                                        static_cast<uint32_t>(((qq + 1) / NSTAGE) & 1));
        const Ctx cc = column_ctx(it.x0 + tx, (it.pzb + kk) * TY + ty, vd);
        const bool fin = kk >= 1 && cp.col_ok;
        const bool all_g = __all_sync(0xffffffffu, !cp.col_ok || sd.G >= 1.0e-30f);
        const bool all_live = __all_sync(0xffffffffu, cp.col_ok);
        const bool any_live = __any_sync(0xffffffffu, cp.col_ok);
        const bool fast = kk >= 1 && all_g && k.m_is_2 && any_live;
        if (ok) {
          const float* xs = xs_of(qq % NSTAGE);
          const float* us = us_of(qq % NSTAGE);
          const float x_mid = xs[cidx];
          const int sdi = (qq + NSTAGE - 1) % NSTAGE;
          if (fast && all_live) {
            finalize_centre<C, NP, UL, true>(sd, us_of(sdi), cidx, xs_of(sdi)[cidx], 0, true, vd,
                                             it, s_ic, cp, k, acc);
            accumulate_plane<C, NP, UL, false>(xs, us, cidx, 0.0f, x_mid, 0.0f, sl, sm, sh);
          } else if (fast) {
            finalize_centre<C, NP, UL, true, true>(sd, us_of(sdi), cidx, xs_of(sdi)[cidx], 0,
                                                   true, vd, it, s_ic, cp, k, acc, cp.col_ok);
            accumulate_plane<C, NP, UL, false>(xs, us, cidx, 0.0f, x_mid, 0.0f, sl, sm, sh);
          } else {
            if (fin)
              finalize_centre<C, NP, UL, false>(sd, us_of(sdi), cidx, xs_of(sdi)[cidx], 0,
                                                cp.col_interior, vd, it, s_ic, cp, k, acc);
            accumulate_plane<C, NP, UL, false>(xs, us, cidx, 0.0f, x_mid, 0.0f, sl, sm, sh);
          }
        }
        if (!landed1) ok = ok && wait_full(qq + 1);
        if (kk >= 1) release(qq - 1);
        sd = sm;
        sm.clear();
        cp = cc;
      }
      const int ql = q0 + np - 1;
      if (cp.col_ok && !*reinterpret_cast<volatile int*>(&s_abort))
        finalize_centre<C, NP, UL, false>(sd, us_of(ql % NSTAGE), cidx, xs_of(ql % NSTAGE)[cidx],
                                          0, cp.col_interior, vd, it, s_ic, cp, k, acc);
      release(ql);
    } else {
      // sd / sl / sm / sh = centres pz - 2 (complete), pz - 1, pz, pz + 1 while
      // plane pz is consumed.  The centre completed by plane pz - 1 is finalised
      // in the same basic block as plane pz's stencil so that its dependency
      // chain (Eqs 4 and 2) overlaps the stencil arithmetic.  Each stage is
      // waited for once and one plane early: plane pz consumes stages pz - 2 ..
      // pz + 1 (pz + 1 supplies x of the centre above), and the full barrier of
      // stage pz + 2 is tested without blocking when plane pz starts, its result
      // read only after plane pz's arithmetic; only a stage that had not landed
      // by then is waited for (bounded).
      bool ok = wait_full(q0) && (np < 2 || wait_full(q0 + 1));
      // One plane: finalise centre pz - 2 (slot sd), add plane pz to the centres
      // pz - 1, pz and pz + 1 (slots sl, sm and sh; sh starts cleared).
      auto step = [&](int kk, Slot<C, NP>& sd, Slot<C, NP>& sl, Slot<C, NP>& sm,
                      Slot<C, NP>& sh) {
        const int qq = q0 + kk;
        const int pz = it.pzb + kk;
        const bool has_next = kk + 1 < np;
        const bool need2 = kk + 2 < np;
        const bool landed2 =
            !need2 || mbar_test_wait(&full[(qq + 2) % NSTAGE],
                                     static_cast<uint32_t>(((qq + 2) / NSTAGE) & 1));
        // centre pz - 2 is finalised here when it lies in the item's z-range;
        // the whole warp takes the fast form when every lane can (voted by all
        // 32 lanes, before any lane may skip the plane)
        const int zd = pz - 2;
        const bool fin_z = kk >= 2 && zd >= it.z0 && zd < it.z1;
        const bool fin = fin_z && cx.col_ok;
        const bool zin = zd > 0 && zd < vd.nz - 1;
        const bool inter = cx.col_interior && zin;
        const bool all_g = __all_sync(0xffffffffu, !cx.col_ok || sd.G >= 1.0e-30f);
        const bool fast = fin_z && zin && all_g && k.m_is_2 && warp_any_live;
        if (ok) {
          const float* xs = xs_of(qq % NSTAGE);
          const float* us = us_of(qq % NSTAGE);
          const float x_mid = xs[cidx];
          const float x_lo = kk > 0 ? xs_of((qq + NSTAGE - 1) % NSTAGE)[cidx] : 0.0f;
          const float x_hi = has_next ? xs_of((qq + 1) % NSTAGE)[cidx] : 0.0f;
          const int sdi = (qq + NSTAGE - 2) % NSTAGE;
          if (fast && warp_all_live) {
            finalize_centre<C, NP, UL, true>(sd, us_of(sdi), cidx, xs_of(sdi)[cidx], zd, true, vd,
                                             it, s_ic, cx, k, acc);
            accumulate_plane<C, NP, UL, true>(xs, us, cidx, x_lo, x_mid, x_hi, sl, sm, sh);
          } else if (fast) {      // a tile overhanging the volume: some lanes outside
            finalize_centre<C, NP, UL, true, true>(sd, us_of(sdi), cidx, xs_of(sdi)[cidx], zd,
                                                   true, vd, it, s_ic, cx, k, acc, cx.col_ok);
            accumulate_plane<C, NP, UL, true>(xs, us, cidx, x_lo, x_mid, x_hi, sl, sm, sh);
          } else {
            if (fin)
              finalize_centre<C, NP, UL, false>(sd, us_of(sdi), cidx, xs_of(sdi)[cidx], zd, inter,
                                                vd, it, s_ic, cx, k, acc);
            accumulate_plane<C, NP, UL, true>(xs, us, cidx, x_lo, x_mid, x_hi, sl, sm, sh);
          }
        }
        if (!landed2) ok = ok && wait_full(qq + 2);
        if (kk >= 2) release(qq - 2);
      };
      for (int kk = 0; kk < np; ++kk) {
        step(kk, sd, sl, sm, sh);
        sd = sl;
        sl = sm;
        sm = sh;
        sh.clear();
      }
      // After the last plane: sd = centre pze - 1 (complete) and sl = centre pze
      // (complete only when pze is the last plane of the volume).
      {
        const int ql = q0 + np - 1;
        const bool live = cx.col_ok && !*reinterpret_cast<volatile int*>(&s_abort);
        if (live && np >= 2 && it.pze - 1 >= it.z0 && it.pze - 1 < it.z1) {
          const int sdi = (ql + NSTAGE - 1) % NSTAGE;
          finalize_centre<C, NP, UL, false>(sd, us_of(sdi), cidx, xs_of(sdi)[cidx], it.pze - 1,
                                 cx.col_interior && it.pze - 1 > 0 && it.pze - 1 < vd.nz - 1, vd,
                                 it, s_ic, cx, k, acc);
        }
        if (live && it.pze == vd.nz - 1 && it.pze >= it.z0 && it.pze < it.z1) {
          const int sli = ql % NSTAGE;
          finalize_centre<C, NP, UL, false>(sl, us_of(sli), cidx, xs_of(sli)[cidx], it.pze,
                                 false, vd, it, s_ic, cx, k, acc);   // the top z face
        }
        if (np >= 2) release(ql - 1);
        release(ql);
      }
    }
    q = q0 + np;

    // Item partial sums: FP32 within a thread and a warp, FP64 across warps.
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const float v0 = warp_sum(pick<C, NP>(acc.s0, p, j));
        const float v1 = warp_sum(pick<C, NP>(acc.s1, p, j));
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
      if (p == 0 ? it.on0 : it.two) {
        const int pid = p == 0 ? it.p0 : it.p1;
        const long long rec = vd.rec_base + static_cast<long long>(pid) * vd.n_tiles + it.tile;
        if (!IFCM_CHECK(rec >= 0 && rec < a.n_records, a.status, 23)) {
        } else if (v < 2 * C + 1) {
          if (a.reduce == IFCM_REDUCE_FP64) {
            double sum = 0.0;
#pragma unroll
            for (int wv = 0; wv < NCW; ++wv) sum += static_cast<double>(s_red[wv][tid]);
            a.partials[rec * (2 * C + 1) + v] = sum;
          } else {   // compensated FP32 (Neumaier) across the warps
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
  // wait (bounded) for the copies still landing in its shared memory.  The
  // producer issues no load after the abort, so each stage has at most one.
  __syncthreads();
  if (tid == 0 && *reinterpret_cast<volatile int*>(&s_abort)) {
    for (int s = 0; s < NSTAGE; ++s)
      if (lastq[s] >= 0) mbar_wait_bounded(&full[s], static_cast<uint32_t>((lastq[s] / NSTAGE) & 1));
  }
}
// ---------------------------------------------------------------------------
// One iteration over the launch's volumes: the 3D kernel if it has 3D
// volumes, the 2D kernel if it has 2D images (both, one after the other on
// the stream, for a batch that mixes them).
// With deep_ok false the 3D volumes are left to another kernel.
template <int C, int NP, int UL>
cudaError_t launch_c(const StencilArgs& a, int grid, cudaStream_t s, bool deep_ok = true) {
  constexpr int smem = smem_total<C, NP, UL>();
  bool flat = false, deep = false;
  for (int v = 0; v < a.n_vol; ++v) (a.vol[v].nz == 1 ? flat : deep) = true;
  if (deep && deep_ok) {
    cudaError_t e = cudaFuncSetAttribute(stencil_kernel<C, NP, UL, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = launch_dependent(stencil_kernel<C, NP, UL, false>, dim3(grid), dim3(NT), smem, s, a);
    if (e != cudaSuccess) return e;
  }
  if (flat) {
    cudaError_t e = cudaFuncSetAttribute(stencil_kernel<C, NP, UL, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return launch_dependent(stencil_kernel<C, NP, UL, true>, dim3(grid), dim3(NT), smem, s, a);
  }
  return cudaSuccess;
}

// CTAs per SM (the 3D kernel; both have the same shared memory and block).
template <int C, int NP, int UL>
int blocks_per_sm_c() {
  int n = 0;
  constexpr int smem = smem_total<C, NP, UL>();
  cudaFuncSetAttribute(stencil_kernel<C, NP, UL, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stencil_kernel<C, NP, UL, false>, NT,
                                                    smem) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

}  // namespace
}  // namespace pifcm
