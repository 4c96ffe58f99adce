// Host-side launchers of the library's kernels (one per translation unit),
// called by the C ABI in api.cu.  Each returns the cudaError_t of its launch.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace pifcm {

// ------------------------------------------------ stencil iteration (batched)
// Tile of one stencil work item: TX x TY columns of voxels marched along z.
// kTY rows = kTY consumer warps (+ one producer warp) per CTA.
#ifndef PIFCM_STENCIL_TY
#define PIFCM_STENCIL_TY 11
#endif
constexpr int kTX = 32;
constexpr int kTY = PIFCM_STENCIL_TY;
constexpr int kThreads = kTX * kTY;

// One volume of a stencil launch.  A launch covers up to kMaxVols volumes of
// the same c; particle state arrays (centres, active) are shared by the
// launch and indexed by the volume's first particle pbase.
constexpr int kMaxVols = 64;
constexpr int kMaxBatchParticles = 4096;

struct VolDesc {
  int nx, ny, nz, pitch;
  int tiles_x, tiles_y, tz, n_tiles;   // 32x8 column tiles x z-chunks of tz planes
  int P;                        // particles of this volume in the batch
  int pbase;                    // index of its particle 0 in the launch's state arrays
  long long rec_base;           // first partial record: record = rec_base + p * n_tiles + tile
  const double* lam_xi;         // [P][2]
  float* u_dst;                 // [P][c][nz][ny][pitch]  U^{t+1}
  const float* u_src;           // particle 0's U^t (for the rare flat-neighbourhood path)
  long long src_pstride;        // elements between particles' U^t (0: one shared U^t)
  int src_cstride;              // TMA cluster-coordinate step per particle (c or 0)
  int src_planes;               // planes of the U^t tensor map (checked build)
  long long dst_elems;          // 4-byte elements of the U^{t+1} buffer (checked build)
  DevStatus* status;            // the launch's status word (checked build)
};

// Kernel parameter block (passed as __grid_constant__, so the tensor maps
// stay in parameter space): the volumes, their TMA maps, the shared state.
struct StencilArgs {
  CUtensorMap tm_x[kMaxVols];   // normalised volume (NaN outside)
  CUtensorMap tm_u[kMaxVols];   // memberships U^t (zero outside)
  CUtensorMap tm_s[kMaxVols];   // 1/G per voxel (gsum_kernel), 32 x TY boxes (3D kernel)
  VolDesc vol[kMaxVols];
  int n_vol;
  const double* centres;        // [particles of the launch][c]  C^t
  const int32_t* active;        // [particles of the launch]
  double* partials;             // [records][2c+1]
  float* dmax;                  // [records]
  long long n_records;          // records of the workspace (checked build)
  float dist_floor, m, inv_m1;
  int m_is_2;
  int reduce;                   // IFCM_REDUCE_FP64 or IFCM_REDUCE_COMP32 across warps
  int sum_one;                  // U^t comes from Eq 2 (memberships of a voxel sum to one)
  unsigned long long wait_ns;   // bound of one mbarrier wait (0: about one second)
  DevStatus* status;
};
static_assert(sizeof(StencilArgs) <= 32000, "kernel parameter block must stay below 32 KB");

// Layout of the memberships between iterations (see stencil_kernel.cuh):
// FP32 planes per particle, bf16 pair words, or float2 pair words.
constexpr int UL_PLANAR = 0, UL_BF16 = 1, UL_F32P = 2;

// Whether a stencil launch runs the lean plane step (stencil3d_kernel for 3D
// volumes, stencil2d_kernel for 2D images): pair words (one or two particles
// per item), m = 2, and -- for float2 words, whose last cluster's H is taken
// by complement -- U^t from Eq 2 (every iteration after the first); bf16
// words take every iteration.  Its volume maps are zero-filled outside the
// volume; the general kernel's are NaN-filled.
inline bool stencil_lean(int layout, int np, int m_is_2, int sum_one) {
  return ((layout == UL_F32P && sum_one) || layout == UL_BF16) && (np == 1 || np == 2) &&
         m_is_2;
}
inline bool stencil3d_eligible(int layout, int np, int m_is_2, int sum_one, int nz) {
  return stencil_lean(layout, np, m_is_2, sum_one) && nz > 1;
}

// np = particles sharing one work item: 1 for every c, 2 for c <= 5.
bool stencil_np_supported(int c, int np);
int stencil_default_np(int c);
size_t stencil_smem_bytes(int c, int np, int layout);
int stencil_blocks_per_sm(int c, int np, int layout);
cudaError_t launch_stencil(int c, int np, int layout, const StencilArgs& a, int grid,
                           cudaStream_t s);
// Pair words per voxel of one pair-word membership buffer of P particles
// laid out for np: ceil(P/2) * c (np = 2) or P * ceil(c/2) (np = 1).
long long pair_unit_words(int c, int np, int P);

// ------------------------------------- plain iteration (one thread per voxel)
constexpr int kMaxV = 4;            // neighbourhood shells (Eq 10) of the shell kernel

struct PlainArgs {
  int nx, ny, nz, pitch;
  const float* x;
  const float* u_src;           // U^t, or NULL for u = 1/c
  float* u_dst;                 // U^{t+1}
  const double* lam_xi;         // device (lambda, xi) [P][2], or NULL: use lam / xi below
  float lam, xi;
  const double* centres;        // [P][c] C^t
  const int32_t* active;        // [P]
  double* partials;             // [P][n_rec][2c+1]
  float* dmax;                  // [P][n_rec]
  long long n_records;          // records from partials on (checked build)
  long long dst_elems;          // elements of u_dst (checked build)
  float dist_floor, m, inv_m1;
  int m_is_2;
  int vpt;                      // voxels per thread
  int stencil;                  // 0: lambda = xi = 0, no neighbourhood terms
  DevStatus* status;
};

// The V > 1 shell kernel's extra arguments.  Particle p of a launch is
// blockIdx.y: its U^t at u_src + p * src_pstride, U^{t+1} at u_dst + p *
// dst_pstride, (lambda, xi) at lam_xi[2p], C^t at centres[p c], records
// p * n_rec + blockIdx.x.
struct ShellArgs {
  int P;                        // particles (grid y)
  long long src_pstride;        // elements between particles' U^t (0: one shared U^t)
  long long dst_pstride;        // elements between particles' U^{t+1}
  int n_rec;                    // records per particle (grid x)
  int V;                        // shells, 1..kMaxV
  float W[kMaxV];               // Eq 10 weights W_1..W_V
};

int plain_blocks(long long nvox, int vpt);
// One particle, V = 1 (sh.V == 1, sh.P == 1), or the shell kernel (sh.V > 1).
cudaError_t launch_plain(int c, const PlainArgs& a, const ShellArgs& sh, int blocks,
                         cudaStream_t s);

// ---------------------------------------------- per-particle finalisation
// One volume of a reduce launch (particle p of the volume is state index
// pbase + p; its records are rec_base + p * n_rec ... + n_rec - 1).
struct ReduceVol {
  int pbase, P, n_rec;
  long long rec_base;
  long long nvox;
  double* fitness;              // [P] or NULL
  int32_t* iters_out;           // [P] or NULL
  double* c_out;                // [P][c] or NULL
  double* trace;                // [P][max_iter][2c+1] C^{t+1}, S0^{t+1}, J^t, or NULL
};

struct ReduceArgs {
  int n_vol;
  int P_total;                  // particles of the launch (one CTA each)
  const double* partials;       // [records][2c+1]
  const float* dmax;            // [records]
  long long n_records;          // records of the workspace (checked build)
  RunState st;                  // arrays over the launch's particles
  int max_iter;
  double eps;
  int reduce;                   // IFCM_REDUCE_FP64 or IFCM_REDUCE_COMP32 across records
  DevStatus* status;
  ReduceVol vol[kMaxVols];
};

cudaError_t launch_reduce(int c, const ReduceArgs& a, cudaStream_t s);

// ------------------------------------------- resident runs (resident.cu)
// Whole runs of volumes small enough for shared memory: CTA gp runs particle
// gp of the launch (volume v's particle p is gp = pbase_v + p) through every
// iteration of its run with x, U^t and U^{t+1} held in shared memory.
constexpr int kResidentThreads = 512;
constexpr size_t kResidentSmemBytes = 225 * 1024;     // dynamic shared memory, at most

struct ResidentVol {
  const float* x;               // normalised volume [nz][ny][pitch]
  const float* u0;              // shared start [c][nz][ny][pitch], or NULL for u = 1/c
  const double* c0;             // [c] C^0, or NULL for c_j = (j + 1/2) / c
  const double* lam_xi;         // [P][2], or NULL for lambda = xi = 0
  double* fitness;              // [P] J of the last iteration, or NULL
  int32_t* iters_out;           // [P] iterations executed, or NULL
  double* c_out;                // [P][c] final centres, or NULL
  float* u_final;               // [c][nz][ny][pitch] final U of particle 0, or NULL
  int nx, ny, nz, pitch;
  int P, pbase;
};

struct ResidentArgs {
  ResidentVol vol[kMaxVols];
  int n_vol;
  RunState st;                  // [particles of the launch]: written at the end of each run
  float dist_floor, m, inv_m1;
  int m_is_2;
  int max_iter;
  double eps;
  int reduce;                   // IFCM_REDUCE_FP64 or IFCM_REDUCE_COMP32 across warps
  int stencil;                  // 0: no neighbourhood terms (the FCM start)
  DevStatus* status;
};

// Dynamic shared memory of a resident run: x plus two membership fields.
size_t resident_smem_bytes(int c, long long nvox);
// One launch of P_total CTAs; max_nvox = the largest volume of the launch.
cudaError_t launch_resident(int c, const ResidentArgs& a, int P_total, long long max_nvox,
                            cudaStream_t s);

// ------------------------------------------------ reverse pass (adjoint.cu)
// One iteration t of the reverse pass over K unrolled IFCM iterations.
struct AdjointArgs {
  int nx, ny, nz, pitch;
  const float* x;               // normalised volume
  const float* u;               // U^t (checkpoint)
  const float* ubar_next;       // adjoint of U^{t+1}, or NULL (zero)
  const double* lam_xi;         // device (lambda, xi)
  const double* c_t;            // C^t [c]
  const double* c_next;         // C^{t+1} [c]
  const double* s0_next;        // S0^{t+1} = sum_i u^m [c]
  const double* cbar_next;      // adjoint of C^{t+1} [c], or NULL (zero)
  float J_bar;                  // dL/dJ^t: 1 for the last iteration, else 0
  float* A;                     // [c][plane] H_bar / G (point kernel out, gather in)
  float* B;                     // [c][plane] F_bar / Q
  float* e;                     // [plane] 1 where G = 0 (flat neighbourhood)
  float* ubar_out;              // [c][plane] adjoint of U^t (gather kernel out)
  double* partials;             // [blocks][2 + c] lambda_bar, xi_bar, c_bar^t
  float dist_floor, m, inv_m1;
  int m_is_2;
};

// Blocks (and partial records) of the reverse pass's point kernel: 32 x 8
// column tiles times z-chunks of 32 planes.
int adjoint_blocks(int nx, int ny, int nz);
cudaError_t launch_adjoint_point(int c, const AdjointArgs& a, int blocks, cudaStream_t s);
cudaError_t launch_adjoint_gather(int c, const AdjointArgs& a, cudaStream_t s);
cudaError_t launch_adjoint_reduce(int c, const double* partials, int blocks, double* grad,
                                  double* cbar_out, cudaStream_t s);
// mode 0: start (best = current, +inf); 1: keep the best, take a step; 2: keep
// the best and write it to lam_xi.
cudaError_t launch_polish_step(double* lam_xi, const double* grad, const double* J, double* best,
                               double alpha, int mode, cudaStream_t s);

// ------------------------------------------------------- auxiliary kernels
cudaError_t launch_run_init(int c, int P, const double* c0, RunState st, double* J_clear,
                            cudaStream_t s);
cudaError_t launch_minmax(const float* v, int nx, int ny, int nz, int pitch, float* pmin,
                          float* pmax, int32_t* pbad, int blocks, cudaStream_t s);
cudaError_t launch_scale(const float* v, float* x, int nx, int ny, int nz, int pitch,
                         const float* pmin, const float* pmax, const int32_t* pbad, int nparts,
                         DevStatus* st, cudaStream_t s);
cudaError_t launch_fill(float* dst, float value, long long n, cudaStream_t s);
// s_i = 1/G_i with G_i = sum of |x_i - x_k| over the in-volume 26-neighbourhood
// (FP64), or -1/n_i where G_i = 0 (n_i in-volume neighbours, 0 for none), for
// every voxel of a 3D volume [nz][ny][pitch] (padding columns untouched).
cudaError_t launch_gsum(const float* x, int nx, int ny, int nz, int pitch, float* s_out,
                        cudaStream_t s);
cudaError_t launch_select_copy(const float* a, const float* b, const int32_t* iters,
                               float* dst, long long n, cudaStream_t s);
// Pair words of a shared start: u0 [c][plane] FP32 -> [c][plane] words (u, u)
// for np = 2, or [ceil(c/2)][plane] words (u_2k, u_2k+1) for np = 1; bf16x2
// (layout UL_BF16) or float2 (UL_F32P) words.
cudaError_t launch_pack_start(const float* u0, void* out, int c, int np, int layout,
                              long long plane, cudaStream_t s);
// Particle 0's memberships from the pair-word buffer its last iteration wrote
// (a after an odd number of iterations, else b) as FP32 [c][plane].
cudaError_t launch_unpack_select(const void* a, const void* b, const int32_t* iters, float* dst,
                                 int c, int np, int layout, long long plane, cudaStream_t s);
cudaError_t launch_pso_init(const pso_state& st, cudaStream_t s);
cudaError_t launch_pso_step(const pso_state& st, const double* fitness, cudaStream_t s);
cudaError_t launch_pso_best(const double* pbest_x, const double* pbest_f, int P,
                            double* lam_xi, int32_t* best, cudaStream_t s);
cudaError_t launch_result(int c, const double* centres, const double* lam_xi, const double* J,
                          const double* pbest_f, int P, const int32_t* iters_final,
                          const int32_t* iters_init, const unsigned long long* updates,
                          const int32_t* best, const DevStatus* status, pifcm_result* out,
                          cudaStream_t s);

}  // namespace pifcm
