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
constexpr int kTX = 32;
constexpr int kTY = 8;
constexpr int kThreads = kTX * kTY;

struct StencilArgs {
  int nx, ny, nz, pitch;
  int tiles_x, tiles_y, zchunks, tz;
  int n_tiles;                  // tiles_x * tiles_y * zchunks, per particle
  int P;                        // particles in the batch
  const double* lam_xi;         // [P][2]
  const double* centres;        // [P][c]  C^t
  const int32_t* active;        // [P]
  float* u_dst;                 // [P][c][nz][ny][pitch]  U^{t+1}
  const float* u_src;           // particle 0's U^t (for the rare flat-neighbourhood path)
  long long src_pstride;        // elements between particles' U^t (0: one shared U^t)
  int src_cstride;              // TMA cluster-coordinate step per particle (c or 0)
  double* partials;             // [P][n_tiles][2c+1]
  float* dmax;                  // [P][n_tiles]
  float dist_floor, m, inv_m1;
  int m_is_2;
  DevStatus* status;
};

int stencil_particles_per_item(int c);   // particles sharing one work item
size_t stencil_smem_bytes(int c);
int stencil_blocks_per_sm(int c);
cudaError_t launch_stencil(int c, const CUtensorMap& tm_x, const CUtensorMap& tm_u,
                           const StencilArgs& a, int grid, cudaStream_t s);

// ------------------------------------- plain iteration (one thread per voxel)
struct PlainArgs {
  int nx, ny, nz, pitch;
  const float* x;
  const float* u_src;           // U^t, or NULL for u = 1/c
  float* u_dst;                 // U^{t+1}
  const double* lam_xi;         // device (lambda, xi), or NULL: use lam / xi below
  float lam, xi;
  const double* centres;        // [c] C^t
  const int32_t* active;        // [1]
  double* partials;             // [blocks][2c+1]
  float* dmax;                  // [blocks]
  float dist_floor, m, inv_m1;
  int m_is_2;
  int vpt;                      // voxels per thread
  int stencil;                  // 0: lambda = xi = 0, no neighbourhood terms
  DevStatus* status;
};

int plain_blocks(long long nvox, int vpt);
cudaError_t launch_plain(int c, const PlainArgs& a, int blocks, cudaStream_t s);

// ---------------------------------------------- per-particle finalisation
struct ReduceArgs {
  int P, n_rec;                 // particles; partial records per particle
  const double* partials;       // [P][n_rec][2c+1]
  const float* dmax;            // [P][n_rec]
  RunState st;
  double* fitness;              // [P] or NULL
  int32_t* iters_out;           // [P] or NULL
  double* c_out;                // [P][c] or NULL
  int max_iter;
  double eps;
  long long nvox;
  DevStatus* status;
};

cudaError_t launch_reduce(int c, const ReduceArgs& a, cudaStream_t s);

// ------------------------------------------------------- auxiliary kernels
cudaError_t launch_run_init(int c, int P, const double* c0, RunState st, double* J_clear,
                            cudaStream_t s);
cudaError_t launch_minmax(const float* v, int nx, int ny, int nz, int pitch, float* pmin,
                          float* pmax, int32_t* pbad, int blocks, cudaStream_t s);
cudaError_t launch_scale(const float* v, float* x, int nx, int ny, int nz, int pitch,
                         const float* pmin, const float* pmax, const int32_t* pbad, int nparts,
                         DevStatus* st, cudaStream_t s);
cudaError_t launch_fill(float* dst, float value, long long n, cudaStream_t s);
cudaError_t launch_select_copy(const float* a, const float* b, const int32_t* iters,
                               float* dst, long long n, cudaStream_t s);
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
