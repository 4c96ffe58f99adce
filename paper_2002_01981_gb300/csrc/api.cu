// C ABI of the 3DPIFCM library (declared in include/pifcm.h): argument checks,
// workspace layout, TMA tensor maps and the launch sequences of the path.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "launch.h"

using namespace pifcm;

namespace {

thread_local char g_msg[512] = "";

ifcm_status fail(ifcm_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return s;
}

#define CU_TRY(expr)                                                                  \
  do {                                                                                \
    cudaError_t e_ = (expr);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(IFCM_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),     \
                  __FILE__, __LINE__);                                                \
  } while (0)

#define ST_TRY(expr)                 \
  do {                               \
    ifcm_status s_ = (expr);         \
    if (s_ != IFCM_OK) return s_;    \
  } while (0)

// ------------------------------------------------------------ validation
ifcm_status check_shape(const ifcm_shape& s) {
  if (s.nx < 1 || s.ny < 1 || s.nz < 1)
    return fail(IFCM_ERR_INVALID, "shape %dx%dx%d: every extent must be >= 1", s.nx, s.ny, s.nz);
  if (s.pitch_x < s.nx || s.pitch_x % 4 != 0)
    return fail(IFCM_ERR_INVALID, "pitch_x %d must be >= nx (%d) and a multiple of 4",
                s.pitch_x, s.nx);
  const double elems = static_cast<double>(s.pitch_x) * s.ny * s.nz;
  if (elems > 4.0e9)
    return fail(IFCM_ERR_INVALID, "volume of %.0f elements exceeds the 4e9 limit", elems);
  return IFCM_OK;
}

ifcm_status check_params(const ifcm_params* p) {
  if (!p) return fail(IFCM_ERR_INVALID, "params is NULL");
  if (p->c < 2 || p->c > kMaxC) return fail(IFCM_ERR_INVALID, "c = %d outside 2..%d", p->c, kMaxC);
  if (!(p->m > 1.0) || !std::isfinite(p->m))
    return fail(IFCM_ERR_INVALID, "fuzzifier m = %g must be finite and > 1", p->m);
  if (p->V < 1 || p->V > kMaxV)
    return fail(IFCM_ERR_UNSUPPORTED, "V = %d shells: 1..%d are built", p->V, kMaxV);
  if (p->V > 1 && (!(p->h > 0.0) || !std::isfinite(p->h)))
    return fail(IFCM_ERR_INVALID, "h = %g must be finite and > 0 for V > 1", p->h);
  if (p->V > 1 && p->u_dtype != IFCM_U_FP32)
    return fail(IFCM_ERR_UNSUPPORTED, "V > 1 shells are built for FP32 memberships only");
  if (p->max_iter < 1) return fail(IFCM_ERR_INVALID, "max_iter = %d must be >= 1", p->max_iter);
  if (!(p->eps_u >= 0.0)) return fail(IFCM_ERR_INVALID, "eps_u = %g must be >= 0", p->eps_u);
  if (!(p->dist_floor > 0.0) || !(p->dist_floor < 1.0))
    return fail(IFCM_ERR_INVALID, "dist_floor = %g must lie in (0, 1)", p->dist_floor);
  if (p->u_dtype != IFCM_U_FP32 && p->u_dtype != IFCM_U_BF16)
    return fail(IFCM_ERR_INVALID, "u_dtype = %d: expected IFCM_U_FP32 or IFCM_U_BF16", p->u_dtype);
  if (p->reduce != IFCM_REDUCE_FP64 && p->reduce != IFCM_REDUCE_COMP32)
    return fail(IFCM_ERR_INVALID, "reduce = %d: expected IFCM_REDUCE_FP64 or IFCM_REDUCE_COMP32",
                p->reduce);
  return IFCM_OK;
}

bool is_bf16(const ifcm_params* p) { return p->u_dtype == IFCM_U_BF16; }

// Layout of the memberships between iterations for a batch of P_total
// particles: bf16 pair words when asked for; FP32 planes for V > 1 shells (the
// plain kernel); float2 pair words for every other FP32 run, one particle
// included (its clusters paired in the words).
int run_layout(const ifcm_params* p, int P_total) {
  (void)P_total;
  if (is_bf16(p)) return UL_BF16;
  if (p->V > 1) return UL_PLANAR;
  return UL_F32P;
}

// The kernels index one particle's c membership planes with 32-bit offsets.
ifcm_status check_extent(const ifcm_shape& s, const ifcm_params* p) {
  const double elems = static_cast<double>(p->c) * s.pitch_x * s.ny * s.nz;
  if (elems >= 2147483647.0)
    return fail(IFCM_ERR_INVALID,
                "c * pitch_x * ny * nz = %.0f must stay below 2^31 (memberships of one run)",
                elems);
  return IFCM_OK;
}

ifcm_status check_aligned(const void* ptr, const char* what) {
  if (!ptr) return fail(IFCM_ERR_INVALID, "%s is NULL", what);
  if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0)
    return fail(IFCM_ERR_INVALID, "%s must be 16-byte aligned", what);
  return IFCM_OK;
}

// ------------------------------------------------------------- workspace
struct Carver {
  uintptr_t base;
  size_t off = 0;
  explicit Carver(void* b) : base(reinterpret_cast<uintptr_t>(b)) {}
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~static_cast<size_t>(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
    return p;
  }
};

size_t plane_elems(const ifcm_shape& s) {
  return static_cast<size_t>(s.nz) * s.ny * s.pitch_x;
}

struct Tiling {
  int tiles_x, tiles_y, zchunks, tz, n_tiles;
};

// A work item covers ceil(nz / chunks) planes of one 32 x kTY column tile,
// with at most ceil(nz / kMinTileZ) chunks.  In a 2D image (nz = 1) an item is
// instead a run of 32 x kTY tiles down the image, one tile per ring stage:
// chunks cut each column of tiles into runs of ceil(y-tiles / chunks) tiles.
// The planning rule keeps those runs near kMinTileRun tiles or longer, but
// tiling() accepts any cut, down to one tile per item (the cut of images too
// small to fill the GPU).
constexpr int kMinTileZ = 8;
constexpr int kMinTileRun = 4;

int y_tiles(const ifcm_shape& s) { return (s.ny + kTY - 1) / kTY; }

// Steps of a whole item column: planes in 3D, tiles down the image in 2D.
int column_depth(const ifcm_shape& s) { return s.nz == 1 ? y_tiles(s) : s.nz; }

int max_chunks(const ifcm_shape& s) {
  const int d = column_depth(s), m = s.nz == 1 ? kMinTileRun : kMinTileZ;
  return d <= m ? 1 : (d + m - 1) / m;
}

// Most chunks tiling() accepts.
int chunk_limit(const ifcm_shape& s) { return s.nz == 1 ? column_depth(s) : max_chunks(s); }

Tiling tiling(const ifcm_shape& s, int chunks) {
  Tiling t;
  t.tiles_x = (s.nx + kTX - 1) / kTX;
  t.tiles_y = s.nz == 1 ? 1 : y_tiles(s);
  const int d = column_depth(s), mk = chunk_limit(s);
  const int k = chunks < 1 ? 1 : (chunks > mk ? mk : chunks);
  t.tz = (d + k - 1) / k;
  t.zchunks = (d + t.tz - 1) / t.tz;
  t.n_tiles = t.tiles_x * t.tiles_y * t.zchunks;
  return t;
}

// Most records one particle of this volume can have (any plan).
int max_tiles(const ifcm_shape& s) { return tiling(s, chunk_limit(s)).n_tiles; }

constexpr int kPlainVpt = 32;

// Buffers of a batch of IFCM runs over n volumes of the same c: two membership
// buffers per volume (P particles each), the partial records of every
// particle's tiles, and the per-particle run state (particle p of volume v is
// state index pbase[v] + p).
// With a pair-word layout ua / ub hold words for either plan (np = 1 or 2,
// whichever is larger) and u0p the packed shared start; np is the plan the
// last run used (it fixes the word layout).
struct RunBufs {
  int n;
  int layout;
  int np;
  float* ua[kMaxVols];
  float* ub[kMaxVols];
  float* u0p[kMaxVols];
  float* gs[kMaxVols];          // 1/G per voxel (gsum_kernel), one plane per volume
  const float* gs_of[kMaxVols]; // the volume gs holds 1/G of (the runs of one call reuse it)
  int pbase[kMaxVols];
  long long rec_base[kMaxVols];
  int rec_per_particle[kMaxVols];
  double* partials;
  float* dmax;
  long long n_records;          // records carved (all volumes)
  long long buf_elems[kMaxVols];   // 4-byte elements of each ua / ub buffer
  RunState st;
};

// 4-byte elements per voxel of one membership buffer of P particles; pairs2:
// the batch (two or more particles) may run two particles per item.
size_t run_buffer_elems(int c, int P, int layout, bool pairs2) {
  if (layout == UL_PLANAR) return static_cast<size_t>(P) * c;
  long long w = pair_unit_words(c, 1, P);
  if (pairs2 && c <= 5 && pair_unit_words(c, 2, P) > w) w = pair_unit_words(c, 2, P);
  if (layout == UL_F32P) w *= 2;          // 8-byte words
  // the FCM start (FP32 planes, one particle) also runs in these buffers
  if (w < c) w = c;
  return static_cast<size_t>(w);
}

int forced_np();

RunBufs carve_runs(Carver& cv, const ifcm_shape* shapes, const int* P, int n, int c,
                   int layout) {
  RunBufs r{};
  r.n = n;
  r.layout = layout;
  int P_total = 0;
  for (int v = 0; v < n; ++v) P_total += P[v];
  const bool pairs2 = P_total >= 2 || forced_np() == 2;
  long long recs = 0;
  int pb = 0;
  for (int v = 0; v < n; ++v) {
    const size_t pl = plane_elems(shapes[v]);
    const size_t be = run_buffer_elems(c, P[v], layout, pairs2) * pl;
    r.buf_elems[v] = static_cast<long long>(be);
    r.ua[v] = cv.take<float>(be);
    r.ub[v] = cv.take<float>(be);
    r.u0p[v] = layout == UL_PLANAR ? nullptr
               : cv.take<float>(static_cast<size_t>(c) * pl * (layout == UL_F32P ? 2 : 1));
    r.gs[v] = cv.take<float>(pl);
    const long long nvox = static_cast<long long>(shapes[v].nx) * shapes[v].ny * shapes[v].nz;
    int nrec = max_tiles(shapes[v]);
    const int nplain = plain_blocks(nvox, kPlainVpt);      // the plain kernel's records (P = 1)
    if (nplain > nrec) nrec = nplain;
    r.pbase[v] = pb;
    r.rec_base[v] = recs;
    r.rec_per_particle[v] = nrec;
    recs += static_cast<long long>(P[v]) * nrec;
    pb += P[v];
  }
  r.n_records = recs;
  r.partials = cv.take<double>(static_cast<size_t>(recs) * (2 * c + 1));
  r.dmax = cv.take<float>(static_cast<size_t>(recs));
  r.st.centres = cv.take<double>(static_cast<size_t>(pb) * c);
  r.st.J = cv.take<double>(pb);
  r.st.active = cv.take<int32_t>(pb);
  r.st.iters = cv.take<int32_t>(pb);
  r.st.updates = cv.take<unsigned long long>(1);
  return r;
}

RunBufs carve_run(Carver& cv, const ifcm_shape& s, int c, int P, int layout) {
  return carve_runs(cv, &s, &P, 1, c, layout);
}

RunState shifted(const RunState& st, int pbase, int c) {
  RunState r = st;
  r.centres += static_cast<size_t>(pbase) * c;
  r.J += pbase;
  r.active += pbase;
  r.iters += pbase;
  return r;
}

DevStatus* carve_status(Carver& cv) { return cv.take<DevStatus>(1); }

struct NormBufs {
  float* pmin;
  float* pmax;
  int32_t* pbad;
  int nparts;
};

NormBufs carve_norm(Carver& cv, const ifcm_shape& s) {
  NormBufs n;
  const long long rows = static_cast<long long>(s.ny) * s.nz;
  n.nparts = static_cast<int>(rows < 1024 ? rows : 1024);
  n.pmin = cv.take<float>(n.nparts);
  n.pmax = cv.take<float>(n.nparts);
  n.pbad = cv.take<int32_t>(n.nparts);
  return n;
}

// ------------------------------------------------------------ tensor maps
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

ifcm_status get_encode() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!g_encode) return fail(IFCM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  return IFCM_OK;
}

// Box of one stencil plane: TX + 8 columns (4-voxel aligned margins) by TY + 2 rows.
constexpr cuuint32_t kBoxX = kTX + 8, kBoxY = kTY + 2;

// planes <= 0: the volume x; else a membership map of `planes` planes of
// elem_bytes-byte elements (4: FP32 or a bf16x2 word; 8: a float2 word).
ifcm_status make_map(CUtensorMap* m, const float* base, const ifcm_shape& s, int planes,
                     int box_planes, int elem_bytes = 4, bool nan_fill = true) {
  ST_TRY(get_encode());
  const cuuint64_t row = static_cast<cuuint64_t>(s.pitch_x) * (planes <= 0 ? 4 : elem_bytes);
  if (planes <= 0) {   // 3D volume map: positions outside the volume read as NaN (or 0)
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(s.nx), static_cast<cuuint64_t>(s.ny),
                          static_cast<cuuint64_t>(s.nz)};
    cuuint64_t strides[2] = {row, row * s.ny};
    cuuint32_t box[3] = {kBoxX, kBoxY, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims,
                          strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          nan_fill ? CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA
                                   : CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(IFCM_ERR_CUDA, "tensor map (volume) failed: %d", (int)r);
    return IFCM_OK;
  }
  cuuint64_t dims[4] = {static_cast<cuuint64_t>(s.nx), static_cast<cuuint64_t>(s.ny),
                        static_cast<cuuint64_t>(s.nz), static_cast<cuuint64_t>(planes)};
  cuuint64_t strides[3] = {row, row * s.ny, row * s.ny * s.nz};
  cuuint32_t box[4] = {kBoxX, kBoxY, 1, static_cast<cuuint32_t>(box_planes)};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = g_encode(m, elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                           : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        4, const_cast<float*>(base), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(IFCM_ERR_CUDA, "tensor map (memberships) failed: %d", (int)r);
  return IFCM_OK;
}

// The 1/G planes of a volume (gsum_kernel's output): one 32 x TY box of the
// tile's centres per plane; positions outside the volume read as 0.
ifcm_status make_smap(CUtensorMap* m, const float* base, const ifcm_shape& s) {
  ST_TRY(get_encode());
  const cuuint64_t row = static_cast<cuuint64_t>(s.pitch_x) * 4;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(s.nx), static_cast<cuuint64_t>(s.ny),
                        static_cast<cuuint64_t>(s.nz)};
  cuuint64_t strides[2] = {row, row * s.ny};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(kTX), static_cast<cuuint32_t>(kTY), 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(IFCM_ERR_CUDA, "tensor map (1/G) failed: %d", (int)r);
  return IFCM_OK;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// ------------------------------------------------------------ profiling
// Event pairs around kernel launches of four kinds (IFCM_PROF_*): the
// stencil iteration, the adjoint point kernel, the adjoint gather kernel, and
// the stencil iterations of 3D batches that run stencil3d_kernel alone (those
// launches are in the first kind as well).
struct Profiler {
  std::mutex mu;
  bool on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> used[4];
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spare;
} g_prof;

cudaEvent_t prof_begin(cudaStream_t s, cudaEvent_t* end_out, int kind = IFCM_PROF_STENCIL) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (!g_prof.on) return nullptr;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return nullptr;                              // launches of a graph are not timed here
  std::pair<cudaEvent_t, cudaEvent_t> ev;
  if (!g_prof.spare.empty()) {
    ev = g_prof.spare.back();
    g_prof.spare.pop_back();
  } else {
    cudaEventCreate(&ev.first);
    cudaEventCreate(&ev.second);
  }
  g_prof.used[kind].push_back(ev);
  cudaEventRecord(ev.first, s);
  *end_out = ev.second;
  return ev.first;
}

// ------------------------------------------------------------ tracing
// NVTX ranges on the host thread around the enqueueing of a run's phases
// (the run, the FCM start, each generation, each IFCM iteration, the final
// run).  They cost a few instructions when no tool is attached; a profiler
// that records NVTX (e.g. Nsight Systems) shows them beside the launches.
struct Trace {
  explicit Trace(const char* name) { nvtxRangePushA(name); }
  Trace(const char* fmt, int i) {
    char buf[48];
    std::snprintf(buf, sizeof(buf), fmt, i);
    nvtxRangePushA(buf);
  }
  ~Trace() { nvtxRangePop(); }
  Trace(const Trace&) = delete;
  Trace& operator=(const Trace&) = delete;
};

// ------------------------------------------------------------ run loops
void fill_method(StencilArgs& a, const ifcm_params* p) {
  a.dist_floor = static_cast<float>(p->dist_floor);
  a.m = static_cast<float>(p->m);
  a.inv_m1 = static_cast<float>(1.0 / (p->m - 1.0));
  a.m_is_2 = p->m == 2.0;
  a.reduce = p->reduce;
}

// One volume of a batch of IFCM runs (host view).
struct BatchVol {
  const float* x;
  ifcm_shape shape;
  int P;
  const double* lam_xi;   // device [P][2]
  const float* u0;        // device [c][plane]: the shared start of the volume's runs
  const double* c0;       // device [c] or NULL
  double* fitness;        // device [P] or NULL
  int32_t* iters;         // device [P] or NULL
  double* c_out;          // device [P][c] or NULL
  bool start_eq2 = false; // u0 comes from Eq 2 (the memberships of a voxel sum to one)
};

// ------------------------------------------------------- stencil plans
// How one batched stencil launch is cut into work items: particles per item
// (np) and z-chunks per column tile (every volume of the launch is cut into
// the same number of chunks, each at least kMinTileZ planes deep).
struct StencilPlan {
  int np;
  int chunks;
};

long long plan_items(const BatchVol* vols, int n, const StencilPlan& pl) {
  long long items = 0;
  for (int v = 0; v < n; ++v)
    items += static_cast<long long>((vols[v].P + pl.np - 1) / pl.np) *
             tiling(vols[v].shape, pl.chunks).n_tiles;
  return items;
}

int plan_grid(int c, int layout, const StencilPlan& pl, long long items) {
  long long g = static_cast<long long>(sm_count()) * stencil_blocks_per_sm(c, pl.np, layout);
  if (g > items) g = items;
  return g < 1 ? 1 : static_cast<int>(g);
}

int most_chunks(const BatchVol* vols, int n) {
  int k = 1;
  for (int v = 0; v < n; ++v)
    if (max_chunks(vols[v].shape) > k) k = max_chunks(vols[v].shape);
  return k;
}

// Built-in choice: the deepest chunks that still give every CTA of the
// persistent grid at least four items (whole columns when the batch is big
// enough: fewer halo planes and pipeline fills per voxel).
StencilPlan heuristic_plan(const BatchVol* vols, int n, int c, int layout) {
  int P_total = 0;
  for (int v = 0; v < n; ++v) P_total += vols[v].P;
  // one particle: its clusters in pairs (two particles per item would
  // compute a duplicate lane)
  StencilPlan pl{P_total == 1 ? 1 : stencil_default_np(c), 1};
  const long long grid =
      static_cast<long long>(sm_count()) * stencil_blocks_per_sm(c, pl.np, layout);
  const int kmax = most_chunks(vols, n);
  while (pl.chunks < kmax && plan_items(vols, n, pl) < 4 * grid) ++pl.chunks;
  // 2D images whose one-tile items would not even fill the grid: a launch is
  // then one round of items, bound by its latency, so the shortest runs win
  int depth = 1;
  for (int v = 0; v < n; ++v) {
    if (vols[v].shape.nz != 1) return pl;
    if (column_depth(vols[v].shape) > depth) depth = column_depth(vols[v].shape);
  }
  const StencilPlan one{pl.np, depth};
  if (plan_items(vols, n, one) <= grid) return one;
  return pl;
}

struct Tuner {
  std::mutex mu;
  int mode = 0;
  StencilPlan force{0, 0};       // np > 0: every launch uses this plan
  std::map<std::vector<long long>, StencilPlan> cache;
} g_tune;

// Particles per item of the forced plan, 0 when none is forced.
int forced_np() {
  std::lock_guard<std::mutex> lk(g_tune.mu);
  return g_tune.force.np;
}

// Cache key: element type of the memberships (an IFCM_U_* value), c, and
// every volume's extent and particle count.
std::vector<long long> plan_key(const BatchVol* vols, int n, int c, int u_dtype) {
  std::vector<long long> k{u_dtype, c, n};
  for (int v = 0; v < n; ++v) {
    const ifcm_shape& s = vols[v].shape;
    k.insert(k.end(), {s.nx, s.ny, s.nz, vols[v].P});
  }
  return k;
}

// Parameter block of one iteration kind: 0 reads the shared start U0 and
// writes ua, 1 reads ua and writes ub, 2 reads ub and writes ua.
// Bound of every mbarrier wait of the stencil kernels (ifcm_set_wait_limit_ns).
std::atomic<unsigned long long> g_wait_ns{0};
// Whole runs of small volumes in one launch (ifcm_resident_enable): on by default.
std::atomic<int> g_resident{1};

ifcm_status build_args(StencilArgs& a, const BatchVol* vols, int n, const ifcm_params* p,
                       const RunBufs& rb, const StencilPlan& pl, int kind, DevStatus* status) {
  const int c = p->c;
  std::memset(static_cast<void*>(&a), 0, sizeof(StencilArgs));
  a.n_vol = n;
  a.centres = rb.st.centres;
  a.active = rb.st.active;
  a.partials = rb.partials;
  a.dmax = rb.dmax;
  a.n_records = rb.n_records;
  a.status = status;
  // iterations after the first read Eq 2's memberships; the first reads the
  // start, which may come from Eq 2 as well (pifcm3d's FCM start)
  bool starts_eq2 = true;
  for (int v = 0; v < n; ++v) starts_eq2 = starts_eq2 && vols[v].start_eq2;
  a.sum_one = kind != 0 || starts_eq2;
  a.wait_ns = g_wait_ns.load();
  fill_method(a, p);
  for (int v = 0; v < n; ++v) {
    const BatchVol& bv = vols[v];
    const ifcm_shape& s = bv.shape;
    const Tiling t = tiling(s, pl.chunks);
    const size_t plane = plane_elems(s);
    VolDesc& d = a.vol[v];
    d.nx = s.nx;
    d.ny = s.ny;
    d.nz = s.nz;
    d.pitch = s.pitch_x;
    d.tiles_x = t.tiles_x;
    d.tiles_y = t.tiles_y;
    d.tz = t.tz;
    d.n_tiles = t.n_tiles;
    d.P = bv.P;
    d.pbase = rb.pbase[v];
    d.rec_base = rb.rec_base[v];
    d.lam_xi = bv.lam_xi;
    d.u_dst = kind == 1 ? rb.ub[v] : rb.ua[v];
    d.dst_elems = rb.buf_elems[v];
    d.status = status;
    const bool lean = stencil_lean(rb.layout, pl.np, a.m_is_2, a.sum_one);
    ST_TRY(make_map(&a.tm_x[v], bv.x, s, 0, 0, 4, !lean));
    ST_TRY(make_smap(&a.tm_s[v], rb.gs[v], s));
    if (rb.layout != UL_PLANAR) {
      // pair words: K planes per unit (a particle pair for np = 2, a particle
      // for np = 1); iteration 0 reads the packed shared start (one unit)
      const int K = pl.np == 2 ? c : (c + 1) / 2;
      const int units = pl.np == 2 ? (bv.P + 1) / 2 : bv.P;
      const int wb = rb.layout == UL_F32P ? 8 : 4;
      const float* src = kind == 0 ? rb.u0p[v] : (kind == 1 ? rb.ua[v] : rb.ub[v]);
      d.u_src = src;
      d.src_pstride = kind == 0 ? 0 : static_cast<long long>(K) * plane;   // in words
      d.src_cstride = kind == 0 ? 0 : K;
      d.src_planes = kind == 0 ? K : units * K;
      ST_TRY(make_map(&a.tm_u[v], src, s, kind == 0 ? K : units * K, K, wb));
    } else {
      const float* src = kind == 0 ? bv.u0 : (kind == 1 ? rb.ua[v] : rb.ub[v]);
      d.u_src = src;
      d.src_pstride = kind == 0 ? 0 : static_cast<long long>(c) * plane;
      d.src_cstride = kind == 0 ? 0 : c;
      d.src_planes = kind == 0 ? c : bv.P * c;
      ST_TRY(make_map(&a.tm_u[v], src, s, kind == 0 ? c : bv.P * c, c));
    }
  }
  return IFCM_OK;
}

// Pair-word runs: each volume's shared start as pair words laid out for np.
ifcm_status pack_starts(const BatchVol* vols, int n, int c, const RunBufs& rb, int np,
                        cudaStream_t st) {
  if (rb.layout == UL_PLANAR) return IFCM_OK;
  for (int v = 0; v < n; ++v)
    CU_TRY(launch_pack_start(vols[v].u0, rb.u0p[v], c, np, rb.layout,
                             static_cast<long long>(plane_elems(vols[v].shape)), st));
  return IFCM_OK;
}

// Time every candidate plan on the batch itself: one launch from the shared
// start (fills ua), then two timed launches ua -> ub, as in any later
// iteration.  Only the stencil kernel runs, so the run state is untouched
// and the real run that follows starts from iteration 0 again.
ifcm_status tune_plan(const BatchVol* vols, int n, const ifcm_params* p, const RunBufs& rb,
                      DevStatus* status, cudaStream_t st, StencilPlan* best) {
  const int c = p->c;
  const int lay = rb.layout;
  const StencilPlan h = heuristic_plan(vols, n, c, lay);
  const int kmax = most_chunks(vols, n);
  std::vector<StencilPlan> cand;
  int P_total = 0;
  for (int v = 0; v < n; ++v) P_total += vols[v].P;
  for (int np = 1; np <= (P_total >= 2 ? 2 : 1); ++np) {
    if (!stencil_np_supported(c, np)) continue;
    for (int k : {1, 2, 3, 4, 6, 8, 12, 16}) {
      if (k > kmax) break;
      const StencilPlan pl{np, k};
      if (plan_items(vols, n, pl) < sm_count() && k < kmax) continue;
      cand.push_back(pl);
    }
    if (np == h.np && h.chunks > 16) cand.push_back(h);
  }
  std::vector<StencilArgs> args(2);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU_TRY(cudaEventCreate(&e0));
  CU_TRY(cudaEventCreate(&e1));
  float best_ms = 0.0f;
  *best = h;
  ifcm_status rc = IFCM_OK;
  for (const StencilPlan& pl : cand) {
    rc = build_args(args[0], vols, n, p, rb, pl, 0, status);
    if (rc == IFCM_OK) rc = build_args(args[1], vols, n, p, rb, pl, 1, status);
    if (rc != IFCM_OK) break;
    const int grid = plan_grid(c, lay, pl, plan_items(vols, n, pl));
    rc = pack_starts(vols, n, c, rb, pl.np, st);
    if (rc != IFCM_OK) break;
    cudaError_t e = launch_stencil(c, pl.np, lay, args[0], grid, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r)
      e = launch_stencil(c, pl.np, lay, args[1], grid, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = fail(IFCM_ERR_CUDA, "stencil plan timing: %s", cudaGetErrorString(e));
      break;
    }
    if (best_ms == 0.0f || ms < best_ms) {
      best_ms = ms;
      *best = pl;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

ifcm_status choose_plan_any(const BatchVol* vols, int n, const ifcm_params* p, const RunBufs& rb,
                            DevStatus* status, cudaStream_t st, StencilPlan* out);

// The plan of a batch; a single particle runs one per item (its buffers hold
// no second particle) unless a plan is forced.
ifcm_status choose_plan(const BatchVol* vols, int n, const ifcm_params* p, const RunBufs& rb,
                        DevStatus* status, cudaStream_t st, StencilPlan* out) {
  ST_TRY(choose_plan_any(vols, n, p, rb, status, st, out));
  int P_total = 0;
  for (int v = 0; v < n; ++v) P_total += vols[v].P;
  if (P_total < 2 && forced_np() == 0) out->np = 1;
  return IFCM_OK;
}

ifcm_status choose_plan_any(const BatchVol* vols, int n, const ifcm_params* p, const RunBufs& rb,
                            DevStatus* status, cudaStream_t st, StencilPlan* out) {
  const std::vector<long long> key = plan_key(vols, n, p->c, p->u_dtype);
  int mode;
  {
    std::lock_guard<std::mutex> lk(g_tune.mu);
    if (g_tune.force.np > 0 && stencil_np_supported(p->c, g_tune.force.np)) {
      *out = g_tune.force;
      return IFCM_OK;
    }
    auto it = g_tune.cache.find(key);
    if (it != g_tune.cache.end()) {
      *out = it->second;
      return IFCM_OK;
    }
    mode = g_tune.mode;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CU_TRY(cudaStreamIsCapturing(st, &cap));
  if (mode == 0 || cap != cudaStreamCaptureStatusNone) {
    *out = heuristic_plan(vols, n, p->c, rb.layout);   // a captured stream is never timed
    return IFCM_OK;
  }
  ST_TRY(tune_plan(vols, n, p, rb, status, st, out));
  std::lock_guard<std::mutex> lk(g_tune.mu);
  g_tune.cache[key] = *out;
  return IFCM_OK;
}

void fill_plain_method(PlainArgs& a, ShellArgs& sh, const ifcm_params* p);

// A prepared batch of IFCM runs of every particle of n volumes (same c,
// n <= kMaxVols): run state initialised from each volume's c0, the launch
// plan, the three parameter blocks of the stencil kernel (iteration 0: U0 ->
// ua, odd: ua -> ub, even: ub -> ua) or, for V > 1 shells, of the plain
// kernel, and the per-particle finalisation.  iteration(it) queues one
// iteration of every running particle.
struct BatchRun {
  const BatchVol* vols = nullptr;
  int n = 0;
  const ifcm_params* p = nullptr;
  RunBufs* rb = nullptr;
  DevStatus* status = nullptr;
  bool wide = false;                 // V > 1: plain kernel
  StencilPlan pl{1, 1};
  std::vector<StencilArgs> args;
  int grid = 1;
  ReduceArgs r{};

  ifcm_status prepare(const BatchVol* vols_, int n_, const ifcm_params* p_, RunBufs& rb_,
                      DevStatus* status_, int max_iter, double eps, cudaStream_t st) {
    vols = vols_;
    n = n_;
    p = p_;
    rb = &rb_;
    status = status_;
    wide = p->V > 1;
    const int c = p->c;
    int P_total = 0;
    for (int v = 0; v < n; ++v) {
      CU_TRY(launch_run_init(c, vols[v].P, vols[v].c0, shifted(rb->st, rb->pbase[v], c),
                             nullptr, st));
      P_total += vols[v].P;
    }
    if (!wide) {
      // 1/G of each volume for the lean pair-word kernels (plans are timed on them)
      if (rb->layout == UL_F32P || rb->layout == UL_BF16)
        for (int v = 0; v < n; ++v) {
          const ifcm_shape& s = vols[v].shape;
          if (rb->gs_of[v] != vols[v].x) {
            CU_TRY(launch_gsum(vols[v].x, s.nx, s.ny, s.nz, s.pitch_x, rb->gs[v], st));
            rb->gs_of[v] = vols[v].x;
          }
        }
      ST_TRY(choose_plan(vols, n, p, *rb, status, st, &pl));
      rb->np = pl.np;
      ST_TRY(pack_starts(vols, n, c, *rb, pl.np, st));
      args.resize(3);
      for (int k = 0; k < 3; ++k) ST_TRY(build_args(args[k], vols, n, p, *rb, pl, k, status));
      grid = plan_grid(c, rb->layout, pl, plan_items(vols, n, pl));
    } else {
      rb->np = 1;
    }
    r = ReduceArgs{};
    r.n_vol = n;
    r.P_total = P_total;
    r.partials = rb->partials;
    r.dmax = rb->dmax;
    r.n_records = rb->n_records;
    r.st = rb->st;
    r.max_iter = max_iter;
    r.eps = eps;
    r.reduce = p->reduce;
    r.status = status;
    for (int v = 0; v < n; ++v) {
      ReduceVol& rv = r.vol[v];
      const ifcm_shape& s = vols[v].shape;
      rv.pbase = rb->pbase[v];
      rv.P = vols[v].P;
      rv.nvox = static_cast<long long>(s.nx) * s.ny * s.nz;
      rv.n_rec = wide ? plain_blocks(rv.nvox, kPlainVpt) : tiling(s, pl.chunks).n_tiles;
      rv.rec_base = rb->rec_base[v];
      rv.fitness = vols[v].fitness;
      rv.iters_out = vols[v].iters;
      rv.c_out = vols[v].c_out;
    }
    return IFCM_OK;
  }

  ifcm_status iteration(int it, cudaStream_t st) {
    const Trace tr("ifcm iteration %d", it);
    const int c = p->c;
    const int kind = it == 0 ? 0 : (it % 2 == 1 ? 1 : 2);
    if (!wide) {
      bool k3 = true;   // the launch is one stencil3d_kernel launch
      for (int v = 0; v < n; ++v)
        k3 = k3 && stencil3d_eligible(rb->layout, pl.np, args[kind].m_is_2, args[kind].sum_one,
                                      vols[v].shape.nz);
      cudaEvent_t ev_end = nullptr, ev3_end = nullptr;
      cudaEvent_t ev_beg = prof_begin(st, &ev_end);
      cudaEvent_t ev3_beg = k3 ? prof_begin(st, &ev3_end, IFCM_PROF_STENCIL3D) : nullptr;
      CU_TRY(launch_stencil(c, pl.np, rb->layout, args[kind], grid, st));
      if (ev3_beg) cudaEventRecord(ev3_end, st);
      if (ev_beg) cudaEventRecord(ev_end, st);
    } else {
      for (int v = 0; v < n; ++v) {
        const BatchVol& bv = vols[v];
        const ifcm_shape& s = bv.shape;
        const long long plane = static_cast<long long>(plane_elems(s));
        const int blocks = r.vol[v].n_rec;
        PlainArgs a{};
        a.nx = s.nx;
        a.ny = s.ny;
        a.nz = s.nz;
        a.pitch = s.pitch_x;
        a.x = bv.x;
        ShellArgs sh;
        fill_plain_method(a, sh, p);
        a.u_src = kind == 0 ? bv.u0 : (kind == 1 ? rb->ua[v] : rb->ub[v]);
        sh.src_pstride = kind == 0 ? 0 : c * plane;
        a.u_dst = kind == 1 ? rb->ub[v] : rb->ua[v];
        sh.dst_pstride = c * plane;
        a.lam_xi = bv.lam_xi;
        a.centres = rb->st.centres + static_cast<size_t>(rb->pbase[v]) * c;
        a.active = rb->st.active + rb->pbase[v];
        a.partials = rb->partials + static_cast<size_t>(rb->rec_base[v]) * (2 * c + 1);
        a.dmax = rb->dmax + rb->rec_base[v];
        a.n_records = rb->n_records - rb->rec_base[v];
        a.dst_elems = rb->buf_elems[v];
        a.stencil = 1;
        sh.P = bv.P;
        sh.n_rec = blocks;
        a.status = status;
        CU_TRY(launch_plain(c, a, sh, blocks, st));
      }
    }
    CU_TRY(launch_reduce(c, r, st));
    return IFCM_OK;
  }
};

// A batch whose every volume fits one CTA's shared memory (x, U^t and U^{t+1}),
// with FP32 memberships and the first neighbourhood shell, runs whole: one
// launch of one CTA per particle instead of two launches per iteration.
bool resident_eligible(const BatchVol* vols, int n, const ifcm_params* p) {
  if (!g_resident.load() || forced_np() > 0 || p->V != 1 || p->u_dtype != IFCM_U_FP32)
    return false;
  for (int v = 0; v < n; ++v) {
    const ifcm_shape& s = vols[v].shape;
    const long long nvox = static_cast<long long>(s.nx) * s.ny * s.nz;
    if (resident_smem_bytes(p->c, nvox) > kResidentSmemBytes) return false;
  }
  return true;
}

// The resident form of a batch (resident.cu): every particle's run (Alg 1
// step 4, reading R5) inside one launch; u_final (or NULL) receives particle
// 0's final memberships of volume 0 as FP32 [c][plane].
// stencil = false, max_iter >= 0: the FCM start instead (lambda = xi = 0, no
// neighbourhood terms, max_iter iterations at most).
ifcm_status run_resident(const BatchVol* vols, int n, const ifcm_params* p, RunBufs& rb,
                         DevStatus* status, float* u_final, cudaStream_t st,
                         bool stencil = true, int max_iter = -1) {
  const Trace tr("resident runs");
  ResidentArgs a{};
  a.n_vol = n;
  a.st = rb.st;
  a.dist_floor = static_cast<float>(p->dist_floor);
  a.m = static_cast<float>(p->m);
  a.inv_m1 = static_cast<float>(1.0 / (p->m - 1.0));
  a.m_is_2 = p->m == 2.0;
  a.max_iter = max_iter >= 0 ? max_iter : p->max_iter;
  a.eps = p->eps_u;
  a.reduce = p->reduce;
  a.stencil = stencil ? 1 : 0;
  a.status = status;
  int P_total = 0;
  long long max_nvox = 0;
  for (int v = 0; v < n; ++v) {
    const BatchVol& bv = vols[v];
    ResidentVol& rv = a.vol[v];
    rv.x = bv.x;
    rv.u0 = bv.u0;
    rv.c0 = bv.c0;
    rv.lam_xi = bv.lam_xi;
    rv.fitness = bv.fitness;
    rv.iters_out = bv.iters;
    rv.c_out = bv.c_out;
    rv.u_final = v == 0 ? u_final : nullptr;
    rv.nx = bv.shape.nx;
    rv.ny = bv.shape.ny;
    rv.nz = bv.shape.nz;
    rv.pitch = bv.shape.pitch_x;
    rv.P = bv.P;
    rv.pbase = P_total;
    P_total += bv.P;
    const long long nvox = static_cast<long long>(bv.shape.nx) * bv.shape.ny * bv.shape.nz;
    if (nvox > max_nvox) max_nvox = nvox;
  }
  CU_TRY(launch_resident(p->c, a, P_total, max_nvox, st));
  return IFCM_OK;
}

// IFCM runs of every particle of n volumes with the stencil kernel (the plain
// kernel for V > 1): one launch per iteration covers all volumes' work items.
// Batches of small volumes run resident instead (resident_eligible); then,
// when u_final is given, particle 0's final memberships of volume 0 go there
// and *u_written is set.
ifcm_status run_stencil_batch(const BatchVol* vols, int n, const ifcm_params* p, RunBufs& rb,
                              DevStatus* status, cudaStream_t st, float* u_final = nullptr,
                              bool* u_written = nullptr) {
  if (u_written) *u_written = false;
  if (resident_eligible(vols, n, p)) {
    ST_TRY(run_resident(vols, n, p, rb, status, u_final, st));
    if (u_written) *u_written = u_final != nullptr;
    return IFCM_OK;
  }
  BatchRun br;
  ST_TRY(br.prepare(vols, n, p, rb, status, p->max_iter, p->eps_u, st));
  for (int it = 0; it < p->max_iter; ++it) ST_TRY(br.iteration(it, st));
  return IFCM_OK;
}

// The runs of P particles of one volume from the shared start (u0, c0).
// start_eq2: u0 is a membership field from Eq 2 (e.g. the FCM start).
ifcm_status run_stencil(const float* x, const ifcm_shape& s, const ifcm_params* p,
                        const double* lam_xi, int P, const float* u0, const double* c0,
                        RunBufs& rb, double* fitness, int32_t* iters, double* c_out,
                        DevStatus* status, cudaStream_t st, bool start_eq2 = false,
                        float* u_final = nullptr, bool* u_written = nullptr) {
  BatchVol bv{x, s, P, lam_xi, u0, c0, fitness, iters, c_out, start_eq2};
  return run_stencil_batch(&bv, 1, p, rb, status, st, u_final, u_written);
}

// Method constants of a plain-kernel launch, and the shells with their Eq 10
// weights (one particle unless the caller sets more).
void fill_plain_method(PlainArgs& a, ShellArgs& sh, const ifcm_params* p) {
  a.dist_floor = static_cast<float>(p->dist_floor);
  a.m = static_cast<float>(p->m);
  a.inv_m1 = static_cast<float>(1.0 / (p->m - 1.0));
  a.m_is_2 = p->m == 2.0;
  a.vpt = kPlainVpt;
  sh = ShellArgs{};
  sh.P = 1;
  sh.V = p->V;
  double e[kMaxV], sum = 0.0;
  for (int r = 1; r <= p->V; ++r) sum += (e[r - 1] = std::exp(-r / (p->V > 1 ? p->h : 1.0)));
  for (int r = 1; r <= p->V; ++r) sh.W[r - 1] = static_cast<float>(e[r - 1] / sum);
}

// Particle 0's final memberships (P = 1 runs) as FP32 [c][plane].
ifcm_status copy_out(const RunBufs& rb, int c, size_t plane, float* u_out, cudaStream_t st) {
  if (rb.layout != UL_PLANAR)
    CU_TRY(launch_unpack_select(rb.ua[0], rb.ub[0], rb.st.iters, u_out, c, rb.np, rb.layout,
                                static_cast<long long>(plane), st));
  else
    CU_TRY(launch_select_copy(rb.ua[0], rb.ub[0], rb.st.iters, u_out,
                              static_cast<long long>(c) * plane, st));
  return IFCM_OK;
}

// One run with the plain kernel (P = 1).  host_check: read max|du| after
// every iteration and stop on the host (the paper's Algorithm 2 loop).
ifcm_status run_plain(const float* x, const ifcm_shape& s, const ifcm_params* p,
                      const double* lam_xi_dev, float lam, float xi, bool stencil,
                      const float* u_init, const double* c_init, int max_iter, RunBufs& rb,
                      int32_t* iters_out, double* c_out, double* J_out, DevStatus* status,
                      bool host_check, cudaStream_t st) {
  const int c = p->c;
  const long long nvox = static_cast<long long>(s.nx) * s.ny * s.nz;
  const int blocks = plain_blocks(nvox, kPlainVpt);
  CU_TRY(launch_run_init(c, 1, c_init, rb.st, nullptr, st));
  PlainArgs a{};
  a.nx = s.nx;
  a.ny = s.ny;
  a.nz = s.nz;
  a.pitch = s.pitch_x;
  a.x = x;
  a.lam_xi = lam_xi_dev;
  a.lam = lam;
  a.xi = xi;
  a.centres = rb.st.centres;
  a.active = rb.st.active;
  a.partials = rb.partials;
  a.dmax = rb.dmax;
  a.n_records = rb.n_records;
  a.dst_elems = rb.buf_elems[0];
  ShellArgs sh;
  fill_plain_method(a, sh, p);
  sh.n_rec = blocks;
  a.stencil = stencil ? 1 : 0;
  a.status = status;
  ReduceArgs r{};
  r.n_vol = 1;
  r.P_total = 1;
  r.partials = rb.partials;
  r.dmax = rb.dmax;
  r.n_records = rb.n_records;
  r.st = rb.st;
  r.max_iter = max_iter;
  r.eps = p->eps_u;
  r.status = status;
  r.vol[0].pbase = 0;
  r.vol[0].P = 1;
  r.vol[0].n_rec = blocks;
  r.vol[0].rec_base = 0;
  r.vol[0].nvox = nvox;
  r.vol[0].fitness = J_out;
  r.vol[0].iters_out = iters_out;
  r.vol[0].c_out = c_out;
  for (int it = 0; it < max_iter; ++it) {
    a.u_dst = (it % 2 == 0) ? rb.ua[0] : rb.ub[0];
    a.u_src = it == 0 ? u_init : ((it % 2 == 1) ? rb.ua[0] : rb.ub[0]);
    CU_TRY(launch_plain(c, a, sh, blocks, st));
    CU_TRY(launch_reduce(c, r, st));
    if (host_check) {
      int32_t act = 0;
      CU_TRY(cudaMemcpyAsync(&act, rb.st.active, sizeof(act), cudaMemcpyDeviceToHost, st));
      CU_TRY(cudaStreamSynchronize(st));
      if (!act) break;
    }
  }
  return IFCM_OK;
}

// ------------------------------------------------------------ pifcm3d layout
struct PifcmBufs {
  DevStatus* status;
  float* x;
  float* u0;
  double* c0;
  double* sw_x;
  double* sw_v;
  double* sw_pbx;
  double* sw_pbf;
  int32_t* sw_gen;
  double* fitness;
  int32_t* iters;
  double* lam_best;
  int32_t* best;
  int32_t* iters_init;
  int32_t* iters_final;
  double* J_final;
  double* c_final;
  double* J_init;
  unsigned long long* updates;
  NormBufs norm;
  RunBufs run;
};

ifcm_shape run_shape(const ifcm_shape& s, const pifcm_options* o) {
  ifcm_shape r = s;
  if (o->slice_z >= 0) r.nz = 1;
  return r;
}

PifcmBufs carve_pifcm(Carver& cv, const ifcm_shape& s, const ifcm_params* p,
                      const pifcm_options* o) {
  PifcmBufs b;
  const int c = p->c, P = o->P;
  const ifcm_shape rs = run_shape(s, o);
  b.status = carve_status(cv);
  b.x = cv.take<float>(plane_elems(s));
  b.u0 = cv.take<float>(static_cast<size_t>(c) * plane_elems(rs));
  b.c0 = cv.take<double>(c);
  b.sw_x = cv.take<double>(2 * P);
  b.sw_v = cv.take<double>(2 * P);
  b.sw_pbx = cv.take<double>(2 * P);
  b.sw_pbf = cv.take<double>(P);
  b.sw_gen = cv.take<int32_t>(1);
  b.fitness = cv.take<double>(P);
  b.iters = cv.take<int32_t>(P);
  b.lam_best = cv.take<double>(2);
  b.best = cv.take<int32_t>(1);
  b.iters_init = cv.take<int32_t>(1);
  b.iters_final = cv.take<int32_t>(1);
  b.J_final = cv.take<double>(1);
  b.c_final = cv.take<double>(c);
  b.J_init = cv.take<double>(1);
  b.updates = cv.take<unsigned long long>(1);
  b.norm = carve_norm(cv, s);
  b.run = carve_run(cv, rs, c, P, run_layout(p, P));
  return b;
}

ifcm_status check_options(const pifcm_options* o, const ifcm_shape& s) {
  if (!o) return fail(IFCM_ERR_INVALID, "options is NULL");
  if (o->P < 1 || o->P > kMaxP) return fail(IFCM_ERR_INVALID, "P = %d outside 1..%d", o->P, kMaxP);
  if (o->generations < 1) return fail(IFCM_ERR_INVALID, "generations must be >= 1");
  if (o->radius < 0) return fail(IFCM_ERR_INVALID, "radius must be >= 0");
  if (!(o->vmax > 0.0)) return fail(IFCM_ERR_INVALID, "vmax must be > 0");
  if (o->init_max_iter < 1) return fail(IFCM_ERR_INVALID, "init_max_iter must be >= 1");
  if (o->slice_z >= s.nz) return fail(IFCM_ERR_INVALID, "slice_z %d >= nz %d", o->slice_z, s.nz);
  if (o->fitness_mode != PIFCM_FITNESS_RESTART && o->fitness_mode != PIFCM_FITNESS_ONESTEP)
    return fail(IFCM_ERR_INVALID, "fitness_mode = %d: expected PIFCM_FITNESS_RESTART or "
                "PIFCM_FITNESS_ONESTEP", o->fitness_mode);
  return IFCM_OK;
}

}  // namespace

namespace pifcm {
// Sets the thread-local message ifcm_last_error() returns (for entry points
// defined in other translation units).
void set_error_message(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
}
}  // namespace pifcm

// ============================================================== C ABI
extern "C" {

const char* ifcm_status_string(ifcm_status s) {
  switch (s) {
    case IFCM_OK: return "ok";
    case IFCM_ERR_INVALID: return "invalid argument or input";
    case IFCM_ERR_NOMEM: return "workspace too small";
    case IFCM_ERR_CUDA: return "CUDA error";
    case IFCM_ERR_TIMEOUT: return "device wait timed out";
    case IFCM_ERR_BOUNDS: return "index out of bounds";
    case IFCM_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

const char* ifcm_last_error(void) { return g_msg; }

ifcm_status ifcm_device_status(const void* ws, void* stream) {
  if (!ws) return fail(IFCM_ERR_INVALID, "ws is NULL");
  DevStatus h{};
  CU_TRY(cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost,
                         static_cast<cudaStream_t>(stream)));
  CU_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  if (h.status != 0)
    return fail(static_cast<ifcm_status>(h.status), "device status %d (site %d)", h.status,
                h.where);
  return IFCM_OK;
}

// ---------------------------------------------------------- normalise
size_t ifcm_normalize_workspace_bytes(ifcm_shape shape) {
  Carver cv(nullptr);
  carve_status(cv);
  carve_norm(cv, shape);
  return cv.off + 256;
}

ifcm_status ifcm_normalize(const float* vol, float* x_out, ifcm_shape shape, void* ws,
                           size_t ws_bytes, void* stream) {
  ST_TRY(check_shape(shape));
  ST_TRY(check_aligned(vol, "vol"));
  ST_TRY(check_aligned(x_out, "x_out"));
  ST_TRY(check_aligned(ws, "ws"));
  if (ws_bytes < ifcm_normalize_workspace_bytes(shape))
    return fail(IFCM_ERR_NOMEM, "workspace %zu < %zu bytes", ws_bytes,
                ifcm_normalize_workspace_bytes(shape));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  DevStatus* status = carve_status(cv);
  NormBufs n = carve_norm(cv, shape);
  CU_TRY(cudaMemsetAsync(status, 0, sizeof(DevStatus), st));
  CU_TRY(launch_minmax(vol, shape.nx, shape.ny, shape.nz, shape.pitch_x, n.pmin, n.pmax, n.pbad,
                       n.nparts, st));
  CU_TRY(launch_scale(vol, x_out, shape.nx, shape.ny, shape.nz, shape.pitch_x, n.pmin, n.pmax,
                      n.pbad, n.nparts, status, st));
  return IFCM_OK;
}

// ----------------------------------------------------------- ifcm_fit
size_t ifcm_fit_workspace_bytes(ifcm_shape shape, const ifcm_params* p) {
  if (!p || p->c < 2 || p->c > kMaxC) return 0;
  Carver cv(nullptr);
  carve_status(cv);
  cv.take<float>(static_cast<size_t>(p->c) * plane_elems(shape));   // uniform start
  carve_run(cv, shape, p->c, 1, run_layout(p, 1));
  return cv.off + 256;
}

ifcm_status ifcm_fit(const float* x, ifcm_shape shape, const ifcm_params* p,
                     const double* lam_xi, const float* u_init, const double* c_init,
                     float* u_out, double* c_out, double* J_out, int32_t* iters_out, void* ws,
                     size_t ws_bytes, void* stream) {
  ST_TRY(check_shape(shape));
  ST_TRY(check_params(p));
  ST_TRY(check_extent(shape, p));
  ST_TRY(check_aligned(x, "x"));
  ST_TRY(check_aligned(ws, "ws"));
  if (!lam_xi) return fail(IFCM_ERR_INVALID, "lam_xi is NULL");
  if (u_init) ST_TRY(check_aligned(u_init, "u_init"));
  if (u_out) ST_TRY(check_aligned(u_out, "u_out"));
  const size_t need = ifcm_fit_workspace_bytes(shape, p);
  if (ws_bytes < need) return fail(IFCM_ERR_NOMEM, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  DevStatus* status = carve_status(cv);
  float* uni = cv.take<float>(static_cast<size_t>(p->c) * plane_elems(shape));
  RunBufs rb = carve_run(cv, shape, p->c, 1, run_layout(p, 1));
  CU_TRY(cudaMemsetAsync(status, 0, sizeof(DevStatus), st));
  CU_TRY(cudaMemsetAsync(rb.st.updates, 0, sizeof(unsigned long long), st));
  const float* start = u_init;
  if (!start) {
    CU_TRY(launch_fill(uni, 1.0f / p->c, static_cast<long long>(p->c) * plane_elems(shape), st));
    start = uni;
  }
  bool written = false;
  ST_TRY(run_stencil(x, shape, p, lam_xi, 1, start, c_init, rb, J_out, iters_out, c_out, status,
                     st, false, u_out, &written));
  if (u_out && !written) ST_TRY(copy_out(rb, p->c, plane_elems(shape), u_out, st));
  return IFCM_OK;
}

ifcm_status ifcm_fit_plain(const float* x, ifcm_shape shape, const ifcm_params* p, double lambda,
                           double xi, const float* u_init, const double* c_init, float* u_out,
                           double* c_out, double* J_out, int32_t* iters_out, void* ws,
                           size_t ws_bytes, void* stream) {
  ST_TRY(check_shape(shape));
  ST_TRY(check_params(p));
  if (p->u_dtype != IFCM_U_FP32)
    return fail(IFCM_ERR_UNSUPPORTED, "the plain form stores FP32 memberships only");
  ST_TRY(check_extent(shape, p));
  ST_TRY(check_aligned(x, "x"));
  ST_TRY(check_aligned(ws, "ws"));
  if (u_out) ST_TRY(check_aligned(u_out, "u_out"));
  const size_t need = ifcm_fit_workspace_bytes(shape, p);
  if (ws_bytes < need) return fail(IFCM_ERR_NOMEM, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  DevStatus* status = carve_status(cv);
  cv.take<float>(static_cast<size_t>(p->c) * plane_elems(shape));
  RunBufs rb = carve_run(cv, shape, p->c, 1, UL_PLANAR);
  CU_TRY(cudaMemsetAsync(status, 0, sizeof(DevStatus), st));
  CU_TRY(cudaMemsetAsync(rb.st.updates, 0, sizeof(unsigned long long), st));
  ST_TRY(run_plain(x, shape, p, nullptr, static_cast<float>(lambda), static_cast<float>(xi),
                   true, u_init, c_init, p->max_iter, rb, iters_out, c_out, J_out, status,
                   true, st));
  if (u_out)
    CU_TRY(launch_select_copy(rb.ua[0], rb.ub[0], rb.st.iters, u_out,
                              static_cast<long long>(p->c) * plane_elems(shape), st));
  return IFCM_OK;
}

// -------------------------------------------------- pso_fitness_batch
size_t pso_fitness_batch_workspace_bytes(ifcm_shape shape, const ifcm_params* p, int32_t P) {
  if (!p || p->c < 2 || p->c > kMaxC || P < 1) return 0;
  Carver cv(nullptr);
  carve_status(cv);
  carve_run(cv, shape, p->c, P, run_layout(p, P));
  return cv.off + 256;
}

ifcm_status pso_fitness_batch(const float* x, ifcm_shape shape, const ifcm_params* p,
                              const double* lam_xi, int32_t P, const float* u0,
                              const double* c0, double* fitness, int32_t* iters,
                              double* c_out, void* ws, size_t ws_bytes, void* stream) {
  ST_TRY(check_shape(shape));
  ST_TRY(check_params(p));
  ST_TRY(check_extent(shape, p));
  if (P < 1 || P > kMaxP) return fail(IFCM_ERR_INVALID, "P = %d outside 1..%d", P, kMaxP);
  ST_TRY(check_aligned(x, "x"));
  ST_TRY(check_aligned(u0, "u0"));
  ST_TRY(check_aligned(ws, "ws"));
  if (!lam_xi || !c0 || !fitness)
    return fail(IFCM_ERR_INVALID, "lam_xi, c0 and fitness must not be NULL");
  const size_t need = pso_fitness_batch_workspace_bytes(shape, p, P);
  if (ws_bytes < need) return fail(IFCM_ERR_NOMEM, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  DevStatus* status = carve_status(cv);
  RunBufs rb = carve_run(cv, shape, p->c, P, run_layout(p, P));
  CU_TRY(cudaMemsetAsync(status, 0, sizeof(DevStatus), st));
  CU_TRY(cudaMemsetAsync(rb.st.updates, 0, sizeof(unsigned long long), st));
  return run_stencil(x, shape, p, lam_xi, P, u0, c0, rb, fitness, iters, c_out, status, st);
}

}  // extern "C"

// ------------------------------------------------------- plan selection
extern "C" {

void ifcm_autotune_enable(int32_t mode) {
  std::lock_guard<std::mutex> lk(g_tune.mu);
  g_tune.mode = mode ? 1 : 0;
}

void ifcm_autotune_reset(void) {
  std::lock_guard<std::mutex> lk(g_tune.mu);
  g_tune.cache.clear();
}

ifcm_status ifcm_stencil_force_plan(int32_t np, int32_t chunks) {
  if (np == 0) {
    std::lock_guard<std::mutex> lk(g_tune.mu);
    g_tune.force = StencilPlan{0, 0};
    return IFCM_OK;
  }
  if ((np != 1 && np != 2) || chunks < 1)
    return fail(IFCM_ERR_INVALID, "forced plan np = %d, chunks = %d", np, chunks);
  std::lock_guard<std::mutex> lk(g_tune.mu);
  g_tune.force = StencilPlan{np, chunks};
  return IFCM_OK;
}

int32_t ifcm_stencil_plan(ifcm_shape shape, int32_t c, int32_t P, int32_t* np, int32_t* tz) {
  if (check_shape(shape) != IFCM_OK || c < 2 || c > kMaxC || P < 1) return -1;
  BatchVol bv{};
  bv.shape = shape;
  bv.P = P;
  StencilPlan pl = heuristic_plan(&bv, 1, c, UL_F32P);
  int32_t tuned = 0;
  {
    std::lock_guard<std::mutex> lk(g_tune.mu);
    auto it = g_tune.cache.find(plan_key(&bv, 1, c, IFCM_U_FP32));
    if (g_tune.force.np > 0 && stencil_np_supported(c, g_tune.force.np)) {
      pl = g_tune.force;
    } else if (it != g_tune.cache.end()) {
      pl = it->second;
      tuned = 1;
    }
  }
  if (P < 2 && forced_np() == 0) pl.np = 1;
  if (np) *np = pl.np;
  if (tz) *tz = tiling(shape, pl.chunks).tz;
  return tuned;
}

}  // extern "C"

// -------------------------------------------------- pso_fitness_multi
namespace {

// Multi-volume batches: the layout depends on the parameters only (a wave's
// particle count changes while waves are packed).
int multi_layout(const ifcm_params* p) { return run_layout(p, 2); }

size_t wave_bytes(const ifcm_batch_volume* vols, const int* idx, int n, int c, int layout) {
  ifcm_shape shapes[kMaxVols];
  int P[kMaxVols];
  for (int i = 0; i < n; ++i) {
    shapes[i] = vols[idx[i]].shape;
    P[i] = vols[idx[i]].P;
  }
  Carver cv(nullptr);
  carve_status(cv);
  carve_runs(cv, shapes, P, n, c, layout);
  return cv.off + 256;
}

ifcm_status check_multi(const ifcm_batch_volume* vols, int32_t n, const ifcm_params* p) {
  if (!vols || n < 1) return fail(IFCM_ERR_INVALID, "need at least one volume");
  if (!p) return fail(IFCM_ERR_INVALID, "params is NULL");
  for (int i = 0; i < n; ++i) {
    const ifcm_batch_volume& v = vols[i];
    ifcm_params pv = *p;
    pv.c = v.c;
    ST_TRY(check_shape(v.shape));
    ST_TRY(check_params(&pv));
    ST_TRY(check_extent(v.shape, &pv));
    ST_TRY(check_aligned(v.x, "volume x"));
    ST_TRY(check_aligned(v.u0, "volume u0"));
    if (v.P < 1 || v.P > kMaxBatchParticles)
      return fail(IFCM_ERR_INVALID, "volume %d: P = %d outside 1..%d", i, v.P, kMaxBatchParticles);
    if (!v.lam_xi || !v.c0 || !v.fitness)
      return fail(IFCM_ERR_INVALID, "volume %d: lam_xi, c0 and fitness must not be NULL", i);
  }
  return IFCM_OK;
}

// Volumes in the wave that starts at g[b]: as many as fit one launch
// (kMaxVols volumes, kMaxBatchParticles particles) and ws_bytes.
int wave_size(const ifcm_batch_volume* vols, const std::vector<int>& g, size_t b, int c,
              int layout, size_t ws_bytes) {
  int cnt = 0, parts = 0;
  while (b + cnt < g.size() && cnt < kMaxVols &&
         parts + vols[g[b + cnt]].P <= kMaxBatchParticles &&
         wave_bytes(vols, g.data() + b, cnt + 1, c, layout) <= ws_bytes)
    parts += vols[g[b + cnt++]].P;
  return cnt;
}

// Volumes of cluster count c, in input order.
std::vector<int> group_of(const ifcm_batch_volume* vols, int n, int c) {
  std::vector<int> g;
  for (int i = 0; i < n; ++i)
    if (vols[i].c == c) g.push_back(i);
  return g;
}

}  // namespace

extern "C" {

size_t pso_fitness_multi_workspace_bytes(const ifcm_batch_volume* vols, int32_t n,
                                         const ifcm_params* p) {
  if (check_multi(vols, n, p) != IFCM_OK) return 0;
  size_t need = 0;
  for (int c = 2; c <= kMaxC; ++c) {
    const std::vector<int> g = group_of(vols, n, c);
    // whole group, in launch-sized pieces
    for (size_t b = 0; b < g.size();) {
      const int cnt = wave_size(vols, g, b, c, multi_layout(p), static_cast<size_t>(-1));
      const size_t w = wave_bytes(vols, g.data() + b, cnt, c, multi_layout(p));
      if (w > need) need = w;
      b += cnt;
    }
  }
  return need;
}

size_t pso_fitness_multi_min_workspace_bytes(const ifcm_batch_volume* vols, int32_t n,
                                             const ifcm_params* p) {
  if (check_multi(vols, n, p) != IFCM_OK) return 0;
  size_t need = 0;
  for (int i = 0; i < n; ++i) {
    const size_t w = wave_bytes(vols, &i, 1, vols[i].c, multi_layout(p));
    if (w > need) need = w;
  }
  return need;
}

int32_t pso_fitness_multi_waves(const ifcm_batch_volume* vols, int32_t n, const ifcm_params* p,
                                size_t ws_bytes) {
  if (check_multi(vols, n, p) != IFCM_OK) return -1;
  if (ws_bytes < pso_fitness_multi_min_workspace_bytes(vols, n, p)) return -1;
  int32_t waves = 0;
  for (int c = 2; c <= kMaxC; ++c) {
    const std::vector<int> g = group_of(vols, n, c);
    for (size_t b = 0; b < g.size(); ++waves)
      b += wave_size(vols, g, b, c, multi_layout(p), ws_bytes);
  }
  return waves;
}

ifcm_status pso_fitness_multi(const ifcm_batch_volume* vols, int32_t n, const ifcm_params* p,
                              void* ws, size_t ws_bytes, void* stream) {
  ST_TRY(check_multi(vols, n, p));
  ST_TRY(check_aligned(ws, "ws"));
  const size_t min_need = pso_fitness_multi_min_workspace_bytes(vols, n, p);
  if (ws_bytes < min_need)
    return fail(IFCM_ERR_NOMEM, "workspace %zu < %zu bytes (the largest volume alone)",
                ws_bytes, min_need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    // one status word for the whole call: a later wave must not clear an
    // earlier wave's error
    Carver cv(ws);
    CU_TRY(cudaMemsetAsync(carve_status(cv), 0, sizeof(DevStatus), st));
  }
  for (int c = 2; c <= kMaxC; ++c) {
    const std::vector<int> g = group_of(vols, n, c);
    ifcm_params pc = *p;
    pc.c = c;
    for (size_t b = 0; b < g.size();) {
      const int cnt = wave_size(vols, g, b, c, multi_layout(p), ws_bytes);
      std::vector<BatchVol> bv(cnt);
      ifcm_shape shapes[kMaxVols];
      int P[kMaxVols];
      for (int i = 0; i < cnt; ++i) {
        const ifcm_batch_volume& v = vols[g[b + i]];
        bv[i] = BatchVol{v.x, v.shape, v.P, v.lam_xi, v.u0, v.c0, v.fitness, v.iters, nullptr};
        shapes[i] = v.shape;
        P[i] = v.P;
      }
      Carver cv(ws);
      DevStatus* status = carve_status(cv);
      RunBufs rb = carve_runs(cv, shapes, P, cnt, c, multi_layout(p));
      CU_TRY(cudaMemsetAsync(rb.st.updates, 0, sizeof(unsigned long long), st));
      ST_TRY(run_stencil_batch(bv.data(), cnt, &pc, rb, status, st));
      b += cnt;
    }
  }
  return IFCM_OK;
}

}  // extern "C"

// ------------------------------------------------------------ CUDA graphs
struct ifcm_graph_t {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

namespace {

// Captures body(stream) on a private stream into an instantiated graph.
template <class Body>
ifcm_status capture_graph(Body body, ifcm_graph* out) {
  cudaStream_t cs = nullptr;
  CU_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return fail(IFCM_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
  }
  const ifcm_status rc = body(cs);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (rc != IFCM_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != IFCM_OK ? rc : fail(IFCM_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(IFCM_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
  }
  *out = new ifcm_graph_t{g, ex};
  return IFCM_OK;
}

}  // namespace

extern "C" {

ifcm_status pso_fitness_multi_graph(const ifcm_batch_volume* vols, int32_t n,
                                    const ifcm_params* p, void* ws, size_t ws_bytes,
                                    ifcm_graph* out) {
  if (!out) return fail(IFCM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  ST_TRY(check_multi(vols, n, p));
  return capture_graph(
      [&](cudaStream_t cs) { return pso_fitness_multi(vols, n, p, ws, ws_bytes, cs); }, out);
}

ifcm_status ifcm_graph_launch(ifcm_graph g, void* stream) {
  if (!g) return fail(IFCM_ERR_INVALID, "graph is NULL");
  CU_TRY(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
  return IFCM_OK;
}

void ifcm_graph_destroy(ifcm_graph g) {
  if (!g) return;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
}

// ------------------------------------------------------------- swarm
static ifcm_status check_swarm(const pso_state* s) {
  if (!s) return fail(IFCM_ERR_INVALID, "swarm is NULL");
  if (s->P < 1 || s->P > kMaxP) return fail(IFCM_ERR_INVALID, "P = %d outside 1..%d", s->P, kMaxP);
  if (s->radius < 0) return fail(IFCM_ERR_INVALID, "radius must be >= 0");
  if (!(s->vmax > 0.0)) return fail(IFCM_ERR_INVALID, "vmax must be > 0");
  if (!s->x || !s->v || !s->pbest_x || !s->pbest_f || !s->gen)
    return fail(IFCM_ERR_INVALID, "swarm arrays must not be NULL");
  return IFCM_OK;
}

ifcm_status pso_init(const pso_state* s, void* stream) {
  ST_TRY(check_swarm(s));
  CU_TRY(launch_pso_init(*s, static_cast<cudaStream_t>(stream)));
  return IFCM_OK;
}

ifcm_status pso_step(const pso_state* s, const double* fitness, void* stream) {
  ST_TRY(check_swarm(s));
  if (!fitness) return fail(IFCM_ERR_INVALID, "fitness is NULL");
  CU_TRY(launch_pso_step(*s, fitness, static_cast<cudaStream_t>(stream)));
  return IFCM_OK;
}

// ------------------------------------------------------------ pifcm3d
size_t pifcm3d_workspace_bytes(ifcm_shape shape, const ifcm_params* p, const pifcm_options* o) {
  if (!p || !o || p->c < 2 || p->c > kMaxC || o->P < 1) return 0;
  Carver cv(nullptr);
  carve_pifcm(cv, shape, p, o);
  return cv.off + 256;
}

ifcm_status pifcm3d(const float* vol, ifcm_shape shape, const ifcm_params* p,
                    const pifcm_options* o, float* u_out, pifcm_result* result, void* ws,
                    size_t ws_bytes, void* stream) {
  const Trace trace_run("pifcm3d");
  ST_TRY(check_shape(shape));
  ST_TRY(check_params(p));
  ST_TRY(check_extent(shape, p));
  ST_TRY(check_options(o, shape));
  ST_TRY(check_aligned(vol, "vol"));
  ST_TRY(check_aligned(ws, "ws"));
  if (u_out) ST_TRY(check_aligned(u_out, "u_out"));
  if (!result) return fail(IFCM_ERR_INVALID, "result is NULL");
  const size_t need = pifcm3d_workspace_bytes(shape, p, o);
  if (ws_bytes < need) return fail(IFCM_ERR_NOMEM, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int c = p->c, P = o->P;
  Carver cv(ws);
  PifcmBufs b = carve_pifcm(cv, shape, p, o);
  const ifcm_shape rs = run_shape(shape, o);
  const size_t rpl = plane_elems(rs);

  CU_TRY(cudaMemsetAsync(b.status, 0, sizeof(DevStatus), st));
  CU_TRY(cudaMemsetAsync(b.updates, 0, sizeof(unsigned long long), st));
  // Algorithm 2 step 1: normalise over the whole volume, then (Alg 1 step 1) slice.
  CU_TRY(launch_minmax(vol, shape.nx, shape.ny, shape.nz, shape.pitch_x, b.norm.pmin,
                       b.norm.pmax, b.norm.pbad, b.norm.nparts, st));
  CU_TRY(launch_scale(vol, b.x, shape.nx, shape.ny, shape.nz, shape.pitch_x, b.norm.pmin,
                      b.norm.pmax, b.norm.pbad, b.norm.nparts, b.status, st));
  const float* xr =
      o->slice_z >= 0 ? b.x + static_cast<size_t>(o->slice_z) * shape.ny * shape.pitch_x : b.x;

  RunBufs rb = b.run;
  rb.st.updates = b.updates;
  // Algorithm 1 step 2: FCM start (lambda = xi = 0) from u = 1/c, c_j = (j+1/2)/c;
  // one resident launch when the (sliced) volume fits a CTA's shared memory.
  {
    const Trace tr("fcm start");
    const long long nvox = static_cast<long long>(rs.nx) * rs.ny * rs.nz;
    if (g_resident.load() && resident_smem_bytes(c, nvox) <= kResidentSmemBytes) {
      BatchVol sv{xr, rs, 1, nullptr, nullptr, nullptr, b.J_init, b.iters_init, b.c0};
      ST_TRY(run_resident(&sv, 1, p, rb, b.status, b.u0, st, false, o->init_max_iter));
    } else {
      ST_TRY(run_plain(xr, rs, p, nullptr, 0.0f, 0.0f, false, nullptr, nullptr,
                       o->init_max_iter, rb, b.iters_init, b.c0, b.J_init, b.status, false, st));
      CU_TRY(launch_select_copy(rb.ua[0], rb.ub[0], rb.st.iters, b.u0,
                                static_cast<long long>(c) * rpl, st));
    }
  }

  // Algorithm 1 steps 3-9.
  pso_state sw{};
  sw.P = P;
  sw.radius = o->radius;
  sw.vmax = o->vmax;
  sw.seed = o->seed;
  sw.x = b.sw_x;
  sw.v = b.sw_v;
  sw.pbest_x = b.sw_pbx;
  sw.pbest_f = b.sw_pbf;
  sw.gen = b.sw_gen;
  CU_TRY(launch_pso_init(sw, st));
  if (o->fitness_mode == PIFCM_FITNESS_ONESTEP) {
    // each particle's (U, C) persists: generation g is iteration g of its run
    BatchVol bv{xr, rs, P, sw.x, b.u0, b.c0, b.fitness, b.iters, nullptr, true};
    BatchRun br;
    ST_TRY(br.prepare(&bv, 1, p, rb, b.status, o->generations, 0.0, st));
    for (int g = 0; g < o->generations; ++g) {
      const Trace tr("generation %d", g);
      ST_TRY(br.iteration(g, st));
      CU_TRY(launch_pso_step(sw, b.fitness, st));
    }
  } else {
    for (int g = 0; g < o->generations; ++g) {
      const Trace tr("generation %d", g);
      ST_TRY(run_stencil(xr, rs, p, sw.x, P, b.u0, b.c0, rb, b.fitness, b.iters, nullptr,
                         b.status, st, true));
      CU_TRY(launch_pso_step(sw, b.fitness, st));
    }
  }
  // Algorithm 1 step 11: final IFCM at the best personal best.
  const Trace tr("final run");
  CU_TRY(launch_pso_best(sw.pbest_x, sw.pbest_f, P, b.lam_best, b.best, st));
  bool written = false;
  ST_TRY(run_stencil(xr, rs, p, b.lam_best, 1, b.u0, b.c0, rb, b.J_final, b.iters_final,
                     b.c_final, b.status, st, true, u_out, &written));
  if (u_out && !written) ST_TRY(copy_out(rb, c, rpl, u_out, st));
  CU_TRY(launch_result(c, b.c_final, b.lam_best, b.J_final, sw.pbest_f, P, b.iters_final,
                       b.iters_init, b.updates, b.best, b.status, result, st));
  return IFCM_OK;
}

ifcm_status pifcm3d_graph(const float* vol, ifcm_shape shape, const ifcm_params* p,
                          const pifcm_options* o, float* u_out, pifcm_result* result, void* ws,
                          size_t ws_bytes, ifcm_graph* out) {
  if (!out) return fail(IFCM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  return capture_graph(
      [&](cudaStream_t cs) {
        return pifcm3d(vol, shape, p, o, u_out, result, ws, ws_bytes, cs);
      },
      out);
}

size_t pifcm3d_host_workspace_bytes(ifcm_shape shape, const ifcm_params* p,
                                    const pifcm_options* o) {
  if (!p || !o || p->c < 2 || p->c > kMaxC || o->P < 1) return 0;
  Carver cv(nullptr);
  cv.take<float>(plane_elems(shape));
  cv.take<float>(static_cast<size_t>(p->c) * plane_elems(run_shape(shape, o)));
  cv.take<pifcm_result>(1);
  cv.take<unsigned char>(pifcm3d_workspace_bytes(shape, p, o));
  return cv.off + 256;
}

ifcm_status pifcm3d_host(const float* vol_host, ifcm_shape shape, const ifcm_params* p,
                         const pifcm_options* o, float* u_out_host, pifcm_result* result_host,
                         void* ws, size_t ws_bytes, void* stream) {
  ST_TRY(check_shape(shape));
  ST_TRY(check_params(p));
  ST_TRY(check_extent(shape, p));
  ST_TRY(check_options(o, shape));
  ST_TRY(check_aligned(ws, "ws"));
  if (!vol_host || !result_host) return fail(IFCM_ERR_INVALID, "vol_host / result_host is NULL");
  const size_t need = pifcm3d_host_workspace_bytes(shape, p, o);
  if (ws_bytes < need) return fail(IFCM_ERR_NOMEM, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  const size_t upl = static_cast<size_t>(p->c) * plane_elems(run_shape(shape, o));
  float* vol = cv.take<float>(plane_elems(shape));
  float* u = cv.take<float>(upl);
  pifcm_result* res = cv.take<pifcm_result>(1);
  const size_t inner = pifcm3d_workspace_bytes(shape, p, o);
  void* iws = cv.take<unsigned char>(inner);
  CU_TRY(cudaMemcpyAsync(vol, vol_host, plane_elems(shape) * sizeof(float),
                         cudaMemcpyHostToDevice, st));
  ST_TRY(pifcm3d(vol, shape, p, o, u_out_host ? u : nullptr, res, iws, inner, stream));
  if (u_out_host)
    CU_TRY(cudaMemcpyAsync(u_out_host, u, upl * sizeof(float), cudaMemcpyDeviceToHost, st));
  CU_TRY(cudaMemcpyAsync(result_host, res, sizeof(pifcm_result), cudaMemcpyDeviceToHost, st));
  CU_TRY(cudaStreamSynchronize(st));
  if (result_host->status != 0)
    return fail(static_cast<ifcm_status>(result_host->status), "device status %d",
                result_host->status);
  return IFCM_OK;
}

void ifcm_set_wait_limit_ns(uint64_t ns) { g_wait_ns.store(ns); }

void ifcm_resident_enable(int32_t mode) { g_resident.store(mode ? 1 : 0); }

// ------------------------------------------------------------ profiling
void ifcm_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.on = on != 0;
}

ifcm_status ifcm_profile_read_kind(int32_t kind, double* kernel_ms, int64_t* launches) {
  if (kind < 0 || kind > 3) return fail(IFCM_ERR_INVALID, "profile kind %d outside 0..3", kind);
  std::lock_guard<std::mutex> lk(g_prof.mu);
  double total = 0.0;
  auto& used = g_prof.used[kind];
  for (auto& ev : used) {
    CU_TRY(cudaEventSynchronize(ev.second));
    float ms = 0.0f;
    CU_TRY(cudaEventElapsedTime(&ms, ev.first, ev.second));
    total += ms;
    g_prof.spare.push_back(ev);
  }
  if (kernel_ms) *kernel_ms = total;
  if (launches) *launches = static_cast<int64_t>(used.size());
  used.clear();
  return IFCM_OK;
}

ifcm_status ifcm_profile_read(double* kernel_ms, int64_t* launches) {
  return ifcm_profile_read_kind(IFCM_PROF_STENCIL, kernel_ms, launches);
}

}  // extern "C"

// ------------------------------------------------------- differentiation
namespace {

// Plan of a launch without timing: a forced plan, the tuning cache, else the rule.
StencilPlan peek_plan(const BatchVol* vols, int n, const ifcm_params* p) {
  std::lock_guard<std::mutex> lk(g_tune.mu);
  if (g_tune.force.np > 0 && stencil_np_supported(p->c, g_tune.force.np)) return g_tune.force;
  auto it = g_tune.cache.find(plan_key(vols, n, p->c, p->u_dtype));
  if (it != g_tune.cache.end()) return it->second;
  return heuristic_plan(vols, n, p->c, is_bf16(p) ? UL_BF16 : UL_PLANAR);
}

// Scratch of a gradient evaluation: the run state of one particle, the
// checkpoints U^1 .. U^K, the trace of C^{t+1}, S0^{t+1}, J^t, and the reverse
// pass's coefficient planes, adjoint ping-pong and partial sums.
struct GradBufs {
  DevStatus* status;
  RunBufs run;
  float* ckpt;          // [K][c][plane]
  double* trace;        // [K][2c+1]
  float* A;             // [c][plane]
  float* B;             // [c][plane]
  float* e;             // [plane]
  float* ubar[2];       // [c][plane] each
  double* partials;     // [blocks][2+c]
  double* cbar;         // [c]
  double* best;         // polish: lambda*, xi*, J*
  double* grad;         // polish: gradient at the current point
  double* J;            // polish: J at the current point
};

GradBufs carve_grad(Carver& cv, const ifcm_shape& s, int c, int K) {
  GradBufs g;
  const size_t pl = plane_elems(s);
  const long long nvox = static_cast<long long>(s.nx) * s.ny * s.nz;
  g.status = carve_status(cv);
  g.run = carve_run(cv, s, c, 1, UL_PLANAR);
  g.ckpt = cv.take<float>(static_cast<size_t>(K) * c * pl);
  g.trace = cv.take<double>(static_cast<size_t>(K) * (2 * c + 1));
  g.A = cv.take<float>(static_cast<size_t>(c) * pl);
  g.B = cv.take<float>(static_cast<size_t>(c) * pl);
  g.e = cv.take<float>(pl);
  g.ubar[0] = cv.take<float>(static_cast<size_t>(c) * pl);
  g.ubar[1] = cv.take<float>(static_cast<size_t>(c) * pl);
  g.partials = cv.take<double>(static_cast<size_t>(adjoint_blocks(s.nx, s.ny, s.nz)) * (2 + c));
  g.cbar = cv.take<double>(c);
  g.best = cv.take<double>(3);
  g.grad = cv.take<double>(2);
  g.J = cv.take<double>(1);
  return g;
}

// K iterations of one run from (u0, c0) with the stencil kernel: U^{t+1} into
// checkpoint t, C^{t+1}, S0^{t+1}, J^t into the trace, J^{K-1} into J_out.
ifcm_status grad_forward(const float* x, const ifcm_shape& s, const ifcm_params* p, int K,
                         const double* lam_xi, const float* u0, const double* c0, GradBufs& g,
                         double* J_out, cudaStream_t st) {
  const int c = p->c;
  const size_t pl = plane_elems(s);
  ifcm_params pk = *p;
  pk.max_iter = K;
  pk.eps_u = 0.0;
  RunBufs& rb = g.run;
  CU_TRY(launch_run_init(c, 1, c0, rb.st, nullptr, st));
  BatchVol bv{x, s, 1, lam_xi, u0, c0, J_out, nullptr, nullptr};
  const StencilPlan plan = peek_plan(&bv, 1, &pk);
  rb.np = plan.np;
  ReduceArgs r{};
  r.n_vol = 1;
  r.P_total = 1;
  r.partials = rb.partials;
  r.dmax = rb.dmax;
  r.n_records = rb.n_records;
  r.st = rb.st;
  r.max_iter = K;
  r.eps = 0.0;
  r.reduce = p->reduce;
  r.status = g.status;
  r.vol[0].P = 1;
  r.vol[0].n_rec = tiling(s, plan.chunks).n_tiles;
  r.vol[0].rec_base = rb.rec_base[0];
  r.vol[0].nvox = static_cast<long long>(s.nx) * s.ny * s.nz;
  r.vol[0].fitness = J_out;
  r.vol[0].trace = g.trace;
  std::vector<StencilArgs> args(1);
  const int grid = plan_grid(c, rb.layout, plan, plan_items(&bv, 1, plan));
  for (int t = 0; t < K; ++t) {
    bv.u0 = t == 0 ? u0 : g.ckpt + static_cast<size_t>(t - 1) * c * pl;
    rb.ua[0] = g.ckpt + static_cast<size_t>(t) * c * pl;
    ST_TRY(build_args(args[0], &bv, 1, &pk, rb, plan, 0, g.status));
    cudaEvent_t ev_end = nullptr;
    cudaEvent_t ev_beg = prof_begin(st, &ev_end);
    CU_TRY(launch_stencil(c, plan.np, rb.layout, args[0], grid, st));
    if (ev_beg) cudaEventRecord(ev_end, st);
    CU_TRY(launch_reduce(c, r, st));
  }
  return IFCM_OK;
}

// Reverse pass over the K iterations grad_forward recorded: grad = (dJ/dlambda,
// dJ/dxi) of J^{K-1}.
ifcm_status grad_reverse(const float* x, const ifcm_shape& s, const ifcm_params* p, int K,
                         const double* lam_xi, const float* u0, const double* c0, GradBufs& g,
                         double* grad, cudaStream_t st) {
  const int c = p->c;
  const size_t pl = plane_elems(s);
  const long long nvox = static_cast<long long>(s.nx) * s.ny * s.nz;
  const int blocks = adjoint_blocks(s.nx, s.ny, s.nz);
  const size_t tw = 2 * c + 1;
  CU_TRY(cudaMemsetAsync(grad, 0, 2 * sizeof(double), st));
  AdjointArgs a{};
  a.nx = s.nx;
  a.ny = s.ny;
  a.nz = s.nz;
  a.pitch = s.pitch_x;
  a.x = x;
  a.lam_xi = lam_xi;
  a.A = g.A;
  a.B = g.B;
  a.e = g.e;
  a.partials = g.partials;
  a.dist_floor = static_cast<float>(p->dist_floor);
  a.m = static_cast<float>(p->m);
  a.inv_m1 = static_cast<float>(1.0 / (p->m - 1.0));
  a.m_is_2 = p->m == 2.0;
  for (int t = K - 1; t >= 0; --t) {
    a.u = t == 0 ? u0 : g.ckpt + static_cast<size_t>(t - 1) * c * pl;
    a.ubar_next = t == K - 1 ? nullptr : g.ubar[(t + 1) & 1];
    a.c_t = t == 0 ? c0 : g.trace + static_cast<size_t>(t - 1) * tw;
    a.c_next = g.trace + static_cast<size_t>(t) * tw;
    a.s0_next = a.c_next + c;
    a.cbar_next = t == K - 1 ? nullptr : g.cbar;
    a.J_bar = t == K - 1 ? 1.0f : 0.0f;
    a.ubar_out = g.ubar[t & 1];
    cudaEvent_t ev_end = nullptr;
    cudaEvent_t ev_beg = prof_begin(st, &ev_end, IFCM_PROF_ADJOINT_POINT);
    CU_TRY(launch_adjoint_point(c, a, blocks, st));
    if (ev_beg) cudaEventRecord(ev_end, st);
    CU_TRY(launch_adjoint_reduce(c, g.partials, blocks, grad, g.cbar, st));
    if (t > 0) {
      ev_beg = prof_begin(st, &ev_end, IFCM_PROF_ADJOINT_GATHER);
      CU_TRY(launch_adjoint_gather(c, a, st));
      if (ev_beg) cudaEventRecord(ev_end, st);
    }
  }
  return IFCM_OK;
}

ifcm_status check_grad(const float* x, const ifcm_shape& shape, const ifcm_params* p, int K,
                       const double* lam_xi, const float* u0, const double* c0, const void* ws) {
  ST_TRY(check_shape(shape));
  ST_TRY(check_params(p));
  if (p->u_dtype != IFCM_U_FP32)
    return fail(IFCM_ERR_UNSUPPORTED, "gradients are built for FP32 memberships only");
  ST_TRY(check_extent(shape, p));
  if (K < 1) return fail(IFCM_ERR_INVALID, "K = %d must be >= 1", K);
  ST_TRY(check_aligned(x, "x"));
  ST_TRY(check_aligned(u0, "u0"));
  ST_TRY(check_aligned(ws, "ws"));
  if (!lam_xi || !c0) return fail(IFCM_ERR_INVALID, "lam_xi and c0 must not be NULL");
  return IFCM_OK;
}

}  // namespace

extern "C" {

size_t ifcm_grad_workspace_bytes(ifcm_shape shape, const ifcm_params* p, int32_t K) {
  if (!p || p->c < 2 || p->c > kMaxC || K < 1) return 0;
  Carver cv(nullptr);
  carve_grad(cv, shape, p->c, K);
  return cv.off + 256;
}

ifcm_status ifcm_grad(const float* x, ifcm_shape shape, const ifcm_params* p, int32_t K,
                      const double* lam_xi, const float* u0, const double* c0, double* J_out,
                      double* grad_out, void* ws, size_t ws_bytes, void* stream) {
  ST_TRY(check_grad(x, shape, p, K, lam_xi, u0, c0, ws));
  if (!grad_out) return fail(IFCM_ERR_INVALID, "grad_out is NULL");
  const size_t need = ifcm_grad_workspace_bytes(shape, p, K);
  if (ws_bytes < need) return fail(IFCM_ERR_NOMEM, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  GradBufs g = carve_grad(cv, shape, p->c, K);
  CU_TRY(cudaMemsetAsync(g.status, 0, sizeof(DevStatus), st));
  CU_TRY(cudaMemsetAsync(g.run.st.updates, 0, sizeof(unsigned long long), st));
  ST_TRY(grad_forward(x, shape, p, K, lam_xi, u0, c0, g, J_out ? J_out : g.J, st));
  ST_TRY(grad_reverse(x, shape, p, K, lam_xi, u0, c0, g, grad_out, st));
  return IFCM_OK;
}

ifcm_status ifcm_polish(const float* x, ifcm_shape shape, const ifcm_params* p, int32_t K,
                        int32_t steps, double step0, double decay, double* lam_xi,
                        const float* u0, const double* c0, double* J_out, void* ws,
                        size_t ws_bytes, void* stream) {
  ST_TRY(check_grad(x, shape, p, K, lam_xi, u0, c0, ws));
  if (steps < 0) return fail(IFCM_ERR_INVALID, "steps = %d must be >= 0", steps);
  if (!(step0 > 0.0) || !(decay > 0.0) || !(decay <= 1.0))
    return fail(IFCM_ERR_INVALID, "step0 must be > 0 and decay in (0, 1]");
  const size_t need = ifcm_grad_workspace_bytes(shape, p, K);
  if (ws_bytes < need) return fail(IFCM_ERR_NOMEM, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  GradBufs g = carve_grad(cv, shape, p->c, K);
  CU_TRY(cudaMemsetAsync(g.status, 0, sizeof(DevStatus), st));
  CU_TRY(cudaMemsetAsync(g.run.st.updates, 0, sizeof(unsigned long long), st));
  CU_TRY(launch_polish_step(lam_xi, g.grad, g.J, g.best, 0.0, 0, st));
  double alpha = step0;
  for (int k = 0; k < steps; ++k, alpha *= decay) {
    ST_TRY(grad_forward(x, shape, p, K, lam_xi, u0, c0, g, g.J, st));
    ST_TRY(grad_reverse(x, shape, p, K, lam_xi, u0, c0, g, g.grad, st));
    CU_TRY(launch_polish_step(lam_xi, g.grad, g.J, g.best, alpha, 1, st));
  }
  ST_TRY(grad_forward(x, shape, p, K, lam_xi, u0, c0, g, g.J, st));
  CU_TRY(launch_polish_step(lam_xi, g.grad, g.J, g.best, 0.0, 2, st));
  if (J_out)
    CU_TRY(cudaMemcpyAsync(J_out, g.best + 2, sizeof(double), cudaMemcpyDeviceToDevice, st));
  return IFCM_OK;
}

}  // extern "C"
