// lbm_core.cu -- 2D grid path of the MRT-FD D2V16 scheme: the launches of the
// step kernels (lbm_step_kernels.cuh; two steps per launch: lbm_fused.cu),
// the auxiliary kernels (initial state, moments, audit, Dirichlet ghosts,
// status, repitch) and the C ABI declared in include/lbm.h.
//
// Data layout in HBM: populations are structure-of-arrays,
//   f[i][y][x] at offset i * plane + y * pitch + x,
// pitch = nx rounded up to 32 elements (rows start on 128-byte (FP32) or
// 256-byte (FP64) boundaries), plane = ny * pitch. There is no ghost ring in
// memory: the step computes boundary ghosts on the fly from the time-n
// interior (or reads the fixed Dirichlet ghosts), so one launch per step
// carries the whole update. Two buffers alternate (time n -> n+1).
//
// One step (one launch of k_step) per node:
//   load the node's 16 populations -> 4-point group transforms -> conserved
//   moments -> Eq. 14 equilibria -> relaxation folded into the back-map (Eq. 3)
//   -> f(1 - cx^2 - cy^2) + collision -> Lax-Wendroff neighbour terms of
//   Eq. A.1b (12 x-neighbours, 12 y-neighbours, ghosts at the domain edge)
//   -> store; epilogue: watchdog flags and, every audit_every steps, block
//   partial sums of (rho, j, e) in FP64 with a fixed-order final pass done by
//   the last block to finish (no floating-point atomics).
#include "lbm_step.cuh"
#include "lbm_step_kernels.cuh"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>  // header-only; ranges cost nothing without a profiler attached

#include <climits>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

using namespace lbmk;

namespace {

constexpr int GRAPH_CHUNK = 64;  // steps per captured graph (even)

// ---------------------------------------------------------------------------
// Initial state, moments out, standalone audit, Dirichlet ghosts
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_init(R* __restrict__ f, const double* __restrict__ rho,
                       const double* __restrict__ u, const double* __restrict__ v,
                       const double* __restrict__ T, const Coeffs<double> K,
                       int nx, int ny, long long pitch, long long plane) {
  const int x = blockIdx.x * AUX_X + threadIdx.x;
  const int y = blockIdx.y * AUX_Y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const long long k = (long long)y * nx + x;
  const double r = rho[k], uu = u[k], vv = v[k];
  double g[16];
  feq(K, r, r * uu, r * vv, r * T[k] + 0.5 * r * (uu * uu + vv * vv), g);
  const long long c = (long long)y * pitch + x;
#pragma unroll
  for (int i = 0; i < 16; ++i) f[i * plane + c] = (R)g[i];
}

template <typename R>
__global__ void k_moments(const R* __restrict__ f, double* rho, double* u,
                          double* v, double* T, int nx, int ny, long long pitch,
                          long long plane, const Coeffs<double> K) {
  const int x = blockIdx.x * AUX_X + threadIdx.x;
  const int y = blockIdx.y * AUX_Y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const long long c = (long long)y * pitch + x;
  double g[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) g[i] = (double)f[i * plane + c];
  Groups<double> d;
  transform(g, d);
  const Cons<double> m = conserved(K, d);
  const double r = 1.0 / m.rho;
  const double uu = m.jx * r, vv = m.jy * r;
  const long long k = (long long)y * nx + x;
  if (rho) rho[k] = m.rho;
  if (u) u[k] = uu;
  if (v) v[k] = vv;
  if (T) T[k] = m.e * r - 0.5 * (uu * uu + vv * vv);
}

template <typename R>
__global__ void __launch_bounds__(AUX_N) k_audit(const R* __restrict__ f, int nx,
                                                 int ny, long long pitch,
                                                 long long plane, double area,
                                                 DevStatus* st, double* partial,
                                                 const Coeffs<double> K) {
  __shared__ double sm[AUX_N / 4][4];
  __shared__ int s_last;
  const int x = blockIdx.x * AUX_X + threadIdx.x;
  const int y = blockIdx.y * AUX_Y + threadIdx.y;
  const int t = threadIdx.y * AUX_X + threadIdx.x;
  double tot[4] = {0.0, 0.0, 0.0, 0.0};
  if (x < nx && y < ny) {
    const long long c = (long long)y * pitch + x;
    double g[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = (double)f[i * plane + c];
    Groups<double> d;
    transform(g, d);
    const Cons<double> m = conserved(K, d);
    tot[0] = m.rho; tot[1] = m.jx; tot[2] = m.jy; tot[3] = m.e;
  }
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  const double bs = block_sum4<AUX_N>(tot, sm);
  if (t < 4) partial[4 * bid + t] = bs;
  __syncthreads();
  if (t == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&st->arrive_audit, 1u);
    s_last = (prev == (unsigned)nblocks - 1);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    const double tot4 = final_sum4<AUX_N>(partial, nblocks, sm);
    if (t < 4) st->audit_now[t] = tot4 * area;
    if (t == 0) st->arrive_audit = 0;
  }
}

// Dirichlet ghost populations; g3 (LBM_DF64, else NULL) gets the third word
// of each one's double-word split.
template <typename R>
__global__ void k_ghost_eq(R* g, const Coeffs<double> K, const double* states, float* g3) {
  const int side = threadIdx.x;
  if (side >= 4) return;
  const double r = states[4 * side], u = states[4 * side + 1],
               v = states[4 * side + 2], T = states[4 * side + 3];
  double out[16];
  feq(K, r, r * u, r * v, r * T + 0.5 * r * (u * u + v * v), out);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    g[16 * side + i] = (R)out[i];
    if (g3) g3[16 * side + i] = third_word(out[i]);
  }
}

// ---------------------------------------------------------------------------
// Host-side constants
// ---------------------------------------------------------------------------
// Dense M of Eqs. 5a-5p on the velocities of Eq. 4 (row n = moment n + 1,
// column i = velocity i + 1) and its inverse by Gauss-Jordan elimination with
// partial pivoting in long double; used by the tensor-core step.
bool dense_moment_matrices(double (&M)[16][16], double (&Minv)[16][16]) {
  for (int i = 0; i < 16; ++i) {
    const double x = vel_x(i), y = vel_y(i), q = x * x + y * y;
    const double r[16] = {1.0, x, y, q / 2, x * x - y * y, x * y, x * q / 2, y * q / 2,
                          x * (x * x - 3 * y * y), y * (3 * x * x - y * y), q * q / 4,
                          x * x * x * x - 6 * x * x * y * y + y * y * y * y, q * (x * x - y * y),
                          q * x * y, x * (x * x - 3 * y * y) * q, y * (3 * x * x - y * y) * q};
    for (int n = 0; n < 16; ++n) M[n][i] = r[n];
  }
  long double a[16][32];
  for (int i = 0; i < 16; ++i)
    for (int j = 0; j < 32; ++j) a[i][j] = j < 16 ? (long double)M[i][j] : (long double)(j - 16 == i);
  for (int col = 0; col < 16; ++col) {
    int p = col;
    for (int r = col + 1; r < 16; ++r)
      if (fabsl(a[r][col]) > fabsl(a[p][col])) p = r;
    if (a[p][col] == 0.0L) return false;
    for (int j = 0; j < 32; ++j) { const long double t = a[col][j]; a[col][j] = a[p][j]; a[p][j] = t; }
    const long double piv = a[col][col];
    for (int j = 0; j < 32; ++j) a[col][j] /= piv;
    for (int r = 0; r < 16; ++r) {
      if (r == col || a[r][col] == 0.0L) continue;
      const long double fac = a[r][col];
      for (int j = 0; j < 32; ++j) a[r][j] -= fac * a[col][j];
    }
  }
  for (int i = 0; i < 16; ++i)
    for (int j = 0; j < 16; ++j) Minv[i][j] = (double)a[i][16 + j];
  return true;
}

bool build_coeffs(const lbm_config& cfg, Coeffs<double>& K) {
  if (!lattice_constants(K)) return false;
  set_rates(K, cfg.dt, cfg.s);
  set_advection(K, cfg.dt, cfg.dx, cfg.dy);
  return true;
}

template <typename R>
Coeffs<R> cast_coeffs(const Coeffs<double>& K) {
  Coeffs<R> o;
  const double* s = reinterpret_cast<const double*>(&K);
  R* d = reinterpret_cast<R*>(&o);
  for (size_t k = 0; k < sizeof(Coeffs<double>) / sizeof(double); ++k) d[k] = (R)s[k];
  return o;
}

thread_local std::string g_create_error = "no error";

}  // namespace

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct lbm_ctx {
  lbm_config cfg;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int esize = 8;
  long long pitch = 0, plane = 0;
  void* f[2] = {nullptr, nullptr};
  int cur = 0;
  void* geq = nullptr;
  DevStatus* st = nullptr;
  double* partial = nullptr;
  double* gpartial = nullptr;     // audit group sums (audit_block_done)
  unsigned* gcount = nullptr;     // audit group counters
  int ngroups = 0;
  int agroup = 0;                 // tiles per audit group
  double* staging = nullptr;
  void* pstage = nullptr;  // contiguous populations for host transfers (on first use)
  int nblocks = 0;      // blocks of one step launch
  int ntiles = 0, tiles_x = 0;  // node tiles of the grid
  int sms = 0;          // multiprocessors of the device
  dim3 grid, aux_grid;  // step grid; init / moments / audit grid
  bool wide = false;    // 64-bit element offsets needed
  Coeffs<double> Kd;
  CUtensorMap tmap[2];        // TMA descriptors of the two population buffers
  bool tc = false;            // tensor-core transforms (LBM_TC_TF32X3)
  bool dwp = false;           // double-word populations and arithmetic (LBM_DF64)
  bool dwmom = false;         // FP32 step, double-word moments (LBM_FP32_DWMOM)
  unsigned char* tc_b = nullptr;  // TF32 parts of M and M^-1 (16 KB)
  TcWeights tc_w = {};           // -dt s_k, 0 for the conserved k
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int fuse = 1;                   // time steps per FP32 launch (1 or 2)
  CUtensorMap tmap2[2];           // two-step kernel: tile + two-row halo
  cudaGraphExec_t graph2[2] = {nullptr, nullptr};  // GRAPH_CHUNK steps, two per launch
  std::string err = "no error";
};

namespace {

int fail(lbm_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg; else g_create_error = msg;
  return code;
}

int cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(c, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, m);
}

#define CK(ctx, call)                                       \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

// Third words of the double-word split of every constant (LBM_DF64).
Coeffs<float> third_words(const Coeffs<double>& K) {
  Coeffs<float> o;
  const double* s = reinterpret_cast<const double*>(&K);
  float* d = reinterpret_cast<float*>(&o);
  for (size_t k = 0; k < sizeof(Coeffs<double>) / sizeof(double); ++k) d[k] = third_word(s[k]);
  return o;
}

template <typename R>
StepArgs<R> make_args(lbm_ctx* c, int slot) {
  StepArgs<R> A;
  A.K = cast_coeffs<R>(c->Kd);
  if (std::is_same<R, dw>::value) A.K3 = third_words(c->Kd);
  else memset(&A.K3, 0, sizeof(A.K3));
  A.nx = c->cfg.nx;
  A.ny = c->cfg.ny;
  A.pitch = c->pitch;
  A.plane = c->plane;
  A.hx = (R)c->cfg.dx;
  A.hy = (R)c->cfg.dy;
  A.dtr = (R)c->cfg.dt;
  for (int s = 0; s < 4; ++s) {
    A.bc[s] = c->cfg.bc[s].kind;
    A.split[s] = c->cfg.bc[s].split;
    A.far[s] = c->cfg.bc[s].far_kind;
    A.s0[s] = (R)c->cfg.bc[s].split0;
    A.s1[s] = (R)c->cfg.bc[s].split_rate;
    A.wall[s][0] = (R)c->cfg.bc[s].u;
    A.wall[s][1] = (R)c->cfg.bc[s].v;
    A.wall[s][2] = (R)c->cfg.bc[s].T;
  }
  A.geq = (const R*)c->geq;
  A.geq3 = c->dwp ? (const float*)((const dw*)c->geq + 64) : nullptr;
  A.st = c->st;
  A.partial = c->partial;
  A.gpartial = c->gpartial;
  A.gcount = c->gcount;
  A.ngroups = c->ngroups;
  A.agroup = c->agroup;
  A.audit_every = c->cfg.audit_every;
  A.nblocks = c->nblocks;
  A.ntiles = c->ntiles;
  A.tiles_x = c->tiles_x;
  A.area = c->cfg.dx * c->cfg.dy;
  A.slot = slot;
  return A;
}

template <typename R, int VAR = 0>
int launch_persistent(lbm_ctx* c, cudaStream_t s, int from, void* fout, const StepArgs<R>& A) {
  const dim3 blk(Shape<R>::X, Shape<R>::TY);
  const R* fi = (const R*)c->f[from];
  const CUtensorMap& tm = c->tmap[from];
  if (A.nblocks >= A.ntiles) {
    if (c->wide) k_step<R, long long, VAR><<<A.ntiles, blk, 0, s>>>(tm, fi, (R*)fout, A);
    else k_step<R, unsigned, VAR><<<A.ntiles, blk, 0, s>>>(tm, fi, (R*)fout, A);
  } else {
    const size_t smem = pipe_smem_bytes<R>();
    if (c->wide) k_step_pipe<R, long long, VAR><<<A.nblocks, blk, smem, s>>>(tm, fi, (R*)fout, A);
    else k_step_pipe<R, unsigned, VAR><<<A.nblocks, blk, smem, s>>>(tm, fi, (R*)fout, A);
  }
  CK(c, cudaGetLastError());
  return LBM_OK;
}

int launch_step(lbm_ctx* c, cudaStream_t s, int from) {
  const int to = 1 - from;
  if (c->tc) {
    CK(c, tc_launch(c->tmap[from], (const float*)c->f[from], (float*)c->f[to],
                    make_args<float>(c, from), c->tc_b, c->tc_w, c->grid, s));
    return LBM_OK;
  }
  if (c->dwp) return launch_persistent<dw>(c, s, from, c->f[to], make_args<dw>(c, from));
  if (c->dwmom) return launch_persistent<float, 1>(c, s, from, c->f[to], make_args<float>(c, from));
  if (c->esize == 8) return launch_persistent<double>(c, s, from, c->f[to], make_args<double>(c, from));
  return launch_persistent<float>(c, s, from, c->f[to], make_args<float>(c, from));
}

// Blocks of a step launch when none were chosen: one per tile (k_step).
int default_blocks(const lbm_ctx* c) { return c->ntiles; }

template <typename R, int VAR = 0>
cudaError_t allow_pipe_smem() {
  const int b = (int)pipe_smem_bytes<R>();
  cudaError_t e = cudaFuncSetAttribute(k_step_pipe<R, unsigned, VAR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step_pipe<R, long long, VAR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  return e;
}

int ensure_graph(lbm_ctx* c, int from) {
  if (c->graph[from]) return LBM_OK;
  cudaGraph_t g;
  CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  int f = from, rc = LBM_OK;
  for (int k = 0; k < GRAPH_CHUNK && rc == LBM_OK; ++k) {
    rc = launch_step(c, c->stream, f);
    f = 1 - f;
  }
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (rc != LBM_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&c->graph[from], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  return LBM_OK;
}

// Two time steps in one launch (FP32, one block per tile).
int launch_fused(lbm_ctx* c, cudaStream_t s, int from) {
  StepArgs<float> A = make_args<float>(c, from);
  A.nblocks = c->ntiles;
  CK(c, fused_launch(c->tmap2[from], (const float*)c->f[from], (float*)c->f[1 - from], A, c->wide, s));
  return LBM_OK;
}

int ensure_graph2(lbm_ctx* c, int from) {
  if (c->graph2[from]) return LBM_OK;
  cudaGraph_t g;
  CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  int f = from, rc = LBM_OK;
  for (int k = 0; k < GRAPH_CHUNK / 2 && rc == LBM_OK; ++k) {
    rc = launch_fused(c, c->stream, f);
    f = 1 - f;
  }
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (rc != LBM_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&c->graph2[from], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  return LBM_OK;
}
static_assert(GRAPH_CHUNK % 4 == 0, "graphs of fused launches leave the buffer parity unchanged");

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Tensor map of population buffer b: dims (pitch, ny, 16), box = one tile
// with its halo (`rows` rows, Tile<R>::BXP columns, 16 populations).
int encode_map(lbm_ctx* c, int b, cuuint32_t rows, CUtensorMap* out) {
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return fail(c, LBM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const bool dbl = c->esize == 8;  // FP64 or double-word (8-byte elements)
  const cuuint64_t dims[3] = {(cuuint64_t)c->pitch, (cuuint64_t)c->cfg.ny, 16};
  const cuuint64_t strides[2] = {(cuuint64_t)c->pitch * c->esize, (cuuint64_t)c->plane * c->esize};
  const cuuint32_t bxp = c->dwp ? Tile<dw>::BXP : (dbl ? Tile<double>::BXP : Tile<float>::BXP);
  const cuuint32_t box[3] = {bxp, rows, 16};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(out, dbl ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                         3, c->f[b], dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, LBM_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return LBM_OK;
}

// The step kernels' maps of buffer b (and, for FP32, the two-step kernel's).
int encode_tile_map(lbm_ctx* c, int b) {
  const bool dbl = c->esize == 8;
  const cuuint32_t rows = c->tc ? (cuuint32_t)(TC_Y + 2)
                    : (cuuint32_t)(c->dwp ? Tile<dw>::ROWS
                                          : (dbl ? Tile<double>::ROWS : Tile<float>::ROWS));
  int rc = encode_map(c, b, rows, &c->tmap[b]);
  if (rc == LBM_OK && !dbl && !c->tc)
    rc = encode_map(c, b, (cuuint32_t)fused_halo_rows(), &c->tmap2[b]);
  return rc;
}

// Resets the status block for time level `step` in slot `cur` (a kernel, so
// that a restart needs no host round trip).
__global__ void k_reset_status(DevStatus* st, int cur, unsigned long long step, int phase) {
  constexpr int WORDS = (int)(offsetof(DevStatus, audit_totals) / sizeof(unsigned long long));
  static_assert(offsetof(DevStatus, audit_totals) % sizeof(unsigned long long) == 0, "prefix");
  unsigned long long* w = reinterpret_cast<unsigned long long*>(st);
  for (int i = threadIdx.x; i < WORDS; i += blockDim.x) w[i] = 0ull;
  __syncthreads();
  if (threadIdx.x == 0) {
    st->step[cur] = step;
    st->audit_phase[cur] = phase;
    st->first_bad = NONE;
    st->first_negT = NONE;
  }
}

int reset_status(lbm_ctx* c, unsigned long long step) {
  const int phase =
      c->cfg.audit_every > 0 ? (int)(step % (unsigned long long)c->cfg.audit_every) : 0;
  k_reset_status<<<1, 64, 0, c->stream>>>(c->st, c->cur, step, phase);
  CK(c, cudaGetLastError());
  CK(c, cudaMemsetAsync(c->gcount, 0, sizeof(unsigned) * c->ngroups, c->stream));
  return LBM_OK;
}

// Copies `rows` rows of nx elements between row pitches sp and dp (elements).
template <typename T>
__global__ void k_repitch(const T* __restrict__ src, long long sp, T* __restrict__ dst,
                          long long dp, int nx, long long rows) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  for (long long r = blockIdx.y; r < rows; r += gridDim.y) dst[r * dp + x] = src[r * sp + x];
}

int repitch(lbm_ctx* c, const void* src, long long sp, void* dst, long long dp) {
  const long long rows = 16ll * c->cfg.ny;
  const dim3 grid((c->cfg.nx + 255) / 256, (unsigned)std::min(rows, 65535ll));
  if (c->esize == 8)
    k_repitch<double><<<grid, 256, 0, c->stream>>>((const double*)src, sp, (double*)dst, dp,
                                                   c->cfg.nx, rows);
  else
    k_repitch<float><<<grid, 256, 0, c->stream>>>((const float*)src, sp, (float*)dst, dp,
                                                  c->cfg.nx, rows);
  CK(c, cudaGetLastError());
  return LBM_OK;
}

// Device buffer for one contiguous copy of the populations (host transfers).
int population_stage(lbm_ctx* c) {
  if (!c->pstage)
    CK(c, cudaMalloc(&c->pstage, (size_t)16 * c->cfg.nx * c->cfg.ny * c->esize));
  return LBM_OK;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

extern "C" {

int lbm_create(const lbm_config* cfg, void* cuda_stream, lbm_ctx** out) {
  if (!out) return fail(nullptr, LBM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, LBM_ERR_INVALID, "cfg is NULL");
  const lbm_config& C = *cfg;
  if (C.nx < 1 || C.ny < 1) return fail(nullptr, LBM_ERR_INVALID, "nx and ny must be >= 1");
  if ((long long)C.nx * C.ny > (1ll << 31))
    return fail(nullptr, LBM_ERR_INVALID, "grid too large");
  if (!finite_pos(C.dx) || !finite_pos(C.dy) || !finite_pos(C.dt))
    return fail(nullptr, LBM_ERR_INVALID, "dx, dy, dt must be finite and > 0");
  for (int k = 0; k < 16; ++k)
    if (!std::isfinite(C.s[k]) || C.s[k] < 0.0)
      return fail(nullptr, LBM_ERR_INVALID, "relaxation rates must be finite and >= 0");
  if (6.0 * C.dt / C.dx > 1.0 || 6.0 * C.dt / C.dy > 1.0)
    return fail(nullptr, LBM_ERR_INVALID, "Courant number 6 dt / dx exceeds 1");
  if (C.internal_dof != 0)
    return fail(nullptr, LBM_ERR_UNSUPPORTED,
                "internal_dof != 0: the D2V16 moment set fixes gamma = 2");
  if (C.precision != LBM_FP64 && C.precision != LBM_FP32 && C.precision != LBM_TC_TF32X3 &&
      C.precision != LBM_DF64 && C.precision != LBM_FP32_DWMOM)
    return fail(nullptr, LBM_ERR_UNSUPPORTED, "precision not built for the 2D grid path");
  if (C.audit_every < 0) return fail(nullptr, LBM_ERR_INVALID, "audit_every < 0");
  for (int s = 0; s < 4; ++s) {
    const lbm_bc& b = C.bc[s];
    if (b.kind < LBM_BC_PERIODIC || b.kind > LBM_BC_OUTFLOW)
      return fail(nullptr, LBM_ERR_INVALID, "bad boundary kind");
    if (b.split != 0 && b.split != 1) return fail(nullptr, LBM_ERR_INVALID, "split must be 0 or 1");
    if (b.split && (b.far_kind <= LBM_BC_PERIODIC || b.far_kind > LBM_BC_OUTFLOW ||
                    b.kind == LBM_BC_PERIODIC || !std::isfinite(b.split0) ||
                    !std::isfinite(b.split_rate)))
      return fail(nullptr, LBM_ERR_INVALID,
                  "a split side needs two non-periodic kinds and a finite split position");
    const bool eq = b.kind == LBM_BC_EQ || (b.split && b.far_kind == LBM_BC_EQ);
    const bool wall = b.kind == LBM_BC_WALL || (b.split && b.far_kind == LBM_BC_WALL);
    if (eq && !(finite_pos(b.rho) && finite_pos(b.T) && std::isfinite(b.u) && std::isfinite(b.v)))
      return fail(nullptr, LBM_ERR_INVALID, "Dirichlet state needs rho > 0, T > 0");
    if (wall && !(finite_pos(b.T) && std::isfinite(b.u) && std::isfinite(b.v)))
      return fail(nullptr, LBM_ERR_INVALID, "wall state needs T > 0");
  }
  if ((C.bc[0].kind == LBM_BC_PERIODIC) != (C.bc[1].kind == LBM_BC_PERIODIC) ||
      (C.bc[2].kind == LBM_BC_PERIODIC) != (C.bc[3].kind == LBM_BC_PERIODIC))
    return fail(nullptr, LBM_ERR_INVALID, "periodic must be set on both opposite sides");
  if (C.precision == LBM_TC_TF32X3 && 16ll * (((long long)C.nx + 31) / 32 * 32) * C.ny >= (1ll << 32))
    return fail(nullptr, LBM_ERR_UNSUPPORTED,
                "tensor-core step: 16 x pitch x ny must stay below 2^32 elements");

  lbm_ctx* c = new lbm_ctx();
  c->cfg = C;
  c->esize = (C.precision == LBM_FP64 || C.precision == LBM_DF64) ? 8 : 4;
  c->tc = C.precision == LBM_TC_TF32X3;
  c->dwp = C.precision == LBM_DF64;
  c->dwmom = C.precision == LBM_FP32_DWMOM;
  if (!build_coeffs(C, c->Kd)) {
    delete c;
    return fail(nullptr, LBM_ERR_INVALID, "singular moment block");
  }
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreate(&c->stream);  // blocking: ordered with the default stream
    c->own_stream = true;
  }
  c->pitch = ((long long)C.nx + 31) / 32 * 32;
  c->plane = c->pitch * C.ny;
  const int bx = c->tc ? TC_X : (c->dwp ? Shape<dw>::X : (c->esize == 8 ? Shape<double>::X : Shape<float>::X));
  const int by = c->tc ? TC_Y : (c->dwp ? Shape<dw>::Y : (c->esize == 8 ? Shape<double>::Y : Shape<float>::Y));
  c->tiles_x = (C.nx + bx - 1) / bx;
  c->ntiles = c->tiles_x * ((C.ny + by - 1) / by);
  c->aux_grid = dim3((C.nx + AUX_X - 1) / AUX_X, (C.ny + AUX_Y - 1) / AUX_Y);
  c->wide = 16ll * c->plane >= (1ll << 32);
  {
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (c->tc) {  // persistent CTAs, each taking every G-th tile
    c->nblocks = std::max(1, std::min(c->ntiles, TC_CTAS_PER_SM * std::max(1, c->sms)));
    c->grid = dim3(c->nblocks);
    if (e == cudaSuccess) e = tc_prepare();
  } else {
    c->nblocks = default_blocks(c);
    c->grid = dim3(c->nblocks);
    if (e == cudaSuccess)
      e = c->dwp ? allow_pipe_smem<dw>()
                 : c->dwmom ? allow_pipe_smem<float, 1>()
                            : (c->esize == 8 ? allow_pipe_smem<double>() : allow_pipe_smem<float>());
    if (e == cudaSuccess && c->esize == 4) e = fused_prepare();
  }
  const int npartial = std::max(c->ntiles, (int)(c->aux_grid.x * c->aux_grid.y));
  const size_t fbytes = (size_t)16 * c->plane * c->esize;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&c->f[b], fbytes);
  // Dirichlet ghosts: 64 elements (LBM_DF64: then 64 third words)
  if (e == cudaSuccess) e = cudaMalloc(&c->geq, 64 * c->esize + (c->dwp ? 64 * sizeof(float) : 0));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->st, sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->partial, sizeof(double) * 4 * npartial);
  c->agroup = (c->esize == 8 && !c->dwp) ? AUDIT_GROUP_FP64 : AUDIT_GROUP_REDUCED;
  c->ngroups = audit_groups(c->ntiles, c->agroup);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->gpartial, sizeof(double) * 4 * c->ngroups);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->gcount, sizeof(unsigned) * c->ngroups);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->gcount, 0, sizeof(unsigned) * c->ngroups, c->stream);
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&c->staging, sizeof(double) * 4 * (size_t)C.nx * C.ny);
  if (e == cudaSuccess && c->tc) {
    double M[16][16], Minv[16][16];
    unsigned char bconst[4][4096];
    if (!dense_moment_matrices(M, Minv)) {
      lbm_destroy(c);
      return fail(nullptr, LBM_ERR_INVALID, "singular moment matrix");
    }
    tc_prepare_constants(M, Minv, bconst);
    float w[16];
    for (int k = 0; k < 16; ++k) w[k] = k < 4 ? 0.f : (float)(-C.dt * C.s[k]);
    e = cudaMalloc((void**)&c->tc_b, sizeof(bconst));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->tc_b, bconst, sizeof(bconst), cudaMemcpyHostToDevice, c->stream);
    memcpy(c->tc_w.w, w, sizeof(w));
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMemsetAsync(c->f[b], 0, fbytes, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->st, 0, sizeof(DevStatus), c->stream);
  if (e == cudaSuccess) {
    double states[16];
    double* dstates = nullptr;
    for (int s = 0; s < 4; ++s) {
      const bool eq = C.bc[s].kind == LBM_BC_EQ || (C.bc[s].split && C.bc[s].far_kind == LBM_BC_EQ);
      states[4 * s] = eq ? C.bc[s].rho : 1.0;
      states[4 * s + 1] = eq ? C.bc[s].u : 0.0;
      states[4 * s + 2] = eq ? C.bc[s].v : 0.0;
      states[4 * s + 3] = eq ? C.bc[s].T : 1.0;
    }
    e = cudaMalloc((void**)&dstates, sizeof(states));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dstates, states, sizeof(states), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
      if (c->dwp)
        k_ghost_eq<dw><<<1, 32, 0, c->stream>>>((dw*)c->geq, c->Kd, dstates,
                                                (float*)((dw*)c->geq + 64));
      else if (c->esize == 8)
        k_ghost_eq<double><<<1, 32, 0, c->stream>>>((double*)c->geq, c->Kd, dstates, nullptr);
      else
        k_ghost_eq<float><<<1, 32, 0, c->stream>>>((float*)c->geq, c->Kd, dstates, nullptr);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (dstates) cudaFree(dstates);
  }
  if (e != cudaSuccess) {
    const int rc = cuda_fail(nullptr, e, "lbm_create");
    lbm_destroy(c);
    return rc;
  }
  if (encode_tile_map(c, 0) != LBM_OK || encode_tile_map(c, 1) != LBM_OK ||
      reset_status(c, 0) != LBM_OK) {
    g_create_error = c->err;
    lbm_destroy(c);
    return LBM_ERR_CUDA;
  }
  *out = c;
  return LBM_OK;
}

int lbm_set_init(lbm_ctx* c, const double* rho, const double* u, const double* v,
                 const double* T, int on_device) {
  if (!c) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
  if (!rho || !u || !v || !T) return fail(c, LBM_ERR_INVALID, "NULL field");
  const size_t n = (size_t)c->cfg.nx * c->cfg.ny;
  const double* p[4] = {rho, u, v, T};
  if (!on_device) {
    for (int k = 0; k < 4; ++k) {
      CK(c, cudaMemcpyAsync(c->staging + k * n, p[k], n * sizeof(double),
                            cudaMemcpyHostToDevice, c->stream));
      p[k] = c->staging + k * n;
    }
  }
  const dim3 blk(AUX_X, AUX_Y);
  c->cur = 0;
  if (c->dwp)
    k_init<dw><<<c->aux_grid, blk, 0, c->stream>>>((dw*)c->f[0], p[0], p[1], p[2], p[3], c->Kd,
                                                c->cfg.nx, c->cfg.ny, c->pitch, c->plane);
  else if (c->esize == 8)
    k_init<double><<<c->aux_grid, blk, 0, c->stream>>>((double*)c->f[0], p[0], p[1], p[2], p[3],
                                                    c->Kd, c->cfg.nx, c->cfg.ny, c->pitch, c->plane);
  else
    k_init<float><<<c->aux_grid, blk, 0, c->stream>>>((float*)c->f[0], p[0], p[1], p[2], p[3],
                                                   c->Kd, c->cfg.nx, c->cfg.ny, c->pitch, c->plane);
  CK(c, cudaGetLastError());
  const int rc = reset_status(c, 0);
  if (rc == LBM_OK && !on_device) CK(c, cudaStreamSynchronize(c->stream));  // host fields free again
  return rc;
}

namespace {
// Profiler range around one lbm_step call ("lbm_step n=<steps>").
struct StepRange {
  explicit StepRange(long long n) {
    char name[48];
    snprintf(name, sizeof(name), "lbm_step n=%lld", n);
    nvtxRangePushA(name);
  }
  ~StepRange() { nvtxRangePop(); }
};
}  // namespace

int lbm_step(lbm_ctx* c, long long nsteps) {
  if (!c) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
  if (nsteps < 0) return fail(c, LBM_ERR_INVALID, "nsteps < 0");
  const StepRange range(nsteps);
  if (c->fuse == 2 && c->cfg.audit_every != 1) {
    while (nsteps >= GRAPH_CHUNK) {
      int rc = ensure_graph2(c, c->cur);
      if (rc != LBM_OK) return rc;
      CK(c, cudaGraphLaunch(c->graph2[c->cur], c->stream));
      nsteps -= GRAPH_CHUNK;
    }
    for (; nsteps >= 2; nsteps -= 2) {
      int rc = launch_fused(c, c->stream, c->cur);
      if (rc != LBM_OK) return rc;
      c->cur = 1 - c->cur;
    }
  }
  while (nsteps >= GRAPH_CHUNK) {
    int rc = ensure_graph(c, c->cur);
    if (rc != LBM_OK) return rc;
    CK(c, cudaGraphLaunch(c->graph[c->cur], c->stream));
    nsteps -= GRAPH_CHUNK;
  }
  for (; nsteps > 0; --nsteps) {
    int rc = launch_step(c, c->stream, c->cur);
    if (rc != LBM_OK) return rc;
    c->cur = 1 - c->cur;
  }
  return LBM_OK;
}

int lbm_moments(lbm_ctx* c, double* rho, double* u, double* v, double* T, int on_device) {
  if (!c) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
  const size_t n = (size_t)c->cfg.nx * c->cfg.ny;
  double* d[4] = {rho, u, v, T};
  double* h[4] = {rho, u, v, T};
  if (!on_device)
    for (int k = 0; k < 4; ++k) d[k] = h[k] ? c->staging + k * n : nullptr;
  const dim3 blk(AUX_X, AUX_Y);
  if (c->dwp)
    k_moments<dw><<<c->aux_grid, blk, 0, c->stream>>>((const dw*)c->f[c->cur], d[0], d[1], d[2],
                                                   d[3], c->cfg.nx, c->cfg.ny, c->pitch,
                                                   c->plane, c->Kd);
  else if (c->esize == 8)
    k_moments<double><<<c->aux_grid, blk, 0, c->stream>>>((const double*)c->f[c->cur], d[0], d[1],
                                                       d[2], d[3], c->cfg.nx, c->cfg.ny,
                                                       c->pitch, c->plane, c->Kd);
  else
    k_moments<float><<<c->aux_grid, blk, 0, c->stream>>>((const float*)c->f[c->cur], d[0], d[1],
                                                      d[2], d[3], c->cfg.nx, c->cfg.ny,
                                                      c->pitch, c->plane, c->Kd);
  CK(c, cudaGetLastError());
  if (!on_device) {
    // Four host fields that are consecutive blocks of one array come back in
    // one copy (the staging blocks are consecutive too).
    const bool one = h[0] && h[1] == h[0] + n && h[2] == h[1] + n && h[3] == h[2] + n;
    if (one) {
      CK(c, cudaMemcpyAsync(h[0], d[0], 4 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    } else {
      for (int k = 0; k < 4; ++k)
        if (h[k])
          CK(c, cudaMemcpyAsync(h[k], d[k], n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}

int lbm_destroy(lbm_ctx* c) {
  if (!c) return LBM_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (int k = 0; k < 2; ++k) {
    if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
    if (c->graph2[k]) cudaGraphExecDestroy(c->graph2[k]);
    if (c->f[k]) cudaFree(c->f[k]);
  }
  if (c->geq) cudaFree(c->geq);
  if (c->st) cudaFree(c->st);
  if (c->partial) cudaFree(c->partial);
  if (c->gpartial) cudaFree(c->gpartial);
  if (c->gcount) cudaFree(c->gcount);
  if (c->staging) cudaFree(c->staging);
  if (c->pstage) cudaFree(c->pstage);
  if (c->tc_b) cudaFree(c->tc_b);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return LBM_OK;
}

int lbm_audit(lbm_ctx* c, double totals[4]) {
  if (!c || !totals) return fail(c, LBM_ERR_INVALID, "NULL argument");
  const dim3 blk(AUX_X, AUX_Y);
  const double area = c->cfg.dx * c->cfg.dy;
  if (c->dwp)
    k_audit<dw><<<c->aux_grid, blk, 0, c->stream>>>((const dw*)c->f[c->cur], c->cfg.nx, c->cfg.ny,
                                                 c->pitch, c->plane, area, c->st, c->partial,
                                                 c->Kd);
  else if (c->esize == 8)
    k_audit<double><<<c->aux_grid, blk, 0, c->stream>>>((const double*)c->f[c->cur], c->cfg.nx,
                                                     c->cfg.ny, c->pitch, c->plane, area,
                                                     c->st, c->partial, c->Kd);
  else
    k_audit<float><<<c->aux_grid, blk, 0, c->stream>>>((const float*)c->f[c->cur], c->cfg.nx,
                                                    c->cfg.ny, c->pitch, c->plane, area,
                                                    c->st, c->partial, c->Kd);
  CK(c, cudaGetLastError());
  CK(c, cudaMemcpyAsync(totals, c->st->audit_now, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_audit_log(lbm_ctx* c, double* totals, long long* steps, int max_entries, int* count) {
  if (!c || !count || max_entries < 0) return fail(c, LBM_ERR_INVALID, "bad argument");
  std::vector<DevStatus> h(1);
  CK(c, cudaMemcpyAsync(h.data(), c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const DevStatus& s = h[0];
  const unsigned long long n = s.audit_count < LBM_AUDIT_RING ? s.audit_count : LBM_AUDIT_RING;
  const unsigned long long first = s.audit_count - n;
  int k = 0;
  for (unsigned long long a = first; a < s.audit_count && k < max_entries; ++a, ++k) {
    const unsigned long long slot = a % LBM_AUDIT_RING;
    if (totals)
      for (int q = 0; q < 4; ++q) totals[4 * k + q] = s.audit_totals[slot][q];
    if (steps) steps[k] = s.audit_steps[slot];
  }
  *count = k;
  return LBM_OK;
}

int lbm_status(lbm_ctx* c, long long* first_bad_step, long long* first_negT_step) {
  if (!c) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
  DevStatus h;
  CK(c, cudaMemcpyAsync(&h, c->st, offsetof(DevStatus, audit_totals), cudaMemcpyDeviceToHost,
                        c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (h.tma_timeout) {
    c->err = "a tile load (TMA) did not complete within its time limit";
    return LBM_ERR_TIMEOUT;
  }
  const long long bad = h.first_bad == NONE ? -1 : (long long)h.first_bad;
  const long long neg = h.first_negT == NONE ? -1 : (long long)h.first_negT;
  if (first_bad_step) *first_bad_step = bad;
  if (first_negT_step) *first_negT_step = neg;
  if (bad >= 0) {
    c->err = "state non-finite or rho <= 0 at time level " + std::to_string(bad);
    return LBM_ERR_NONFINITE;
  }
  return LBM_OK;
}

long long lbm_step_count(lbm_ctx* c) {
  if (!c) return -1;
  unsigned long long s = 0;
  if (cudaMemcpyAsync(&s, &c->st->step[c->cur], sizeof(s), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return -1;
  return (long long)s;
}

int lbm_get_populations(lbm_ctx* c, void* f, long long* step, int on_device) {
  if (!c || !f) return fail(c, LBM_ERR_INVALID, "NULL argument");
  const size_t w = (size_t)c->cfg.nx * c->esize;
  const size_t bytes = w * 16 * c->cfg.ny;
  if (on_device) {
    CK(c, cudaMemcpy2DAsync(f, w, c->f[c->cur], (size_t)c->pitch * c->esize, w,
                            (size_t)16 * c->cfg.ny, cudaMemcpyDeviceToDevice, c->stream));
  } else if (c->pitch == c->cfg.nx) {  // rows unpadded: one contiguous copy
    CK(c, cudaMemcpyAsync(f, c->f[c->cur], bytes, cudaMemcpyDeviceToHost, c->stream));
  } else {  // gather into a contiguous stage, then one copy (not 16 ny short rows)
    int rc = population_stage(c);
    if (rc == LBM_OK) rc = repitch(c, c->f[c->cur], c->pitch, c->pstage, c->cfg.nx);
    if (rc != LBM_OK) return rc;
    CK(c, cudaMemcpyAsync(f, c->pstage, bytes, cudaMemcpyDeviceToHost, c->stream));
  }
  if (step) {
    unsigned long long s = 0;
    CK(c, cudaMemcpyAsync(&s, &c->st->step[c->cur], sizeof(s), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *step = (long long)s;
  } else if (!on_device) {
    CK(c, cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, const void* f, long long step, int on_device) {
  if (!c || !f || step < 0) return fail(c, LBM_ERR_INVALID, "bad argument");
  const size_t w = (size_t)c->cfg.nx * c->esize;
  const size_t bytes = w * 16 * c->cfg.ny;
  c->cur = 0;
  if (on_device) {
    CK(c, cudaMemcpy2DAsync(c->f[0], (size_t)c->pitch * c->esize, f, w, w,
                            (size_t)16 * c->cfg.ny, cudaMemcpyDeviceToDevice, c->stream));
  } else if (c->pitch == c->cfg.nx) {
    CK(c, cudaMemcpyAsync(c->f[0], f, bytes, cudaMemcpyHostToDevice, c->stream));
  } else {  // one contiguous copy into a stage, then spread to the row pitch
    int rc = population_stage(c);
    if (rc != LBM_OK) return rc;
    CK(c, cudaMemcpyAsync(c->pstage, f, bytes, cudaMemcpyHostToDevice, c->stream));
    if ((rc = repitch(c, c->pstage, c->cfg.nx, c->f[0], c->pitch)) != LBM_OK) return rc;
  }
  const int rc = reset_status(c, (unsigned long long)step);
  if (rc == LBM_OK && !on_device) CK(c, cudaStreamSynchronize(c->stream));  // host f is free again
  return rc;
}

int lbm_element_size(lbm_ctx* c) { return c ? c->esize : 0; }

}  // extern "C"

namespace {

// Sets the number of blocks of the step launch: later steps are issued with
// `g` blocks and the captured graphs are rebuilt.
int apply_blocks(lbm_ctx* c, int g) {
  CK(c, cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 2; ++k)
    if (c->graph[k]) {
      cudaGraphExecDestroy(c->graph[k]);
      c->graph[k] = nullptr;
    }
  c->nblocks = g;
  c->grid = dim3(g);
  return LBM_OK;
}

// Times `launches` step launches with `g` blocks that read the current buffer
// and write the spare one, against a scratch status (no audit), so the
// state, the step counter and the audit log are untouched. Mean ms / launch.
template <typename R, int VAR = 0>
int time_blocks(lbm_ctx* c, int g, int launches, DevStatus* scratch, cudaEvent_t e0,
                cudaEvent_t e1, float* ms) {
  CK(c, cudaMemsetAsync(scratch, 0, offsetof(DevStatus, audit_totals), c->stream));
  StepArgs<R> A = make_args<R>(c, 0);
  A.st = scratch;
  A.audit_every = 0;
  A.nblocks = g;
  for (int j = 0; j < 2 + launches; ++j) {
    if (j == 2) CK(c, cudaEventRecord(e0, c->stream));
    A.slot = j & 1;
    const int rc = launch_persistent<R, VAR>(c, c->stream, c->cur, c->f[1 - c->cur], A);
    if (rc != LBM_OK) return rc;
  }
  CK(c, cudaEventRecord(e1, c->stream));
  CK(c, cudaEventSynchronize(e1));
  CK(c, cudaEventElapsedTime(ms, e0, e1));
  *ms /= (float)launches;
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_set_step_blocks(lbm_ctx* c, int blocks) {
  if (!c) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
  if (blocks < 0) return fail(c, LBM_ERR_INVALID, "blocks < 0");
  if (c->tc) return fail(c, LBM_ERR_UNSUPPORTED, "the tensor-core step sets its own launch");
  return apply_blocks(c, blocks == 0 ? default_blocks(c) : std::min(blocks, c->ntiles));
}

int lbm_step_blocks(lbm_ctx* c) { return c ? c->nblocks : -1; }

int lbm_set_fused_steps(lbm_ctx* c, int steps) {
  if (!c) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
  if (steps != 1 && steps != 2) return fail(c, LBM_ERR_INVALID, "steps per launch must be 1 or 2");
  if (steps == 2 && (c->tc || c->dwmom || c->esize != 4))
    return fail(c, LBM_ERR_UNSUPPORTED, "two steps per launch: LBM_FP32 contexts only");
  c->fuse = steps;
  return LBM_OK;
}

int lbm_fused_steps(lbm_ctx* c) { return c ? c->fuse : -1; }

int lbm_autotune(lbm_ctx* c, int launches) {
  if (!c) return fail(nullptr, LBM_ERR_INVALID, "ctx is NULL");
  if (launches < 1) return fail(c, LBM_ERR_INVALID, "launches < 1");
  if (c->tc) return LBM_OK;  // nothing to choose
  // Candidates: one tile per block (k_step), and for k_step_pipe 1 ..
  // MINB_PIPE blocks per SM and ceil(ntiles / m) blocks for m = 2 .. 8 tiles
  // per block.
  const int per_sm = c->dwp ? Shape<dw>::MINB_PIPE
                            : (c->esize == 8 ? Shape<double>::MINB_PIPE : Shape<float>::MINB_PIPE);
  std::vector<int> cand;
  auto add = [&](long long g) {
    const int v = (int)std::max(1ll, std::min((long long)c->ntiles, g));
    if (std::find(cand.begin(), cand.end(), v) == cand.end()) cand.push_back(v);
  };
  for (int m = 1; m <= 8; ++m) add(((long long)c->ntiles + m - 1) / m);
  for (int m = 1; m <= per_sm; ++m) add((long long)m * c->sms);
  DevStatus* scratch = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(c, cudaMalloc((void**)&scratch, sizeof(DevStatus)));
  int rc = LBM_OK, best = cand[0];
  float best_ms = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = fail(c, LBM_ERR_CUDA, "cudaEventCreate failed");
  for (size_t i = 0; i < cand.size() && rc == LBM_OK; ++i) {
    float ms = 0.f;
    rc = c->dwp ? time_blocks<dw>(c, cand[i], launches, scratch, e0, e1, &ms)
         : c->dwmom ? time_blocks<float, 1>(c, cand[i], launches, scratch, e0, e1, &ms)
         : c->esize == 8 ? time_blocks<double>(c, cand[i], launches, scratch, e0, e1, &ms)
                         : time_blocks<float>(c, cand[i], launches, scratch, e0, e1, &ms);
    if (rc == LBM_OK && (i == 0 || ms < best_ms)) {
      best_ms = ms;
      best = cand[i];
    }
  }
  cudaStreamSynchronize(c->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(scratch);
  if (rc != LBM_OK) return rc;
  return apply_blocks(c, best);
}

const char* lbm_last_error(lbm_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
