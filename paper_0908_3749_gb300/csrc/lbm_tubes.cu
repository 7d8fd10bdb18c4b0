// lbm_tubes.cu -- batches of quasi-1D shock tubes (include/lbm_batch.h) in one
// persistent, graph-captured kernel launch per call.
//
// Layout: FP32 populations SoA f[i][p], p running over all tubes; tube t owns
// nodes off[t] .. off[t] + nx[t] - 1 with off[t] a multiple of 32 (128-byte
// aligned rows), and 32 unused nodes lie before the first tube and after the
// last, so that the staged copies below never leave the allocation. Work items
// are tiles of `tile` consecutive nodes of one tube; the item list is ordered
// tube by tube.
//
// Per node the arithmetic is the 2D step with every y-derivative zero (one
// node deep, y periodic): the collision of Eq. 3 through the factorised
// transforms of d2v16.cuh, then f+ = (1 - c^2) f + (c^2 - c)/2 f(x+dx)
// + (c^2 + c)/2 f(x-dx) + df with c = v_x dt / dx (Eq. A.1b). The per-tube
// constants are the relaxation weights w_k = -dt s_k and lambda = dt / dx;
// the scaled block inverses of M are lattice constants shared by all tubes.
//
// The persistent kernel runs all requested steps: each resident block takes
// items blockIdx, blockIdx + gridDim, ...; the 16 population rows of an item
// and 4 halo nodes on each side come into shared memory by bulk TMA copies
// (two stages: the next item's copy runs while the current one is computed);
// each thread updates node pairs (x, x + threads) in paired FP32 arithmetic.
// After each step all blocks meet at a grid barrier whose spin is bounded in
// time. Co-residency is guaranteed by a cooperative launch sized from the
// occupancy calculator.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>  // header-only; ranges cost nothing without a profiler attached

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/lbm_batch.h"
#include "coeffs.h"
#include "d2v16.cuh"
#include "tma.cuh"

using namespace d2v16;
using namespace gbtma;

namespace {

constexpr unsigned long long NONE = ~0ull;
constexpr long long TUBE_PAD = 32;  // unused nodes before the first and after the last tube

struct TubeDesc {
  long long off;   // first population index of the tube
  long long out;   // first index in the concatenated field arrays
  int nx;
  float lam;       // dt / dx
  float w[12];     // -dt s_k for k = 5..16
};

struct BatchStatus {
  unsigned long long step;  // time level of the current buffer
  int cur;                  // which buffer holds it
  unsigned bar_count;       // arrivals at the running barrier
  unsigned bar_gen;         // barrier generation
  int timeout;              // a barrier wait expired
  unsigned long long first_timeout_step;
};

struct BatchArgs {
  Coeffs<float> E;            // only E0/EX/EY/EC/ES are used (lattice constants)
  const TubeDesc* tubes;
  const int2* items;          // (tube, first node of the tile)
  const float* ghost;         // [ntubes][2][16]: x- and x+ Dirichlet ghosts
  unsigned long long* bad;    // [ntubes] first bad time level
  BatchStatus* st;
  long long plane;            // populations per buffer plane
  int nitems;
  int skip_block;             // test hook: block that skips one barrier arrival
  long long skip_step;
  long long spin_cycles;      // barrier wait limit in SM clock cycles
};

// Velocity magnitude class of population i along x: 0 (v_x = 0), or the
// group index + 1; and the sign of v_x.
__host__ __device__ constexpr int xclass(int i) { return has_x(i) ? (i >> 2) + 1 : 0; }
__host__ __device__ constexpr float xsign(int i) {
  return vel_x(i) > 0.0 ? 1.0f : (vel_x(i) < 0.0 ? -1.0f : 0.0f);
}
__host__ __device__ constexpr double xmag(int g) {
  return g == 0 ? 1.0 : (g == 1 ? 6.0 : (g == 2 ? SQ2 : 3.0 / SQ2));
}

// Bounded grid barrier. Returns false (and every block leaves) when the wait
// exceeded A.spin_cycles or another block already reported a timeout.
__device__ bool grid_barrier(const BatchArgs& A, unsigned& gen, bool skip) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = gen;
    if (!skip) {
      __threadfence();
      const unsigned prev = atomicAdd(&A.st->bar_count, 1u);
      if (prev == gridDim.x - 1) {
        A.st->bar_count = 0;
        __threadfence();
        atomicExch(&A.st->bar_gen, g + 1);
      } else {
        const long long t0 = clock64();
        while (*(volatile unsigned*)&A.st->bar_gen == g) {
          if (*(volatile int*)&A.st->timeout || clock64() - t0 > A.spin_cycles) {
            atomicExch(&A.st->timeout, 1);
            ok = 0;
            break;
          }
          __nanosleep(256);
        }
        __threadfence();
      }
    } else {
      ok = 0;  // the skipping block leaves without waiting
    }
    gen = g + 1;
  }
  __syncthreads();
  return ok != 0;
}

// Staged width of an item: its TILE nodes plus 4 halo nodes on each side.
template <int TILE>
__host__ __device__ constexpr int stage_width() { return TILE + 8; }

// Thread 0: copies item `item` (16 population rows of its valid nodes plus
// 4 halo nodes on each side, rounded up to 16 bytes) into `stage`. The
// source start off + x0 - 4 is a multiple of 4 floats (off and x0 are
// multiples of 32 and of TILE), so both ends are 16-byte aligned.
template <int TILE>
__device__ __forceinline__ void issue_item(const BatchArgs& A, const float* fin, float* stage,
                                           int item, unsigned long long* bar) {
  const int2 it = A.items[item];
  const TubeDesc& D = A.tubes[it.x];
  const int valid = min(TILE, D.nx - it.y);
  const unsigned n = (unsigned)((valid + 8 + 3) & ~3);  // floats per row, <= TILE + 8
  mbar_expect_tx(bar, 16u * 4u * n);
  const float* src = fin + D.off + it.y - 4;
#pragma unroll 1
  for (int i = 0; i < 16; ++i)
    bulk_load(stage + i * stage_width<TILE>(), src + i * A.plane, 4u * n, bar);
}

// Updates one item from its staged copy: thread t takes node pairs
// (x, x + BT) of each 2 BT-node chunk in paired arithmetic.
template <int BT, int TILE>
__device__ __forceinline__ void tube_item(const BatchArgs& A, float* __restrict__ fout,
                                          const float* stage, int item, unsigned long long level) {
  constexpr int W = stage_width<TILE>();
  const int2 it = A.items[item];
  const TubeDesc& D = A.tubes[it.x];
  const long long off = D.off;
  const int nx = D.nx;
  const float lam = D.lam;
  float w[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) w[k] = D.w[k];
  // Lax-Wendroff weights per |v_x| class: a0 = 1 - 2 b, aE = b - s a, aW = b + s a
  float al[4], be[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const float c = (float)xmag(g) * lam;
    al[g] = 0.5f * c;
    be[g] = 0.5f * c * c;
  }
  const float* gL = A.ghost + (size_t)it.x * 32;
  const float* gR = gL + 16;
  const long long P = A.plane;
  const Coeffs<float>& E = A.E;
  bool bad = false;
#pragma unroll 1
  for (int c0 = 0; c0 < TILE; c0 += 2 * BT) {
    const int la = c0 + threadIdx.x, lb = la + BT;  // node index within the item
    const int xa = it.y + la, xb = it.y + lb;
    if (xa >= nx) continue;
    const bool actb = xb < nx;
    const float* sa = stage + la + 4;
    const float* sb = stage + lb + 4;
    F2 f[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i] = F2(sa[i * W], sb[i * W]);
    Groups<F2> d;
    transform(f, d);
    const Cons<F2> m = conserved(E, d);
    const Eq<F2> q = equilibria(m.rho, m.jx, m.jy, m.e);
    // deviations from equilibrium of the non-conserved moments, relaxed
    const F2 r11 = w[6] * (row4(E.F0, 2, d.S) - q.m11);
    const F2 r12 = w[7] * row4(E.F0, 3, d.S);
    const F2 r7 = w[2] * (row4(E.FX, 1, d.X) - q.m7);
    const F2 r9 = w[4] * (row4(E.FX, 2, d.X) - q.m9);
    const F2 r15 = w[10] * row4(E.FX, 3, d.X);
    const F2 r8 = w[3] * (row4(E.FY, 1, d.Y) - q.m8);
    const F2 r10 = w[5] * (row4(E.FY, 2, d.Y) - q.m10);
    const F2 r16 = w[11] * row4(E.FY, 3, d.Y);
    const F2 r5 = w[0] * (E.FC[0][0] * d.C[0] + E.FC[0][1] * d.C[1] - q.m5);
    const F2 r13 = w[8] * (E.FC[1][0] * d.C[0] + E.FC[1][1] * d.C[1] - q.m13);
    const F2 r6 = w[1] * (E.FS[0][0] * d.C[2] + E.FS[0][1] * d.C[3] - q.m6);
    const F2 r14 = w[9] * (E.FS[1][0] * d.C[2] + E.FS[1][1] * d.C[3] - q.m14);
    F2 S[4], C[4], X[4], Y[4], df[16];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      S[g] = E.E0[g][2] * r11 + E.E0[g][3] * r12;
      X[g] = E.EX[g][1] * r7 + E.EX[g][2] * r9 + E.EX[g][3] * r15;
      Y[g] = E.EY[g][1] * r8 + E.EY[g][2] * r10 + E.EY[g][3] * r16;
    }
    C[0] = E.EC[0][0] * r5 + E.EC[0][1] * r13;
    C[1] = E.EC[1][0] * r5 + E.EC[1][1] * r13;
    C[2] = E.ES[0][0] * r6 + E.ES[0][1] * r14;
    C[3] = E.ES[1][0] * r6 + E.ES[1][1] * r14;
    inverse_transform(S, C, X, Y, df);
    bad |= !(m.rho.v.x > 0.0f) || !isfinite(m.rho.v.x + m.jx.v.x + m.jy.v.x + m.e.v.x);
    bad |= actb && (!(m.rho.v.y > 0.0f) || !isfinite(m.rho.v.y + m.jx.v.y + m.jy.v.y + m.e.v.y));
    const bool wa = xa > 0, ea = xa < nx - 1, wb = xb > 0, eb = xb < nx - 1;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      F2 out;
      if (xclass(i) == 0) {
        out = f[i] + df[i];
      } else {
        const int g = xclass(i) - 1;
        const float s = xsign(i);
        const F2 fe(ea ? sa[i * W + 1] : gR[i], eb ? sb[i * W + 1] : gR[i]);
        const F2 fw(wa ? sa[i * W - 1] : gL[i], wb ? sb[i * W - 1] : gL[i]);
        out = (1.0f - 2.0f * be[g]) * f[i] + df[i];
        out = (be[g] - s * al[g]) * fe + out;
        out = (be[g] + s * al[g]) * fw + out;
      }
      fout[i * P + off + xa] = out.v.x;
      if (actb) fout[i * P + off + xb] = out.v.y;
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
    atomicMin(&A.bad[it.x], level);
}

template <int BT, int TILE>
__global__ void __launch_bounds__(BT) k_tubes(float* f0, float* f1, const BatchArgs A,
                                              long long nsteps) {
  extern __shared__ __align__(16) unsigned char tube_smem[];
  float* const stages = reinterpret_cast<float*>(tube_smem);  // [2][16][stage_width]
  constexpr int SE = 16 * stage_width<TILE>();
  __shared__ unsigned long long bar[2];
  __shared__ unsigned long long s_level;
  __shared__ int s_cur;
  __shared__ unsigned s_gen;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_level = *(volatile unsigned long long*)&A.st->step;
    s_cur = *(volatile int*)&A.st->cur;
    s_gen = *(volatile unsigned*)&A.st->bar_gen;
  }
  __syncthreads();
  const unsigned long long level0 = s_level;
  const int cur = s_cur;
  unsigned gen = s_gen;
  long long k = 0;  // items processed by this block: stage k & 1, phase (k >> 1) & 1
  // All blocks read the state above before anyone can pass this barrier.
  if (!grid_barrier(A, gen, false)) return;
  for (long long s = 0; s < nsteps; ++s) {
    const bool even = ((s + cur) & 1) == 0;
    const float* fin = even ? f0 : f1;
    float* fout = even ? f1 : f0;
    // Plain stores of the previous step are read below by bulk copies.
    fence_proxy_async();
    if (threadIdx.x == 0 && (int)blockIdx.x < A.nitems)
      issue_item<TILE>(A, fin, stages + (k & 1) * SE, blockIdx.x, &bar[k & 1]);
    for (int item = blockIdx.x; item < A.nitems; item += gridDim.x, ++k) {
      const int st = (int)(k & 1);
      const int next = item + (int)gridDim.x;
      // Stage 1 - st was released at the end of the previous item.
      if (threadIdx.x == 0 && next < A.nitems)
        issue_item<TILE>(A, fin, stages + (1 - st) * SE, next, &bar[1 - st]);
      if (!__syncthreads_and(mbar_wait_bounded(&bar[st], (unsigned)((k >> 1) & 1), TMA_WAIT_CYCLES))) {
        // A copy did not land: record it (the other blocks leave at the next
        // barrier), wait once more for this block's copies, leave.
        if (threadIdx.x == 0) {
          atomicExch(&A.st->timeout, 1);
          atomicMin(&A.st->first_timeout_step, level0 + s);
          mbar_wait_bounded(&bar[st], (unsigned)((k >> 1) & 1), TMA_WAIT_CYCLES);
          if (next < A.nitems)
            mbar_wait_bounded(&bar[1 - st], (unsigned)(((k + 1) >> 1) & 1), TMA_WAIT_CYCLES);
        }
        return;
      }
      tube_item<BT, TILE>(A, fout, stages + st * SE, item, level0 + (unsigned long long)s);
      __syncthreads();  // stage st is free again
    }
    fence_proxy_async();
    const bool skip = (int)blockIdx.x == A.skip_block && s == A.skip_step;
    if (!grid_barrier(A, gen, skip)) {
      if (threadIdx.x == 0) atomicMin(&A.st->first_timeout_step, level0 + s);
      return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.st->step = level0 + (unsigned long long)nsteps;
    A.st->cur = (int)((cur + nsteps) & 1);
  }
}

// ---------------------------------------------------------------------------
// Init, moments, audit, ghosts (one block per item / per tube)
// ---------------------------------------------------------------------------
constexpr int AUX_T = 128;

__global__ void k_tubes_init(float* f, const TubeDesc* tubes, const int2* items, long long P,
                             int tile, const double* rho, const double* u, const double* v,
                             const double* T, const Coeffs<double> K) {
  const int2 it = items[blockIdx.x];
  const TubeDesc D = tubes[it.x];
  for (int j = threadIdx.x; j < tile; j += blockDim.x) {
    const int x = it.y + j;
    if (x >= D.nx) break;
    const long long k = D.out + x;
    const double r = rho[k], uu = u[k], vv = v[k];
    double g[16];
    feq(K, r, r * uu, r * vv, r * T[k] + 0.5 * r * (uu * uu + vv * vv), g);
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i * P + D.off + x] = (float)g[i];
  }
}

__global__ void k_tubes_moments(const float* f, const TubeDesc* tubes, const int2* items,
                                long long P, int tile, double* rho, double* u, double* v,
                                double* T, const Coeffs<double> K) {
  const int2 it = items[blockIdx.x];
  const TubeDesc D = tubes[it.x];
  for (int j = threadIdx.x; j < tile; j += blockDim.x) {
    const int x = it.y + j;
    if (x >= D.nx) break;
    double g[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = (double)f[i * P + D.off + x];
    Groups<double> d;
    transform(g, d);
    const Cons<double> m = conserved(K, d);
    const double r = 1.0 / m.rho, uu = m.jx * r, vv = m.jy * r;
    const long long k = D.out + x;
    if (rho) rho[k] = m.rho;
    if (u) u[k] = uu;
    if (v) v[k] = vv;
    if (T) T[k] = m.e * r - 0.5 * (uu * uu + vv * vv);
  }
}

// One block per tube: FP64 totals over the tube's nodes in a fixed order.
__global__ void __launch_bounds__(AUX_T) k_tubes_audit(const float* f, const TubeDesc* tubes,
                                                       const double* dx, long long P,
                                                       double* totals, const Coeffs<double> K) {
  __shared__ double sm[AUX_T][4];
  const TubeDesc D = tubes[blockIdx.x];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int x = threadIdx.x; x < D.nx; x += AUX_T) {
    double g[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = (double)f[i * P + D.off + x];
    Groups<double> d;
    transform(g, d);
    const Cons<double> m = conserved(K, d);
    s[0] += m.rho; s[1] += m.jx; s[2] += m.jy; s[3] += m.e;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) sm[threadIdx.x][q] = s[q];
  __syncthreads();
  for (int stride = AUX_T / 2; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride)
#pragma unroll
      for (int q = 0; q < 4; ++q) sm[threadIdx.x][q] += sm[threadIdx.x + stride][q];
    __syncthreads();
  }
  if (threadIdx.x < 4) totals[4 * blockIdx.x + threadIdx.x] = sm[0][threadIdx.x] * dx[blockIdx.x];
}

__global__ void k_tubes_ghost(float* ghost, const double* states, int ntubes,
                              const Coeffs<double> K) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;  // (tube, side)
  if (k >= 2 * ntubes) return;
  const double* s = states + 4 * k;
  const double r = s[0], u = s[1], v = s[2], T = s[3];
  double g[16];
  feq(K, r, r * u, r * v, r * T + 0.5 * r * (u * u + v * v), g);
#pragma unroll
  for (int i = 0; i < 16; ++i) ghost[16 * k + i] = (float)g[i];
}

// ---------------------------------------------------------------------------
// Tiling candidates
// ---------------------------------------------------------------------------
using KernelFn = void (*)(float*, float*, const BatchArgs, long long);
struct Variant {
  int tile, threads;
  KernelFn fn;
};
const Variant VARIANTS[] = {
    {128, 64, k_tubes<64, 128>},     {256, 64, k_tubes<64, 256>},
    {256, 128, k_tubes<128, 256>},   {512, 128, k_tubes<128, 512>},
    {512, 256, k_tubes<256, 512>},   {1024, 256, k_tubes<256, 1024>},
    {1024, 512, k_tubes<512, 1024>}, {1024, 128, k_tubes<128, 1024>},
};
size_t variant_smem(int v) {
  return 2 * 16 * sizeof(float) * (size_t)(VARIANTS[v].tile + 8) + 16;
}
constexpr int NVARIANTS = sizeof(VARIANTS) / sizeof(VARIANTS[0]);

int find_variant(int tile, int threads) {
  for (int k = 0; k < NVARIANTS; ++k)
    if (VARIANTS[k].tile == tile && VARIANTS[k].threads == threads) return k;
  return -1;
}

thread_local std::string g_batch_create_error = "no error";

}  // namespace

struct lbm_batch {
  int ntubes = 0;
  std::vector<int> nx;
  std::vector<double> dx;
  std::vector<TubeDesc> h_tubes;
  long long plane = 0, total = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float* f[2] = {nullptr, nullptr};
  TubeDesc* tubes = nullptr;
  int2* items = nullptr;
  int nitems = 0;
  float* ghost = nullptr;
  unsigned long long* bad = nullptr;
  BatchStatus* st = nullptr;
  double* d_dx = nullptr;
  double* staging = nullptr;   // 4 * total doubles
  double* d_totals = nullptr;  // 4 * ntubes
  Coeffs<double> Kd;
  int variant = 3;             // tile 256, 128 threads
  int blocks = 0;
  int sms = 0;
  long long spin_cycles = 0;
  int skip_block = -1;
  long long skip_step = -1;
  std::map<std::pair<long long, int>, cudaGraphExec_t> graphs;
  std::string err = "no error";
};

namespace {

int bfail(lbm_batch* b, int code, const std::string& m) {
  if (b) b->err = m; else g_batch_create_error = m;
  return code;
}
int bcuda(lbm_batch* b, cudaError_t e, const char* what) {
  return bfail(b, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}
#define BCK(b, call)                                  \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return bcuda(b, e_, #call); \
  } while (0)

int build_items(lbm_batch* b) {
  const int tile = VARIANTS[b->variant].tile;
  std::vector<int2> items;
  for (int t = 0; t < b->ntubes; ++t)
    for (int x0 = 0; x0 < b->nx[t]; x0 += tile) items.push_back(make_int2(t, x0));
  if (b->items) cudaFree(b->items);
  b->items = nullptr;
  b->nitems = (int)items.size();
  BCK(b, cudaMalloc((void**)&b->items, sizeof(int2) * items.size()));
  BCK(b, cudaMemcpyAsync(b->items, items.data(), sizeof(int2) * items.size(),
                         cudaMemcpyHostToDevice, b->stream));
  int per_sm = 0;
  const Variant& V = VARIANTS[b->variant];
  const size_t smem = variant_smem(b->variant);
  BCK(b, cudaFuncSetAttribute((const void*)V.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem));
  BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, V.fn, V.threads, smem));
  if (per_sm < 1) return bfail(b, LBM_ERR_CUDA, "tube kernel does not fit on an SM");
  b->blocks = std::min(per_sm * b->sms, b->nitems);
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
  b->graphs.clear();
  BCK(b, cudaStreamSynchronize(b->stream));
  return LBM_OK;
}

BatchArgs make_batch_args(lbm_batch* b) {
  BatchArgs A;
  const double* s = reinterpret_cast<const double*>(&b->Kd);
  float* d = reinterpret_cast<float*>(&A.E);
  for (size_t k = 0; k < sizeof(Coeffs<double>) / sizeof(double); ++k) d[k] = (float)s[k];
  A.tubes = b->tubes;
  A.items = b->items;
  A.ghost = b->ghost;
  A.bad = b->bad;
  A.st = b->st;
  A.plane = b->plane;
  A.nitems = b->nitems;
  A.skip_block = b->skip_block;
  A.skip_step = b->skip_step;
  A.spin_cycles = b->spin_cycles;
  return A;
}

int launch_tubes(lbm_batch* b, long long nsteps) {
  const Variant& V = VARIANTS[b->variant];
  BatchArgs A = make_batch_args(b);
  float* f0 = b->f[0];
  float* f1 = b->f[1];
  void* args[] = {&f0, &f1, &A, &nsteps};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->blocks);
  cfg.blockDim = dim3(V.threads);
  cfg.dynamicSmemBytes = variant_smem(b->variant);
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BCK(b, cudaLaunchKernelExC(&cfg, (const void*)V.fn, args));
  return LBM_OK;
}

int reset_batch_status(lbm_batch* b) {
  BatchStatus h;
  memset(&h, 0, sizeof(h));
  h.first_timeout_step = NONE;
  BCK(b, cudaMemcpyAsync(b->st, &h, sizeof(h), cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaMemsetAsync(b->bad, 0xff, sizeof(unsigned long long) * b->ntubes, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  return LBM_OK;
}

unsigned long long fnv1a(const void* p, size_t n, unsigned long long h = 1469598103934665603ull) {
  const unsigned char* c = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
  return h;
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_batch_config* cfg, void* cuda_stream, lbm_batch** out) {
  if (!out) return bfail(nullptr, LBM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!cfg || cfg->ntubes < 1 || !cfg->nx || !cfg->dx || !cfg->s || !cfg->left || !cfg->right)
    return bfail(nullptr, LBM_ERR_INVALID, "incomplete batch configuration");
  if (!(std::isfinite(cfg->dt) && cfg->dt > 0.0))
    return bfail(nullptr, LBM_ERR_INVALID, "dt must be finite and > 0");
  for (int t = 0; t < cfg->ntubes; ++t) {
    if (cfg->nx[t] < 2) return bfail(nullptr, LBM_ERR_INVALID, "every tube needs nx >= 2");
    if (!(std::isfinite(cfg->dx[t]) && cfg->dx[t] > 0.0))
      return bfail(nullptr, LBM_ERR_INVALID, "dx must be finite and > 0");
    if (6.0 * cfg->dt / cfg->dx[t] > 1.0)
      return bfail(nullptr, LBM_ERR_INVALID, "Courant number 6 dt / dx exceeds 1");
    for (int k = 0; k < 16; ++k)
      if (!(std::isfinite(cfg->s[16 * t + k]) && cfg->s[16 * t + k] >= 0.0))
        return bfail(nullptr, LBM_ERR_INVALID, "relaxation rates must be finite and >= 0");
    for (int side = 0; side < 2; ++side) {
      const double* q = (side ? cfg->right : cfg->left) + 4 * t;
      if (!(q[0] > 0.0 && q[3] > 0.0 && std::isfinite(q[0] + q[1] + q[2] + q[3])))
        return bfail(nullptr, LBM_ERR_INVALID, "boundary states need rho > 0 and T > 0");
    }
  }
  lbm_batch* b = new lbm_batch();
  b->ntubes = cfg->ntubes;
  b->nx.assign(cfg->nx, cfg->nx + cfg->ntubes);
  b->dx.assign(cfg->dx, cfg->dx + cfg->ntubes);
  if (!lattice_constants(b->Kd)) {
    delete b;
    return bfail(nullptr, LBM_ERR_INVALID, "singular moment block");
  }
  long long off = TUBE_PAD, outo = 0;
  for (int t = 0; t < b->ntubes; ++t) {
    TubeDesc D;
    D.off = off;
    D.out = outo;
    D.nx = b->nx[t];
    D.lam = (float)(cfg->dt / cfg->dx[t]);
    for (int k = 0; k < 12; ++k) D.w[k] = (float)(-cfg->dt * cfg->s[16 * t + 4 + k]);
    b->h_tubes.push_back(D);
    off += (D.nx + 31) / 32 * 32;
    outo += D.nx;
  }
  b->plane = off + TUBE_PAD;
  b->total = outo;
  cudaError_t e = cudaSuccess;
  int dev = 0, clk_khz = 0;
  if (cuda_stream) b->stream = (cudaStream_t)cuda_stream;
  else { e = cudaStreamCreate(&b->stream); b->own_stream = true; }
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  b->spin_cycles = (long long)clk_khz * 1000ll;  // about one second at the peak clock
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    e = cudaMalloc((void**)&b->f[k], sizeof(float) * 16 * b->plane);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    e = cudaMemsetAsync(b->f[k], 0, sizeof(float) * 16 * b->plane, b->stream);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->tubes, sizeof(TubeDesc) * b->ntubes);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->tubes, b->h_tubes.data(), sizeof(TubeDesc) * b->ntubes,
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->ghost, sizeof(float) * 32 * b->ntubes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->bad, sizeof(unsigned long long) * b->ntubes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->st, sizeof(BatchStatus));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_dx, sizeof(double) * b->ntubes);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_dx, cfg->dx, sizeof(double) * b->ntubes, cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->staging, sizeof(double) * 4 * b->total);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_totals, sizeof(double) * 4 * b->ntubes);
  double* dstates = nullptr;
  if (e == cudaSuccess) e = cudaMalloc((void**)&dstates, sizeof(double) * 8 * b->ntubes);
  if (e == cudaSuccess) {
    std::vector<double> states(8 * (size_t)b->ntubes);
    for (int t = 0; t < b->ntubes; ++t)
      for (int q = 0; q < 4; ++q) {
        states[8 * t + q] = cfg->left[4 * t + q];
        states[8 * t + 4 + q] = cfg->right[4 * t + q];
      }
    e = cudaMemcpyAsync(dstates, states.data(), sizeof(double) * states.size(),
                        cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) {
      k_tubes_ghost<<<(2 * b->ntubes + 127) / 128, 128, 0, b->stream>>>(b->ghost, dstates,
                                                                         b->ntubes, b->Kd);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  }
  if (dstates) cudaFree(dstates);
  if (e != cudaSuccess) {
    const int rc = bcuda(nullptr, e, "lbm_batch_create");
    lbm_batch_destroy(b);
    return rc;
  }
  if (build_items(b) != LBM_OK || reset_batch_status(b) != LBM_OK) {
    g_batch_create_error = b->err;
    lbm_batch_destroy(b);
    return LBM_ERR_CUDA;
  }
  *out = b;
  return LBM_OK;
}

int lbm_batch_set_init(lbm_batch* b, const double* rho, const double* u, const double* v,
                       const double* T, int on_device) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID, "batch is NULL");
  if (!rho || !u || !v || !T) return bfail(b, LBM_ERR_INVALID, "NULL field");
  const double* p[4] = {rho, u, v, T};
  if (!on_device)
    for (int k = 0; k < 4; ++k) {
      BCK(b, cudaMemcpyAsync(b->staging + k * b->total, p[k], sizeof(double) * b->total,
                             cudaMemcpyHostToDevice, b->stream));
      p[k] = b->staging + k * b->total;
    }
  const int tile = VARIANTS[b->variant].tile;
  k_tubes_init<<<b->nitems, AUX_T, 0, b->stream>>>(b->f[0], b->tubes, b->items, b->plane, tile,
                                                    p[0], p[1], p[2], p[3], b->Kd);
  BCK(b, cudaGetLastError());
  return reset_batch_status(b);
}

int lbm_batch_step(lbm_batch* b, long long nsteps) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID, "batch is NULL");
  if (nsteps < 0) return bfail(b, LBM_ERR_INVALID, "nsteps < 0");
  if (nsteps == 0) return LBM_OK;
  if (b->skip_block >= 0) {  // test hook: plain launch, never cached
    const int rc = launch_tubes(b, nsteps);
    b->skip_block = -1;
    b->skip_step = -1;
    return rc;
  }
  char range[64];
  snprintf(range, sizeof(range), "lbm_batch_step n=%lld (graph)", nsteps);
  nvtxRangePushA(range);
  struct Pop { ~Pop() { nvtxRangePop(); } } pop;
  auto key = std::make_pair(nsteps, b->variant);
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    cudaGraph_t g;
    BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = launch_tubes(b, nsteps);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc != LBM_OK) return rc;
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
    cudaGraphExec_t ex;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
    it = b->graphs.emplace(key, ex).first;
  }
  BCK(b, cudaGraphLaunch(it->second, b->stream));
  return LBM_OK;
}

int lbm_batch_moments(lbm_batch* b, double* rho, double* u, double* v, double* T,
                      int on_device) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID, "batch is NULL");
  double* h[4] = {rho, u, v, T};
  double* d[4] = {rho, u, v, T};
  if (!on_device)
    for (int k = 0; k < 4; ++k) d[k] = h[k] ? b->staging + k * b->total : nullptr;
  BatchStatus hs;
  BCK(b, cudaMemcpyAsync(&hs, b->st, sizeof(hs), cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  const int tile = VARIANTS[b->variant].tile;
  k_tubes_moments<<<b->nitems, AUX_T, 0, b->stream>>>(b->f[hs.cur], b->tubes, b->items,
                                                       b->plane, tile, d[0], d[1], d[2], d[3], b->Kd);
  BCK(b, cudaGetLastError());
  if (!on_device) {
    for (int k = 0; k < 4; ++k)
      if (h[k])
        BCK(b, cudaMemcpyAsync(h[k], d[k], sizeof(double) * b->total, cudaMemcpyDeviceToHost,
                               b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
  }
  return LBM_OK;
}

int lbm_batch_audit(lbm_batch* b, double* totals) {
  if (!b || !totals) return bfail(b, LBM_ERR_INVALID, "NULL argument");
  BatchStatus hs;
  BCK(b, cudaMemcpyAsync(&hs, b->st, sizeof(hs), cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  k_tubes_audit<<<b->ntubes, AUX_T, 0, b->stream>>>(b->f[hs.cur], b->tubes, b->d_dx, b->plane,
                                                     b->d_totals, b->Kd);
  BCK(b, cudaGetLastError());
  BCK(b, cudaMemcpyAsync(totals, b->d_totals, sizeof(double) * 4 * b->ntubes,
                         cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  return LBM_OK;
}

int lbm_batch_status(lbm_batch* b, long long* first_bad, int* nbad, int* timeout) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID, "batch is NULL");
  std::vector<unsigned long long> bad(b->ntubes);
  BatchStatus hs;
  BCK(b, cudaMemcpyAsync(bad.data(), b->bad, sizeof(unsigned long long) * b->ntubes,
                         cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaMemcpyAsync(&hs, b->st, sizeof(hs), cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  int n = 0;
  for (int t = 0; t < b->ntubes; ++t) {
    if (bad[t] != NONE) ++n;
    if (first_bad) first_bad[t] = bad[t] == NONE ? -1 : (long long)bad[t];
  }
  if (nbad) *nbad = n;
  if (timeout) *timeout = hs.timeout;
  if (hs.timeout) {
    b->err = "grid barrier wait expired";
    return LBM_ERR_TIMEOUT;
  }
  return LBM_OK;
}

int lbm_batch_set_tiling(lbm_batch* b, int tile, int threads) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID, "batch is NULL");
  const int k = find_variant(tile, threads);
  if (k < 0) return bfail(b, LBM_ERR_INVALID, "unsupported (tile, threads)");
  // keep the populations: items only change the work split, not the layout
  b->variant = k;
  return build_items(b);
}

int lbm_batch_get_tiling(lbm_batch* b, int* tile, int* threads, int* blocks) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID, "batch is NULL");
  if (tile) *tile = VARIANTS[b->variant].tile;
  if (threads) *threads = VARIANTS[b->variant].threads;
  if (blocks) *blocks = b->blocks;
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int trial_steps, const char* cache_path, int* chosen) {
  if (!b || trial_steps < 1) return bfail(b, LBM_ERR_INVALID, "bad argument");
  cudaDeviceProp prop;
  int dev = 0;
  BCK(b, cudaGetDevice(&dev));
  BCK(b, cudaGetDeviceProperties(&prop, dev));
  unsigned long long h = fnv1a(b->nx.data(), sizeof(int) * b->nx.size());
  h = fnv1a(b->dx.data(), sizeof(double) * b->dx.size(), h);
  char key[512];
  snprintf(key, sizeof(key), "%s|%016llx", prop.name, h);
  // cache lookup: one JSON object {"<key>": [tile, threads], ...}
  std::string text;
  if (cache_path) {
    FILE* fp = fopen(cache_path, "rb");
    if (fp) {
      char buf[4096];
      size_t n;
      while ((n = fread(buf, 1, sizeof(buf), fp)) > 0) text.append(buf, n);
      fclose(fp);
      const std::string pat = std::string("\"") + key + "\": [";
      const size_t at = text.find(pat);
      if (at != std::string::npos) {
        int tl = 0, th = 0;
        if (sscanf(text.c_str() + at + pat.size(), "%d, %d", &tl, &th) == 2 &&
            find_variant(tl, th) >= 0) {
          const int rc = lbm_batch_set_tiling(b, tl, th);
          if (rc != LBM_OK) return rc;
          if (chosen) { chosen[0] = tl; chosen[1] = th; }
          return LBM_OK;
        }
      }
    }
  }
  // save the populations and the status, time every candidate, restore
  float* save = nullptr;
  const size_t fb = sizeof(float) * 16 * b->plane;
  BCK(b, cudaMalloc((void**)&save, fb));
  BatchStatus hs;
  std::vector<unsigned long long> bad_save(b->ntubes);
  BCK(b, cudaMemcpyAsync(&hs, b->st, sizeof(hs), cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaMemcpyAsync(bad_save.data(), b->bad, sizeof(unsigned long long) * b->ntubes,
                         cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  BCK(b, cudaMemcpyAsync(save, b->f[hs.cur], fb, cudaMemcpyDeviceToDevice, b->stream));
  cudaEvent_t e0, e1;
  BCK(b, cudaEventCreate(&e0));
  BCK(b, cudaEventCreate(&e1));
  int best = -1;
  float best_ms = 1e30f;
  int rc = LBM_OK;
  for (int k = 0; k < NVARIANTS && rc == LBM_OK; ++k) {
    b->variant = k;
    if ((rc = build_items(b)) != LBM_OK) break;
    if ((rc = launch_tubes(b, 1)) != LBM_OK) break;  // warm-up
    cudaEventRecord(e0, b->stream);
    if ((rc = launch_tubes(b, trial_steps)) != LBM_OK) break;
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    BatchStatus chk;
    cudaMemcpy(&chk, b->st, sizeof(chk), cudaMemcpyDeviceToHost);
    if (!chk.timeout && ms < best_ms) { best_ms = ms; best = k; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore state and status
  if (rc == LBM_OK) {
    BatchStatus restore = hs;
    cudaMemcpyAsync(b->f[hs.cur], save, fb, cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(b->st, &restore, sizeof(restore), cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(b->bad, bad_save.data(), sizeof(unsigned long long) * b->ntubes,
                    cudaMemcpyHostToDevice, b->stream);
    cudaStreamSynchronize(b->stream);
  }
  cudaFree(save);
  if (rc != LBM_OK) return rc;
  if (best < 0) return bfail(b, LBM_ERR_TIMEOUT, "no tiling candidate completed");
  b->variant = best;
  if ((rc = build_items(b)) != LBM_OK) return rc;
  if (chosen) { chosen[0] = VARIANTS[best].tile; chosen[1] = VARIANTS[best].threads; }
  if (cache_path) {
    // append or replace the entry, keeping the file a flat JSON object
    std::string body;
    if (!text.empty()) {
      const size_t lb = text.find('{'), rb = text.rfind('}');
      if (lb != std::string::npos && rb != std::string::npos && rb > lb) {
        body = text.substr(lb + 1, rb - lb - 1);
        const std::string pat = std::string("\"") + key + "\"";
        const size_t at = body.find(pat);
        if (at != std::string::npos) {
          size_t end = body.find(']', at);
          size_t start = at;
          while (start > 0 && (body[start - 1] == ' ' || body[start - 1] == '\n' || body[start - 1] == ',')) --start;
          body.erase(start, end == std::string::npos ? std::string::npos : end + 1 - start);
        }
      }
    }
    while (!body.empty() && (body.back() == ' ' || body.back() == '\n' || body.back() == ',')) body.pop_back();
    while (!body.empty() && (body[0] == ' ' || body[0] == '\n' || body[0] == ',')) body.erase(0, 1);
    char entry[600];
    snprintf(entry, sizeof(entry), "\"%s\": [%d, %d]", key, VARIANTS[best].tile,
             VARIANTS[best].threads);
    FILE* fp = fopen(cache_path, "wb");
    if (fp) {
      fprintf(fp, "{%s%s%s}\n", body.c_str(), body.empty() ? "" : ",\n ", entry);
      fclose(fp);
    }
  }
  return LBM_OK;
}

int lbm_batch_debug_skip_arrival(lbm_batch* b, int block, long long step) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID, "batch is NULL");
  if (block >= b->blocks) return bfail(b, LBM_ERR_INVALID, "block out of range");
  b->skip_block = block;
  b->skip_step = step;
  return LBM_OK;
}

long long lbm_batch_step_count(lbm_batch* b) {
  if (!b) return -1;
  BatchStatus hs;
  if (cudaMemcpyAsync(&hs, b->st, sizeof(hs), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return -1;
  return (long long)hs.step;
}

int lbm_batch_total_nodes(lbm_batch* b, long long* total) {
  if (!b || !total) return bfail(b, LBM_ERR_INVALID, "NULL argument");
  *total = b->total;
  return LBM_OK;
}

int lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
  for (int k = 0; k < 2; ++k)
    if (b->f[k]) cudaFree(b->f[k]);
  if (b->tubes) cudaFree(b->tubes);
  if (b->items) cudaFree(b->items);
  if (b->ghost) cudaFree(b->ghost);
  if (b->bad) cudaFree(b->bad);
  if (b->st) cudaFree(b->st);
  if (b->d_dx) cudaFree(b->d_dx);
  if (b->staging) cudaFree(b->staging);
  if (b->d_totals) cudaFree(b->d_totals);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return LBM_OK;
}

const char* lbm_batch_last_error(lbm_batch* b) {
  return b ? b->err.c_str() : g_batch_create_error.c_str();
}

}  // extern "C"
