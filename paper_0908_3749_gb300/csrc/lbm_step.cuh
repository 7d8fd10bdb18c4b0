// lbm_step.cuh -- device code shared by the fused step kernels (FP64/FP32 in
// lbm_core.cu, tensor-core in lbm_tc.cu): status block and kernel arguments,
// fixed-order FP64 reductions, boundary ghosts, TMA tile loads, the
// Lax-Wendroff neighbour terms and the watchdog / audit epilogue.
#pragma once

#include <cuda.h>  // CUtensorMap (the encoder is fetched at run time; libcuda is not linked)
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "coeffs.h"
#include "d2v16.cuh"
#include "dw.cuh"
#include "tma.cuh"

namespace lbmk {

using namespace d2v16;
using namespace gbtma;

constexpr unsigned long long NONE = ~0ull;
// Node tiles of X x Y nodes handled by blocks of X x TY threads, and the
// blocks per SM each launch form is compiled for: MINB for one tile per block
// (one shared-memory stage), MINB_PIPE for the persistent form (two stages).
// FP32: 32 x 8 tiles, each thread two nodes (rows y and y + 4) in paired
// FP32 arithmetic (memory-bound: fewer instructions per node). FP64: 32 x 2
// tiles, one node per thread (FP64-ALU-bound: small tiles spread the work
// evenly over the SMs).
template <typename R> struct Shape;
// FP32 node tiles are 32 x LBM_F32_TILE_Y nodes (4, 8 or 16 rows), two rows
// per thread; the launch bounds keep 128 registers per thread (one-tile form)
// and 170 (persistent form, two tile stages).
#ifndef LBM_F32_TILE_Y
#define LBM_F32_TILE_Y 8
#endif
template <> struct Shape<float> {
  static constexpr int X = 32, Y = LBM_F32_TILE_Y, TY = Y / 2;
  static constexpr int MINB = 512 / (X * TY);
  static constexpr int MINB_PIPE = 384 / (X * TY) > 0 ? 384 / (X * TY) : 1;
  static_assert(Y == 4 || Y == 8 || Y == 16, "FP32 tile rows: 4, 8 or 16");
};
template <> struct Shape<double> {
  static constexpr int X = 32, Y = 2, TY = 2, MINB = 8, MINB_PIPE = 6;
};
// Double-word (LBM_DF64): 32 x 4 tiles of 8-byte elements (below the 48 KB
// of static shared memory), FP32-ALU-bound. LBM_DW_LANES = 1: one node per
// thread; 2: two rows per thread in paired f32x2 instructions (half the
// instructions issued, twice the registers; the FP32 units retire the same
// lanes per clock either way).
#ifndef LBM_DW_LANES
#define LBM_DW_LANES 1
#endif
// Blocks per SM of the one-tile double-word form (4: 128 registers, no
// spills; 5 spills in the node update).
#ifndef LBM_DW_MINB
#define LBM_DW_MINB 4
#endif
template <> struct Shape<dw> {
  static constexpr int X = 32, Y = 4, TY = Y / LBM_DW_LANES;
  static constexpr int MINB = LBM_DW_LANES == 1 ? LBM_DW_MINB : 6, MINB_PIPE = 3;
  static_assert(LBM_DW_LANES == 1 || LBM_DW_LANES == 2, "one or two nodes per thread");
};
constexpr int AUX_X = 32, AUX_Y = 8, AUX_N = AUX_X * AUX_Y;  // init / moments / audit

// Device-resident status block of one context.
// The time level and the audit phase are kept in two slots, one per
// population buffer: a step reading buffer p reads slot p, and its block 0
// writes slot 1 - p for the next step. A block learns both with two loads, no
// division and no atomic; the arrival ticket is used on audit steps only.
struct DevStatus {
  unsigned long long step[2];     // time level of buffer 0 / 1 when it is current
  int audit_phase[2];             // step mod audit_every (0 when audits are off)
  unsigned int arrive_step;       // blocks of a running audit step finished
  unsigned int arrive_audit;      // blocks finished in a standalone audit
  unsigned long long first_bad;   // first level with non-finite / rho <= 0
  unsigned long long first_negT;  // first level with T <= 0
  unsigned long long audit_count; // fused audits written so far
  int tma_timeout;                // a tile load did not complete in time
  int pad2;
  double audit_now[4];            // result of the standalone audit
  double audit_totals[LBM_AUDIT_RING][4];
  long long audit_steps[LBM_AUDIT_RING];
};

template <typename R>
struct StepArgs {
  Coeffs<R> K;
  Coeffs<float> K3;   // LBM_DF64: third words of K (K = K.h + K.l + K3); else unused
  int nx, ny;
  long long pitch, plane;
  int bc[4];          // x-, x+, y-, y+
  int split[4];       // side split into bc (s <= s0 + s1 t) and far (beyond)
  int far[4];
  R s0[4], s1[4];
  R hx, hy, dtr;      // dx, dy, dt (positions along a side, time)
  R wall[4][3];       // (u, v, T) of LBM_BC_WALL sides
  const R* geq;       // [4][16] Dirichlet ghost populations
  const float* geq3;  // LBM_DF64: their third words; else unused
  DevStatus* st;
  double* partial;    // [ntiles][4] audit scratch: one partial sum per tile
  double* gpartial;   // [ngroups][4]: the sums of groups of `agroup` tiles
  int agroup;         // tiles per audit group
  unsigned* gcount;   // [ngroups]: tiles of the group done in this audit step
  int ngroups;
  int audit_every;
  int nblocks;        // blocks of the launch
  int ntiles, tiles_x; // node tiles of the grid (x fastest)
  double area;        // dx * dy
  int slot;           // index of the buffer read by this step (0 or 1)
};

// Tiles per group of the two-level audit sums (audit_block_done).
// Tiles per group of the two-level audit sums: 256 for the FP64 step (one
// tile per block: small groups only lengthen the final sum over the
// groups), 64 for the persistent reduced-precision steps (whose blocks count
// their tiles at the end of the launch, so that the last blocks complete
// many groups at once; smaller groups are summed faster). Measured on
// 2048 x 1024: the tensor-core step 1.2 % faster with 64 than with 256, the
// FP64 step 0.08 % slower.
constexpr int AUDIT_GROUP_FP64 = 256, AUDIT_GROUP_REDUCED = 64;
constexpr int AUDIT_GROUP_MAX = 256;  // rows per warp sum of the final level
inline int audit_groups(int ntiles, int agroup) { return (ntiles + agroup - 1) / agroup; }

// FP32 -> FP64 conversion that stays inside the branch that needs it. A plain
// conversion may be hoisted above an audit-step test by the compiler, and
// conversions to FP64 run on the FP64 pipe, which is slow on GB300: hoisted,
// they cost every step (measured: 4 per node, 15-30 % of that pipe's time).
__device__ __forceinline__ double widen(float x) {
  double d;
  asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d) : "f"(x));
  return d;
}
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(dw x) { return widen(x.h) + widen(x.l); }

// ---------------------------------------------------------------------------
// Fixed-order FP64 reductions of four sums (bitwise reproducible)
// ---------------------------------------------------------------------------
// Warp sum of v[0..3] by a transposing butterfly: the first two exchange
// levels halve the number of live sums, so a lane does 6 additions instead of
// 20. Afterwards lanes 0, 8, 16, 24 hold the warp totals of sums 0, 1, 2, 3.
__device__ __forceinline__ double warp_sum4(const double v[4], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8;
  const double s0 = h16 ? v[0] : v[2], s1 = h16 ? v[1] : v[3];
  double k0 = (h16 ? v[2] : v[0]) + __shfl_xor_sync(0xffffffffu, s0, 16);
  double k1 = (h16 ? v[3] : v[1]) + __shfl_xor_sync(0xffffffffu, s1, 16);
  double k = (h8 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;
}

// The same for FP32 values, exactly to double-word accuracy on the FP32
// units: each value is an unevaluated pair h + l; an addition keeps the exact
// rounding error of the high words (TwoSum) and adds it and the low words
// into the low word, so a warp total of FP32 values carries about 48
// significant bits (errors of order 2^-48 of the summed magnitudes), and
// the FP64 units, slow on GB300, see only the warp totals.
__device__ __forceinline__ void dw_acc(float& h, float& l, float h2, float l2) {
  float s, e;
  two_sum(h, h2, s, e);
  h = s;
  l = (l + l2) + e;
}
__device__ __forceinline__ double warp_sum4_dw(const float (&h)[4], const float (&l)[4], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8;
  float k0h = h16 ? h[2] : h[0], k0l = h16 ? l[2] : l[0];
  float k1h = h16 ? h[3] : h[1], k1l = h16 ? l[3] : l[1];
  const float s0h = h16 ? h[0] : h[2], s0l = h16 ? l[0] : l[2];
  const float s1h = h16 ? h[1] : h[3], s1l = h16 ? l[1] : l[3];
  dw_acc(k0h, k0l, __shfl_xor_sync(0xffffffffu, s0h, 16), __shfl_xor_sync(0xffffffffu, s0l, 16));
  dw_acc(k1h, k1l, __shfl_xor_sync(0xffffffffu, s1h, 16), __shfl_xor_sync(0xffffffffu, s1l, 16));
  float kh = h8 ? k1h : k0h, kl = h8 ? k1l : k0l;
  const float sh = h8 ? k0h : k1h, sl = h8 ? k0l : k1l;
  dw_acc(kh, kl, __shfl_xor_sync(0xffffffffu, sh, 8), __shfl_xor_sync(0xffffffffu, sl, 8));
#pragma unroll
  for (int o = 4; o > 0; o >>= 1)
    dw_acc(kh, kl, __shfl_xor_sync(0xffffffffu, kh, o), __shfl_xor_sync(0xffffffffu, kl, o));
  return widen(kh) + widen(kl);  // exact in FP64
}

// Block sum of v[0..3] (N threads); threads 0..3 return sums 0..3.
template <int N>
__device__ __forceinline__ double block_sum4(const double v[4], double (*sm)[4]) {
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const double k = warp_sum4(v, lane);
  if ((lane & 7) == 0) sm[warp][lane >> 3] = k;
  __syncthreads();
  double s = 0.0;
  if (t < 4)
    for (int w = 0; w < N / 32; ++w) s += sm[w][t];
  return s;
}

// Sum of partial[b][q] over b by all N threads of one block, in a fixed
// order: thread t takes q = t % 4 and blocks b = t/4, t/4 + N/4, ...; then a
// fixed tree. Threads 0..3 return the totals of q = 0..3.
template <int N>
__device__ __forceinline__ double final_sum4(const double* partial, int nblocks,
                                             double (*sm)[4]) {
  constexpr int G = N / 4;
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int q = t & 3, j = t >> 2;
  double s = 0.0;
#pragma unroll 4
  for (int b = j; b < nblocks; b += G) s += __ldcg(partial + 4 * b + q);
  sm[j][q] = s;
  __syncthreads();
#pragma unroll
  for (int stride = G / 2; stride > 0; stride >>= 1) {
    if (j < stride) sm[j][q] += sm[j + stride][q];
    __syncthreads();
  }
  return t < 4 ? sm[0][t] : 0.0;
}

// ---------------------------------------------------------------------------
// Boundary ghosts
// ---------------------------------------------------------------------------
template <typename R, typename Off>
__device__ __forceinline__ Cons<R> load_cons(const Coeffs<R>& K, const R* __restrict__ fin,
                                             Off plane, Off idx) {
  R f[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) f[i] = fin[i * plane + idx];
  Groups<R> d;
  transform(f, d);
  return conserved(K, d);
}

// Boundary kind of the ghost next to node `along` (its index along the side)
// at time t: the side's kind, or its far kind beyond a split.
template <typename R>
__device__ __forceinline__ int side_kind(const StepArgs<R>& A, int side, int along, R t) {
  if (!A.split[side]) return A.bc[side];
  const R s = (R(along) + R(0.5)) * (side < 2 ? A.hy : A.hx);
  return s <= A.s0[side] + A.s1[side] * t ? A.bc[side] : A.far[side];
}

// Ghost populations of boundary kind `kind` outside `side` of the node with
// conserved moments `own`. `inward()` gives the conserved moments of the next
// node inwards (EXTRAP only; called only for that kind).
template <typename R, typename InFn>
__device__ __forceinline__ void ghost_with(const StepArgs<R>& A, int side, int kind, Cons<R> own,
                                           InFn inward, R g[16]) {
  if (kind == LBM_BC_EQ) {
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = A.geq[side * 16 + i];
    return;
  }
  Cons<R> s = own;
  if (kind == LBM_BC_REFLECT) {
    if (side < 2) s.jx = -s.jx; else s.jy = -s.jy;
  } else if (kind == LBM_BC_WALL) {
    const R u = A.wall[side][0], v = A.wall[side][1], T = A.wall[side][2];
    s.jx = own.rho * u;
    s.jy = own.rho * v;
    s.e = own.rho * T + R(0.5) * own.rho * (u * u + v * v);
  } else if (kind == LBM_BC_OUTFLOW) {
    // the adjacent node's state unchanged
  } else {  // LBM_BC_EXTRAP
    const Cons<R> in = inward();
    const R r1 = recip(own.rho), r2 = recip(in.rho);
    const R u1 = own.jx * r1, v1 = own.jy * r1, u2 = in.jx * r2, v2 = in.jy * r2;
    const R T1 = own.e * r1 - R(0.5) * (u1 * u1 + v1 * v1);
    const R T2 = in.e * r2 - R(0.5) * (u2 * u2 + v2 * v2);
    R rho = R(2) * own.rho - in.rho, u = R(2) * u1 - u2, v = R(2) * v1 - v2,
      T = R(2) * T1 - T2;
    if (!(rho > R(0) && T > R(0))) {
      rho = own.rho; u = u1; v = v1; T = T1;
    }
    s.rho = rho;
    s.jx = rho * u;
    s.jy = rho * v;
    s.e = rho * T + R(0.5) * rho * (u * u + v * v);
  }
  feq(A.K, s.rho, s.jx, s.jy, s.e, g);
}

// ghost_with whose inward node is element `inward` of the global population
// buffer (`has_inward` false when the grid is one node deep that way).
template <typename R, typename Off>
__device__ __forceinline__ void ghost(const StepArgs<R>& A, const R* __restrict__ fin,
                                      Off plane, int side, int kind, Cons<R> own, Off inward,
                                      bool has_inward, R g[16]) {
  ghost_with(A, side, kind, own,
             [&]() { return has_inward ? load_cons(A.K, fin, plane, inward) : own; }, g);
}

// ---------------------------------------------------------------------------
// Tile loads: TMA (cp.async.bulk.tensor) into shared memory, mbarrier-tracked
// ---------------------------------------------------------------------------
// The populations are a 3D tensor (x: pitch, y: ny, i: 16). A block's tile is
// its BX x BY nodes plus a halo: rows y0-1 .. y0+BY, columns x0-4 .. x0+BX+3
// (4 columns instead of 1 so that the box starts on a 16-byte boundary), all
// 16 populations, landing in shared memory as [16][BY+2][BX+8]. Boxes that
// reach outside the tensor are filled with zeros; those values are never
// used (boundary nodes take ghosts, periodic wraps read global memory).
constexpr int HALO_X = 4;
template <typename R>
struct Tile {
  static constexpr int BXP = Shape<R>::X + 2 * HALO_X;
  static constexpr int ROWS = Shape<R>::Y + 2;
  static constexpr int ELEMS = 16 * ROWS * BXP;
  static constexpr unsigned BYTES = ELEMS * sizeof(R);
};
// ---------------------------------------------------------------------------
// Lax-Wendroff neighbour terms (Eq. A.1b) with boundary ghosts
// ---------------------------------------------------------------------------
// acc[i] += aW f(x-dx) + aE f(x+dx) + aS f(y-dy) + aN f(y+dy) for the node at
// tile pointer `ctr` (population i at ctr[i * PS], rows BXP apart). Interior
// nodes read the tile only; edge nodes wrap (periodic, global memory) or use
// the ghost populations of their side.
template <typename R, typename Off, int BXP>
__device__ __forceinline__ void neighbour_terms(const StepArgs<R>& A, const R* __restrict__ fin,
                                                const R* ctr, int PS, Off P, Off pitch, Off c,
                                                int x, int y, const Cons<R>& m, R t,
                                                R (&acc)[16]) {
  if (x > 0 && x < A.nx - 1 && y > 0 && y < A.ny - 1) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      R a = acc[i];
      if (has_x(i)) {
        a += A.K.aW[i] * ctr[i * PS - 1];
        a += A.K.aE[i] * ctr[i * PS + 1];
      }
      if (has_y(i)) {
        a += A.K.aS[i] * ctr[i * PS - BXP];
        a += A.K.aN[i] * ctr[i * PS + BXP];
      }
      acc[i] = a;
    }
    return;
  }
  // x- neighbour (west)
  if (x > 0) {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (has_x(i)) acc[i] += A.K.aW[i] * ctr[i * PS - 1];
  } else if (A.bc[0] == LBM_BC_PERIODIC) {
    const Off n = c + (Off)(A.nx - 1);
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (has_x(i)) acc[i] += A.K.aW[i] * fin[i * P + n];
  } else {
    R g[16];
    ghost(A, fin, P, 0, side_kind(A, 0, y, t), m, c + 1, A.nx > 1, g);
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (has_x(i)) acc[i] += A.K.aW[i] * g[i];
  }
  // x+ neighbour (east)
  if (x < A.nx - 1) {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (has_x(i)) acc[i] += A.K.aE[i] * ctr[i * PS + 1];
  } else if (A.bc[1] == LBM_BC_PERIODIC) {
    const Off n = c - (Off)(A.nx - 1);
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (has_x(i)) acc[i] += A.K.aE[i] * fin[i * P + n];
  } else {
    R g[16];
    ghost(A, fin, P, 1, side_kind(A, 1, y, t), m, c - 1, A.nx > 1, g);
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (has_x(i)) acc[i] += A.K.aE[i] * g[i];
  }
  // y- neighbour (south)
  if (y > 0) {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (has_y(i)) acc[i] += A.K.aS[i] * ctr[i * PS - BXP];
  } else if (A.bc[2] == LBM_BC_PERIODIC) {
    const Off n = c + (Off)(A.ny - 1) * pitch;
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (has_y(i)) acc[i] += A.K.aS[i] * fin[i * P + n];
  } else {
    R g[16];
    ghost(A, fin, P, 2, side_kind(A, 2, x, t), m, c + pitch, A.ny > 1, g);
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (has_y(i)) acc[i] += A.K.aS[i] * g[i];
  }
  // y+ neighbour (north)
  if (y < A.ny - 1) {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (has_y(i)) acc[i] += A.K.aN[i] * ctr[i * PS + BXP];
  } else if (A.bc[3] == LBM_BC_PERIODIC) {
    const Off n = c - (Off)(A.ny - 1) * pitch;
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (has_y(i)) acc[i] += A.K.aN[i] * fin[i * P + n];
  } else {
    R g[16];
    ghost(A, fin, P, 3, side_kind(A, 3, x, t), m, c - pitch, A.ny > 1, g);
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (has_y(i)) acc[i] += A.K.aN[i] * g[i];
  }
}

// ---------------------------------------------------------------------------
// Watchdog and audit epilogue of a step block (N threads)
// ---------------------------------------------------------------------------
// Time level of this launch and whether it audits, read by one thread at the
// start of a step block; block 0 also writes both for the next step into the
// other slot (no block of this launch reads that slot; the previous launch is
// done).
template <typename R>
__device__ __forceinline__ unsigned long long read_step(const StepArgs<R>& A, int* audit) {
  const unsigned long long step = *(volatile unsigned long long*)&A.st->step[A.slot];
  const int ph = *(volatile int*)&A.st->audit_phase[A.slot];
  *audit = A.audit_every > 0 && ph == 0;
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    A.st->step[1 - A.slot] = step + 1;
    A.st->audit_phase[1 - A.slot] = ph + 1 >= A.audit_every ? 0 : ph + 1;
  }
  return step;
}

// A block that leaves an audit step early (a wait timed out) still counts
// its tiles (`first`, first + stride, ...; one thread), so that the group and
// step counters return to zero for later audit steps (the failed step's
// totals are not valid; the step reports the timeout).
template <typename R>
__device__ __forceinline__ void audit_ticket_on_exit(const StepArgs<R>& A, bool audit, int first,
                                                     int stride) {
  if (!audit) return;
  for (int tile = first; tile < A.ntiles; tile += stride) {
    const int g = tile / A.agroup, g0 = g * A.agroup;
    const int gn = min(A.ntiles - g0, A.agroup);
    if (atomicAdd(&A.gcount[g], 1u) == (unsigned)gn - 1) {
      A.gcount[g] = 0u;
      if (atomicAdd(&A.st->arrive_step, 1u) == (unsigned)A.ngroups - 1) A.st->arrive_step = 0u;
    }
  }
}

// Watchdog: records the step as the first with a bad / T <= 0 node (one
// atomic per warp that saw one).
__device__ __forceinline__ void watchdog_flags(DevStatus* st, unsigned long long step, bool bad,
                                               bool negT) {
  const unsigned badm = __ballot_sync(0xffffffffu, bad);
  const unsigned negm = __ballot_sync(0xffffffffu, negT);
  if ((threadIdx.x & 31) == 0) {
    if (badm) atomicMin(&st->first_bad, step);
    if (negm) atomicMin(&st->first_negT, step);
  }
}

// Audit steps, per tile, for FP32 or double-word values (h + l): warp totals
// by warp_sum4_dw, then the warps' totals in FP64 in order.
template <int N, typename R>
__device__ __forceinline__ void audit_tile_dw(const StepArgs<R>& A, int tile, const float (&h)[4],
                                              const float (&l)[4], double (*sm)[4]) {
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const double k = warp_sum4_dw(h, l, lane);
  if ((lane & 7) == 0) sm[warp][lane >> 3] = k;
  __syncthreads();
  if (t < 4) {
    double s = 0.0;
    for (int w = 0; w < N / 32; ++w) s += sm[w][t];
    A.partial[4 * tile + t] = s;
  }
}

// Audit steps, per tile: the block's FP64 sums of (rho, j_x, j_y, e) over the
// tile go to partial[tile]. Per tile rather than per block, so the totals do
// not depend on which block handled which tile. `v` is zero for inactive
// threads. The caller synchronises the block before `sm` is reused.
template <int N, typename R>
__device__ __forceinline__ void audit_tile(const StepArgs<R>& A, int tile, const double (&v)[4],
                                           double (*sm)[4]) {
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const double bs = block_sum4<N>(v, sm);
  if (t < 4) A.partial[4 * tile + t] = bs;
}

// Sum over a warp (fixed butterfly: every lane ends with the same value).
__device__ __forceinline__ double warp_total(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The (rho, j_x, j_y, e) sums of rows first .. first + n - 1 of p[][4] by one
// warp in a fixed order (lane l takes rows l, l + 32, ..., then the
// butterfly), whichever warp of whichever block runs it; n <= AUDIT_GROUP_MAX.
__device__ __forceinline__ void warp_sum_rows(const double* p, int first, int n, int lane,
                                              double (&out)[4]) {
  double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 8
  for (int j = lane; j < n; j += 32)
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] += __ldcg(p + 4 * (first + j) + q);
#pragma unroll
  for (int q = 0; q < 4; ++q) out[q] = warp_total(s[q]);
}

// Audit steps, once per block after its last tile (every thread calls it;
// the block's tiles are first, first + stride, ...): two levels of
// fixed-order sums, so that no warp sums more than A.agroup partials.
// The tiles are grouped by index (group g = tiles g agroup .. (g + 1)
// agroup - 1). Warp 0 counts the block's tiles into their groups'
// counters (one lane per tile, the atomics in flight together); the groups
// this block completes are summed in order into gpartial[], one warp per
// group; the warp that completes the last group sums the group sums in order
// into the audit ring. The totals do not depend on which block handled which
// tile, and no block sums every tile's partial (which took hundreds of
// microseconds on a 2048 x 1024 grid). Counters are reset by the warp that
// completes them. `s_list` (32 ints) and `s_n` are shared scratch.
template <typename R>
__device__ __forceinline__ void audit_block_done(const StepArgs<R>& A, int first, int stride,
                                                 unsigned long long step, int* s_list, int* s_n) {
  const int t = threadIdx.y * blockDim.x + threadIdx.x, lane = t & 31, warp = t >> 5;
  const int nwarps = (int)(blockDim.x * blockDim.y) >> 5;
  __syncthreads();  // the partials of the block's tiles are written
  if (warp == 0) __threadfence();
  for (int base = first; base < A.ntiles; base += 32 * stride) {
    if (warp == 0) {
      const int tile = base + lane * stride;
      int g = -1;
      if (tile < A.ntiles) {
        const int gt = tile / A.agroup, gn = min(A.ntiles - gt * A.agroup, A.agroup);
        if (atomicAdd(&A.gcount[gt], 1u) == (unsigned)gn - 1) g = gt;
      }
      const unsigned done = __ballot_sync(0xffffffffu, g >= 0);
      if (g >= 0) s_list[__popc(done & ((1u << lane) - 1u))] = g;
      if (lane == 0) *s_n = __popc(done);
    }
    __syncthreads();
    const int n = *s_n;
    if (n > 0) {
      __threadfence();  // the groups' partials, released by the blocks that wrote them
      for (int k = warp; k < n; k += nwarps) {
        const int gg = s_list[k];
        const int g0 = gg * A.agroup, gn = min(A.ntiles - g0, A.agroup);
        double s4[4];
        warp_sum_rows(A.partial, g0, gn, lane, s4);
        if (lane < 4)
          A.gpartial[4 * gg + lane] = lane == 0 ? s4[0] : lane == 1 ? s4[1] : lane == 2 ? s4[2] : s4[3];
        __syncwarp();
        int last = 0;
        if (lane == 0) {
          A.gcount[gg] = 0u;
          __threadfence();
          last = atomicAdd(&A.st->arrive_step, 1u) == (unsigned)A.ngroups - 1;
        }
        if (__shfl_sync(0xffffffffu, last, 0)) {
          __syncwarp();
          __threadfence();
          double tot[4] = {0.0, 0.0, 0.0, 0.0};
          for (int c = 0; c < A.ngroups; c += AUDIT_GROUP_MAX) {  // chunks of groups, in order
            double part[4];
            warp_sum_rows(A.gpartial, c, min(A.ngroups - c, AUDIT_GROUP_MAX), lane, part);
#pragma unroll
            for (int q = 0; q < 4; ++q) tot[q] += part[q];
          }
          const unsigned slot = (unsigned)(A.st->audit_count & (LBM_AUDIT_RING - 1));
          if (lane < 4)
            A.st->audit_totals[slot][lane] =
                (lane == 0 ? tot[0] : lane == 1 ? tot[1] : lane == 2 ? tot[2] : tot[3]) * A.area;
          __syncwarp();
          if (lane == 0) {
            A.st->audit_steps[slot] = (long long)step;
            A.st->audit_count += 1;
            A.st->arrive_step = 0u;
          }
        }
      }
    }
    __syncthreads();  // s_list and s_n are reused in the next round
  }
}

// Audit partial of a tile whose threads each hold two nodes (rows y and
// y + BYD/2), FP32 or double-word values (h + l): the thread's two nodes
// added exactly to double-word accuracy, the warp totals by warp_sum4_dw,
// then the warps (rows 0 .. BYD/2 - 1) in FP64 in order.
template <int BXD, int BYD, typename R>
__device__ __forceinline__ void audit_pair_rows(const StepArgs<R>& A, int cur,
                                                const float (&ha)[4], const float (&la)[4],
                                                const float (&hb)[4], const float (&lb)[4],
                                                double (*sm)[4]) {
  constexpr int HY = BYD / 2;
  const int lane = threadIdx.x;
  float h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    h[q] = ha[q];
    l[q] = la[q];
    dw_acc(h[q], l[q], hb[q], lb[q]);
  }
  const double k = warp_sum4_dw(h, l, lane);
  if ((lane & 7) == 0) sm[threadIdx.y][lane >> 3] = k;
  __syncthreads();
  const int t = threadIdx.y * BXD + threadIdx.x;
  if (t < 4) {
    double s = 0.0;
    for (int w = 0; w < HY; ++w) s += sm[w][t];
    A.partial[4 * cur + t] = s;
  }
}

// ---------------------------------------------------------------------------
// Tensor-core step (lbm_tc.cu)
// ---------------------------------------------------------------------------
constexpr int TC_X = 32, TC_Y = 8;  // nodes per tile: 32 x 8 = 256 (two per thread)
#ifndef LBM_TC_CTAS_PER_SM
#define LBM_TC_CTAS_PER_SM 3
#endif
constexpr int TC_CTAS_PER_SM = LBM_TC_CTAS_PER_SM;  // persistent CTAs per SM
cudaError_t tc_prepare();           // shared-memory attribute of the kernel
// TF32 high/low parts of M and M^-1 in the layout the kernel stages (4 x 4 KB).
void tc_prepare_constants(const double (&M)[16][16], const double (&Minv)[16][16],
                          unsigned char (&out)[4][4096]);
// Relaxation weights w_k = -dt s_k (0 for the conserved k), passed by value
// (kernel parameter space).
struct TcWeights {
  float w[16];
};
cudaError_t tc_launch(const CUtensorMap& tm, const float* fin, float* fout,
                      const StepArgs<float>& A, const unsigned char* bconst, const TcWeights& wk,
                      dim3 grid, cudaStream_t s);

// ---------------------------------------------------------------------------
// Two steps per launch (lbm_fused.cu)
// ---------------------------------------------------------------------------
size_t fused_smem_bytes();
int fused_halo_rows();  // rows of the fused kernel's tile copy (tensor-map box)
cudaError_t fused_prepare();
cudaError_t fused_launch(const CUtensorMap& tm, const float* fin, float* fout,
                         const StepArgs<float>& A, bool wide, cudaStream_t s);

}  // namespace lbmk
