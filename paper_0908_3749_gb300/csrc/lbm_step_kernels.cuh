// lbm_step_kernels.cuh -- the one-step grid kernels of the fused step
// (k_step, k_step_pipe) and the per-tile node updates they share, for the
// FP64 and FP32 paths of include/lbm.h; included by lbm_core.cu, which
// launches them (the only translation unit that includes this header).
#pragma once

#include <type_traits>

#include "lbm_dw_step.cuh"
#include "lbm_step.cuh"

namespace lbmk {

// ---------------------------------------------------------------------------
// The fused step
// ---------------------------------------------------------------------------
// A step launch covers the grid's node tiles of Shape<R>::X x Shape<R>::Y
// nodes, one thread per node, each tile and its halo copied into shared
// memory by one TMA. Two launch forms, chosen per grid by lbm_autotune:
//  k_step       one tile per block (grid = all tiles); the copy of a tile
//               overlaps other blocks' compute through the hardware's block
//               scheduling. Best for grids that fit on the device in about
//               one wave.
//  k_step_pipe  persistent: nblocks < ntiles blocks, block b takes tiles b,
//               b + nblocks, ... and copies its next tile into a second
//               shared-memory stage while it computes the current one.
// Which block computes which tile changes no result: each node's update is
// the same, and audit partials are kept per tile.
// Off: unsigned (32-bit element offsets, grids with 16 * plane < 2^32) or
// long long.
template <typename R>
__device__ __forceinline__ void load_tile(R* stage, const CUtensorMap* tmap, unsigned long long* bar,
                                          int tile, int tiles_x) {
  const int x0 = (tile % tiles_x) * Shape<R>::X, y0 = (tile / tiles_x) * Shape<R>::Y;
  mbar_expect_tx(bar, Tile<R>::BYTES);
  tma_load_tile(stage, tmap, x0 - HALO_X, y0 - 1, bar);
}

// Updates the nodes of tile `cur` from its copy in shared memory `stage`:
// group transforms, conserved moments, Eq. 14 equilibria, relaxation and
// back-map, f (1 - cx^2 - cy^2) + collision + Lax-Wendroff neighbour terms,
// store. Accumulates the watchdog flags; on audit steps writes the tile's
// partial sums (a block-wide reduction: every thread of the block calls it).
template <typename R, typename Off>
__device__ __forceinline__ void step_tile(const StepArgs<R>& A, const R* __restrict__ fin,
                                          R* __restrict__ fout, const R* stage, int cur, bool audit,
                                          R t, double (*sm)[4], bool& bad, bool& negT) {
  constexpr int BXD = Shape<R>::X, BYD = Shape<R>::Y, N = BXD * BYD;
  constexpr int BXP = Tile<R>::BXP, PS = Tile<R>::ROWS * BXP;
  const int x = (cur % A.tiles_x) * BXD + threadIdx.x;
  const int y = (cur / A.tiles_x) * BYD + threadIdx.y;
  R mc[4] = {R(0), R(0), R(0), R(0)};  // conserved moments, widened on audit steps
  if (x < A.nx && y < A.ny) {
    const Off P = (Off)A.plane, pitch = (Off)A.pitch;
    const Off c = (Off)y * pitch + (Off)x;
    const R* ctr = stage + (threadIdx.y + 1) * BXP + threadIdx.x + HALO_X;
    R f[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i] = ctr[i * PS];
    Groups<R> d;
    transform(f, d);
    const Cons<R> m = conserved(A.K, d);
    R acc[16];
    const R press = collide(A.K, d, m, acc);
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = A.K.a0[i] * f[i] + acc[i];

    const bool b = !(m.rho > R(0)) || !isfinite(m.rho + m.jx + m.jy + m.e);
    bad |= b;
    negT |= !b && !(press > R(0));
    mc[0] = m.rho; mc[1] = m.jx; mc[2] = m.jy; mc[3] = m.e;
    neighbour_terms<R, Off, BXP>(A, fin, ctr, PS, P, pitch, c, x, y, m, t, acc);
#pragma unroll
    for (int i = 0; i < 16; ++i) fout[i * P + c] = acc[i];
  }
  if (audit) {  // FP64 only on audit steps
    const double tot[4] = {widen(mc[0]), widen(mc[1]), widen(mc[2]), widen(mc[3])};
    audit_tile<N>(A, cur, tot, sm);
  }
}

// FP32 tiles: thread (tx, ty) updates nodes (x, y) and (x, y + Y/2) together
// in paired arithmetic (F2). Interior pairs take their Lax-Wendroff terms from
// shared memory in paired form; a pair with a node on the domain edge
// finishes node by node through the scalar neighbour_terms (ghosts, periodic
// wraps). Audit steps: per-tile sums of the Y rows in a fixed order (two warp
// passes, then rows 0 .. Y-1).
// MAC (precision LBM_FP32_DWMOM): the conserved moments (rho, j, e) of the
// FP32 populations, the Eq. 14 equilibria and P = rho T in double-word
// arithmetic (lbm_dw_step.cuh), rounded to FP32 only where they enter the
// FP32 relaxation; audits sum the double-word moments.
template <typename Off, bool MAC = false>
__device__ __forceinline__ void step_tile_x2(const StepArgs<float>& A, const float* __restrict__ fin,
                                             float* __restrict__ fout, const float* stage, int cur,
                                             bool audit, float t, double (*sm)[4], bool& bad,
                                             bool& negT) {
  constexpr int BXD = Shape<float>::X, BYD = Shape<float>::Y, HY = BYD / 2;
  constexpr int BXP = Tile<float>::BXP, PS = Tile<float>::ROWS * BXP;
  static_assert(Shape<float>::TY == HY, "two rows per thread");
  const int x = (cur % A.tiles_x) * BXD + threadIdx.x;
  const int ya = (cur / A.tiles_x) * BYD + threadIdx.y, yb = ya + HY;
  const bool act_a = x < A.nx && ya < A.ny, act_b = x < A.nx && yb < A.ny;  // act_b => act_a
  float mca[4] = {0.f, 0.f, 0.f, 0.f}, mcb[4] = {0.f, 0.f, 0.f, 0.f};
  dw wca[4], wcb[4];  // MAC: the double-word conserved moments for the audit
  if (act_a) {
    const Off P = (Off)A.plane, pitch = (Off)A.pitch;
    const Off ca = (Off)ya * pitch + (Off)x, cb = ca + (Off)HY * pitch;
    const float* sa = stage + (threadIdx.y + 1) * BXP + threadIdx.x + HALO_X;
    const float* sb = sa + HY * BXP;
    F2 f[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i] = F2(sa[i * PS], sb[i * PS]);
    Groups<F2> d;
    transform(f, d);
    Cons<F2> m;
    F2 acc[16];
    F2 press;
    if constexpr (MAC) {
      float2 fv[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) fv[i] = f[i].v;
      DW<float2> rho, jx, jy, e;
      dw_conserved_of(fv, rho, jx, jy, e);
      rho = dnorm(rho); jx = dnorm(jx); jy = dnorm(jy); e = dnorm(e);
      const DwEq<float2> qd = dw_equilibria(rho, jx, jy, e);
      auto r32 = [](DW<float2> v) { return F2(dnorm(v).h); };
      Eq<F2> q;
      q.m5 = r32(qd.m5); q.m6 = r32(qd.m6); q.m7 = r32(qd.m7); q.m8 = r32(qd.m8);
      q.m9 = r32(qd.m9); q.m10 = r32(qd.m10); q.m11 = r32(qd.m11); q.m13 = r32(qd.m13);
      q.m14 = r32(qd.m14); q.P = r32(qd.P);
      m.rho = F2(rho.h); m.jx = F2(jx.h); m.jy = F2(jy.h); m.e = F2(e.h);
      press = collide_q(A.K, d, q, acc);
      wca[0] = dw(rho.h.x, rho.l.x); wca[1] = dw(jx.h.x, jx.l.x);
      wca[2] = dw(jy.h.x, jy.l.x); wca[3] = dw(e.h.x, e.l.x);
      wcb[0] = dw(rho.h.y, rho.l.y); wcb[1] = dw(jx.h.y, jx.l.y);
      wcb[2] = dw(jy.h.y, jy.l.y); wcb[3] = dw(e.h.y, e.l.y);
    } else {
      m = conserved(A.K, d);
      press = collide(A.K, d, m, acc);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = A.K.a0[i] * f[i] + acc[i];

    const bool ba = !(m.rho.v.x > 0.f) || !isfinite(m.rho.v.x + m.jx.v.x + m.jy.v.x + m.e.v.x);
    const bool bb = act_b && (!(m.rho.v.y > 0.f) || !isfinite(m.rho.v.y + m.jx.v.y + m.jy.v.y + m.e.v.y));
    bad |= ba || bb;
    negT |= (!ba && !(press.v.x > 0.f)) || (act_b && !bb && !(press.v.y > 0.f));
    mca[0] = m.rho.v.x; mca[1] = m.jx.v.x; mca[2] = m.jy.v.x; mca[3] = m.e.v.x;
    if (act_b) { mcb[0] = m.rho.v.y; mcb[1] = m.jx.v.y; mcb[2] = m.jy.v.y; mcb[3] = m.e.v.y; }

    if (act_b && x > 0 && x < A.nx - 1 && ya > 0 && yb < A.ny - 1) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        F2 a = acc[i];
        if (has_x(i)) {
          a = A.K.aW[i] * F2(sa[i * PS - 1], sb[i * PS - 1]) + a;
          a = A.K.aE[i] * F2(sa[i * PS + 1], sb[i * PS + 1]) + a;
        }
        if (has_y(i)) {
          a = A.K.aS[i] * F2(sa[i * PS - BXP], sb[i * PS - BXP]) + a;
          a = A.K.aN[i] * F2(sa[i * PS + BXP], sb[i * PS + BXP]) + a;
        }
        fout[i * P + ca] = a.v.x;
        fout[i * P + cb] = a.v.y;
      }
    } else {
      float acc1[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) acc1[i] = acc[i].v.x;
      const Cons<float> m1 = {m.rho.v.x, m.jx.v.x, m.jy.v.x, m.e.v.x};
      neighbour_terms<float, Off, BXP>(A, fin, sa, PS, P, pitch, ca, x, ya, m1, t, acc1);
#pragma unroll
      for (int i = 0; i < 16; ++i) fout[i * P + ca] = acc1[i];
      if (act_b) {
#pragma unroll
        for (int i = 0; i < 16; ++i) acc1[i] = acc[i].v.y;
        const Cons<float> m2 = {m.rho.v.y, m.jx.v.y, m.jy.v.y, m.e.v.y};
        neighbour_terms<float, Off, BXP>(A, fin, sb, PS, P, pitch, cb, x, yb, m2, t, acc1);
#pragma unroll
        for (int i = 0; i < 16; ++i) fout[i * P + cb] = acc1[i];
      }
    }
  }
  if (audit) {  // double-word warp sums, FP64 across warps, only on audit steps
    float ha[4], la[4], hb[4], lb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if constexpr (MAC) {
        ha[q] = act_a ? wca[q].h : 0.f;
        la[q] = act_a ? wca[q].l : 0.f;
        hb[q] = act_b ? wcb[q].h : 0.f;
        lb[q] = act_b ? wcb[q].l : 0.f;
      } else {
        ha[q] = mca[q];
        hb[q] = mcb[q];
        la[q] = lb[q] = 0.f;
      }
    }
    audit_pair_rows<BXD, BYD>(A, cur, ha, la, hb, lb, sm);
  }
}

// VAR selects a variant of the FP32 step: 0 the plain one, 1 the one with
// double-word conserved moments and equilibria (LBM_FP32_DWMOM).
template <typename R, typename Off, int VAR>
__device__ __forceinline__ void step_any(const StepArgs<R>& A, const R* __restrict__ fin,
                                         R* __restrict__ fout, const R* stage, int cur, bool audit,
                                         R t, double (*sm)[4], bool& bad, bool& negT) {
  if constexpr (std::is_same<R, dw>::value)
    step_tile_dw<Off>(A, fin, fout, stage, cur, audit, t, sm, bad, negT);
  else if constexpr (Shape<R>::TY == Shape<R>::Y)
    step_tile<R, Off>(A, fin, fout, stage, cur, audit, t, sm, bad, negT);
  else
    step_tile_x2<Off, VAR == 1>(A, fin, fout, stage, cur, audit, t, sm, bad, negT);
}

// Blocks per SM the one-tile form is compiled for: the FP32 form with 64-bit
// offsets needs more than 128 registers (it spilled at 4 blocks per SM).
template <typename R, typename Off>
constexpr int step_minb() {
  return (sizeof(R) == 4 && sizeof(Off) == 8) ? Shape<R>::MINB - 1 : Shape<R>::MINB;
}

template <typename R, typename Off, int VAR = 0>
__global__ void __launch_bounds__(Shape<R>::X * Shape<R>::TY, (step_minb<R, Off>()))
    k_step(const __grid_constant__ CUtensorMap tmap, const R* __restrict__ fin,
           R* __restrict__ fout, const StepArgs<R> A) {
  constexpr int N = Shape<R>::X * Shape<R>::TY;
  __shared__ __align__(128) R tile[Tile<R>::ELEMS];
  __shared__ double sm[N / 4][4];
  __shared__ unsigned long long bar;
  __shared__ unsigned long long s_step;
  __shared__ int s_audit, s_alist[32], s_an;
  const int t = threadIdx.y * Shape<R>::X + threadIdx.x;
  if (t == 0) {
    // Start the tile copy first so that its latency overlaps the read of
    // the step counter.
    mbar_init(&bar, 1);
    load_tile(tile, &tmap, &bar, blockIdx.x, A.tiles_x);
    s_step = read_step(A, &s_audit);
  }
  __syncthreads();
  const bool audit = s_audit != 0;
  // Every thread waits for the tile (bounded); the block decides together.
  if (!__syncthreads_and(mbar_wait_bounded(&bar, 0, TMA_WAIT_CYCLES))) {
    // The copy did not land: record it, give it a second bounded wait so that
    // no copy is left writing into shared memory, and leave without output.
    if (t == 0) {
      atomicExch(&A.st->tma_timeout, 1);
      mbar_wait_bounded(&bar, 0, TMA_WAIT_CYCLES);
      audit_ticket_on_exit(A, audit, (int)blockIdx.x, A.ntiles);
    }
    return;
  }
  bool bad = false, negT = false;
  step_any<R, Off, VAR>(A, fin, fout, tile, blockIdx.x, audit, A.dtr * R(s_step), sm, bad, negT);
  const unsigned long long step = s_step;
  watchdog_flags(A.st, step, bad, negT);
  if (audit) audit_block_done(A, (int)blockIdx.x, A.ntiles, step, s_alist, &s_an);
}

// Two tile stages (each a multiple of 128 bytes) plus room to align the first
// to 128 bytes, as TMA destinations require.
template <typename R>
constexpr size_t pipe_smem_bytes() { return 2 * sizeof(R) * (size_t)Tile<R>::ELEMS + 128; }
static_assert(sizeof(float) * Tile<float>::ELEMS % 128 == 0, "stage size");
static_assert(sizeof(double) * Tile<double>::ELEMS % 128 == 0, "stage size");

template <typename R, typename Off, int VAR = 0>
__global__ void __launch_bounds__(Shape<R>::X * Shape<R>::TY, Shape<R>::MINB_PIPE)
    k_step_pipe(const __grid_constant__ CUtensorMap tmap, const R* __restrict__ fin,
                R* __restrict__ fout, const StepArgs<R> A) {
  constexpr int N = Shape<R>::X * Shape<R>::TY;
  extern __shared__ __align__(128) unsigned char pipe_smem[];
  R* const stages = reinterpret_cast<R*>(  // [2][Tile<R>::ELEMS], 128-byte aligned
      pipe_smem + ((128u - (smem_addr(pipe_smem) & 127u)) & 127u));
  __shared__ double sm[N / 4][4];
  __shared__ unsigned long long bar[2];
  __shared__ unsigned long long s_step;
  __shared__ int s_audit, s_alist[32], s_an;
  const int t = threadIdx.y * Shape<R>::X + threadIdx.x;
  const int G = (int)gridDim.x;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    load_tile(stages, &tmap, &bar[0], blockIdx.x, A.tiles_x);  // nblocks <= ntiles
    s_step = read_step(A, &s_audit);
  }
  __syncthreads();
  bool bad = false, negT = false;
  int k = 0;
  for (int cur = blockIdx.x; cur < A.ntiles; cur += G, ++k) {
    const int s = k & 1;
    const bool more = cur + G < A.ntiles;
    // Stage 1 - s was released at the end of the previous tile.
    if (t == 0 && more)
      load_tile(stages + (1 - s) * Tile<R>::ELEMS, &tmap, &bar[1 - s], cur + G, A.tiles_x);
    // Every thread waits for the tile (bounded); the block decides together.
    if (!__syncthreads_and(mbar_wait_bounded(&bar[s], (k >> 1) & 1, TMA_WAIT_CYCLES))) {
      // A copy did not land: record it, give the copies issued a second
      // bounded wait so that none is left writing into shared memory, leave.
      if (t == 0) {
        atomicExch(&A.st->tma_timeout, 1);
        mbar_wait_bounded(&bar[s], (k >> 1) & 1, TMA_WAIT_CYCLES);
        if (more) mbar_wait_bounded(&bar[1 - s], ((k + 1) >> 1) & 1, TMA_WAIT_CYCLES);
        audit_ticket_on_exit(A, s_audit != 0, (int)blockIdx.x, G);
      }
      return;
    }
    step_any<R, Off, VAR>(A, fin, fout, stages + s * Tile<R>::ELEMS, cur, s_audit != 0,
                     A.dtr * R(s_step), sm, bad, negT);
    __syncthreads();  // stage s and sm are free again
  }
  watchdog_flags(A.st, s_step, bad, negT);
  if (s_audit) audit_block_done(A, (int)blockIdx.x, G, s_step, s_alist, &s_an);
}

}  // namespace lbmk
