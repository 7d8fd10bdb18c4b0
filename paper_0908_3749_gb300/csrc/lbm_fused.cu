// lbm_fused.cu -- two time steps of the FP32 grid step in one launch
// (temporal blocking), selected by lbm_set_fused_steps (include/lbm.h).
//
// One block of 32 x 4 threads per 32 x 8 node tile, as k_step<float>. Per
// launch, from time level n in buffer fin to level n + 2 in fout:
//   1. TMA: the tile with a halo of 2 rows and 4 columns, all 16 populations
//      (S0: rows y0-2 .. y0+9, columns x0-4 .. x0+35). On a tile that reaches
//      across a periodic side the halo positions outside the grid are then
//      filled from the wrapped positions (plain loads), so that every
//      neighbour the two steps read is in shared memory.
//   2. Step A (level n -> n+1) for the tile and a ring of one node around it
//      (S1: rows y0-1 .. y0+8, columns x0-1 .. x0+32; the ring is computed
//      again by the neighbouring tiles). Ring positions outside the grid are
//      skipped unless a periodic side wraps them.
//   3. Step B (level n+1 -> n+2) for the tile from S1, stored to fout.
// Every node update is the arithmetic of the one-step kernel (group
// transforms, conserved moments, Eq. 14 equilibria, relaxation, back-map,
// Lax-Wendroff terms of Eq. A.1 in the same order; boundary ghosts of Sec. V
// from the node's own moments or, for extrapolation, its inward neighbour in
// shared memory). Watchdog flags are taken on the input state of both
// levels; an audit on level n or n + 1 (at most one: the host does not fuse
// when audit_every = 1) uses the tile nodes' moments of that level.
#include "lbm_step.cuh"

namespace lbmk {
namespace {

constexpr int FX = Shape<float>::X, FY = Shape<float>::Y, FHY = FY / 2;
constexpr int NT = FX * FHY;                   // threads per block
constexpr int R0 = FY + 4, B0 = FX + 2 * HALO_X;  // S0 rows x columns
constexpr int R1 = FY + 2, B1 = FX + 4;           // S1 rows x columns
constexpr int PS0 = R0 * B0, PS1 = R1 * B1;       // population strides
constexpr int C0 = HALO_X, C1 = 2;                // column of x0 in S0 / S1
constexpr int RING = 2 * (FX + 2) + 2 * FY;       // ring positions
constexpr unsigned S0_BYTES = 16u * PS0 * 4u;
static_assert(RING <= NT, "one ring position per thread");
static_assert(S0_BYTES % 128 == 0, "S1 starts 128-byte aligned");

__device__ __forceinline__ int wrap(int v, int n) {
  const int r = v % n;
  return r < 0 ? r + n : r;
}

template <int PS>
__device__ __forceinline__ Cons<float> stage_cons(const Coeffs<float>& K, const float* p) {
  float f[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) f[i] = p[i * PS];
  Groups<float> d;
  transform(f, d);
  return conserved(K, d);
}

// acc += aW f(x-dx) + aE f(x+dx) + aS f(y-dy) + aN f(y+dy) for the node at
// stage pointer ctr (rows BXP apart, populations PS apart) whose grid position
// is (xm, ym): neighbours inside the grid or across a periodic side come from
// the stage, the others are ghosts of the side (extrapolation reads the
// inward node from the stage). Same order of operations as neighbour_terms.
template <int BXP, int PS>
__device__ __forceinline__ void stage_neighbours(const StepArgs<float>& A, const float* ctr, int xm,
                                                 int ym, const Cons<float>& m, float t,
                                                 float (&acc)[16]) {
  const bool px = A.bc[0] == LBM_BC_PERIODIC, py = A.bc[2] == LBM_BC_PERIODIC;
  const int sx[4] = {-1, 1, -BXP, BXP};
  const bool in[4] = {px || xm > 0, px || xm < A.nx - 1, py || ym > 0, py || ym < A.ny - 1};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const float* w = d == 0 ? A.K.aW : d == 1 ? A.K.aE : d == 2 ? A.K.aS : A.K.aN;
    if (in[d]) {
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (d < 2 ? has_x(i) : has_y(i)) acc[i] += w[i] * ctr[i * PS + sx[d]];
    } else {
      const bool has_inward = d < 2 ? A.nx > 1 : A.ny > 1;
      const float* inward = ctr - sx[d];
      float g[16];
      ghost_with(A, d, side_kind(A, d, d < 2 ? ym : xm, t), m,
                 [&]() { return has_inward ? stage_cons<PS>(A.K, inward) : m; }, g);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (d < 2 ? has_x(i) : has_y(i)) acc[i] += w[i] * g[i];
    }
  }
}

// One node (scalar FP32): the new populations into out[i * PO].
template <int BXP, int PS, int PO>
__device__ __forceinline__ void node_step(const StepArgs<float>& A, const float* ctr, int xm, int ym,
                                          float t, float* out) {
  float f[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) f[i] = ctr[i * PS];
  Groups<float> d;
  transform(f, d);
  const Cons<float> m = conserved(A.K, d);
  float acc[16];
  collide(A.K, d, m, acc);
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = A.K.a0[i] * f[i] + acc[i];
  stage_neighbours<BXP, PS>(A, ctr, xm, ym, m, t, acc);
#pragma unroll
  for (int i = 0; i < 16; ++i) out[i * PO] = acc[i];
}

// Nodes a = (x, ya) and b = (x, ya + FHY) of a tile column advanced one step
// from their stage copies sa, sb (paired FP32 arithmetic, as step_tile_x2).
// (xm, yma, ymb): grid positions; use_a / use_b: compute the node; real_a /
// real_b: the node is a grid node of this tile (watchdog and audit).
// put(node, i, value) stores population i of node a (0) or b (1).
template <int BXP, int PS, typename Put>
__device__ __forceinline__ void pair_step(const StepArgs<float>& A, const float* sa, const float* sb,
                                          int xm, int yma, int ymb, bool use_a, bool use_b,
                                          bool real_a, bool real_b, float t, Put put,
                                          float (&mca)[4], float (&mcb)[4], bool& bad,
                                          bool& negT) {
  if (!use_a) return;  // use_b implies use_a
  F2 f[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) f[i] = F2(sa[i * PS], sb[i * PS]);
  Groups<F2> d;
  transform(f, d);
  const Cons<F2> m = conserved(A.K, d);
  F2 acc[16];
  const F2 press = collide(A.K, d, m, acc);
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = A.K.a0[i] * f[i] + acc[i];
  if (real_a) {
    const bool ba = !(m.rho.v.x > 0.f) || !isfinite(m.rho.v.x + m.jx.v.x + m.jy.v.x + m.e.v.x);
    bad |= ba;
    negT |= !ba && !(press.v.x > 0.f);
    mca[0] = m.rho.v.x; mca[1] = m.jx.v.x; mca[2] = m.jy.v.x; mca[3] = m.e.v.x;
  }
  if (real_b) {
    const bool bb = !(m.rho.v.y > 0.f) || !isfinite(m.rho.v.y + m.jx.v.y + m.jy.v.y + m.e.v.y);
    bad |= bb;
    negT |= !bb && !(press.v.y > 0.f);
    mcb[0] = m.rho.v.y; mcb[1] = m.jx.v.y; mcb[2] = m.jy.v.y; mcb[3] = m.e.v.y;
  }
  const bool px = A.bc[0] == LBM_BC_PERIODIC, py = A.bc[2] == LBM_BC_PERIODIC;
  const bool inner_x = px || (xm > 0 && xm < A.nx - 1);
  const bool inner_y = py || (yma > 0 && ymb < A.ny - 1);
  if (use_b && inner_x && inner_y) {
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
      put(0, i, a.v.x);
      put(1, i, a.v.y);
    }
    return;
  }
  {
    float acc1[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc1[i] = acc[i].v.x;
    const Cons<float> m1 = {m.rho.v.x, m.jx.v.x, m.jy.v.x, m.e.v.x};
    stage_neighbours<BXP, PS>(A, sa, xm, yma, m1, t, acc1);
#pragma unroll
    for (int i = 0; i < 16; ++i) put(0, i, acc1[i]);
  }
  if (use_b) {
    float acc2[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc2[i] = acc[i].v.y;
    const Cons<float> m2 = {m.rho.v.y, m.jx.v.y, m.jy.v.y, m.e.v.y};
    stage_neighbours<BXP, PS>(A, sb, xm, ymb, m2, t, acc2);
#pragma unroll
    for (int i = 0; i < 16; ++i) put(1, i, acc2[i]);
  }
}

// Time levels and audit flags of the two steps; block 0 writes level n + 2
// and its audit phase into the other slot for the next launch.
__device__ __forceinline__ unsigned long long read_step2(const StepArgs<float>& A, int* audit0,
                                                         int* audit1) {
  const unsigned long long step = *(volatile unsigned long long*)&A.st->step[A.slot];
  const int ph = *(volatile int*)&A.st->audit_phase[A.slot];
  const int ae = A.audit_every;
  const int ph1 = ph + 1 >= ae ? 0 : ph + 1;
  *audit0 = ae > 0 && ph == 0;
  *audit1 = ae > 0 && ph1 == 0;
  if (blockIdx.x == 0) {
    A.st->step[1 - A.slot] = step + 2;
    A.st->audit_phase[1 - A.slot] = ph1 + 1 >= ae ? 0 : ph1 + 1;
  }
  return step;
}

// The tile's audit partial from the tile nodes' conserved moments, by the
// one-step kernel's reduction (audit_pair_rows), so that fused and single
// steps audit bit for bit alike.
__device__ __forceinline__ void audit_pair(const StepArgs<float>& A, int tile,
                                           const float (&mca)[4], const float (&mcb)[4],
                                           double (*sm)[4]) {
  const float z[4] = {0.f, 0.f, 0.f, 0.f};
  audit_pair_rows<FX, FY>(A, tile, mca, z, mcb, z, sm);
}

template <typename Off>
__global__ void __launch_bounds__(NT, 4)
    k_step2(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ fin,
            float* __restrict__ fout, const StepArgs<float> A) {
  extern __shared__ __align__(128) unsigned char fused_smem[];
  float* const S0 = reinterpret_cast<float*>(
      fused_smem + ((128u - (smem_addr(fused_smem) & 127u)) & 127u));
  float* const S1 = S0 + 16 * PS0;
  __shared__ double sm[NT / 4][4];
  __shared__ unsigned long long bar, s_step;
  __shared__ int s_audit0, s_audit1, s_alist[32], s_an;
  const int tx = threadIdx.x, ty = threadIdx.y, t = ty * FX + tx;
  const int tile = blockIdx.x;
  const int x0 = (tile % A.tiles_x) * FX, y0 = (tile / A.tiles_x) * FY;
  if (t == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, S0_BYTES);
    tma_load_tile(S0, &tmap, x0 - HALO_X, y0 - 2, &bar);
    s_step = read_step2(A, &s_audit0, &s_audit1);
  }
  __syncthreads();
  const bool audit0 = s_audit0 != 0, audit1 = s_audit1 != 0;
  if (!__syncthreads_and(mbar_wait_bounded(&bar, 0, TMA_WAIT_CYCLES))) {
    if (t == 0) {
      atomicExch(&A.st->tma_timeout, 1);
      mbar_wait_bounded(&bar, 0, TMA_WAIT_CYCLES);
      audit_ticket_on_exit(A, audit0 || audit1, tile, A.ntiles);
    }
    return;
  }
  const int nx = A.nx, ny = A.ny;
  const bool px = A.bc[0] == LBM_BC_PERIODIC, py = A.bc[2] == LBM_BC_PERIODIC;
  const Off P = (Off)A.plane, pitch = (Off)A.pitch;

  // 1. wrapped halo of tiles that reach across a periodic side
  if ((px && (x0 - HALO_X < 0 || x0 + FX + HALO_X > nx)) || (py && (y0 - 2 < 0 || y0 + FY + 2 > ny))) {
    for (int k = t; k < R0 * B0; k += NT) {
      const int r = k / B0, col = k - r * B0;
      const int x = x0 - HALO_X + col, y = y0 - 2 + r;
      const bool ox = x < 0 || x >= nx, oy = y < 0 || y >= ny;
      if ((!ox && !oy) || (ox && !px) || (oy && !py)) continue;
      const Off g = (Off)wrap(y, ny) * pitch + (Off)wrap(x, nx);
#pragma unroll
      for (int i = 0; i < 16; ++i) S0[i * PS0 + k] = fin[i * P + g];
    }
    __syncthreads();
  }

  // 2. step A: level n -> n + 1 into S1 (tile and ring)
  const float tA = A.dtr * (float)s_step, tB = A.dtr * (float)(s_step + 1);
  bool bad = false, negT = false;
  float mca[4] = {0.f, 0.f, 0.f, 0.f}, mcb[4] = {0.f, 0.f, 0.f, 0.f};
  const int x = x0 + tx, ya = y0 + ty, yb = ya + FHY;
  {
    const bool ux = x < nx || px;
    const bool use_a = ux && (ya < ny || py), use_b = ux && (yb < ny || py);
    const bool real_a = x < nx && ya < ny, real_b = x < nx && yb < ny;
    const float* sa = S0 + (ya - y0 + 2) * B0 + tx + C0;
    const float* sb = sa + FHY * B0;
    float* da = S1 + (ya - y0 + 1) * B1 + tx + C1;
    float* db = da + FHY * B1;
    pair_step<B0, PS0>(
        A, sa, sb, wrap(x, nx), wrap(ya, ny), wrap(yb, ny), use_a, use_b, real_a, real_b, tA,
        [&](int which, int i, float v) { (which ? db : da)[i * PS1] = v; },
        mca, mcb, bad, negT);
  }
  if (t < RING) {
    int rx, ry;
    if (t < FX + 2) { rx = x0 - 1 + t; ry = y0 - 1; }
    else if (t < 2 * (FX + 2)) { rx = x0 - 1 + (t - (FX + 2)); ry = y0 + FY; }
    else if (t < 2 * (FX + 2) + FY) { rx = x0 - 1; ry = y0 + (t - 2 * (FX + 2)); }
    else { rx = x0 + FX; ry = y0 + (t - 2 * (FX + 2) - FY); }
    const bool use = (px || (rx >= 0 && rx < nx)) && (py || (ry >= 0 && ry < ny));
    if (use)
      node_step<B0, PS0, PS1>(A, S0 + (ry - y0 + 2) * B0 + (rx - x0) + C0, wrap(rx, nx), wrap(ry, ny),
                              tA, S1 + (ry - y0 + 1) * B1 + (rx - x0) + C1);
  }
  const unsigned long long step = s_step;
  watchdog_flags(A.st, step, bad, negT);
  if (audit0) audit_pair(A, tile, mca, mcb, sm);
  __syncthreads();  // S1 complete

  // 3. step B: level n + 1 -> n + 2 from S1 into fout
  bad = false;
  negT = false;
  {
    const bool real_a = x < nx && ya < ny, real_b = x < nx && yb < ny;
    const float* sa = S1 + (ya - y0 + 1) * B1 + tx + C1;
    const float* sb = sa + FHY * B1;
    const Off ca = (Off)ya * pitch + (Off)x, cb = ca + (Off)FHY * pitch;
    float nb[4] = {0.f, 0.f, 0.f, 0.f}, nbb[4] = {0.f, 0.f, 0.f, 0.f};
    pair_step<B1, PS1>(
        A, sa, sb, x, ya, yb, real_a, real_b, real_a, real_b, tB,
        [&](int which, int i, float v) { fout[i * P + (which ? cb : ca)] = v; },
        nb, nbb, bad, negT);
    watchdog_flags(A.st, step + 1, bad, negT);
    if (audit1) audit_pair(A, tile, nb, nbb, sm);
  }
  if (audit0 || audit1)
    audit_block_done(A, tile, A.ntiles, audit0 ? step : step + 1, s_alist, &s_an);
}

}  // namespace

size_t fused_smem_bytes() { return S0_BYTES + 16u * PS1 * 4u + 128u; }
int fused_halo_rows() { return R0; }

cudaError_t fused_prepare() {
  const int b = (int)fused_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_step2<unsigned>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step2<long long>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  return e;
}

cudaError_t fused_launch(const CUtensorMap& tm, const float* fin, float* fout,
                         const StepArgs<float>& A, bool wide, cudaStream_t s) {
  const dim3 blk(FX, FHY);
  if (wide) k_step2<long long><<<A.ntiles, blk, fused_smem_bytes(), s>>>(tm, fin, fout, A);
  else k_step2<unsigned><<<A.ntiles, blk, fused_smem_bytes(), s>>>(tm, fin, fout, A);
  return cudaGetLastError();
}

}  // namespace lbmk
