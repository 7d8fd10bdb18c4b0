// lbm_tc.cu -- the fused step with the two 16 x 16 moment transforms on the
// 5th-generation tensor cores (tcgen05.mma, TMEM accumulators), precision
// LBM_TC_TF32X3 of include/lbm.h.
//
// Persistent CTAs of 128 threads (4 warps, TC_CTAS_PER_SM per SM), each taking
// node tiles b, b + G, b + 2G, ... (G CTAs); a tile is 32 x 4 = 128 nodes,
// node t of the tile is row t of the MMA and lane t of tensor memory. Once
// per CTA: 32 TMEM columns are allocated, the transform constants copied to
// shared memory and the first tile's copy started. Per tile:
//   0. TMA: the next tile and its halo into the other shared-memory stage
//      (double buffering: the copy runs under this tile's work);
//   1. wait for this tile's copy;
//   2. A = f (128 x 16) split into TF32 high and low parts (round to nearest,
//      ties away, by integer rounding of the bit pattern), written to shared
//      memory in the canonical K-major layout without swizzle;
//   3. m = f M^T: three products A_hi B_hi + A_hi B_lo + A_lo B_hi (the
//      3xTF32 split, error ~ the FP32 one), each two K = 8 MMAs issued by one
//      thread into TMEM columns 0..15 (FP32 accumulation); tcgen05.ld gives
//      every thread the 16 moments of its node;
//   4. Eq. 14 equilibria and the relaxation of Eq. 3 on the CUDA cores:
//      dm_k = -dt s_k (m_k - m_k^eq);
//   5. df = dm (M^-1)^T, the same split, into TMEM columns 16..31; ld;
//   6. Lax-Wendroff update with the tile's neighbours, ghosts at the domain
//      edge, store; audit partial of the tile on audit steps.
// Watchdog and audit epilogue once per CTA. Every wait (TMA, MMA completion)
// is bounded in time; on expiry the kernel records LBM_ERR_TIMEOUT, waits
// once more for the copies and products it issued (bounded), frees its
// tensor memory and returns.
#include "lbm_step.cuh"

#include <cstring>

namespace lbmk {
namespace {

constexpr int TC_N = TC_X * TC_Y;   // 128 nodes per CTA
constexpr int TC_BXP = TC_X + 2 * HALO_X, TC_ROWS = TC_Y + 2;
constexpr int TC_TILE = 16 * TC_ROWS * TC_BXP;
constexpr unsigned TC_TILE_BYTES = TC_TILE * 4;
constexpr unsigned TC_TMEM_COLS = 32;

// Byte offset of element (row, k) of a rows x 16 TF32 operand in the
// canonical K-major, no-swizzle layout: core matrices of 8 rows x 4 elements
// (128 contiguous bytes), 4 core matrices along K per 8-row group.
__device__ __host__ constexpr unsigned canon(int row, int k) {
  return (unsigned)((((row >> 3) * 4 + (k >> 2)) * 128) + (row & 7) * 16 + (k & 3) * 4);
}
constexpr unsigned CANON_LBO = 128;  // next core matrix along K
constexpr unsigned CANON_SBO = 512;  // next 8-row group

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading-dimension
// byte offset >> 4 (16-29), stride-dimension byte offset >> 4 (32-45), the
// fixed value 0b001 at bits 46-48, base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
  return (unsigned long long)((addr >> 4) & 0x3FFF) |
         ((unsigned long long)((CANON_LBO >> 4) & 0x3FFF) << 16) |
         ((unsigned long long)((CANON_SBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 = 2, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
constexpr unsigned TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) |
                              ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(unsigned tmem_d, unsigned long long a, unsigned long long b,
                                       unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 16 consecutive TMEM columns of this warp's 32 lanes (lane = thread).
__device__ __forceinline__ void tc_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Six MMAs: D = A_hi B_hi + A_hi B_lo + A_lo B_hi over K = 16 (two K = 8 halves).
__device__ __forceinline__ void tc_product(unsigned tmem_d, unsigned a_hi, unsigned a_lo,
                                           unsigned b_hi, unsigned b_lo) {
  const unsigned As[3] = {a_hi, a_hi, a_lo}, Bs[3] = {b_hi, b_lo, b_hi};
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int h = 0; h < 2; ++h)
      tc_mma(tmem_d, smem_desc(As[p] + h * 2 * CANON_LBO), smem_desc(Bs[p] + h * 2 * CANON_LBO),
             (p | h) ? 1u : 0u);
}

// TF32 rounding of an FP32 value (nearest, ties away from zero: half of the
// last kept bit added to the magnitude's bit pattern, the 13 low bits
// cleared): two integer operations instead of a conversion.
__device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Writes the TF32 high and low parts of v (16 values of row `row`) into the
// two operand buffers: hi = tf32(v), lo = tf32(v - hi) (v - hi is exact).
__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, int row,
                                              const float (&v)[16]) {
#pragma unroll
  for (int kq = 0; kq < 4; ++kq) {
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      h[e] = tf32_rna(v[4 * kq + e]);
      l[e] = tf32_rna(__fsub_rn(v[4 * kq + e], h[e]));
    }
    *reinterpret_cast<float4*>(hi + canon(row, 4 * kq)) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(lo + canon(row, 4 * kq)) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

struct TcSmem {
  float tile[2][TC_TILE];                      // two stages: populations + halo (TMA)
  alignas(128) unsigned char a_hi[TC_N * 64];  // 128 x 16 TF32, canonical layout
  alignas(128) unsigned char a_lo[TC_N * 64];
  alignas(128) unsigned char b[4][16 * 64];    // M hi, M lo, M^-1 hi, M^-1 lo (16 x 16)
  unsigned long long bar_tma[2], bar_mma;
  unsigned tmem_base;
  double red[TC_N / 4][4];
  unsigned long long step;
  int audit, last;
};
static_assert(TC_TILE * sizeof(float) % 128 == 0, "stages stay 128-byte aligned");

__device__ __forceinline__ void tc_load_tile(float* dst, const CUtensorMap* tmap,
                                             unsigned long long* bar, int tile, int tiles_x) {
  mbar_expect_tx(bar, TC_TILE_BYTES);
  tma_load_tile(dst, tmap, (tile % tiles_x) * TC_X - HALO_X, (tile / tiles_x) * TC_Y - 1, bar);
}

__global__ void __launch_bounds__(TC_N, TC_CTAS_PER_SM)
    k_step_tc(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ fin,
              float* __restrict__ fout, const StepArgs<float> A,
              const unsigned char* __restrict__ bconst, const float* __restrict__ wk) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5;
  const int G = (int)gridDim.x;

  if (warp == 0) {  // tensor memory: 32 columns for this CTA, for all its tiles
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&S.tmem_base)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    mbar_init(&S.bar_tma[0], 1);
    mbar_init(&S.bar_tma[1], 1);
    mbar_init(&S.bar_mma, 1);
    tc_load_tile(S.tile[0], &tmap, &S.bar_tma[0], blockIdx.x, A.tiles_x);  // grid <= ntiles
    S.step = read_step(A, &S.audit);
  }
  // transform constants into shared memory (4 KB)
  for (int i = t; i < 4 * 16 * 64 / 16; i += TC_N)
    reinterpret_cast<uint4*>(&S.b[0][0])[i] = reinterpret_cast<const uint4*>(bconst)[i];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = S.tmem_base;
  const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);
  const unsigned long long step = S.step;
  const bool audit = S.audit != 0;
  const float tnow = A.dtr * (float)step;
  const int tx = t & 31, ty = t >> 5;
  constexpr int PS = TC_ROWS * TC_BXP;
  const unsigned P = (unsigned)A.plane, pitch = (unsigned)A.pitch;

  bool bad = false, negT = false;
  unsigned mma_done = 0;  // MMA batches committed to bar_mma and waited for
  // Failure state: which waits gave up (-1: none) and what is still in flight.
  int failed = 0, wait_tma = -1, wait_next = -1, wait_mma = 0;
  int k = 0;
  for (int cur = blockIdx.x; cur < A.ntiles; cur += G, ++k) {
    const int s = k & 1;
    const bool more = cur + G < A.ntiles;
    // Stage 1 - s was released at the end of the previous tile.
    if (t == 0 && more) tc_load_tile(S.tile[1 - s], &tmap, &S.bar_tma[1 - s], cur + G, A.tiles_x);
    if (!__syncthreads_and(mbar_wait_bounded(&S.bar_tma[s], (k >> 1) & 1, TMA_WAIT_CYCLES))) {
      failed = 1;
      wait_tma = s * 2 + ((k >> 1) & 1);
      if (more) wait_next = (1 - s) * 2 + (((k + 1) >> 1) & 1);
      break;
    }
    const int x = (cur % A.tiles_x) * TC_X + tx, y = (cur / A.tiles_x) * TC_Y + ty;
    const bool active = x < A.nx && y < A.ny;
    const float* ctr = S.tile[s] + (ty + 1) * TC_BXP + tx + HALO_X;
    float f[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i] = ctr[i * PS];

    // m = f M^T on the tensor cores
    put_split(S.a_hi, S.a_lo, t, f);
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      tc_product(tmem, smem_addr(S.a_hi), smem_addr(S.a_lo), smem_addr(S.b[0]), smem_addr(S.b[1]));
      tc_commit(&S.bar_mma);
    }
    if (!__syncthreads_and(mbar_wait_bounded(&S.bar_mma, mma_done & 1, TMA_WAIT_CYCLES))) {
      failed = 1;
      wait_mma = 1;
      if (more) wait_next = (1 - s) * 2 + (((k + 1) >> 1) & 1);
      break;
    }
    ++mma_done;
    tc_fence_after();
    float m[16];
    tc_ld16(trow, m);

    // equilibria and relaxation on the CUDA cores
    Cons<float> c;
    c.rho = m[0]; c.jx = m[1]; c.jy = m[2]; c.e = m[3];
    const Eq<float> q = equilibria(c.rho, c.jx, c.jy, c.e);
    {
      const float meq[16] = {m[0], m[1], m[2], m[3], q.m5, q.m6, q.m7, q.m8, q.m9, q.m10,
                             q.m11, 0.f, q.m13, q.m14, 0.f, 0.f};
      float dm[16];
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) dm[kk] = wk[kk] * (m[kk] - meq[kk]);
      tc_fence_before();  // the tcgen05.ld above completes before A is rewritten
      put_split(S.a_hi, S.a_lo, t, dm);
      fence_async_smem();
    }
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      tc_product(tmem + 16, smem_addr(S.a_hi), smem_addr(S.a_lo), smem_addr(S.b[2]),
                 smem_addr(S.b[3]));
      tc_commit(&S.bar_mma);
    }
    if (!__syncthreads_and(mbar_wait_bounded(&S.bar_mma, mma_done & 1, TMA_WAIT_CYCLES))) {
      failed = 1;
      wait_mma = 1;
      if (more) wait_next = (1 - s) * 2 + (((k + 1) >> 1) & 1);
      break;
    }
    ++mma_done;
    tc_fence_after();
    float df[16];
    tc_ld16(trow + 16, df);

    float cons[4] = {0.f, 0.f, 0.f, 0.f};
    if (active) {
      const unsigned cidx = (unsigned)y * pitch + (unsigned)x;
      float acc[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[i] = A.K.a0[i] * f[i] + df[i];
      const bool b = !(c.rho > 0.f) ||
                     ((__float_as_uint(c.rho + c.jx + c.jy + c.e) & 0x7f800000u) == 0x7f800000u);
      bad |= b;
      negT |= !b && !(q.P > 0.f);
      cons[0] = c.rho; cons[1] = c.jx; cons[2] = c.jy; cons[3] = c.e;
      neighbour_terms<float, unsigned, TC_BXP>(A, fin, ctr, PS, P, pitch, cidx, x, y, c, tnow, acc);
#pragma unroll
      for (int i = 0; i < 16; ++i) fout[i * P + cidx] = acc[i];
    }
    if (audit) {  // per-tile partial (fixed order whatever the CTA)
      const double v[4] = {widen(cons[0]), widen(cons[1]), widen(cons[2]), widen(cons[3])};
      audit_tile<TC_N>(A, cur, v, S.red);
    }
    // stage s, the operand buffers and TMEM are free for the next tile
    tc_fence_before();
    __syncthreads();
  }

  if (failed) {
    // A copy or a product did not finish in time: record it, wait once more
    // (bounded) for what this CTA issued, free tensor memory, leave.
    if (t == 0) {
      atomicExch(&A.st->tma_timeout, 1);
      if (wait_tma >= 0) mbar_wait_bounded(&S.bar_tma[wait_tma >> 1], wait_tma & 1, TMA_WAIT_CYCLES);
      if (wait_next >= 0) mbar_wait_bounded(&S.bar_tma[wait_next >> 1], wait_next & 1, TMA_WAIT_CYCLES);
      if (wait_mma) mbar_wait_bounded(&S.bar_mma, mma_done & 1, TMA_WAIT_CYCLES);
      audit_ticket_on_exit(A, audit);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(TC_TMEM_COLS)
                   : "memory");
    return;
  }

  // free tensor memory (every tcgen05.ld of this CTA is complete)
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TC_TMEM_COLS)
                 : "memory");

  watchdog_flags(A.st, step, bad, negT);
  if (audit) audit_finish<TC_N>(A, step, S.red, &S.last);
}

}  // namespace

// Host side ------------------------------------------------------------------
namespace {

float tf32_host(float x) {  // round to nearest (ties away), 10 mantissa bits kept
  unsigned u;
  memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

}  // namespace

// Canonical-layout TF32 hi/lo parts of M and M^-1 as the K-major B operands
// (row n of B^T = row n of M for m = f M^T; row p of M^-1 for df = dm M^-T),
// 4 x 1 KB, and the relaxation weights w_k = -dt s_k (0 for k < 4).
void tc_prepare_constants(const double (&M)[16][16], const double (&Minv)[16][16],
                          unsigned char (&out)[4][1024]) {
  memset(out, 0, sizeof(out));
  for (int n = 0; n < 16; ++n)
    for (int k = 0; k < 16; ++k) {
      const float vm = (float)M[n][k], vi = (float)Minv[n][k];
      const float mh = tf32_host(vm), ih = tf32_host(vi);
      const float ml = tf32_host((float)(M[n][k] - (double)mh));
      const float il = tf32_host((float)(Minv[n][k] - (double)ih));
      const unsigned off = canon(n, k);
      memcpy(out[0] + off, &mh, 4);
      memcpy(out[1] + off, &ml, 4);
      memcpy(out[2] + off, &ih, 4);
      memcpy(out[3] + off, &il, 4);
    }
}

cudaError_t tc_prepare() {
  static_assert(sizeof(TcSmem) * TC_CTAS_PER_SM <= 220 * 1024,
                "tensor-core step: TC_CTAS_PER_SM CTAs must fit in one SM's shared memory");
  return cudaFuncSetAttribute(k_step_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(TcSmem));
}

cudaError_t tc_launch(const CUtensorMap& tm, const float* fin, float* fout,
                      const StepArgs<float>& A, const unsigned char* bconst, const float* wk,
                      dim3 grid, cudaStream_t s) {
  k_step_tc<<<grid, TC_N, sizeof(TcSmem), s>>>(tm, fin, fout, A, bconst, wk);
  return cudaGetLastError();
}

}  // namespace lbmk
