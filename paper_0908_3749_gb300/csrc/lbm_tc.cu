// lbm_tc.cu -- the fused step with the two 16 x 16 moment transforms on the
// 5th-generation tensor cores (tcgen05.mma, TMEM operands and accumulators),
// precision LBM_TC_TF32X3 of include/lbm.h.
//
// Persistent CTAs of 128 threads (4 warps, TC_CTAS_PER_SM per SM), each taking
// node tiles b, b + G, b + 2G, ... (G CTAs). A tile is 32 x 8 = 256 nodes;
// thread t = (tx, ty) holds two of them, rows ty and ty + 4 (nodes a and b),
// and computes both in paired f32x2 instructions, as the FP32 step does.
// Both nodes of thread t are row t of the MMAs (lane t of tensor memory):
// the A row holds the two nodes' 16 values interleaved (K = 2j for value j of
// node a, 2j + 1 for node b: the thread's register pairs, split in pairs),
// and B (32 x 32) maps them to interleaved output columns, 2k for moment k
// of node a and 2k + 1 for node b, so that one 32-column load gives every
// thread its pairs ready for the paired arithmetic. (The other node's values
// enter each output with zero coefficients: a non-finite population of one
// node makes its partner non-finite in the same step, which the watchdog
// reports at that step either way.) Once per CTA: 128 TMEM columns are
// allocated, the transform constants copied to shared memory and the first
// tile's copy started. TMEM columns:
//   [0, 32) A high parts (node a, node b), [32, 64) A low parts,
//   [64, 96) D, interleaved.
// Per tile:
//   0. TMA: the next tile and its halo (two stages: into the other stage at
//      the start, so that the copy runs under this tile's work; one stage:
//      at the end, the other CTAs on the SM working meanwhile);
//   1. wait for this tile's copy;
//   2. A = f split into TF32 high and low parts (high: round to nearest,
//      ties away, by integer rounding of the bit pattern; low = f - high,
//      exact, whose 13 low bits the TF32 product ignores), written by each
//      thread into its own TMEM lane (tcgen05.st);
//   3. m = f M^T: three products A_hi B_hi + A_hi B_lo + A_lo B_hi (the
//      3xTF32 split), each four K = 8 MMAs with A from TMEM and B from
//      shared memory, issued by one thread; FP32 accumulation in TMEM;
//      tcgen05.ld gives every thread the 16 moments of its two nodes;
//   4. Eq. 14 equilibria and the relaxation of Eq. 3 on the CUDA cores
//      (paired): dm_k = -dt s_k (m_k - m_k^eq);
//   5. df = dm (M^-1)^T, the same split and products; ld;
//   6. Lax-Wendroff update with the tile's neighbours (paired for interior
//      pairs), ghosts at the domain edge, store; audit partial of the tile
//      on audit steps.
// Watchdog and audit epilogue once per CTA. Every wait (TMA, MMA completion)
// is bounded in time; on expiry the kernel records LBM_ERR_TIMEOUT, waits
// once more for the copies and products it issued (bounded), frees its
// tensor memory and returns.
#include "lbm_step.cuh"
#include "tc05.cuh"

#include <cstring>

namespace lbmk {
namespace {

constexpr int TC_HY = TC_Y / 2;                      // node b is TC_HY rows below node a
constexpr int TC_T = TC_X * TC_HY;                   // 128 threads
constexpr int TC_BXP = TC_X + 2 * HALO_X, TC_ROWS = TC_Y + 2;
constexpr int TC_TILE = 16 * TC_ROWS * TC_BXP;
constexpr unsigned TC_TILE_BYTES = TC_TILE * 4;
constexpr unsigned TC_TMEM_COLS = 128;
// Shared-memory stages of the tile copy: 2 (the default, with 3 CTAs per SM)
// overlaps the next tile's copy with this tile's work inside the CTA; 1
// leaves room (and tensor memory) for TC_CTAS_PER_SM = 4 CTAs, which overlap
// one another's copies instead. Measured on 2048 x 1024: 0.072 against
// 0.089 ms per step.
#ifndef LBM_TC_STAGES
#define LBM_TC_STAGES 2
#endif
constexpr int TC_STAGES = LBM_TC_STAGES;
static_assert(TC_STAGES == 1 || TC_STAGES == 2, "one or two stages");
constexpr unsigned TM_HI = 0, TM_LO = 32, TM_D = 64;  // column bases (see above)
static_assert(TC_T == 128, "one MMA row per thread");

// Byte offset of element (row, k) of a rows x 32 TF32 operand in the
// canonical K-major, no-swizzle layout: core matrices of 8 rows x 4 elements
// (128 contiguous bytes), 8 core matrices along K per 8-row group.
__device__ __host__ constexpr unsigned canon(int row, int k) {
  return (unsigned)((((row >> 3) * 8 + (k >> 2)) * 128) + (row & 7) * 16 + (k & 3) * 4);
}
constexpr unsigned CANON_LBO = 128;   // next core matrix along K
constexpr unsigned CANON_SBO = 1024;  // next 8-row group
constexpr unsigned TC_B_BYTES = 32 * 32 * 4;

__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
  return tc05::smem_desc(addr, CANON_LBO, CANON_SBO);
}
// kind::tf32, M = 128 nodes, N = 32 (16 moments x 2 nodes, interleaved).
constexpr unsigned TC_IDESC = tc05::idesc_f32acc(tc05::FMT_TF32, 128, 32);

// Twelve MMAs: D = A_hi B_hi + A_hi B_lo + A_lo B_hi over K = 32 (four
// K = 8 slices), A from TMEM.
__device__ __forceinline__ void tc_product(unsigned tmem, unsigned b_hi, unsigned b_lo) {
  const unsigned As[3] = {tmem + TM_HI, tmem + TM_HI, tmem + TM_LO}, Bs[3] = {b_hi, b_lo, b_hi};
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      tc05::mma_tf32_ta(tmem + TM_D, As[p] + 8 * q, smem_desc(Bs[p] + q * 2 * CANON_LBO), TC_IDESC,
                        (p | q) ? 1u : 0u);
}

// TF32 rounding of an FP32 value (nearest, ties away from zero: half of the
// last kept bit added to the magnitude's bit pattern, the 13 low bits
// cleared): two integer operations instead of a conversion.
__device__ __forceinline__ unsigned tf32_rna_bits(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

// The TF32 high and low parts of the two nodes' 16 values into this
// thread's lane of the A columns, interleaved: hi = tf32(v), lo = v - hi
// (exact, one paired subtraction for both nodes; the product reads its 19
// high bits).
__device__ __forceinline__ void put_split(unsigned tmem_lane, const F2 (&v)[16]) {
  unsigned h[32], l[32];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    h[2 * k] = tf32_rna_bits(v[k].v.x);
    h[2 * k + 1] = tf32_rna_bits(v[k].v.y);
    const F2 lo = v[k] - F2(__uint_as_float(h[2 * k]), __uint_as_float(h[2 * k + 1]));
    l[2 * k] = __float_as_uint(lo.v.x);
    l[2 * k + 1] = __float_as_uint(lo.v.y);
  }
  tc05::st32(tmem_lane + TM_HI, h);
  tc05::st32(tmem_lane + TM_LO, l);
  tc05::st_wait();
}

// The 16 values of both nodes, as pairs, from this thread's lane of D.
__device__ __forceinline__ void get_pair(unsigned tmem_lane, F2 (&out)[16]) {
  float r[32];
  tc05::ld32(tmem_lane + TM_D, r);
#pragma unroll
  for (int k = 0; k < 16; ++k) out[k] = F2(r[2 * k], r[2 * k + 1]);
}

struct TcSmem {
  float tile[TC_STAGES][TC_TILE];              // populations + halo (TMA)
  alignas(128) unsigned char b[4][TC_B_BYTES];  // M hi, M lo, M^-1 hi, M^-1 lo (32 x 32)
  unsigned long long bar_tma[TC_STAGES], bar_mma;
  unsigned tmem_base;
  double red[TC_Y][4];                         // audit sums of a tile's rows
  unsigned long long step;
  int audit, alist[32], an;       // audit: groups completed by this CTA
};
static_assert(TC_TILE * sizeof(float) % 128 == 0, "stages stay 128-byte aligned");

__device__ __forceinline__ void tc_load_tile(float* dst, const CUtensorMap* tmap,
                                             unsigned long long* bar, int tile, int tiles_x) {
  mbar_expect_tx(bar, TC_TILE_BYTES);
  tma_load_tile(dst, tmap, (tile % tiles_x) * TC_X - HALO_X, (tile / tiles_x) * TC_Y - 1, bar);
}

__global__ void __launch_bounds__(TC_T, TC_CTAS_PER_SM)
    k_step_tc(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ fin,
              float* __restrict__ fout, const StepArgs<float> A,
              const unsigned char* __restrict__ bconst, const TcWeights wk) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y, t = ty * TC_X + tx, warp = ty;
  const int G = (int)gridDim.x;

  if (warp == 0) tc05::alloc(&S.tmem_base, TC_TMEM_COLS);  // for all this CTA's tiles
  if (t == 0) {
    for (int i = 0; i < TC_STAGES; ++i) mbar_init(&S.bar_tma[i], 1);
    mbar_init(&S.bar_mma, 1);
    tc_load_tile(S.tile[0], &tmap, &S.bar_tma[0], blockIdx.x, A.tiles_x);  // grid <= ntiles
    S.step = read_step(A, &S.audit);
  }
  // transform constants into shared memory (16 KB)
  for (int i = t; i < 4 * (int)TC_B_BYTES / 16; i += TC_T)
    reinterpret_cast<uint4*>(&S.b[0][0])[i] = reinterpret_cast<const uint4*>(bconst)[i];
  tc05::fence_before();
  __syncthreads();
  tc05::fence_after();
  const unsigned tmem = S.tmem_base;
  const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);  // this thread's lane
  const unsigned long long step = S.step;
  const bool audit = S.audit != 0;
  const float tnow = A.dtr * (float)step;
  constexpr int PS = TC_ROWS * TC_BXP;
  const unsigned P = (unsigned)A.plane, pitch = (unsigned)A.pitch;

  bool bad = false, negT = false;
  unsigned mma_done = 0;  // MMA batches committed to bar_mma and waited for
  // Failure state: which waits gave up (-1: none) and what is still in flight.
  int failed = 0, wait_tma = -1, wait_next = -1, wait_mma = 0;
  int k = 0;
  for (int cur = blockIdx.x; cur < A.ntiles; cur += G, ++k) {
    const int s = k % TC_STAGES, ph = (k / TC_STAGES) & 1;
    const int next_wait = TC_STAGES == 2 && cur + G < A.ntiles ? (1 - s) * 2 + (((k + 1) >> 1) & 1) : -1;
    const bool more = cur + G < A.ntiles;
    // Two stages: stage 1 - s was released at the end of the previous tile.
    if (TC_STAGES == 2 && t == 0 && more)
      tc_load_tile(S.tile[1 - s], &tmap, &S.bar_tma[1 - s], cur + G, A.tiles_x);
    if (!__syncthreads_and(mbar_wait_bounded(&S.bar_tma[s], ph, TMA_WAIT_CYCLES))) {
      failed = 1;
      wait_tma = s * 2 + ph;
      wait_next = next_wait;
      break;
    }
    const int x = (cur % A.tiles_x) * TC_X + tx;
    const int ya = (cur / A.tiles_x) * TC_Y + ty, yb = ya + TC_HY;
    const bool act_a = x < A.nx && ya < A.ny, act_b = x < A.nx && yb < A.ny;  // act_b => act_a
    const float* sa = S.tile[s] + (ty + 1) * TC_BXP + tx + HALO_X;
    const float* sb = sa + TC_HY * TC_BXP;
    F2 f[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i] = F2(sa[i * PS], sb[i * PS]);

    // m = f M^T on the tensor cores
    put_split(trow, f);
    tc05::fence_before();
    __syncthreads();
    if (t == 0) {
      tc05::fence_after();
      tc_product(tmem, smem_addr(S.b[0]), smem_addr(S.b[1]));
      tc05::commit(&S.bar_mma);
    }
    if (!__syncthreads_and(mbar_wait_bounded(&S.bar_mma, mma_done & 1, TMA_WAIT_CYCLES))) {
      failed = 1;
      wait_mma = 1;
      wait_next = next_wait;
      break;
    }
    ++mma_done;
    tc05::fence_after();
    F2 m[16];
    get_pair(trow, m);

    // equilibria and relaxation on the CUDA cores (the A columns are free:
    // the products that read them have completed). A node outside the grid
    // (zeros from the copy) gets density 1, so that its relaxation stays
    // finite: its partner's products multiply it by zero coefficients.
    if (!act_a) m[0].v.x = 1.f;
    if (!act_b) m[0].v.y = 1.f;
    const Eq<F2> q = equilibria(m[0], m[1], m[2], m[3]);
    {
      F2 dm[16];
      const F2 meq[16] = {m[0], m[1], m[2], m[3], q.m5, q.m6, q.m7, q.m8, q.m9, q.m10,
                          q.m11, F2(0.0), q.m13, q.m14, F2(0.0), F2(0.0)};
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) dm[kk] = wk.w[kk] * (m[kk] - meq[kk]);
      put_split(trow, dm);
    }
    tc05::fence_before();
    __syncthreads();
    if (t == 0) {
      tc05::fence_after();
      tc_product(tmem, smem_addr(S.b[2]), smem_addr(S.b[3]));
      tc05::commit(&S.bar_mma);
    }
    if (!__syncthreads_and(mbar_wait_bounded(&S.bar_mma, mma_done & 1, TMA_WAIT_CYCLES))) {
      failed = 1;
      wait_mma = 1;
      wait_next = next_wait;
      break;
    }
    ++mma_done;
    tc05::fence_after();
    F2 acc[16];
    get_pair(trow, acc);

    float mca[4] = {0.f, 0.f, 0.f, 0.f}, mcb[4] = {0.f, 0.f, 0.f, 0.f};
    if (act_a) {
      const unsigned ca = (unsigned)ya * pitch + (unsigned)x, cb = ca + TC_HY * pitch;
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[i] = A.K.a0[i] * f[i] + acc[i];
      const bool ba = !(m[0].v.x > 0.f) || !isfinite(m[0].v.x + m[1].v.x + m[2].v.x + m[3].v.x);
      const bool bb = act_b && (!(m[0].v.y > 0.f) || !isfinite(m[0].v.y + m[1].v.y + m[2].v.y + m[3].v.y));
      bad |= ba || bb;
      negT |= (!ba && !(q.P.v.x > 0.f)) || (act_b && !bb && !(q.P.v.y > 0.f));
#pragma unroll
      for (int c = 0; c < 4; ++c) mca[c] = m[c].v.x;
      if (act_b)
#pragma unroll
        for (int c = 0; c < 4; ++c) mcb[c] = m[c].v.y;

      if (act_b && x > 0 && x < A.nx - 1 && ya > 0 && yb < A.ny - 1) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          F2 a = acc[i];
          if (has_x(i)) {
            a = A.K.aW[i] * F2(sa[i * PS - 1], sb[i * PS - 1]) + a;
            a = A.K.aE[i] * F2(sa[i * PS + 1], sb[i * PS + 1]) + a;
          }
          if (has_y(i)) {
            a = A.K.aS[i] * F2(sa[i * PS - TC_BXP], sb[i * PS - TC_BXP]) + a;
            a = A.K.aN[i] * F2(sa[i * PS + TC_BXP], sb[i * PS + TC_BXP]) + a;
          }
          fout[i * P + ca] = a.v.x;
          fout[i * P + cb] = a.v.y;
        }
      } else {
        float acc1[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) acc1[i] = acc[i].v.x;
        const Cons<float> m1 = {m[0].v.x, m[1].v.x, m[2].v.x, m[3].v.x};
        neighbour_terms<float, unsigned, TC_BXP>(A, fin, sa, PS, P, pitch, ca, x, ya, m1, tnow, acc1);
#pragma unroll
        for (int i = 0; i < 16; ++i) fout[i * P + ca] = acc1[i];
        if (act_b) {
#pragma unroll
          for (int i = 0; i < 16; ++i) acc1[i] = acc[i].v.y;
          const Cons<float> m2 = {m[0].v.y, m[1].v.y, m[2].v.y, m[3].v.y};
          neighbour_terms<float, unsigned, TC_BXP>(A, fin, sb, PS, P, pitch, cb, x, yb, m2, tnow, acc1);
#pragma unroll
          for (int i = 0; i < 16; ++i) fout[i * P + cb] = acc1[i];
        }
      }
    }
    if (audit) {  // per-tile partial (fixed order whatever the CTA)
      const float z[4] = {0.f, 0.f, 0.f, 0.f};
      audit_pair_rows<TC_X, TC_Y>(A, cur, mca, z, mcb, z, S.red);
    }
    // stage s and TMEM are free for the next tile
    tc05::fence_before();
    __syncthreads();
    if (TC_STAGES == 1 && t == 0 && more)
      tc_load_tile(S.tile[0], &tmap, &S.bar_tma[0], cur + G, A.tiles_x);
  }

  if (failed) {
    // A copy or a product did not finish in time: record it, wait once more
    // (bounded) for what this CTA issued, free tensor memory, leave.
    if (t == 0) {
      atomicExch(&A.st->tma_timeout, 1);
      if (wait_tma >= 0) mbar_wait_bounded(&S.bar_tma[wait_tma >> 1], wait_tma & 1, TMA_WAIT_CYCLES);
      if (wait_next >= 0) mbar_wait_bounded(&S.bar_tma[wait_next >> 1], wait_next & 1, TMA_WAIT_CYCLES);
      if (wait_mma) mbar_wait_bounded(&S.bar_mma, mma_done & 1, TMA_WAIT_CYCLES);
      audit_ticket_on_exit(A, audit, (int)blockIdx.x, G);
    }
    tc05::fence_before();
    __syncthreads();
    if (warp == 0) tc05::dealloc(tmem, TC_TMEM_COLS);
    return;
  }

  // free tensor memory (every tcgen05.ld of this CTA is complete)
  tc05::fence_before();
  __syncthreads();
  if (warp == 0) tc05::dealloc(tmem, TC_TMEM_COLS);

  watchdog_flags(A.st, step, bad, negT);
  if (audit) audit_block_done(A, (int)blockIdx.x, G, step, S.alist, &S.an);
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

// Canonical-layout TF32 hi/lo parts of the 32 x 32 B operands of M and
// M^-1, 4 x 4 KB. Row n of B^T (output column n = 2k + node) takes K index
// 2j + node (population or moment j of that node): the entry of row k,
// column j of M (m = f M^T) or of M^-1 (df = dm M^-T); zero for the other
// node. Relaxation weights w_k = -dt s_k are applied on the CUDA cores.
void tc_prepare_constants(const double (&M)[16][16], const double (&Minv)[16][16],
                          unsigned char (&out)[4][4096]) {
  memset(out, 0, sizeof(out));
  for (int k = 0; k < 16; ++k)
    for (int j = 0; j < 16; ++j) {
      const float vm = (float)M[k][j], vi = (float)Minv[k][j];
      const float mh = tf32_host(vm), ih = tf32_host(vi);
      const float ml = tf32_host((float)(M[k][j] - (double)mh));
      const float il = tf32_host((float)(Minv[k][j] - (double)ih));
      for (int node = 0; node < 2; ++node) {
        const unsigned off = canon(2 * k + node, 2 * j + node);
        memcpy(out[0] + off, &mh, 4);
        memcpy(out[1] + off, &ml, 4);
        memcpy(out[2] + off, &ih, 4);
        memcpy(out[3] + off, &il, 4);
      }
    }
}

cudaError_t tc_prepare() {
  static_assert(sizeof(TcSmem) * TC_CTAS_PER_SM <= 220 * 1024,
                "tensor-core step: TC_CTAS_PER_SM CTAs must fit in one SM's shared memory");
  return cudaFuncSetAttribute(k_step_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(TcSmem));
}

cudaError_t tc_launch(const CUtensorMap& tm, const float* fin, float* fout,
                      const StepArgs<float>& A, const unsigned char* bconst, const TcWeights& wk,
                      dim3 grid, cudaStream_t s) {
  k_step_tc<<<grid, dim3(TC_X, TC_HY), sizeof(TcSmem), s>>>(tm, fin, fout, A, bconst, wk);
  return cudaGetLastError();
}

}  // namespace lbmk
