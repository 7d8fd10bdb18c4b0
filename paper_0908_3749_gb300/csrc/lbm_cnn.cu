// lbm_cnn.cu -- training and inference kernels of the coarse-grid corrector
// (include/lbm_cnn.h).
//
// Activations are BF16, pixel-major (NHWC, one image): a[p][c], p = y W + x;
// the input features stay FP32 and the first layer (4 -> 32) runs in FP32 on
// the CUDA cores. The other 3 x 3 convolutions are implicit GEMMs on the tensor cores
// (mma.sync m16n8k16, BF16 inputs, FP32 accumulation): rows are pixels, the
// reduction index k = tap * CIN + ci runs over the 9 taps and the input
// channels, columns are output channels. The weights of a layer are packed
// once per update into [COUT][K] BF16 (K contiguous, the "col" operand) for
// the forward pass and into the tap-flipped, channel-transposed [CIN][K'] for
// the input-gradient pass, which is the same GEMM run on the output
// gradients. Weight gradients are contractions over the pixels on the
// 5th-generation tensor cores (tcgen05, BF16 inputs, FP32 accumulation in
// tensor memory; the first layer's FP32 features as three BF16 parts), as
// per-CTA partials, then a fixed-order sum (reproducible). Adam keeps FP32
// master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>  // header-only; ranges cost nothing without a profiler attached

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm_cnn.h"
#include "tc05.cuh"

namespace {

constexpr int NL = LBM_CNN_LAYERS;
constexpr int CH[NL + 1] = {4, 32, 32, 32, 32, 4};
__host__ __device__ constexpr int ru(int a, int m) { return (a + m - 1) / m * m; }

__host__ __device__ constexpr int wsize(int l) { return 9 * (l == 0 ? 4 : 32) * (l == NL - 1 ? 4 : 32); }
__host__ __device__ constexpr int cin_of(int l) { return l == 0 ? 4 : 32; }
__host__ __device__ constexpr int cout_of(int l) { return l == NL - 1 ? 4 : 32; }

int param_offset(int l) {  // start of layer l in the packed parameter vector
  int o = 0;
  for (int k = 0; k < l; ++k) o += wsize(k) + cout_of(k);
  return o;
}

// ---------------------------------------------------------------------------
// Tensor-core implicit-GEMM 3 x 3 convolution
// ---------------------------------------------------------------------------
enum Epi { EPI_RELU_BF16 = 0, EPI_LINEAR_F32 = 1, EPI_MASK_BF16 = 2 };

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4],
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Two consecutive channels (k, k+1) of the patch element of pixel (y, x) for
// reduction index k (k even, CIN even so both share a tap); zero outside the
// image or beyond the real K.
template <int CIN>
__device__ __forceinline__ unsigned patch2(const __nv_bfloat16* __restrict__ in, int H, int W,
                                           bool valid, int y, int x, int k) {
  if (!valid || k >= 9 * CIN) return 0u;
  const int tap = k / CIN, ci = k - tap * CIN;
  const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
  if (yy < 0 || yy >= H || xx < 0 || xx >= W) return 0u;
  return *reinterpret_cast<const unsigned*>(in + ((long long)yy * W + xx) * CIN + ci);
}

// out[p][c] (c < COUT) = epilogue(sum_k patch(p, k) * Wt[c][k]). Each warp
// computes 16 pixels x COUTP columns; a block of 4 warps covers 64 pixels.
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(128) k_conv(const __nv_bfloat16* __restrict__ in, int H, int W,
                                              const __nv_bfloat16* __restrict__ Wt,
                                              const float* __restrict__ bias,
                                              const __nv_bfloat16* __restrict__ mask,
                                              __nv_bfloat16* __restrict__ out_bf,
                                              float* __restrict__ out_f) {
  constexpr int KP = ru(9 * CIN, 16), COUTP = ru(COUT, 8), NF = COUTP / 8, KS = KP / 16;
  __shared__ __align__(16) __nv_bfloat16 sw[COUTP * KP];
  for (int i = threadIdx.x; i < COUTP * KP / 2; i += blockDim.x)
    reinterpret_cast<unsigned*>(sw)[i] = reinterpret_cast<const unsigned*>(Wt)[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tig = lane & 3;
  const int npix = H * W;
  const int p0 = blockIdx.x * 64 + warp * 16;
  const int pa = p0 + g, pb = p0 + g + 8;
  const bool va = pa < npix, vb = pb < npix;
  const int ya = va ? pa / W : 0, xa = va ? pa - ya * W : 0;
  const int yb = vb ? pb / W : 0, xb = vb ? pb - yb * W : 0;
  float acc[NF][4];
#pragma unroll
  for (int j = 0; j < NF; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll 2
  for (int ks = 0; ks < KS; ++ks) {
    const int k0 = ks * 16 + tig * 2, k1 = k0 + 8;
    unsigned a[4];
    a[0] = patch2<CIN>(in, H, W, va, ya, xa, k0);
    a[1] = patch2<CIN>(in, H, W, vb, yb, xb, k0);
    a[2] = patch2<CIN>(in, H, W, va, ya, xa, k1);
    a[3] = patch2<CIN>(in, H, W, vb, yb, xb, k1);
#pragma unroll
    for (int j = 0; j < NF; ++j) {
      const __nv_bfloat16* col = sw + (j * 8 + g) * KP;
      const unsigned b0 = *reinterpret_cast<const unsigned*>(col + k0);
      const unsigned b1 = *reinterpret_cast<const unsigned*>(col + k1);
      mma_bf16(acc[j], a, b0, b1);
    }
  }
#pragma unroll
  for (int j = 0; j < NF; ++j) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int p = h ? pb : pa;
      if (!(h ? vb : va)) continue;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = j * 8 + tig * 2 + e;
        if (c >= COUT) continue;
        float v = acc[j][2 * h + e];
        if (EPI == EPI_RELU_BF16) {
          v = fmaxf(v + bias[c], 0.f);
          out_bf[(long long)p * COUT + c] = __float2bfloat16(v);
        } else if (EPI == EPI_LINEAR_F32) {
          out_f[(long long)p * COUT + c] = v + bias[c];
        } else {
          const float keep = __bfloat162float(mask[(long long)p * COUT + c]) > 0.f ? 1.f : 0.f;
          out_bf[(long long)p * COUT + c] = __float2bfloat16(v * keep);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Weight and bias gradients on the tensor cores (tcgen05)
// ---------------------------------------------------------------------------
// dW[tap][ci][co] = sum_p act[p + off(tap)][ci] dz[p][co] is a contraction
// over the pixels: D (M x N) = A (M x K) B (K x N) with K = the pixels, N =
// the output channels (32, or 4 padded to 16 with zero rows of B) and the
// rows m of A:
//   32-channel layers (BF16 activations): m = tap * 32 + ci, 288 rows as
//     three M = 128 tiles (taps 0-3, taps 4-7, tap 8 and 96 zero rows);
//   first layer (FP32 features, 4 channels): each feature split into three
//     BF16 parts x = x0 + x1 + x2 (x0 = bf16(x), x1 = bf16(x - x0), x2 =
//     bf16(x - x0 - x1), the differences exact in FP32; 24 significant bits
//     together), m = part * 36 + tap * 4 + ci, 108 rows of one M = 128 tile;
//     the epilogue adds the three parts' sums (x2 first), which gives the
//     contraction of the FP32 features.
// Persistent CTAs of 128 threads take chunks of WG_CHUNK pixels (WG_CHUNK /
// 16 MMA steps of K = 16): the threads gather the chunk's shifted features
// and output gradients as blocks of 8 channels x 8 consecutive pixels (eight
// 16-byte loads, one per pixel, transposed in registers by byte permutes)
// and store them in the canonical K-major layout; one thread issues the
// chunk's MMAs into the CTA's TMEM accumulators and commits them to an
// mbarrier, which every thread waits for (bounded) before the next chunk is
// gathered. At the end each thread reads its rows of the accumulators
// (tcgen05.ld) into the CTA's partial sums, with the bias gradient (sum_p
// dz[p][co], FP32, a fixed order); k_sum_partials adds the partials of all
// CTAs in a fixed order.
constexpr int WG_T = 128, WG_CHUNK = 64, WG_KS = WG_CHUNK / 16;
constexpr int WG_CTAS_PER_SM = 4;
constexpr unsigned WG_TMEM_COLS = 128;
constexpr unsigned WG_A_TILE = 128 * 16 * 2;  // one M tile x one K step, BF16 (4 KB)

template <int CIN>
__host__ __device__ constexpr int wg_mt() { return CIN == 32 ? 3 : 1; }  // M tiles

template <int CIN, int NP>
struct WgSmem {
  unsigned char a[wg_mt<CIN>() * WG_KS][WG_A_TILE];  // reused by the epilogue
  unsigned char b[WG_KS][NP * 16 * 2];                // reused for the bias sums
  unsigned long long bar;
  unsigned tmem;
};

// Byte offset of element (row, k) of a rows x 16 BF16 operand tile in the
// canonical K-major layout without swizzle (core matrices of 8 rows x 8
// elements, 128 contiguous bytes; the next core matrix along K 128 bytes on,
// the next 8-row group 256 bytes on).
__device__ __forceinline__ unsigned wg_off(int row, int k) {
  return (unsigned)((row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Transposes 8 pixels x 8 channels (v[j] = channels 0..7 of pixel j, two per
// word) into 8 rows (channels) of 8 pixels: out[c] = pixels 0..7 of channel c.
__device__ __forceinline__ void wg_transpose8(const uint4 (&v)[8], uint4 (&out)[8]) {
#pragma unroll
  for (int cp = 0; cp < 4; ++cp) {
    unsigned lo[4], hi[4];
#pragma unroll
    for (int pp = 0; pp < 4; ++pp) {
      const unsigned a = (&v[2 * pp].x)[cp], b = (&v[2 * pp + 1].x)[cp];
      lo[pp] = __byte_perm(a, b, 0x5410);  // channel 2 cp of pixels 2 pp, 2 pp + 1
      hi[pp] = __byte_perm(a, b, 0x7632);  // channel 2 cp + 1
    }
    out[2 * cp] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    out[2 * cp + 1] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  }
}

__device__ __forceinline__ float bf_lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(unsigned w) { return __uint_as_float(w & 0xFFFF0000u); }
__device__ __forceinline__ unsigned bf_bits(__nv_bfloat16 h) {
  return (unsigned)__bfloat16_as_ushort(h);
}

// The three BF16 parts of x (bit patterns).
__device__ __forceinline__ void split3(float x, unsigned (&p)[3]) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h0);
  const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
  const __nv_bfloat16 h2 = __float2bfloat16_rn(r1 - __bfloat162float(h1));
  p[0] = bf_bits(h0);
  p[1] = bf_bits(h1);
  p[2] = bf_bits(h2);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(WG_T, WG_CTAS_PER_SM)
    k_wgrad_tc(const void* __restrict__ act_, const __nv_bfloat16* __restrict__ dz, int H, int W,
               float* __restrict__ partial) {
  constexpr int NP = COUT == 32 ? 32 : 16;  // N of the MMA
  constexpr int MT = wg_mt<CIN>();
  constexpr int ROWS = CIN == 32 ? 9 * 32 : 3 * 36;  // used rows of A
  constexpr int NOUT = 9 * CIN * COUT + COUT;
  constexpr unsigned IDESC = tc05::idesc_f32acc(tc05::FMT_BF16, 128, NP);
  static_assert(CIN == 32 || (CIN == 4 && COUT == 32), "layer shapes of the corrector");
  extern __shared__ __align__(1024) unsigned char wg_raw[];
  WgSmem<CIN, NP>& S = *reinterpret_cast<WgSmem<CIN, NP>*>(wg_raw);
  const int t = threadIdx.x, warp = t >> 5;
  const int npix = H * W, nchunks = (npix + WG_CHUNK - 1) / WG_CHUNK;
  if (warp == 0) tc05::alloc(&S.tmem, WG_TMEM_COLS);
  if (t == 0) gbtma::mbar_init(&S.bar, 1);
  // Zero the rows that no gather writes: A rows ROWS .. MT * 128 - 1 (in the
  // last M tile), B rows COUT .. NP - 1.
  constexpr int AZ = MT * 128 - ROWS, AZ0 = 128 - AZ;
  for (int i = t; i < WG_KS * AZ * 2; i += WG_T) {
    const int ks = i / (AZ * 2), r = AZ0 + (i % (AZ * 2)) / 2, half = i & 1;
    *reinterpret_cast<uint4*>(&S.a[(MT - 1) * WG_KS + ks][wg_off(r, 8 * half)]) = make_uint4(0, 0, 0, 0);
  }
  for (int i = t; i < WG_KS * (NP - COUT) * 2; i += WG_T) {
    const int ks = i / ((NP - COUT) * 2), r = COUT + (i % ((NP - COUT) * 2)) / 2, half = i & 1;
    *reinterpret_cast<uint4*>(&S.b[ks][wg_off(r, 8 * half)]) = make_uint4(0, 0, 0, 0);
  }
  tc05::fence_before();
  __syncthreads();
  tc05::fence_after();
  const unsigned tmem = S.tmem;

  float db[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // bias sums of this thread's B block
  constexpr int NBB = COUT == 32 ? 32 : 8;                 // B blocks per chunk
  unsigned done = 0;                                      // chunks whose MMAs completed
  bool ok = true;
  for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int pbase = ch * WG_CHUNK;
    if constexpr (CIN == 32) {
      // A: 288 blocks (tap, pixel group of 8, channel group of 8), channel
      // group fastest so that neighbouring threads read one pixel's 64 bytes.
      const __nv_bfloat16* act = static_cast<const __nv_bfloat16*>(act_);
      for (int q = t; q < 288; q += WG_T) {
        const int cg = q & 3, pg = (q >> 2) & 7, tap = q >> 5;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        uint4 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int p = pbase + pg * 8 + j;
          const int y = p / W, x = p - y * W, yy = y + dy, xx = x + dx;
          v[j] = (p < npix && yy >= 0 && yy < H && xx >= 0 && xx < W)
                     ? __ldg(reinterpret_cast<const uint4*>(act + ((long long)yy * W + xx) * 32 + cg * 8))
                     : make_uint4(0, 0, 0, 0);
        }
        uint4 o[8];
        wg_transpose8(v, o);
        const int mt = tap < 8 ? tap / 4 : 2, rbase = (tap < 8 ? (tap % 4) * 32 : 0) + cg * 8;
        unsigned char* tile = S.a[mt * WG_KS + pg / 2];
#pragma unroll
        for (int c = 0; c < 8; ++c)
          *reinterpret_cast<uint4*>(tile + wg_off(rbase + c, (pg & 1) * 8)) = o[c];
      }
    } else {
      // A: 72 blocks (tap, pixel group of 8): 8 pixels x 4 features, each
      // split into three BF16 parts, give rows part * 36 + tap * 4 + ci.
      const float* act = static_cast<const float*>(act_);
      if (t < 72) {
        const int pg = t & 7, tap = t >> 3;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        unsigned part[8][4][3];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int p = pbase + pg * 8 + j;
          const int y = p / W, x = p - y * W, yy = y + dy, xx = x + dx;
          const float4 v = (p < npix && yy >= 0 && yy < H && xx >= 0 && xx < W)
                               ? __ldg(reinterpret_cast<const float4*>(act + ((long long)yy * W + xx) * 4))
                               : make_float4(0.f, 0.f, 0.f, 0.f);
          split3(v.x, part[j][0]);
          split3(v.y, part[j][1]);
          split3(v.z, part[j][2]);
          split3(v.w, part[j][3]);
        }
        unsigned char* tile = S.a[pg / 2];
#pragma unroll
        for (int pt = 0; pt < 3; ++pt)
#pragma unroll
          for (int ci = 0; ci < 4; ++ci) {
            uint4 o;
            o.x = part[0][ci][pt] | (part[1][ci][pt] << 16);
            o.y = part[2][ci][pt] | (part[3][ci][pt] << 16);
            o.z = part[4][ci][pt] | (part[5][ci][pt] << 16);
            o.w = part[6][ci][pt] | (part[7][ci][pt] << 16);
            *reinterpret_cast<uint4*>(tile + wg_off(pt * 36 + tap * 4 + ci, (pg & 1) * 8)) = o;
          }
      }
    }
    // B: the output gradients of the chunk's pixels (and the bias sums).
    if (t < NBB) {
      const int pg = COUT == 32 ? t >> 2 : t, cg = COUT == 32 ? t & 3 : 0;
      unsigned char* tile = S.b[pg / 2];
      if constexpr (COUT == 32) {
        uint4 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int p = pbase + pg * 8 + j;
          v[j] = p < npix ? __ldg(reinterpret_cast<const uint4*>(dz + (long long)p * 32 + cg * 8))
                          : make_uint4(0, 0, 0, 0);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const unsigned w = (&v[j].x)[c];
            db[2 * c] += bf_lo(w);
            db[2 * c + 1] += bf_hi(w);
          }
        }
        uint4 o[8];
        wg_transpose8(v, o);
#pragma unroll
        for (int c = 0; c < 8; ++c)
          *reinterpret_cast<uint4*>(tile + wg_off(cg * 8 + c, (pg & 1) * 8)) = o[c];
      } else {
        uint2 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int p = pbase + pg * 8 + j;
          v[j] = p < npix ? __ldg(reinterpret_cast<const uint2*>(dz + (long long)p * 4))
                          : make_uint2(0, 0);
          db[0] += bf_lo(v[j].x);
          db[1] += bf_hi(v[j].x);
          db[2] += bf_lo(v[j].y);
          db[3] += bf_hi(v[j].y);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          unsigned w[4];
#pragma unroll
          for (int pp = 0; pp < 4; ++pp) {
            const unsigned a = (&v[2 * pp].x)[c >> 1], b = (&v[2 * pp + 1].x)[c >> 1];
            w[pp] = __byte_perm(a, b, (c & 1) ? 0x7632 : 0x5410);
          }
          *reinterpret_cast<uint4*>(tile + wg_off(c, (pg & 1) * 8)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
    }
    tc05::fence_async_smem();
    __syncthreads();
    if (t == 0) {
      tc05::fence_after();
#pragma unroll
      for (int ks = 0; ks < WG_KS; ++ks)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
          tc05::mma_f16(tmem + mt * NP,
                        tc05::smem_desc(gbtma::smem_addr(S.a[mt * WG_KS + ks]), 128, 256),
                        tc05::smem_desc(gbtma::smem_addr(S.b[ks]), 128, 256), IDESC,
                        (done > 0 || ks > 0) ? 1u : 0u);
      tc05::commit(&S.bar);
    }
    ok = __syncthreads_and(gbtma::mbar_wait_bounded(&S.bar, done & 1, gbtma::TMA_WAIT_CYCLES));
    if (!ok) break;
    ++done;
    tc05::fence_after();
  }
  if (!ok) {
    // The products did not complete in time: wait once more (bounded), mark
    // this CTA's partials not-a-number (the training loss turns non-finite
    // and the host reports it), free tensor memory.
    if (t == 0) gbtma::mbar_wait_bounded(&S.bar, done & 1, gbtma::TMA_WAIT_CYCLES);
    for (int i = t; i < NOUT; i += WG_T) partial[(long long)blockIdx.x * NOUT + i] = __int_as_float(0x7fc00000);
    tc05::fence_before();
    __syncthreads();
    if (warp == 0) tc05::dealloc(tmem, WG_TMEM_COLS);
    return;
  }
  float* out = partial + (long long)blockIdx.x * NOUT;
  if constexpr (CIN == 32) {
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const int row = mt * 128 + t;  // = tap * 32 + ci
#pragma unroll
      for (int cb = 0; cb < NP / 16; ++cb) {
        float v[16];
        tc05::ld16(tmem + ((unsigned)(warp * 32) << 16) + mt * NP + cb * 16, v);
        if (row < ROWS)
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (cb * 16 + c < COUT) out[row * COUT + cb * 16 + c] = done ? v[c] : 0.f;
      }
    }
  } else {
    // rows of the three parts through shared memory (the A tiles are free:
    // every product has completed), then out[r][co] = D2 + D1 + D0.
    float* sD = reinterpret_cast<float*>(S.a[0]);  // 128 x 32 FP32 = 16 KB
    static_assert(sizeof(S.a) >= 128 * 32 * sizeof(float), "epilogue scratch");
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
      float v[16];
      tc05::ld16(tmem + ((unsigned)(warp * 32) << 16) + cb * 16, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) sD[t * 32 + ((cb * 16 + c + t) & 31)] = done ? v[c] : 0.f;
    }
    __syncthreads();
    for (int i = t; i < 36 * 32; i += WG_T) {
      const int r = i >> 5, co = i & 31;
      auto at = [&](int row) { return sD[row * 32 + ((co + row) & 31)]; };
      out[r * 32 + co] = (at(72 + r) + at(36 + r)) + at(r);
    }
  }
  // bias: thread t (t < NBB) holds 8 (COUT 32) or 4 (COUT 4) channel sums of
  // pixel group pg; add the pixel groups in order.
  float* sdb = reinterpret_cast<float*>(S.b[0]);  // the B tiles are free now
  tc05::fence_before();
  __syncthreads();
  if (t < NBB)
#pragma unroll
    for (int c = 0; c < 8; ++c) sdb[t * 8 + c] = db[c];
  __syncthreads();
  if (t < COUT) {
    float s = 0.f;
    if constexpr (COUT == 32) {
      const int cg = t >> 3, c = t & 7;
      for (int pg = 0; pg < 8; ++pg) s += sdb[(pg * 4 + cg) * 8 + c];
    } else {
      for (int pg = 0; pg < 8; ++pg) s += sdb[pg * 8 + t];
    }
    out[9 * CIN * COUT + t] = s;
  }
  if (warp == 0) tc05::dealloc(tmem, WG_TMEM_COLS);
}

template <int CIN, int COUT>
constexpr size_t wg_smem() { return sizeof(WgSmem<CIN, COUT == 32 ? 32 : 16>); }

// First layer (4 -> 32 channels) in FP32 on the CUDA cores, straight from the
// FP32 input features [p][4]: 3 x 3 correlation with zero padding, bias,
// ReLU, stored BF16 [p][32] for the tensor-core layers. Keeping the input in
// FP32 keeps differences between neighbouring nodes that are below one BF16
// step of the fields (smooth regions of fine-grained coarse grids).
// w: the layer's FP32 parameters, (3, 3, 4, 32) then 32 biases.
constexpr int C0_T = 128;
__global__ void __launch_bounds__(C0_T) k_conv0(const float* __restrict__ xf, int H, int W,
                                                const float* __restrict__ w,
                                                __nv_bfloat16* __restrict__ out) {
  __shared__ float sw[9 * 4 * 32 + 32];
  for (int i = threadIdx.x; i < 9 * 4 * 32 + 32; i += C0_T) sw[i] = w[i];
  __syncthreads();
  const int p = blockIdx.x * C0_T + threadIdx.x;
  if (p >= H * W) return;
  const int y = p / W, x = p - y * W;
  float acc[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc[c] = sw[9 * 4 * 32 + c];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
    const float4 q = *reinterpret_cast<const float4*>(xf + 4 * ((long long)yy * W + xx));
    const float qi[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int ci = 0; ci < 4; ++ci)
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[c] += qi[ci] * sw[(tap * 4 + ci) * 32 + c];
  }
  __nv_bfloat16* o = out + (long long)p * 32;
#pragma unroll
  for (int c = 0; c < 32; c += 2)
    *reinterpret_cast<__nv_bfloat162*>(o + c) =
        __floats2bfloat162_rn(fmaxf(acc[c], 0.f), fmaxf(acc[c + 1], 0.f));
}

// grad[i] = sum over blocks b (in order) of partial[b][i].
__global__ void k_sum_partials(const float* __restrict__ partial, int nblocks, int n,
                               float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int b = 0; b < nblocks; ++b) s += partial[(long long)b * n + i];
  grad[i] = s;
}

// ---------------------------------------------------------------------------
// Features, loss, Adam, packing, correction, restriction
// ---------------------------------------------------------------------------
// Planes [4][H][W] (rho, u, v, T) -> features (log rho, u, v, log T) in FP32
// [p][4] and BF16 [p][4].
__global__ void k_features(const double* __restrict__ f, int npix, float* __restrict__ xf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npix) return;
  xf[4 * p] = (float)log(f[p]);
  xf[4 * p + 1] = (float)f[npix + p];
  xf[4 * p + 2] = (float)f[2 * npix + p];
  xf[4 * p + 3] = (float)log(f[3 * npix + p]);
}

// out = x + z; d = out - target; dz = 2 d / N (BF16); block partial of sum d^2.
// Per-channel output scale: the network predicts the correction of feature
// c in units of s[c] (out = x + s z).
struct Scale4 {
  float s[4];
};

// Loss per element of out - target, d: d^2 (LBM_CNN_LOSS_MSE) or |d|
// (LBM_CNN_LOSS_L1, whose gradient is sign(d), 0 at d = 0); summed per block.
__global__ void k_loss(const float* __restrict__ xf, const float* __restrict__ z,
                       const float* __restrict__ tf, int n, __nv_bfloat16* __restrict__ dz,
                       double* __restrict__ partial, const Scale4 sc, int l1) {
  __shared__ double sm[256];
  const int i = blockIdx.x * 256 + threadIdx.x;
  double s = 0.0;
  if (i < n) {
    const float k = sc.s[i & 3];
    const float d = xf[i] + k * z[i] - tf[i];
    if (l1) {
      s = fabs((double)d);
      const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
      if (dz) dz[i] = __float2bfloat16(k * sg / (float)n);
    } else {
      s = (double)d * d;
      if (dz) dz[i] = __float2bfloat16(2.f * k * d / (float)n);
    }
  }
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void k_sum_d(const double* __restrict__ partial, int n, double scale, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partial[i];
    *out = s * scale;
  }
}

__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Packs layer l's FP32 w[3][3][cin][cout] into the forward operand
// Wt[cout_p][kp] (k = tap cin + ci) and the input-gradient operand
// Wb[cin_p][kb] (k' = tap' cout + co with tap' = 8 - tap), BF16, zero padded.
__global__ void k_pack(const float* __restrict__ w, int cin, int cout, int kp, int coutp,
                       int kb, int cinp, __nv_bfloat16* __restrict__ wt,
                       __nv_bfloat16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < coutp * kp) {
    const int c = i / kp, k = i % kp;
    float val = 0.f;
    if (c < cout && k < 9 * cin) {
      const int tap = k / cin, ci = k % cin;
      val = w[(tap * cin + ci) * cout + c];
    }
    wt[i] = __float2bfloat16(val);
  }
  if (wb && i < cinp * kb) {
    const int ci = i / kb, k = i % kb;
    float val = 0.f;
    if (ci < cin && k < 9 * cout) {
      const int tp = k / cout, co = k % cout, tap = 8 - tp;
      val = w[(tap * cin + ci) * cout + co];
    }
    wb[i] = __float2bfloat16(val);
  }
}

// corrected planes from output features x + z; block partial sums of rho.
__global__ void k_apply(const float* __restrict__ xf, const float* __restrict__ z, int npix,
                        double* __restrict__ out, const double* __restrict__ coarse,
                        double* __restrict__ partial, const Scale4 sc) {
  __shared__ double sm[2][256];
  const int p = blockIdx.x * 256 + threadIdx.x;
  double r = 0.0, r0 = 0.0;
  if (p < npix) {
    const float q0 = xf[4 * p] + sc.s[0] * z[4 * p], q1 = xf[4 * p + 1] + sc.s[1] * z[4 * p + 1];
    const float q2 = xf[4 * p + 2] + sc.s[2] * z[4 * p + 2];
    const float q3 = xf[4 * p + 3] + sc.s[3] * z[4 * p + 3];
    r = exp((double)q0);
    out[p] = r;
    out[npix + p] = q1;
    out[2 * npix + p] = q2;
    out[3 * npix + p] = exp((double)q3);
    r0 = coarse[p];
    if (!isfinite(r + q1 + q2 + q3)) r = nan("");
  }
  sm[0][threadIdx.x] = r;
  sm[1][threadIdx.x] = r0;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + st];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sm[0][0];
    partial[2 * blockIdx.x + 1] = sm[1][0];
  }
}

// Block partial sums of (t - x)^2 per feature channel, [block][4].
__global__ void k_residual_sq(const float* __restrict__ xf, const float* __restrict__ tf, int npix,
                              double* __restrict__ partial) {
  __shared__ double sm[4][256];
  const int p = blockIdx.x * 256 + threadIdx.x;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double d = p < npix ? (double)tf[4 * p + c] - (double)xf[4 * p + c] : 0.0;
    sm[c][threadIdx.x] = d * d;
  }
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
#pragma unroll
      for (int c = 0; c < 4; ++c) sm[c][threadIdx.x] += sm[c][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < 4) partial[4 * blockIdx.x + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void k_restrict(const double* __restrict__ f, int Hf, int Wf, int r,
                           double* __restrict__ c) {
  const int Hc = Hf / r, Wc = Wf / r;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Hc * Wc) return;
  const int Y = p / Wc, X = p % Wc;
  const long long nf = (long long)Hf * Wf;
  double R = 0, JX = 0, JY = 0, E = 0;
  for (int a = 0; a < r; ++a)
    for (int b = 0; b < r; ++b) {
      const long long q = (long long)(Y * r + a) * Wf + (X * r + b);
      const double rho = f[q], u = f[nf + q], v = f[2 * nf + q], T = f[3 * nf + q];
      R += rho;
      JX += rho * u;
      JY += rho * v;
      E += rho * T + 0.5 * rho * (u * u + v * v);
    }
  const double inv = 1.0 / (r * r);
  R *= inv; JX *= inv; JY *= inv; E *= inv;
  const double U = JX / R, V = JY / R;
  const long long nc = (long long)Hc * Wc;
  c[p] = R;
  c[nc + p] = U;
  c[2 * nc + p] = V;
  c[3 * nc + p] = E / R - 0.5 * (U * U + V * V);
}

thread_local std::string g_cnn_error = "no error";

}  // namespace

struct lbm_cnn {
  int H = 0, W = 0, npix = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float* w = nullptr;        // FP32 master parameters (packed)
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* wt[NL] = {};
  __nv_bfloat16* wb[NL] = {};
  __nv_bfloat16* act[NL] = {};  // act[l] = relu output of layer l-1 (act[0] unused)
  __nv_bfloat16* dz[2] = {};    // ping-pong output gradients
  float* xf = nullptr;          // input features FP32 [p][4]
  float* tf = nullptr;          // target features FP32 [p][4]
  float* z = nullptr;           // last layer output FP32 [p][4]
  float* wpartial = nullptr;    // weight-gradient partials
  double* dpart = nullptr;      // loss / mass partials
  double* dloss = nullptr;
  int wblocks = 0;              // persistent CTAs of the weight gradients
  long long step = 0;
  float lr = 1e-3f, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  Scale4 scale = {{1.f, 1.f, 1.f, 1.f}};
  int loss_kind = LBM_CNN_LOSS_MSE;
  std::string err = "no error";
};

namespace {

int cfail(lbm_cnn* n, int code, const std::string& msg) {
  if (n) n->err = msg; else g_cnn_error = msg;
  return code;
}
#define CCK(n, call)                                                              \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return cfail(n, e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, \
                   std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

int kp_of(int l) { return ru(9 * cin_of(l), 16); }
int kb_of(int l) { return ru(9 * cout_of(l), 16); }

int pack_all(lbm_cnn* n) {
  for (int l = 0; l < NL; ++l) {
    const int cin = cin_of(l), cout = cout_of(l);
    const int kp = kp_of(l), coutp = ru(cout, 8), kb = kb_of(l), cinp = ru(cin, 8);
    const int total = std::max(coutp * kp, cinp * kb);
    k_pack<<<(total + 255) / 256, 256, 0, n->stream>>>(n->w + param_offset(l), cin, cout, kp,
                                                        coutp, kb, cinp, n->wt[l], n->wb[l]);
    CCK(n, cudaGetLastError());
  }
  return LBM_OK;
}

template <int CIN, int COUT, int EPI>
void conv(lbm_cnn* n, const __nv_bfloat16* in, const __nv_bfloat16* wt, const float* bias,
          const __nv_bfloat16* mask, __nv_bfloat16* ob, float* of) {
  k_conv<CIN, COUT, EPI><<<(n->npix + 63) / 64, 128, 0, n->stream>>>(in, n->H, n->W, wt, bias,
                                                                      mask, ob, of);
}

int forward(lbm_cnn* n, const double* coarse) {
  k_features<<<(n->npix + 255) / 256, 256, 0, n->stream>>>(coarse, n->npix, n->xf);
  const float* w = n->w;
  k_conv0<<<(n->npix + C0_T - 1) / C0_T, C0_T, 0, n->stream>>>(n->xf, n->H, n->W,
                                                               w + param_offset(0), n->act[1]);
  conv<32, 32, EPI_RELU_BF16>(n, n->act[1], n->wt[1], w + param_offset(1) + wsize(1), nullptr, n->act[2], nullptr);
  conv<32, 32, EPI_RELU_BF16>(n, n->act[2], n->wt[2], w + param_offset(2) + wsize(2), nullptr, n->act[3], nullptr);
  conv<32, 32, EPI_RELU_BF16>(n, n->act[3], n->wt[3], w + param_offset(3) + wsize(3), nullptr, n->act[4], nullptr);
  conv<32, 4, EPI_LINEAR_F32>(n, n->act[4], n->wt[4], w + param_offset(4) + wsize(4), nullptr, nullptr, n->z);
  CCK(n, cudaGetLastError());
  return LBM_OK;
}

template <int CIN, int COUT>
void wgrad(lbm_cnn* n, const void* act, const __nv_bfloat16* dzl, float* grad) {
  constexpr int NOUT = 9 * CIN * COUT + COUT;
  k_wgrad_tc<CIN, COUT><<<n->wblocks, WG_T, wg_smem<CIN, COUT>(), n->stream>>>(act, dzl, n->H,
                                                                              n->W, n->wpartial);
  k_sum_partials<<<(NOUT + 255) / 256, 256, 0, n->stream>>>(n->wpartial, n->wblocks, NOUT, grad);
}

// Loss against the target features and all gradients into n->grad.
int loss_backward(lbm_cnn* n, const double* target) {
  k_features<<<(n->npix + 255) / 256, 256, 0, n->stream>>>(target, n->npix, n->tf);
  const int nel = 4 * n->npix, nb = (nel + 255) / 256;
  k_loss<<<nb, 256, 0, n->stream>>>(n->xf, n->z, n->tf, nel, n->dz[0], n->dpart, n->scale,
                                    n->loss_kind == LBM_CNN_LOSS_L1);
  k_sum_d<<<1, 32, 0, n->stream>>>(n->dpart, nb, 1.0 / nel, n->dloss);
  float* g = n->grad;
  // layer 5 (32 -> 4): dz[0] holds d loss / d z5
  wgrad<32, 4>(n, n->act[4], n->dz[0], g + param_offset(4));
  conv<4, 32, EPI_MASK_BF16>(n, n->dz[0], n->wb[4], nullptr, n->act[4], n->dz[1], nullptr);
  wgrad<32, 32>(n, n->act[3], n->dz[1], g + param_offset(3));
  conv<32, 32, EPI_MASK_BF16>(n, n->dz[1], n->wb[3], nullptr, n->act[3], n->dz[0], nullptr);
  wgrad<32, 32>(n, n->act[2], n->dz[0], g + param_offset(2));
  conv<32, 32, EPI_MASK_BF16>(n, n->dz[0], n->wb[2], nullptr, n->act[2], n->dz[1], nullptr);
  wgrad<32, 32>(n, n->act[1], n->dz[1], g + param_offset(1));
  conv<32, 32, EPI_MASK_BF16>(n, n->dz[1], n->wb[1], nullptr, n->act[1], n->dz[0], nullptr);
  wgrad<4, 32>(n, n->xf, n->dz[0], g + param_offset(0));
  CCK(n, cudaGetLastError());
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_cnn_create(int H, int W, void* cuda_stream, lbm_cnn** out) {
  if (!out) return cfail(nullptr, LBM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (H < 1 || W < 1 || (long long)H * W > (1ll << 26))
    return cfail(nullptr, LBM_ERR_INVALID, "bad image size");
  lbm_cnn* n = new lbm_cnn();
  n->H = H;
  n->W = W;
  n->npix = H * W;
  cudaError_t e = cudaSuccess;
  if (cuda_stream) n->stream = (cudaStream_t)cuda_stream;
  else { e = cudaStreamCreate(&n->stream); n->own_stream = true; }
  const size_t P = n->npix;
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto allow = [&](const void* k, size_t bytes) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  allow((const void*)k_wgrad_tc<32, 32>, wg_smem<32, 32>());
  allow((const void*)k_wgrad_tc<32, 4>, wg_smem<32, 4>());
  allow((const void*)k_wgrad_tc<4, 32>, wg_smem<4, 32>());
  n->wblocks = (int)std::min<long long>((P + WG_CHUNK - 1) / WG_CHUNK,
                                        (long long)WG_CTAS_PER_SM * std::max(sms, 1));
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, bytes, n->stream);
  };
  A((void**)&n->w, sizeof(float) * LBM_CNN_NPARAMS);
  A((void**)&n->m, sizeof(float) * LBM_CNN_NPARAMS);
  A((void**)&n->v, sizeof(float) * LBM_CNN_NPARAMS);
  A((void**)&n->grad, sizeof(float) * LBM_CNN_NPARAMS);
  for (int l = 0; l < NL; ++l) {
    A((void**)&n->wt[l], 2 * (size_t)ru(cout_of(l), 8) * kp_of(l));
    A((void**)&n->wb[l], 2 * (size_t)ru(cin_of(l), 8) * kb_of(l));
    A((void**)&n->act[l], 2 * P * CH[l]);
  }
  A((void**)&n->dz[0], 2 * P * 32);
  A((void**)&n->dz[1], 2 * P * 32);
  A((void**)&n->xf, 4 * P * 4);
  A((void**)&n->tf, 4 * P * 4);
  A((void**)&n->z, 4 * P * 4);
  A((void**)&n->wpartial, sizeof(float) * (size_t)n->wblocks * (9 * 32 * 32 + 32));
  A((void**)&n->dpart, sizeof(double) * 2 * ((4 * P + 255) / 256 + 1));
  A((void**)&n->dloss, sizeof(double));
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) {
    g_cnn_error = std::string("lbm_cnn_create: ") + cudaGetErrorString(e);
    lbm_cnn_destroy(n);
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
  }
  if (pack_all(n) != LBM_OK) {
    g_cnn_error = n->err;
    lbm_cnn_destroy(n);
    return LBM_ERR_CUDA;
  }
  *out = n;
  return LBM_OK;
}

int lbm_cnn_destroy(lbm_cnn* n) {
  if (!n) return LBM_OK;
  if (n->stream) cudaStreamSynchronize(n->stream);
  void* ps[] = {n->w, n->m, n->v, n->grad, n->dz[0], n->dz[1], n->xf, n->tf, n->z,
                n->wpartial, n->dpart, n->dloss};
  for (void* p : ps)
    if (p) cudaFree(p);
  for (int l = 0; l < NL; ++l) {
    if (n->wt[l]) cudaFree(n->wt[l]);
    if (n->wb[l]) cudaFree(n->wb[l]);
    if (n->act[l]) cudaFree(n->act[l]);
  }
  if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
  delete n;
  return LBM_OK;
}

int lbm_cnn_set_params(lbm_cnn* n, const float* params, int on_device) {
  if (!n || !params) return cfail(n, LBM_ERR_INVALID, "NULL argument");
  CCK(n, cudaMemcpyAsync(n->w, params, sizeof(float) * LBM_CNN_NPARAMS,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, n->stream));
  CCK(n, cudaMemsetAsync(n->m, 0, sizeof(float) * LBM_CNN_NPARAMS, n->stream));
  CCK(n, cudaMemsetAsync(n->v, 0, sizeof(float) * LBM_CNN_NPARAMS, n->stream));
  n->step = 0;
  const int rc = pack_all(n);
  if (rc != LBM_OK) return rc;
  if (!on_device) CCK(n, cudaStreamSynchronize(n->stream));
  return LBM_OK;
}

int lbm_cnn_get_params(lbm_cnn* n, float* params, int on_device) {
  if (!n || !params) return cfail(n, LBM_ERR_INVALID, "NULL argument");
  CCK(n, cudaMemcpyAsync(params, n->w, sizeof(float) * LBM_CNN_NPARAMS,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->stream));
  if (!on_device) CCK(n, cudaStreamSynchronize(n->stream));
  return LBM_OK;
}

int lbm_cnn_set_adam(lbm_cnn* n, double lr, double beta1, double beta2, double eps) {
  if (!n || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return cfail(n, LBM_ERR_INVALID, "bad Adam hyper-parameters");
  n->lr = (float)lr; n->b1 = (float)beta1; n->b2 = (float)beta2; n->eps = (float)eps;
  return LBM_OK;
}

int lbm_cnn_loss_grad(lbm_cnn* n, const double* coarse, const double* target, double* loss,
                      float* grads) {
  if (!n || !coarse || !target) return cfail(n, LBM_ERR_INVALID, "NULL argument");
  nvtxRangePushA("lbm_cnn_train_step");
  struct Pop { ~Pop() { nvtxRangePop(); } } pop;
  int rc = forward(n, coarse);
  if (rc == LBM_OK) rc = loss_backward(n, target);
  if (rc != LBM_OK) return rc;
  if (loss) CCK(n, cudaMemcpyAsync(loss, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
  if (grads)
    CCK(n, cudaMemcpyAsync(grads, n->grad, sizeof(float) * LBM_CNN_NPARAMS, cudaMemcpyDeviceToHost,
                           n->stream));
  CCK(n, cudaStreamSynchronize(n->stream));
  return LBM_OK;
}

int lbm_cnn_train_step(lbm_cnn* n, const double* coarse, const double* target, double* loss) {
  if (!n || !coarse || !target) return cfail(n, LBM_ERR_INVALID, "NULL argument");
  int rc = forward(n, coarse);
  if (rc == LBM_OK) rc = loss_backward(n, target);
  if (rc != LBM_OK) return rc;
  n->step += 1;
  const float c1 = 1.f - powf(n->b1, (float)n->step), c2 = 1.f - powf(n->b2, (float)n->step);
  k_adam<<<(LBM_CNN_NPARAMS + 255) / 256, 256, 0, n->stream>>>(n->w, n->m, n->v, n->grad,
                                                               LBM_CNN_NPARAMS, n->lr, n->b1,
                                                               n->b2, n->eps, c1, c2);
  CCK(n, cudaGetLastError());
  rc = pack_all(n);
  if (rc != LBM_OK) return rc;
  if (loss) {
    CCK(n, cudaMemcpyAsync(loss, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    CCK(n, cudaStreamSynchronize(n->stream));
  }
  return LBM_OK;
}

int lbm_cnn_set_output_scale(lbm_cnn* n, const double* scale) {
  if (!n || !scale) return cfail(n, LBM_ERR_INVALID, "NULL argument");
  for (int c = 0; c < 4; ++c)
    if (!(std::isfinite(scale[c]) && scale[c] > 0.0))
      return cfail(n, LBM_ERR_INVALID, "output scales must be finite and > 0");
  for (int c = 0; c < 4; ++c) n->scale.s[c] = (float)scale[c];
  return LBM_OK;
}

int lbm_cnn_set_loss(lbm_cnn* n, int kind) {
  if (!n) return cfail(nullptr, LBM_ERR_INVALID, "NULL argument");
  if (kind != LBM_CNN_LOSS_MSE && kind != LBM_CNN_LOSS_L1)
    return cfail(n, LBM_ERR_INVALID, "unknown loss kind");
  n->loss_kind = kind;
  return LBM_OK;
}

int lbm_cnn_residual_rms(lbm_cnn* n, const double* coarse, const double* target, double* rms) {
  if (!n || !coarse || !target || !rms) return cfail(n, LBM_ERR_INVALID, "NULL argument");
  const int nb = (n->npix + 255) / 256;
  k_features<<<nb, 256, 0, n->stream>>>(coarse, n->npix, n->xf);
  k_features<<<nb, 256, 0, n->stream>>>(target, n->npix, n->tf);
  std::vector<double> part(4 * (size_t)nb);
  double* dpart = nullptr;
  CCK(n, cudaMalloc((void**)&dpart, sizeof(double) * part.size()));
  k_residual_sq<<<nb, 256, 0, n->stream>>>(n->xf, n->tf, n->npix, dpart);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part.data(), dpart, sizeof(double) * part.size(), cudaMemcpyDeviceToHost,
                        n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  cudaFree(dpart);
  CCK(n, e);
  for (int c = 0; c < 4; ++c) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[4 * b + c];
    rms[c] = std::sqrt(s / n->npix);
  }
  return LBM_OK;
}

int lbm_cnn_correct(lbm_cnn* n, const double* coarse, double* corrected, double mass_tol,
                    int* used_fallback) {
  if (!n || !coarse || !corrected) return cfail(n, LBM_ERR_INVALID, "NULL argument");
  int rc = forward(n, coarse);
  if (rc != LBM_OK) return rc;
  const int nb = (n->npix + 255) / 256;
  k_apply<<<nb, 256, 0, n->stream>>>(n->xf, n->z, n->npix, corrected, coarse, n->dpart, n->scale);
  CCK(n, cudaGetLastError());
  std::vector<double> part(2 * (size_t)nb);
  CCK(n, cudaMemcpyAsync(part.data(), n->dpart, sizeof(double) * part.size(),
                         cudaMemcpyDeviceToHost, n->stream));
  CCK(n, cudaStreamSynchronize(n->stream));
  double m1 = 0, m0 = 0;
  for (int b = 0; b < nb; ++b) { m1 += part[2 * b]; m0 += part[2 * b + 1]; }
  const bool fallback = !std::isfinite(m1) || std::fabs(m1 - m0) > mass_tol * std::fabs(m0);
  if (fallback) {
    CCK(n, cudaMemcpyAsync(corrected, coarse, sizeof(double) * 4 * n->npix,
                           cudaMemcpyDeviceToDevice, n->stream));
    CCK(n, cudaStreamSynchronize(n->stream));
  }
  if (used_fallback) *used_fallback = fallback ? 1 : 0;
  return LBM_OK;
}

int lbm_restrict(const double* fine, int Hf, int Wf, int r, double* coarse, void* cuda_stream) {
  if (!fine || !coarse || r < 1 || Hf < r || Wf < r || Hf % r || Wf % r)
    return cfail(nullptr, LBM_ERR_INVALID, "lbm_restrict: bad sizes");
  const int nc = (Hf / r) * (Wf / r);
  k_restrict<<<(nc + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(fine, Hf, Wf, r, coarse);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cfail(nullptr, LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}

const char* lbm_cnn_last_error(lbm_cnn* n) { return n ? n->err.c_str() : g_cnn_error.c_str(); }

}  // extern "C"
