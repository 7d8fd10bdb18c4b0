// lbm_vn.cu -- linear (von Neumann) stability analysis of Sec. IV on the
// device (include/lbm_vn.h).
//
// k_vn_jacobian: one block of 16 threads per case. Thread j pushes the dual
//   number f + eps e_j through the per-node collision code of the step kernels
//   (d2v16::transform / conserved / collide) at f = f^eq(state); the
//   derivative part of the result is column j of the collision Jacobian
//   d(Delta f^coll)/df = -dt M^-1 S_hat (M - dfhat^eq/df) of Sec. IV.
// k_vn_eig: 16 threads per matrix (8 matrices per 128-thread block, each in
//   shared memory). G = diag(Lax-Wendroff symbol of Eq. A.1) + Jacobian, then
//   Householder reduction to upper Hessenberg form and explicit single-shift
//   complex QR sweeps (Wilkinson shift from the trailing 2 x 2 block,
//   exceptional shifts after 10 and 20 sweeps without deflation, deflation
//   where |h_{l,l-1}| <= u (|h_{l-1,l-1}| + |h_{l,l}|), u = 2^-52), the
//   textbook complex Schur iteration (Golub and Van Loan, Matrix
//   Computations, Secs. 7.4-7.5), in FP64. Every loop is bounded; a matrix
//   that does not converge within 30 x 16 sweeps gets NaN results.
// The 16 threads of a matrix synchronise with __syncwarp on their own
// half-warp mask, so the two matrices of a warp proceed independently.

#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/lbm_vn.h"
#include "coeffs.h"
#include "d2v16.cuh"

using namespace d2v16;

namespace {

thread_local std::string g_vn_error = "no error";

int vfail(int code, const std::string& m) {
  g_vn_error = m;
  return code;
}
int vcuda(cudaError_t e, const char* what) {
  return vfail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}
#define VCK(call)                                  \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return vcuda(e_, #call); \
  } while (0)

// ---------------------------------------------------------------------------
// Forward-mode dual numbers: (value, derivative along one direction)
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() = default;
  __device__ Dual(double x) : v(x), d(0.0) {}
  __device__ Dual(double x, double dx) : v(x), d(dx) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) {
  return Dual(a.v * b.v, a.d * b.v + a.v * b.d);
}
__device__ __forceinline__ Dual operator*(double k, Dual b) { return Dual(k * b.v, k * b.d); }
// (1/x)' = -x' / x^2
__device__ __forceinline__ Dual recip(Dual x) {
  const double r = d2v16::recip(x.v);
  return Dual(r, -x.d * r * r);
}

// Lax-Wendroff weights of Eq. A.1 per population (set_advection).
struct LW {
  double a0[16], aE[16], aW[16], aN[16], aS[16];
};

constexpr int VN_T = 128;           // threads per eigen block
constexpr int MPB = VN_T / 16;      // matrices per block
constexpr int SWEEPS_PER_EIG = 30;  // average QR sweeps allowed per eigenvalue

__global__ void __launch_bounds__(16) k_vn_jacobian(const lbm_vn_case* cases, const Coeffs<double> base,
                                                    double dt, double* Jc) {
  __shared__ Coeffs<double> K;
  const int c = blockIdx.x, j = threadIdx.x;
  const lbm_vn_case cs = cases[c];
  if (j == 0) {
    K = base;
    set_rates(K, dt, cs.s);
  }
  __syncthreads();
  bool ok = cs.rho > 0.0 && cs.T > 0.0 && isfinite(cs.rho) && isfinite(cs.T) &&
            isfinite(cs.u) && isfinite(cs.v);
  for (int k = 0; k < 16; ++k) ok = ok && isfinite(cs.s[k]);
  double* col = Jc + (size_t)c * 256;
  if (!ok) {
    for (int i = 0; i < 16; ++i) col[i * 16 + j] = nan("");
    return;
  }
  const double rho = cs.rho, jx = rho * cs.u, jy = rho * cs.v;
  const double e = rho * cs.T + 0.5 * rho * (cs.u * cs.u + cs.v * cs.v);
  double f0[16];
  feq<double, double>(K, rho, jx, jy, e, f0);
  Dual f[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) f[i] = Dual(f0[i], i == j ? 1.0 : 0.0);
  Groups<Dual> g;
  transform(f, g);
  const Cons<Dual> m = conserved(K, g);
  Dual df[16];
  collide(K, g, m, df);
#pragma unroll
  for (int i = 0; i < 16; ++i) col[i * 16 + j] = df[i].d;
}

// ---------------------------------------------------------------------------
// Complex arithmetic and the 16 x 16 eigenvalue solver
// ---------------------------------------------------------------------------
struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx mk(double r, double i) { return cplx{r, i}; }
__device__ __forceinline__ cplx operator+(cplx a, cplx b) { return mk(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ cplx operator-(cplx a, cplx b) { return mk(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cplx operator-(cplx a) { return mk(-a.re, -a.im); }
__device__ __forceinline__ cplx operator*(cplx a, cplx b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ cplx operator*(double k, cplx a) { return mk(k * a.re, k * a.im); }
__device__ __forceinline__ cplx conj(cplx a) { return mk(a.re, -a.im); }
__device__ __forceinline__ double cabs(cplx a) { return hypot(a.re, a.im); }
__device__ __forceinline__ double cabs1(cplx a) { return fabs(a.re) + fabs(a.im); }
__device__ __forceinline__ double norm2(cplx a) { return a.re * a.re + a.im * a.im; }
// a / b by scaling with the larger component of b (Smith's method).
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, den = b.re + b.im * r;
    return mk((a.re + a.im * r) / den, (a.im - a.re * r) / den);
  }
  const double r = b.re / b.im, den = b.im + b.re * r;
  return mk((a.re * r + a.im) / den, (a.im * r - a.re) / den);
}
// Principal square root: for z = x + i y, |z| = r, sqrt z = (t, y / (2 t)) with
// t = sqrt((r + x) / 2) when x >= 0, else (|y| / (2 t), sign(y) t) with
// t = sqrt((r - x) / 2).
__device__ __forceinline__ cplx csqrt(cplx z) {
  const double r = cabs(z);
  if (r == 0.0) return mk(0.0, 0.0);
  if (z.re >= 0.0) {
    const double t = sqrt(0.5 * (r + z.re));
    return mk(t, z.im / (2.0 * t));
  }
  const double t = sqrt(0.5 * (r - z.re));
  return mk(fabs(z.im) / (2.0 * t), copysign(t, z.im));
}
// Givens rotation G = [[c, s], [-conj(s), c]], c real, with G (a, b)^T = (r, 0)^T:
// c = |a| / n, s = (a / |a|) conj(b) / n, r = (a / |a|) n, n^2 = |a|^2 + |b|^2,
// from two reciprocal square roots. The solver scales its matrix to entries
// below 2 in magnitude first, so the squares cannot overflow.
__device__ __forceinline__ void givens(cplx a, cplx b, double& c, cplx& s, cplx& r) {
  const double na2 = norm2(a), nb2 = norm2(b);
  if (nb2 == 0.0) {
    c = 1.0;
    s = mk(0.0, 0.0);
    r = a;
    return;
  }
  if (na2 == 0.0) {
    const double ib = rsqrt(nb2);
    c = 0.0;
    s = ib * conj(b);
    r = mk(nb2 * ib, 0.0);
    return;
  }
  const double n2 = na2 + nb2;
  const double inv = rsqrt(n2), ia = rsqrt(na2);
  const cplx ph = ia * a;  // a / |a|
  c = na2 * ia * inv;
  s = inv * (ph * conj(b));
  r = (n2 * inv) * ph;
}

struct EigWork {
  cplx A[16][16];
  cplx v[16];      // Householder vector
  cplx rs[16];     // Givens sines of the current sweep
  double rc[16];   // Givens cosines
  double norm;     // max |a_ij|_1 after the reduction
  double scale;    // power of two the matrix was divided by
  int finite;
};

// Eigenvalues of W.A by the 16 lanes in `mask` (lane l = 0..15 of them). On
// a true return the eigenvalues are W.A's diagonal (scaled back). Every lane
// returns the same value.
__device__ bool eig16(EigWork& W, int l, unsigned mask, int base) {
  constexpr double U = 2.220446049250313e-16;  // 2^-52
  __syncwarp(mask);
  if (l == 0) {
    int fin = 1;
    double amax = 0.0;
    for (int i = 0; i < 256; ++i) {
      const cplx a = W.A[i >> 4][i & 15];
      fin &= isfinite(a.re) && isfinite(a.im);
      amax = fmax(amax, fmax(fabs(a.re), fabs(a.im)));
    }
    W.finite = fin;
    // 2^e with amax / 2^e in [1, 2): an exact scaling (e clamped so that
    // 2^-e stays a normal number)
    W.scale = (fin && amax > 0.0) ? ldexp(1.0, max(-1000, min(1000, ilogb(amax)))) : 1.0;
  }
  __syncwarp(mask);
  if (!W.finite) return false;
  {
    const double inv_scale = 1.0 / W.scale;  // a power of two: exact
    for (int j = 0; j < 16; ++j) W.A[l][j] = inv_scale * W.A[l][j];
  }

  // Householder reduction to upper Hessenberg form: A <- H A H, H = I - tau v v^H.
  for (int c = 0; c < 14; ++c) {
    __syncwarp(mask);
    double tail = 0.0;
    for (int i = c + 2; i < 16; ++i) tail += norm2(W.A[i][c]);
    if (tail == 0.0) continue;  // the same decision in every lane
    const cplx x0 = W.A[c + 1][c];
    const double ax0 = cabs(x0);
    const double sigma = sqrt(ax0 * ax0 + tail);
    const cplx ph = ax0 > 0.0 ? (1.0 / ax0) * x0 : mk(1.0, 0.0);
    const cplx alpha = -(sigma * ph);
    const double tau = 1.0 / (sigma * (sigma + ax0));
    if (l >= c + 1) W.v[l] = l == c + 1 ? (ax0 + sigma) * ph : W.A[l][c];
    __syncwarp(mask);
    if (l == c) {
      W.A[c + 1][c] = alpha;
      for (int i = c + 2; i < 16; ++i) W.A[i][c] = mk(0.0, 0.0);
    } else if (l > c) {  // column l: A[:, l] -= tau v (v^H A[:, l])
      cplx w = mk(0.0, 0.0);
      for (int i = c + 1; i < 16; ++i) w = w + conj(W.v[i]) * W.A[i][l];
      w = tau * w;
      for (int i = c + 1; i < 16; ++i) W.A[i][l] = W.A[i][l] - W.v[i] * w;
    }
    __syncwarp(mask);
    {  // row l: A[l, :] -= tau (A[l, :] v) v^H
      cplx z = mk(0.0, 0.0);
      for (int j = c + 1; j < 16; ++j) z = z + W.A[l][j] * W.v[j];
      z = tau * z;
      for (int j = c + 1; j < 16; ++j) W.A[l][j] = W.A[l][j] - z * conj(W.v[j]);
    }
  }
  __syncwarp(mask);
  if (l == 0) {
    double nrm = 0.0;
    for (int i = 0; i < 256; ++i) nrm = fmax(nrm, cabs1(W.A[i >> 4][i & 15]));
    W.norm = nrm;
  }
  __syncwarp(mask);
  const double nrm = W.norm;

  // Shifted QR sweeps on the active block [lo, hi].
  int hi = 15, its = 0, total = 0;
  while (hi > 0) {
    if (total >= SWEEPS_PER_EIG * 16) return false;
    __syncwarp(mask);
    bool small = false;
    if (l >= 1 && l <= hi) {
      double ref = cabs1(W.A[l - 1][l - 1]) + cabs1(W.A[l][l]);
      if (ref == 0.0) ref = nrm;
      small = cabs1(W.A[l][l - 1]) <= U * ref;
    }
    const unsigned bits = (__ballot_sync(mask, small) >> base) & ((2u << hi) - 1u);
    const int lo = bits ? 31 - __clz(bits) : 0;
    __syncwarp(mask);
    if (small) W.A[l][l - 1] = mk(0.0, 0.0);
    if (lo == hi) {
      --hi;
      its = 0;
      continue;
    }
    __syncwarp(mask);
    cplx mu;
    const cplx d = W.A[hi][hi], sub = W.A[hi][hi - 1];
    if (its == 10 || its == 20) {
      mu = mk(d.re + 0.75 * fabs(sub.re), d.im);
    } else {
      // Eigenvalue of [[a, b], [sub, d]] nearer d: d + h -+ sqrt(h^2 + b sub),
      // h = (a - d)/2, written as d - b sub / (h +- sqrt(...)) with the larger
      // denominator (no cancellation).
      const cplx a = W.A[hi - 1][hi - 1], b = W.A[hi - 1][hi];
      const cplx h = 0.5 * (a - d);
      const cplx bc = b * sub;
      const cplx r = csqrt(h * h + bc);
      const cplx den = (h.re * r.re + h.im * r.im) >= 0.0 ? h + r : h - r;
      mu = cabs1(den) > 0.0 ? d - cdiv(bc, den) : d;
    }
    __syncwarp(mask);
    if (l >= lo && l <= hi) W.A[l][l] = W.A[l][l] - mu;
    for (int k = lo; k < hi; ++k) {  // H - mu I = Q R, rows rotated in turn
      __syncwarp(mask);
      double c;
      cplx s, r;
      givens(W.A[k][k], W.A[k + 1][k], c, s, r);
      __syncwarp(mask);
      if (l == k) {
        W.A[k][k] = r;
        W.A[k + 1][k] = mk(0.0, 0.0);
      } else if (l > k && l <= hi) {
        const cplx x = W.A[k][l], y = W.A[k + 1][l];
        W.A[k][l] = c * x + s * y;
        W.A[k + 1][l] = c * y - conj(s) * x;
      }
      if (l == 0) {
        W.rc[k] = c;
        W.rs[k] = s;
      }
    }
    __syncwarp(mask);
    for (int k = lo; k < hi; ++k) {  // R Q: columns rotated in turn, lane = row
      if (l >= lo && l <= k + 1 && l <= hi) {
        const double c = W.rc[k];
        const cplx s = W.rs[k];
        const cplx x = W.A[l][k], y = W.A[l][k + 1];
        W.A[l][k] = c * x + conj(s) * y;
        W.A[l][k + 1] = c * y - s * x;
      }
    }
    __syncwarp(mask);
    if (l >= lo && l <= hi) W.A[l][l] = W.A[l][l] + mu;
    ++its;
    ++total;
  }
  __syncwarp(mask);
  W.A[l][l] = W.scale * W.A[l][l];
  __syncwarp(mask);
  return true;
}

// Input modes of k_vn_eig.
enum { SRC_VN = 0, SRC_MATRIX = 1 };

// One matrix per 16 threads. SRC_VN: G of item (case, wave vector) from the
// case's collision Jacobian and the Lax-Wendroff symbol; writes G if Gout,
// else solves. SRC_MATRIX: the item's input matrix.
__global__ void __launch_bounds__(VN_T) k_vn_eig(int src, long long nitems, int nk,
                                                 const double* __restrict__ Jc,
                                                 const double* __restrict__ kvec, LW lw, double dx,
                                                 double dy, const double* __restrict__ Ain,
                                                 double* Gout, double* omega, double* radius,
                                                 unsigned long long* failed) {
  __shared__ EigWork work[MPB];
  const int half = threadIdx.x >> 4, l = threadIdx.x & 15;
  const long long item = (long long)blockIdx.x * MPB + half;
  if (item >= nitems) return;  // the whole half-warp leaves together
  const int base = (threadIdx.x & 31) & ~15;
  const unsigned mask = 0xFFFFu << base;
  EigWork& W = work[half];
  if (src == SRC_VN) {
    const long long c = item / nk;
    const int q = (int)(item - c * nk);
    const double* J = Jc + c * 256;
    for (int i = l; i < 256; i += 16) W.A[i >> 4][i & 15] = mk(J[i], 0.0);
    double sx, cx, sy, cy;
    sincos(kvec[2 * q] * dx, &sx, &cx);
    sincos(kvec[2 * q + 1] * dy, &sy, &cy);
    // a0 + aE e^{i tx} + aW e^{-i tx} + aN e^{i ty} + aS e^{-i ty}
    const cplx diag = mk(lw.a0[l] + (lw.aE[l] + lw.aW[l]) * cx + (lw.aN[l] + lw.aS[l]) * cy,
                         (lw.aE[l] - lw.aW[l]) * sx + (lw.aN[l] - lw.aS[l]) * sy);
    __syncwarp(mask);
    W.A[l][l] = W.A[l][l] + diag;
    if (Gout) {
      __syncwarp(mask);
      double* g = Gout + item * 512;
      for (int i = l; i < 256; i += 16) {
        g[2 * i] = W.A[i >> 4][i & 15].re;
        g[2 * i + 1] = W.A[i >> 4][i & 15].im;
      }
      return;
    }
  } else {
    const double* a = Ain + item * 512;
    for (int i = l; i < 256; i += 16) W.A[i >> 4][i & 15] = mk(a[2 * i], a[2 * i + 1]);
  }
  const bool ok = eig16(W, l, mask, base);
  const cplx w = ok ? W.A[l][l] : mk(nan(""), nan(""));
  if (omega) {
    omega[item * 32 + 2 * l] = w.re;
    omega[item * 32 + 2 * l + 1] = w.im;
  }
  double r = ok ? cabs(w) : nan("");
  for (int off = 8; off > 0; off >>= 1) r = fmax(r, __shfl_xor_sync(mask, r, off, 16));
  if (l == 0) {
    if (radius) radius[item] = ok ? r : nan("");
    if (!ok && failed) atomicAdd(failed, 1ull);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, s);
  }
};

int check_grid(double dx, double dy, double dt) {
  if (!(std::isfinite(dx) && dx > 0.0 && std::isfinite(dy) && dy > 0.0 && std::isfinite(dt) &&
        dt > 0.0))
    return vfail(LBM_ERR_INVALID, "dx, dy and dt must be finite and > 0");
  return LBM_OK;
}

int check_cases(const lbm_vn_case* cases, int n) {
  for (int c = 0; c < n; ++c) {
    const lbm_vn_case& k = cases[c];
    bool ok = std::isfinite(k.rho) && k.rho > 0.0 && std::isfinite(k.T) && k.T > 0.0 &&
              std::isfinite(k.u) && std::isfinite(k.v);
    for (int i = 0; i < 16; ++i) ok = ok && std::isfinite(k.s[i]);
    if (!ok) return vfail(LBM_ERR_INVALID, "case " + std::to_string(c) +
                                               ": needs finite rates, rho > 0 and T > 0");
  }
  return LBM_OK;
}

int check_k(const double* k, int nk) {
  for (int q = 0; q < 2 * nk; ++q)
    if (!std::isfinite(k[q])) return vfail(LBM_ERR_INVALID, "non-finite wave vector");
  return LBM_OK;
}

// Copies n bytes of host data to a new device buffer (or aliases device data).
int stage_in(const void* src, size_t n, int on_device, cudaStream_t s, DevBuf& buf,
             const void** out) {
  if (on_device) {
    *out = src;
    return LBM_OK;
  }
  buf.s = s;
  VCK(cudaMallocAsync(&buf.p, n, s));
  VCK(cudaMemcpyAsync(buf.p, src, n, cudaMemcpyHostToDevice, s));
  *out = buf.p;
  return LBM_OK;
}

int alloc_out(void* host, size_t n, int on_device, cudaStream_t s, DevBuf& buf, void** out) {
  if (!host) {
    *out = nullptr;
    return LBM_OK;
  }
  if (on_device) {
    *out = host;
    return LBM_OK;
  }
  buf.s = s;
  VCK(cudaMallocAsync(&buf.p, n, s));
  *out = buf.p;
  return LBM_OK;
}

int copy_out(void* host, const void* dev, size_t n, int on_device, cudaStream_t s) {
  if (host && !on_device) VCK(cudaMemcpyAsync(host, dev, n, cudaMemcpyDeviceToHost, s));
  return LBM_OK;
}

unsigned grid_of(long long nitems) { return (unsigned)((nitems + MPB - 1) / MPB); }

// Shared body of lbm_vn_matrices (G != nullptr) and lbm_vn_spectrum.
int vn_run(const lbm_vn_case* cases, int ncases, const double* k, int nk, double dx, double dy,
           double dt, double* G, double* radius, double* omega, int on_device, void* stream,
           long long* nonconverged) {
  if (ncases < 1 || nk < 1 || !cases || !k)
    return vfail(LBM_ERR_INVALID, "need ncases >= 1, nk >= 1, cases and k");
  int rc = check_grid(dx, dy, dt);
  if (rc != LBM_OK) return rc;
  if (!on_device) {
    if ((rc = check_cases(cases, ncases)) != LBM_OK) return rc;
    if ((rc = check_k(k, nk)) != LBM_OK) return rc;
  }
  const long long nitems = (long long)ncases * nk;
  if ((nitems + MPB - 1) / MPB > 0x7FFFFFFFLL) return vfail(LBM_ERR_INVALID, "too many items");
  Coeffs<double> K;
  if (!lattice_constants(K)) return vfail(LBM_ERR_CUDA, "singular lattice block");
  set_advection(K, dt, dx, dy);
  LW lw;
  for (int i = 0; i < 16; ++i) {
    lw.a0[i] = K.a0[i];
    lw.aE[i] = K.aE[i];
    lw.aW[i] = K.aW[i];
    lw.aN[i] = K.aN[i];
    lw.aS[i] = K.aS[i];
  }
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf bc, bk, bj, bg, br, bo, bf;
  const void *dcases = nullptr, *dk = nullptr;
  if ((rc = stage_in(cases, sizeof(lbm_vn_case) * ncases, on_device, s, bc, &dcases)) ||
      (rc = stage_in(k, sizeof(double) * 2 * nk, on_device, s, bk, &dk)))
    return rc;
  bj.s = s;
  VCK(cudaMallocAsync(&bj.p, sizeof(double) * 256 * (size_t)ncases, s));
  void *dG = nullptr, *dr = nullptr, *dw = nullptr;
  if ((rc = alloc_out(G, sizeof(double) * 512 * (size_t)nitems, on_device, s, bg, &dG)) ||
      (rc = alloc_out(radius, sizeof(double) * (size_t)nitems, on_device, s, br, &dr)) ||
      (rc = alloc_out(omega, sizeof(double) * 32 * (size_t)nitems, on_device, s, bo, &dw)))
    return rc;
  unsigned long long* dfail = nullptr;
  if (nonconverged) {
    bf.s = s;
    VCK(cudaMallocAsync(&bf.p, sizeof(unsigned long long), s));
    dfail = (unsigned long long*)bf.p;
    VCK(cudaMemsetAsync(dfail, 0, sizeof(unsigned long long), s));
  }
  k_vn_jacobian<<<ncases, 16, 0, s>>>((const lbm_vn_case*)dcases, K, dt, (double*)bj.p);
  VCK(cudaGetLastError());
  k_vn_eig<<<grid_of(nitems), VN_T, 0, s>>>(SRC_VN, nitems, nk, (const double*)bj.p,
                                            (const double*)dk, lw, dx, dy, nullptr,
                                            (double*)dG, (double*)dw, (double*)dr, dfail);
  VCK(cudaGetLastError());
  if ((rc = copy_out(G, dG, sizeof(double) * 512 * (size_t)nitems, on_device, s)) ||
      (rc = copy_out(radius, dr, sizeof(double) * (size_t)nitems, on_device, s)) ||
      (rc = copy_out(omega, dw, sizeof(double) * 32 * (size_t)nitems, on_device, s)))
    return rc;
  unsigned long long nf = 0;
  if (nonconverged) VCK(cudaMemcpyAsync(&nf, dfail, sizeof(nf), cudaMemcpyDeviceToHost, s));
  if (!on_device || nonconverged) VCK(cudaStreamSynchronize(s));
  if (nonconverged) *nonconverged = (long long)nf;
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_vn_matrices(const lbm_vn_case* cases, int ncases, const double* k, int nk, double dx,
                    double dy, double dt, double* G, int on_device, void* cuda_stream) {
  if (!G) return vfail(LBM_ERR_INVALID, "G is required");
  return vn_run(cases, ncases, k, nk, dx, dy, dt, G, nullptr, nullptr, on_device, cuda_stream,
                nullptr);
}

int lbm_vn_spectrum(const lbm_vn_case* cases, int ncases, const double* k, int nk, double dx,
                    double dy, double dt, double* radius, double* omega, int on_device,
                    void* cuda_stream, long long* nonconverged) {
  if (!radius && !omega && !nonconverged)
    return vfail(LBM_ERR_INVALID, "no output requested");
  return vn_run(cases, ncases, k, nk, dx, dy, dt, nullptr, radius, omega, on_device, cuda_stream,
                nonconverged);
}

int lbm_eig16(const double* A, long long n, double* omega, double* radius, int on_device,
              void* cuda_stream, long long* nonconverged) {
  if (n < 1 || !A) return vfail(LBM_ERR_INVALID, "need n >= 1 and A");
  if (!omega && !radius && !nonconverged) return vfail(LBM_ERR_INVALID, "no output requested");
  if ((n + MPB - 1) / MPB > 0x7FFFFFFFLL) return vfail(LBM_ERR_INVALID, "too many matrices");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  DevBuf ba, bo, br, bf;
  const void* dA = nullptr;
  int rc;
  if ((rc = stage_in(A, sizeof(double) * 512 * (size_t)n, on_device, s, ba, &dA))) return rc;
  void *dw = nullptr, *dr = nullptr;
  if ((rc = alloc_out(omega, sizeof(double) * 32 * (size_t)n, on_device, s, bo, &dw)) ||
      (rc = alloc_out(radius, sizeof(double) * (size_t)n, on_device, s, br, &dr)))
    return rc;
  unsigned long long* dfail = nullptr;
  if (nonconverged) {
    bf.s = s;
    VCK(cudaMallocAsync(&bf.p, sizeof(unsigned long long), s));
    dfail = (unsigned long long*)bf.p;
    VCK(cudaMemsetAsync(dfail, 0, sizeof(unsigned long long), s));
  }
  LW lw = {};
  k_vn_eig<<<grid_of(n), VN_T, 0, s>>>(SRC_MATRIX, n, 1, nullptr, nullptr, lw, 1.0, 1.0,
                                       (const double*)dA, nullptr, (double*)dw, (double*)dr,
                                       dfail);
  VCK(cudaGetLastError());
  if ((rc = copy_out(omega, dw, sizeof(double) * 32 * (size_t)n, on_device, s)) ||
      (rc = copy_out(radius, dr, sizeof(double) * (size_t)n, on_device, s)))
    return rc;
  unsigned long long nf = 0;
  if (nonconverged) VCK(cudaMemcpyAsync(&nf, dfail, sizeof(nf), cudaMemcpyDeviceToHost, s));
  if (!on_device || nonconverged) VCK(cudaStreamSynchronize(s));
  if (nonconverged) *nonconverged = (long long)nf;
  return LBM_OK;
}

const char* lbm_vn_last_error(void) { return g_vn_error.c_str(); }

}  // extern "C"
