// lbm_dw_step.cuh -- the per-node update of precision LBM_DF64 in
// double-word arithmetic (dw.cuh): populations stored as pairs (h, l) of
// FP32 values, every operation of the step on the FP32 units through
// error-free transformations, two nodes per thread in paired f32x2
// instructions. Included by lbm_step_kernels.cuh (the tile update of the
// generic k_step / k_step_pipe kernels for R = dw).
//
// Per node, in the order of Eq. 3 with Eq. A.1 (the same factorisation as
// d2v16.cuh, written out for the double-word form):
//   4-point group transforms of the 16 populations (S, C, X, Y per group);
//   the 16 moments of Eqs. 5a-5p as dot products of those with the groups'
//   radial factors (the diagonal groups' sqrt 2 and 3 / sqrt 2 taken into X
//   and Y once, so that every coefficient left is an exact FP32 number);
//   the Eq. 14 equilibria from (rho, j, e); the deviations m_k - m_k^eq;
//   the back-map M^-1 (-dt S_hat (m - m^eq)) through the scaled block
//   inverses (constants of Coeffs<dw>) and the inverse 4-point transform;
//   the update f + [df + aW (f(x-dx) - f) + aE (f(x+dx) - f) + aS (f(y-dy) - f)
//   + aN (f(y+dy) - f)] (Eq. A.1 with a0 = 1 - aW - aE - aS - aN, in increment
//   form so that rounding scales with the change of f).
#pragma once

#include <type_traits>

#include "dw.cuh"
#include "lbm_step.cuh"

namespace lbmk {

// Radial factors taken into the diagonal groups' X and Y.
__host__ __device__ constexpr dw dw_sq2() { return dw(SQ2); }
__host__ __device__ constexpr dw dw_3_sq2() { return dw(3.0 / SQ2); }
__host__ __device__ constexpr double radial(int g) { return g == 2 ? SQ2 : (g == 3 ? 3.0 / SQ2 : 1.0); }
// Coefficient of group g in row r of the x (y) block after that scaling:
// small integers and halves, exact in FP32.
__host__ __device__ constexpr float bxs(int r, int g) { return (float)(bx(r, g) / radial(g)); }
__host__ __device__ constexpr float bys(int r, int g) { return (float)(by(r, g) / radial(g)); }

template <typename V>
__device__ __forceinline__ DW<V> dot4f(float c0, float c1, float c2, float c3, const DW<V> (&v)[4]) {
  DW<V> s = dmulf(v[0], c0);
  s = dadd(s, dmulf(v[1], c1));
  s = dadd(s, dmulf(v[2], c2));
  return dadd(s, dmulf(v[3], c3));
}
template <typename V>
__device__ __forceinline__ DW<V> dot2k(dw k0, float t0, DW<V> a, dw k1, float t1, DW<V> b) {
  return dadd(dmulk(a, k0, t0), dmulk(b, k1, t1));
}
template <typename V>
__device__ __forceinline__ DW<V> dot3k(dw k0, float t0, DW<V> a, dw k1, float t1, DW<V> b, dw k2,
                                       float t2, DW<V> c) {
  return dadd(dadd(dmulk(a, k0, t0), dmulk(b, k1, t1)), dmulk(c, k2, t2));
}

// The 16 moments from the populations f_i = ld(i): mom[k - 1] = m_k
// (rho, j_x, j_y, e, m5 .. m16 in the paper's numbering).
template <typename V, typename Load>
__device__ __forceinline__ void dw_moments(Load ld, DW<V> (&mom)[16]) {
  DW<V> S[4], C[4], X[4], Y[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const DW<V> f0 = ld(4 * g), f1 = ld(4 * g + 1), f2 = ld(4 * g + 2), f3 = ld(4 * g + 3);
    const DW<V> p = dadd(f0, f2), q = dadd(f1, f3), a = dsub(f0, f2), b = dsub(f1, f3);
    S[g] = dadd(p, q);
    C[g] = dsub(p, q);
    if (g < 2) {
      X[g] = a;
      Y[g] = b;
    } else {
      X[g] = dsub(a, b);
      Y[g] = dadd(a, b);
    }
  }
  X[2] = dmulk(X[2], dw_sq2(), third_word(SQ2));
  Y[2] = dmulk(Y[2], dw_sq2(), third_word(SQ2));
  X[3] = dmulk(X[3], dw_3_sq2(), third_word(3.0 / SQ2));
  Y[3] = dmulk(Y[3], dw_3_sq2(), third_word(3.0 / SQ2));
  mom[0] = dadd(dadd(S[0], S[1]), dadd(S[2], S[3]));                                   // rho
  mom[3] = dot4f((float)b0(1, 0), (float)b0(1, 1), (float)b0(1, 2), (float)b0(1, 3), S);  // e
  mom[10] = dot4f((float)b0(2, 0), (float)b0(2, 1), (float)b0(2, 2), (float)b0(2, 3), S); // m11
  mom[11] = dot4f((float)b0(3, 0), (float)b0(3, 1), (float)b0(3, 2), (float)b0(3, 3), S); // m12
  mom[1] = dot4f(bxs(0, 0), bxs(0, 1), bxs(0, 2), bxs(0, 3), X);    // j_x
  mom[6] = dot4f(bxs(1, 0), bxs(1, 1), bxs(1, 2), bxs(1, 3), X);    // m7
  mom[8] = dot4f(bxs(2, 0), bxs(2, 1), bxs(2, 2), bxs(2, 3), X);    // m9
  mom[14] = dot4f(bxs(3, 0), bxs(3, 1), bxs(3, 2), bxs(3, 3), X);   // m15
  mom[2] = dot4f(bys(0, 0), bys(0, 1), bys(0, 2), bys(0, 3), Y);    // j_y
  mom[7] = dot4f(bys(1, 0), bys(1, 1), bys(1, 2), bys(1, 3), Y);    // m8
  mom[9] = dot4f(bys(2, 0), bys(2, 1), bys(2, 2), bys(2, 3), Y);    // m10
  mom[15] = dot4f(bys(3, 0), bys(3, 1), bys(3, 2), bys(3, 3), Y);   // m16
  mom[4] = dadd(dmulf(C[0], (float)bc2(0, 0)), dmulf(C[1], (float)bc2(0, 1)));   // m5
  mom[12] = dadd(dmulf(C[0], (float)bc2(1, 0)), dmulf(C[1], (float)bc2(1, 1)));  // m13
  mom[5] = dadd(dmulf(C[2], (float)bs2(0, 0)), dmulf(C[3], (float)bs2(0, 1)));   // m6
  mom[13] = dadd(dmulf(C[2], (float)bs2(1, 0)), dmulf(C[3], (float)bs2(1, 1)));  // m14
}

// (rho, j_x, j_y, e) of FP32 populations in double-word arithmetic: the
// group butterflies of the inputs by two_sum (exact), then the same radial
// dot products as dw_moments. For the FP32 step of precision
// LBM_FP32_DWMOM: its conserved moments carry no rounding of the transform.
template <typename V>
__device__ __forceinline__ void dw_conserved_of(const V (&f)[16], DW<V>& rho, DW<V>& jx,
                                                DW<V>& jy, DW<V>& e) {
  DW<V> S[4], X[4], Y[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    DW<V> p, q, a, b;
    two_sum(f[4 * g], f[4 * g + 2], p.h, p.l);
    two_sum(f[4 * g + 1], f[4 * g + 3], q.h, q.l);
    two_sum(f[4 * g], lneg(f[4 * g + 2]), a.h, a.l);
    two_sum(f[4 * g + 1], lneg(f[4 * g + 3]), b.h, b.l);
    S[g] = dadd(p, q);
    if (g < 2) {
      X[g] = a;
      Y[g] = b;
    } else {
      X[g] = dsub(a, b);
      Y[g] = dadd(a, b);
    }
  }
  X[2] = dmulk(X[2], dw_sq2(), third_word(SQ2));
  Y[2] = dmulk(Y[2], dw_sq2(), third_word(SQ2));
  X[3] = dmulk(X[3], dw_3_sq2(), third_word(3.0 / SQ2));
  Y[3] = dmulk(Y[3], dw_3_sq2(), third_word(3.0 / SQ2));
  rho = dadd(dadd(S[0], S[1]), dadd(S[2], S[3]));
  e = dot4f((float)b0(1, 0), (float)b0(1, 1), (float)b0(1, 2), (float)b0(1, 3), S);
  jx = dot4f(bxs(0, 0), bxs(0, 1), bxs(0, 2), bxs(0, 3), X);
  jy = dot4f(bys(0, 0), bys(0, 1), bys(0, 2), bys(0, 3), Y);
}

// Eq. 14 from (rho, j, e) with P = rho T = e - |j|^2 / (2 rho) (gamma = 2);
// the same expressions as d2v16.cuh `equilibria`, in double-word arithmetic.
template <typename V>
struct DwEq {
  DW<V> m5, m6, m7, m8, m9, m10, m11, m13, m14, P;
};
template <typename V>
__device__ __forceinline__ DwEq<V> dw_equilibria(DW<V> rho, DW<V> jx, DW<V> jy, DW<V> e) {
  DwEq<V> q;
  const DW<V> r = drecip(rho);
  const DW<V> ux = dmul(jx, r), uy = dmul(jy, r);
  const DW<V> ux2 = dmul(ux, ux), uy2 = dmul(uy, uy), usq = dadd(ux2, uy2);
  const DW<V> er = dmul(e, r);
  q.P = dsub(e, dmul(dscale(rho, 0.5f), usq));
  const DW<V> eP = dadd(e, q.P);
  q.m5 = dmul(rho, dsub(ux2, uy2));
  q.m6 = dmul(jx, uy);
  q.m7 = dmul(eP, ux);
  q.m8 = dmul(eP, uy);
  q.m9 = dmul(jx, dsub(ux2, dmulf(uy2, 3.0f)));
  q.m10 = dmul(jy, dsub(dmulf(ux2, 3.0f), uy2));
  q.m11 = dsub(dscale(dmul(e, er), 2.0f), dmul(dscale(rho, 0.25f), dmul(usq, usq)));
  const DW<V> A = dsub(dmulf(er, 6.0f), dscale(usq, 2.0f));
  q.m13 = dmul(A, q.m5);
  q.m14 = dmul(A, q.m6);
  return q;
}

// Inverse 4-point transform from scaled group values to populations (the
// double-word form of d2v16.cuh `inverse_transform`).
template <typename V>
__device__ __forceinline__ void dw_inverse_transform(const DW<V> (&S)[4], const DW<V> (&C)[4],
                                                     const DW<V> (&X)[4], const DW<V> (&Y)[4],
                                                     DW<V> (&out)[16]) {
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const DW<V> P = dadd(S[g], C[g]), Q = dsub(S[g], C[g]);
    if (g < 2) {
      out[4 * g] = dadd(P, X[g]);
      out[4 * g + 2] = dsub(P, X[g]);
      out[4 * g + 1] = dadd(Q, Y[g]);
      out[4 * g + 3] = dsub(Q, Y[g]);
    } else {
      const DW<V> A = dadd(X[g], Y[g]), B = dsub(Y[g], X[g]);
      out[4 * g] = dadd(P, A);
      out[4 * g + 2] = dsub(P, A);
      out[4 * g + 1] = dadd(Q, B);
      out[4 * g + 3] = dsub(Q, B);
    }
  }
}

// Collision of Eq. 3 from the moments: df = M^-1 (-dt S_hat (m - m^eq)),
// through the w-scaled block inverses K* of Coeffs<dw> and the inverse
// 4-point transform. Returns P = rho T.
template <typename V>
__device__ __forceinline__ DW<V> dw_collide(const Coeffs<dw>& K, const Coeffs<float>& T,
                                            const DW<V> (&m)[16], DW<V> (&df)[16]) {
  const DwEq<V> q = dw_equilibria(m[0], m[1], m[2], m[3]);
  const DW<V> d11 = dsub(m[10], q.m11), d12 = m[11];
  const DW<V> d7 = dsub(m[6], q.m7), d9 = dsub(m[8], q.m9), d15 = m[14];
  const DW<V> d8 = dsub(m[7], q.m8), d10 = dsub(m[9], q.m10), d16 = m[15];
  const DW<V> d5 = dsub(m[4], q.m5), d13 = dsub(m[12], q.m13);
  const DW<V> d6 = dsub(m[5], q.m6), d14 = dsub(m[13], q.m14);
  DW<V> S[4], C[4], X[4], Y[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    S[g] = dot2k(K.K0[g][0], T.K0[g][0], d11, K.K0[g][1], T.K0[g][1], d12);
    X[g] = dot3k(K.KX[g][0], T.KX[g][0], d7, K.KX[g][1], T.KX[g][1], d9, K.KX[g][2], T.KX[g][2], d15);
    Y[g] = dot3k(K.KY[g][0], T.KY[g][0], d8, K.KY[g][1], T.KY[g][1], d10, K.KY[g][2], T.KY[g][2], d16);
  }
  C[0] = dot2k(K.KC[0][0], T.KC[0][0], d5, K.KC[0][1], T.KC[0][1], d13);
  C[1] = dot2k(K.KC[1][0], T.KC[1][0], d5, K.KC[1][1], T.KC[1][1], d13);
  C[2] = dot2k(K.KS[0][0], T.KS[0][0], d6, K.KS[0][1], T.KS[0][1], d14);
  C[3] = dot2k(K.KS[1][0], T.KS[1][0], d6, K.KS[1][1], T.KS[1][1], d14);
  dw_inverse_transform(S, C, X, Y, df);
  return q.P;
}

__device__ __forceinline__ bool dw_finite(float h, float l) { return ::isfinite(h) && ::isfinite(l); }

// ---------------------------------------------------------------------------
// Edge nodes: the neighbour terms of Eq. A.1 with boundary ghosts, in the
// double-word form with three-word constants (the double-word counterpart of
// lbm_step.cuh `neighbour_terms` / `ghost_with`). A two-word weight or
// ghost population at a boundary is off by up to 2^-48 of itself at every
// step, and on a supersonic inflow that bias is carried into the domain and
// grows linearly with time; three words take it below 2^-70.
// ---------------------------------------------------------------------------
using DWf = DW<float>;

__device__ __forceinline__ DWf dwf(dw v) { return {v.h, v.l}; }

// f^eq = M^-1 f_hat^eq of (rho, j, e) (d2v16.cuh `feq` in double-word, the
// scaled block inverses E* with their third words).
__device__ __forceinline__ void dw_feq(const Coeffs<dw>& K, const Coeffs<float>& T, DWf rho, DWf jx,
                                       DWf jy, DWf e, DWf (&out)[16]) {
  const DwEq<float> q = dw_equilibria(rho, jx, jy, e);
  DWf S[4], C[4], X[4], Y[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    S[g] = dot3k(K.E0[g][0], T.E0[g][0], rho, K.E0[g][1], T.E0[g][1], e, K.E0[g][2], T.E0[g][2], q.m11);
    X[g] = dot3k(K.EX[g][0], T.EX[g][0], jx, K.EX[g][1], T.EX[g][1], q.m7, K.EX[g][2], T.EX[g][2], q.m9);
    Y[g] = dot3k(K.EY[g][0], T.EY[g][0], jy, K.EY[g][1], T.EY[g][1], q.m8, K.EY[g][2], T.EY[g][2], q.m10);
  }
  C[0] = dot2k(K.EC[0][0], T.EC[0][0], q.m5, K.EC[0][1], T.EC[0][1], q.m13);
  C[1] = dot2k(K.EC[1][0], T.EC[1][0], q.m5, K.EC[1][1], T.EC[1][1], q.m13);
  C[2] = dot2k(K.ES[0][0], T.ES[0][0], q.m6, K.ES[0][1], T.ES[0][1], q.m14);
  C[3] = dot2k(K.ES[1][0], T.ES[1][0], q.m6, K.ES[1][1], T.ES[1][1], q.m14);
  dw_inverse_transform(S, C, X, Y, out);
}

// Conserved moments (rho, j_x, j_y, e) of node idx of the global populations.
template <typename Off>
__device__ __forceinline__ void dw_load_cons(const dw* __restrict__ fin, Off plane, Off idx,
                                             DWf (&c)[4]) {
  auto ld = [&](int i) { return dwf(fin[i * plane + idx]); };
  DWf m[16];
  dw_moments(ld, m);
  c[0] = dnorm(m[0]); c[1] = dnorm(m[1]); c[2] = dnorm(m[2]); c[3] = dnorm(m[3]);
}

// Primitive (rho, u, v, T) of conserved moments; T = e / rho - |u|^2 / 2.
__device__ __forceinline__ void dw_primitive(const DWf (&c)[4], DWf& rho, DWf& u, DWf& v, DWf& T) {
  const DWf r = drecip(c[0]);
  rho = c[0];
  u = dmul(c[1], r);
  v = dmul(c[2], r);
  T = dsub(dmul(c[3], r), dscale(dadd(dmul(u, u), dmul(v, v)), 0.5f));
}

// Ghost populations g (+ third words gt, the Dirichlet ghosts only) of kind
// `kind` outside `side` of a node with conserved moments `own`; `inward` is
// the next node inwards (linear extrapolation only).
template <typename Off>
__device__ __forceinline__ void dw_ghost(const StepArgs<dw>& A, const dw* __restrict__ fin, Off plane,
                                         int side, int kind, const DWf (&own)[4], Off inward,
                                         bool has_inward, DWf (&g)[16], float (&gt)[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) gt[i] = 0.f;
  if (kind == LBM_BC_EQ) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      g[i] = dwf(A.geq[side * 16 + i]);
      gt[i] = A.geq3[side * 16 + i];
    }
    return;
  }
  DWf rho = own[0], jx = own[1], jy = own[2], e = own[3];
  if (kind == LBM_BC_REFLECT) {
    if (side < 2) jx = {-jx.h, -jx.l}; else jy = {-jy.h, -jy.l};
  } else if (kind == LBM_BC_WALL) {
    const DWf u = dwf(A.wall[side][0]), v = dwf(A.wall[side][1]), T = dwf(A.wall[side][2]);
    jx = dmul(rho, u);
    jy = dmul(rho, v);
    e = dadd(dmul(rho, T), dmul(dscale(rho, 0.5f), dadd(dmul(u, u), dmul(v, v))));
  } else if (kind == LBM_BC_EXTRAP) {
    DWf in[4] = {own[0], own[1], own[2], own[3]};
    if (has_inward) dw_load_cons(fin, plane, inward, in);
    DWf r1, u1, v1, T1, r2, u2, v2, T2;
    dw_primitive(own, r1, u1, v1, T1);
    dw_primitive(in, r2, u2, v2, T2);
    DWf r = dnorm(dsub(dscale(r1, 2.f), r2)), u = dsub(dscale(u1, 2.f), u2),
        v = dsub(dscale(v1, 2.f), v2), T = dnorm(dsub(dscale(T1, 2.f), T2));
    if (!(r.h > 0.f && T.h > 0.f)) {
      r = r1; u = u1; v = v1; T = T1;
    }
    rho = r;
    jx = dmul(r, u);
    jy = dmul(r, v);
    e = dadd(dmul(r, T), dmul(dscale(r, 0.5f), dadd(dmul(u, u), dmul(v, v))));
  }  // LBM_BC_OUTFLOW: the node's own state
  dw_feq(A.K, A.K3, rho, jx, jy, e, g);
}

// acc[i] += aW (f(x-dx) - f) + aE (f(x+dx) - f) + aS (f(y-dy) - f) +
// aN (f(y+dy) - f) for an edge node with populations f (its tile pointer
// ctr, global index c, conserved moments m at time t): the increment form
// of the interior update.
template <typename Off, int BXP>
__device__ __forceinline__ void dw_edge_terms(const StepArgs<dw>& A, const dw* __restrict__ fin,
                                              const dw* ctr, int PS, Off P, Off pitch, Off c, int x,
                                              int y, const DWf (&m)[4], dw t, DWf (&acc)[16]) {
  auto f = [&](int i) { return dwf(ctr[i * PS]); };  // the node's own populations
  // side: 0 x-, 1 x+, 2 y-, 3 y+ ; the neighbour lies inside when the node
  // is not on that side
  const bool inside[4] = {x > 0, x < A.nx - 1, y > 0, y < A.ny - 1};
  const int toff[4] = {-1, 1, -BXP, BXP};
  const Off wrap[4] = {(Off)(A.nx - 1), (Off)0 - (Off)(A.nx - 1), (Off)(A.ny - 1) * pitch,
                       (Off)0 - (Off)(A.ny - 1) * pitch};
  const Off inw[4] = {c + 1, c - 1, c + pitch, c - pitch};
  const bool deep[4] = {A.nx > 1, A.nx > 1, A.ny > 1, A.ny > 1};
#pragma unroll
  for (int side = 0; side < 4; ++side) {
    const bool xs = side < 2;
    const dw* wgt = side == 0 ? A.K.aW : side == 1 ? A.K.aE : side == 2 ? A.K.aS : A.K.aN;
    const float* wgt3 = side == 0 ? A.K3.aW : side == 1 ? A.K3.aE : side == 2 ? A.K3.aS : A.K3.aN;
    auto use = [&](int i) { return xs ? has_x(i) : has_y(i); };
    if (inside[side]) {
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (use(i))
          acc[i] = dadd(acc[i], dmulk(dsub(dwf(ctr[i * PS + toff[side]]), f(i)), wgt[i], wgt3[i]));
    } else if (A.bc[side] == LBM_BC_PERIODIC) {
      const Off n = c + wrap[side];
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (use(i)) acc[i] = dadd(acc[i], dmulk(dsub(dwf(fin[i * P + n]), f(i)), wgt[i], wgt3[i]));
    } else {
      DWf g[16];
      float gt[16];
      dw_ghost(A, fin, P, side, side_kind(A, side, xs ? y : x, t), m, inw[side], deep[side], g, gt);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (use(i)) {
          DWf d = dsub(g[i], f(i));
          d.l = ladd(d.l, gt[i]);   // the ghost's third word
          acc[i] = dadd(acc[i], dmulk(d, wgt[i], wgt3[i]));
        }
    }
  }
}


// Lane access: V = float holds one node, V = float2 two (rows y and y + Y/2).
__device__ __forceinline__ DW<float> lanes(const dw* sa, const dw*, int off) {
  const dw a = sa[off];
  return {a.h, a.l};
}
__device__ __forceinline__ DW<float2> lanes2(const dw* sa, const dw* sb, int off) {
  const dw a = sa[off], b = sb[off];
  return {make_float2(a.h, b.h), make_float2(a.l, b.l)};
}
template <typename V>
__device__ __forceinline__ DW<V> ldn(const dw* sa, const dw* sb, int off) {
  if constexpr (std::is_same<V, float>::value) return lanes(sa, sb, off);
  else return lanes2(sa, sb, off);
}
template <typename V>
__device__ __forceinline__ dw lane(DW<V> v, int k) {
  if constexpr (std::is_same<V, float>::value) return dw(v.h, v.l);
  else return k == 0 ? dw(v.h.x, v.l.x) : dw(v.h.y, v.l.y);
}
template <typename V>
__device__ __forceinline__ float lane_h(V v, int k) {
  if constexpr (std::is_same<V, float>::value) return v;
  else return k == 0 ? v.x : v.y;
}

template <typename V>
__device__ __forceinline__ DWf lane_dw(DW<V> v, int k) {
  const dw d = lane(v, k);
  return {d.h, d.l};
}

// Double-word tile update. Each thread updates NL = 1 node (V = float) or
// NL = 2 nodes (V = float2: rows y and y + Y/2 of the tile in paired f32x2
// instructions). Interior nodes take their neighbour terms from shared
// memory in the lane form; a thread with a node on the domain edge finishes
// node by node through the generic neighbour_terms (ghosts and periodic wraps
// on the normalised scalar type dw). Watchdog and audit as in the FP32 update.
template <typename Off>
__device__ __forceinline__ void step_tile_dw(const StepArgs<dw>& A, const dw* __restrict__ fin,
                                             dw* __restrict__ fout, const dw* stage, int cur,
                                             bool audit, dw t, double (*sm)[4], bool& bad,
                                             bool& negT) {
  constexpr int BXD = Shape<dw>::X, BYD = Shape<dw>::Y, TY = Shape<dw>::TY, NL = BYD / TY;
  using V = typename std::conditional<NL == 2, float2, float>::type;
  constexpr int BXP = Tile<dw>::BXP, PS = Tile<dw>::ROWS * BXP;
  static_assert(NL == 1 || NL == 2, "one or two nodes per thread");
  const int x = (cur % A.tiles_x) * BXD + threadIdx.x;
  int y[NL];
  bool act[NL];
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    y[k] = (cur / A.tiles_x) * BYD + threadIdx.y + k * TY;
    act[k] = x < A.nx && y[k] < A.ny;  // act[1] => act[0]
  }
  dw mc[NL][4];
#pragma unroll
  for (int k = 0; k < NL; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q) mc[k][q] = dw(0.f, 0.f);
  if (act[0]) {
    const Off P = (Off)A.plane, pitch = (Off)A.pitch;
    const Off c0 = (Off)y[0] * pitch + (Off)x;
    const dw* sa = stage + (threadIdx.y + 1) * BXP + threadIdx.x + HALO_X;
    const dw* sb = sa + TY * BXP;
    auto ld = [&](int i) { return ldn<V>(sa, sb, i * PS); };
    DW<V> m[16];
    dw_moments(ld, m);
    DW<V> df[16];
    const DW<V> press = dnorm(dw_collide(A.K, A.K3, m, df));
    const DW<V> rho = dnorm(m[0]), jx = dnorm(m[1]), jy = dnorm(m[2]), e = dnorm(m[3]);
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      if (!act[k]) continue;
      const bool b = !(lane_h(rho.h, k) > 0.f) ||
                     !dw_finite(lane_h(rho.h, k) + lane_h(jx.h, k) + lane_h(jy.h, k) + lane_h(e.h, k),
                                lane_h(rho.l, k));
      bad |= b;
      negT |= !b && !(lane_h(press.h, k) > 0.f);
      mc[k][0] = lane(rho, k); mc[k][1] = lane(jx, k); mc[k][2] = lane(jy, k); mc[k][3] = lane(e, k);
    }
    const bool inner = act[NL - 1] && x > 0 && x < A.nx - 1 && y[0] > 0 && y[NL - 1] < A.ny - 1;
    if (inner) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        // f+ = f + [df + sum_n a_n (f_n - f)]: the Lax-Wendroff update of
        // Eq. A.1 in increment form (a0 = 1 - sum_n a_n), so that rounding
        // scales with the change of f, not with f (populations reach 50 rho
        // in supersonic flow), and a uniform state stays uniform.
        const DW<V> fi = ld(i);
        DW<V> a = df[i];
        if (has_x(i)) {
          a = dadd(a, dmulk(dsub(ldn<V>(sa, sb, i * PS - 1), fi), A.K.aW[i], A.K3.aW[i]));
          a = dadd(a, dmulk(dsub(ldn<V>(sa, sb, i * PS + 1), fi), A.K.aE[i], A.K3.aE[i]));
        }
        if (has_y(i)) {
          a = dadd(a, dmulk(dsub(ldn<V>(sa, sb, i * PS - BXP), fi), A.K.aS[i], A.K3.aS[i]));
          a = dadd(a, dmulk(dsub(ldn<V>(sa, sb, i * PS + BXP), fi), A.K.aN[i], A.K3.aN[i]));
        }
        a = dnorm(dadd(fi, a));
#pragma unroll
        for (int k = 0; k < NL; ++k) fout[i * P + c0 + (Off)(k * TY) * pitch] = lane(a, k);
      }
    } else {
#pragma unroll
      for (int k = 0; k < NL; ++k) {
        if (!act[k]) continue;
        DWf acc1[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) acc1[i] = lane_dw(df[i], k);
        const DWf mk[4] = {dwf(mc[k][0]), dwf(mc[k][1]), dwf(mc[k][2]), dwf(mc[k][3])};
        const Off ck = c0 + (Off)(k * TY) * pitch;
        const dw* ctrk = k == 0 ? sa : sb;
        dw_edge_terms<Off, BXP>(A, fin, ctrk, PS, P, pitch, ck, x, y[k], mk, t, acc1);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const DWf a = dnorm(dadd(dwf(ctrk[i * PS]), acc1[i]));
          fout[i * P + ck] = dw(a.h, a.l);
        }
      }
    }
  }
  if (audit) {  // double-word warp sums, FP64 across warps, only on audit steps
    float h[NL][4], l[NL][4];
#pragma unroll
    for (int k = 0; k < NL; ++k)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        h[k][q] = mc[k][q].h;
        l[k][q] = mc[k][q].l;
      }
    if constexpr (NL == 2) {
      audit_pair_rows<BXD, BYD>(A, cur, h[0], l[0], h[1], l[1], sm);
    } else {
      constexpr int N = BXD * BYD;
      audit_tile_dw<N>(A, cur, h[0], l[0], sm);
    }
  }
}

}  // namespace lbmk
