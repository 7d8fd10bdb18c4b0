// d2v16.cuh -- per-node arithmetic of the D2V16 MRT-FD scheme, factorised.
//
// Velocity set (Eq. 4): population i = 4 g + k, group g = 0..3 with k = 0..3
// counter-clockwise:
//   g = 0: speed 1 on the axes    (1,0) (0,1) (-1,0) (0,-1)
//   g = 1: speed 6 on the axes    x 6
//   g = 2: speed 2 on diagonals   sqrt2 (1,1) (-1,1) (-1,-1) (1,-1)
//   g = 3: speed 3 on diagonals   3/sqrt2 x the same
//
// Factorisation of M (Eqs. 5a-5p). The moment basis is built from the SO(2)
// harmonics, and each group is a 90-degree rotation orbit, so M splits into a
// 4-point transform inside every group followed by small mixes across the
// groups. Per group, with p = f0 + f2, q = f1 + f3, a = f0 - f2, b = f1 - f3:
//   S = p + q                    (angular frequency 0)
//   C = p - q                    (frequency 2; cos 2theta on the axes,
//                                  sin 2theta on the diagonals)
//   X = a,     Y = b             (frequency 1, axis groups)
//   X = a - b, Y = a + b         (frequency 1, diagonal groups)
// Evaluating Eqs. 5a-5p on each group gives every moment as a dot product of
// one of these group vectors with the group's radial factors:
//   frequency 0 (S): rho = m1, e = m4, m11, m12
//   x-frequency 1 (X): j_x = m2, m7, m9, m15
//   y-frequency 1 (Y): j_y = m3, m8, m10, m16
//   cos 2theta (C of the axis groups): m5, m13
//   sin 2theta (C of the diagonal groups): m6, m14
// The coefficient tables below are those evaluations (e.g. m9 = v_x (v_x^2 -
// 3 v_y^2) is c^3 on the axis group of speed c and -2 h^3 on a diagonal group
// with components +-h). M^-1 is the inverse of each small block followed by
// the inverse 4-point transform; the host inverts the blocks once per context.
// Cost per node: 28 add/sub for the transform, 56 for the mixes, against 256
// multiply-adds for the dense product M f.
#pragma once

#include <cstdint>

namespace d2v16 {

constexpr double SQ2 = 1.41421356237309504880;

// Radial coefficient tables, rows = moments, columns = groups g = 0..3
// (constexpr functions so that host and device code read the same table).
// Frequency 0 block over S: rows rho, e, m11, m12.
__host__ __device__ constexpr double b0(int r, int g) {
  constexpr double t[4][4] = {{1.0, 1.0, 1.0, 1.0},
                              {0.5, 18.0, 2.0, 4.5},
                              {0.25, 324.0, 4.0, 20.25},
                              {1.0, 1296.0, -16.0, -81.0}};
  return t[r][g];
}
// x block over X: rows j_x, m7, m9, m15.
__host__ __device__ constexpr double bx(int r, int g) {
  constexpr double t[4][4] = {{1.0, 6.0, SQ2, 3.0 / SQ2},
                              {0.5, 108.0, 2.0 * SQ2, 27.0 / (2.0 * SQ2)},
                              {1.0, 216.0, -4.0 * SQ2, -27.0 / SQ2},
                              {1.0, 7776.0, -16.0 * SQ2, -243.0 / SQ2}};
  return t[r][g];
}
// y block over Y: rows j_y, m8, m10, m16.
__host__ __device__ constexpr double by(int r, int g) {
  constexpr double t[4][4] = {{1.0, 6.0, SQ2, 3.0 / SQ2},
                              {0.5, 108.0, 2.0 * SQ2, 27.0 / (2.0 * SQ2)},
                              {-1.0, -216.0, 4.0 * SQ2, 27.0 / SQ2},
                              {-1.0, -7776.0, 16.0 * SQ2, 243.0 / SQ2}};
  return t[r][g];
}
// cos 2theta block over (C0, C1): rows m5, m13.
__host__ __device__ constexpr double bc2(int r, int g) {
  constexpr double t[2][2] = {{1.0, 36.0}, {1.0, 1296.0}};
  return t[r][g];
}
// sin 2theta block over (C2, C3): rows m6, m14.
__host__ __device__ constexpr double bs2(int r, int g) {
  constexpr double t[2][2] = {{2.0, 4.5}, {8.0, 40.5}};
  return t[r][g];
}

// Velocities of Eq. 4 in the order above (host use: Lax-Wendroff weights).
__host__ __device__ constexpr double vel_x(int i) {
  constexpr double t[16] = {1, 0, -1, 0, 6, 0, -6, 0,
                            SQ2, -SQ2, -SQ2, SQ2,
                            3.0 / SQ2, -3.0 / SQ2, -3.0 / SQ2, 3.0 / SQ2};
  return t[i];
}
__host__ __device__ constexpr double vel_y(int i) {
  constexpr double t[16] = {0, 1, 0, -1, 0, 6, 0, -6,
                            SQ2, SQ2, -SQ2, -SQ2,
                            3.0 / SQ2, 3.0 / SQ2, -3.0 / SQ2, -3.0 / SQ2};
  return t[i];
}

// Population has a non-zero x (y) velocity component.
__host__ __device__ constexpr bool has_x(int i) { return !((i < 8) && (i & 1)); }
__host__ __device__ constexpr bool has_y(int i) { return !((i < 8) && !(i & 1)); }

// Per-context constants of the scheme, in the arithmetic type R.
//  E*   : scaled inverses of the blocks (rows give S/4, C/4 and X, Y divided
//         by 2 on axis groups, by 4 on diagonal groups, so that the inverse
//         4-point transform needs only additions);
//  K*   : the same columns of the non-conserved moments, each multiplied by
//         w_k = -dt s_k (the relaxation of Eq. 3 folded into the back-map);
//  a*   : Lax-Wendroff weights of Eq. A.1 per population,
//         f+ = a0 f + aE f(x+dx) + aW f(x-dx) + aN f(y+dy) + aS f(y-dy) + df.
template <typename R>
struct Coeffs {
  R F0[4][4];  // forward blocks (b0, bx, by, bc2, bs2 in the type R)
  R FX[4][4];
  R FY[4][4];
  R FC[2][2];
  R FS[2][2];
  R E0[4][4];  // rows S'_g; columns rho, e, m11, m12
  R EX[4][4];  // rows X'_g; columns j_x, m7, m9, m15
  R EY[4][4];  // rows Y'_g; columns j_y, m8, m10, m16
  R EC[2][2];  // rows C'_0, C'_1; columns m5, m13
  R ES[2][2];  // rows C'_2, C'_3; columns m6, m14
  R K0[4][2];  // w-scaled columns m11, m12 of E0
  R KX[4][3];  // w-scaled columns m7, m9, m15 of EX
  R KY[4][3];  // w-scaled columns m8, m10, m16 of EY
  R KC[2][2];  // w-scaled EC
  R KS[2][2];  // w-scaled ES
  R a0[16], aE[16], aW[16], aN[16], aS[16];
};

// Fills the forward blocks of K from the coefficient tables above.
template <typename R>
inline void fill_forward(Coeffs<R>& K) {
  for (int r = 0; r < 4; ++r)
    for (int g = 0; g < 4; ++g) {
      K.F0[r][g] = (R)b0(r, g);
      K.FX[r][g] = (R)bx(r, g);
      K.FY[r][g] = (R)by(r, g);
    }
  for (int r = 0; r < 2; ++r)
    for (int g = 0; g < 2; ++g) {
      K.FC[r][g] = (R)bc2(r, g);
      K.FS[r][g] = (R)bs2(r, g);
    }
}

// ---------------------------------------------------------------------------
// Device arithmetic
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

// Reciprocal. FP64: hardware approximation refined by two Newton-Raphson
// steps r <- r + r (1 - x r) (quadratic convergence of Newton's method for
// 1/x), within about one ulp; FP32: the hardware approximation.
__device__ __forceinline__ double recip(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Two FP32 values carried together (two nodes): every operation is one paired
// instruction of the FP32 units (add / mul / fma on .f32x2), so two nodes cost
// the instructions of one. A product is kept unevaluated (P2) until it meets a
// sum, which then becomes one paired fused multiply-add, as the compiler does
// for scalar float; scalar coefficients are broadcast to both lanes.
struct F2 {
  float2 v;
  __device__ __forceinline__ F2() {}
  __device__ __forceinline__ explicit F2(float2 x) : v(x) {}
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ F2(double s) : v(make_float2((float)s, (float)s)) {}
};
struct P2 {
  float2 a, b;
  __device__ __forceinline__ operator F2() const { return F2(__fmul2_rn(a, b)); }
};
__device__ __forceinline__ float2 bcast(float k) { return make_float2(k, k); }
__device__ __forceinline__ F2 operator-(F2 x) { return F2(-x.v.x, -x.v.y); }
__device__ __forceinline__ F2 operator+(F2 x, F2 y) { return F2(__fadd2_rn(x.v, y.v)); }
__device__ __forceinline__ F2 operator-(F2 x, F2 y) { return F2(__fadd2_rn(x.v, (-y).v)); }
__device__ __forceinline__ P2 operator*(F2 x, F2 y) { return {x.v, y.v}; }
__device__ __forceinline__ P2 operator*(float k, F2 y) { return {bcast(k), y.v}; }
__device__ __forceinline__ P2 operator*(F2 y, float k) { return {y.v, bcast(k)}; }
__device__ __forceinline__ P2 operator*(P2 p, F2 y) { return {F2(p).v, y.v}; }
__device__ __forceinline__ P2 operator*(F2 y, P2 p) { return {y.v, F2(p).v}; }
__device__ __forceinline__ P2 operator*(P2 p, P2 q) { return {F2(p).v, F2(q).v}; }
__device__ __forceinline__ F2 operator+(P2 p, F2 c) { return F2(__ffma2_rn(p.a, p.b, c.v)); }
__device__ __forceinline__ F2 operator+(F2 c, P2 p) { return F2(__ffma2_rn(p.a, p.b, c.v)); }
__device__ __forceinline__ F2 operator+(P2 p, P2 q) { return F2(__ffma2_rn(p.a, p.b, F2(q).v)); }
__device__ __forceinline__ F2 operator-(P2 p, F2 c) { return F2(__ffma2_rn(p.a, p.b, (-c).v)); }
__device__ __forceinline__ F2 operator-(F2 c, P2 p) {
  return F2(__ffma2_rn((-F2(p.a)).v, p.b, c.v));
}
__device__ __forceinline__ F2 operator-(P2 p, P2 q) { return F2(__ffma2_rn(p.a, p.b, (-F2(q)).v)); }
__device__ __forceinline__ F2 recip(F2 x) { return F2(recip(x.v.x), recip(x.v.y)); }

template <typename R>
struct Groups {
  R S[4], C[4], X[4], Y[4];
};

template <typename R>
__device__ __forceinline__ void transform(const R f[16], Groups<R>& d) {
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const R p = f[4 * g] + f[4 * g + 2], q = f[4 * g + 1] + f[4 * g + 3];
    const R a = f[4 * g] - f[4 * g + 2], b = f[4 * g + 1] - f[4 * g + 3];
    d.S[g] = p + q;
    d.C[g] = p - q;
    if (g < 2) {
      d.X[g] = a;
      d.Y[g] = b;
    } else {
      d.X[g] = a - b;
      d.Y[g] = a + b;
    }
  }
}

// Inverse 4-point transform from scaled group values to populations.
template <typename R>
__device__ __forceinline__ void inverse_transform(const R S[4], const R C[4],
                                                  const R X[4], const R Y[4],
                                                  R out[16]) {
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const R P = S[g] + C[g], Q = S[g] - C[g];
    if (g < 2) {
      out[4 * g] = P + X[g];
      out[4 * g + 2] = P - X[g];
      out[4 * g + 1] = Q + Y[g];
      out[4 * g + 3] = Q - Y[g];
    } else {
      const R A = X[g] + Y[g], B = Y[g] - X[g];
      out[4 * g] = P + A;
      out[4 * g + 2] = P - A;
      out[4 * g + 1] = Q + B;
      out[4 * g + 3] = Q - B;
    }
  }
}

// Eq. 14 equilibria of the non-conserved moments from (rho, j, e), with
// P = rho T = e - |j|^2 / (2 rho) (gamma = 2, R = 1); m12 = m15 = m16 = 0.
template <typename R>
struct Eq {
  R m5, m6, m7, m8, m9, m10, m11, m13, m14, P;
};

template <typename R>
__device__ __forceinline__ Eq<R> equilibria(R rho, R jx, R jy, R e) {
  Eq<R> q;
  const R r = recip(rho);
  const R ux = jx * r, uy = jy * r;
  const R ux2 = ux * ux, uy2 = uy * uy, usq = ux2 + uy2;
  const R er = e * r;
  q.P = e - R(0.5) * rho * usq;
  const R eP = e + q.P;
  q.m5 = rho * (ux2 - uy2);                      // (jx^2 - jy^2) / rho
  q.m6 = jx * uy;                                // jx jy / rho
  q.m7 = eP * ux;                                // (e + P) jx / rho
  q.m8 = eP * uy;
  q.m9 = jx * (ux2 - R(3) * uy2);                // (jx^2 - 3 jy^2) jx / rho^2
  q.m10 = jy * (R(3) * ux2 - uy2);               // (3 jx^2 - jy^2) jy / rho^2
  q.m11 = R(2) * e * er - R(0.25) * rho * usq * usq;  // 2e^2/rho - |j|^4/(4 rho^3)
  const R A = R(6) * er - R(2) * usq;            // (6 rho e - 2|j|^2) / rho^2
  q.m13 = A * q.m5;
  q.m14 = A * q.m6;
  return q;
}

// f^eq = M^-1 f_hat^eq for the conserved moments (rho, j, e). KT: the
// coefficient type (R itself, or float for R = F2).
template <typename KT, typename R>
__device__ __forceinline__ void feq(const Coeffs<KT>& K, R rho, R jx, R jy, R e,
                                    R out[16]) {
  const Eq<R> q = equilibria(rho, jx, jy, e);
  R S[4], C[4], X[4], Y[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    S[g] = K.E0[g][0] * rho + K.E0[g][1] * e + K.E0[g][2] * q.m11;
    X[g] = K.EX[g][0] * jx + K.EX[g][1] * q.m7 + K.EX[g][2] * q.m9;
    Y[g] = K.EY[g][0] * jy + K.EY[g][1] * q.m8 + K.EY[g][2] * q.m10;
  }
  C[0] = K.EC[0][0] * q.m5 + K.EC[0][1] * q.m13;
  C[1] = K.EC[1][0] * q.m5 + K.EC[1][1] * q.m13;
  C[2] = K.ES[0][0] * q.m6 + K.ES[0][1] * q.m14;
  C[3] = K.ES[1][0] * q.m6 + K.ES[1][1] * q.m14;
  inverse_transform(S, C, X, Y, out);
}

// Conserved moments (rho, j_x, j_y, e) from the group values.
template <typename R>
struct Cons {
  R rho, jx, jy, e;
};

// Row r of a forward block (coefficients of type KT) times a group vector.
template <typename KT, typename R>
__device__ __forceinline__ R row4(const KT (&b)[4][4], int r, const R (&v)[4]) {
  return b[r][0] * v[0] + b[r][1] * v[1] + b[r][2] * v[2] + b[r][3] * v[3];
}

template <typename KT, typename R>
__device__ __forceinline__ Cons<R> conserved(const Coeffs<KT>& K, const Groups<R>& d) {
  Cons<R> c;
  c.rho = (d.S[0] + d.S[1]) + (d.S[2] + d.S[3]);
  c.e = row4(K.F0, 1, d.S);
  c.jx = row4(K.FX, 0, d.X);
  c.jy = row4(K.FY, 0, d.Y);
  return c;
}

// Collision of Eq. 3 at one node: df = M^-1 (-dt S_hat (m - m^eq)), given the
// group values and the equilibria q of the node. Returns P = rho T.
template <typename KT, typename R>
__device__ __forceinline__ R collide_q(const Coeffs<KT>& K, const Groups<R>& d, const Eq<R>& q,
                                       R df[16]) {
  const R d11 = row4(K.F0, 2, d.S) - q.m11;
  const R d12 = row4(K.F0, 3, d.S);                // m12^eq = 0
  const R d7 = row4(K.FX, 1, d.X) - q.m7;
  const R d9 = row4(K.FX, 2, d.X) - q.m9;
  const R d15 = row4(K.FX, 3, d.X);                // m15^eq = 0
  const R d8 = row4(K.FY, 1, d.Y) - q.m8;
  const R d10 = row4(K.FY, 2, d.Y) - q.m10;
  const R d16 = row4(K.FY, 3, d.Y);                // m16^eq = 0
  const R d5 = K.FC[0][0] * d.C[0] + K.FC[0][1] * d.C[1] - q.m5;
  const R d13 = K.FC[1][0] * d.C[0] + K.FC[1][1] * d.C[1] - q.m13;
  const R d6 = K.FS[0][0] * d.C[2] + K.FS[0][1] * d.C[3] - q.m6;
  const R d14 = K.FS[1][0] * d.C[2] + K.FS[1][1] * d.C[3] - q.m14;
  R S[4], C[4], X[4], Y[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    S[g] = K.K0[g][0] * d11 + K.K0[g][1] * d12;
    X[g] = K.KX[g][0] * d7 + K.KX[g][1] * d9 + K.KX[g][2] * d15;
    Y[g] = K.KY[g][0] * d8 + K.KY[g][1] * d10 + K.KY[g][2] * d16;
  }
  C[0] = K.KC[0][0] * d5 + K.KC[0][1] * d13;
  C[1] = K.KC[1][0] * d5 + K.KC[1][1] * d13;
  C[2] = K.KS[0][0] * d6 + K.KS[0][1] * d14;
  C[3] = K.KS[1][0] * d6 + K.KS[1][1] * d14;
  inverse_transform(S, C, X, Y, df);
  return q.P;
}

// The same, with the equilibria from the node's conserved moments c.
template <typename KT, typename R>
__device__ __forceinline__ R collide(const Coeffs<KT>& K, const Groups<R>& d,
                                     const Cons<R>& c, R df[16]) {
  return collide_q(K, d, equilibria(c.rho, c.jx, c.jy, c.e), df);
}

#endif  // __CUDACC__

}  // namespace d2v16
