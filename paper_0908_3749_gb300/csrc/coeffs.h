// coeffs.h -- per-context constants of the D2V16 scheme (d2v16::Coeffs),
// shared by the grid step, the tube batch and the stability analysis.
//
//  lattice_constants : forward blocks and the scaled block inverses E* (the
//                      lattice alone: Eqs. 4, 5a-5p);
//  set_rates         : the back-map columns K* = E* w_k, w_k = -dt s_k (the
//                      relaxation of Eq. 3); host and device;
//  set_advection     : the Lax-Wendroff weights of Eq. A.1 per population.
#pragma once

#include <cmath>
#include <cstring>

#include "d2v16.cuh"

namespace d2v16 {

// Gauss-Jordan inverse with partial pivoting in long double (n <= 4).
inline bool invert_block(int n, const double* a, double* out) {
  long double m[4][8];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j)
      m[i][j] = j < n ? (long double)a[i * n + j] : (long double)(j - n == i);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(m[r][c]) > fabsl(m[p][c])) p = r;
    if (m[p][c] == 0.0L) return false;
    for (int j = 0; j < 2 * n; ++j) {
      const long double t = m[c][j];
      m[c][j] = m[p][j];
      m[p][j] = t;
    }
    const long double piv = m[c][c];
    for (int j = 0; j < 2 * n; ++j) m[c][j] /= piv;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const long double fac = m[r][c];
      for (int j = 0; j < 2 * n; ++j) m[r][j] -= fac * m[c][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) out[i * n + j] = (double)m[i][n + j];
  return true;
}

// Zeroes K, then fills the forward blocks and E* (K* and the weights stay 0).
inline bool lattice_constants(Coeffs<double>& K) {
  double m0[16], mx[16], my[16], mc[4], ms[4];
  for (int r = 0; r < 4; ++r)
    for (int g = 0; g < 4; ++g) {
      m0[4 * r + g] = b0(r, g);
      mx[4 * r + g] = bx(r, g);
      my[4 * r + g] = by(r, g);
    }
  for (int r = 0; r < 2; ++r)
    for (int g = 0; g < 2; ++g) {
      mc[2 * r + g] = bc2(r, g);
      ms[2 * r + g] = bs2(r, g);
    }
  double i0[16], ix[16], iy[16], ic[4], is[4];
  if (!invert_block(4, m0, i0) || !invert_block(4, mx, ix) || !invert_block(4, my, iy) ||
      !invert_block(2, mc, ic) || !invert_block(2, ms, is))
    return false;
  memset(&K, 0, sizeof(K));
  fill_forward(K);
  const double sx[4] = {0.5, 0.5, 0.25, 0.25};
  for (int g = 0; g < 4; ++g)
    for (int c = 0; c < 4; ++c) {
      K.E0[g][c] = 0.25 * i0[g * 4 + c];
      K.EX[g][c] = sx[g] * ix[g * 4 + c];
      K.EY[g][c] = sx[g] * iy[g * 4 + c];
    }
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      K.EC[r][c] = 0.25 * ic[r * 2 + c];
      K.ES[r][c] = 0.25 * is[r * 2 + c];
    }
  return true;
}

// K* = E* w for the non-conserved moments, w_k = -dt s_k; s holds s_1..s_16.
__host__ __device__ inline void set_rates(Coeffs<double>& K, double dt, const double* s) {
  const double w5 = -dt * s[4], w6 = -dt * s[5], w7 = -dt * s[6], w8 = -dt * s[7];
  const double w9 = -dt * s[8], w10 = -dt * s[9], w11 = -dt * s[10], w12 = -dt * s[11];
  const double w13 = -dt * s[12], w14 = -dt * s[13], w15 = -dt * s[14], w16 = -dt * s[15];
  for (int g = 0; g < 4; ++g) {
    K.K0[g][0] = K.E0[g][2] * w11;
    K.K0[g][1] = K.E0[g][3] * w12;
    K.KX[g][0] = K.EX[g][1] * w7;
    K.KX[g][1] = K.EX[g][2] * w9;
    K.KX[g][2] = K.EX[g][3] * w15;
    K.KY[g][0] = K.EY[g][1] * w8;
    K.KY[g][1] = K.EY[g][2] * w10;
    K.KY[g][2] = K.EY[g][3] * w16;
  }
  for (int r = 0; r < 2; ++r) {
    K.KC[r][0] = K.EC[r][0] * w5;
    K.KC[r][1] = K.EC[r][1] * w13;
    K.KS[r][0] = K.ES[r][0] * w6;
    K.KS[r][1] = K.ES[r][1] * w14;
  }
}

// Eq. A.1: f+ = a0 f + aE f(x+dx) + aW f(x-dx) + aN f(y+dy) + aS f(y-dy) + df,
// with the Courant numbers a_x = v_x dt / dx, a_y = v_y dt / dy.
inline void set_advection(Coeffs<double>& K, double dt, double dx, double dy) {
  for (int i = 0; i < 16; ++i) {
    const double ax = vel_x(i) * dt / dx, ay = vel_y(i) * dt / dy;
    K.a0[i] = 1.0 - ax * ax - ay * ay;
    K.aE[i] = 0.5 * (ax * ax - ax);
    K.aW[i] = 0.5 * (ax * ax + ax);
    K.aN[i] = 0.5 * (ay * ay - ay);
    K.aS[i] = 0.5 * (ay * ay + ay);
  }
}

}  // namespace d2v16
