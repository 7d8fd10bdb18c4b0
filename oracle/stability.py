"""Linear (von Neumann) stability of the scheme, Sec. IV, in plain FP64 numpy.

Test infrastructure only (see ``oracle/__init__``).

Passage followed
----------------
Sec. IV: about a uniform state (rho, u, v, T) every population is split into
its constant equilibrium value plus a small disturbance Delta f_i; a Fourier
mode Delta f_i = F_i exp(i k.x) then grows by F^{t+dt} = G F^t per step with

  G_ij = delta_ij [1 - sum_a (v_ia dt / (2 dx_a)) (e^{i k_a dx_a} - e^{-i k_a dx_a})
                      + sum_a (1/2) (v_ia dt / dx_a)^2 (e^{i k_a dx_a} - 2 + e^{-i k_a dx_a})]
         - dt [M^-1 S_hat (dfhat/df - dfhat^eq/df)]_ij,

dfhat/df = M and dfhat^eq/df the derivative of the Eq. 14 equilibria
through the conserved moments. The scheme is von Neumann stable at the state
when max |omega| <= 1 over the eigenvalues omega of G and all k.

Readings
--------
V1  The paper differentiates f_hat^eq through (rho, T, u_a); the equilibria
    are functions of the conserved moments (rho, j, e) = rows 1-4 of M f, and
    (rho, u, T) <-> (rho, j, e) is one-to-one, so the chain rule through
    (rho, j, e) gives the same matrix: dfhat^eq/df = J M[0:4], J the 16 x 4
    derivative of Eq. 14 with respect to (rho, j_x, j_y, e).
V2  J is taken by complex-step differentiation (Squire and Trapp, SIAM Rev.
    40, 1998): for a real-analytic F, F'(x) = Im F(x + i h) / h + O(h^2) with
    no subtractive cancellation, so h = 1e-30 gives J to rounding.
V3  The advective part is summed over both axes (the formula's repeated
    index a), with no mixed x-y term, as in Eq. A.1.
V4  The single-relaxation-time version sets every s_k = 1 / tau.

Pins (tests/test_oracle_stability.py): with S_hat = 0 the eigenvalues are the
Lax-Wendroff factors 1 - i C sin(theta) - C^2 (1 - cos theta) per velocity
(closed form); at k = 0 they are 1 (four times, the conserved moments) and
1 - dt s_k (block-triangular structure of S_hat (I - J)); G applied to a
Fourier mode equals the linear part of one step of ``scheme.step`` on a
periodic grid (brute force through the nonlinear scheme).
"""
import numpy as np

from .lattice import matrices
from .scheme import conserved_from_state, moment_equilibria

__all__ = ["equilibrium_jacobian", "amplification_matrix", "eigenvalues", "spectral_radius"]


def equilibrium_jacobian(rho, u, v, T, h=1e-30):
    """dfhat^eq / d(rho, j_x, j_y, e) (16 x 4) of Eq. 14 at the state
    (readings V1, V2)."""
    c = np.array(conserved_from_state(rho, u, v, T), dtype=np.float64)
    J = np.empty((16, 4))
    for q in range(4):
        z = c.astype(np.complex128)
        z[q] += 1j * h
        J[:, q] = np.imag(moment_equilibria(*z)) / h
    return J


def amplification_matrix(state, s, dx, dy, dt, kx, ky):
    """G (16 x 16 complex) of Sec. IV for the uniform state (rho, u, v, T),
    rates s (16), grid spacings and time step, wave vector (kx, ky)."""
    vel, M, Minv = matrices()
    Cx = vel[:, 0] * dt / dx
    Cy = vel[:, 1] * dt / dy
    ex, ey = np.exp(1j * kx * dx), np.exp(1j * ky * dy)
    diag = (1.0
            - 0.5 * Cx * (ex - 1.0 / ex) + 0.5 * Cx ** 2 * (ex - 2.0 + 1.0 / ex)
            - 0.5 * Cy * (ey - 1.0 / ey) + 0.5 * Cy ** 2 * (ey - 2.0 + 1.0 / ey))
    dfeq_df = equilibrium_jacobian(*state) @ M[0:4, :]
    S = np.diag(np.asarray(s, dtype=np.float64))
    return np.diag(diag) - dt * (Minv @ S @ (M - dfeq_df))


def eigenvalues(G):
    """The eigenvalues omega of G (LAPACK through numpy)."""
    return np.linalg.eigvals(G)


def spectral_radius(state, s, dx, dy, dt, kx, ky):
    """max |omega| over the eigenvalues of G(kx, ky)."""
    return float(np.abs(eigenvalues(amplification_matrix(state, s, dx, dy, dt, kx, ky))).max())
