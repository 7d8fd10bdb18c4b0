"""GPU tests of the von Neumann tool (include/lbm_vn.h) against the oracle of
Sec. IV (oracle/stability.py) and against closed forms.

Eigenvalue solver (lbm_eig16) on matrices with known spectra: triangular
(the diagonal, bit for bit), scaled identity and zero (exact), Hermitian (real,
equal to LAPACK's), a companion matrix (its polynomial's roots), random complex
matrices (LAPACK's eigenvalues, and the trace), a non-finite entry (NaN,
counted, neighbours unaffected).

Bars. G entries: 1e-13 relative to max |G| (G is built from the same
formula in two evaluation orders; entries are O(1)). Eigenvalues of random
Gaussian matrices: 1e-11 relative to the spectral norm (their condition
numbers are moderate; LAPACK's backward error is ~1e-15). Spectral radii of
G: the first-order perturbation bound kappa_max * 3 * 16 u ||G||_2 (u =
2^-53; kappa the eigenvalue condition numbers of the oracle's G from its left
and right eigenvectors; three backward errors of 16 u ||G||: the two
constructions of G and the two solvers). At the Sec. IV example (u = 10)
||G||_2 ~ 3e3 and kappa ~ 3e4, so rounding alone moves the eigenvalues by
~1e-8 there.
"""
import numpy as np
import pytest

from oracle import stability

pytestmark = pytest.mark.gpu

import workloads as W


U53 = 2.0 ** -53


def _radius_bar(G):
    """First-order bound on rounding-induced changes of G's eigenvalues."""
    import scipy.linalg as sl
    _, vl, vr = sl.eig(G, left=True, right=True)
    kappa = (np.linalg.norm(vl, axis=0) * np.linalg.norm(vr, axis=0)
             / np.abs(np.sum(vl.conj() * vr, axis=0)))
    return float(kappa.max() * 3 * 16 * U53 * np.linalg.norm(G, 2))


def _match(a, b):
    """Max distance between two multisets of complex numbers (optimal matching)."""
    from scipy.optimize import linear_sum_assignment
    d = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(d)
    return float(d[r, c].max())


def test_eig16_known_spectra():
    from paper_0908_3749_gb300 import lbm
    rng = np.random.default_rng(7)
    mats = []
    U = np.triu(rng.normal(size=(16, 16)) + 1j * rng.normal(size=(16, 16)))
    mats.append(U)
    mats.append((2.0 + 3.0j) * np.eye(16))
    mats.append(np.zeros((16, 16), complex))
    H = rng.normal(size=(16, 16)) + 1j * rng.normal(size=(16, 16))
    mats.append(H + H.conj().T)
    roots = 0.9 * np.exp(2j * np.pi * (np.arange(16) + 0.25) / 16)
    coef = np.poly(roots)                       # monic, degree 16
    Cm = np.zeros((16, 16), complex)
    Cm[0, :] = -coef[1:]
    Cm[1:, :-1] = np.eye(15)
    mats.append(Cm)
    omega, radius, nf = lbm.lbm_eig16(np.stack(mats))
    assert nf == 0
    key = lambda z: np.lexsort((z.imag, z.real))
    d = np.diag(U)
    assert np.array_equal(omega[0][key(omega[0])], d[key(d)])
    assert np.all(omega[1] == 2.0 + 3.0j) and abs(radius[1] - abs(2.0 + 3.0j)) <= 1e-15
    assert np.all(omega[2] == 0) and radius[2] == 0
    herm = mats[3]
    assert np.abs(omega[3].imag).max() <= 1e-13 * np.linalg.norm(herm, 2)
    np.testing.assert_allclose(np.sort(omega[3].real), np.linalg.eigvalsh(herm),
                               rtol=0, atol=1e-12 * np.linalg.norm(herm, 2))
    assert _match(omega[4], roots) < 1e-12
    assert abs(radius[4] - 0.9) < 1e-12


def test_eig16_random_matrices_match_lapack():
    from paper_0908_3749_gb300 import lbm
    rng = np.random.default_rng(11)
    n = 257                                      # 33 blocks, last one ragged
    A = rng.normal(size=(n, 16, 16)) + 1j * rng.normal(size=(n, 16, 16))
    A *= np.exp(rng.uniform(-3, 3, n))[:, None, None]
    omega, radius, nf = lbm.lbm_eig16(A)
    assert nf == 0
    worst = 0.0
    for i in range(n):
        nrm = np.linalg.norm(A[i], 2)
        ref = np.linalg.eigvals(A[i])
        worst = max(worst, _match(omega[i], ref) / nrm)
        assert abs(omega[i].sum() - np.trace(A[i])) <= 1e-13 * 16 * nrm
        assert abs(radius[i] - np.abs(omega[i]).max()) <= 1e-15 * radius[i]
    print("eig16: %d random matrices, worst eigenvalue error / ||A|| = %.3g" % (n, worst))
    assert worst < 1e-11


def test_eig16_nonfinite_matrix_is_reported():
    from paper_0908_3749_gb300 import lbm
    rng = np.random.default_rng(3)
    A = rng.normal(size=(3, 16, 16)).astype(complex)
    A[1, 4, 9] = np.nan
    omega, radius, nf = lbm.lbm_eig16(A)
    assert nf == 1
    assert np.isnan(radius[1]) and np.all(np.isnan(omega[1]))
    for i in (0, 2):
        assert _match(omega[i], np.linalg.eigvals(A[i])) < 1e-11 * np.linalg.norm(A[i], 2)


def _sweep_cases(seed, ncases):
    rng = np.random.default_rng(seed)
    states = np.stack([np.exp(rng.uniform(np.log(0.5), np.log(2.0), ncases)),
                       rng.uniform(-1, 1, ncases), rng.uniform(-1, 1, ncases),
                       np.exp(rng.uniform(np.log(0.5), np.log(2.0), ncases))], 1)
    rates = np.exp(rng.uniform(np.log(1e2), np.log(1e5), (ncases, 16)))
    k = np.stack([rng.uniform(-np.pi, np.pi, 24) / 2e-3, rng.uniform(-np.pi, np.pi, 24) / 3e-3], 1)
    k[0] = 0.0
    return states, rates, k


def test_vn_matrices_match_oracle():
    from paper_0908_3749_gb300 import lbm
    states, rates, k = _sweep_cases(1, 5)
    dx, dy, dt = 2e-3, 3e-3, 1e-5
    G = lbm.lbm_vn_matrices(lbm.vn_cases(states, rates), k, dx, dy, dt)
    worst = 0.0
    for c in range(len(states)):
        for q in range(len(k)):
            ref = stability.amplification_matrix(states[c], rates[c], dx, dy, dt, *k[q])
            worst = max(worst, float(np.abs(G[c, q] - ref).max() / np.abs(ref).max()))
    print("G: worst relative entry error %.3g" % worst)
    assert worst <= 1e-13


def test_vn_spectrum_matches_oracle_and_zero_k_closed_form():
    from paper_0908_3749_gb300 import lbm
    states, rates, k = _sweep_cases(2, 6)
    dx, dy, dt = 2e-3, 3e-3, 1e-5
    radius, omega, nf = lbm.lbm_vn_spectrum(lbm.vn_cases(states, rates), k, dx, dy, dt)
    assert nf == 0
    worst = 0.0
    for c in range(len(states)):
        for q in range(len(k)):
            G = stability.amplification_matrix(states[c], rates[c], dx, dy, dt, *k[q])
            ref = float(np.abs(stability.eigenvalues(G)).max())
            err = abs(radius[c, q] - ref)
            worst = max(worst, err)
            assert err <= _radius_bar(G), (c, q, err)
        closed = np.concatenate([np.ones(4), 1.0 - dt * rates[c, 4:]])
        assert _match(omega[c, 0], closed.astype(complex)) < 1e-12
    print("spectral radius: worst |GPU - oracle| = %.3g" % worst)


def test_paper_example_mrt_and_srt():
    """The Sec. IV example: both sides' max |omega| over k dx in [0, pi] along x
    agree; the values are reported (the paper's MRT-stable / SRT-unstable
    ordering is not reproduced under this reading of G)."""
    from paper_0908_3749_gb300 import lbm
    ex = W.vn_example(181)
    k = ex["k"]
    cases = lbm.vn_cases(ex["states"], ex["rates"])
    radius, _, nf = lbm.lbm_vn_spectrum(cases, k, ex["dx"], ex["dy"], ex["dt"], want_omega=False)
    assert nf == 0
    for c in range(2):
        for q in range(0, len(k), 4):
            G = stability.amplification_matrix(ex["states"][c], ex["rates"][c], ex["dx"], ex["dy"],
                                               ex["dt"], *k[q])
            ref = float(np.abs(stability.eigenvalues(G)).max())
            assert abs(radius[c, q] - ref) <= _radius_bar(G), (c, q)
    print("Sec. IV example: max |omega| MRT %.10f, SRT %.10f" % (radius[0].max(), radius[1].max()))


def test_device_pointers_give_the_host_results():
    import torch
    from paper_0908_3749_gb300 import lbm
    states, rates, k = _sweep_cases(3, 4)
    dx, dy, dt = 2e-3, 3e-3, 1e-5
    cases = lbm.vn_cases(states, rates)
    r_host, w_host, _ = lbm.lbm_vn_spectrum(cases, k, dx, dy, dt)
    dc = torch.from_numpy(cases).cuda()
    dk = torch.from_numpy(np.ascontiguousarray(k)).cuda()
    n = cases.shape[0] * k.shape[0]
    rr = torch.empty(n, dtype=torch.float64, device="cuda")
    ww = torch.empty(n * 32, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    lbm.lbm_vn_spectrum(dc, dk, dx, dy, dt, radius=rr, omega=ww, stream=s, count_nonconverged=False)
    torch.cuda.synchronize()
    assert np.array_equal(rr.cpu().numpy().reshape(r_host.shape), r_host)
    w = ww.cpu().numpy().view(np.complex128).reshape(w_host.shape)
    assert np.array_equal(w, w_host)


def test_eig16_power_of_two_scaling_is_exact():
    """The solver normalises each matrix by an exact power of two, so scaling
    the input by 2^k scales the computed eigenvalues by exactly 2^k, far into
    the ranges where squares of the raw entries would overflow or underflow."""
    from paper_0908_3749_gb300 import lbm
    rng = np.random.default_rng(5)
    A = rng.normal(size=(4, 16, 16)) + 1j * rng.normal(size=(4, 16, 16))
    w0, r0, _ = lbm.lbm_eig16(A)
    for k in (600, -600):
        w, r, nf = lbm.lbm_eig16(A * 2.0 ** k)
        assert nf == 0
        assert np.array_equal(w, w0 * 2.0 ** k)
        assert np.array_equal(r, r0 * 2.0 ** k)
