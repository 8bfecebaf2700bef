"""Independent reference computations that pin the oracle (test-side only).

None of these reuse the oracle's FFT, right-hand side or Dormand-Prince stepper:
* ``dense_march``   builds the full semi-discrete Hamiltonian as a dense matrix from explicit
                    spectral-differentiation sums and integrates it with scipy's DOP853 at a
                    tight tolerance (brute force on tiny grids);
* ``mode_march``    integrates the 4x4 Dirac equation of one Fourier mode for a field of t alone;
* ``sauter_pair_density``  the exact pair spectrum of the Sauter pulse E(t) = E sech^2(omega t)
                    (Narozhny and Nikishov), used to check ``mode_march`` itself;
* ``mode_pair_density``    the same quantity from ``mode_march`` by projecting on the
                    eigenvectors of the asymptotic Hamiltonians (numpy.linalg.eigh, no spinor
                    formula of the oracle).
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import solve_ivp

S1 = np.array([[0, 1], [1, 0]], dtype=complex)
S2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
S3 = np.array([[1, 0], [0, -1]], dtype=complex)
Z2 = np.zeros((2, 2), dtype=complex)
I2 = np.eye(2, dtype=complex)
# alpha^k and beta written directly in the Dirac representation
ALPHA_D = [np.block([[Z2, s], [s, Z2]]) for s in (S1, S2, S3)]
BETA_D = np.block([[I2, Z2], [Z2, -I2]])


def spectral_diff_matrix(n: int, L: float) -> np.ndarray:
    """Periodic spectral d/dx on n points as an explicit n x n matrix (no FFT routine).

    D[j, l] = (1/n) sum_m (i kappa_m) exp(i kappa_m (x_j - x_l)), kappa_m = 2 pi m'/L with
    m' = m for m < n/2 and m - n otherwise (the Nyquist mode taken negative).
    """
    if n == 1:
        return np.zeros((1, 1), dtype=complex)
    dx = L / n
    x = np.arange(n) * dx
    m = np.arange(n)
    mp = np.where(m < (n + 1) // 2, m, m - n)
    if n % 2 == 0:
        mp[n // 2] = -n // 2
    kap = 2 * np.pi * mp / L
    diff = x[:, None] - x[None, :]
    return np.einsum("m,jlm->jl", 1j * kap, np.exp(1j * kap[None, None, :] * diff[:, :, None])) / n


def dense_h0(n, L, K=(0.0, 0.0, 0.0)) -> np.ndarray:
    """-i alpha.grad + alpha.K_trivial + beta as a dense (4N x 4N) matrix, index (comp, x, y, z)."""
    N = int(np.prod(n))
    eye = [np.eye(v, dtype=complex) for v in n]
    D = [spectral_diff_matrix(n[a], L[a]) for a in range(3)]
    H = np.kron(BETA_D, np.eye(N))
    for a in range(3):
        if n[a] > 1:
            ops = [eye[0], eye[1], eye[2]]
            ops[a] = -1j * D[a]
            H = H + np.kron(ALPHA_D[a], np.kron(ops[0], np.kron(ops[1], ops[2])))
        else:
            H = H + np.kron(ALPHA_D[a], np.eye(N)) * K[a]
    return H


def dense_march(A_func, n, L, t_in, t_out, psi_b_func, K=(0.0, 0.0, 0.0), rtol=1e-12, atol=1e-14):
    """psi_scat(t_in) of i d psi_s/dt = (H0 + V) psi_s + V psi_b by DOP853 (dense matrices).

    ``A_func(t)`` returns the four covariant potentials on the (nx, ny, nz) grid,
    ``psi_b_func(t)`` the background on the grid, shape (4, nx, ny, nz).
    """
    N = int(np.prod(n))
    H0 = dense_h0(n, L, K)

    def vmat(t):
        A = A_func(t)
        V = np.kron(np.eye(4), np.diag(A[0].ravel()))
        for k in range(3):
            if np.any(A[k + 1] != 0):
                V = V + np.kron(ALPHA_D[k], np.diag(A[k + 1].ravel()))
        return V

    def f(t, y):
        V = vmat(t)
        return -1j * ((H0 + V) @ y + V @ psi_b_func(t).reshape(4 * N))

    sol = solve_ivp(f, (t_out, t_in), np.zeros(4 * N, dtype=complex), method="DOP853",
                    rtol=rtol, atol=atol)
    assert sol.success
    return sol.y[:, -1].reshape((4,) + tuple(n))


def mode_march(a1_func, kappa, t_start, t_end, phi0, rtol=1e-12, atol=1e-14):
    """One Fourier mode of i d phi/dt = (alpha.kappa + beta + alpha^x A_1(t)) phi."""
    kappa = np.asarray(kappa, dtype=float)
    H0 = sum(ALPHA_D[a] * kappa[a] for a in range(3)) + BETA_D

    def f(t, y):
        return -1j * ((H0 + ALPHA_D[0] * a1_func(t)) @ y)

    sol = solve_ivp(f, (t_start, t_end), np.asarray(phi0, dtype=complex), method="DOP853",
                    rtol=rtol, atol=atol)
    assert sol.success
    return sol.y[:, -1]


def sauter_pair_density(E, omega, p_par, p_perp2=0.0):
    """Pair number per mode and spin for E(t) = E sech^2(omega t) (Narozhny-Nikishov).

    n = sinh[pi (2E/omega + w_- - w_+)/(2 omega)] sinh[pi (2E/omega - w_- + w_+)/(2 omega)]
        / [sinh(pi w_+/omega) sinh(pi w_-/omega)],   w_+- = sqrt(1 + p_perp^2 + (p_par +- E/omega)^2).
    """
    wp = np.sqrt(1 + p_perp2 + (p_par + E / omega) ** 2)
    wm = np.sqrt(1 + p_perp2 + (p_par - E / omega) ** 2)
    a = np.pi * (2 * E / omega + wm - wp) / (2 * omega)
    b = np.pi * (2 * E / omega - wm + wp) / (2 * omega)
    c = np.pi * wp / omega
    d = np.pi * wm / omega

    def log_sinh(x):  # log sinh(x) for x > 0 without overflow
        return x + np.log1p(-np.exp(-2 * x)) - np.log(2.0)

    return float(np.exp(log_sinh(a) + log_sinh(b) - log_sinh(c) - log_sinh(d)))


def mode_pair_density(E, omega, p_par, T):
    """Same quantity from ``mode_march``: A_1 = (E/omega) tanh(omega t) (E_x = dA_1/dt).

    Start in a negative-energy eigenvector of H(-T), evolve to +T, and return the weight on the
    positive-energy eigenspace of H(+T) (one spin state; the spin along x is conserved).
    """
    a1 = lambda t: (E / omega) * np.tanh(omega * t)

    def hmat(t):
        return ALPHA_D[0] * (p_par + a1(t)) + BETA_D

    w0, v0 = np.linalg.eigh(hmat(-T))
    phi0 = v0[:, 0]  # a negative-energy state
    phi = mode_march(a1, (p_par, 0.0, 0.0), -T, T, phi0)
    w1, v1 = np.linalg.eigh(hmat(T))
    pos = v1[:, w1 > 0]
    return float(np.sum(np.abs(pos.conj().T @ phi) ** 2))
