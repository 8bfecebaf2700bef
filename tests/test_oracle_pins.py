"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the property it checks.  The references used here (closed forms, dense-matrix
brute force, an independent per-mode ODE, the exact Sauter spectrum) share no code with the
oracle's FFT, right-hand side or stepper.
"""
import json
import os

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import swf_oracle as O
from tests import pin_references as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ Dirac algebra and spinors
def test_clifford_algebra():
    for mu in range(4):
        for nu in range(4):
            ac = O.GAMMA[mu] @ O.GAMMA[nu] + O.GAMMA[nu] @ O.GAMMA[mu]
            assert np.allclose(ac, 2 * O.ETA[mu, nu] * np.eye(4), atol=1e-15)
    for k in range(3):
        assert np.allclose(O.ALPHA[k], R.ALPHA_D[k])
    assert np.allclose(O.BETA, R.BETA_D)


def test_spin_basis_relations():
    # Eq. A45: gamma^0 gamma^1 R_s = R_s, i gamma^2 gamma^3 R_s = s R_s, R_r^+ R_s = delta_rs
    g01 = O.GAMMA[0] @ O.GAMMA[1]
    g23 = 1j * O.GAMMA[2] @ O.GAMMA[3]
    for s in (+1, -1):
        Rs = O.R_SPIN[s]
        assert np.allclose(g01 @ Rs, Rs)
        assert np.allclose(g23 @ Rs, s * Rs)
        for r in (+1, -1):
            assert np.isclose(np.vdot(O.R_SPIN[r], Rs), 1.0 if r == s else 0.0)


@pytest.mark.parametrize("p", [(0.0, 0.0, 0.0), (0.3, -0.7, 0.2), (-1.5, 0.4, 0.0), (2.0, 0.0, 1.0)])
def test_free_spinors(p):
    p = np.array(p)
    p0 = O.energy(p)
    for s in (+1, -1):
        u = O.u_spinor(p, s)
        v = O.v_spinor(p, s)
        assert np.isclose(np.vdot(u, u).real, 1.0, atol=1e-14)  # unit norm (reading C-3)
        assert np.isclose(np.vdot(v, v).real, 1.0, atol=1e-14)
        assert np.allclose(O.h0_matrix(p) @ u, p0 * u, atol=1e-13)       # positive energy, momentum p
        assert np.allclose(O.h0_matrix(-p) @ v, -p0 * v, atol=1e-13)     # negative energy, momentum -p
        assert np.allclose((O.pslash(p) - np.eye(4)) @ u, 0, atol=1e-13)
        assert np.allclose((O.pslash(p) + np.eye(4)) @ v, 0, atol=1e-13)
        for r in (+1, -1):
            assert np.isclose(np.vdot(O.u_spinor(p, r), u), 1.0 if r == s else 0.0, atol=1e-14)
            assert np.isclose(np.vdot(O.v_spinor(p, r), v), 1.0 if r == s else 0.0, atol=1e-14)
    # completeness at one mode kappa: u_s(kappa) and v_s(-kappa) span C^4
    P = sum(np.outer(O.u_spinor(p, s), O.u_spinor(p, s).conj()) for s in (1, -1))
    P = P + sum(np.outer(O.v_spinor(-p, s), O.v_spinor(-p, s).conj()) for s in (1, -1))
    assert np.allclose(P, np.eye(4), atol=1e-13)
    # projectors (Eq. 23 up to the mode-label sign)
    Pp, Pm = O.energy_projector(p, +1), O.energy_projector(p, -1)
    assert np.allclose(Pp @ Pp, Pp) and np.allclose(Pm @ Pm, Pm)
    assert np.allclose(Pp + Pm, np.eye(4)) and np.allclose(Pp @ Pm, 0, atol=1e-14)
    assert np.allclose(Pp @ O.u_spinor(p, 1), O.u_spinor(p, 1))
    assert np.allclose(Pm @ O.v_spinor(-p, 1), O.v_spinor(-p, 1))


def test_polarisation_basis():
    # Eq. A58 with e = x and the photon along -y (the Breit-Wheeler workload): right-handed set
    perp, par = O.polarisation_basis((1, 0, 0), (0, -2, 0))
    assert np.allclose(perp, (0, 0, -1)) and np.allclose(par, (-1, 0, 0))
    assert np.allclose(np.cross(par, perp), (0, -1, 0))


def test_field_values():
    # spot values of the analytic fields
    f = O.Field("sauter_gauss", (0.3, 0.5, 5.0))
    a = O.gauge_potential(f, 0.0, np.array(0.0), np.array(0.0), np.array(0.0))
    assert np.isclose(a[1], 0.6) and a[0] == 0 and a[2] == 0
    a = O.gauge_potential(f, np.arccosh(2.0) / 0.5, np.array(5.0), np.array(0.0), np.array(0.0))
    assert np.isclose(a[1], 0.6 / 4 * np.exp(-1.0))
    g = O.Field("single_e", (0.25, 0.25, 0.125, 0.125, 0.0))
    a = O.gauge_potential(g, 0.0, np.array(4 * np.pi), np.array(0.0), np.array(0.0))
    assert np.isclose(a[0], -2.0 * np.sin(np.pi / 2) * np.exp(-(np.pi / 2) ** 2))
    d = O.Field("double_e", (0.25, 0.25, 0.125, 0.125, 0.0, 3.0))
    a = O.gauge_potential(d, 0.0, np.array(0.0), np.array(0.0), np.array(0.0))
    assert np.isclose(a[0], 0.0)  # odd single pulses at +-Dx cancel at x = 0
    pg = O.Field("pulse_gauss", (1.0, 0.5, 10.0, 8.0))
    a = O.gauge_potential(pg, 3.0, np.array(0.0), np.array(3.0 - np.pi), np.array(0.0))
    assert np.isclose(a[1], np.sin(0.5 * np.pi) * np.exp(-(np.pi ** 2) / 100.0))


# ------------------------------------------------------------------ spectral derivative (Eq. 10)
def test_spectral_derivative_sign_and_plane_waves():
    grid = O.Grid((8, 6, 1), (4.0, 3.0, 1.0))
    X, Y, Z = grid.coords()
    # d/dx sin(2 pi x/L) = (2 pi/L) cos(2 pi x/L): the i kappa convention of the FFT
    f = np.zeros((4,) + grid.n, dtype=complex)
    f[0] = np.sin(2 * np.pi * X / 4.0)
    h0 = O.h0_field(grid)
    hf = O.apply_h0(f, h0)
    # alpha^x maps component 0 to 3: (alpha^x (-i d/dx) f)_3 = -i (2 pi/L) cos
    assert np.allclose(hf[3], -1j * (2 * np.pi / 4.0) * np.cos(2 * np.pi * X / 4.0), atol=1e-12)
    # every grid plane wave is an eigenfunction with matrix alpha.kappa + beta, incl. trivial offset
    rng = np.random.default_rng(0)
    K = (0.0, 0.0, 0.37)
    h0K = O.h0_field(grid, K)
    for (ix, iy) in [(1, 0), (0, 2), (3, 5), (4, 3)]:
        kap = np.array([grid.kappa[0][ix], grid.kappa[1][iy], 0.37])
        spin = rng.normal(size=4) + 1j * rng.normal(size=4)
        wave = np.exp(1j * (kap[0] * X + kap[1] * Y))
        psi = spin[:, None, None, None] * wave[None]
        out = O.apply_h0(psi, h0K)
        assert np.allclose(out, (O.h0_matrix(kap) @ spin)[:, None, None, None] * wave[None], atol=1e-12)


def test_transform_on_grid_equals_direct_sum():
    grid = O.Grid((6, 4, 1), (5.0, 3.0, 1.0))
    rng = np.random.default_rng(1)
    psi = rng.normal(size=(4,) + grid.n) + 1j * rng.normal(size=(4,) + grid.n)
    spec = O.transform_on_grid(psi, grid)
    for ix in range(6):
        for iy in range(4):
            kap = (grid.kappa[0][ix], grid.kappa[1][iy], 0.0)
            assert np.allclose(spec[:, ix, iy, 0], O.transform_at(psi, grid, kap), atol=1e-12)


# ------------------------------------------------------------------ Dormand-Prince stepper
def _free_evolution_error(n_steps):
    grid = O.Grid((8, 4, 1), (6.0, 5.0, 1.0))
    rng = np.random.default_rng(2)
    y0 = rng.normal(size=(4,) + grid.n) + 1j * rng.normal(size=(4,) + grid.n)
    h0 = O.h0_field(grid)
    T0, T1 = 1.0, -2.0
    y, _ = O.dopri5_march(lambda t, y: -1j * O.apply_h0(y, h0), y0, T0, T1, n_steps)
    # exact: per mode exp(-i H0(kappa) (T1 - T0))
    spec0 = np.fft.fftn(y0, axes=(1, 2, 3))
    exact = np.zeros_like(spec0)
    for idx in np.ndindex(*grid.n):
        kap = [grid.kappa[a][idx[a]] for a in range(3)]
        exact[(slice(None),) + idx] = expm(-1j * O.h0_matrix(kap) * (T1 - T0)) @ spec0[(slice(None),) + idx]
    exact = np.fft.ifftn(exact, axes=(1, 2, 3))
    return np.max(np.abs(y - exact)) / np.max(np.abs(exact))


def test_dopri5_free_evolution_exact_and_fifth_order():
    e1 = _free_evolution_error(40)
    e2 = _free_evolution_error(80)
    assert e1 < 1e-5 and e2 < e1
    # global error of a 5th-order method falls by ~2^5 when the step halves
    assert 20.0 < e1 / e2 < 45.0, (e1, e2)


def test_dopri5_tableau_consistency():
    for i in range(1, 7):
        assert sum(O.DP_A[i]) == O.DP_C[i]
    assert sum(O.DP_B) == 1 and sum(O.DP_BSTAR) == 1
    assert O.DP_A[6] == O.DP_B[:6]
    # 5th-order conditions sum b_i c_i^k = 1/(k+1), k = 0..4
    for kk in range(5):
        assert sum(b * c ** kk for b, c in zip(O.DP_B, O.DP_C)) == O.Fraction(1, kk + 1)


# ------------------------------------------------------------------ the SWF march
def test_zero_field_gives_zero():
    grid = O.Grid((8, 8, 1), (8.0, 8.0, 1.0))
    psi = O.march_scattered(O.Field("zero"), grid, O.Background("U", (0.3, 0.1, 0.0), 1), -2.0, 2.0, 10)
    assert np.all(psi == 0)


def test_march_matches_dense_brute_force():
    """Whole semi-discrete system on a 4x4 grid: oracle Dopri5 vs dense Hamiltonian + DOP853."""
    grid = O.Grid((4, 4, 1), (6.0, 5.0, 1.0))
    fld = O.Field("sauter_gauss", (0.8, 0.6, 1.5))
    for bg in (O.Background("U", (0.4, -0.2, 0.0), 1), O.Background("V", (-0.3, 0.5, 0.0), -1)):
        t_in, t_out = -5.0, 5.0
        psi = O.march_scattered(fld, grid, bg, t_in, t_out, 400)
        X, Y, Z = grid.coords()
        ref = R.dense_march(lambda t: O.gauge_potential(fld, t, X, Y, Z), grid.n, grid.L, t_in, t_out,
                            lambda t: bg.values(grid, t), K=bg.offset())
        err = np.max(np.abs(psi - ref)) / np.max(np.abs(ref))
        assert err < 1e-8, err


def test_march_matches_dense_brute_force_1d_trivial_axes_and_a0():
    """A_0 field (Eq. 11) on a 1D grid with a trivial y axis carrying momentum p_y."""
    grid = O.Grid((8, 1, 1), (12.0, 1.0, 1.0))
    fld = O.Field("single_e", (0.6, 0.5, 0.4, 0.0, 0.0))
    bg = O.Background("U", (0.3, 0.6, 0.0), -1)
    psi = O.march_scattered(fld, grid, bg, -6.0, 6.0, 600)
    X, Y, Z = grid.coords()
    ref = R.dense_march(lambda t: O.gauge_potential(fld, t, X, Y, Z), grid.n, grid.L, -6.0, 6.0,
                        lambda t: bg.values(grid, t), K=bg.offset())
    assert np.max(np.abs(psi - ref)) / np.max(np.abs(ref)) < 1e-8


def test_time_only_field_matches_single_mode_solver():
    """Field of t alone: the SWF wave stays in the mode p; compare C at q = -p with a 4x4 ODE."""
    L = 2 * np.pi * 4
    grid = O.Grid((8, 8, 1), (L, L, 1.0))
    E, om = 0.5, 0.5
    fld = O.Field("sauter_gauss", (E, om, np.inf))
    p = np.array([grid.kappa[0][1], 0.0, 0.0])
    t_in, t_out = -14.0, 14.0
    for s in (+1, -1):
        bg = O.Background("U", tuple(p), s)
        psi = O.march_scattered(fld, grid, bg, t_in, t_out, 1400)
        C = O.c_spectrum(psi, grid, t_in)
        # mode of positron q = -p is kappa = p  -> index (1, 0, 0)
        a1 = lambda t: (E / om) / np.cosh(om * t) ** 2
        p0 = O.energy(p)
        phi = R.mode_march(a1, p, t_out, t_in, O.u_spinor(p, s) * np.exp(-1j * p0 * t_out))
        c = phi - O.u_spinor(p, s) * np.exp(-1j * p0 * t_in)
        for ir, r in enumerate((+1, -1)):
            ref = grid.volume * np.exp(1j * p0 * t_in) * (np.conj(c) @ O.v_spinor(-p, r))
            got = C[ir, 1, 0, 0]
            if r == s:
                assert abs(got - ref) / abs(ref) < 1e-7, (got, ref)
                assert abs(ref) ** 2 / grid.volume ** 2 > 1e-6
            else:  # spin along x is conserved for p_perp = 0 (cf. Eq. A46)
                assert abs(got) < 1e-12 * grid.volume and abs(ref) < 1e-12 * grid.volume


def test_single_mode_solver_matches_exact_sauter_spectrum():
    """Pins the independent mode solver itself against the exact Sauter-pulse spectrum."""
    E, om = 0.5, 0.5
    for p_par in (0.0, 0.4, -0.8):
        exact = R.sauter_pair_density(E, om, p_par)
        got = R.mode_pair_density(E, om, p_par, T=40.0)
        assert abs(got - exact) / exact < 1e-6, (p_par, got, exact)
    # constant-field limit of the closed form: exp(-pi (1 + p_perp^2)/E)
    assert np.isclose(R.sauter_pair_density(0.2, 0.002, 0.0), np.exp(-np.pi / 0.2), rtol=1e-3)


def test_norm_of_full_wave_is_conserved():
    """Grid p: psi_b + psi_s evolves unitarily, so its norm stays L^d (to stepper error)."""
    grid = O.Grid((16, 16, 1), (16.0, 16.0, 1.0))
    fld = O.Field("sauter_gauss", (1.0, 0.6, 2.5))
    p = (grid.kappa[0][2], grid.kappa[1][1], 0.0)
    bg = O.Background("U", p, 1)
    t_in, t_out = -6.0, 6.0
    psi = O.march_scattered(fld, grid, bg, t_in, t_out, 400)
    full = psi + bg.values(grid, t_in)
    assert abs(O.inner(full, full, grid).real / grid.volume - 1.0) < 1e-8
    assert O.inner(psi, psi, grid).real / grid.volume > 1e-4  # the field did scatter


def test_pair_number_two_lines_agree():
    """Eq. 8: |A + B|^2 = |C + D|^2 for grid momenta (reading C-1: the lines are equal)."""
    grid = O.Grid((16, 16, 1), (16.0, 16.0, 1.0))
    fld = O.Field("sauter_gauss", (1.2, 0.6, 2.5))
    t_in, t_out, nst = -6.0, 6.0, 400
    p = (grid.kappa[0][1], 0.0, 0.0)
    q = (-grid.kappa[0][1], grid.kappa[1][1], 0.0)
    for s, r in ((1, 1), (1, -1), (-1, 1)):
        bu = O.Background("U", p, s)
        bv = O.Background("V", q, r)
        pu = O.march_scattered(fld, grid, bu, t_in, t_out, nst)
        pv = O.march_scattered(fld, grid, bv, t_in, t_out, nst)
        res = O.pair_number(pu, pv, grid, t_in, p, s, q, r, bu.offset(), bv.offset())
        assert res["N_line2"] > 1e-8
        assert abs(res["N_line1"] - res["N_line2"]) / res["N_line2"] < 1e-7, res
        # C from the full spectrum equals the direct overlap at the grid mode of -q
        C = O.c_spectrum(pu, grid, t_in)
        # q = (-kappa_1, kappa_1): its mode kappa = -q sits at index (1, n_y - 1)
        assert np.isclose(C[0 if r == 1 else 1, 1, grid.n[1] - 1, 0],
                          res["C"], rtol=1e-10)


# ------------------------------------------------------------------ Breit-Wheeler (Sec. IV)
def _bw_setup_2d():
    grid = O.Grid((16, 16, 1), (8 * np.pi, 8 * np.pi, 1.0))
    fld = O.Field("sauter_gauss", (1.0, 0.7, 2.0))
    k = (0.0, -4 * grid.kappa[1][1], 0.0)  # grid mode
    perp, par = O.polarisation_basis((1, 0, 0), k)
    return grid, fld, O.Photon(k, tuple(par))


def test_bw_zero_field_gives_zero():
    grid, _, ph = _bw_setup_2d()
    res = O.bw_amplitude(O.Field("zero"), grid, (0.25, -1.0, 0), 1, (-0.25, -1.0, 0), 1, ph, -3.0, 3.0, 20)
    assert res["M"] == 0


def test_bw_t_in_independence():
    """Eq. 24: the t_in dependence cancels in M_past + M_finite."""
    grid, fld, ph = _bw_setup_2d()
    p, q = (0.25, -1.0, 0.0), (-0.25, -1.0, 0.0)
    t_out = 12.0
    # the field is sech^2(0.7 t) ~ 2e-7 at |t| = 12: the sum must agree to that level
    r1 = O.bw_amplitude(fld, grid, p, 1, q, 1, ph, -12.0, t_out, 600)
    r2 = O.bw_amplitude(fld, grid, p, 1, q, 1, ph, -15.0, t_out, 675)
    assert abs(r1["M"]) > 1e-3
    # the split between the two parts moves by O(1), the sum does not
    assert abs(r1["finite"][1] - r2["finite"][1]) > 0.1 * abs(r1["M"])
    assert abs(r1["M"] - r2["M"]) / abs(r1["M"]) < 2e-6, (r1["M"], r2["M"])


def test_bw_partial_integration_form_equals_past_finite_split():
    """The two ways of Sec. IV to handle t < t_in give the same amplitude: the partial-integration
    integrals of Eqs. 30-32 equal finite (Eq. 17) plus past (Eqs. 25-27) parts term by term, up to
    the time quadrature, whose error falls at least as fast as h^5 (Dormand-Prince)."""
    grid, fld, ph = _bw_setup_2d()
    p, q = (0.25, -1.0, 0.0), (-0.25, -1.0, 0.0)
    gaps = []
    for n_steps in (100, 200):
        r1 = O.bw_amplitude(fld, grid, p, 1, q, 1, ph, -9.0, 9.0, n_steps)
        r2 = O.bw_amplitude(fld, grid, p, 1, q, 1, ph, -9.0, 9.0, n_steps, form=2)
        assert np.all(r2["past"] == 0)
        # the split between finite and past parts is O(1); the partial-integration terms match the sums
        assert abs(r1["past"][0]) > 0.05 * abs(r1["M"])
        gaps.append(np.max(np.abs(r1["terms"] - r2["terms"])) / abs(r1["M"]))
    assert gaps[1] < 1e-6, gaps
    assert gaps[0] / gaps[1] > 20.0, gaps


def test_bw_step_size_controlled_march_converges_to_the_fixed_step_amplitude():
    """Breit-Wheeler with the paper's step-size-controlled Dopri5 (Sec. II.A) and M appended
    (Eq. 35): the amplitude approaches the fine fixed-step one as the tolerances tighten."""
    grid, fld, ph = _bw_setup_2d()
    p, q = (0.25, -1.0, 0.0), (-0.25, -1.0, 0.0)
    ref = O.bw_amplitude(fld, grid, p, 1, q, 1, ph, -9.0, 9.0, 800)["M"]
    gaps, steps = [], []
    for tol in ((1e-5, 1e-10), (1e-7, 1e-12)):
        r = O.bw_amplitude(fld, grid, p, 1, q, 1, ph, -9.0, 9.0, 50, adaptive=tol)
        gaps.append(abs(r["M"] - ref) / abs(ref))
        steps.append(r["accepted"])
    assert gaps[0] < 1e-5 and gaps[1] < gaps[0] / 20, gaps
    assert steps[1] > steps[0] > 50, steps


def test_bw_forms_agree_on_an_odd_axis_length():
    """On a grid with an odd axis length a V mode that wraps around the grid pairs with its U mode
    through the grid sum of their plane waves, N e^{i(kappa_v + k - kappa_u).x0} = -N: with that
    factor in the mode sums the past/finite split and the partial-integration form are again the
    same number (for grid momenta), up to the time quadrature."""
    grid = O.Grid((15, 12, 1), (7.5, 6.0, 1.0))
    fld = O.Field("sauter_gauss", (1.0, 0.7, 2.0))
    ux, uy = 2 * np.pi / 7.5, 2 * np.pi / 6.0
    k = (3 * ux, -uy, 0.0)
    perp, par = O.polarisation_basis((0, 0, 1), k)
    ph = O.Photon(k, tuple(par))
    p, q = (ux, -2 * uy, 0.0), (-2 * ux, -uy, 0.0)
    gaps = []
    for n_steps in (200, 400):
        r1 = O.bw_amplitude(fld, grid, p, 1, q, -1, ph, -10.0, 10.0, n_steps)
        r2 = O.bw_amplitude(fld, grid, p, 1, q, -1, ph, -10.0, 10.0, n_steps, form=2)
        gaps.append(np.max(np.abs(r1["terms"] - r2["terms"])) / abs(r1["terms"][0]))
    assert gaps[1] < 1e-7 and gaps[0] / gaps[1] > 20.0, gaps


def test_bw_t_in_independence_on_an_odd_axis_length():
    """Eq. 24 on a 15 x 12 grid, where V modes that wrap around the grid carry the factor
    N e^{i(kappa_v + k - kappa_u).x0} = -N in the scat-scat mode sum of Eq. 25.  The finite part
    (Eq. 17, an x-space integral without mode pairing) and the past part must still add up to an
    amplitude that does not depend on t_in.  Moving t_in from -12 to -15 shifts the finite parts
    by O(|M|) while the sum moves by 1e-7 |M| (the field's tail, sech^2(0.7 t) ~ 2e-7 at |t| = 12);
    with the wrap factor set to 1 the ss term moves by 7.7e-5 |M|, so this pins the factor against
    the x-space integral, independently of the partial-integration form."""
    grid = O.Grid((15, 12, 1), (7.5, 6.0, 1.0))
    fld = O.Field("sauter_gauss", (1.0, 0.7, 2.0))
    ux, uy = 2 * np.pi / 7.5, 2 * np.pi / 6.0
    k = (3 * ux, -uy, 0.0)
    perp, par = O.polarisation_basis((0, 0, 1), k)
    ph = O.Photon(k, tuple(par))
    p, q = (ux, -2 * uy, 0.0), (-2 * ux, -uy, 0.0)
    r1 = O.bw_amplitude(fld, grid, p, 1, q, -1, ph, -12.0, 12.0, 600)
    r2 = O.bw_amplitude(fld, grid, p, 1, q, -1, ph, -15.0, 12.0, 675)
    M = abs(r1["M"])
    assert M > 1e-3
    assert abs(r1["finite"][0] - r2["finite"][0]) > 1.0 * M
    assert np.max(np.abs(r1["terms"] - r2["terms"])) < 1e-6 * M, (r1["terms"], r2["terms"])


def test_bw_partial_integration_zero_field_gives_zero():
    grid, _, ph = _bw_setup_2d()
    res = O.bw_amplitude(O.Field("zero"), grid, (0.25, -1.0, 0), 1, (-0.25, -1.0, 0), 1, ph, -3.0, 3.0, 20, form=2)
    assert res["M"] == 0


def _photon_list(grid):
    du = grid.kappa[0][1]
    out = []
    for k in ((0.0, -4 * du, 0.0), (du, -4 * du, 0.0), (-2 * du, -3 * du, 0.0)):
        perp, par = O.polarisation_basis((1, 0, 0), k)
        out.append(O.Photon(k, tuple(par)))
        out.append(O.Photon(k, tuple(perp)))
    return out


def test_bw_photon_scan_equals_single_photon_solves():
    """One march serves every photon (the photon enters only the integrals of Eq. 14): the scan's
    amplitudes equal separate solves photon by photon."""
    grid, fld, _ = _bw_setup_2d()
    p, q = (0.25, -1.0, 0.0), (-0.25, -1.0, 0.0)
    photons = _photon_list(grid)[::2]
    scan = O.bw_photon_scan(fld, grid, p, 1, q, -1, photons, -6.0, 6.0, 80)
    for ph, got in zip(photons, scan):
        ref = O.bw_amplitude(fld, grid, p, 1, q, -1, ph, -6.0, 6.0, 80)
        assert abs(got["M"]) > 1e-3
        assert np.max(np.abs(got["terms"] - ref["terms"])) <= 1e-13 * abs(ref["M"])


def test_bw_wave_packet_finite_term_is_one_space_time_integral():
    """A photon wave packet sampled on grid momenta (Sec. IV, closing paragraphs): the finite-time
    terms with eps e^{-ikx} replaced by the packet f(t, x) = sum_j w_j eps_j e^{-i k_j x} equal the
    weighted sum of the plane-wave finite terms; and M is linear in the polarisation."""
    grid, fld, _ = _bw_setup_2d()
    p, q = (0.25, -1.0, 0.0), (-0.25, -1.0, 0.0)
    photons = _photon_list(grid)
    rng = np.random.default_rng(3)
    w = rng.normal(size=len(photons)) + 1j * rng.normal(size=len(photons))
    scan = O.bw_photon_scan(fld, grid, p, 1, q, 1, photons, -6.0, 6.0, 60)
    direct = O.bw_packet_finite(fld, grid, p, 1, q, 1, photons, w, -6.0, 6.0, 60)
    summed = sum(wj * r["finite"] for wj, r in zip(w, scan))
    assert np.max(np.abs(direct - summed)) <= 1e-12 * np.max(np.abs(summed))
    # photons 0 and 1 share k: their weighted sum is the photon with polarisation w0 eps0 + w1 eps1
    mix = O.Photon(photons[0].k, tuple(w[0] * np.asarray(photons[0].eps) + w[1] * np.asarray(photons[1].eps)))
    one = O.bw_amplitude(fld, grid, p, 1, q, 1, mix, -6.0, 6.0, 60)["M"]
    assert abs(one - (w[0] * scan[0]["M"] + w[1] * scan[1]["M"])) <= 1e-12 * abs(one)


@pytest.mark.parametrize("form", [1, 2])
def test_bw_spin_ratio_is_exact_in_1p1d(form):
    """Eq. A81 for the (1+1)D example of Sec. IV (golden fixture): |M(r != s)|^2/|M(r = s)|^2 = p_2^2,
    with either treatment of the times before t_in."""
    with open(os.path.join(GOLDEN, "bw_spin_ratio_1p1d.json")) as fh:
        gold = json.load(fh)
    c = gold["case"]
    E0, om = c["E0"], c["omega"]
    fld = O.Field("single_e", (E0, om, c["kappa_x"], 0.0, 0.0))
    n, L = 64, 64.0
    grid = O.Grid((n, 1, 1), (L, 1.0, 1.0))
    P = grid.kappa[0][2]
    rho = c["p2"]
    p, q = (P, rho, 0.0), (-P, rho, 0.0)
    k = (0.0, c["k2"], 0.0)
    perp, par = O.polarisation_basis((1, 0, 0), k)
    ph = O.Photon(k, tuple(par))
    amps = {}
    for r in (1, -1):
        for s in (1, -1):
            amps[(r, s)] = O.bw_amplitude(fld, grid, p, r, q, s, ph, -20.0, 20.0, 800, form=form)["M"]
    diag = abs(amps[(1, 1)]) ** 2
    assert diag > 1e-12
    assert np.isclose(abs(amps[(-1, -1)]) ** 2, diag, rtol=1e-6)
    for off in ((1, -1), (-1, 1)):
        assert np.isclose(abs(amps[off]) ** 2 / diag, gold["expected_ratio"], rtol=1e-5), amps


def test_bw_out_states_orthogonal():
    """(U_r^out | V_s^out) = 0 at t_in for grid momenta (the orthogonality used with Eq. A77)."""
    grid, fld, ph = _bw_setup_2d()
    p = (grid.kappa[0][1], grid.kappa[1][2], 0.0)
    q = (-grid.kappa[0][1], grid.kappa[1][3], 0.0)
    t_in, t_out = -5.0, 5.0
    bu, bv = O.Background("U", p, 1), O.Background("V", q, -1)
    pu, pv, _ = O.bw_march(fld, grid, bu, bv, ph, t_in, t_out, 300)
    uo = pu + bu.values(grid, t_in)
    vo = pv + bv.values(grid, t_in)
    assert abs(O.inner(uo, vo, grid)) / grid.volume < 1e-8
    assert abs(O.inner(pu, bv.values(grid, t_in), grid)) / grid.volume > 1e-6


def test_rhs_solves_covariant_equation():
    """The Hamiltonian right-hand side satisfies Eq. 6 as printed:
    (i gamma^mu (d_mu + i A_mu) - 1) psi_s = A-slash psi_b, with A-slash = gamma^mu A_mu."""
    grid = O.Grid((6, 5, 1), (5.0, 4.0, 1.0))
    rng = np.random.default_rng(3)
    psi = rng.normal(size=(4,) + grid.n) + 1j * rng.normal(size=(4,) + grid.n)
    # a field with all four components, to exercise every coupling term
    X, Y, Z = grid.coords()
    t0 = 0.3
    A = [0.4 * np.cos(X) * np.exp(-Y * Y / 4), 0.7 * np.exp(-X * X / 3), -0.5 * np.sin(Y), 0.2 + 0 * X]

    bg = O.Background("U", (0.3, -0.2, 0.0), -1)
    fld = O.Field("zero")
    orig = O.gauge_potential
    try:
        O.gauge_potential = lambda f, t, X_, Y_, Z_: tuple(a + 0 * X_ for a in A)
        dt = O.rhs(fld, grid, bg, O.h0_field(grid), t0, psi)
    finally:
        O.gauge_potential = orig
    # spatial derivatives by the explicit spectral matrix (no FFT routine)
    Dx = R.spectral_diff_matrix(grid.n[0], grid.L[0])
    Dy = R.spectral_diff_matrix(grid.n[1], grid.L[1])
    d = [dt, np.einsum("ij,ajk...->aik...", Dx, psi), np.einsum("jk,aik...->aij...", Dy, psi)]
    lhs = np.zeros_like(psi)
    for mu in range(3):  # d_3 = 0 on the trivial axis
        lhs += 1j * np.einsum("ab,b...->a...", O.GAMMA[mu], d[mu])
    for mu in range(4):
        lhs -= np.einsum("ab,b...->a...", O.GAMMA[mu], A[mu][None] * psi)
    lhs -= psi
    psib = bg.values(grid, t0)
    rhs = sum(np.einsum("ab,b...->a...", O.GAMMA[mu], A[mu][None] * psib) for mu in range(4))
    assert np.allclose(lhs, rhs, atol=1e-11)


def test_gauge_transformation_leaves_amplitudes_unchanged():
    """A_mu -> A_mu + d_mu chi with chi localised in space and time (negligible at t_in and
    t_out): psi -> exp(-i chi) psi, so the amplitudes at t_in (Eq. 8) do not change.  On the grid
    the spectral derivative and the multiplication by exp(-i chi) commute only up to aliasing,
    so the agreement improves with refinement; mid-march, where chi is large, the waves differ."""
    fld = O.Field("sauter_gauss", (0.8, 0.6, 2.5))
    shifted = O.GaugeShift(fld, chi0=0.6, tau=1.2, sigma=1.8)
    bg = O.Background("U", (0.3, -0.2, 0.0), 1)
    errs = []
    for n in (16, 32):
        grid = O.Grid((n, n, 1), (14.0, 14.0, 1.0))
        c0 = O.c_spectrum(O.march_scattered(fld, grid, bg, -6.0, 6.0, 300), grid, -6.0)
        c1 = O.c_spectrum(O.march_scattered(shifted, grid, bg, -6.0, 6.0, 300), grid, -6.0)
        errs.append(np.max(np.abs(c1 - c0)) / np.max(np.abs(c0)))
    assert errs[1] < 1e-5 and errs[1] < errs[0] / 100, errs
    grid = O.Grid((16, 16, 1), (14.0, 14.0, 1.0))
    m0 = O.c_spectrum(O.march_scattered(fld, grid, bg, 0.0, 6.0, 150), grid, 0.0)
    m1 = O.c_spectrum(O.march_scattered(shifted, grid, bg, 0.0, 6.0, 150), grid, 0.0)
    assert np.max(np.abs(m1 - m0)) / np.max(np.abs(m0)) > 0.1


@pytest.mark.parametrize("gam", [0.5, 1.0, 2.0])
def test_weak_field_exponent_of_the_sauter_spectrum(gam):
    """Weak field at fixed gamma = omega/E: ln n(p = 0) of E(t) = E sech^2(omega t) falls linearly
    in 1/E with the worldline-instanton exponent pi (2/(1 + sqrt(1 + gamma^2))) (constant-field
    limit pi).  Pins the closed form that pins the mode solver, which pins the oracle (above)."""
    Es = (0.05, 0.04, 0.03)
    ln = [np.log(R.sauter_pair_density(E, gam * E, 0.0)) for E in Es]
    slope = (ln[2] - ln[0]) / (1 / Es[2] - 1 / Es[0])
    expo = np.pi * 2 / (1 + np.sqrt(1 + gam ** 2))
    assert abs(slope + expo) < 1e-6 * expo, (slope, expo)
    assert abs((ln[1] - ln[0]) / (1 / Es[1] - 1 / Es[0]) + expo) < 1e-6 * expo


def test_spectral_convergence_under_grid_refinement():
    """Fixed box and a field negligible at its edge (exp(-36)): the amplitude C at fixed physical
    positron modes converges faster than any power as the grid is refined (brute force on tiny
    grids, 12^2 .. 36^2 against 48^2; measured 2e-2, 1.4e-4, 2.9e-6, 1.2e-11)."""
    fld = O.Field("sauter_gauss", (0.8, 0.6, 1.2))
    L = 12.0
    bg = O.Background("U", (2 * np.pi / L, 0.0, 0.0), 1)

    def c_at(n):
        grid = O.Grid((n, n, 1), (L, L, 1.0))
        C = O.c_spectrum(O.march_scattered(fld, grid, bg, -5.0, 5.0, 200), grid, -5.0)
        return C[0, 1, 0, 0], C[0, n - 1, 1, 0]  # modes (1, 0) and (-1, 1) in units of 2 pi / L

    ref = np.array(c_at(48))
    errs = [np.max(np.abs(np.array(c_at(n)) - ref)) / np.max(np.abs(ref)) for n in (12, 18, 24, 36)]
    assert all(errs[i] > 10 * errs[i + 1] for i in range(3)), errs
    assert errs[-1] < 1e-9, errs


def test_adaptive_dopri5_error_follows_the_tolerance():
    """The step-size-controlled march: its global error against a converged fixed-step march
    falls in proportion to the tolerance (Dormand-Prince 5(4) with the integral controller), a
    too-large first step is rejected and retried, and A = 0 stays exactly zero in a few steps."""
    fld = O.Field("sauter_gauss", (0.8, 0.6, 2.5))
    grid = O.Grid((16, 16, 1), (12.0, 12.0, 1.0))
    bg = O.Background("U", (0.3, -0.2, 0.0), 1)
    ref = O.march_scattered(fld, grid, bg, -6.0, 6.0, 4000)
    errs, steps = [], []
    for rtol in (1e-4, 1e-6):
        y, na, nr = O.march_scattered_adaptive(fld, grid, bg, -6.0, 6.0, 0.1, rtol, 1e-10)
        errs.append(np.max(np.abs(y - ref)) / np.max(np.abs(ref)))
        steps.append(na)
    assert errs[0] < 20 * 1e-4 and errs[1] < 20 * 1e-6 and errs[1] < errs[0] / 50, errs
    assert steps[1] > steps[0]
    y, na, nr = O.march_scattered_adaptive(fld, grid, bg, -6.0, 6.0, 3.0, 1e-5, 1e-10)
    assert nr > 0 and np.max(np.abs(y - ref)) / np.max(np.abs(ref)) < 2e-3
    y0, na0, nr0 = O.march_scattered_adaptive(O.Field("zero"), grid, bg, -6.0, 6.0, 0.1, 1e-5, 1e-10)
    assert np.all(y0 == 0) and na0 <= 4 and nr0 == 0
