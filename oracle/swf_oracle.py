"""Plain, slow FP64 CPU oracle of the scattered-wave-function (SWF) Dirac method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  The product path (the CUDA library and its Python
binding) never imports it, and this module imports nothing from the product package.

It restates, in numpy float64/complex128 and in the paper's order, what the GPU path computes
(G. Torgrimsson, "Solving the Dirac equation on a GPU for strong-field processes in
multidimensional background fields"):

* Sec. II, Eqs. 2-9: dressed Dirac equation (i D-slash - 1) psi = 0 with D_mu = d_mu + i A_mu,
  split psi = psi_back + psi_scat (Eq. 4), inhomogeneous equation
  (i D-slash - 1) psi_scat = A-slash psi_back (Eq. 6) with psi_scat(t_out) = 0 (Eq. 7),
  pair number N(m, n) (Eq. 8) and the inner product (Eq. 9).
* Sec. II.A: pseudo-spectral spatial derivative (Eq. 10) and a Dormand-Prince 5(4) march from
  t_out back to t_in, here at a fixed step.
* Sec. III, Eqs. 11-12: the paper's example fields.
* Sec. IV, Eqs. 13-36: Breit-Wheeler amplitude M = M_ss + M_bs + M_sb, finite-time part by an
  integrand appended to the ODE state (Eqs. 33-35) and the analytic past part (Eqs. 24-27) built
  with the energy projectors of Eq. 23.
* App. A.5, Eqs. A44-A45: spinor basis u_s(p), v_s(p), R_s;  App. A.6, Eq. A58: photon
  polarisation basis.

Conventions (readings where the paper leaves a choice open):
* metric (+,-,-,-); A_mu covariant; Dirac representation of the gamma matrices;
  alpha^k = gamma^0 gamma^k, beta = gamma^0.
* Hamiltonian form of Eq. 6:  d psi_s/dt = -i [ H0 psi_s + V (psi_s + psi_b) ],
  H0 = alpha.kappa + beta applied per Fourier mode e^{i kappa.x}, V = A_0 + alpha^k A_k.
* Arrays are (4, nx, ny, nz) complex128 (the paper's (g, n_x, n_y, n_z) layout).  An axis with
  n = 1 is trivial: the field does not depend on it, its cell width is 1 (the delta function of
  that direction is stripped) and the marched wave carries a fixed momentum K along it
  (K = p for an electron wave U, K = -q for a positron wave V).
* Grid: x_j = -L/2 + j L/n, Fourier modes kappa = 2 pi fftfreq(n, L/n) (Nyquist negative).
* Discrete Fourier transform with the continuum normalisation
  psi~(kappa) = dx^d sum_x psi(x) e^{-i kappa.x}.
"""
from __future__ import annotations

from dataclasses import dataclass, field as dc_field
from fractions import Fraction

import numpy as np

# --------------------------------------------------------------------------------------------
# Dirac algebra (Sec. II; Dirac representation)
# --------------------------------------------------------------------------------------------
SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=complex),
    np.array([[0, -1j], [1j, 0]], dtype=complex),
    np.array([[1, 0], [0, -1]], dtype=complex),
)
_Z2 = np.zeros((2, 2), dtype=complex)
GAMMA0 = np.diag([1, 1, -1, -1]).astype(complex)
GAMMA = (GAMMA0,) + tuple(np.block([[_Z2, s], [-s, _Z2]]) for s in SIGMA)
ALPHA = tuple(GAMMA0 @ GAMMA[k] for k in (1, 2, 3))
BETA = GAMMA0
ETA = np.diag([1.0, -1.0, -1.0, -1.0])
ID4 = np.eye(4, dtype=complex)


def energy(p) -> float:
    """On-shell energy p_0 = sqrt(1 + |p|^2) (units c = hbar = m = 1, Sec. I)."""
    p = np.asarray(p, dtype=float)
    return float(np.sqrt(1.0 + p @ p))


def pslash(p) -> np.ndarray:
    """p-slash = gamma^mu p_mu = gamma^0 p_0 - gamma^k p^k for the on-shell momentum p."""
    p = np.asarray(p, dtype=float)
    return GAMMA0 * energy(p) - sum(GAMMA[k + 1] * p[k] for k in range(3))


# R_s of Eq. A45: gamma^0 gamma^1 R_s = R_s, i gamma^2 gamma^3 R_s = s R_s, R_r^+ R_s = delta_rs.
R_SPIN = {
    +1: np.array([1, 1, 1, 1], dtype=complex) / 2.0,
    -1: np.array([1, -1, -1, 1], dtype=complex) / 2.0,
}


def _spinor_norm(p) -> float:
    # sqrt(2 p_0 (p_0 + p_1)) of Eq. A44 with the covariant p_1 = -p^x.
    return float(np.sqrt(2.0 * energy(p) * (energy(p) - float(p[0]))))


def u_spinor(p, s: int) -> np.ndarray:
    """Electron spinor u_s(p) = (1 + p-slash) R_s / sqrt(2 p_0 (p_0 + p_1))  (Eq. A44)."""
    return (ID4 + pslash(p)) @ R_SPIN[s] / _spinor_norm(p)


def v_spinor(p, s: int) -> np.ndarray:
    """Positron spinor v_s(p) = (1 - p-slash) R_s / sqrt(2 p_0 (p_0 + p_1))  (Eq. A44)."""
    return (ID4 - pslash(p)) @ R_SPIN[s] / _spinor_norm(p)


def h0_matrix(kappa) -> np.ndarray:
    """Free Dirac Hamiltonian alpha.kappa + beta for the mode e^{i kappa.x} (Eq. 10 applied)."""
    kappa = np.asarray(kappa, dtype=float)
    return sum(ALPHA[k] * kappa[k] for k in range(3)) + BETA


def energy_projector(kappa, sign: int) -> np.ndarray:
    """Projector onto the energy-sign eigenspace of H0(kappa): (1 + sign H0/E)/2.

    sign = +1 picks the part evolving as e^{-iEt}, sign = -1 the part evolving as e^{+iEt}.
    In the paper's labelling (Eq. 23, modes e^{i Q_j x^j} = e^{-i Q.x}) this is Lambda_{-sign}.
    """
    return 0.5 * (ID4 + sign * h0_matrix(kappa) / energy(kappa))


def polarisation_basis(e_dir, k):
    """(eps_perp, eps_par) of Eq. A58 for the field direction e and photon momentum k."""
    e_dir = np.asarray(e_dir, dtype=float)
    k = np.asarray(k, dtype=float)
    perp = np.cross(e_dir, k)
    perp = perp / np.linalg.norm(perp)
    par = np.cross(perp, k)
    par = par / np.linalg.norm(par)
    return perp, par


# --------------------------------------------------------------------------------------------
# Grid (Sec. II.A)
# --------------------------------------------------------------------------------------------
@dataclass
class Grid:
    """Periodic box with n[a] points on [-L/2, L/2) per axis; n[a] = 1 marks a trivial axis."""

    n: tuple
    L: tuple

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        self.L = tuple(float(v) for v in self.L)
        assert len(self.n) == 3 and len(self.L) == 3
        self.dx = tuple(self.L[a] / self.n[a] if self.n[a] > 1 else 1.0 for a in range(3))
        self.x = tuple(
            (-self.L[a] / 2.0 + np.arange(self.n[a]) * self.dx[a]) if self.n[a] > 1 else np.zeros(1)
            for a in range(3)
        )
        self.kappa = tuple(
            (2.0 * np.pi * np.fft.fftfreq(self.n[a], self.dx[a])) if self.n[a] > 1 else np.zeros(1)
            for a in range(3)
        )
        self.cell = float(np.prod(self.dx))
        self.volume = float(np.prod([self.L[a] for a in range(3) if self.n[a] > 1]))

    def coords(self):
        return np.meshgrid(*self.x, indexing="ij")

    def modes(self, K=(0.0, 0.0, 0.0)):
        """Mode wave vectors on the grid; trivial axes carry the fixed momentum K."""
        ks = [self.kappa[a] + (K[a] if self.n[a] == 1 else 0.0) for a in range(3)]
        return np.meshgrid(*ks, indexing="ij")


# --------------------------------------------------------------------------------------------
# Background fields (Sec. III Eqs. 11-12, and the analytic workloads of the benchmarks)
# --------------------------------------------------------------------------------------------
@dataclass
class Field:
    """Analytic gauge potential A_mu(t, x) (covariant components).

    kind = "zero":          A = 0.
    kind = "sauter_gauss":  prm (E, omega, lam): A_1 = (E/omega) sech^2(omega t) exp(-r^2/lam^2),
                            r^2 over the non-trivial axes (lam = inf gives a field of t alone).
    kind = "pulse_gauss":   prm (a0, omega0, tau, w, wy): A_1 = a0 sin(omega0 (t - y))
                            exp(-(t - y)^2/tau^2 - x^2/w^2) [times exp(-y^2/wy^2) when wy > 0].
    kind = "single_e":      prm (E0, omega, kx, ky, kz): Eq. 11,
                            A_0 = -(E0/kx) sin(kx x) exp(-(omega t)^2 - (kx x)^2 - (ky y)^2 - (kz z)^2).
    kind = "double_e":      prm (E0, omega, kx, ky, kz, Dx): Eq. 12, A_0^one(x + Dx) + A_0^one(x - Dx).
    """

    kind: str
    prm: tuple = ()


@dataclass
class GaugeShift:
    """The potential of `base` plus the gradient of chi(t, x) = chi0 exp(-t^2/tau^2 - r^2/sigma^2)
    (r over the non-trivial axes): A_mu -> A_mu + d_mu chi, covariant components, so that with
    D_mu = d_mu + i A_mu (Eq. 2) a solution psi becomes exp(-i chi) psi."""

    base: Field
    chi0: float
    tau: float
    sigma: float


def gauge_potential(fld, t: float, X, Y, Z):
    """Return (A_0, A_1, A_2, A_3) on the coordinate arrays at time t."""
    zero = np.zeros(np.broadcast(X, Y, Z).shape)
    if isinstance(fld, GaugeShift):
        a = list(gauge_potential(fld.base, t, X, Y, Z))
        chi = fld.chi0 * np.exp(-t * t / fld.tau**2 - (X * X + Y * Y + Z * Z) / fld.sigma**2)
        a[0] = a[0] + (-2.0 * t / fld.tau**2) * chi          # d_t chi
        for k, xk in enumerate((X, Y, Z)):
            a[k + 1] = a[k + 1] + (-2.0 * xk / fld.sigma**2) * chi  # d_k chi = d chi / d x^k
        return tuple(a)
    if fld.kind == "zero":
        return zero, zero, zero, zero
    if fld.kind == "sauter_gauss":
        E, om, lam = fld.prm[:3]
        r2 = X * X + Y * Y + Z * Z
        a1 = (E / om) / np.cosh(om * t) ** 2 * np.exp(-r2 / lam**2)
        return zero, a1 + zero, zero, zero
    if fld.kind == "pulse_gauss":
        a0, om0, tau, w = fld.prm[:4]
        wy = fld.prm[4] if len(fld.prm) > 4 else 0.0
        u = t - Y
        a1 = a0 * np.sin(om0 * u) * np.exp(-(u * u) / tau**2 - (X * X) / w**2)
        if wy > 0:
            a1 = a1 * np.exp(-(Y * Y) / wy**2)
        return zero, a1 + zero, zero, zero
    if fld.kind in ("single_e", "double_e"):
        E0, om, kx, ky, kz = fld.prm[:5]

        def one(xs):
            return -(E0 / kx) * np.sin(kx * xs) * np.exp(
                -(om * t) ** 2 - (kx * xs) ** 2 - (ky * Y) ** 2 - (kz * Z) ** 2
            )

        if fld.kind == "single_e":
            a0 = one(X)
        else:
            dxs = fld.prm[5]
            a0 = one(X + dxs) + one(X - dxs)
        return a0 + zero, zero, zero, zero
    raise ValueError(f"unknown field kind {fld.kind!r}")


# --------------------------------------------------------------------------------------------
# Plane-wave backgrounds (Sec. II, Eqs. 3-5)
# --------------------------------------------------------------------------------------------
@dataclass
class Background:
    """psi_back of Eq. 5: kind "U" -> u_s(p) e^{-i(p_0 t - p.x)}, kind "V" -> v_s(p) e^{+i(p_0 t - p.x)}."""

    kind: str
    p: tuple
    s: int

    def spinor(self):
        return u_spinor(self.p, self.s) if self.kind == "U" else v_spinor(self.p, self.s)

    def offset(self):
        """Momentum carried along trivial axes: +p for U (mode e^{ipx}), -p for V (mode e^{-ipx})."""
        p = np.asarray(self.p, dtype=float)
        return tuple(p) if self.kind == "U" else tuple(-p)

    def values(self, grid: Grid, t: float):
        X, Y, Z = grid.coords()
        p = np.asarray(self.p, dtype=float)
        # trivial axes sit at x = 0: their plane-wave factor is carried by the mode offset
        px = [p[a] if grid.n[a] > 1 else 0.0 for a in range(3)]
        phase = energy(self.p) * t - (px[0] * X + px[1] * Y + px[2] * Z)
        sign = -1.0 if self.kind == "U" else 1.0
        return self.spinor()[:, None, None, None] * np.exp(1j * sign * phase)[None]


# --------------------------------------------------------------------------------------------
# Right-hand side of Eq. 6 with the spectral derivative of Eq. 10
# --------------------------------------------------------------------------------------------
def h0_field(grid: Grid, K=(0.0, 0.0, 0.0)):
    """H0(kappa) on every grid mode, shape (4, 4, nx, ny, nz)."""
    KX, KY, KZ = grid.modes(K)
    return (
        ALPHA[0][:, :, None, None, None] * KX[None, None]
        + ALPHA[1][:, :, None, None, None] * KY[None, None]
        + ALPHA[2][:, :, None, None, None] * KZ[None, None]
        + BETA[:, :, None, None, None]
    )


def apply_h0(psi, h0):
    """H0 psi by FFT -> (alpha.kappa + beta) -> inverse FFT (Eq. 10)."""
    spec = np.fft.fftn(psi, axes=(1, 2, 3))
    spec = np.einsum("ab...,b...->a...", h0, spec)
    return np.fft.ifftn(spec, axes=(1, 2, 3))


def apply_v(fld: Field, grid: Grid, t: float, phi):
    """V(t, x) phi with V = A_0 + alpha^k A_k (A covariant)."""
    X, Y, Z = grid.coords()
    a = gauge_potential(fld, t, X, Y, Z)
    out = a[0][None] * phi
    for k in range(3):
        if np.any(a[k + 1] != 0.0):
            out = out + np.einsum("ab,b...->a...", ALPHA[k], a[k + 1][None] * phi)
    return out


def rhs(fld: Field, grid: Grid, bg: Background, h0, t: float, psi_s):
    """d psi_s/dt = -i [ H0 psi_s + V (psi_s + psi_b) ]  (Eq. 6 in Hamiltonian form)."""
    return -1j * (apply_h0(psi_s, h0) + apply_v(fld, grid, t, psi_s + bg.values(grid, t)))


# --------------------------------------------------------------------------------------------
# Dormand-Prince 5(4) at a fixed step (Sec. II.A; Dormand & Prince 1980 tableau)
# --------------------------------------------------------------------------------------------
_F = Fraction
DP_C = [_F(0), _F(1, 5), _F(3, 10), _F(4, 5), _F(8, 9), _F(1), _F(1)]
DP_A = [
    [],
    [_F(1, 5)],
    [_F(3, 40), _F(9, 40)],
    [_F(44, 45), _F(-56, 15), _F(32, 9)],
    [_F(19372, 6561), _F(-25360, 2187), _F(64448, 6561), _F(-212, 729)],
    [_F(9017, 3168), _F(-355, 33), _F(46732, 5247), _F(49, 176), _F(-5103, 18656)],
    [_F(35, 384), _F(0), _F(500, 1113), _F(125, 192), _F(-2187, 6784), _F(11, 84)],
]
DP_B = [_F(35, 384), _F(0), _F(500, 1113), _F(125, 192), _F(-2187, 6784), _F(11, 84), _F(0)]
DP_BSTAR = [_F(5179, 57600), _F(0), _F(7571, 16695), _F(393, 640), _F(-92097, 339200),
            _F(187, 2100), _F(1, 40)]


def dopri5_march(f, y0, t_out: float, t_in: float, n_steps: int, stage_hook=None):
    """Fixed-step Dormand-Prince from t_out down to t_in (h < 0), first-same-as-last.

    ``f(t, y)`` is the right-hand side.  ``stage_hook(t_i, Y_i)`` (optional) returns the
    derivative of an appended quadrature variable at each stage, integrated with the same
    weights b_i (Eq. 35's Y = (psi, M) form).  Returns (y(t_in), appended integral).
    """
    h = (t_in - t_out) / n_steps
    c = [float(v) for v in DP_C]
    a = [[float(v) for v in row] for row in DP_A]
    b = [float(v) for v in DP_B]
    y = y0.copy()
    t = t_out
    k = [f(t, y)] + [None] * 6
    g = [stage_hook(t, y) if stage_hook else 0.0] + [0.0] * 6
    acc = 0.0
    for n in range(n_steps):
        t = t_out + n * h
        for i in range(1, 7):
            yi = y.copy()
            for j in range(i):
                if a[i][j] != 0.0:
                    yi = yi + (h * a[i][j]) * k[j]
            k[i] = f(t + c[i] * h, yi)
            if stage_hook is not None:
                g[i] = stage_hook(t + c[i] * h, yi)
            if i == 6:
                y_next = yi  # the 5th-order solution equals the last stage value (a_7j = b_j)
        if stage_hook is not None:
            acc = acc + h * sum(b[j] * g[j] for j in range(7))
        y = y_next
        k[0] = k[6]
        g[0] = g[6]
    return y, acc


def dopri5_adaptive(f, y0, t_out: float, t_in: float, h0: float, rtol: float, atol: float, max_attempts: int,
                    stage_hook=None, fields_axis0: bool = False):
    """Dormand-Prince 5(4) with step-size control (the integrator Sec. II.A names: Dopri5 with
    relative and absolute tolerances), from t_out down to t_in (h < 0), first-same-as-last.

    Error of a step: e = h sum_i (b_i - b*_i) k_i (fifth- minus fourth-order solution); scaled
    norm err = sqrt(mean(|e|^2 / (atol + rtol max(|y_n|, |y_n+1|))^2)) over all complex entries
    (with fields_axis0: over each field y[f] separately, err the largest of them).
    The step is accepted when err <= 1; the next step is h * min(10, max(0.2, 0.9 err^(-1/5)))
    (the standard integral controller), never passing t_in.  Returns (y(t_in), accepted,
    rejected), and with ``stage_hook(t_i, Y_i)`` also the appended quadrature variable, integrated
    with the weights b_i over the accepted steps (Eq. 35's Y = (psi, M) form).
    """
    c = [float(v) for v in DP_C]
    a = [[float(v) for v in row] for row in DP_A]
    db = [float(DP_B[j] - DP_BSTAR[j]) for j in range(7)]
    y = y0.copy()
    t = t_out
    span = abs(t_in - t_out)
    h = -abs(h0) if t_in < t_out else abs(h0)
    b = [float(v) for v in DP_B]
    k = [f(t, y)] + [None] * 6
    g = [stage_hook(t, y) if stage_hook else 0.0] + [0.0] * 6
    acc = 0.0
    accepted = rejected = 0
    while abs(t_in - t) > 1e-12 * span:
        if accepted + rejected >= max_attempts:
            raise RuntimeError("adaptive march: too many attempts")
        if abs(h) > abs(t_in - t):
            h = t_in - t
        for i in range(1, 7):
            yi = y.copy()
            for j in range(i):
                if a[i][j] != 0.0:
                    yi = yi + (h * a[i][j]) * k[j]
            k[i] = f(t + c[i] * h, yi)
            if stage_hook is not None:
                g[i] = stage_hook(t + c[i] * h, yi)
        y_new = yi
        e = h * sum(db[j] * k[j] for j in range(7) if db[j] != 0.0)
        sc = atol + rtol * np.maximum(np.abs(y), np.abs(y_new))
        q = (np.abs(e) / sc) ** 2
        if fields_axis0:
            err = float(max(np.sqrt(np.mean(q[fi])) for fi in range(q.shape[0])))
        else:
            err = float(np.sqrt(np.mean(q)))
        fac = 10.0 if err == 0.0 else min(10.0, max(0.2, 0.9 * err ** -0.2))
        if err <= 1.0:
            if stage_hook is not None:
                acc = acc + h * sum(b[j] * g[j] for j in range(7))
                g[0] = g[6]
            t = t + h
            y = y_new
            k[0] = k[6]
            accepted += 1
        else:
            rejected += 1
        h = h * fac
    if stage_hook is not None:
        return y, accepted, rejected, acc
    return y, accepted, rejected


def march_scattered_adaptive(fld: Field, grid: Grid, bg: Background, t_in, t_out, h0, rtol, atol,
                             max_attempts=100000):
    """psi_scat(t_in) of Eqs. 6-7 with the step-size-controlled march."""
    h0f = h0_field(grid, bg.offset())
    y0 = np.zeros((4,) + grid.n, dtype=complex)
    return dopri5_adaptive(lambda t, y: rhs(fld, grid, bg, h0f, t, y), y0, t_out, t_in, h0, rtol, atol,
                           max_attempts)


def march_scattered(fld: Field, grid: Grid, bg: Background, t_in, t_out, n_steps):
    """psi_scat(t_in) for psi_scat(t_out) = 0 (Eq. 7), marched backward through Eq. 6."""
    h0 = h0_field(grid, bg.offset())
    y0 = np.zeros((4,) + grid.n, dtype=complex)
    y, _ = dopri5_march(lambda t, y: rhs(fld, grid, bg, h0, t, y), y0, t_out, t_in, n_steps)
    return y


# --------------------------------------------------------------------------------------------
# Overlaps at t_in (Eqs. 8-9) and the Schwinger pair number
# --------------------------------------------------------------------------------------------
def inner(psi, phi, grid: Grid):
    """(psi|phi) = integral d^dx psi^+ phi on the grid (Eq. 9)."""
    return grid.cell * np.sum(np.conj(psi) * phi)


def transform_on_grid(psi, grid: Grid):
    """psi~(kappa) = dx^d sum_x psi(x) e^{-i kappa.x} on every grid mode (library FFT)."""
    spec = np.fft.fftn(psi, axes=(1, 2, 3)) * grid.cell
    KX, KY, KZ = np.meshgrid(*grid.kappa, indexing="ij")
    # the grid starts at x = -L/2 instead of 0
    shift = np.exp(1j * (KX * grid.x[0][0] + KY * grid.x[1][0] + KZ * grid.x[2][0]))
    return spec * np.conj(shift)[None]


def transform_at(psi, grid: Grid, kappa):
    """psi~(kappa) at one arbitrary wave vector by the direct sum (off-grid momenta)."""
    X, Y, Z = grid.coords()
    kappa = np.asarray(kappa, dtype=float)
    kk = [kappa[a] if grid.n[a] > 1 else 0.0 for a in range(3)]
    ph = np.exp(-1j * (kk[0] * X + kk[1] * Y + kk[2] * Z))
    return grid.cell * np.sum(psi * ph[None], axis=(1, 2, 3))


def c_spectrum(psi_u, grid: Grid, t_in: float, K=(0.0, 0.0, 0.0)):
    """C(m, (r, q)) = (U_scat^out(m) | V_back(r, q)) at t_in for every grid positron.

    The positron with momentum q occupies the grid mode kappa = -q, so the entry at mode
    index j belongs to q = -kappa_j.  Shape (2, nx, ny, nz); r = +1 first.
    """
    spec = transform_on_grid(psi_u, grid)
    KX, KY, KZ = grid.modes(K)
    out = np.zeros((2,) + grid.n, dtype=complex)
    for idx in np.ndindex(*grid.n):
        q = -np.array([KX[idx], KY[idx], KZ[idx]])
        for ir, r in enumerate((+1, -1)):
            v = v_spinor(q, r)
            out[(ir,) + idx] = np.exp(1j * energy(q) * t_in) * (np.conj(spec[(slice(None),) + idx]) @ v)
    return out


def overlap_u_scat_v_back(psi_u, grid, t_in, q, r):
    """(U_scat | V_back(r, q)) at t_in for any q (direct transform at kappa = -q)."""
    spec = transform_at(psi_u, grid, -np.asarray(q, dtype=float))
    return np.exp(1j * energy(q) * t_in) * (np.conj(spec) @ v_spinor(q, r))


def overlap_u_back_v_scat(psi_v, grid, t_in, p, s):
    """A(m, n) = (U_back(s, p) | V_scat) at t_in for any p (direct transform at kappa = p)."""
    spec = transform_at(psi_v, grid, np.asarray(p, dtype=float))
    return np.exp(1j * energy(p) * t_in) * (np.conj(u_spinor(p, s)) @ spec)


def pair_number(psi_u, psi_v, grid: Grid, t_in, p, s, q, r, K_u=(0, 0, 0), K_v=(0, 0, 0)):
    """Both lines of Eq. 8 for electron m = (s, p), positron n = (r, q).

    Line 1: A + B, A = (U_back m | V_scat n), B = sum_i (U_scat m | U_back i)(U_back i | V_scat n).
    Line 2: C + D, C = (U_scat m | V_back n), D = sum_i (U_scat m | V_back i)(V_back i | V_scat n).
    The sum over i = (s', Q) runs over both spins and every grid mode with the weight L^{-d}
    (a resolution of the identity on the grid).  Returns dict with A, B, C, D and both |.|^2.
    """
    su = transform_on_grid(psi_u, grid)
    sv = transform_on_grid(psi_v, grid)
    KXu, KYu, KZu = grid.modes(K_u)
    KXv, KYv, KZv = grid.modes(K_v)
    A = overlap_u_back_v_scat(psi_v, grid, t_in, p, s)
    C = overlap_u_scat_v_back(psi_u, grid, t_in, q, r)
    B = 0.0 + 0.0j
    D = 0.0 + 0.0j
    for idx in np.ndindex(*grid.n):
        sl = (slice(None),) + idx
        Q = np.array([KXu[idx], KYu[idx], KZu[idx]])   # U_back(s', Q) lives in mode Q
        for sp in (+1, -1):
            u = u_spinor(Q, sp)
            e = energy(Q)
            uu = np.exp(-1j * e * t_in) * (np.conj(su[sl]) @ u)     # (U_scat | U_back i)
            uv = np.exp(1j * e * t_in) * (np.conj(u) @ sv[sl])      # (U_back i | V_scat)
            B += uu * uv
        Qv = -np.array([KXv[idx], KYv[idx], KZv[idx]])  # V_back(s', Q) lives in mode -Q
        for sp in (+1, -1):
            v = v_spinor(Qv, sp)
            e = energy(Qv)
            cu = np.exp(1j * e * t_in) * (np.conj(su[sl]) @ v)      # (U_scat | V_back i)
            wv = np.exp(-1j * e * t_in) * (np.conj(v) @ sv[sl])     # (V_back i | V_scat)
            D += cu * wv
    B /= grid.volume
    D /= grid.volume
    return {"A": A, "B": B, "C": C, "D": D,
            "N_line1": abs(A + B) ** 2, "N_line2": abs(C + D) ** 2}


# --------------------------------------------------------------------------------------------
# Nonlinear Breit-Wheeler (Sec. IV)
# --------------------------------------------------------------------------------------------
@dataclass
class Photon:
    """Plane-wave photon e^{-ikx} with polarisation eps_mu = (0, eps) (Eq. 13)."""

    k: tuple
    eps: tuple

    def k0(self):
        return float(np.linalg.norm(self.k))

    def alpha_eps(self):
        # gamma^0 eps-slash = gamma^0 gamma^k eps_k = alpha . eps
        return sum(ALPHA[a] * self.eps[a] for a in range(3))


def bw_integrand(grid, photon, bg_u, bg_v, t, psi_u, psi_v):
    """dM_{a,b}/dt of the finite-time terms (the integrand of Eq. 17): dx^d sum_x U_a^+ (alpha.eps) V_b e^{-ikx}.

    Returns the three terms (ss, bs, sb) as a complex array of length 3.
    """
    X, Y, Z = grid.coords()
    k = np.asarray(photon.k, dtype=float)
    kk = [k[a] if grid.n[a] > 1 else 0.0 for a in range(3)]
    ph = np.exp(-1j * photon.k0() * t + 1j * (kk[0] * X + kk[1] * Y + kk[2] * Z))
    ae = photon.alpha_eps()
    ub = bg_u.values(grid, t)
    vb = bg_v.values(grid, t)

    def term(uu, vv):
        return grid.cell * np.sum(np.einsum("a...,ab,b...->...", np.conj(uu), ae, vv) * ph)

    return np.array([term(psi_u, psi_v), term(ub, psi_v), term(psi_u, vb)])


class PartialIntegrationTables:
    """Time-independent pieces of the partial-integration integrand (Sec. IV, Eqs. 28-33).

    For every U grid mode kappa_u (index idx) the V mode is kappa_v = kappa_u - k (index
    idx - shift, periodic, as in the past terms).  Holds the energy projectors of both modes,
    the four denominators Omega = sigma E_u - sigma' E_v - k0 and the factor
    e^{i(kappa_v + k - kappa_u).x0} that the grid sum of the pair's plane waves carries (1 unless
    the V mode wrapped around the grid, then -1 on an odd axis length).
    """

    def __init__(self, grid, photon, bg_u, bg_v):
        k = np.asarray(photon.k, dtype=float)
        self.shift = []
        for a in range(3):
            if grid.n[a] > 1:
                m = k[a] * grid.L[a] / (2.0 * np.pi)
                assert abs(m - round(m)) < 1e-9, "photon momentum must be a grid mode"
                self.shift.append(int(round(m)))
            else:
                self.shift.append(0)
        ku = np.stack(grid.modes(bg_u.offset()))
        kv = np.stack(grid.modes(bg_v.offset()))
        # V quantities moved onto the U mode they pair with: entry idx holds mode idx - shift
        kv = np.roll(kv, self.shift, axis=(1, 2, 3))
        self.eu = np.sqrt(1.0 + np.sum(ku * ku, axis=0))
        self.ev = np.sqrt(1.0 + np.sum(kv * kv, axis=0))

        def proj(kk, e, sign):
            h = sum(ALPHA[a][:, :, None, None, None] * kk[a][None, None] for a in range(3)) + BETA[:, :, None, None, None]
            return 0.5 * (ID4[:, :, None, None, None] + sign * h / e[None, None])

        self.pu = {sg: proj(ku, self.eu, sg) for sg in (1, -1)}
        self.pv = {sg: proj(kv, self.ev, sg) for sg in (1, -1)}
        k0 = photon.k0()
        self.omega = {(sg, sgp): sg * self.eu - sgp * self.ev - k0 for sg in (1, -1) for sgp in (1, -1)}
        X0 = [grid.x[a][0] if grid.n[a] > 1 else 0.0 for a in range(3)]
        kk = [k[a] if grid.n[a] > 1 else 0.0 for a in range(3)]
        self.wrap = np.exp(1j * sum((kv[a] + kk[a] - ku[a]) * X0[a] for a in range(3)))

    def on_u_modes(self, spec_v):
        """A V spectrum re-indexed so that entry idx holds V~(kappa_u(idx) - k)."""
        return np.roll(spec_v, self.shift, axis=(1, 2, 3))


def bw_integrand_partial(fld, grid, photon, bg_u, bg_v, tabs, t, psi_u, psi_v):
    """dM_{a,b}/dt of the partial-integration form (Eqs. 30-33) for (ss, bs, sb).

    With the grid transform psi~(kappa) and the energy projectors P_sigma of Eq. 23, the split
    parts of Eq. 29 are P_sigma psi~ e^{+i sigma E t} (free oscillation removed).  Their time
    derivative is P_sigma (d/dt + i H0) psi~ = P_sigma F[-i V (psi_s + psi_b)] (Eq. 6), so
    (i e^{i Omega t} / Omega) d/dt[...] of Eq. 33 becomes, after the phases cancel against
    e^{i Omega t},
        ss: (i e^{-i k0 t} / L^d) sum_kappa sum_{sigma,sigma'}
            [(P_s dU~)^+ (alpha.eps) P_s' V~ + (P_s U~)^+ (alpha.eps) P_s' dV~] / Omega_{s s'}
        bs: i e^{i (p0 - k0) t} sum_s' u^+ (alpha.eps) P_s'(p - k) dV~(p - k) / (p0 - s' E - k0)
        sb: i e^{i (q0 - k0) t} sum_s (P_s(k - q) dU~(k - q))^+ (alpha.eps) v / (s E + q0 - k0)
    with dU = -i V (U_scat + U_back), dV = -i V (V_scat + V_back) at time t.
    """
    k0 = photon.k0()
    ae = photon.alpha_eps()
    du = -1j * apply_v(fld, grid, t, psi_u + bg_u.values(grid, t))
    dv = -1j * apply_v(fld, grid, t, psi_v + bg_v.values(grid, t))
    su = transform_on_grid(psi_u, grid)
    sdu = transform_on_grid(du, grid)
    sv = tabs.on_u_modes(transform_on_grid(psi_v, grid))
    sdv = tabs.on_u_modes(transform_on_grid(dv, grid))

    def proj(P, x):
        return np.einsum("ab...,b...->a...", P, x)

    def form(x, y):
        return np.einsum("a...,ab,b...->...", np.conj(x), ae, y)

    ss = 0.0 + 0.0j
    for sg in (1, -1):
        pu, pdu = proj(tabs.pu[sg], su), proj(tabs.pu[sg], sdu)
        for sgp in (1, -1):
            pv, pdv = proj(tabs.pv[sgp], sv), proj(tabs.pv[sgp], sdv)
            ss += np.sum(tabs.wrap * (form(pdu, pv) + form(pu, pdv)) / tabs.omega[(sg, sgp)])
    ss = 1j * np.exp(-1j * k0 * t) * ss / grid.volume
    k = np.asarray(photon.k, dtype=float)
    p = np.asarray(bg_u.p, dtype=float)
    kv = p - k
    dvk = transform_at(dv, grid, kv)
    u = bg_u.spinor()
    bs = 0.0 + 0.0j
    for sgp in (1, -1):
        bs += (np.conj(u) @ ae @ (energy_projector(kv, sgp) @ dvk)) / (energy(p) - sgp * energy(kv) - k0)
    bs = 1j * np.exp(1j * (energy(p) - k0) * t) * bs
    q = np.asarray(bg_v.p, dtype=float)
    ku = k - q
    duk = transform_at(du, grid, ku)
    v = bg_v.spinor()
    sb = 0.0 + 0.0j
    for sg in (1, -1):
        sb += (np.conj(energy_projector(ku, sg) @ duk) @ ae @ v) / (sg * energy(ku) + energy(q) - k0)
    sb = 1j * np.exp(1j * (energy(q) - k0) * t) * sb
    return np.array([ss, bs, sb])


def bw_march(fld, grid, bg_u, bg_v, photon, t_in, t_out, n_steps, form: int = 1):
    """March (U_scat, V_scat) together with M appended (Eqs. 34-35).

    The appended variable obeys dM/dt = M-dot(t), M(t_out) = 0, so its integral over the march
    is -M(t_in).  form = 1: M-dot is the integrand of Eq. 17 (finite-time terms; the past terms
    are added at t_in).  form = 2: M-dot is the partial-integration integrand of Eqs. 30-33,
    which vanishes outside the field, so -M(t_in) is the whole amplitude.
    Returns (U_scat(t_in), V_scat(t_in), -M(t_in)[3]).
    """
    h0u = h0_field(grid, bg_u.offset())
    h0v = h0_field(grid, bg_v.offset())
    shape = (4,) + grid.n

    def f(t, y):
        return np.stack([rhs(fld, grid, bg_u, h0u, t, y[0]), rhs(fld, grid, bg_v, h0v, t, y[1])])

    if form == 2:
        tabs = PartialIntegrationTables(grid, photon, bg_u, bg_v)

        def g(t, y):
            return bw_integrand_partial(fld, grid, photon, bg_u, bg_v, tabs, t, y[0], y[1])
    else:
        def g(t, y):
            return bw_integrand(grid, photon, bg_u, bg_v, t, y[0], y[1])

    y0 = np.zeros((2,) + shape, dtype=complex)
    y, m = dopri5_march(f, y0, t_out, t_in, n_steps, stage_hook=g)
    return y[0], y[1], -m


def bw_march_adaptive(fld, grid, bg_u, bg_v, photon, t_in, t_out, h0, rtol, atol, max_attempts=100000):
    """bw_march with the step-size-controlled Dormand-Prince march: one step for both waves, the
    error norm the larger of the U and V fields' (the appended integral is left out of it: three
    numbers against 8 n^d), the integrand of Eq. 17 integrated over the accepted steps.
    Returns (U_scat(t_in), V_scat(t_in), M_finite[3], accepted, rejected)."""
    h0u = h0_field(grid, bg_u.offset())
    h0v = h0_field(grid, bg_v.offset())

    def f(t, y):
        return np.stack([rhs(fld, grid, bg_u, h0u, t, y[0]), rhs(fld, grid, bg_v, h0v, t, y[1])])

    def g(t, y):
        return bw_integrand(grid, photon, bg_u, bg_v, t, y[0], y[1])

    y0 = np.zeros((2, 4) + grid.n, dtype=complex)
    y, acc_n, rej_n, m = dopri5_adaptive(f, y0, t_out, t_in, h0, rtol, atol, max_attempts, stage_hook=g,
                                         fields_axis0=True)
    return y[0], y[1], -m, acc_n, rej_n


def bw_past(grid, photon, bg_u, bg_v, psi_u, psi_v, t_in):
    """Analytic t < t_in parts of Eqs. 25-27 with the energy projectors of Eq. 23.

    For t < t_in every grid mode of U_scat, V_scat evolves freely, psi~(t, kappa) =
    sum_sigma P_sigma(kappa) psi~(t_in, kappa) e^{-i sigma E (t - t_in)}, and the time integral
    from -infinity to t_in of e^{i Omega (t - t_in)} is 1/(i Omega).  The photon momentum k must
    be a grid mode (the V mode is the U mode minus k).  Returns (ss, bs, sb).
    """
    k = np.asarray(photon.k, dtype=float)
    k0 = photon.k0()
    ae = photon.alpha_eps()
    Ku = bg_u.offset()
    Kv = bg_v.offset()
    su = transform_on_grid(psi_u, grid)
    sv = transform_on_grid(psi_v, grid)
    KXu, KYu, KZu = grid.modes(Ku)
    KXv, KYv, KZv = grid.modes(Kv)
    # integer mode shift of k along the non-trivial axes
    shift = []
    for a in range(3):
        if grid.n[a] > 1:
            m = k[a] * grid.L[a] / (2.0 * np.pi)
            assert abs(m - round(m)) < 1e-9, "photon momentum must be a grid mode"
            shift.append(int(round(m)))
        else:
            shift.append(0)
    ss = 0.0 + 0.0j
    x0 = [grid.x[a][0] for a in range(3)]
    for idx in np.ndindex(*grid.n):
        jdx = tuple((idx[a] - shift[a]) % grid.n[a] for a in range(3))  # mode kappa - k
        ku = np.array([KXu[idx], KYu[idx], KZu[idx]])
        kv = np.array([KXv[jdx], KYv[jdx], KZv[jdx]])
        eu, ev = energy(ku), energy(kv)
        uu = su[(slice(None),) + idx]
        vv = sv[(slice(None),) + jdx]
        # the grid sum of e^{i(kappa_v + k - kappa_u).x} over N points is N e^{i(kappa_v + k - kappa_u).x0}:
        # 1 unless the V mode wrapped around the grid (then -1 on an odd axis length)
        wrap = np.exp(1j * sum((kv[a] + k[a] - ku[a]) * x0[a] for a in range(3) if grid.n[a] > 1))
        for sg in (+1, -1):
            pu = energy_projector(ku, sg) @ uu
            for sgp in (+1, -1):
                pv = energy_projector(kv, sgp) @ vv
                om = sg * eu - sgp * ev - k0
                ss += wrap * (np.conj(pu) @ ae @ pv) / (1j * om)
    ss = ss * np.exp(-1j * k0 * t_in) / grid.volume
    # back, scat: U_back = u(p) e^{-i p0 t} in mode p, so V_scat is needed at mode p - k
    p = np.asarray(bg_u.p, dtype=float)
    u = bg_u.spinor()
    kv = p - k
    vv = transform_at(psi_v, grid, kv)
    bs = 0.0 + 0.0j
    for sgp in (+1, -1):
        pv = energy_projector(kv, sgp) @ vv
        om = energy(p) - sgp * energy(kv) - k0
        bs += (np.conj(u) @ ae @ pv) / (1j * om)
    bs = bs * np.exp(1j * energy(p) * t_in) * np.exp(-1j * k0 * t_in)
    # scat, back: V_back = v(q) e^{+i q0 t} in mode -q, so U_scat is needed at mode k - q
    q = np.asarray(bg_v.p, dtype=float)
    v = bg_v.spinor()
    ku = k - q
    uu = transform_at(psi_u, grid, ku)
    sb = 0.0 + 0.0j
    for sg in (+1, -1):
        pu = energy_projector(ku, sg) @ uu
        om = sg * energy(ku) + energy(q) - k0
        sb += (np.conj(pu) @ ae @ v) / (1j * om)
    sb = sb * np.exp(1j * energy(q) * t_in) * np.exp(-1j * k0 * t_in)
    return np.array([ss, bs, sb])


def bw_amplitude(fld, grid, p, s, q, r, photon, t_in, t_out, n_steps, form: int = 1, adaptive=None):
    """M = M_ss + M_bs + M_sb (Eq. 13).

    form = 1: each term is the sum of its finite (Eq. 17) and past (Eqs. 25-27) part.
    form = 2: each term is the time integral of the partial-integration integrand (Eqs. 30-33);
    "past" is then zero.
    adaptive = (rtol, atol) (form 1): the step-size-controlled march, first step
    (t_in - t_out)/n_steps; the result then also holds "accepted" and "rejected".
    """
    bg_u = Background("U", tuple(p), s)
    bg_v = Background("V", tuple(q), r)
    if adaptive is not None:
        rtol, atol = adaptive
        psi_u, psi_v, m_fin, acc_n, rej_n = bw_march_adaptive(fld, grid, bg_u, bg_v, photon, t_in, t_out,
                                                              (t_in - t_out) / n_steps, rtol, atol)
        m_past = bw_past(grid, photon, bg_u, bg_v, psi_u, psi_v, t_in)
        return {"finite": m_fin, "past": m_past, "terms": m_fin + m_past, "M": complex(np.sum(m_fin + m_past)),
                "psi_u": psi_u, "psi_v": psi_v, "accepted": acc_n, "rejected": rej_n}
    if form == 2:
        psi_u, psi_v, m = bw_march(fld, grid, bg_u, bg_v, photon, t_in, t_out, n_steps, form=2)
        return {"finite": m, "past": np.zeros(3, dtype=complex), "terms": m, "M": complex(np.sum(m)),
                "psi_u": psi_u, "psi_v": psi_v}
    psi_u, psi_v, m_fin = bw_march(fld, grid, bg_u, bg_v, photon, t_in, t_out, n_steps)
    m_past = bw_past(grid, photon, bg_u, bg_v, psi_u, psi_v, t_in)
    return {"finite": m_fin, "past": m_past, "terms": m_fin + m_past,
            "M": complex(np.sum(m_fin + m_past)), "psi_u": psi_u, "psi_v": psi_v}


def bw_photon_scan(fld, grid, p, s, q, r, photons, t_in, t_out, n_steps):
    """Amplitudes M(k_j, eps_j) for a list of plane-wave photons from one march of U and V.

    The photon enters only the integrals of Eq. 14, not the Dirac equations for U and V (Sec. IV,
    closing paragraphs), so the appended integral carries the finite-time integrands of every
    photon and the past terms (Eqs. 25-27) are added per photon at t_in.
    Returns a list of dicts like bw_amplitude's (without the wave functions).
    """
    bg_u = Background("U", tuple(p), s)
    bg_v = Background("V", tuple(q), r)
    h0u = h0_field(grid, bg_u.offset())
    h0v = h0_field(grid, bg_v.offset())

    def f(t, y):
        return np.stack([rhs(fld, grid, bg_u, h0u, t, y[0]), rhs(fld, grid, bg_v, h0v, t, y[1])])

    def g(t, y):
        return np.concatenate([bw_integrand(grid, ph, bg_u, bg_v, t, y[0], y[1]) for ph in photons])

    y0 = np.zeros((2, 4) + grid.n, dtype=complex)
    y, m = dopri5_march(f, y0, t_out, t_in, n_steps, stage_hook=g)
    out = []
    for j, ph in enumerate(photons):
        fin = -m[3 * j:3 * j + 3]
        past = bw_past(grid, ph, bg_u, bg_v, y[0], y[1], t_in)
        out.append({"finite": fin, "past": past, "terms": fin + past, "M": complex(np.sum(fin + past))})
    return out


def bw_packet_finite(fld, grid, p, s, q, r, photons, weights, t_in, t_out, n_steps):
    """Finite-time terms (Eq. 17) for a photon wave packet: eps_mu e^{-ikx} replaced by the packet
    f(t, x) = sum_j w_j eps_j e^{-i k_j x} (Sec. IV, closing paragraphs), integrated as one
    space-time integral dx^d sum_x U_a^+ (alpha.f) V_b per stage.  Returns (ss, bs, sb)."""
    bg_u = Background("U", tuple(p), s)
    bg_v = Background("V", tuple(q), r)
    h0u = h0_field(grid, bg_u.offset())
    h0v = h0_field(grid, bg_v.offset())
    X, Y, Z = grid.coords()

    def packet(t):
        fv = np.zeros((3,) + grid.n, dtype=complex)
        for ph, w in zip(photons, weights):
            k = np.asarray(ph.k, dtype=float)
            kk = [k[a] if grid.n[a] > 1 else 0.0 for a in range(3)]
            wave = w * np.exp(-1j * ph.k0() * t + 1j * (kk[0] * X + kk[1] * Y + kk[2] * Z))
            for a in range(3):
                fv[a] = fv[a] + ph.eps[a] * wave
        return fv

    def f(t, y):
        return np.stack([rhs(fld, grid, bg_u, h0u, t, y[0]), rhs(fld, grid, bg_v, h0v, t, y[1])])

    def g(t, y):
        fv = packet(t)
        ub = bg_u.values(grid, t)
        vb = bg_v.values(grid, t)

        def term(uu, vv):
            av = sum(np.einsum("ab,b...->a...", ALPHA[a], vv) * fv[a][None] for a in range(3))
            return grid.cell * np.sum(np.conj(uu) * av)

        return np.array([term(y[0], y[1]), term(ub, y[1]), term(y[0], vb)])

    y0 = np.zeros((2, 4) + grid.n, dtype=complex)
    _, m = dopri5_march(f, y0, t_out, t_in, n_steps, stage_hook=g)
    return -m


# --------------------------------------------------------------------------------------------
# Convenience drivers used by tests and by the CPU baseline
# --------------------------------------------------------------------------------------------
@dataclass
class SchwingerResult:
    psi_u: np.ndarray
    spectrum: np.ndarray = dc_field(default=None)


def schwinger_spectrum(fld, grid, p, s, t_in, t_out, n_steps):
    """One electron march and its C-spectrum |C(m, (r, q))|^2 over all grid positrons."""
    bg = Background("U", tuple(p), s)
    psi = march_scattered(fld, grid, bg, t_in, t_out, n_steps)
    C = c_spectrum(psi, grid, t_in, bg.offset())
    return psi, C
