"""Seeded synthetic workloads (instance tables only; none of the method's arithmetic).

Each function returns a list of plain dicts, one per instance:
    field: (kind_name, params)     grid: n (3 ints), L (3 floats), t_in, t_out, n_steps
    p, s: electron;  q, r: positron;  k, eps: Breit-Wheeler photon;  flags: list of strings
Both the CUDA path and the CPU oracle consume these dicts, each through its own code.

Workloads (shapes follow the paper's runs: 128^2 (x, y) grids with momentum scans, 128^3 in
(3+1)D; the field kinds are the benchmark's analytic pulses):
* ``schwinger_fp64_single``: (2+1)D, A_1 = (E/omega) sech^2(omega t) exp(-(x^2+y^2)/lambda^2),
  E = 0.3, omega = 0.5, lambda = 5, 128^2 grid on a 40 x 40 box, 1000 steps over [-20, 20],
  electron p = (0.2, 0, 0), s = +1.
* ``schwinger_batched``: (2+1)D 256^2 grid, box 40, same window, 64 electron momenta on an
  8 x 8 grid in [-1, 1]^2 times both spins (128 instances), E per instance drawn from
  {0.2, 0.3, 0.4} by numpy default_rng(20251216) in (p_x, p_y, s) row-major order.
* ``bw_uneven``: (2+1)D Breit-Wheeler, A_1 = a0 sin(omega0 (t - y)) exp(-(t-y)^2/tau^2 - x^2/w^2),
  a0 = 1, omega0 = 0.5, tau = 10, w = 8, photon k = (0, -2, 0), 128 pairs p = (P, -1, 0),
  q = (-P, -1, 0), P in linspace(-1.5, 1.5, 128), parallel polarisation, grids n^2 with n drawn
  from {192, 256, 320, 384} by default_rng(7), box 16 pi, t_out = -t_in = 8 pi + 4 tau, h ~ 0.05.
* ``bw_photon_scan``: one pair of ``bw_uneven`` (192^2) with 64 photons k = (2 pi m/L, -2, 0),
  m = -16 .. 15, parallel and perpendicular polarisation each.
* ``schwinger_3d``: (3+1)D 256^3 grid, box 48, E = 0.3, omega = 0.4, lambda = 6, [-25, 25] in
  2000 steps, 16 electrons p = (p_x, 0, 0), p_x in linspace(-1, 1, 16), s = +1.
* ``surrogate_samples``: field parameters and momenta for the surrogate's training set,
  E ~ U[0.15, 0.45], omega ~ U[0.2, 0.8], lambda ~ U[3, 8], p ~ U[-1, 1]^2, s = +-1 (default_rng(4)).
"""
from __future__ import annotations

import math

import numpy as np


def _inst(field, n, L, t_in, t_out, n_steps, p=(0.0, 0.0, 0.0), s=1, q=(0.0, 0.0, 0.0), r=1,
          k=(0.0, 0.0, 0.0), eps=(0.0, 0.0, 0.0), flags=()):
    return {"field": field, "n": tuple(int(v) for v in n), "L": tuple(float(v) for v in L),
            "t_in": float(t_in), "t_out": float(t_out), "n_steps": int(n_steps),
            "p": tuple(float(v) for v in p), "s": int(s), "q": tuple(float(v) for v in q), "r": int(r),
            "k": tuple(float(v) for v in k), "eps": tuple(float(v) for v in eps), "flags": tuple(flags)}


def schwinger_fp64_single(n=128, L=40.0, n_steps=1000, t_window=20.0):
    return [_inst(("sauter_gauss", (0.3, 0.5, 5.0)), (n, n, 1), (L, L, 1.0), -t_window, t_window, n_steps,
                  p=(0.2, 0.0, 0.0), s=1, q=(-0.2, 0.0, 0.0), r=1, flags=("spectrum",))]


def batched_field_strengths(count=128, seed=20251216):
    return np.random.default_rng(seed).choice([0.2, 0.3, 0.4], count)


def schwinger_batched(n=256, L=40.0, n_steps=1000, t_window=20.0, n_p=8, omega=0.5, lam=5.0):
    es = batched_field_strengths(n_p * n_p * 2)
    ps = np.linspace(-1.0, 1.0, n_p)
    out = []
    i = 0
    for px in ps:
        for py in ps:
            for s in (1, -1):
                out.append(_inst(("sauter_gauss", (float(es[i]), omega, lam)), (n, n, 1), (L, L, 1.0),
                                 -t_window, t_window, n_steps, p=(px, py, 0.0), s=s,
                                 q=(-px, -py, 0.0), r=s, flags=("spectrum",)))
                i += 1
    return out


def pair_scan(n=256, L=40.0, n_steps=1000, t_window=20.0, n_p=8, E=0.3, omega=0.5, lam=5.0):
    """A momentum scan in one field (the batched workload's grid and window at E = 0.3):
    electrons (s, p) over an n_p x n_p lattice of grid momenta (every second mode, 2 pi k/L,
    k = -8, -6, .., 6: p in [-1.26, 0.94]) and both spins, and the positrons (r, q = -p) of the
    same lattice, for the all-pairs full pair number (grid momenta, so that both lines of Eq. 8
    agree)."""
    ps = 2 * np.pi / L * 2 * (np.arange(n_p) - n_p // 2)
    base = (("sauter_gauss", (E, omega, lam)), (n, n, 1), (L, L, 1.0), -t_window, t_window, n_steps)
    els, pos = [], []
    for px in ps:
        for py in ps:
            for s in (1, -1):
                els.append(_inst(*base, p=(px, py, 0.0), s=s, q=(0.0, 0.0, 0.0), r=1))
                pos.append(_inst(*base, p=(0.0, 0.0, 0.0), s=1, q=(-px, -py, 0.0), r=s))
    return els, pos


def paper_cross_section(kind="single_e", n_p=100, h=0.1):
    """The (2+1)D momentum cross sections of Sec. V (Eqs. 11-12): E0 = 1/4, omega = E0,
    kappa_x = kappa_y = E0/2 (and Delta x = 1.75/kappa_x for the double field), p_2 = p_3 = q_2 =
    q_3 = 0, spins s = r = +1, and an n_p x n_p grid of (p_1, q_1).  Box and window are readings
    (the text gives neither): a 128 x 64 box at 0.5 spacing (the field's Gaussian is below
    exp(-16) at its edge, also for the double field's peaks at +-14), the window where exp(-(omega
    t)^2) falls below exp(-20), fixed step h.  The momenta are the box's modes p_1 = 2 pi k/128,
    k = -n_p/2 .. n_p/2 - 1 (p_1 in [-2.45, 2.40] for n_p = 100), so that both lines of Eq. 8
    agree on the grid.  Returns (electrons, positrons)."""
    E0 = 0.25
    kx = ky = E0 / 2
    if kind == "single_e":
        field = ("single_e", (E0, E0, kx, ky, 0.0))
    else:
        field = ("double_e", (E0, E0, kx, ky, 0.0, 1.75 / kx))
    Lx, Ly = 128.0, 64.0
    nx, ny = 256, 128
    t_w = 4.0 / E0 + 2.0
    n_steps = int(round(2 * t_w / h))
    ps = 2 * np.pi / Lx * np.arange(-(n_p // 2), n_p - n_p // 2)
    base = (field, (nx, ny, 1), (Lx, Ly, 1.0), -t_w, t_w, n_steps)
    els = [_inst(*base, p=(float(p), 0.0, 0.0), s=1, q=(0.0, 0.0, 0.0), r=1) for p in ps]
    pos = [_inst(*base, p=(0.0, 0.0, 0.0), s=1, q=(float(q), 0.0, 0.0), r=1) for q in ps]
    return els, pos


def bw_uneven(count=128, sizes=(192, 256, 320, 384), seed=7, h=0.05, a0=1.0, omega0=0.5, tau=10.0, w=8.0):
    L = 16.0 * math.pi
    ns = np.random.default_rng(seed).choice(list(sizes), count)
    t_out = L / 2 + 4 * tau
    n_steps = int(round(2 * t_out / h))
    Ps = np.linspace(-1.5, 1.5, count)
    return [_inst(("pulse_gauss", (a0, omega0, tau, w, 0.0)), (int(ns[i]), int(ns[i]), 1), (L, L, 1.0),
                  -t_out, t_out, n_steps, p=(Ps[i], -1.0, 0.0), s=1, q=(-Ps[i], -1.0, 0.0), r=1,
                  k=(0.0, -2.0, 0.0), eps=(-1.0, 0.0, 0.0)) for i in range(count)]


def bw_photon_scan(m_range=16):
    """One pair of the uneven-grid Breit-Wheeler workload (the first on a 192^2 grid) and a list of
    photons k = (2 pi m / L, -2, 0), m = -m_range .. m_range - 1, each with the polarisations
    transverse to k in the plane of k and x (parallel: (-2, -k_x, 0)/|.|) and along -z
    (perpendicular).  Returns (instance, k [n][3], eps [n][3])."""
    ds = bw_uneven()
    d = next(x for x in ds if x["n"][0] == 192)
    ks, es = [], []
    for m in range(-m_range, m_range):
        kx = 2.0 * math.pi * m / d["L"][0]
        k = (kx, -2.0, 0.0)
        nrm = math.sqrt(4.0 + kx * kx)
        for e in ((-2.0 / nrm, -kx / nrm, 0.0), (0.0, 0.0, -1.0)):
            ks.append(k)
            es.append(e)
    return d, ks, es


def schwinger_3d(n=256, L=48.0, n_steps=2000, t_window=25.0, count=16):
    return [_inst(("sauter_gauss", (0.3, 0.4, 6.0)), (n, n, n), (L, L, L), -t_window, t_window, n_steps,
                  p=(px, 0.0, 0.0), s=1, q=(-px, 0.0, 0.0), r=1, flags=("spectrum",))
            for px in np.linspace(-1.0, 1.0, count)]


def surrogate_samples(count, seed=4):
    rng = np.random.default_rng(seed)
    return {"E": rng.uniform(0.15, 0.45, count), "omega": rng.uniform(0.2, 0.8, count),
            "lam": rng.uniform(3.0, 8.0, count), "px": rng.uniform(-1.0, 1.0, count),
            "py": rng.uniform(-1.0, 1.0, count), "s": rng.choice([1, -1], count)}


def small_parity_cases():
    """Reduced grids and windows that the oracle finishes in seconds, spanning several tiles and
    a non-power-of-two length."""
    base = []
    base.append(_inst(("sauter_gauss", (0.8, 0.6, 2.5)), (32, 24, 1), (16.0, 12.0, 1.0), -6.0, 6.0, 120,
                      p=(0.3, -0.2, 0.0), s=1, q=(-0.25, 0.1, 0.0), r=-1, flags=("spectrum",)))
    base.append(_inst(("sauter_gauss", (0.5, 0.5, 3.0)), (40, 30, 1), (20.0, 15.0, 1.0), -7.0, 7.0, 140,
                      p=(-0.4, 0.5, 0.0), s=-1, q=(0.3, -0.6, 0.0), r=1, flags=("spectrum",)))
    base.append(_inst(("single_e", (0.6, 0.5, 0.3, 0.3, 0.0)), (36, 20, 1), (24.0, 14.0, 1.0), -5.0, 5.0, 100,
                      p=(0.1, 0.2, 0.0), s=1, q=(-0.1, 0.2, 0.0), r=1, flags=("spectrum",)))
    return base
