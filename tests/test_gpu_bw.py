"""GPU parity of the Breit-Wheeler amplitude (Sec. IV) against the FP64 oracle."""
import json
import os

import numpy as np
import pytest

from oracle import swf_oracle as O

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Tolerances: complex128 runs the oracle's scheme and steps (only the summation order differs):
# 1e-10 relative on M and on each term (measured: 1e-15 on the small grids, 4e-13 on the full-size
# instance).  complex64: 5e-5 relative on M and the terms, so that |M|^2 is within 1e-4 (measured:
# at most 9e-7 on the small grids, 6e-6 at full size).


def _precs(swf):
    return ((swf.C128, 1e-10), (swf.C64, 5e-5))


def _check_prob(prob, M, tol):
    """|M|^2 within 2 tol relative (1e-4 for complex64, 2e-10 for complex128)."""
    assert abs(prob - abs(M) ** 2) <= 2 * tol * abs(M) ** 2, (prob, abs(M) ** 2)


@pytest.fixture(scope="module")
def env():
    from paper_2512_16889_gb300 import build, swf
    build.build()
    ctx = swf.Context(0)
    yield swf, ctx
    ctx.close()


def _bw_inst(swf, fld_kind, prm, n, L, t_in, t_out, n_steps, p, s, q, r, k, eps, flags=0):
    code = swf.FIELD_CODES[fld_kind]
    return swf.make_instance(code, prm, n, L, t_in, t_out, n_steps, p=p, s=s, q=q, r=r, k=k, eps=eps, flags=flags)


CASE2D = dict(fld=("sauter_gauss", (1.0, 0.7, 2.0)), n=(16, 16, 1), L=(8 * np.pi, 8 * np.pi, 1.0), t_in=-9.0,
              t_out=9.0, n_steps=450, p=(0.25, -1.0, 0.0), q=(-0.25, -1.0, 0.0), k=(0.0, -2.0, 0.0))


def _oracle(c, s, r, form=1):
    fld = O.Field(*c["fld"])
    grid = O.Grid(c["n"], c["L"])
    perp, par = O.polarisation_basis((1, 0, 0), c["k"])
    ph = O.Photon(c["k"], tuple(par))
    return O.bw_amplitude(fld, grid, c["p"], s, c["q"], r, ph, c["t_in"], c["t_out"], c["n_steps"], form=form), par


def _amps(res):
    return [complex(res.amp[2 * j], res.amp[2 * j + 1]) for j in range(4)]


@pytest.mark.parametrize("spins", [(1, 1), (-1, 1)])
def test_bw_partial_integration_form_matches_oracle_2d(env, spins):
    """The partial-integration form (Eqs. 30-33) on the GPU against the oracle's, term by term."""
    swf, ctx = env
    s, r = spins
    ref, par = _oracle(CASE2D, s, r, form=2)
    c = CASE2D
    inst = _bw_inst(swf, *c["fld"], c["n"], c["L"], c["t_in"], c["t_out"], c["n_steps"], c["p"], s, c["q"], r,
                    c["k"], par, flags=swf.BW_PARTIAL)
    M = ref["M"]
    for prec, tol in _precs(swf):
        res, _ = ctx.solve([inst], swf.BREIT_WHEELER, prec)
        got = _amps(res[0])
        assert abs(got[3] - M) <= tol * abs(M), (prec, got[3], M)
        _check_prob(res[0].prob[0], M, tol)
        for j in range(3):
            assert abs(got[j] - ref["terms"][j]) <= tol * max(abs(ref["terms"][j]), abs(M)), (prec, j)


def test_bw_both_forms_in_one_call_agree(env):
    """Instances of both forms in one call are solved in separate groups; on the GPU the two forms
    agree term by term to the time-quadrature gap (Sec. IV: both handle t < t_in exactly)."""
    swf, ctx = env
    c = CASE2D
    perp, par = O.polarisation_basis((1, 0, 0), c["k"])
    insts = [_bw_inst(swf, *c["fld"], c["n"], c["L"], c["t_in"], c["t_out"], c["n_steps"], c["p"], 1, c["q"], 1,
                      c["k"], par, flags=f) for f in (0, swf.BW_PARTIAL, 0)]
    res, _ = ctx.solve(insts, swf.BREIT_WHEELER, swf.C128)
    a1, a2, a3 = _amps(res[0]), _amps(res[1]), _amps(res[2])
    assert a1 == a3
    M = a1[3]
    for j in range(4):
        assert abs(a1[j] - a2[j]) <= 1e-6 * abs(M), (j, a1[j], a2[j])
    single, _ = ctx.solve([insts[1]], swf.BREIT_WHEELER, swf.C128)
    assert _amps(single[0]) == a2


@pytest.mark.parametrize("spins", [(1, 1), (1, -1)])
def test_bw_amplitude_matches_oracle_2d(env, spins):
    swf, ctx = env
    s, r = spins
    ref, par = _oracle(CASE2D, s, r)
    c = CASE2D
    inst = _bw_inst(swf, *c["fld"], c["n"], c["L"], c["t_in"], c["t_out"], c["n_steps"], c["p"], s, c["q"], r,
                    c["k"], par)
    for prec, tol in _precs(swf):
        res, _ = ctx.solve([inst], swf.BREIT_WHEELER, prec)
        got = [complex(res[0].amp[2 * j], res[0].amp[2 * j + 1]) for j in range(4)]
        M = ref["M"]
        assert abs(got[3] - M) <= tol * abs(M), (prec, got[3], M)
        _check_prob(res[0].prob[0], M, tol)
        for j in range(3):  # each of ss, bs, sb (finite + past)
            assert abs(got[j] - ref["terms"][j]) <= tol * max(abs(ref["terms"][j]), abs(M)), (prec, j)


@pytest.mark.parametrize("partial", [False, True])
def test_bw_exact_spin_ratio_1p1d_on_gpu(env, partial):
    """Eq. A81 on the (1+1)D example of Sec. IV, computed by the CUDA path (either integrand form)."""
    swf, ctx = env
    gold = json.load(open(os.path.join(GOLDEN, "bw_spin_ratio_1p1d.json")))
    c = gold["case"]
    n, L = 64, 64.0
    P = 2 * np.pi * 2 / L
    rho = c["p2"]
    k = (0.0, c["k2"], 0.0)
    perp, par = O.polarisation_basis((1, 0, 0), k)
    insts = [_bw_inst(swf, "single_e", (c["E0"], c["omega"], c["kappa_x"], 0.0, 0.0), (n, 1, 1), (L, 1.0, 1.0),
                      -20.0, 20.0, 800, (P, rho, 0.0), rs[0], (-P, rho, 0.0), rs[1], k, par,
                      flags=swf.BW_PARTIAL if partial else 0)
             for rs in ((1, 1), (1, -1), (-1, 1), (-1, -1))]
    res, _ = ctx.solve(insts, swf.BREIT_WHEELER, swf.C128)
    prob = [res[i].prob[0] for i in range(4)]
    assert prob[0] > 1e-12
    assert np.isclose(prob[3], prob[0], rtol=1e-6)
    assert np.isclose(prob[1] / prob[0], gold["expected_ratio"], rtol=1e-5)
    assert np.isclose(prob[2] / prob[0], gold["expected_ratio"], rtol=1e-5)


def test_bw_zero_field_and_validation(env):
    swf, ctx = env
    c = CASE2D
    inst = _bw_inst(swf, "zero", (), c["n"], c["L"], c["t_in"], c["t_out"], 20, c["p"], 1, c["q"], 1, c["k"],
                    (-1.0, 0.0, 0.0))
    res, _ = ctx.solve([inst], swf.BREIT_WHEELER, swf.C64)
    assert res[0].prob[0] == 0.0
    bad = _bw_inst(swf, *c["fld"], c["n"], c["L"], c["t_in"], c["t_out"], 20, c["p"], 1, c["q"], 1,
                   (0.0, -2.05, 0.0), (-1.0, 0.0, 0.0))
    with pytest.raises(swf.SwfError) as ei:
        ctx.solve([bad], swf.BREIT_WHEELER, swf.C64)
    assert ei.value.status == swf.SWF_EINVAL and "grid mode" in str(ei.value)


@pytest.mark.parametrize("partial", [False, True])
def test_bw_graph_replay_matches_plain_launches(partial):
    """The Breit-Wheeler march replayed from CUDA graphs gives the same amplitudes as kernel-by-
    kernel launches (kernel timing on), for an odd step count, in both integrand forms."""
    from paper_2512_16889_gb300 import build, swf
    build.build()
    c = CASE2D
    perp, par = O.polarisation_basis((1, 0, 0), c["k"])
    inst = _bw_inst(swf, *c["fld"], c["n"], c["L"], c["t_in"], c["t_out"], 451, c["p"], 1, c["q"], 1, c["k"], par,
                    flags=swf.BW_PARTIAL if partial else 0)
    res = []
    for timed in (False, True):
        ctx = swf.Context(0)
        ctx.profile_enable(timed)
        r, _ = ctx.solve([inst], swf.BREIT_WHEELER, swf.C64)
        res.append(list(r[0].amp) + list(r[0].prob))
        ctx.close()
    assert res[0] == res[1]


def test_full_size_instance_matches_stored_oracle(env):
    """One instance of the Breit-Wheeler uneven-grid workload at full size (192^2, 2605 steps),
    against oracle values written by tests/golden/make_full_size_reference.py, in complex128 and
    in the workload's complex64."""
    swf, ctx = env
    from paper_2512_16889_gb300 import workloads as W
    golden = json.load(open(os.path.join(GOLDEN, "bw_uneven_sample.json")))
    d = W.bw_uneven()[golden["instance"]]
    M = complex(*golden["M"])
    for prec, tol in _precs(swf):
        res, _ = ctx.solve([swf.from_workload(d)], swf.BREIT_WHEELER, prec)
        got = [complex(res[0].amp[2 * j], res[0].amp[2 * j + 1]) for j in range(4)]
        assert abs(got[3] - M) <= tol * abs(M), (prec, got[3], M)
        _check_prob(res[0].prob[0], M, tol)
        for j in range(3):
            ref = complex(*golden["terms"][j])
            assert abs(got[j] - ref) <= tol * max(abs(ref), abs(M)), (prec, j)
        assert abs(res[0].diag[0] - golden["norm_u"]) <= 10 * tol * golden["norm_u"]


def test_full_size_partial_integration_form_matches_stored_oracle(env):
    """The same full-size instance in the partial-integration form (Eqs. 30-33), against the oracle's
    values of that form (written by tests/golden/make_full_size_reference.py --bw-partial)."""
    swf, ctx = env
    from paper_2512_16889_gb300 import workloads as W
    golden = json.load(open(os.path.join(GOLDEN, "bw_uneven_partial_sample.json")))
    d = W.bw_uneven()[golden["instance"]]
    M = complex(*golden["M"])
    inst = swf.from_workload(d)
    inst.flags = swf.BW_PARTIAL
    for prec, tol in _precs(swf):
        res, _ = ctx.solve([inst], swf.BREIT_WHEELER, prec)
        got = _amps(res[0])
        assert abs(got[3] - M) <= tol * abs(M), (prec, got[3], M)
        _check_prob(res[0].prob[0], M, tol)
        for j in range(3):
            ref = complex(*golden["terms"][j])
            assert abs(got[j] - ref) <= tol * max(abs(ref), abs(M)), (prec, j)


def _scan_photons():
    du = 2 * np.pi / CASE2D["L"][0]
    ks, es = [], []
    for k in ((0.0, -2.0, 0.0), (du, -2.0, 0.0), (-2 * du, -1.75, 0.0)):
        perp, par = O.polarisation_basis((1, 0, 0), k)
        for e in (par, perp):
            ks.append(k)
            es.append(tuple(e))
    return np.array(ks), np.array(es)


def test_bw_photon_scan_matches_oracle(env):
    """Six photons from one march (Sec. IV: the photon enters only the integrals of Eq. 14), and
    their wave-packet sum, against the oracle's photon scan."""
    swf, ctx = env
    c = dict(CASE2D, n_steps=300)
    ks, es = _scan_photons()
    photons = [O.Photon(tuple(k), tuple(e)) for k, e in zip(ks, es)]
    ref = O.bw_photon_scan(O.Field(*c["fld"]), O.Grid(c["n"], c["L"]), c["p"], 1, c["q"], -1, photons,
                           c["t_in"], c["t_out"], c["n_steps"])
    rng = np.random.default_rng(11)
    w = rng.normal(size=len(photons)) + 1j * rng.normal(size=len(photons))
    inst = _bw_inst(swf, *c["fld"], c["n"], c["L"], c["t_in"], c["t_out"], c["n_steps"], c["p"], 1, c["q"], -1,
                    ks[0], es[0])
    pk_ref = sum(wj * np.append(r["terms"], r["M"]) for wj, r in zip(w, ref))
    for prec, tol in _precs(swf):
        amps, packet = ctx.bw_photons(inst, ks, es, prec, weights=w)
        for j, r in enumerate(ref):
            M = r["M"]
            assert abs(amps[j, 3] - M) <= tol * abs(M), (prec, j, amps[j, 3], M)
            for t in range(3):
                assert abs(amps[j, t] - r["terms"][t]) <= tol * max(abs(r["terms"][t]), abs(M)), (prec, j, t)
        scale = np.max(np.abs([r["M"] for r in ref])) * np.sum(np.abs(w))
        assert np.max(np.abs(packet - pk_ref)) <= tol * scale, (prec, packet, pk_ref)


def test_bw_photon_scan_equals_solves_bitwise(env):
    """Each photon of a scan gives the same bits as a solve of that photon alone (shared march,
    the same split of the integrand sums), and invalid scans are refused."""
    swf, ctx = env
    c = dict(CASE2D, n_steps=120)
    ks, es = _scan_photons()
    insts = [_bw_inst(swf, *c["fld"], c["n"], c["L"], c["t_in"], c["t_out"], c["n_steps"], c["p"], 1, c["q"], 1, k, e)
             for k, e in zip(ks, es)]
    amps, packet = ctx.bw_photons(insts[0], ks, es, swf.C64)
    assert packet is None
    res, _ = ctx.solve(insts, swf.BREIT_WHEELER, swf.C64)
    for j in range(len(insts)):
        assert list(amps[j]) == _amps(res[j]), j
    with pytest.raises(swf.SwfError) as ei:
        ctx.bw_photons(insts[0], [(0.0, -2.05, 0.0)], [(1.0, 0.0, 0.0)], swf.C64)
    assert ei.value.status == swf.SWF_EINVAL and "grid mode" in str(ei.value)
    bad = _bw_inst(swf, *c["fld"], c["n"], c["L"], c["t_in"], c["t_out"], c["n_steps"], c["p"], 1, c["q"], 1, ks[0],
                   es[0], flags=swf.BW_PARTIAL)
    with pytest.raises(swf.SwfError) as ei:
        ctx.bw_photons(bad, ks, es, swf.C64)
    assert ei.value.status == swf.SWF_EUNSUPPORTED


EDGE_CASES = {
    # (3+1)D: every axis non-trivial, the photon a grid mode along x and y
    "3d": dict(fld=("sauter_gauss", (0.9, 0.7, 1.5)), n=(8, 6, 6), L=(6.0, 5.0, 5.0), t_in=-4.0, t_out=4.0,
               n_steps=80, p=(0.3, 0.2, -0.1), q=(-0.2, 0.1, 0.3), k=(2 * np.pi / 6.0, 4 * np.pi / 5.0, 0.0)),
    # an odd axis length (15 = 3 x 5): V modes that wrap around the grid carry the sign of the
    # grid origin's phase
    "odd": dict(fld=("sauter_gauss", (1.0, 0.7, 2.0)), n=(15, 12, 1), L=(7.5, 6.0, 1.0), t_in=-6.0, t_out=6.0,
                n_steps=150, p=(0.3, -0.5, 0.0), q=(-0.2, -0.5, 0.0), k=(6 * np.pi / 7.5, -2 * np.pi / 6.0, 0.0)),
}


@pytest.mark.parametrize("case", sorted(EDGE_CASES))
@pytest.mark.parametrize("partial", [False, True])
def test_bw_edge_grids_match_oracle(env, case, partial):
    """Both integrand forms on a (3+1)D grid and on an odd axis length, against the oracle."""
    swf, ctx = env
    c = EDGE_CASES[case]
    perp, par = O.polarisation_basis((0, 0, 1), c["k"])
    ph = O.Photon(c["k"], tuple(par))
    ref = O.bw_amplitude(O.Field(*c["fld"]), O.Grid(c["n"], c["L"]), c["p"], 1, c["q"], -1, ph, c["t_in"],
                         c["t_out"], c["n_steps"], form=2 if partial else 1)
    inst = _bw_inst(swf, *c["fld"], c["n"], c["L"], c["t_in"], c["t_out"], c["n_steps"], c["p"], 1, c["q"], -1,
                    c["k"], par, flags=swf.BW_PARTIAL if partial else 0)
    M = ref["M"]
    for prec, tol in _precs(swf):
        res, _ = ctx.solve([inst], swf.BREIT_WHEELER, prec)
        got = _amps(res[0])
        assert abs(got[3] - M) <= tol * abs(M), (prec, got[3], M)
        _check_prob(res[0].prob[0], M, tol)
        for j in range(3):
            assert abs(got[j] - ref["terms"][j]) <= tol * max(abs(ref["terms"][j]), abs(M)), (prec, j)


def test_bw_step_size_controlled_march_matches_oracle(env):
    """Breit-Wheeler with the paper's step-size control (Sec. II.A, rtol 1e-5, atol 1e-10) and
    the integral appended (Eq. 35): the same accepted and rejected steps and amplitude as the
    oracle's controlled march in complex128; complex64 within its tolerance."""
    swf, ctx = env
    c = CASE2D
    perp, par = O.polarisation_basis((1, 0, 0), c["k"])
    ph = O.Photon(c["k"], tuple(par))
    ref = O.bw_amplitude(O.Field(*c["fld"]), O.Grid(c["n"], c["L"]), c["p"], 1, c["q"], 1, ph, c["t_in"],
                         c["t_out"], 50, adaptive=(1e-5, 1e-10))
    inst = _bw_inst(swf, *c["fld"], c["n"], c["L"], c["t_in"], c["t_out"], 50, c["p"], 1, c["q"], 1, c["k"], par,
                    flags=swf.ADAPTIVE)
    M = ref["M"]
    for prec, tol in _precs(swf):
        res, _ = ctx.solve([inst], swf.BREIT_WHEELER, prec)
        got = _amps(res[0])
        if prec == swf.C128:
            assert ctx.march_stats() == (ref["accepted"], ref["rejected"])
            assert ctx.device_loop_marches() > 0  # decided on the device, one graph launch
        assert abs(got[3] - M) <= tol * abs(M), (prec, got[3], M)
        _check_prob(res[0].prob[0], M, tol)
        for j in range(3):
            assert abs(got[j] - ref["terms"][j]) <= tol * max(abs(ref["terms"][j]), abs(M)), (prec, j)
    bad = _bw_inst(swf, *c["fld"], c["n"], c["L"], c["t_in"], c["t_out"], 50, c["p"], 1, c["q"], 1, c["k"], par,
                   flags=swf.ADAPTIVE | swf.BW_PARTIAL)
    with pytest.raises(swf.SwfError) as ei:
        ctx.solve([bad], swf.BREIT_WHEELER, swf.C64)
    assert ei.value.status == swf.SWF_EUNSUPPORTED


def test_uneven_grids_share_one_multi_grid_march(env):
    """Breit-Wheeler instances on three grids with one time grid (the uneven-grid workload's
    pattern): one launch per pass and one integrand launch per stage for all of them, bitwise the
    amplitudes of marching each grid group alone, in both precisions; one instance against the
    oracle."""
    swf, _ = env
    c = CASE2D
    perp, par = O.polarisation_basis((1, 0, 0), c["k"])
    L = c["L"]
    insts, cases = [], []
    for n in (24, 16, 20):
        for P in (-0.3, 0.25):
            d = dict(n=(n, n, 1), p=(P, -1.0, 0.0), q=(-P, -1.0, 0.0))
            cases.append(d)
            insts.append(_bw_inst(swf, *c["fld"], d["n"], L, c["t_in"], c["t_out"], 150, d["p"], 1, d["q"], 1, c["k"],
                                  par))
    for prec in (swf.C64, swf.C128):
        out = {}
        for multi in (True, False):
            ctx = swf.Context(0)
            ctx.set_multi_grid(2 if multi else 0)
            ctx.profile_enable(True)
            ctx.profile_read()
            res, _ = ctx.solve(insts, swf.BREIT_WHEELER, prec)
            prof, _ = ctx.profile_read()
            ctx.close()
            out[multi] = ([list(r.amp) + list(r.prob) for r in res], prof)
        assert "k_mdot_multi" in out[True][1] and "k_mdot_multi" not in out[False][1]
        assert out[True][0] == out[False][0], prec
    # the second instance of the 16^2 group (not the first group in the call) against the oracle
    d = cases[3]
    ph = O.Photon(c["k"], tuple(par))
    ref = O.bw_amplitude(O.Field(*c["fld"]), O.Grid(d["n"], L), d["p"], 1, d["q"], 1, ph, c["t_in"], c["t_out"], 150)
    M = ref["M"]
    got = complex(out[True][0][3][6], out[True][0][3][7])  # last precision run: complex128
    assert abs(got - M) <= 1e-10 * abs(M), (got, M)


def test_multi_grid_march_on_3d_grids(env):
    """(3+1)D Breit-Wheeler instances on two grids with one time grid (3 y/z passes and the
    integrand per stage: the longest launch sequence of a grouped step pair) give bitwise the
    amplitudes of marching each grid alone, in both precisions."""
    swf, _ = env
    c = EDGE_CASES["3d"]
    perp, par = O.polarisation_basis((0, 0, 1), c["k"])
    insts = []
    for n in ((8, 6, 6), (10, 8, 6)):
        for P in (0.3, -0.2):
            insts.append(_bw_inst(swf, *c["fld"], n, c["L"], c["t_in"], c["t_out"], 40, (P, 0.2, -0.1), 1,
                                  (-0.2, 0.1, 0.3), -1, c["k"], par))
    for prec in (swf.C64, swf.C128):
        out = {}
        for mode in (2, 0):
            ctx = swf.Context(0)
            ctx.set_multi_grid(mode)
            ctx.profile_enable(True)
            ctx.profile_read()
            res, _ = ctx.solve(insts, swf.BREIT_WHEELER, prec)
            prof, _ = ctx.profile_read()
            ctx.close()
            out[mode] = ([list(r.amp) + list(r.prob) for r in res], prof)
        assert "k_mid_multi" in out[2][1] and "k_mdot_multi" in out[2][1]
        assert out[2][0] == out[0][0], prec
        assert np.all(np.isfinite(out[2][0]))
