"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (from the arithmetic of the two paths):
* complex128 path: same scheme and steps as the oracle, only the summation order differs ->
  1e-10 relative (state: max|diff| / max|ref|; scalars: |diff| / |ref|).
* complex64 march: single-precision rounding accumulated over the march -> 1e-4 relative on
  |C|^2 for entries at or above 1e-2 of the spectrum maximum (below, an absolute noise floor of
  the single-precision march), 2e-5 relative on the state.
"""
import numpy as np
import pytest

from oracle import swf_oracle as O
from paper_2512_16889_gb300 import workloads as W
from tests import oracle_adapter as OA

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2512_16889_gb300 import build, swf
    build.build()
    ctx = swf.Context(0)
    yield torch, swf, ctx
    ctx.close()


def to_complex(t):
    a = t.cpu().numpy()
    return a.view(np.complex128) if a.dtype == np.float64 else a.view(np.complex64).astype(np.complex128)


def rel_state(got, ref):
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


RHS_CASES = [
    dict(field=("sauter_gauss", (0.8, 0.6, 2.5)), n=(32, 24, 1), L=(16.0, 12.0, 1.0), p=(0.3, -0.2, 0.0), s=1),
    dict(field=("single_e", (0.6, 0.5, 0.3, 0.3, 0.0)), n=(36, 20, 1), L=(24.0, 14.0, 1.0), p=(0.1, 0.2, 0.0), s=-1),
    dict(field=("double_e", (0.5, 0.4, 0.3, 0.2, 0.0, 3.0)), n=(40, 30, 1), L=(30.0, 20.0, 1.0), p=(-0.3, 0.2, 0.0), s=1),
    dict(field=("pulse_gauss", (1.0, 0.5, 4.0, 3.0, 0.0)), n=(48, 20, 1), L=(20.0, 18.0, 1.0), p=(0.4, -1.0, 0.0), s=1),
    dict(field=("sauter_gauss", (0.7, 0.5, 2.0)), n=(12, 10, 8), L=(8.0, 7.0, 6.0), p=(0.2, 0.1, -0.3), s=-1),
    dict(field=("single_e", (0.4, 0.5, 0.25, 0.0, 0.0)), n=(64, 1, 1), L=(30.0, 1.0, 1.0), p=(0.3, 0.6, 0.0), s=1),
]


def _full(d):
    base = dict(t_in=-4.0, t_out=4.0, n_steps=10, q=(-0.2, 0.1, 0.0), r=1, k=(0, 0, 0), eps=(0, 0, 0), flags=())
    base.update(d)
    return base


@pytest.mark.parametrize("case", range(len(RHS_CASES)))
@pytest.mark.parametrize("bg", [0, 1])
def test_rhs_matches_oracle(env, case, bg):
    torch, swf, ctx = env
    d = _full(RHS_CASES[case])
    rng = np.random.default_rng(10 + case)
    grid = OA.grid(d)
    psi = rng.normal(size=(4,) + grid.n) + 1j * rng.normal(size=(4,) + grid.n)
    t = 0.37
    ref = O.rhs(OA.field(d), grid, OA.background(d, bg), O.h0_field(grid, OA.background(d, bg).offset()), t, psi)
    ref_g = OA.to_gpu_layout(ref)
    inst = swf.from_workload(d)
    for prec, tol in ((swf.C128, 1e-12), (swf.C64, 2e-6)):
        dt = np.complex128 if prec == swf.C128 else np.complex64
        src = OA.to_gpu_layout(psi).astype(dt)
        x = torch.from_numpy(src.view(np.float64 if prec == swf.C128 else np.float32).copy()).cuda()
        out = torch.zeros_like(x)
        ctx.rhs_dev(inst, t, x, out, bg=bg, prec=prec)
        torch.cuda.synchronize()
        got = to_complex(out).reshape(ref_g.shape)
        assert rel_state(got, ref_g) < tol, (prec, rel_state(got, ref_g))


@pytest.mark.parametrize("case", range(3))
def test_march_matches_oracle(env, case):
    torch, swf, ctx = env
    d = W.small_parity_cases()[case]
    grid = OA.grid(d)
    for bg in (0, 1):
        ref = O.march_scattered(OA.field(d), grid, OA.background(d, bg), d["t_in"], d["t_out"], d["n_steps"])
        ref_g = OA.to_gpu_layout(ref)
        for prec, tol in ((swf.C128, 1e-10), (swf.C64, 2e-5)):
            elems = 2 * 4 * int(np.prod(d["n"]))
            out = torch.zeros(elems, dtype=torch.float64 if prec == swf.C128 else torch.float32, device="cuda")
            ctx.march_dev([swf.from_workload(d)], out, bg=bg, prec=prec)
            got = to_complex(out).reshape(ref_g.shape)
            assert rel_state(got, ref_g) < tol, (bg, prec, rel_state(got, ref_g))


def test_march_batch_of_distinct_fields(env):
    """A batch of instances with different field strengths and momenta marches each one alone."""
    torch, swf, ctx = env
    ds = W.schwinger_batched(n=24, L=12.0, n_steps=30, t_window=3.0, n_p=2)
    N = int(np.prod(ds[0]["n"]))
    out = torch.zeros(len(ds) * 8 * N, dtype=torch.float64, device="cuda")
    ctx.march_dev([swf.from_workload(d) for d in ds], out, bg=0, prec=swf.C128)
    got = to_complex(out).reshape(len(ds), 4, 1, 24, 24)
    for i, d in enumerate(ds):
        ref = OA.to_gpu_layout(O.march_scattered(OA.field(d), OA.grid(d), OA.background(d, 0),
                                                 d["t_in"], d["t_out"], d["n_steps"]))
        assert rel_state(got[i], ref) < 1e-10, i


def test_spectrum_matches_oracle(env):
    torch, swf, ctx = env
    d = W.small_parity_cases()[1]
    grid = OA.grid(d)
    rng = np.random.default_rng(5)
    psi = rng.normal(size=(4,) + grid.n) + 1j * rng.normal(size=(4,) + grid.n)
    ref = O.c_spectrum(psi, grid, d["t_in"])
    x = torch.from_numpy(OA.to_gpu_layout(psi).view(np.float64).copy()).cuda()
    N = int(np.prod(d["n"]))
    c_out = torch.zeros(2 * 2 * N, dtype=torch.float64, device="cuda")
    p_out = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    ctx.spectrum_dev([swf.from_workload(d)], x, c_out, p_out, prec=swf.C128)
    got = to_complex(c_out).reshape(2, d["n"][2], d["n"][1], d["n"][0])
    ref_g = np.transpose(ref, (0, 3, 2, 1))
    assert rel_state(got, ref_g) < 1e-12
    assert np.allclose(p_out.cpu().numpy(), (np.abs(ref_g) ** 2).ravel(), rtol=1e-11, atol=0)


def test_solve_full_pair_number_matches_oracle(env):
    torch, swf, ctx = env
    ds = [dict(d, flags=("spectrum", "full_n")) for d in W.small_parity_cases()[:2]]
    res, spec = ctx.solve([swf.from_workload(d) for d in ds], swf.SCHWINGER, swf.C128)
    off = 0
    for i, d in enumerate(ds):
        grid = OA.grid(d)
        bu, bv = OA.background(d, 0), OA.background(d, 1)
        pu = O.march_scattered(OA.field(d), grid, bu, d["t_in"], d["t_out"], d["n_steps"])
        pv = O.march_scattered(OA.field(d), grid, bv, d["t_in"], d["t_out"], d["n_steps"])
        ref = O.pair_number(pu, pv, grid, d["t_in"], d["p"], d["s"], d["q"], d["r"], bu.offset(), bv.offset())
        r = res[i]
        for j, key in enumerate(("C", "D", "A", "B")):
            got = complex(r.amp[2 * j], r.amp[2 * j + 1])
            assert abs(got - ref[key]) <= 1e-10 * max(abs(ref[key]), abs(ref["C"] + ref["D"])), (key, got, ref[key])
        assert abs(r.prob[0] - ref["N_line2"]) <= 1e-10 * ref["N_line2"]
        assert abs(r.prob[1] - ref["N_line1"]) <= 1e-10 * ref["N_line1"]
        assert abs(r.diag[0] - O.inner(pu, pu, grid).real) <= 1e-10 * r.diag[0]
        n = int(np.prod(d["n"]))
        C = O.c_spectrum(pu, grid, d["t_in"])
        ref_spec = np.transpose(np.abs(C) ** 2, (0, 3, 2, 1)).ravel()
        assert np.max(np.abs(spec[off:off + 2 * n] - ref_spec)) <= 1e-10 * np.max(ref_spec)
        off += 2 * n


def binned_rel_errors(got, ref):
    """Max relative error of |C|^2 per decade of |C|^2 / max|C|^2 (key: decade exponent)."""
    rel = np.abs(got - ref) / np.maximum(ref, 1e-300)
    dec = np.floor(np.log10(np.maximum(ref / ref.max(), 1e-300)))
    return {int(d): float(rel[dec == d].max()) for d in np.unique(dec) if d > -12}


def test_c64_spectrum_within_tolerance(env):
    torch, swf, ctx = env
    d = W.small_parity_cases()[0]
    grid = OA.grid(d)
    res, spec = ctx.solve([swf.from_workload(d)], swf.SCHWINGER, swf.C64)
    pu = O.march_scattered(OA.field(d), grid, OA.background(d, 0), d["t_in"], d["t_out"], d["n_steps"])
    ref = np.transpose(np.abs(O.c_spectrum(pu, grid, d["t_in"])) ** 2, (0, 3, 2, 1)).ravel()
    bins = binned_rel_errors(spec, ref)
    print("c64 |C|^2 max rel error per decade below the maximum:", bins)
    # 1e-4 relative holds for |C|^2 >= 1e-2 of the spectrum maximum (below it, the absolute floor)
    assert max(v for k, v in bins.items() if k >= -2) < 1e-4, bins
    # below the floor the error is an absolute single-precision noise floor of the whole wave
    assert np.max(np.abs(spec - ref)) < 5e-6 * ref.max()


def test_zero_field_is_exactly_zero(env):
    torch, swf, ctx = env
    d = dict(W.small_parity_cases()[0], field=("zero", ()))
    for prec in (swf.C128, swf.C64):
        res, spec = ctx.solve([swf.from_workload(d)], swf.SCHWINGER, prec)
        assert res[0].prob[0] == 0.0 and res[0].diag[0] == 0.0
        assert np.all(spec == 0.0)


def test_uneven_grids_in_one_call(env):
    """Instances with different grids are grouped; each result matches its own solo solve."""
    torch, swf, ctx = env
    cases = W.small_parity_cases()
    insts = [swf.from_workload(d) for d in cases]
    res_all, spec_all = ctx.solve(insts, swf.SCHWINGER, swf.C128)
    off = 0
    for i, inst in enumerate(insts):
        res1, spec1 = ctx.solve([inst], swf.SCHWINGER, swf.C128)
        n = 2 * int(np.prod(cases[i]["n"]))
        assert res_all[i].prob[0] == res1[0].prob[0]
        assert np.array_equal(spec_all[off:off + n], spec1)
        off += n


def test_validation_errors_are_reported(env):
    torch, swf, ctx = env
    d = W.small_parity_cases()[0]
    bad = [dict(d, n=(7, 24, 1)), dict(d, n_steps=0), dict(d, t_in=5.0, t_out=-5.0), dict(d, s=0),
           dict(d, n=(1024, 8, 1)), dict(d, L=(0.0, 12.0, 1.0))]
    for b in bad:
        with pytest.raises(swf.SwfError) as ei:
            ctx.solve([swf.from_workload(b)], swf.SCHWINGER, swf.C64)
        assert ei.value.status == swf.SWF_EINVAL
    # empty input is a no-op
    res, spec = ctx.solve([], swf.SCHWINGER, swf.C64)
    assert len(res) == 0
    # device buffers too short, of the wrong dtype or not contiguous are refused before any launch
    inst = [swf.from_workload(d)]
    N = int(np.prod(d["n"]))
    with pytest.raises(ValueError, match="needed"):
        ctx.march_dev(inst, torch.zeros(8 * N - 1, dtype=torch.float32, device="cuda"), prec=swf.C64)
    with pytest.raises(ValueError, match="dtype"):
        ctx.march_dev(inst, torch.zeros(8 * N, dtype=torch.float32, device="cuda"), prec=swf.C128)
    with pytest.raises(ValueError, match="contiguous"):
        ctx.march_dev(inst, torch.zeros(16 * N, dtype=torch.float32, device="cuda")[::2], prec=swf.C64)
    with pytest.raises(ValueError, match="needed"):
        ctx.spectrum_dev(inst, torch.zeros(8 * N, dtype=torch.float64, device="cuda"),
                         torch.zeros(4 * N - 2, dtype=torch.float64, device="cuda"), prec=swf.C128)


def test_workspace_limit_gives_enomem(env):
    torch, swf, ctx = env
    other = swf.Context(0)
    other.set_workspace_limit(1024)
    with pytest.raises(swf.SwfError) as ei:
        other.solve([swf.from_workload(W.small_parity_cases()[0])], swf.SCHWINGER, swf.C64)
    assert ei.value.status == swf.SWF_ENOMEM
    other.close()


# ---------------------------------------------------------------- fused cluster kernel (256^2, c64)
def _fused_cases(n_steps=16):
    ds = W.schwinger_batched(n=256, L=40.0, n_steps=n_steps, t_window=0.5, n_p=2)
    # a field of the paper (A_0, Eq. 11) and an alpha^y-free pulse keep both sector couplings in play
    ds.append(dict(ds[0], field=("single_e", (0.6, 0.5, 0.3, 0.3, 0.0)), p=(0.3, -0.4, 0.0), s=-1))
    ds.append(dict(ds[1], field=("pulse_gauss", (1.0, 0.5, 4.0, 6.0, 0.0)), p=(-0.2, 0.7, 0.0), s=1))
    return ds


def test_fused_march_matches_oracle(env):
    torch, swf, ctx = env
    ds = _fused_cases()
    N = 256 * 256
    out = torch.zeros(len(ds) * 8 * N, dtype=torch.float32, device="cuda")
    ctx.profile_enable(True)
    ctx.profile_read()
    ctx.march_dev([swf.from_workload(d) for d in ds], out, bg=0, prec=swf.C64)
    prof, _ = ctx.profile_read()
    ctx.profile_enable(False)
    assert any(k.startswith("k_fused") for k in prof), prof  # the cluster kernel ran, not the pass kernels
    got = to_complex(out).reshape(len(ds), 4, 1, 256, 256)
    for i in (0, 3, 4, 5):
        d = ds[i]
        ref = OA.to_gpu_layout(O.march_scattered(OA.field(d), OA.grid(d), OA.background(d, 0),
                                                 d["t_in"], d["t_out"], d["n_steps"]))
        assert rel_state(got[i], ref) < 2e-5, (i, rel_state(got[i], ref))


def test_fused_matches_pass_kernels_and_positron_waves(env):
    torch, swf, ctx = env
    ds = _fused_cases(n_steps=30)
    insts = [swf.from_workload(d) for d in ds]
    N = 256 * 256
    for bg in (0, 1):
        a = torch.zeros(len(ds) * 8 * N, dtype=torch.float32, device="cuda")
        b = torch.zeros_like(a)
        ctx.march_dev(insts, a, bg=bg, prec=swf.C64)
        ctx.set_march_path(1)
        try:
            ctx.march_dev(insts, b, bg=bg, prec=swf.C64)
        finally:
            ctx.set_march_path(0)
        ga, gb = to_complex(a).reshape(len(ds), -1), to_complex(b).reshape(len(ds), -1)
        for i in range(len(ds)):
            assert rel_state(ga[i], gb[i]) < 1e-5, (bg, i, rel_state(ga[i], gb[i]))


def test_pushed_transposes_match_pulled_transposes(env):
    """The fused kernel whose transposes the bulk-copy engine pushes while the threads compute
    (path 5) does the arithmetic of the kernel whose threads pull them (path 4) in the same order:
    equal states after 30 steps for 6 fields (12 sectors, so that clusters march more than one),
    and the pushed variant against the oracle."""
    torch, swf, _ = env
    ds = _fused_cases(n_steps=30)
    insts = [swf.from_workload(d) for d in ds]
    N = 256 * 256
    outs = {}
    for path, name in ((4, "k_fused"), (5, "k_fused3")):
        ctx = swf.Context(0)
        ctx.set_dedupe(False)
        ctx.set_march_path(path)
        out = torch.zeros(len(ds) * 8 * N, dtype=torch.float32, device="cuda")
        ctx.profile_enable(True)
        ctx.profile_read()
        ctx.march_dev(insts, out, bg=0, prec=swf.C64)
        prof, _ = ctx.profile_read()
        ctx.close()
        assert name in prof, (path, prof)
        outs[path] = out.cpu().numpy()
    assert np.all(np.isfinite(outs[5]))
    diff = np.abs(outs[5] - outs[4]).max() / np.abs(outs[4]).max()
    print("pushed vs pulled transposes: bitwise equal" if np.array_equal(outs[4], outs[5]) else f"max diff {diff:.3g}")
    assert diff <= 1e-6, diff
    got = to_complex(torch.from_numpy(outs[5])).reshape(len(ds), 4, 1, 256, 256)
    for i in (0, 4, 5):
        d = ds[i]
        ref = OA.to_gpu_layout(O.march_scattered(OA.field(d), OA.grid(d), OA.background(d, 0),
                                                 d["t_in"], d["t_out"], d["n_steps"]))
        assert rel_state(got[i], ref) < 2e-5, (i, rel_state(got[i], ref))


def test_fused_receive_waits_are_bounded(env):
    """The pushed-transpose fused kernel's receive waits end by themselves.  With its copies
    switched off (swf_set_fused_drop), every CTA's first receive wait runs out after about half
    a second.  The kernel still ends, reports status 1 and writes NaN for every sector.  The same
    context marches normally again afterwards, with status 0."""
    import time
    torch, swf, _ = env
    ds = _fused_cases(n_steps=2)[:4]
    insts = [swf.from_workload(d) for d in ds]
    N = 256 * 256
    ctx = swf.Context(0)
    try:
        ctx.set_dedupe(False)
        ctx.set_march_path(5)
        out = torch.zeros(len(ds) * 8 * N, dtype=torch.float32, device="cuda")
        ctx.set_fused_drop(True)
        t0 = time.perf_counter()
        ctx.march_dev(insts, out, bg=0, prec=swf.C64)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        assert ctx.fused_status() == 1
        assert torch.isnan(out).all().item(), "every sector of a march whose waits ran out is NaN"
        assert dt < 60.0, dt
        ctx.set_fused_drop(False)
        out.zero_()
        ctx.march_dev(insts, out, bg=0, prec=swf.C64)
        torch.cuda.synchronize()
        assert ctx.fused_status() == 0
        assert torch.isfinite(out).all().item()
    finally:
        ctx.close()


def test_split_march_is_fused_plus_pass_kernels(env):
    """A large fused march gives its last fields to the pass kernels, run concurrently on the SMs
    the 16-CTA clusters leave free: the result is bit for bit the fused-only march on the first
    fields and the pass-kernel march on the rest."""
    torch, swf, _ = env
    base = _fused_cases(n_steps=12)[0]
    ds = [dict(base, p=(0.05 * (i % 8) - 0.2, 0.04 * (i // 8) - 0.1, 0.0), s=1 if i % 3 else -1) for i in range(32)]
    insts = [swf.from_workload(d) for d in ds]
    N = 256 * 256
    outs, fused = {}, {}
    for path in (0, 1, 2):
        ctx = swf.Context(0)
        ctx.set_dedupe(False)
        ctx.set_march_path(path)
        out = torch.zeros(len(ds) * 8 * N, dtype=torch.float32, device="cuda")
        f0 = ctx.fields_fused()
        ctx.march_dev(insts, out, bg=0, prec=swf.C64)
        torch.cuda.synchronize()
        fused[path] = ctx.fields_fused() - f0
        outs[path] = out.cpu().numpy().reshape(len(ds), -1)
        ctx.close()
    n1 = fused[0]
    assert fused[2] == len(ds) and fused[1] == 0 and 0 < n1 < len(ds), fused
    assert np.array_equal(outs[0][:n1], outs[2][:n1])
    assert np.array_equal(outs[0][n1:], outs[1][n1:])
    assert np.max(np.abs(outs[0][n1:])) > 0


def test_full_size_workload_matches_stored_oracle_samples(env):
    """The benchmark's own solve (128 instances, 256^2, 1000 steps, complex64, fused kernel)
    against FP64 oracle values stored by tests/golden/make_full_size_reference.py."""
    import json
    import os
    torch, swf, ctx = env
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "schwinger_batched_samples.json")))
    ds = W.schwinger_batched()
    res, spec = ctx.solve([swf.from_workload(d) for d in ds], swf.SCHWINGER, swf.C64)
    n = 2 * 256 * 256
    for smp in gold["samples"]:
        i = smp["instance"]
        got = spec[i * n:(i + 1) * n][np.array(smp["modes"])]
        ref = np.array(smp["prob"])
        big = ref >= 1e-2 * smp["max_prob"]
        assert big.sum() >= 16
        rel = np.abs(got[big] - ref[big]) / ref[big]
        assert rel.max() < 1e-4, (i, rel.max())
        absrel = np.max(np.abs(got - ref)) / smp["max_prob"]
        assert absrel < 2e-5, (i, absrel)
        assert abs(res[i].diag[0] - smp["norm"]) < 1e-5 * smp["norm"]


@pytest.mark.parametrize("inst", [0, 77])
def test_full_size_spectrum_by_decade_against_the_oracle(env, inst):
    """Whole C-spectra of two instances of the batched workload at full size (256^2, 1000 steps)
    against the oracle's (every entry at or above 1e-24 of the maximum, stored by
    tests/golden/make_full_size_reference.py --spectrum), decade by decade.  What the accuracy
    counts of the benchmark line rest on:
    * complex128 (the plain FP64 march): 1e-10 relative on every entry >= 1e-7 of the maximum
      and 1e-4 on every entry >= 1e-19 of it (measured: 5e-11 and 6e-5 at those floors); below,
      FP64 rounding of the march sets the error (the probabilities fall far below the state's
      rounding level);
    * complex64 on the fused kernel and on the pass kernels: 1e-4 relative on every entry
      >= 1e-2 of the maximum (measured: at most 8e-5); the benchmark line reports, decade by
      decade, how many entries below that still meet 1e-4.
    Entries the oracle puts below 1e-24 of the maximum stay below 1e-7 of it on the GPU."""
    import json
    import os
    torch, swf, _ = env
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", f"schwinger_batched_spectrum_{inst}.json")))
    modes, ref, mx = np.array(g["modes"]), np.array(g["prob"]), g["max_prob"]
    d = W.schwinger_batched()[inst]
    rows = {}
    for prec, path, name in ((swf.C128, 0, "c128"), (swf.C64, 0, "c64 fused"), (swf.C64, 1, "c64 pass")):
        ctx = swf.Context(0)
        ctx.set_march_path(path)
        res, spec = ctx.solve([swf.from_workload(d)], swf.SCHWINGER, prec)
        ctx.close()
        rel = np.abs(spec[modes] - ref) / ref
        rest = np.ones(spec.size, bool)
        rest[modes] = False
        assert spec[rest].max() <= 1e-7 * mx, (name, spec[rest].max() / mx)
        if prec == swf.C128:
            assert rel[ref >= 1e-7 * mx].max() <= 1e-10, rel[ref >= 1e-7 * mx].max()
            assert rel[ref >= 1e-19 * mx].max() <= 1e-4, rel[ref >= 1e-19 * mx].max()
            assert abs(res[0].diag[0] - g["norm"]) <= 1e-10 * g["norm"]
        else:
            assert rel[ref >= 1e-2 * mx].max() <= 1e-4, (name, rel[ref >= 1e-2 * mx].max())
            assert abs(res[0].diag[0] - g["norm"]) <= 1e-5 * g["norm"]
        dec = np.floor(np.log10(ref / mx))
        rows[name] = {int(k): round(float(np.mean(rel[dec == k] <= 1e-4)), 3) for k in range(0, -25, -4)}
    print("fraction within 1e-4 per decade below the maximum:", rows)


def test_tuned_launch_shapes_give_bitwise_identical_marches(env):
    """The pass kernels' launch shapes (chosen by timing, or by the fixed rule) decide only which
    lines a block transforms: marches agree bit for bit (x-only, 2D, 3D; both precisions)."""
    torch, swf, _ = env
    cases = [W.small_parity_cases()[i] for i in (0, 1)] + [dict(_full(RHS_CASES[i]), flags=()) for i in (4, 5)]
    for d in cases:
        for prec in (swf.C128, swf.C64):
            outs = []
            for tuned in (False, True):
                ctx = swf.Context(0)
                ctx.set_march_path(1)
                ctx.set_autotune(tuned)
                out = torch.zeros(2 * 4 * int(np.prod(d["n"])), device="cuda",
                                  dtype=torch.float64 if prec == swf.C128 else torch.float32)
                ctx.march_dev([swf.from_workload(d)], out, bg=0, prec=prec)
                ctx.march_dev([swf.from_workload(d)], out, bg=0, prec=prec)  # second call: cached shapes
                outs.append(out.cpu().numpy())
                ctx.close()
            assert np.array_equal(outs[0], outs[1]), (d["n"], prec)


def _pair_scan(n=(24, 20, 1), L=(12.0, 10.0, 1.0)):
    """Three electrons and two positrons in one field: off-grid momenta and both spins."""
    base = dict(field=("sauter_gauss", (0.8, 0.6, 2.5)), n=n, L=L, t_in=-5.0, t_out=5.0, n_steps=60,
                k=(0, 0, 0), eps=(0, 0, 0), flags=())
    els = [dict(base, p=p, s=s, q=(0.0, 0.0, 0.0), r=1) for p, s in
           (((0.3, -0.2, 0.0), 1), ((-0.45, 0.1, 0.0), -1), ((0.05, 0.35, 0.0), 1))]
    pos = [dict(base, p=(0.0, 0.0, 0.0), s=1, q=q, r=r) for q, r in (((-0.25, 0.15, 0.0), -1), ((0.4, -0.3, 0.0), 1))]
    return els, pos


def test_pair_matrix_matches_oracle_and_pair_path(env):
    """swf_pair_matrix (n_e + n_p marches, overlaps as FP64 matrix products) against the oracle's
    Eq. 8 per pair (complex128), and against the one-pair-per-instance path (both precisions)."""
    torch, swf, ctx = env
    els, pos = _pair_scan()
    grid = OA.grid(els[0])
    mat = ctx.pair_matrix([swf.from_workload(d) for d in els], [swf.from_workload(d) for d in pos], swf.C128)
    for m, de in enumerate(els):
        bu = OA.background(de, 0)
        pu = O.march_scattered(OA.field(de), grid, bu, de["t_in"], de["t_out"], de["n_steps"])
        for n, dp in enumerate(pos):
            pair = dict(de, q=dp["q"], r=dp["r"])
            bv = OA.background(pair, 1)
            pv = O.march_scattered(OA.field(pair), grid, bv, de["t_in"], de["t_out"], de["n_steps"])
            ref = O.pair_number(pu, pv, grid, de["t_in"], de["p"], de["s"], dp["q"], dp["r"], bu.offset(), bv.offset())
            r = mat[m][n]
            for j, key in enumerate(("C", "D", "A", "B")):
                got = complex(r.amp[2 * j], r.amp[2 * j + 1])
                assert abs(got - ref[key]) <= 1e-10 * max(abs(ref[key]), abs(ref["C"] + ref["D"])), (m, n, key, got, ref[key])
            assert abs(r.prob[0] - ref["N_line2"]) <= 1e-10 * ref["N_line2"]
            assert abs(r.prob[1] - ref["N_line1"]) <= 1e-10 * ref["N_line1"]
    # the same pairs through solve_swf with SWF_WANT_FULL_N: same marches, other summation order
    for prec, tol in ((swf.C128, 1e-11), (swf.C64, 1e-6)):
        mat = ctx.pair_matrix([swf.from_workload(d) for d in els], [swf.from_workload(d) for d in pos], prec)
        pairs = [dict(de, q=dp["q"], r=dp["r"], flags=("full_n",)) for de in els for dp in pos]
        res, _ = ctx.solve([swf.from_workload(d) for d in pairs], swf.SCHWINGER, prec)
        for i, d in enumerate(pairs):
            r, ref = mat[i // len(pos)][i % len(pos)], res[i]
            for k in range(8):
                assert abs(r.amp[k] - ref.amp[k]) <= tol * max(abs(x) for x in ref.amp), (prec, i, k)
            assert abs(r.diag[0] - ref.diag[0]) <= tol * ref.diag[0]
            assert abs(r.diag[1] - ref.diag[1]) <= tol * ref.diag[1]


def test_pair_matrix_validation(env):
    torch, swf, ctx = env
    els, pos = _pair_scan()
    bad = [dict(pos[0], field=("sauter_gauss", (0.7, 0.6, 2.5)))]
    with pytest.raises(swf.SwfError, match="share the field"):
        ctx.pair_matrix([swf.from_workload(d) for d in els], [swf.from_workload(d) for d in bad], swf.C128)
    with pytest.raises(swf.SwfError):
        ctx.pair_matrix([], [swf.from_workload(d) for d in pos], swf.C128)


@pytest.mark.parametrize("n", [(24, 20, 1), (256, 256, 1)])
def test_spin_pairs_are_marched_once_with_identical_results(env, n):
    """Within one call the other spin's march (components {1, 2} negated source) and exact
    repeats are taken from one march; the states agree with marching every field (pass kernels
    at 24 x 20, the fused cluster kernel at 256 x 256)."""
    torch, swf, _ = env
    L = (12.0, 10.0, 1.0) if n[0] == 24 else (40.0, 40.0, 1.0)
    base = dict(field=("sauter_gauss", (0.8, 0.6, 2.5)), n=n, L=L, t_in=-2.0, t_out=2.0, n_steps=8,
                q=(-0.2, 0.1, 0.0), r=1, k=(0, 0, 0), eps=(0, 0, 0), flags=())
    ds = [dict(base, p=(0.3, -0.2, 0.0), s=1), dict(base, p=(0.3, -0.2, 0.0), s=-1),
          dict(base, p=(-0.1, 0.4, 0.0), s=-1), dict(base, p=(0.3, -0.2, 0.0), s=1)]
    precs = (swf.C128, swf.C64) if n[0] == 24 else (swf.C64,)
    for prec in precs:
        outs, marched = [], []
        for dedupe in (False, True):
            ctx = swf.Context(0)
            ctx.set_dedupe(dedupe)
            out = torch.zeros(len(ds) * 8 * int(np.prod(n)), device="cuda",
                              dtype=torch.float64 if prec == swf.C128 else torch.float32)
            before = ctx.fields_marched()
            ctx.march_dev([swf.from_workload(d) for d in ds], out, bg=0, prec=prec)
            marched.append(ctx.fields_marched() - before)
            outs.append(out.cpu().numpy())
            ctx.close()
        assert marched == [4, 2], marched
        assert np.array_equal(outs[0], outs[1]), prec
        assert np.max(np.abs(outs[1])) > 0


def test_graph_replayed_march_matches_plain_launches(env):
    """Pass-kernel marches replay pairs of steps from a CUDA graph with stage times from a device
    clock; with kernel timing on they launch kernel by kernel.  Both give the same bits (odd and
    even step counts)."""
    torch, swf, _ = env
    for d in (W.small_parity_cases()[0], dict(W.small_parity_cases()[1], n_steps=7)):
        for prec in (swf.C128, swf.C64):
            outs = []
            for timed in (False, True):
                ctx = swf.Context(0)
                ctx.profile_enable(timed)
                out = torch.zeros(2 * 4 * int(np.prod(d["n"])), device="cuda",
                                  dtype=torch.float64 if prec == swf.C128 else torch.float32)
                ctx.march_dev([swf.from_workload(d)], out, bg=0, prec=prec)
                torch.cuda.synchronize()
                outs.append(out.cpu().numpy())
                ctx.close()
            assert np.array_equal(outs[0], outs[1]), (d["n_steps"], prec)


@pytest.mark.parametrize("n", [(512, 6, 1), (6, 512, 1), (4, 6, 512)])
def test_march_at_the_maximum_axis_length(env, n):
    """The largest axis length (512 = 16 x 16 x 2 in the line FFTs) along x, y and z, both
    precisions, against the oracle."""
    torch, swf, ctx = env
    L = tuple(40.0 if k == 512 else (6.0 if k > 1 else 1.0) for k in n)
    p = (0.2, 0.1, 0.0) if n[2] == 1 else (0.2, 0.1, 0.05)
    # h = 0.05: |kappa|_max h = 2 at 512 points on a box of 40, inside the Dormand-Prince region
    d = dict(field=("sauter_gauss", (0.6, 0.5, 3.0)), n=n, L=L, t_in=-1.5, t_out=1.5, n_steps=60, p=p, s=1,
             q=(-0.1, 0.0, 0.0), r=1, k=(0, 0, 0), eps=(0, 0, 0), flags=())
    ref = OA.to_gpu_layout(O.march_scattered(OA.field(d), OA.grid(d), OA.background(d, 0), d["t_in"], d["t_out"],
                                             d["n_steps"]))
    for prec, tol in ((swf.C128, 1e-10), (swf.C64, 2e-5)):
        out = torch.zeros(2 * 4 * int(np.prod(n)), dtype=torch.float64 if prec == swf.C128 else torch.float32,
                          device="cuda")
        ctx.march_dev([swf.from_workload(d)], out, bg=0, prec=prec)
        got = to_complex(out).reshape(ref.shape)
        assert rel_state(got, ref) < tol, (n, prec, rel_state(got, ref))


def test_single_fp64_workload_matches_stored_oracle(env):
    """The full-size single FP64 workload (128^2, 1000 steps) with the full pair number for both
    positron spins, against oracle values written by tests/golden/make_full_size_reference.py."""
    import json
    import os
    torch, swf, ctx = env
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "schwinger_fp64_single.json")))
    d0 = W.schwinger_fp64_single()[0]
    ds = [dict(d0, r=pr["r"], flags=("spectrum", "full_n")) for pr in golden["pairs"]]
    res, spec = ctx.solve([swf.from_workload(d) for d in ds], swf.SCHWINGER, swf.C128)
    # r = -1 is forbidden here (spin along x conserved for p_perp = 0): compare on the common scale
    scale = max(np.hypot(*pr[k]) for pr in golden["pairs"] for k in ("C", "D", "A", "B"))
    n_scale = max(max(pr["N_line1"], pr["N_line2"]) for pr in golden["pairs"])
    for r, pr in zip(res, golden["pairs"]):
        for j, key in enumerate(("C", "D", "A", "B")):
            got = complex(r.amp[2 * j], r.amp[2 * j + 1])
            assert abs(got - complex(*pr[key])) <= 1e-10 * scale, (pr["r"], key)
        assert abs(r.prob[0] - pr["N_line2"]) <= 1e-10 * n_scale
        assert abs(r.prob[1] - pr["N_line1"]) <= 1e-10 * n_scale
        assert abs(r.diag[0] - golden["norm_u"]) <= 1e-10 * golden["norm_u"]
        assert abs(r.diag[1] - pr["norm_v"]) <= 1e-10 * pr["norm_v"]
    modes = np.array(golden["spectrum_modes"])
    ref = np.array(golden["spectrum_prob"])
    assert np.max(np.abs(spec[modes] - ref)) <= 1e-10 * ref.max()


def test_full_3d_grid_conserves_the_norm_of_the_full_wave(env):
    """(3+1)D at the workload's full grid (256^3, box 48, its field): for a grid-mode momentum the
    full wave psi_b + psi_s evolves unitarily, so ||psi_b + psi_s||^2 = L^3 at t_in (a property
    that holds at any size), and the zero field gives exactly zero."""
    torch, swf, ctx = env
    L = 48.0
    p = (2 * np.pi / L * 3, 0.0, 0.0)
    # the workload's step (h = 0.025: |kappa|_max h = 0.42, inside the Dormand-Prince region)
    base = dict(n=(256, 256, 256), L=(L, L, L), t_in=-0.75, t_out=0.75, n_steps=60, p=p, s=1,
                q=(-p[0], 0.0, 0.0), r=1, k=(0, 0, 0), eps=(0, 0, 0), flags=())
    d = dict(base, field=("sauter_gauss", (0.3, 0.4, 6.0)))
    N = 256 ** 3
    out = torch.zeros(2 * 4 * N, dtype=torch.float32, device="cuda")
    ctx.march_dev([swf.from_workload(d)], out, bg=0, prec=swf.C64)
    psi = torch.view_as_complex(out.view(4, N, 2))
    assert float(psi.abs().max()) > 1e-3  # the field acts
    dx = L / 256
    x = -L / 2 + dx * torch.arange(256, device="cuda", dtype=torch.float64)
    p0 = float(np.sqrt(1 + p[0] ** 2))
    ph = torch.exp(1j * (p[0] * x - p0 * d["t_in"]))  # e^{-i(p0 t - p.x)} along x
    u = O.u_spinor(np.array(p), 1)
    total = 0.0
    for c in range(4):
        wave = (complex(u[c]) * ph).to(torch.complex128)
        full = psi[c].view(256, 256, 256).to(torch.complex128) + wave.view(1, 1, 256)
        total += float((full.abs() ** 2).sum()) * dx ** 3
        del full
    assert abs(total - L ** 3) <= 2e-5 * L ** 3, (total, L ** 3)
    z = dict(base, field=("zero", (0.0,)))
    out.zero_()
    ctx.march_dev([swf.from_workload(z)], out, bg=0, prec=swf.C64)
    assert float(out.abs().max()) == 0.0


def test_step_size_controlled_march_matches_oracle(env):
    """SWF_ADAPTIVE: the Dormand-Prince 5(4) pair with the integral step controller, decided on
    the device (graph replays).  Against the oracle's controlled march (same tolerances, same first
    step): same accepted/rejected counts and the same state to round-off in complex128; both
    within the tolerance of a converged fixed-step march; a too-large first step is rejected;
    graph replay and kernel-by-kernel launches give the same bits."""
    torch, swf, _ = env
    d0 = dict(field=("sauter_gauss", (0.8, 0.6, 2.5)), n=(16, 16, 1), L=(12.0, 12.0, 1.0), t_in=-6.0, t_out=6.0,
              n_steps=120, p=(0.3, -0.2, 0.0), s=1, q=(-0.2, 0.1, 0.0), r=1, k=(0, 0, 0), eps=(0, 0, 0),
              flags=("adaptive",))
    grid, fld, bg = OA.grid(d0), OA.field(d0), OA.background(d0, 0)
    ref_fixed = OA.to_gpu_layout(O.march_scattered(fld, grid, bg, -6.0, 6.0, 4000))
    for n_steps in (120, 4):  # first step 0.1, and 3.0 (rejected at least once)
        d = dict(d0, n_steps=n_steps)
        y, na, nr = O.march_scattered_adaptive(fld, grid, bg, -6.0, 6.0, 12.0 / n_steps, 1e-5, 1e-10)
        ref = OA.to_gpu_layout(y)
        outs = []
        for timed in (False, True):
            ctx = swf.Context(0)
            ctx.profile_enable(timed)
            out = torch.zeros(2 * 4 * 256, dtype=torch.float64, device="cuda")
            ctx.march_dev([swf.from_workload(d)], out, bg=0, prec=swf.C128)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
            stats = ctx.march_stats()
            # untimed: the attempt loop runs on the device (one graph launch); timed: host chunks
            assert ctx.device_loop_marches() == (0 if timed else 1), timed
            ctx.close()
        assert np.array_equal(outs[0], outs[1])
        assert stats == (na, nr), (stats, na, nr)
        got = to_complex(torch.from_numpy(outs[0])).reshape(ref.shape)
        assert rel_state(got, ref) < 1e-10, rel_state(got, ref)
        assert rel_state(got, ref_fixed) < 20 * 1e-5
        if n_steps == 4:
            assert nr > 0
    # complex64: within the tolerance of the converged march
    ctx = swf.Context(0)
    out = torch.zeros(2 * 4 * 256, dtype=torch.float32, device="cuda")
    ctx.march_dev([swf.from_workload(d0)], out, bg=0, prec=swf.C64)
    got = to_complex(out).reshape(ref_fixed.shape)
    assert rel_state(got, ref_fixed) < 20 * 1e-5
    # tighter tolerance: more steps, smaller error
    ctx.set_tolerances(1e-7, 1e-12)
    out64 = torch.zeros(2 * 4 * 256, dtype=torch.float64, device="cuda")
    ctx.march_dev([swf.from_workload(d0)], out64, bg=0, prec=swf.C128)
    got = to_complex(out64).reshape(ref_fixed.shape)
    assert rel_state(got, ref_fixed) < 20 * 1e-7 and ctx.march_stats()[0] > stats[0]
    ctx.close()


def _multi_solve(swf, ds, process, prec, mode):
    ctx = swf.Context(0)
    ctx.set_multi_grid(mode)
    ctx.profile_enable(True)
    ctx.profile_read()
    res, spec = ctx.solve([swf.from_workload(d) for d in ds], process, prec)
    prof, _ = ctx.profile_read()
    ctx.close()
    return [list(r.amp) + list(r.prob) + list(r.diag) for r in res], spec, prof


@pytest.mark.parametrize("dims", [2, 3])
def test_uneven_grids_share_one_multi_grid_march(env, dims):
    """Batching of uneven grids (Sec. II.A): instance groups on different grids with one time grid
    are marched by one launch per pass (persistent blocks on a device work queue) and give bitwise
    the results of marching each group alone; a 256^2 complex64 group still takes the fused
    kernel beside them.  Spectra and the full pair number, both precisions, 2D and 3D grids."""
    torch, swf, _ = env
    base = dict(field=("sauter_gauss", (0.8, 0.6, 2.5)), t_in=-3.0, t_out=3.0, n_steps=24, k=(0, 0, 0),
                eps=(0, 0, 0), flags=("spectrum", "full_n"))
    if dims == 2:
        grids = [((32, 24, 1), (16.0, 12.0, 1.0)), ((40, 30, 1), (20.0, 15.0, 1.0)), ((20, 20, 1), (10.0, 10.0, 1.0))]
    else:
        grids = [((12, 10, 8), (8.0, 7.0, 6.0)), ((16, 8, 6), (9.0, 6.0, 5.0))]
    ds = []
    for j, (n, L) in enumerate(grids):
        for i in range(3):
            p = (0.1 * i - 0.1, 0.2 - 0.1 * j, 0.0 if dims == 2 else 0.05)
            ds.append(dict(base, n=n, L=L, p=p, s=1 if i % 2 else -1, q=(-0.2, 0.1 * j, 0.0), r=1 if i else -1))
    if dims == 2:  # a group for the fused kernel (complex64) in the same call (|kappa|_max h = 1.6)
        ds.append(dict(base, n=(256, 256, 1), L=(128.0, 128.0, 1.0), p=(0.3, 0.1, 0.0), s=1, q=(-0.3, 0.0, 0.0),
                       r=1, flags=("spectrum",)))
    for prec in (swf.C64, swf.C128):
        r1, s1, prof1 = _multi_solve(swf, ds, swf.SCHWINGER, prec, 2)   # always together
        r0, s0, prof0 = _multi_solve(swf, ds, swf.SCHWINGER, prec, 0)   # one group after another
        ra, sa, profa = _multi_solve(swf, ds, swf.SCHWINGER, prec, 1)   # automatic: small groups go together
        assert "k_first_multi" in prof1 and "k_first_multi" not in prof0, (prof1, prof0)
        assert "k_first_multi" in profa
        assert np.all(np.isfinite(r1)) and np.all(np.isfinite(s1))
        assert r1 == r0 == ra, prec
        assert np.array_equal(s1, s0) and np.array_equal(s1, sa), prec
        assert max(abs(x) for r in r1 for x in r) > 0
