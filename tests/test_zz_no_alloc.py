"""The allocation-free right-hand side (swf_rhs_noalloc) against swf_rhs_dev.

swf_rhs_noalloc serves callers that cannot allocate device memory (host applications that own
all device memory through a pool of their own, loops that cannot absorb cudaFree's device-wide
synchronisation); it takes its workspace from a fixed device array instead of a context.  This file is collected last so that a failure here never hides another test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [
    # field, grid, box, electron momentum: a (2+1)D grid with a non-power-of-two axis and a
    # (3+1)D grid, so that every pass kernel runs
    (("sauter_gauss", (0.8, 0.6, 2.5)), (32, 24, 1), (16.0, 12.0, 1.0), (0.3, -0.2, 0.0)),
    (("single_e", (0.6, 0.5, 0.3, 0.3, 0.2)), (16, 12, 10), (10.0, 8.0, 7.0), (0.1, 0.2, -0.3)),
]


def _case(k):
    from paper_2512_16889_gb300 import swf
    fld, n, L, p = CASES[k]
    d = dict(field=fld, n=n, L=L, t_in=-4.0, t_out=4.0, n_steps=10, p=p, s=1, q=(-0.2, 0.1, 0.0), r=-1,
             k=(0, 0, 0), eps=(0, 0, 0), flags=())
    return swf.from_workload(d), int(np.prod(n))


def test_rhs_noalloc_matches_rhs_dev_twice_in_a_row():
    import torch
    from paper_2512_16889_gb300 import build, swf
    build.build()
    ctx = swf.Context(0)
    rng = np.random.default_rng(42)
    # two calls in a row per precision, on different grids, then the first grid again
    for prec, tol in ((swf.C128, 1e-12), (swf.C64, 2e-6)):
        real = torch.float64 if prec == swf.C128 else torch.float32
        for k in (0, 1, 0):
            inst, N = _case(k)
            psi = torch.from_numpy(rng.normal(size=8 * N)).to(real).cuda()
            ref = torch.zeros_like(psi)
            got = torch.full_like(psi, float("nan"))
            for bg in (0, 1):
                ctx.rhs_dev(inst, 0.37, psi, ref, bg=bg, prec=prec)
                swf.rhs_noalloc(inst, 0.37, psi, got, bg=bg, prec=prec)
                torch.cuda.synchronize()
                err = (got - ref).abs().max().item() / ref.abs().max().item()
                assert err < tol, (prec, k, bg, err)
    ctx.close()


def test_rhs_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2512_16889_gb300 import build, swf
    build.build()
    d = dict(field=("sauter_gauss", (0.3, 0.5, 5.0)), n=(512, 256, 1), L=(40.0, 40.0, 1.0), t_in=-1.0, t_out=1.0,
             n_steps=1, p=(0.0, 0.0, 0.0), s=1, q=(0.0, 0.0, 0.0), r=1, k=(0, 0, 0), eps=(0, 0, 0), flags=())
    x = torch.zeros(8 * 512 * 256, dtype=torch.float32, device="cuda")  # the grid's full size: the
    y = torch.zeros_like(x)                                              # library's own check answers
    with pytest.raises(swf.SwfError) as ei:
        swf.rhs_noalloc(swf.from_workload(d), 0.0, x, y, prec=swf.C64)
    assert ei.value.status == swf.SWF_EINVAL and "exceeds the fixed scratch" in str(ei.value)
