"""The C ABI library builds, loads and exports every declared symbol; the ctypes mirrors match
the C struct layouts; host-side validation and error reporting work without a GPU."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def lib():
    from paper_2512_16889_gb300 import build, swf
    build.build()
    return swf.load_library()


def declared_functions():
    names = []
    for fn in sorted(os.listdir(INCLUDE)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:swf_status|const char\s*\*|int)\s*(\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "solve_swf" in names and "swf_create" in names
    for name in names:
        assert hasattr(lib, name), name


def test_struct_layouts_match_c(lib):
    from paper_2512_16889_gb300 import swf
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "swf.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(swf_field), sizeof(swf_grid), sizeof(swf_instance), sizeof(swf_result));
  printf("%zu %zu %zu %zu %zu\n", offsetof(swf_instance, grid), offsetof(swf_instance, p),
         offsetof(swf_instance, q), offsetof(swf_instance, eps), offsetof(swf_instance, flags));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", INCLUDE, c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    sizes = [int(v) for v in out[:4]]
    offs = [int(v) for v in out[4:]]
    assert sizes == [C.sizeof(swf.Field), C.sizeof(swf.Grid), C.sizeof(swf.Instance), C.sizeof(swf.Result)]
    assert offs == [swf.Instance.grid.offset, swf.Instance.p.offset, swf.Instance.q.offset,
                    swf.Instance.eps.offset, swf.Instance.flags.offset]


def test_errors_without_device(lib):
    from paper_2512_16889_gb300 import swf
    import torch
    if torch.cuda.is_available():
        pytest.skip("checks the no-device path")
    h = C.c_void_p()
    st = lib.swf_create(C.byref(h), 0)
    assert st == swf.SWF_ECUDA and not h
    assert b"not available" in lib.swf_last_error()
    # a NULL context is rejected by validation before any CUDA call
    arr = swf.instance_array([swf.make_instance(1, (0.3, 0.5, 5.0), (8, 8, 1), (4, 4, 1), -1, 1, 2)])
    res = (swf.Result * 1)()
    assert lib.solve_swf(None, 1, arr, 0, 1, res, None) == swf.SWF_EINVAL
    assert b"ctx is NULL" in lib.swf_last_error()
    assert lib.swf_destroy(None) == swf.SWF_OK
    # the fused kernel's status and its diagnostic switch reject a NULL context or output
    status = C.c_int(7)
    assert lib.swf_fused_status(None, C.byref(status)) == swf.SWF_EINVAL
    assert lib.swf_set_fused_drop(None, 1) == swf.SWF_EINVAL


def test_split_plan_of_fused_marches(lib):
    """Host logic of the fused/pass split (default fused kernel, pushed transposes, alpha = 2.0
    sector rounds per pass-kernel field with 40 free SMs): the benchmark's 128 fields on GB300's
    152 SMs and 7 resident 16-CTA clusters give 16 fields to the pass kernels (R = 37 rounds; 32
    rounds leave 16 fields, 16 x 2.0 <= 32, while 31 rounds would leave 20, 20 x 2.0 > 31); the
    fused part always ends in fewer sector rounds than the whole, and the pass part stays within
    the time model."""
    from paper_2512_16889_gb300 import swf
    assert swf.plan_split(128, 7, 152) == 16
    assert swf.plan_split(14, 7, 152) == 0      # too few fields
    assert swf.plan_split(128, 9, 152) == 0     # too few free SMs
    assert swf.plan_split(128, 0, 152) == 0
    for n in range(16, 400):
        n2 = swf.plan_split(n, 7, 152)
        if n2 == 0:
            continue
        n1 = n - n2
        rounds_all = -(-2 * n // 7)
        rounds_fused = -(-2 * n1 // 7)
        assert 0 < n2 < n and rounds_fused < rounds_all, n
        assert 2.0 * n2 <= rounds_fused + 1e-12, n
    with pytest.raises(swf.SwfError) as ei:
        swf.plan_split(-1, 7, 152)
    assert ei.value.status == swf.SWF_EINVAL


def test_rhs_wrappers_check_their_tensors_before_any_call(monkeypatch):
    """The right-hand-side wrappers refuse tensors that would make the kernels read or write out
    of bounds (wrong dtype for the precision, too few values, not contiguous) before a pointer
    reaches the library; the checks need no GPU."""
    import torch
    from paper_2512_16889_gb300 import swf
    d = dict(field=("sauter_gauss", (0.8, 0.6, 2.5)), n=(8, 4, 1), L=(8.0, 4.0, 1.0), t_in=-1.0, t_out=1.0,
             n_steps=2, p=(0.0, 0.0, 0.0), s=1, q=(0.0, 0.0, 0.0), r=1, k=(0, 0, 0), eps=(0, 0, 0), flags=())
    inst = swf.from_workload(d)
    cpu = torch.zeros(8 * 32, dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA tensor"):
        swf._check_state_tensors(inst, cpu, cpu, swf.C64)

    class FakeCuda:  # the attributes the check reads, without a device
        def __init__(self, dtype, numel, contiguous=True, device="cuda:0"):
            self.dtype, self._n, self._c, self.device, self.is_cuda = dtype, numel, contiguous, torch.device(device), True

        def numel(self):
            return self._n

        def is_contiguous(self):
            return self._c

    monkeypatch.setattr(torch, "Tensor", FakeCuda)  # the wrapper's isinstance check
    ok = FakeCuda(torch.float32, 8 * 32)
    assert swf._check_state_tensors(inst, ok, ok, swf.C64) == torch.device("cuda:0")
    with pytest.raises(ValueError, match="dtype"):
        swf._check_state_tensors(inst, ok, ok, swf.C128)
    with pytest.raises(ValueError, match="the grid needs 256"):
        swf._check_state_tensors(inst, FakeCuda(torch.float32, 255), ok, swf.C64)
    with pytest.raises(ValueError, match="contiguous"):
        swf._check_state_tensors(inst, ok, FakeCuda(torch.float32, 256, contiguous=False), swf.C64)
    with pytest.raises(ValueError, match="cuda:1"):
        swf._check_state_tensors(inst, ok, FakeCuda(torch.float32, 256, device="cuda:1"), swf.C64)
