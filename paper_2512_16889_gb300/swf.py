"""Python binding of the C ABI in ``include/swf.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``libswf.so``; this module only mirrors the
C structures with ctypes and passes host pointers or torch device pointers through.  There is
no CPU fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libswf.so")

SWF_OK, SWF_EINVAL, SWF_ENOMEM, SWF_ECUDA, SWF_ENUMERIC, SWF_ETIMEOUT, SWF_EUNSUPPORTED = range(7)
STATUS_NAMES = ["SWF_OK", "SWF_EINVAL", "SWF_ENOMEM", "SWF_ECUDA", "SWF_ENUMERIC", "SWF_ETIMEOUT",
                "SWF_EUNSUPPORTED"]
SCHWINGER, BREIT_WHEELER = 0, 1
C128, C64 = 0, 1
FIELD_ZERO, FIELD_SAUTER_GAUSS, FIELD_PULSE_GAUSS, FIELD_SINGLE_E, FIELD_DOUBLE_E = range(5)
WANT_SPECTRUM, WANT_FULL_N, ADAPTIVE, BW_PARTIAL = 1, 2, 4, 8


class Field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("prm", C.c_double * 8)]


class Grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("n_steps", C.c_int32), ("L", C.c_double * 3),
                ("t_in", C.c_double), ("t_out", C.c_double)]


class Instance(C.Structure):
    _fields_ = [("field", Field), ("grid", Grid),
                ("p", C.c_double * 3), ("s", C.c_int32),
                ("r", C.c_int32), ("q", C.c_double * 3),
                ("k", C.c_double * 3), ("eps", C.c_double * 3),
                ("flags", C.c_int32), ("reserved", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("amp", C.c_double * 8), ("prob", C.c_double * 2), ("diag", C.c_double * 2)]


EXPORTS = ["swf_create", "swf_destroy", "swf_last_error", "solve_swf", "solve_swf_dev", "swf_pair_matrix",
           "swf_bw_photons", "swf_march_dev",
           "swf_rhs_dev", "swf_spectrum_dev", "swf_set_workspace_limit", "swf_profile_enable",
           "swf_profile_read", "swf_set_march_path", "swf_set_autotune", "swf_set_dedupe", "swf_fields_marched",
           "swf_fields_fused", "swf_plan_split", "swf_fused_status", "swf_set_fused_drop",
           "swf_set_tolerances", "swf_march_stats", "swf_set_multi_grid", "swf_device_loop_marches",
           "swf_rhs_noalloc", "swf_mlp_param_count", "swf_mlp_create",
           "swf_mlp_destroy", "swf_mlp_forward", "swf_mlp_activation", "swf_mlp_status", "swf_mlp_gradients", "swf_mlp_train_step",
           "swf_mlp_get_params"]


class SwfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libswf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2512_16889_gb300.build.build()")
    lib = C.CDLL(path)
    vp, ip, dp = C.c_void_p, C.c_int, C.c_double
    inst_p, res_p, dbl_p = C.POINTER(Instance), C.POINTER(Result), C.POINTER(C.c_double)
    lib.swf_create.argtypes = [C.POINTER(vp), ip]
    lib.swf_destroy.argtypes = [vp]
    lib.swf_last_error.restype = C.c_char_p
    lib.solve_swf.argtypes = [vp, ip, inst_p, ip, ip, res_p, dbl_p]
    lib.solve_swf_dev.argtypes = [vp, ip, inst_p, ip, ip, vp, vp, vp]
    lib.swf_pair_matrix.argtypes = [vp, ip, inst_p, ip, inst_p, ip, res_p]
    dptr = C.POINTER(C.c_double)
    lib.swf_bw_photons.argtypes = [vp, inst_p, ip, dptr, dptr, dptr, ip, dptr, dptr]
    lib.swf_march_dev.argtypes = [vp, ip, inst_p, ip, ip, vp, vp]
    lib.swf_rhs_dev.argtypes = [vp, inst_p, ip, ip, dp, vp, vp, vp]
    lib.swf_spectrum_dev.argtypes = [vp, ip, inst_p, ip, vp, vp, vp, vp]
    lib.swf_set_workspace_limit.argtypes = [vp, C.c_size_t]
    lib.swf_profile_enable.argtypes = [vp, ip]
    lib.swf_set_march_path.argtypes = [vp, ip]
    lib.swf_fused_status.argtypes = [vp, C.POINTER(C.c_int)]
    lib.swf_set_fused_drop.argtypes = [vp, ip]
    lib.swf_set_autotune.argtypes = [vp, ip]
    lib.swf_set_dedupe.argtypes = [vp, ip]
    lib.swf_set_multi_grid.argtypes = [vp, ip]
    lib.swf_set_tolerances.argtypes = [vp, dp, dp]
    lib.swf_march_stats.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    lib.swf_fields_marched.argtypes = [vp, C.POINTER(C.c_longlong)]
    lib.swf_device_loop_marches.argtypes = [vp, C.POINTER(C.c_longlong)]
    lib.swf_fields_fused.argtypes = [vp, C.POINTER(C.c_longlong)]
    lib.swf_plan_split.argtypes = [ip, ip, ip, C.POINTER(C.c_int)]
    lib.swf_rhs_noalloc.argtypes = [inst_p, ip, ip, dp, vp, vp, vp]
    fp = C.POINTER(C.c_float)
    lib.swf_mlp_param_count.argtypes = []
    lib.swf_mlp_create.argtypes = [C.POINTER(vp), ip, fp, ip, fp]
    lib.swf_mlp_destroy.argtypes = [vp]
    lib.swf_mlp_forward.argtypes = [vp, vp, ip, vp, vp]
    lib.swf_mlp_status.argtypes = [vp]
    lib.swf_mlp_gradients.argtypes = [vp, vp, vp, ip, vp, vp, vp]
    lib.swf_mlp_train_step.argtypes = [vp, vp, vp, ip, C.c_float, vp, vp]
    lib.swf_mlp_get_params.argtypes = [vp, fp]
    lib.swf_mlp_activation.argtypes = [vp, ip, vp, vp, vp]
    lib.swf_profile_read.argtypes = [vp, ip, C.c_char_p, dbl_p, C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                                     C.POINTER(C.c_longlong)]
    for name in EXPORTS:
        if name != "swf_last_error":
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(status):
    if status != SWF_OK:
        raise SwfError(status, _lib.swf_last_error().decode())


def make_instance(field_kind, prm, n, L, t_in, t_out, n_steps, p=(0, 0, 0), s=1, q=(0, 0, 0), r=1,
                  k=(0, 0, 0), eps=(0, 0, 0), flags=0) -> Instance:
    inst = Instance()
    inst.field.kind = field_kind
    for i, v in enumerate(prm):
        inst.field.prm[i] = float(v)
    for a in range(3):
        inst.grid.n[a] = int(n[a])
        inst.grid.L[a] = float(L[a])
        inst.p[a], inst.q[a], inst.k[a], inst.eps[a] = float(p[a]), float(q[a]), float(k[a]), float(eps[a])
    inst.grid.n_steps = int(n_steps)
    inst.grid.t_in, inst.grid.t_out = float(t_in), float(t_out)
    inst.s, inst.r, inst.flags = int(s), int(r), int(flags)
    return inst


def instance_array(instances):
    arr = (Instance * len(instances))()
    for i, x in enumerate(instances):
        arr[i] = x
    return arr


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _check_state_tensors(instance, psi, out, prec):
    """Checks the device tensors of a right-hand-side call before their pointers are passed on:
    the real dtype of the precision, at least 2 x 4 x N values each (N grid points), contiguous,
    both on one CUDA device.  Returns that device."""
    import torch
    real = torch.float64 if prec == C128 else torch.float32
    need = 8 * int(np.prod([instance.grid.n[a] for a in range(3)]))
    for name, t in (("psi", psi), ("out", out)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != real:
            raise ValueError(f"{name} has dtype {t.dtype}; precision {'C128' if prec == C128 else 'C64'} needs {real}")
        if t.numel() < need:
            raise ValueError(f"{name} holds {t.numel()} values; the grid needs {need}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if psi.device != out.device:
        raise ValueError(f"psi is on {psi.device} and out on {out.device}")
    return psi.device


def _check_device_buffer(name, t, dtype, need, device=None):
    """A contiguous CUDA tensor of `dtype` holding at least `need` elements (on `device` if given)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} has dtype {t.dtype}; {dtype} is needed")
    if t.numel() < need:
        raise ValueError(f"{name} holds {t.numel()} values; {need} are needed")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on {t.device}; this context runs on cuda:{device}")


def _grid_points(inst):
    return int(inst.grid.n[0]) * int(inst.grid.n[1]) * int(inst.grid.n[2])


def rhs_noalloc(instance, t, psi, out, bg=0, prec=C64, stream=None):
    """swf_rhs_noalloc: one right-hand-side evaluation without any device allocation (see swf.h),
    on the tensors' device."""
    import torch
    load_library()
    dev = _check_state_tensors(instance, psi, out, prec)
    arr = instance_array([instance])
    with torch.cuda.device(dev):
        _check(_lib.swf_rhs_noalloc(arr, bg, prec, float(t), C.c_void_p(psi.data_ptr()),
                                    C.c_void_p(out.data_ptr()), _stream_ptr(stream)))


class Context:
    """A solver context on one CUDA device (owns workspace and a stream)."""

    def __init__(self, device: int = 0):
        load_library()
        self.device = int(device)
        self._h = C.c_void_p()
        _check(_lib.swf_create(C.byref(self._h), int(device)))

    def close(self):
        if self._h:
            _lib.swf_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_workspace_limit(self, nbytes: int):
        _check(_lib.swf_set_workspace_limit(self._h, int(nbytes)))

    def set_march_path(self, path: int):
        """0 = automatic (fused cluster kernel where it applies, the pass kernels on the free SMs),
        1 = pass kernels only, 2 = the automatic fused kernel for every field, 3 = two CTAs per SM,
        4 = transposes pulled by the threads, 5 = transposes pushed by the bulk-copy engine."""
        _check(_lib.swf_set_march_path(self._h, int(path)))

    def fused_status(self) -> int:
        """swf_fused_status: 1 if a receive wait of the last pushed-transpose fused march ran out."""
        s = C.c_int(0)
        _check(_lib.swf_fused_status(self._h, C.byref(s)))
        return s.value

    def set_fused_drop(self, on: bool):
        """swf_set_fused_drop (diagnostic): the pushed-transpose fused kernel issues no copies."""
        _check(_lib.swf_set_fused_drop(self._h, 1 if on else 0))

    def set_tolerances(self, rtol, atol):
        """Tolerances of step-size-controlled marches (flag "adaptive")."""
        _check(_lib.swf_set_tolerances(self._h, float(rtol), float(atol)))

    def march_stats(self):
        """(accepted, rejected) steps of the last step-size-controlled march."""
        a, r = C.c_longlong(), C.c_longlong()
        _check(_lib.swf_march_stats(self._h, C.byref(a), C.byref(r)))
        return a.value, r.value

    def set_dedupe(self, on: bool):
        """March repeated fields (the other spin of a z-spin-conserving field) once (True, default)."""
        _check(_lib.swf_set_dedupe(self._h, 1 if on else 0))

    def set_multi_grid(self, mode: int):
        """Instance groups on different grids sharing a time grid: 0 one after another, 1 together
        when they are small enough (default), 2 always together."""
        _check(_lib.swf_set_multi_grid(self._h, int(mode)))

    def device_loop_marches(self):
        """Step-size-controlled marches that ran as one graph launch with the attempt loop on the device."""
        n = C.c_longlong()
        _check(_lib.swf_device_loop_marches(self._h, C.byref(n)))
        return n.value

    def fields_marched(self):
        n = C.c_longlong()
        _check(_lib.swf_fields_marched(self._h, C.byref(n)))
        return n.value

    def fields_fused(self):
        """Fields marched by the fused cluster kernel since the context's creation."""
        n = C.c_longlong()
        _check(_lib.swf_fields_fused(self._h, C.byref(n)))
        return n.value

    def set_autotune(self, on: bool):
        """Pass-kernel launch shapes by timing (True, default) or by the fixed rule (False)."""
        _check(_lib.swf_set_autotune(self._h, 1 if on else 0))

    def profile_enable(self, on=True):
        _check(_lib.swf_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, max_entries=32):
        """{family: (total_ms, launches)} since the last read, and the total launch count."""
        names = C.create_string_buffer(32 * max_entries)
        ms = (C.c_double * max_entries)()
        cnt = (C.c_longlong * max_entries)()
        n = C.c_int()
        total = C.c_longlong()
        _check(_lib.swf_profile_read(self._h, max_entries, names, ms, cnt, C.byref(n), C.byref(total)))
        out = {}
        for i in range(n.value):
            nm = names.raw[32 * i:32 * (i + 1)].split(b"\0")[0].decode()
            out[nm] = (ms[i], cnt[i])
        return out, total.value

    # -- highest level, host buffers
    def solve(self, instances, process=SCHWINGER, prec=C64):
        arr = instance_array(instances)
        res = (Result * len(instances))()
        nspec = sum(2 * x.grid.n[0] * x.grid.n[1] * x.grid.n[2] for x in instances
                    if process == SCHWINGER and (x.flags & WANT_SPECTRUM))
        spec = np.zeros(max(nspec, 1), dtype=np.float64)
        _check(_lib.solve_swf(self._h, len(instances), arr, process, prec, res,
                              spec.ctypes.data_as(C.POINTER(C.c_double))))
        return res, spec[:nspec]

    def pair_matrix(self, electrons, positrons, prec=C64):
        """swf_pair_matrix: full N for every (electron, positron) pair; returns an n_e x n_p list
        of lists of Result."""
        ea, pa = instance_array(electrons), instance_array(positrons)
        res = (Result * (len(electrons) * len(positrons)))()
        _check(_lib.swf_pair_matrix(self._h, len(electrons), ea, len(positrons), pa, prec, res))
        n_p = len(positrons)
        return [[res[m * n_p + n] for n in range(n_p)] for m in range(len(electrons))]

    def bw_photons(self, instance, k, eps, prec=C64, weights=None):
        """swf_bw_photons: Breit-Wheeler amplitudes of n photons from one march of the instance's U
        and V.  k, eps: (n, 3) arrays; weights: optional (n,) complex.  Returns (amps, packet):
        amps (n, 4) complex (M_ss, M_bs, M_sb, M) and packet (4,) complex = sum_j w_j amps[j], or
        None without weights."""
        k = np.ascontiguousarray(np.asarray(k, dtype=np.float64).reshape(-1, 3))
        eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(-1, 3))
        n = k.shape[0]
        if eps.shape[0] != n:
            raise ValueError("k and eps must list the same photons")
        arr = instance_array([instance])
        amps = np.zeros((n, 8), dtype=np.float64)
        dp = C.POINTER(C.c_double)
        wbuf, pbuf = None, None
        if weights is not None:
            w = np.asarray(weights, dtype=np.complex128).reshape(n)
            wbuf = np.ascontiguousarray(np.stack([w.real, w.imag], axis=1))
            pbuf = np.zeros(8, dtype=np.float64)
        _check(_lib.swf_bw_photons(self._h, arr, n, k.ctypes.data_as(dp), eps.ctypes.data_as(dp),
                                   wbuf.ctypes.data_as(dp) if wbuf is not None else None, prec,
                                   amps.ctypes.data_as(dp), pbuf.ctypes.data_as(dp) if pbuf is not None else None))
        out = amps[:, 0::2] + 1j * amps[:, 1::2]
        packet = (pbuf[0::2] + 1j * pbuf[1::2]) if pbuf is not None else None
        return out, packet

    # -- device buffers (torch tensors), asynchronous on `stream`
    def solve_dev(self, instances, results_dev, spectrum_dev=None, process=SCHWINGER, prec=C64, stream=None,
                  arr=None):
        import torch
        arr = arr if arr is not None else instance_array(instances)
        _check_device_buffer("results_dev", results_dev, results_dev.dtype, 0, self.device)
        if results_dev.numel() * results_dev.element_size() < len(arr) * C.sizeof(Result):
            raise ValueError(f"results_dev holds fewer than {len(arr)} results")
        if spectrum_dev is not None:
            nspec = sum(2 * _grid_points(x) for x in arr if process == SCHWINGER and (x.flags & WANT_SPECTRUM))
            _check_device_buffer("spectrum_dev", spectrum_dev, torch.float64, nspec, self.device)
        _check(_lib.solve_swf_dev(self._h, len(arr), arr, process, prec, C.c_void_p(results_dev.data_ptr()),
                                  C.c_void_p(spectrum_dev.data_ptr()) if spectrum_dev is not None else None,
                                  _stream_ptr(stream)))

    def march_dev(self, instances, psi_out, bg=0, prec=C64, stream=None):
        import torch
        arr = instance_array(instances)
        need = sum(8 * _grid_points(x) for x in arr)
        _check_device_buffer("psi_out", psi_out, torch.float64 if prec == C128 else torch.float32, need, self.device)
        _check(_lib.swf_march_dev(self._h, len(instances), arr, bg, prec, C.c_void_p(psi_out.data_ptr()),
                                  _stream_ptr(stream)))

    def rhs_dev(self, instance, t, psi, out, bg=0, prec=C64, stream=None):
        dev = _check_state_tensors(instance, psi, out, prec)
        if dev.index != self.device:
            raise ValueError(f"the tensors are on {dev}; this context runs on cuda:{self.device}")
        arr = instance_array([instance])
        _check(_lib.swf_rhs_dev(self._h, arr, bg, prec, float(t), C.c_void_p(psi.data_ptr()),
                                C.c_void_p(out.data_ptr()), _stream_ptr(stream)))

    def spectrum_dev(self, instances, psi, c_out=None, prob_out=None, prec=C64, stream=None):
        import torch
        arr = instance_array(instances)
        npts = sum(_grid_points(x) for x in arr)
        _check_device_buffer("psi", psi, torch.float64 if prec == C128 else torch.float32, 8 * npts, self.device)
        if c_out is not None:
            _check_device_buffer("c_out", c_out, torch.float64, 4 * npts, self.device)
        if prob_out is not None:
            _check_device_buffer("prob_out", prob_out, torch.float64, 2 * npts, self.device)
        _check(_lib.swf_spectrum_dev(self._h, len(instances), arr, prec, C.c_void_p(psi.data_ptr()),
                                     C.c_void_p(c_out.data_ptr()) if c_out is not None else None,
                                     C.c_void_p(prob_out.data_ptr()) if prob_out is not None else None,
                                     _stream_ptr(stream)))


FIELD_CODES = {"zero": FIELD_ZERO, "sauter_gauss": FIELD_SAUTER_GAUSS, "pulse_gauss": FIELD_PULSE_GAUSS,
               "single_e": FIELD_SINGLE_E, "double_e": FIELD_DOUBLE_E}
FLAG_CODES = {"spectrum": WANT_SPECTRUM, "full_n": WANT_FULL_N, "adaptive": ADAPTIVE, "bw_partial": BW_PARTIAL}


def plan_split(n_fields, clusters, sms):
    """swf_plan_split: fields of a fused march given to the pass kernels on the free SMs."""
    load_library()
    out = C.c_int()
    _check(_lib.swf_plan_split(int(n_fields), int(clusters), int(sms), C.byref(out)))
    return out.value


def from_workload(d) -> Instance:
    """Marshal one workload dict (see ``workloads``) into the C instance struct."""
    kind, prm = d["field"]
    flags = 0
    for f in d.get("flags", ()):
        flags |= FLAG_CODES[f]
    return make_instance(FIELD_CODES[kind], prm, d["n"], d["L"], d["t_in"], d["t_out"], d["n_steps"],
                         p=d["p"], s=d["s"], q=d["q"], r=d["r"], k=d["k"], eps=d["eps"], flags=flags)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class Surrogate:
    """The surrogate network of swf.h (swf_mlp_*); tensors are torch CUDA float32 tensors."""

    def __init__(self, init_params, norm, max_batch=4096, device=0):
        load_library()
        p = np.ascontiguousarray(init_params, dtype=np.float32)
        n = np.ascontiguousarray(norm, dtype=np.float32)
        assert p.size == _lib.swf_mlp_param_count() and n.size == 14
        self._h = C.c_void_p()
        _check(_lib.swf_mlp_create(C.byref(self._h), int(device), p.ctypes.data_as(C.POINTER(C.c_float)),
                                   int(max_batch), n.ctypes.data_as(C.POINTER(C.c_float))))
        self.max_batch = max_batch

    @staticmethod
    def activation(x, gelu_out, grad_out, stream=None):
        """swf_mlp_activation: the network's GELU and its derivative on device float tensors."""
        load_library()
        for t in (x, gelu_out, grad_out):
            if t.dtype.itemsize != 4 or not t.is_cuda or not t.is_contiguous():
                raise ValueError("activation: contiguous float32 CUDA tensors")
        if gelu_out.numel() < x.numel() or grad_out.numel() < x.numel():
            raise ValueError("activation: outputs shorter than the input")
        _check(_lib.swf_mlp_activation(C.c_void_p(x.data_ptr()), int(x.numel()), C.c_void_p(gelu_out.data_ptr()),
                                       C.c_void_p(grad_out.data_ptr()), _stream_ptr(stream)))

    @staticmethod
    def param_count():
        load_library()
        return _lib.swf_mlp_param_count()

    def close(self):
        if self._h:
            _lib.swf_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, x, out, stream=None):
        _check(_lib.swf_mlp_forward(self._h, _ptr(x), x.shape[0], _ptr(out), _stream_ptr(stream)))

    def status(self):
        """Waits for the last inference call; raises SwfError if one of its waits timed out."""
        _check(_lib.swf_mlp_status(self._h))

    def gradients(self, x, y, grad=None, loss=None, stream=None):
        _check(_lib.swf_mlp_gradients(self._h, _ptr(x), _ptr(y), x.shape[0], _ptr(grad), _ptr(loss),
                                      _stream_ptr(stream)))

    def train_step(self, x, y, lr, loss=None, stream=None):
        _check(_lib.swf_mlp_train_step(self._h, _ptr(x), _ptr(y), x.shape[0], float(lr), _ptr(loss),
                                       _stream_ptr(stream)))

    def params(self):
        out = np.zeros(_lib.swf_mlp_param_count(), dtype=np.float32)
        _check(_lib.swf_mlp_get_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out
