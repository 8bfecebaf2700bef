"""Builds the oracle's objects from a workload dict (test side; no CUDA involved)."""
import numpy as np

from oracle import swf_oracle as O


def field(d):
    kind, prm = d["field"]
    prm = tuple(prm)
    if kind == "sauter_gauss" and prm[2] <= 0:
        prm = (prm[0], prm[1], np.inf)
    return O.Field(kind, prm)


def grid(d):
    return O.Grid(d["n"], d["L"])


def background(d, bg):
    return O.Background("U", d["p"], d["s"]) if bg == 0 else O.Background("V", d["q"], d["r"])


def to_gpu_layout(psi):
    """Oracle (4, nx, ny, nz) -> library layout (4, nz, ny, nx)."""
    return np.ascontiguousarray(np.transpose(psi, (0, 3, 2, 1)))


def from_gpu_layout(arr, n):
    """Library layout flat/complex (4, nz, ny, nx) -> oracle (4, nx, ny, nz)."""
    a = np.asarray(arr).reshape(4, n[2], n[1], n[0])
    return np.transpose(a, (0, 3, 2, 1))
