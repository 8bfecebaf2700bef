"""Writes oracle-only reference values for full-size workloads (no CUDA involved).

* batched Schwinger (256^2, 128 instances, 1000 steps): per selected instance the C-spectrum
  |C(m,(r,q))|^2 at the 64 largest modes and 64 modes spread over the spectrum, and
  ||psi_scat(t_in)||^2 -> schwinger_batched_samples.json;
* single FP64 Schwinger (128^2, 1000 steps): the full pair number (both lines of Eq. 8 and the
  amplitudes C, D, A, B) for r = +1 and -1, and C-spectrum samples -> schwinger_fp64_single.json;
* batched Schwinger, whole spectra: for selected instances every C-spectrum entry at or above
  1e-24 of the spectrum's maximum (the range where the complex64 and FP64 marches are compared
  decade by decade) -> schwinger_batched_spectrum_<i>.json;
* Breit-Wheeler uneven grids: the amplitude terms of one instance of the smallest grid (192^2,
  2605 steps) -> bw_uneven_sample.json; the same instance in the partial-integration form of
  Sec. IV (Eqs. 30-33) -> bw_uneven_partial_sample.json.
The GPU tests compare the library's solves of the same instances against these values.

    python tests/golden/make_full_size_reference.py [instance ...]     # batched Schwinger
    python tests/golden/make_full_size_reference.py --spectrum <instance>
    python tests/golden/make_full_size_reference.py --single
    python tests/golden/make_full_size_reference.py --bw
    python tests/golden/make_full_size_reference.py --bw-partial
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import swf_oracle as O  # noqa: E402
from paper_2512_16889_gb300 import workloads as W  # noqa: E402
from tests import oracle_adapter as OA  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "schwinger_batched_samples.json")


def sample(i):
    d = W.schwinger_batched()[i]
    g = OA.grid(d)
    t0 = time.time()
    psi = O.march_scattered(OA.field(d), g, OA.background(d, 0), d["t_in"], d["t_out"], d["n_steps"])
    C = O.c_spectrum(psi, g, d["t_in"])
    prob = np.transpose(np.abs(C) ** 2, (0, 3, 2, 1)).ravel()  # library layout [r][z][y][x]
    top = np.argsort(prob)[::-1][:64]
    spread = np.argsort(prob)[::-1][np.linspace(64, prob.size - 1, 64).astype(int)]
    idx = np.concatenate([top, spread])
    return {"instance": i, "modes": [int(v) for v in idx], "prob": [float(prob[v]) for v in idx],
            "norm": float(O.inner(psi, psi, g).real), "max_prob": float(prob.max()),
            "seconds": time.time() - t0}


def whole_spectrum(i, floor=1e-24):
    """Every C-spectrum entry of instance i with |C|^2 >= floor * max, and the instance's norm."""
    d = W.schwinger_batched()[i]
    g = OA.grid(d)
    t0 = time.time()
    psi = O.march_scattered(OA.field(d), g, OA.background(d, 0), d["t_in"], d["t_out"], d["n_steps"])
    C = O.c_spectrum(psi, g, d["t_in"])
    prob = np.transpose(np.abs(C) ** 2, (0, 3, 2, 1)).ravel()  # library layout [r][z][y][x]
    keep = np.nonzero(prob >= floor * prob.max())[0]
    out = {"citation": "oracle/swf_oracle.py on paper_2512_16889_gb300.workloads.schwinger_batched()",
           "instance": i, "floor": floor, "size": int(prob.size), "max_prob": float(prob.max()),
           "modes": [int(v) for v in keep], "prob": [float(prob[v]) for v in keep],
           "norm": float(O.inner(psi, psi, g).real), "seconds": time.time() - t0}
    name = f"schwinger_batched_spectrum_{i}.json"
    json.dump(out, open(os.path.join(os.path.dirname(OUT), name), "w"))


def single_fp64():
    """Full N of the single FP64 Schwinger workload for both positron spins."""
    d0 = W.schwinger_fp64_single()[0]
    g = OA.grid(d0)
    t0 = time.time()
    pu = O.march_scattered(OA.field(d0), g, OA.background(d0, 0), d0["t_in"], d0["t_out"], d0["n_steps"])
    C = O.c_spectrum(pu, g, d0["t_in"])
    prob = np.transpose(np.abs(C) ** 2, (0, 3, 2, 1)).ravel()
    top = np.argsort(prob)[::-1][:64]
    out = {"citation": "oracle/swf_oracle.py on paper_2512_16889_gb300.workloads.schwinger_fp64_single()",
           "spectrum_modes": [int(v) for v in top], "spectrum_prob": [float(prob[v]) for v in top],
           "norm_u": float(O.inner(pu, pu, g).real), "pairs": []}
    for r in (1, -1):
        d = dict(d0, r=r)
        bv = OA.background(d, 1)
        pv = O.march_scattered(OA.field(d), g, bv, d["t_in"], d["t_out"], d["n_steps"])
        ref = O.pair_number(pu, pv, g, d["t_in"], d["p"], d["s"], d["q"], d["r"], OA.background(d, 0).offset(),
                            bv.offset())
        out["pairs"].append({"r": r, **{k: [ref[k].real, ref[k].imag] for k in ("C", "D", "A", "B")},
                             "N_line1": float(ref["N_line1"]), "N_line2": float(ref["N_line2"]),
                             "norm_v": float(O.inner(pv, pv, g).real)})
    out["seconds"] = time.time() - t0
    json.dump(out, open(os.path.join(os.path.dirname(OUT), "schwinger_fp64_single.json"), "w"), indent=1)


def bw_sample(form=1):
    """Amplitude terms of the first 192^2 instance of the Breit-Wheeler uneven-grid workload."""
    ds = W.bw_uneven()
    i = next(j for j, d in enumerate(ds) if d["n"][0] == 192)
    d = ds[i]
    g = OA.grid(d)
    t0 = time.time()
    ph = O.Photon(tuple(d["k"]), tuple(d["eps"]))
    ref = O.bw_amplitude(OA.field(d), g, d["p"], d["s"], d["q"], d["r"], ph, d["t_in"], d["t_out"], d["n_steps"],
                         form=form)
    name = "bw_uneven_sample.json" if form == 1 else "bw_uneven_partial_sample.json"
    out = {"citation": "oracle/swf_oracle.py on paper_2512_16889_gb300.workloads.bw_uneven()"
                       + ("" if form == 1 else ", partial-integration form (Sec. IV, Eqs. 30-33)"),
           "instance": i, "n": list(d["n"]), "n_steps": d["n_steps"],
           "terms": [[complex(v).real, complex(v).imag] for v in ref["terms"]], "M": [ref["M"].real, ref["M"].imag],
           "norm_u": float(O.inner(ref["psi_u"], ref["psi_u"], g).real),
           "norm_v": float(O.inner(ref["psi_v"], ref["psi_v"], g).real), "seconds": time.time() - t0}
    json.dump(out, open(os.path.join(os.path.dirname(OUT), name), "w"), indent=1)


if __name__ == "__main__":
    if sys.argv[1:] == ["--single"]:
        single_fp64()
        sys.exit(0)
    if sys.argv[1:2] == ["--spectrum"]:
        whole_spectrum(int(sys.argv[2]))
        sys.exit(0)
    if sys.argv[1:] == ["--bw"]:
        bw_sample()
        sys.exit(0)
    if sys.argv[1:] == ["--bw-partial"]:
        bw_sample(form=2)
        sys.exit(0)
    which = [int(v) for v in sys.argv[1:]] or [0, 77]
    data = {"citation": "oracle/swf_oracle.py on paper_2512_16889_gb300.workloads.schwinger_batched()",
            "samples": []}
    if os.path.exists(OUT):
        data = json.load(open(OUT))
    have = {s["instance"] for s in data["samples"]}
    for i in which:
        if i in have:
            continue
        data["samples"].append(sample(i))
        json.dump(data, open(OUT, "w"), indent=1)
        print("instance", i, "done", flush=True)
