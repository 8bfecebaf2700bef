"""Writes oracle-only reference samples for the full-size batched Schwinger workload.

Runs the FP64 oracle (no CUDA involved) on selected instances of the 256^2, 128-instance,
1000-step workload and stores, per instance, the C-spectrum |C(m,(r,q))|^2 at the 64 largest
modes, 64 modes spread over the spectrum, and ||psi_scat(t_in)||^2.  The GPU test compares the
benchmark's own solve against these values.

    python tests/golden/make_full_size_reference.py [instance ...]
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


if __name__ == "__main__":
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
