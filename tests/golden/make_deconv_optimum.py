"""Writes deconv_large_optimum.json: the FP64 optimum of the large 1-D
nonnegative deconvolution (n = 1e6, Gaussian kernel L = 1000, sigma = 100,
1% support, noise 0.01, seed base + 2) from the oracle's exact NNLS solver
(oracle/nnls_conv.py), with its duality bracket and its support.

The cone form's optimal value is t* = sqrt(2 f*), f* the NNLS optimum of
1/2 ||k * x - b_obs||^2 over x >= 0 (Section 5.3's problem).  Calls only the
oracle and the seeded input generator.

    python tests/golden/make_deconv_optimum.py      # ~10 min on 8 cores
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import nnls_conv  # noqa: E402
from paper_1609_03488_b300 import synth  # noqa: E402

INSTANCE = dict(n_x=1_000_000, L=1000, sigma=100.0, support=0.01, noise=0.01, seed=synth.BASE_SEED + 2)


def fingerprint(prob):
    k = np.asarray(prob["meta"]["kernel"], dtype=np.float64)
    b = np.asarray(prob["meta"]["b_obs"], dtype=np.float64)
    return {"kernel_sum": float(k.sum()), "kernel_sq": float(k @ k),
            "b_obs_sum": float(b.sum()), "b_obs_sq": float(b @ b),
            "b_obs_first": float(b[0]), "b_obs_last": float(b[-1])}


def main():
    prob = synth.deconv(**INSTANCE)
    t0 = time.time()
    x, info = nnls_conv.nnls_conv(prob["meta"]["kernel"], prob["meta"]["b_obs"], INSTANCE["n_x"],
                                  rel_gap=1e-13, workers=os.cpu_count())
    el = time.time() - t0
    out = {
        "_what": ("FP64 optimum of the large nonnegative deconvolution cone program: t* = sqrt(2 f*), "
                  "f* = min_{x>=0} 1/2 ||k * x - b_obs||^2 (Section 5.3's problem), from the exact "
                  "active-set NNLS of oracle/nnls_conv.py; [t_lo, t_hi] is its Lagrangian-duality bracket"),
        "_written_by": "tests/golden/make_deconv_optimum.py (oracle and input generator only)",
        "instance": INSTANCE, "fingerprint": fingerprint(prob),
        "f": info["f"], "dual": info["dual"], "t_lo": info["t_lo"], "t_hi": info["t_hi"],
        "kkt_inf": info["kkt_inf"], "outer_steps": info["outer"], "inner_steps": info["inner"],
        "seconds": round(el, 1), "support_size": info["support"],
        "support": [int(i) for i in np.flatnonzero(x)],
    }
    with open(os.path.join(HERE, "deconv_large_optimum.json"), "w") as fh:
        json.dump(out, fh, indent=0)
    print({k: v for k, v in out.items() if k != "support"})


if __name__ == "__main__":
    main()
