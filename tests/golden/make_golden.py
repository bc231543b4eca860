"""Write the oracle's integer outputs for the single n=4096 test signal.

Calls only ``oracle/`` (the FP64 CPU oracle, both tiers) and the seeded input
generator.  Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1802_01359_gb300 import signals  # noqa: E402


def main():
    s = signals.single_4096().astype(np.float64)
    out = {"source": "oracle tiers A and B (FP64), signals.single_4096(), nu=1.6, mask_scale=1, "
                     "delta=1e-3, max_inner=200, max_imfs=10"}
    for name, fn in (("iterative", oracle.iterative), ("direct", oracle.direct)):
        r = fn(s)
        out[name] = {"n_imfs": r["n_imfs"], "status": r["status"], "m": r["m"].tolist(),
                     "L": r["L"].tolist(), "kext": r["kext"].tolist(),
                     "imf_l2": [float(np.linalg.norm(x)) for x in r["imfs"]],
                     "remainder_l2": float(np.linalg.norm(r["remainder"]))}
    r = oracle.direct(s, mask_scale=2)
    out["direct_mask_scale_2"] = {"n_imfs": r["n_imfs"], "status": r["status"], "m": r["m"].tolist(),
                                  "L": r["L"].tolist(), "kext": r["kext"].tolist()}
    # the method's options, direct tier: a-priori N0 (Theorem 5, absolute delta), thresholded
    # IMF (eq. I_gamma), Fourier-peak mask length (end of Sec. 2), shape window (Theorem 4)
    modes = {"apriori_delta2": dict(apriori=True, delta=2.0, max_inner=1 << 16),
             "threshold_gamma0.05": dict(gamma=0.05),
             "peak_mask": dict(peak_mask=True),
             "shape_sine33": dict(shape=np.sin(np.pi * np.linspace(0.0, 1.0, 33)))}
    for name, kw in modes.items():
        r = oracle.direct(s, **kw)
        out["direct_" + name] = {"n_imfs": r["n_imfs"], "status": r["status"], "m": r["m"].tolist(),
                                 "L": r["L"].tolist(), "kext": r["kext"].tolist(),
                                 "imf_l2": [float(np.linalg.norm(x)) for x in r["imfs"]]}
    with open(os.path.join(HERE, "single_4096_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
