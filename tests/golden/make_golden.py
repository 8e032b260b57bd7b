"""Write the stored expected values under tests/golden/.

Calls only the CPU oracle (and the seeded input generators); nothing here
comes from the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ntu_oracle as O  # noqa: E402
from paper_2107_06635_gb300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def one_step_d3():
    """One NTU Trotter step of the 2-site cell: D=3, d=2, iid complex N(0,1)
    site tensors from seed 1 normalised, gate exp(-i 0.01 ZZ) split at r=2,
    10 ALS sweeps, FP64."""
    A, B = I.random_pair(1, 2, 3)
    cfg = O.Config(D=3, r=2, sweeps=10)
    G = I.zz_gate(0.01)
    out = {"workload": "one NTU step, D=3 d=2 r=2, seed 1, exp(-i 0.01 ZZ), 10 sweeps",
           "bonds": []}
    for b in range(4):
        A, B, info = O.update_bond(A, B, b, G, cfg, keep=True)
        out["bonds"].append({"bond": b, "delta": info.delta, "eps": info.eps,
                             "eps0": info.eps0, "tau": info.tau,
                             "g_trace_log": info.diag[2],
                             "g_frob": float(np.linalg.norm(info.g))})
    out["A_after"] = [A.real.reshape(-1).tolist(), A.imag.reshape(-1).tolist()]
    out["B_after"] = [B.real.reshape(-1).tolist(), B.imag.reshape(-1).tolist()]
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "one_step_d3.json"), "w") as f:
        json.dump(one_step_d3(), f, indent=1)
    print("wrote", os.path.join(HERE, "one_step_d3.json"))
