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


def quench(D, steps=200):
    """TFIM quench h=2.5, dt=0.01 to t=2 (Sec. III): the start of
    inputs.quench_start(D) (|+x> zero-padded to D plus the seeded 1e-2
    admixture), second-order Trotter steps, 10 ALS sweeps, FP64; <sigma_x>
    of sites A and B after every step (cluster estimator)."""
    gates2, gate1 = I.tfim_real_time_gates(2.5, 0.01)
    cfg = O.Config(D=D, r=2, sweeps=10)
    A, B = I.quench_start(D)
    xa, xb = [], []
    for _ in range(steps):
        A, B, _ = O.ntu_step(A, B, gates2, gate1, cfg)
        xa.append(O.measure(A, B, 0, I.pauli("X"), 1).real)
        xb.append(O.measure(A, B, 1, I.pauli("X"), 1).real)
    return {"workload": f"TFIM quench h=2.5 dt=0.01, {steps} steps, D={D}, quench_start({D}), "
                        "10 sweeps, FP64 oracle", "D": D, "dt": 0.01, "h": 2.5,
            "sx_A": xa, "sx_B": xb}


def purification(D, steps=100):
    """Thermal state by purification, h = 2.5, d_anc = 2: (|00>+|11>)/sqrt(2) per
    site zero-padded to D plus a seeded 1e-2 admixture (seed 77, both sites
    from one generator, each normalised), imaginary-time gates of h=2.5 with
    dbeta=0.005 to beta=0.5 on the physical index, 10 ALS sweeps, FP64;
    <sigma_x>, <sigma_z> of site A after every step."""
    rng = np.random.default_rng(77)
    A = I.purification_state(D) + 1e-2 * I.random_site_tensor(rng, 4, D)
    B = I.purification_state(D) + 1e-2 * I.random_site_tensor(rng, 4, D)
    A, B = A / np.linalg.norm(A), B / np.linalg.norm(B)
    gates2, gate1 = I.tfim_imag_time_gates(2.5, 0.005)
    cfg = O.Config(D=D, r=2, d_anc=2, sweeps=10)
    sx, sz = [], []
    for _ in range(steps):
        A, B, _ = O.ntu_step(A, B, gates2, gate1, cfg)
        sx.append(O.measure(A, B, 0, I.pauli("X"), 2).real)
        sz.append(O.measure(A, B, 0, I.pauli("Z"), 2).real)
    return {"workload": f"purification h=2.5 dbeta=0.005, {steps} steps, D={D}, seed 77 "
                        "admixture 1e-2, 10 sweeps, FP64 oracle", "D": D, "dbeta": 0.005,
            "h": 2.5, "sx_A": sx, "sz_A": sz}


def write(name, obj):
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(obj, f, indent=1)
    print("wrote", os.path.join(HERE, name))


if __name__ == "__main__":
    write("one_step_d3.json", one_step_d3())
    for D in (4, 5):
        write(f"quench_d{D}.json", quench(D))
    write("purification_d4.json", purification(4))
