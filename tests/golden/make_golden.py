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


def _quench_member(args):
    """One member of a perturbed-oracle ensemble of the quench (see
    quench_spread): <sigma_x> of sites A and B after every step."""
    D, kind, member, steps = args
    gates2, gate1 = I.tfim_real_time_gates(2.5, 0.01)
    A, B = I.quench_start(D)
    if kind == "fp64":
        # rounding-level perturbation of the start, FP64 tolerance grid
        rng = np.random.default_rng(1000 + member)
        A = A + 1e-14 * I.random_site_tensor(rng, 2, D)
        B = B + 1e-14 * I.random_site_tensor(rng, 2, D)
        cfg = O.Config(D=D, r=2, sweeps=10)
    else:
        # the split-BF16 environment: every operand of the metric contraction
        # carried to a 16-bit significand (one hi + lo pair of BF16 values),
        # modelled as independent per-element relative errors of 2^-17; the
        # mixed contexts' tolerance grid 1e-4..1e-8
        rng = np.random.default_rng(5000 + member)
        orig = O.metric_raw

        def pert(x):
            z = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
            return x * (1 + 2.0 ** -17 * z / np.sqrt(2))

        def noisy(Ta, Tb, QA, QB, d_p, D_):
            return orig(pert(Ta), pert(Tb), pert(QA), pert(QB), d_p, D_)

        O.metric_raw = noisy
        cfg = O.Config(D=D, r=2, sweeps=10, tau_exponents=tuple(range(4, 9)))
    out = []
    try:
        for _ in range(steps):
            A, B, _ = O.ntu_step(A, B, gates2, gate1, cfg)
            out.append([O.measure(A, B, 0, I.pauli("X"), 1).real,
                        O.measure(A, B, 1, I.pauli("X"), 1).real])
    finally:
        if kind != "fp64":
            O.metric_raw = orig
    return out


def quench_spread(D, ref, steps=200, members=(4, 8)):
    """How far the oracle's own <sigma_x> moves from the stored quench
    trajectory `ref` when its inputs are perturbed at the level of each GPU
    path's arithmetic: "fp64", 1e-14 relative perturbations of the start
    (members[0] members); "split16", the environment operands perturbed by
    2^-17 per element at every bond update with the mixed tolerance grid
    (members[1] members).  Returns, per kind, the member trajectories and
    the per-step largest deviation over members and both sites."""
    import multiprocessing as mp
    jobs = [(D, "fp64", m, steps) for m in range(members[0])] + \
           [(D, "split16", m, steps) for m in range(members[1])]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = pool.map(_quench_member, jobs)
    center = np.array([ref["sx_A"], ref["sx_B"]]).T
    out = {}
    for kind, n0 in (("fp64", 0), ("split16", members[0])):
        k = members[0] if kind == "fp64" else members[1]
        tr = np.array(res[n0:n0 + k])
        out[f"spread_{kind}"] = np.abs(tr - center[None]).max(axis=(0, 2)).tolist()
        out[f"members_{kind}_first12"] = tr[:, :12].tolist()
    out["spread_recipe"] = (
        "fp64: start + 1e-14 x random_site_tensor(default_rng(1000 + m)), tau 1e-4..1e-15; "
        "split16: every operand of the metric contraction (Ta, Tb, QA, QB) times "
        "(1 + 2^-17 z / sqrt 2), z complex N(0,1) from default_rng(5000 + m), tau 1e-4..1e-8; "
        "spread = max over members and sites of |<sigma_x> - stored trajectory|")
    return out


def write(name, obj):
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(obj, f, indent=1)
    print("wrote", os.path.join(HERE, name))


if __name__ == "__main__":
    write("one_step_d3.json", one_step_d3())
    for D in (4, 5):
        q = quench(D)
        q.update(quench_spread(D, q))
        write(f"quench_d{D}.json", q)
    write("purification_d4.json", purification(4))
