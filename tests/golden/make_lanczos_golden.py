"""Write the oracle's FP64 Lanczos result for the 4x4 Hubbard workload.

Calls only the CPU oracle (oracle/) and the seeded input generators
(workloads/): the start vector is the Philox Gaussian stream of the workload's
seed, the Hamiltonian its term list (t = 1, U = 8, periodic 4x4 square, half
filling, 165,636,900 states).  The run is the oracle's textbook three-term
Lanczos in FP64 with the stopping rule of the library (residual estimate
<= tol * max(1, |theta|)); it takes a few hours on eight cores.  The paper's
ground-state method is Lanczos (Sec. 1, Table 1); no exact value is known at
this size, so this run is the reference the GPU energies are compared with.

Usage: python tests/golden/make_lanczos_golden.py [out.json]
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from workloads import configs, random_vectors  # noqa: E402


def main(out: str) -> None:
    c = configs.hubbard_square4x4()
    m = O.Model(c["model"], c["n_sites"], c["n_up"], c["n_dn"], c["terms"], use_lists=True)
    t0 = time.time()
    v0 = np.ascontiguousarray(random_vectors(m.dim, 1, c["seed"], normalize=False)[:, 0])
    r = m.lanczos(v0, c["max_steps"], c["tol"])
    rec = dict(
        workload=c["name"], dim=m.dim, seed=c["seed"], start_vector="philox gaussian, unnormalised",
        max_steps=c["max_steps"], tol=c["tol"], status=int(r["status"]), steps=int(r["steps"]),
        e0=float(r["e0"]), resid=float(r["resid"]), alpha=[float(a) for a in r["alpha"]],
        beta=[float(b) for b in r["beta"]], oracle_threads=O.num_threads(),
        seconds=round(time.time() - t0, 1),
        source="oracle orc_lanczos (FP64 three-term recurrence, Sturm bisection)",
    )
    with open(out, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(f"E0 = {rec['e0']:.15f} after {rec['steps']} steps (status {rec['status']}), {rec['seconds']} s")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(HERE, "lanczos_hubbard4x4_U8.json"))
