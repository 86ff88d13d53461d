"""Write the oracle's FP64 Lanczos results for the full-size workloads.

Calls only the CPU oracle (oracle/) and the seeded input generators
(workloads/): the start vector is the Philox Gaussian stream of the workload's
seed, the Hamiltonian its term list.  The run is the oracle's textbook
three-term Lanczos in FP64 (the paper's ground-state method, Sec. 1 and
Table 1).

  hubbard4x4 (default): t = 1, U = 8, periodic 4x4 square, half filling,
    165,636,900 states, to the library's stopping rule (residual estimate
    <= tol * max(1, |theta|)); a few hours on eight cores.  No exact value is
    known at this size, so this run is the reference the GPU energies are
    compared with.
  square4x8: the Heisenberg model on the 4x8 periodic square, S^z = 0,
    601,080,390 states, exactly 20 steps from the seed-2 start vector (the
    benchmark's timed Lanczos steps): every alpha, beta and the lowest Ritz
    value after 20 steps.

Usage: python tests/golden/make_lanczos_golden.py [hubbard4x4|square4x8] [out.json]
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


def main(which: str, out: str) -> None:
    if which == "hubbard4x4":
        c = configs.hubbard_square4x4()
        m = O.Model(c["model"], c["n_sites"], c["n_up"], c["n_dn"], c["terms"], use_lists=True)
        max_steps, tol = c["max_steps"], c["tol"]
    elif which == "square4x8":
        c = configs.heisenberg_square4x8()
        m = O.Model(c["model"], c["n_sites"], c["n_up"], c["n_dn"], c["terms"])
        max_steps, tol = 20, 0.0
    else:
        raise SystemExit(f"unknown workload {which}")
    t0 = time.time()
    v0 = np.ascontiguousarray(random_vectors(m.dim, 1, c["seed"], normalize=False)[:, 0])
    r = m.lanczos(v0, max_steps, tol)
    rec = dict(
        workload=c["name"], dim=m.dim, seed=c["seed"], start_vector="philox gaussian, unnormalised",
        max_steps=max_steps, tol=tol, status=int(r["status"]), steps=int(r["steps"]),
        e0=float(r["e0"]), resid=float(r["resid"]), alpha=[float(a) for a in r["alpha"]],
        beta=[float(b) for b in r["beta"]], oracle_threads=O.num_threads(),
        seconds=round(time.time() - t0, 1),
        source="oracle orc_lanczos (FP64 three-term recurrence, Sturm bisection)",
    )
    with open(out, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(f"E0 = {rec['e0']:.15f} after {rec['steps']} steps (status {rec['status']}), {rec['seconds']} s")


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "hubbard4x4"
    name = {"hubbard4x4": "lanczos_hubbard4x4_U8.json", "square4x8": "lanczos_square4x8_20steps.json"}.get(which, "x.json")
    main(which, sys.argv[2] if len(sys.argv) > 2 else os.path.join(HERE, name))
