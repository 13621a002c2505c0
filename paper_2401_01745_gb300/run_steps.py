"""Run a fixed number of emRKC steps on a named synthetic workload.

    python -m paper_2401_01745_gb300.run_steps --workload slab201x71x101_ttp \
        --precision mixed --steps 6 --rho-every 0

Used for profiler captures (one short, deterministic sequence of launches)
and as a minimal example of the Python binding.
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import paper_2401_01745_gb300 as pkg
    from workloads import make_workload

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="slab_ttp")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--rho-every", type=int, default=0)
    ap.add_argument("--h", type=float, default=None, help="mesh size for parametrised workload names")
    ap.add_argument("--method", default="emrkc", choices=["emrkc", "exex", "imex", "mrkc"])
    ap.add_argument("--dt", type=float, default=None)
    ap.add_argument("--rho-s-min", type=float, default=0.0, help="lower bound on rho_S (known stiffness, Sec. 3.1)")
    a = ap.parse_args(argv)
    pkg.build()
    kw = {} if a.h is None else {"h": a.h}
    w = make_workload(a.workload, **kw)
    prec = pkg.PREC_MIXED if a.precision == "mixed" else pkg.PREC_FP64
    method = {"emrkc": pkg.METHOD_EMRKC, "exex": pkg.METHOD_EXEX_RL, "imex": pkg.METHOD_IMEX_RL,
              "mrkc": pkg.METHOD_MRKC}[a.method]
    dt = w.dt if a.dt is None else a.dt
    sol = pkg.Solver.from_workload(w, precision=prec, rho_every=a.rho_every, method=method, rho_S_min=a.rho_s_min)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        sol.step(dt)
    sol.sync()
    el = time.perf_counter() - t0
    st = sol.stats()
    V = sol.get_state(var=0)
    sol.close()
    print(json.dumps({"workload": a.workload, "nodes": w.n, "precision": a.precision, "method": a.method,
                      "steps": a.steps,
                      "s": st["s"], "m": st["m"], "launches": st["launches"], "wall_s": el,
                      "V_min": float(V.min()), "V_max": float(V.max())}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
