"""Writes cg_iterations_<workload>_<precond>.json: the CG iterations per Poisson solve that
the FP64 oracle itself takes on one of the single-run workloads (two RK4 start-up steps,
then AB3), with the given preconditioner:

    shear512_n4    512 x 512 cells, n = 4, double shear layer rho = delta = 0.05, D = 1e-4,
                   dt = 5e-4, CG tol 1e-10
    random1024_n5  1024 x 1024 cells, n = 5, random-phase field (seed 1), D = 0, dt = 2e-4,
                   CG tol 1e-10

Calls only oracle/ and the input generator.  Used to scale the bounded CPU-baseline sample of
bench.py (oracle RHS + a few CG iterations) to one full time step.

    python tests/golden/make_cg_iterations.py [workload] [nsteps] [jacobi|twolevel]
        (shear512_n4, twolevel: about half an hour of CPU; random1024_n5: a few hours)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle.solver as S  # noqa: E402
import oracle.stepper as ST  # noqa: E402
from oracle.operators import Operators  # noqa: E402
from oracle.tables import Grid  # noqa: E402
from paper_1311_7477_gb300 import fields  # noqa: E402


WORKLOADS = {
    "shear512_n4": (512, 4, 1e-4, 5e-4, 1e-10, "shear layer 512x512 cells, n=4, D=1e-4, dt=5e-4, CG tol 1e-10"),
    "random1024_n5": (1024, 5, 0.0, 2e-4, 1e-10,
                      "random phase (seed 1) 1024x1024 cells, n=5, D=0, dt=2e-4, CG tol 1e-10"),
}


def main(workload="shear512_n4", nsteps=4, precond="twolevel"):
    N, n, D, dt, tol, what = WORKLOADS[workload]
    g = Grid(N, N, n)
    ops = Operators(g)
    X, Y = g.mesh()
    w0 = fields.shear_layer(X, Y) if workload.startswith("shear") else fields.random_phase(X, Y, seed=1)
    log = []
    orig = S.solve_poisson

    def logged(ops_, omega, x0, tol_, maxit, fixed_iters=0, pc=None):
        t0 = time.time()
        res = orig(ops_, omega, x0, tol_, maxit, fixed_iters, pc)
        log.append({"iters": res.iters, "relres": res.relres, "seconds": time.time() - t0})
        print("solve", len(log), res.iters, "%.1fs" % log[-1]["seconds"], flush=True)
        return res

    ST.solve_poisson = logged
    sim = ST.Simulation(ops, w0, D, dt, tol=tol, maxit=200000, K=3, precond=precond)
    per_step = []
    for k in range(nsteps):
        before = len(log)
        t0 = time.time()
        sim.step(1)
        per_step.append({"step": k, "kind": "rk4" if k < 2 else "ab3",
                         "solves": log[before:], "seconds": time.time() - t0})
    out = {
        "workload": what + " (FP64 oracle)",
        "preconditioner": precond,
        "initial_solve": log[0],
        "steps": per_step,
        "ab3_iters_mean": float(np.mean([s["solves"][0]["iters"] for s in per_step if s["kind"] == "ab3"]))
        if nsteps > 2 else None,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "cg_iterations_%s_%s.json" % (workload, precond))
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "shear512_n4", int(sys.argv[2]) if len(sys.argv) > 2 else 4,
         sys.argv[3] if len(sys.argv) > 3 else "twolevel")
