"""Writes the stored expected values of the GPU tests by calling only oracle/.

lattice64_history.json: the 64 x 64 lattice of the paper's kind (Sec. 3.1;
bottom row clamped, EA = 1, loads Uniform(-1, 1) from seeds 0-3), 4 x 4 sets
of 16 x 16 nodes, stopped at R1 < 1e-8 (Eq. 19): per seed the number of
upper-level updates and the (R1, R2, Pi) history of the oracle's iteration.

lattice1024_lognormal_history.json (with --full, about 40 minutes of CPU):
the 1024 x 1024 lattice with lognormal(0, 0.3) EA, 16 x 16 sets of 64 x 64
nodes, loads from seed 0, run to R1 < 1e-10: the history, the update counts
at which R1 first drops below 1e-8 and 1e-10, and the displacement at 2000
seeded DOFs after updates 1, 2, 3, 10, 100 and at the end.

Run:  python tests/golden/make_golden.py [--full]
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import hms, truss  # noqa: E402
from workloads import CASES  # noqa: E402


def main():
    c = CASES["lattice64_fp64"]
    tr = truss.Truss(c.nx, c.ny)
    g = hms.SetGrid(c.nx, c.ny, c.sx, c.sy)
    lf = hms.LocalFactors(tr, g)
    out = {"case": c.name, "nx": c.nx, "ny": c.ny, "sx": c.sx, "sy": c.sy, "tol": c.tol, "seeds": {}}
    for seed in range(4):
        from workloads import loads
        p = loads(c.nx, c.ny, seed).reshape(-1)
        res = hms.solve(tr, g, p, c.tol, 1000, factors=lf)
        out["seeds"][str(seed)] = {
            "iterations": res.iterations,
            "history": [[h["R1"], h["R2"], h["Pi"]] for h in res.history],
        }
    with open(os.path.join(HERE, "lattice64_history.json"), "w") as f:
        json.dump(out, f, indent=1)


def main_full():
    import numpy as np
    c = CASES["lattice1024_lognormal_fp64"]
    tr = truss.Truss(c.nx, c.ny, c.ea_array())
    g = hms.SetGrid(c.nx, c.ny, c.sx, c.sy)
    lf = hms.LocalFactors(tr, g)
    p = c.load_array().reshape(-1)
    idx = np.sort(np.random.default_rng(2024).choice(tr.ndof, 2000, replace=False))
    keep = (1, 2, 3, 10, 100)
    samples = {}
    free = tr.free
    pf = free * p
    u = np.zeros(tr.ndof)
    hist = []
    t = 0
    while True:
        r = tr.residual(pf, u)
        R1 = np.abs(r).sum() / np.abs(pf).sum()
        hist.append([R1, np.sqrt(r @ r) / np.sqrt(pf @ pf), -0.5 * (u @ (pf + r))])
        if R1 < 1e-10 or t >= 3000:
            break
        V = hms.modes(tr, g, lf.relax(r))
        Kaa, P = hms.coarse_system(tr, V, r)
        a, _ = hms.coarse_solve(Kaa, P)
        u = u + V @ a
        t += 1
        if t in keep:
            samples[str(t)] = u[idx].tolist()
        if t % 20 == 0:
            print(t, R1, flush=True)
    samples["final"] = u[idx].tolist()
    R1s = [h[0] for h in hist]
    out = {"case": c.name, "nx": c.nx, "ny": c.ny, "sx": c.sx, "sy": c.sy, "seed": c.seed,
           "ea_seed": c.seed + 1000, "iterations": t,
           "first_below_1e-8": next(k for k, v in enumerate(R1s) if v < 1e-8),
           "first_below_1e-10": next((k for k, v in enumerate(R1s) if v < 1e-10), None),
           "history": hist, "sample_dofs": idx.tolist(), "samples": samples}
    with open(os.path.join(HERE, "lattice1024_lognormal_history.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    if "--full" in sys.argv:
        main_full()
    else:
        main()
