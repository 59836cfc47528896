"""Writes paper_scale_181x61_roots.npz: the FP64 oracle's converged surface
elevation zeta at the 181x61 paper-scale configurations (F = 0.7 and 1.5, the
Gaussian bump of amplitude 0.2; Sec. 3.1 discretisation, Sec. 3.2 solver).

It calls only oracle/: the oracle's JFNK with the banded linear Jacobian of
App. A in block storage (half band 3) as preconditioner, from the uniform
stream, to |F|_inf <= 1e-11 -- well below the 1e-8 the GPU tests solve to, so
the stored zeta is the discrete root to within its own rounding.

    python tests/golden/make_paper_scale_roots.py      (several minutes on CPU)
"""
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1709_08803_gb300 import workloads as W  # noqa: E402

TOL = 1e-11
HALF_BAND = 3


def main():
    out, meta = {}, {}
    for F in (0.7, 1.5):
        mesh, topo, Fv = W.config_paper_scale(F)
        P = O.problem(mesh, Fv)
        t0 = time.time()
        u, st = O.jfnk(P, topo, W.flat_guess(mesh), half_band=HALF_BAND, banded=True, tol=TOL,
                       max_newton=40, restart=50, max_krylov=800, eta=1e-4)
        dt = time.time() - t0
        if st["status"] != 0:
            raise SystemExit(f"oracle JFNK did not converge at F = {F}: {st}")
        key = f"F{F:g}".replace(".", "p")
        out[f"zeta_{key}"] = O.nodal_values(P, u)["zeta"].reshape(mesh.M, mesh.N)
        meta[key] = dict(st, seconds=round(dt, 1), F=F, N=mesh.N, M=mesh.M, x1=mesh.x1, y1=mesh.y1,
                         dx=mesh.dx, dy=mesh.dy)
        print(key, meta[key], flush=True)
    meta["how"] = ("oracle.jfnk(banded=True, half_band=3, tol=1e-11, eta=1e-4, restart=50) from the "
                   "uniform stream; zeta at the nodes, shape (M, N)")
    meta["threads"] = O.num_threads()
    meta["host"] = platform.machine()
    np.savez_compressed(os.path.join(HERE, "paper_scale_181x61_roots.npz"), meta=json.dumps(meta), **out)


if __name__ == "__main__":
    main()
