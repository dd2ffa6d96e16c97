"""Writes steel_plate_L10.json: scalars of the Galerkin solution u_h of the 2D steel plate on
2^10 x 2^10 nodes (E = 210 GPa, nu = 0.3, plane strain, clamped -x edge, gravity rho = 7850 plus
a downward traction of 1 MN/m^2 on +x), computed by the CPU oracle only (element-loop assembly
of A_bc, f_bc and V-cycle preconditioned CG; Section 3, Eq. femsys; Section 5.3).

Stored (steel_plate_L<levels>.json):
  uAu      = f_bc^T u_h (= u_h^T A_bc u_h, the squared energy norm of u_h)
  f_norm   = ||f_bc||_2
  samples  = u_h at 64 seeded nodes (node index (i, j), both components)
and (steel_plate_L<levels>_uh_qtt.npz) u_h itself as a QTT train in the layout of Section 4
(component core, then one core per level), from the oracle's TT-SVD at relative accuracy 1e-13;
its own energy-norm distance to u_h is stored as qtt_energy_err.  A solution train u is then
compared by the energy norm of the explicitly formed difference u - u_h (no cancellation).

Run from the repository root:  python tests/golden/make_steel_plate_golden.py [levels]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fem, tt  # noqa: E402
from paper_2501_12151_gb300 import workloads as W  # noqa: E402


def main(levels: int = 10):
    pr = W.steel_plate_2d(levels=levels)
    t0 = time.perf_counter()
    Abc, f = fem.system(pr.grid, pr.material, pr.loads)
    u, info = fem.solve_mg(pr.grid, Abc, f)
    n = pr.grid.n
    nodes = W.rng(2025).integers(0, n, size=(64, 2))
    U = u.reshape(2, n, n)
    cores = tt.tt_svd(tt.to_qtt_order(u, 2, levels), [2] + [4] * levels, eps=1e-13)
    uq = tt.to_natural_order(tt.tt_full(cores), 2, levels)
    qtt_err = fem.energy_norm(Abc, uq - u) / fem.energy_norm(Abc, u)
    out = {
        "what": "Galerkin solution u_h of the 2D steel plate (oracle A: element loop + V-cycle CG)",
        "levels": levels,
        "dofs": int(u.size),
        "uAu": float(f @ u),
        "uAu_direct": float(u @ (Abc @ u)),
        "f_norm": float(np.linalg.norm(f)),
        "cg_iters": info["iters"],
        "rel_residual": info["rel_residual"],
        "sample_nodes": nodes.tolist(),
        "sample_u": [[float(U[0, i, j]), float(U[1, i, j])] for i, j in nodes],
        "qtt_ranks": tt.ranks(cores),
        "qtt_energy_err": qtt_err,
        "seconds": time.perf_counter() - t0,
        "written_by": "tests/golden/make_steel_plate_golden.py",
    }
    here = os.path.dirname(os.path.abspath(__file__))
    np.savez_compressed(os.path.join(here, f"steel_plate_L{levels}_uh_qtt.npz"),
                        **{f"core{k}": c for k, c in enumerate(cores)})
    path = os.path.join(here, f"steel_plate_L{levels}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path, out["uAu"], out["cg_iters"], out["rel_residual"], f"{out['seconds']:.1f} s")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 10)
