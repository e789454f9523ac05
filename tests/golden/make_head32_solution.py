"""Writes head32_ring4_solution.npz: the oracle's converged solution maps of the 32^3 head phantom.

Workload: the head phantom generator of the 64^3 benchmark on a 32^3 grid of 6 mm voxels
(192 mm box), 298 MHz, four z-directed unit dipoles on the 15 cm ring (z = 0).  The oracle
solves each right-hand side with its own FP64 GMRES (restart 100) on P^-1 A x = P^-1 b
(Section IV-B) to a preconditioned relative residual of 1e-11, then takes the PWL field
coefficients e = G^-1 (e_inc + (N - G) x / c_e) and the absorbed-power density (Section IV-C,
Eq. 44).

Stored (tissue voxels only, in C order of (z, y, x)): the voxel-average (l = 1) field
coefficients of the three components, complex64 [R][3][n_tissue]; the absorbed-power density,
float32 [R][n_tissue]; the total absorbed power, float64 [R]; and the oracle's final residual
per right-hand side.  Single precision storage carries a relative rounding of 6e-8, well below
the 1e-6 comparison it serves.

Only the oracle and the seeded input generators are called here.  Run from the repository
root: `python tests/golden/make_head32_solution.py` (about ten minutes on eight cores).
"""

import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "head32_ring4_solution.npz")
N, FREQ, R, TOL = 32, 298e6, 4, 1e-11


def problem():
    sys.path.insert(0, ROOT)
    from oracle import operator as O
    from synth import Grid, head_phantom, ring_dipoles

    h = 0.192 / N
    g = Grid(N, N, N, h, h, h)
    eps, sig = head_phantom(g)
    pos, mom = ring_dipoles(R, 0.15)
    return g, O.Problem(g, FREQ, eps, sig), pos, mom


def solve_one(r):
    sys.path.insert(0, ROOT)
    from oracle import operator as O
    from oracle import post as OP
    from oracle import rhs as OR
    from oracle import solver as OS

    g, prob, pos, mom = problem()
    Nop = O.NOperator(g, prob.k0)
    e_inc = OR.dipoles_tested(g, prob.k0, prob.ce, pos[r : r + 1], mom[r : r + 1])[0]
    b = OR.rhs(prob, e_inc)
    x, info = OS.gmres(lambda v: O.apply_PA(prob, Nop, v), O.apply_Pinv(prob, b), tol=TOL, restart=100, maxit=60)
    e = OP.fields(prob, Nop, x, e_inc)
    p, P = OP.absorbed_power(prob, x)
    return r, e[[0, 4, 8]], p, float(P), float(info["resid"]), int(info["iters"])


def main():
    g, prob, _, _ = problem()
    tissue = (prob.chi != 0).ravel()
    ctx = mp.get_context("spawn")
    with ctx.Pool(R) as pool:
        res = sorted(pool.map(solve_one, range(R)))
    fmap = np.stack([e.reshape(3, -1)[:, tissue] for _, e, _, _, _, _ in res]).astype(np.complex64)
    pabs = np.stack([p.ravel()[tissue] for _, _, p, _, _, _ in res]).astype(np.float32)
    np.savez_compressed(
        OUT,
        field_l1=fmap,
        p_abs=pabs,
        P_abs=np.array([P for *_, P, _, _ in res]),
        resid=np.array([s for *_, s, _ in res]),
        iters=np.array([i for *_, i in res]),
        tol=TOL,
    )
    print("wrote", OUT, "resid", [s for *_, s, _ in res], "iters", [i for *_, i in res])


if __name__ == "__main__":
    main()
