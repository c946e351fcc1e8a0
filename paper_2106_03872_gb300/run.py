"""Command-line runner: one synthetic cell through the GPU path.

    python -m paper_2106_03872_gb300.run --cell gs96 --iterations 1
    python -m paper_2106_03872_gb300.run --cell td128 --td-steps 2
    python -m paper_2106_03872_gb300.run --cell gs96 --iterations 3 --timeline

It builds the grid of a named synthetic cell (plane-wave sphere, local potential, KB
projectors), loads seeded random coefficients, and runs block iterations (Sec. 3: H psi,
orthonormalisation, Rayleigh-Ritz, steepest-descent update) and/or ETRS time steps (Sec. 4,
Eq. 8), then prints one line with the lowest eigenvalue or the step count.  It is the small,
deterministic program that kernel profiles are captured on.
"""
import argparse
import time

import torch

from . import inputs, ks


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--cell", default="gs96", help="named synthetic cell (gs96, td128, ...)")
    ap.add_argument("--prec", default="bf16x3", choices=("bf16x3", "fp64"))
    ap.add_argument("--iterations", type=int, default=1, help="block iterations (ground state)")
    ap.add_argument("--td-steps", type=int, default=0, help="ETRS time steps after the iterations")
    ap.add_argument("--dt", type=float, default=0.05)
    ap.add_argument("--states", type=int, default=0, help="states of the cell (0: the cell's own count)")
    ap.add_argument("--timeline", action="store_true",
                    help="after one warm-up iteration, print the stage spans of the block iterations "
                         "(main and side stream, ms on a common clock)")
    args = ap.parse_args(argv)

    cell = inputs.cell(args.cell, nstates=args.states or None)
    g = ks.Grid(cell, prec=args.prec)
    g.set_states(inputs.random_coeffs(cell["seed"], cell["nstates"], g.nG))
    if args.timeline:
        g.block_iteration(1)
        torch.cuda.synchronize()
        g.profile(1)
        g.profile(3)
    if args.iterations == 0 and args.td_steps > 0:
        g.orthonormalize()                 # the real-time step propagates an orthonormal block
    t0 = time.perf_counter()
    eps = g.block_iteration(args.iterations) if args.iterations > 0 else None
    if args.td_steps > 0:
        g.td_step(args.dt, args.td_steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    line = "cell=%s N=%d states=%d nG=%d iterations=%d td_steps=%d wall=%.3f s" % (
        args.cell, cell["N"], cell["nstates"], g.nG, args.iterations, args.td_steps, dt)
    if eps is not None:
        line += " eps0=%.6f" % float(eps[0])
    print(line)
    if args.timeline:
        for name, a, b in sorted(g.profile_spans(), key=lambda x: x[1]):
            print("%-14s %8.3f %8.3f" % (name, a, b))
        g.profile(4)
        g.profile(0)
    g.close()


if __name__ == "__main__":
    main()
