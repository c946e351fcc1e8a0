"""Writes the stored expected values under tests/golden/ by calling only the FP64 oracle
(oracle/ks_oracle.py) on the seeded inputs of paper_2106_03872_gb300/inputs.py.

    python tests/golden/make_goldens.py gs96     # 20 steepest-descent block iterations, 96^3, 128 states
    python tests/golden/make_goldens.py td64     # 200 ETRS steps with Hartree + Slater, 64^3, 64 states
    python tests/golden/make_goldens.py td128s   # 2 ETRS steps with Hartree + Slater, 128^3 cell, 8 states

The oracle's H application acts on every state independently, and its density is a sum over
states (Eq. 1).  So that the full-size runs finish in hours rather than days, this script
evaluates those two oracle functions over chunks of states in worker processes and joins the
chunks (rows concatenated; partial densities summed in chunk order).  Everything else (CholQR,
Rayleigh-Ritz, the steepest-descent update, the ETRS/Taylor step, Hartree, Slater, energies,
norms, dipoles) runs in the oracle's own functions unchanged.  The joined results equal the
single-process oracle up to the rounding order of the density sum.
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HERE = os.path.dirname(os.path.abspath(__file__))

_CELL = None


def _init(desc):
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    global _CELL
    from oracle import ks_oracle as ko
    _CELL = ko.Cell(desc)


def _apply(args):
    from oracle import ks_oracle as ko
    c, v = args
    return ko.apply_h(_CELL, c, v)


def _density(args):
    from oracle import ks_oracle as ko
    c, occ = args
    return ko.density(_CELL, c, occ)


class Parallel:
    """Replaces the oracle's apply_h and density by chunked evaluations of the same functions."""

    def __init__(self, ko, cell, desc, workers):
        self.ko, self.cell = ko, cell
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_init, initargs=(desc,))
        self.workers = workers
        self.orig_apply, self.orig_density = ko.apply_h, ko.density

    def chunks(self, n):
        k = max(1, (n + self.workers - 1) // self.workers)
        return [(i, min(n, i + k)) for i in range(0, n, k)]

    def apply_h(self, cell, c, v=None):
        import numpy as np
        assert cell is self.cell
        c = np.atleast_2d(np.asarray(c, dtype=np.complex128))
        vv = cell.vloc if v is None else v
        parts = self.pool.map(_apply, [(c[a:b], vv) for a, b in self.chunks(c.shape[0])])
        return np.concatenate(parts, axis=0)

    def density(self, cell, c, occ=None):
        import numpy as np
        assert cell is self.cell
        c = np.atleast_2d(c)
        f = cell.occupations(c.shape[0]) if occ is None else np.asarray(occ, float)
        parts = self.pool.map(_density, [(c[a:b], f[a:b]) for a, b in self.chunks(c.shape[0])])
        out = parts[0].copy()
        for p in parts[1:]:
            out += p
        return out

    def __enter__(self):
        self.ko.apply_h, self.ko.density = self.apply_h, self.density
        return self

    def __exit__(self, *a):
        self.ko.apply_h, self.ko.density = self.orig_apply, self.orig_density
        self.pool.close()
        self.pool.join()


def cplx_list(a):
    import numpy as np
    a = np.asarray(a)
    return [[float(x.real), float(x.imag)] for x in a.ravel()]


def write(name, payload):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        json.dump(payload, f, indent=0)
        f.write("\n")
    print("wrote", path, file=sys.stderr)


def gs96(workers):
    """Sec. "Ground-state solution": the steepest-descent block iteration (CholQR -> H Psi ->
    Rayleigh-Ritz -> Psi - alpha R), 20 iterations from the seeded CN(0,1) start of the 96^3 /
    128-state cell.  Records the Ritz values of every iteration, and the Ritz values of the
    final iterate's subspace (CholQR, then Rayleigh-Ritz with the FP64 H)."""
    import numpy as np
    from oracle import ks_oracle as ko
    from paper_2106_03872_gb300 import inputs
    desc = inputs.cell("gs96")
    cell = ko.Cell(desc)
    c = inputs.random_coeffs(desc["seed"], desc["nstates"], cell.nG)
    eps_hist = []
    t0 = time.time()
    with Parallel(ko, cell, desc, workers):
        for it in range(20):
            eps, c = ko.block_iteration(cell, c, 1)   # one iteration = the loop body of block_iteration
            eps_hist.append([float(x) for x in eps])
            print("gs96 iteration %d  %.0f s  eps0 %.12f" % (it + 1, time.time() - t0, eps[0]), file=sys.stderr)
        q, _ = ko.cholqr(c)
        e_sub, _, _, _ = ko.rayleigh_ritz(q, ko.apply_h(cell, q))
    write("gs96_block_iteration.json", {
        "what": "Ritz values of the steepest-descent block iteration (Sec. Ground-state solution) on the gs96 "
                "cell: L=30, N=96, 128 states, 64 atoms, seeded CN(0,1) start; eps[i] = the Rayleigh-Ritz values "
                "of iteration i+1; eps_subspace = Rayleigh-Ritz of the final iterate after CholQR",
        "command": "python tests/golden/make_goldens.py gs96",
        "cell": "gs96", "nstates": desc["nstates"], "nG": int(cell.nG), "iterations": 20,
        "alpha": float(cell.sd_step_length()),
        "eps": eps_hist, "eps_subspace": [float(x) for x in e_sub]})


def td_run(name, desc, nstates, nsteps, workers, sample_seed, nsample_g):
    """Sec. "Real-time propagation", Eqs. 6-8: ETRS with the 4th-order Taylor exponential and
    shared powers, V = V_loc + v_H + v_x from the density each step (Hartree in Fourier space,
    Slater exchange), dt = 0.05, from the CholQR'd seeded CN(0,1) states.  Records per step the
    norm, the energy (Eq. 5 with expectation values) and the dipole at the step's start, and at
    the end per state the norm, the overlap with the initial state and sampled coefficients."""
    import numpy as np
    from oracle import ks_oracle as ko
    from paper_2106_03872_gb300 import inputs
    desc = dict(desc, nstates=nstates)
    cell = ko.Cell(desc)
    c0 = inputs.random_coeffs(desc["seed"], nstates, cell.nG)
    q, _ = ko.cholqr(c0)
    dt = 0.05
    norms, energies, dips = [], [], []
    c = q
    t0 = time.time()
    with Parallel(ko, cell, desc, workers):
        for s in range(nsteps):
            dips.append(ko.dipole(cell, ko.density(cell, c)))
            c, nrm, e = ko.td_step(cell, c, dt, "etrs", True)
            norms.append(nrm)
            energies.append(e)
            print("%s step %d  %.0f s  norm %.15f  E %.12f" % (name, s + 1, time.time() - t0, nrm, e), file=sys.stderr)
    rng = np.random.default_rng(sample_seed)
    gsel = np.sort(rng.choice(cell.nG, size=nsample_g, replace=False))
    write(name + ".json", {
        "what": "ETRS + Taylor-4 real-time run with Hartree + Slater (Sec. Real-time propagation, Eqs. 6-8) from "
                "the CholQR'd seeded CN(0,1) states; norm/energy/dipole at the start of each step; final per-state "
                "norm, overlap <psi_k(0)|psi_k(T)> and coefficients at the sampled G indices",
        "command": "python tests/golden/make_goldens.py " + ("td64" if name == "td64_etrs" else "td128s"),
        "cell": desc.get("name", name), "L": desc["L"], "N": desc["N"], "nstates": nstates,
        "natoms": int(cell.natoms), "nG": int(cell.nG), "dt": dt, "steps": nsteps,
        "norm": [float(x) for x in norms], "energy": [float(x) for x in energies],
        "dipole": [[float(v) for v in d] for d in dips],
        "final_norm": [float(x) for x in np.sum(np.abs(c) ** 2, axis=1)],
        "final_overlap": cplx_list(np.sum(np.conj(q) * c, axis=1)),
        "g_sample": [int(x) for x in gsel],
        "final_coeff_sample": cplx_list(c[:, gsel])})


def main():
    what = sys.argv[1]
    workers = int(os.environ.get("GOLDEN_WORKERS", "8"))
    from paper_2106_03872_gb300 import inputs
    if what == "gs96":
        gs96(workers)
    elif what == "td64":
        td_run("td64_etrs", dict(inputs.cell("td64"), name="td64"), 64, 200, workers, 64, 32)
    elif what == "td128s":
        td_run("td128_sample_etrs", dict(inputs.cell("td128"), name="td128"), 8, 2, workers, 128, 64)
    else:
        raise SystemExit("unknown golden: " + what)


if __name__ == "__main__":
    main()
