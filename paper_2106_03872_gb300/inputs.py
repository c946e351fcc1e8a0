"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and lays out atoms; it holds none of the
method's arithmetic (no cutoff sphere, no potentials, no transforms).  Every
workload here is synthetic: the paper's own systems (Sec. "Results") need
pseudopotential files and comparison codes, so cells of the same shape are built
from seeded Gaussians instead.

Workload shapes (cubic periodic cell of side L bohr, N^3 grid, 20 Ha cutoff):

* ``small``   L=10,  N=24,  8 states,   4 atoms uniform in the cell, V_loc depth -2 Ha
* ``gs96``    L=30,  N=96,  128 states, 64 atoms on a perturbed fcc lattice, depth -3 Ha
* ``td128``   L=40,  N=128, 512 states, 128 atoms on a perturbed fcc lattice, depth -3 Ha
* ``td64``    L=20,  N=64,  64 states,  32 atoms (reduced real-time case)

All use Gaussian width 0.8 bohr for V_loc and 4 projectors per atom
(s + 3 p Gaussians, sigma 0.5 bohr, sphere radius 2 bohr, coupling 0.5 Ha).
"""
import numpy as np

BASE_SEED = 20210607

FCC_BASIS = np.array([[0.0, 0.0, 0.0],
                      [0.5, 0.5, 0.0],
                      [0.5, 0.0, 0.5],
                      [0.0, 0.5, 0.5]])


def uniform_positions(seed, natoms, L):
    """natoms positions drawn uniformly in [0, L)^3 (bohr), shape [natoms, 3]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, L, size=(natoms, 3))


def fcc_positions(seed, ncells, a, natoms, sigma=0.2):
    """natoms sites picked by a seeded permutation from an ncells^3 conventional fcc
    supercell of lattice constant a, each displaced by N(0, sigma^2) per axis and
    wrapped into the cell [0, ncells*a)^3."""
    rng = np.random.default_rng(seed)
    cells = np.array([[i, j, k] for i in range(ncells) for j in range(ncells) for k in range(ncells)], float)
    sites = (cells[:, None, :] + FCC_BASIS[None, :, :]).reshape(-1, 3) * a
    pick = rng.permutation(len(sites))[:natoms]
    pos = sites[np.sort(pick)] + rng.normal(0.0, sigma, size=(natoms, 3))
    L = ncells * a
    return np.mod(pos, L)


def random_coeffs(seed, nstates, nG):
    """i.i.d. complex Gaussian CN(0,1) coefficients, shape [nstates, nG] complex128."""
    rng = np.random.default_rng(seed)
    re = rng.normal(size=(nstates, nG))
    im = rng.normal(size=(nstates, nG))
    return (re + 1j * im) / np.sqrt(2.0)


def cell(name, nstates=None, natoms=None, seed_offset=0):
    """Cell description for a named workload as a plain dict (atomic units)."""
    spec = {
        "small": dict(L=10.0, N=24, nstates=8, natoms=4, depth=-2.0, lattice=None, cid=1),
        "gs96": dict(L=30.0, N=96, nstates=128, natoms=64, depth=-3.0, lattice=(3, 10.0), cid=2),
        "td128": dict(L=40.0, N=128, nstates=512, natoms=128, depth=-3.0, lattice=(4, 10.0), cid=3),
        "td64": dict(L=20.0, N=64, nstates=64, natoms=32, depth=-3.0, lattice=(2, 10.0), cid=3),
    }[name]
    seed = BASE_SEED + spec["cid"] + seed_offset
    na = natoms if natoms is not None else spec["natoms"]
    if spec["lattice"] is None:
        pos = uniform_positions(seed, na, spec["L"])
    else:
        ncells, a = spec["lattice"]
        pos = fcc_positions(seed, ncells, a, na)
    return dict(L=spec["L"], N=spec["N"], ecut=20.0, pos=pos,
                vloc_depth=spec["depth"], vloc_width=0.8,
                nproj=4, proj_sigma=0.5, proj_rc=2.0, proj_D=0.5,
                nstates=nstates if nstates is not None else spec["nstates"],
                seed=seed)


def thermal_velocities(seed, mass, kT=9.5e-4):
    """Seeded Maxwell-Boltzmann velocities [natoms, 3] (bohr per atomic time unit) for masses
    [natoms] (electron masses) at temperature kT (Ha; the default is 300 K)."""
    m = np.asarray(mass, float)
    rng = np.random.default_rng(seed)
    return rng.normal(size=(len(m), 3)) * np.sqrt(kT / m)[:, None]


def small_cell(L, N, natoms, nstates, seed, depth=-2.0, nproj=4, ecut=20.0):
    """Arbitrary small cell with uniformly placed atoms, for parity sweeps."""
    return dict(L=float(L), N=int(N), ecut=float(ecut), pos=uniform_positions(seed, natoms, L),
                vloc_depth=depth, vloc_width=0.8, nproj=nproj, proj_sigma=0.5, proj_rc=2.0,
                proj_D=0.5, nstates=nstates, seed=seed)


def serve_requests(seed, nreq, h=0.3125, grids=(32, 48, 64, 96), state_range=(8, 256),
                   atom_range=(4, 64), rate_per_s=None):
    """Seeded serving workload: each request is a cell (grid drawn from ``grids``,
    L = N*h), a state count, an atom count, and a kind (0: ground-state block
    iterations, 1: real-time steps).  Poisson arrival times if ``rate_per_s`` is given."""
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for r in range(nreq):
        N = int(rng.choice(grids))
        L = N * h
        ns = int(rng.integers(state_range[0], state_range[1] + 1))
        na = int(rng.integers(atom_range[0], atom_range[1] + 1))
        kind = int(rng.integers(0, 2))
        if rate_per_s:
            t += rng.exponential(1.0 / rate_per_s)
        reqs.append(dict(L=L, N=N, ecut=20.0, pos=rng.uniform(0.0, L, size=(na, 3)),
                         vloc_depth=-3.0, vloc_width=0.8, nproj=4, proj_sigma=0.5, proj_rc=2.0,
                         proj_D=0.5, nstates=ns, kind=kind, count=10 if kind == 0 else 50,
                         dt=0.05, arrival=t, seed=int(rng.integers(1 << 31))))
    return reqs
