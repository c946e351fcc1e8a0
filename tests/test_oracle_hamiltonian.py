"""Pins for the oracle's Hamiltonian (Eq. 2 and Eq. 9), CPU only."""
import numpy as np
import pytest

from oracle import ks_oracle as ko
from paper_2106_03872_gb300 import inputs


def make_cell(L=10.0, N=24, natoms=4, depth=-2.0, nproj=4, D=0.5, seed=11, ecut=20.0):
    pos = inputs.uniform_positions(seed, natoms, L)
    return ko.Cell(dict(L=L, N=N, ecut=ecut, pos=pos, vloc_depth=depth, vloc_width=0.8, nproj=nproj,
                        proj_sigma=0.5, proj_rc=2.0, proj_D=D))


def rand_c(cell, n, seed=0):
    return inputs.random_coeffs(seed, n, cell.nG)


def test_free_plane_waves_are_eigenvectors():
    cell = make_cell(natoms=0)
    for k in [0, 1, 777, cell.nG - 1]:
        c = np.zeros((1, cell.nG), complex)
        c[0, k] = 1.0
        hc = ko.apply_h(cell, c)
        assert np.max(np.abs(hc - 0.5 * cell.g2[k] * c)) < 1e-12


def test_free_spectrum_is_kinetic_shells():
    """Dense matrix of H on a tiny free cell: eigenvalues are the |G|^2/2 list, shells included."""
    cell = make_cell(L=6.0, N=12, natoms=0, ecut=6.0)
    H = ko.apply_h(cell, np.eye(cell.nG)).T
    ev = np.linalg.eigvalsh(0.5 * (H + H.conj().T))
    assert np.allclose(ev, np.sort(0.5 * cell.g2), atol=1e-12)


def test_constant_potential_shifts_spectrum():
    cell = make_cell(natoms=0)
    c = rand_c(cell, 2)
    v0 = -0.37
    assert np.allclose(ko.apply_h(cell, c, np.full((cell.N,) * 3, v0)), ko.apply_h(cell, c) + v0 * c,
                       atol=1e-12)


def test_cosine_potential_couples_g_and_g_plus_minus_q():
    """V(r) = 2 v1 cos(q.r): (V psi)_G = v1 (c_{G-q} + c_{G+q}) for G in S (c = 0 outside S)."""
    cell = make_cell(natoms=0)
    q = np.array([1, 2, 0])
    v1 = 0.3
    r = cell.grid_points()
    V = 2 * v1 * np.cos(r @ (2 * np.pi / cell.L * q))
    c = rand_c(cell, 1, seed=5)[0]
    lookup = {tuple(m): i for i, m in enumerate(cell.m)}
    expect = 0.5 * cell.g2 * c
    for i, m in enumerate(cell.m):
        for s in (-1, +1):
            j = lookup.get(tuple(m - s * q))
            if j is not None:
                expect[i] += v1 * c[j]
    got = ko.apply_h(cell, c[None], V)[0]
    assert np.max(np.abs(got - expect)) < 1e-12


def test_local_potential_integral():
    """dV sum_j V_loc = natoms A (2 pi w^2)^{3/2}: Gaussians narrow against L, periodic
    trapezoid rule spectrally exact."""
    cell = make_cell(natoms=4, depth=-2.0)
    expect = 4 * -2.0 * (2 * np.pi * 0.8 ** 2) ** 1.5
    assert abs(cell.dV * cell.vloc.sum() - expect) < 1e-10 * abs(expect)


def test_projection_matches_bruteforce_loops():
    cell = make_cell(L=8.0, N=16, natoms=3, seed=4)
    c = rand_c(cell, 2, seed=9)
    psi = ko.to_real(cell, c)
    p = ko.nonlocal_projections(cell, psi)
    h = cell.h
    for I, R in enumerate(cell.pos):
        acc = np.zeros((2, 4), complex)
        for jx in range(cell.N):
            for jy in range(cell.N):
                for jz in range(cell.N):
                    d = np.array([jx, jy, jz]) * h - R
                    d = d - cell.L * np.round(d / cell.L)
                    dist2 = d @ d
                    if dist2 >= cell.rc ** 2:
                        continue
                    g = np.exp(-dist2 / (2 * cell.sigma_b ** 2))
                    b = np.array([g, d[0] * g, d[1] * g, d[2] * g])
                    acc += np.outer(psi[:, jx, jy, jz], b)
        # grid normalisation of each projector, recomputed by the loop above's own b
        norms = np.zeros(4)
        for jx in range(cell.N):
            for jy in range(cell.N):
                for jz in range(cell.N):
                    d = np.array([jx, jy, jz]) * h - R
                    d = d - cell.L * np.round(d / cell.L)
                    if d @ d < cell.rc ** 2:
                        g = np.exp(-(d @ d) / (2 * cell.sigma_b ** 2))
                        norms += np.array([g, d[0] * g, d[1] * g, d[2] * g]) ** 2
        ref = cell.dV * acc / np.sqrt(cell.dV * norms)[None, :]
        assert np.max(np.abs(p[:, I, :] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_nonlocal_on_its_own_projector():
    """One atom, one s projector: V_NL beta = D beta (dV sum beta^2 = 1)."""
    cell = make_cell(natoms=1, nproj=1, D=0.7)
    beta = np.zeros(cell.N ** 3)
    beta[cell.proj_index[0]] = cell.proj_beta[0][0]
    out = ko.apply_nonlocal(cell, beta.reshape(1, cell.N, cell.N, cell.N)).reshape(-1)
    assert np.max(np.abs(out - 0.7 * beta)) < 1e-12


def test_nonlocal_psd_and_hamiltonian_hermitian():
    cell = make_cell(natoms=4)
    a = rand_c(cell, 3, seed=1)
    b = rand_c(cell, 3, seed=2)
    ha, hb = ko.apply_h(cell, a), ko.apply_h(cell, b)
    lhs = np.conj(a) @ hb.T
    rhs = np.conj(ha) @ b.T
    assert np.max(np.abs(lhs - rhs)) <= 1e-13 * np.max(np.abs(lhs))
    psi = ko.to_real(cell, a)
    vnl = ko.apply_nonlocal(cell, psi)
    quad = cell.dV * np.sum(np.conj(psi) * vnl, axis=(1, 2, 3))
    assert np.all(quad.real > 0) and np.all(np.abs(quad.imag) < 1e-12 * np.abs(quad.real))


def test_hamiltonian_is_linear():
    cell = make_cell(natoms=2)
    a, b = rand_c(cell, 1, 3), rand_c(cell, 1, 4)
    z = 0.3 - 1.1j
    assert np.allclose(ko.apply_h(cell, a + z * b), ko.apply_h(cell, a) + z * ko.apply_h(cell, b), atol=1e-11)


def _potential_energy(desc, c):
    """sum_k f_k <phi_k| V_loc + V_NL |phi_k> on the grid, orbitals fixed."""
    cell = ko.Cell(desc)
    e_loc = cell.dV * np.sum(cell.vloc * ko.density(cell, c))
    p = ko.nonlocal_projections(cell, ko.to_real(cell, c))
    return e_loc + np.sum(cell.occupations(c.shape[0])[:, None, None] * cell.D * np.abs(p) ** 2)


def _fd_forces(desc, c, atoms, d=1e-3):
    out = np.zeros((len(atoms), 3))
    for n, I in enumerate(atoms):
        for a in range(3):
            pp, pm = desc["pos"].copy(), desc["pos"].copy()
            pp[I, a] += d
            pm[I, a] -= d
            out[n, a] = -(_potential_energy(dict(desc, pos=pp), c) - _potential_energy(dict(desc, pos=pm), c)) / (2 * d)
    return out


def test_forces_local_part_is_minus_energy_derivative():
    """D = 0: Eq. 11's local term equals -dE/dR_I of the grid energy with the orbitals fixed
    (central differences, error O(d^2) ~ 1e-8); this also fixes the overall sign."""
    desc = dict(inputs.small_cell(10.0, 24, 2, 3, 62, depth=-3.0), proj_D=0.0)
    cell = ko.Cell(desc)
    c, _ = ko.cholqr(inputs.random_coeffs(62, 3, cell.nG))
    c = ko.block_iteration(cell, c, 10)[1]
    c, _ = ko.cholqr(c)
    F = ko.forces(cell, c)
    assert np.max(np.abs(F)) > 1e-2
    assert np.max(np.abs(F - _fd_forces(desc, c, [0, 1]))) <= 1e-6


def test_forces_with_projectors_match_energy_derivative():
    """With the KB projectors (about a quarter of each force here) Eq. 11 matches -dE/dR_I to
    the projector spheres' truncation at R_c, where beta is ~5e-4 of its peak, and to the
    grid (N = 32, h = 0.31): 3e-4 absolute on forces of ~4e-2."""
    desc = inputs.small_cell(10.0, 32, 3, 5, 61, depth=-3.0)
    cell = ko.Cell(desc)
    c, _ = ko.cholqr(inputs.random_coeffs(61, 5, cell.nG))
    c = ko.block_iteration(cell, c, 20)[1]
    c, _ = ko.cholqr(c)
    F = ko.forces(cell, c)
    assert np.max(np.abs(F)) > 2e-2
    assert np.max(np.abs(F - _fd_forces(desc, c, [0, 1, 2]))) <= 3e-4
