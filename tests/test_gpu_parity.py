"""GPU parity: every C-ABI operation against the FP64 oracle on the same seeded inputs.

Tolerances: FP64 path 1e-12 relative (eigenvalues and energies relative to max(1, their
largest magnitude); an eigenvector's overlap relative to that over its gap); FP32 (mixed) H psi
2e-5 relative L2 per block.
Other mixed-path tolerances are derived from FP32 rounding (unit roundoff 6e-8, grown by
the FFT depth and the reductions) and stated beside each check.
"""
import numpy as np
import pytest

from oracle import ks_oracle as ko
from paper_2106_03872_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ks():
    from paper_2106_03872_gb300 import ks as mod
    mod.load()
    assert torch.cuda.is_available()
    return mod


TOL_H = {"fp64": 1e-12, "bf16x3": 2e-5}
CDT = {"fp64": torch.complex128, "bf16x3": torch.complex64}


_CELLS = {}


def oracle_cell(name):
    if name not in _CELLS:
        cell = inputs.cell(name)
        _CELLS[name] = (cell, ko.Cell(cell))
    return _CELLS[name]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def apply_dev(ks, g, c, prec):
    psi = torch.from_numpy(c).to("cuda", CDT[prec])
    h = torch.empty_like(psi)
    g.apply_h(psi.data_ptr(), h.data_ptr(), c.shape[0])
    torch.cuda.synchronize()
    return h.cpu().numpy().astype(np.complex128)


CASES = [
    # (L, N, natoms, nstates, nproj, seed)
    (10.0, 24, 4, 8, 4, 1),
    (10.0, 24, 0, 1, 4, 2),          # free electrons, one state
    (12.0, 32, 3, 5, 1, 3),          # s projectors only
    (15.0, 48, 6, 17, 4, 4),         # ragged state count
    (9.0, 36, 2, 3, 4, 5),           # radix-3 grid (36 = 4*9)
    (20.0, 64, 8, 6, 4, 6),          # 64^3: the team plane kernel (8 x 8 plan)
]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("case", CASES)
def test_apply_h_parity(ks, prec, case, meas):
    L, N, na, ns, nproj, seed = case
    cell = inputs.small_cell(L, N, na, ns, seed, nproj=nproj)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec=prec)
    assert g.nG == ref.nG
    assert np.array_equal(g.gvectors(), ref.m)
    meas("np.max(np.abs(g.vloc() - ref.vloc))", np.max(np.abs(g.vloc() - ref.vloc)), 1e-13 * max(1.0, np.max(np.abs(ref.vloc))))
    c = inputs.random_coeffs(seed, ns, ref.nG)
    expect = ko.apply_h(ref, c)
    got = apply_dev(ks, g, c, prec)
    for k in range(ns):
        meas("rel(got[k], expect[k])", rel(got[k], expect[k]), TOL_H[prec])
    # the host entry point gives the same numbers
    got_h = g.apply_h_host(c)
    meas("rel(got_h, expect)", rel(got_h, expect), TOL_H[prec])
    # fewer states than the handle holds
    if ns > 2:
        part = apply_dev(ks, g, c[:2].copy(), prec)
        meas("rel(part, expect[:2])", rel(part, expect[:2]), TOL_H[prec])
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_apply_h_full_size_sampled(ks, prec, meas):
    """96^3 grid, 128 states, 64 atoms: all states on the GPU, 3 sampled states by the oracle."""
    cell, ref = oracle_cell("gs96")
    g = ks.Grid(cell, prec=prec)
    c = inputs.random_coeffs(cell["seed"], cell["nstates"], ref.nG)
    got = apply_dev(ks, g, c, prec)
    for k in (0, 63, 127):
        e = ko.apply_h(ref, c[k:k + 1])[0]
        meas("rel(got[k], e)", rel(got[k], e), TOL_H[prec])
    g.close()


def test_apply_h_128_grid_sampled(ks, meas):
    """128^3 grid (the real-time workload's size, radix plan 8 x 16), 6 states, 8 atoms."""
    cell = inputs.small_cell(40.0, 128, 8, 6, 18, depth=-3.0)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec="bf16x3")
    c = inputs.random_coeffs(18, 6, ref.nG)
    got = apply_dev(ks, g, c, "bf16x3")
    for k in (0, 5):
        e = ko.apply_h(ref, c[k:k + 1])[0]
        meas("rel(got[k], e)", rel(got[k], e), TOL_H["bf16x3"])
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_density_parity(ks, prec, meas):
    cell = inputs.small_cell(12.0, 32, 3, 6, 7)
    occ = np.array([2.0, 2.0, 1.0, 0.5, 0.0, 1.0])
    ref = ko.Cell(dict(cell, occ=occ))
    g = ks.Grid(cell, prec=prec, occ=occ)
    c = inputs.random_coeffs(7, 6, ref.nG)
    g.set_states(c)
    n = torch.empty(32 ** 3, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
    g.density(n.data_ptr())
    torch.cuda.synchronize()
    expect = ko.density(ref, c, occ).reshape(-1)
    # FP32: |psi|^2 from an FP32 FFT, relative error ~ 2 * 7 stages * 6e-8 -> 1e-6 L2; bound 1e-5
    meas("rel(n.cpu().numpy().astype(float), expect)", rel(n.cpu().numpy().astype(float), expect), (1e-12 if prec == "fp64" else 1e-5))
    g.close()


def test_density_clusters_and_ragged_tail(ks, meas):
    """19 states: two full clusters of 8 states and a ragged third (3 states, 5 padding
    slots), with unequal occupations, on the mixed path."""
    cell = inputs.small_cell(10.0, 24, 2, 19, 54)
    occ = np.linspace(0.0, 2.0, 19)
    ref = ko.Cell(dict(cell, occ=occ))
    g = ks.Grid(cell, prec="bf16x3", occ=occ)
    c = inputs.random_coeffs(54, 19, ref.nG)
    g.set_states(c)
    n = torch.empty(24 ** 3, dtype=torch.float32, device="cuda")
    g.density(n.data_ptr())
    torch.cuda.synchronize()
    meas("rel(n.cpu().numpy().astype(float), ko.density(ref, c, occ).reshape(-1))", rel(n.cpu().numpy().astype(float), ko.density(ref, c, occ).reshape(-1)), 1e-5)
    g.close()


def test_density_128_grid(ks, meas):
    """128^3 grid (the real-time workload's size): the chunked density kernel."""
    cell = inputs.small_cell(40.0, 128, 4, 5, 55)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec="bf16x3")
    c = inputs.random_coeffs(55, 5, ref.nG)
    g.set_states(c)
    n = torch.empty(128 ** 3, dtype=torch.float32, device="cuda")
    g.density(n.data_ptr())
    torch.cuda.synchronize()
    meas("rel(n.cpu().numpy().astype(float), ko.density(ref, c).reshape(-1))", rel(n.cpu().numpy().astype(float), ko.density(ref, c).reshape(-1)), 1e-5)
    g.close()


@pytest.mark.parametrize("case", [(20.0, 64, 6, 19, 61), (30.0, 96, 8, 6, 62)])
def test_density_team_grids(ks, meas, case):
    """64^3 and 96^3 grids: the team density kernel (states in chunks, accumulated per point
    in state order), with unequal occupations and a chunk count that leaves a ragged chunk."""
    L, N, na, ns, seed = case
    cell = inputs.small_cell(L, N, na, ns, seed)
    occ = np.linspace(0.2, 2.0, ns)
    ref = ko.Cell(dict(cell, occ=occ))
    g = ks.Grid(cell, prec="bf16x3", occ=occ)
    c = inputs.random_coeffs(seed, ns, ref.nG)
    g.set_states(c)
    n = torch.empty(N ** 3, dtype=torch.float32, device="cuda")
    g.density(n.data_ptr())
    torch.cuda.synchronize()
    meas("team density %d^3, relative L2" % N, rel(n.cpu().numpy().astype(float), ko.density(ref, c, occ).reshape(-1)),
         1e-5)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_orthonormalize_parity(ks, prec, meas):
    cell = inputs.small_cell(10.0, 24, 4, 9, 8)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec=prec)
    c = inputs.random_coeffs(8, 9, ref.nG)
    g.set_states(c)
    S = g.orthonormalize(want_S=True)
    q_ref, S_ref = ko.cholqr(c)
    tol = 1e-12 if prec == "fp64" else 2e-5
    meas("np.max(np.abs(S - S_ref))", np.max(np.abs(S - S_ref)), tol * np.max(np.abs(S_ref)))
    q = g.get_states()
    meas("rel(q, q_ref)", rel(q, q_ref), tol)
    meas("np.max(np.abs(ko.gram(q) - np.eye(9)))", np.max(np.abs(ko.gram(q) - np.eye(9))), (1e-12 if prec == "fp64" else 1e-5))
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_orthonormalize_rejects_dependent_states(ks, prec, meas):
    cell = inputs.small_cell(10.0, 24, 2, 4, 9)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec=prec)
    c = inputs.random_coeffs(9, 4, ref.nG)
    c[2] = c[1]
    g.set_states(c)
    before = g.get_states()
    with pytest.raises(ks.KsError) as e:
        g.orthonormalize()
    assert e.value.status == ks.KS_ERR_NOT_POSDEF
    assert np.array_equal(g.get_states(), before)          # unchanged
    meas("rel(before, c)", rel(before, c), (1e-15 if prec == "fp64" else 1e-7))
    g.close()


@pytest.mark.parametrize("n", [64, 150, 256])
def test_mixed_cholesky_matches_fp64_factor_of_same_S(ks, n, meas):
    """The two-pass FP32 factor against an FP64 Cholesky of the very S the GPU formed, on a
    block with cond(S) ~ 1e4: one FP32 pass would be off by ~eps_32 cond(S) ~ 1e-3."""
    cell = inputs.small_cell(12.0, 32, 2, n, 31)
    ref = ko.Cell(cell)
    rng = np.random.default_rng(31)
    u, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    v, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    c = (u * np.logspace(0.0, -2.0, n)) @ v @ inputs.random_coeffs(31, n, ref.nG)
    g = ks.Grid(cell, prec="bf16x3")
    g.set_states(c)
    c32 = g.get_states()
    S = g.orthonormalize(want_S=True)
    q_ref, _ = ko.cholqr(c32, S=S)
    # tensor-core rotation by M = L^{-1} (cond(L) = 1e2): the state operand is split into two
    # bf16 terms (relative 2^-17 = 7.6e-6 per entry), amplified by at most cond(L) (7.6e-4) and
    # averaged over the n random terms of each row: bound 1e-4
    meas("rel(g.get_states(), q_ref)", rel(g.get_states(), q_ref), 1e-4)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_rayleigh_ritz_parity(ks, prec, meas):
    cell = inputs.small_cell(10.0, 24, 4, 12, 10)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec=prec)
    q, _ = ko.cholqr(inputs.random_coeffs(10, 12, ref.nG))
    g.set_states(q)
    eps = g.rayleigh_ritz()
    eps_ref, U, c_ref, _ = ko.rayleigh_ritz(q, ko.apply_h(ref, q))
    # FP32: H_sub entries carry ~1e-6 relative error of ||H|| <= 25 Ha -> 2.5e-5 Ha bound
    meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)),
         (1e-12 * max(1.0, np.max(np.abs(eps_ref))) if prec == "fp64" else 2.5e-5))
    # rotated states equal up to the phase convention: compare |<ref_i|got_i>|
    got = g.get_states()
    ov = np.abs(np.sum(np.conj(c_ref) * got, axis=1))
    gaps = np.min(np.abs(eps_ref[:, None] - eps_ref[None, :]) + np.eye(12) * 1e9, axis=1)
    well = gaps > 1e-3
    # an eigenvector's error is the eigenvalue error over the gap to its neighbours (Davis-Kahan)
    meas("max |1 - |<ref_i|got_i>|| over well-separated vectors", np.max(np.abs(ov[well] - 1)),
         (1e-12 * max(1.0, np.max(np.abs(eps_ref))) / np.min(gaps[well]) if prec == "fp64" else 1e-3))
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_block_iteration_parity(ks, prec, meas):
    cell = inputs.small_cell(12.0, 32, 4, 10, 11, depth=-3.0)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec=prec)
    c = inputs.random_coeffs(11, 10, ref.nG)
    g.set_states(c)
    eps = g.block_iteration(8)
    eps_ref, c_ref = ko.block_iteration(ref, c, 8)
    if prec == "fp64":
        meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)), 1e-12 * max(1.0, np.max(np.abs(eps_ref))))
    else:
        # refinement: Rayleigh-Ritz of the mixed-precision subspace with the FP64 H
        q, _ = ko.cholqr(g.get_states())
        e_ref_sub, _, _, _ = ko.rayleigh_ritz(q, ko.apply_h(ref, q))
        q2, _ = ko.cholqr(c_ref)
        e_ora, _, _, _ = ko.rayleigh_ritz(q2, ko.apply_h(ref, q2))
        # 8 iterations from a random start are far from converged, so the iterate itself
        # carries the mixed-precision error at first order (bf16x3 products ~3e-6 relative)
        meas("np.max(np.abs(e_ref_sub - e_ora))", np.max(np.abs(e_ref_sub - e_ora)), 1e-5)
        meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)), 1e-4)
    g.close()


def test_fp64_subspace_option_parity(ks, meas):
    """KS_OPT_FP64_SUBSPACE on a mixed handle: the Cholesky factor of S, the subspace products and
    the Rayleigh-Ritz eigensolver in FP64.  Block iteration, Rayleigh-Ritz and CholQR against the
    oracle at the mixed path's tolerances (the states stay complex64, so those bound the result);
    invalid options and values are rejected."""
    cell = inputs.small_cell(12.0, 32, 4, 10, 11, depth=-3.0)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec="bf16x3")
    g.set_option(ks.KS_OPT_FP64_SUBSPACE, 1)
    c = inputs.random_coeffs(11, 10, ref.nG)
    g.set_states(c)
    eps = g.block_iteration(8)
    eps_ref, c_ref = ko.block_iteration(ref, c, 8)
    meas("fp64-subspace block iteration, max |d eps|", np.max(np.abs(eps - eps_ref)), 1e-4)
    q, _ = ko.cholqr(g.get_states())
    e_sub, _, _, _ = ko.rayleigh_ritz(q, ko.apply_h(ref, q))
    q2, _ = ko.cholqr(c_ref)
    e_ora, _, _, _ = ko.rayleigh_ritz(q2, ko.apply_h(ref, q2))
    meas("fp64-subspace refined Ritz values, max |d|", np.max(np.abs(e_sub - e_ora)), 1e-5)
    # CholQR and Rayleigh-Ritz calls with the option
    g.set_states(c)
    g.orthonormalize()
    qq = g.get_states()
    meas("fp64-subspace CholQR orthonormality", np.max(np.abs(ko.gram(qq) - np.eye(10))), 1e-5)
    eps_rr = g.rayleigh_ritz()
    e_rr_ref, _, _, _ = ko.rayleigh_ritz(qq, ko.apply_h(ref, qq))
    meas("fp64-subspace Rayleigh-Ritz, max |d eps|", np.max(np.abs(eps_rr - e_rr_ref)), 2.5e-5)
    for bad in ((ks.KS_OPT_FP64_SUBSPACE, 2), (99, 1)):
        with pytest.raises(ks.KsError) as e:
            g.set_option(*bad)
        assert e.value.status == ks.KS_ERR_ARG
    g.close()


def test_block_iteration_converged_eigenvalues_after_refinement(ks, meas):
    """Mixed path to convergence, then one FP64 Rayleigh-Ritz of its final subspace: the
    converged eigenvalues match the oracle's to 1e-6 Ha (Ritz values are second order in
    the subspace error once converged)."""
    cell = inputs.small_cell(6.0, 18, 2, 4, 17, depth=-3.0)
    ref = ko.Cell(cell)
    c = inputs.random_coeffs(17, 4, ref.nG)
    e250, c250 = ko.block_iteration(ref, c, 250)
    e_ora, _ = ko.block_iteration(ref, c250, 50)
    converged = np.abs(e_ora - e250) < 1e-7
    assert converged[0]
    g = ks.Grid(cell, prec="bf16x3")
    g.set_states(c)
    g.block_iteration(300)
    q, _ = ko.cholqr(g.get_states())
    e_ref, _, _, _ = ko.rayleigh_ritz(q, ko.apply_h(ref, q))
    meas("np.max(np.abs(e_ref[converged] - e_ora[converged]))", np.max(np.abs(e_ref[converged] - e_ora[converged])), 1e-6)
    g.close()


def test_td_step_parity_96_grid(ks, meas):
    """A real-time step on the 96^3 grid of the ground-state workload (3 states, Hartree +
    Slater): the mixed path's packed H applications at N = 96 (the single-cell plane kernel per
    member), the kept Taylor powers summed in the fourth power's epilogue, and the first H
    application starting from the density's z transform, against the oracle."""
    cell = inputs.cell("gs96", nstates=3)
    ref = ko.Cell(cell)
    q, _ = ko.cholqr(inputs.random_coeffs(cell["seed"], 3, ref.nG))
    g = ks.Grid(cell, prec="bf16x3")
    g.set_states(q)
    norms, energies = g.td_step(0.05, 1, "etrs", True)
    c_ref, n_ref, e_ref = ko.td_run(ref, q, 0.05, 1, "etrs", True)
    got = g.get_states()
    meas("rel(got, c_ref)", rel(got, c_ref), 5e-5)
    meas("np.max(np.abs(norms - n_ref))", np.max(np.abs(norms - n_ref)), 1e-5 * n_ref[0])
    meas("np.max(np.abs(energies - e_ref))", np.max(np.abs(energies - e_ref)), 1e-4 * max(1, np.max(np.abs(e_ref))))
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("propagator", ["etrs", "taylor"])
@pytest.mark.parametrize("hxc", [True, False])
def test_td_step_parity(ks, prec, propagator, hxc, meas):
    cell = inputs.small_cell(10.0, 24, 4, 6, 12)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec=prec)
    q, _ = ko.cholqr(inputs.random_coeffs(12, 6, ref.nG))
    g.set_states(q)
    nsteps, dt = 3, 0.05
    norms, energies = g.td_step(dt, nsteps, propagator, hxc)
    c_ref, n_ref, e_ref = ko.td_run(ref, q, dt, nsteps, propagator, hxc)
    got = g.get_states()
    if prec == "fp64":
        meas("rel(got, c_ref)", rel(got, c_ref), 1e-12)
        meas("np.max(np.abs(norms - n_ref))", np.max(np.abs(norms - n_ref)), 1e-12 * n_ref[0])
        meas("np.max(np.abs(energies - e_ref))", np.max(np.abs(energies - e_ref)), 1e-12 * max(1, np.max(np.abs(e_ref))))
    else:
        meas("rel(got, c_ref)", rel(got, c_ref), 5e-5)
        meas("np.max(np.abs(norms - n_ref))", np.max(np.abs(norms - n_ref)), 1e-5 * n_ref[0])
        meas("np.max(np.abs(energies - e_ref))", np.max(np.abs(energies - e_ref)), 1e-4 * max(1, np.max(np.abs(e_ref))))
    g.close()


def test_td_divergence_detected(ks):
    """dt far beyond the Taylor-4 stability bound (x = dt*E > 2 sqrt 2) must report KS_ERR_DIVERGED."""
    cell = inputs.small_cell(10.0, 24, 2, 3, 13)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec="fp64")
    q, _ = ko.cholqr(inputs.random_coeffs(13, 3, ref.nG))
    g.set_states(q)
    with pytest.raises(ks.KsError) as e:
        g.td_step(2.0, 20, "taylor", False)
    assert e.value.status == ks.KS_ERR_DIVERGED
    g.close()


def test_bad_arguments(ks):
    cell = inputs.small_cell(10.0, 24, 2, 3, 14)
    g = ks.Grid(cell, prec="fp64")
    psi = torch.zeros((3, g.nG), dtype=torch.complex128, device="cuda")
    with pytest.raises(ks.KsError) as e:
        g.apply_h(psi.data_ptr(), psi.data_ptr(), 3)
    assert e.value.status == ks.KS_ERR_ARG
    h = torch.empty_like(psi)
    with pytest.raises(ks.KsError):
        g.apply_h(psi.data_ptr(), h.data_ptr(), 4)
    g.close()
    bad = dict(cell, nproj=2)
    with pytest.raises(ks.KsError):
        ks.Grid(bad, prec="fp64")
    for prec in (2, -1):                       # only KS_FP64 and KS_MIXED_BF16X3 exist
        with pytest.raises(ks.KsError) as e:
            ks.Grid(cell, prec=prec)
        assert e.value.status == ks.KS_ERR_ARG


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_orthonormalize_parity_two_tiles(ks, prec, meas):
    """150 states: the overlap and rotation GEMMs span two 128-row tiles with a ragged edge."""
    cell = inputs.small_cell(16.0, 48, 3, 150, 15)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec=prec)
    c = inputs.random_coeffs(15, 150, ref.nG)
    g.set_states(c)
    S = g.orthonormalize(want_S=True)
    q_ref, S_ref = ko.cholqr(c)
    tol = 1e-12 if prec == "fp64" else 2e-5
    meas("np.max(np.abs(S - S_ref))", np.max(np.abs(S - S_ref)), tol * np.max(np.abs(S_ref)))
    q = g.get_states()
    meas("rel(q, q_ref)", rel(q, q_ref), (1e-12 if prec == "fp64" else 1e-4))
    meas("np.max(np.abs(ko.gram(q) - np.eye(150)))", np.max(np.abs(ko.gram(q) - np.eye(150))), (1e-12 if prec == "fp64" else 1e-4))
    g.close()


@pytest.mark.parametrize("L,nstates", [(24.0, 40), (30.0, 21)])
def test_orthonormalize_parity_multi_pass(ks, L, nstates, meas):
    """96^3 grids with 59k and 115k plane waves: the persistent rotation kernel gives each CTA
    several passes over its share of grid rows (ragged shares, a ragged last chunk of states)."""
    cell = inputs.small_cell(L, 96, 2, nstates, 23)
    ref = ko.Cell(cell)
    assert ref.nG > 148 * 256
    g = ks.Grid(cell, prec="bf16x3")
    c = inputs.random_coeffs(23, nstates, ref.nG)
    g.set_states(c)
    S = g.orthonormalize(want_S=True)
    q_ref, S_ref = ko.cholqr(c)
    meas("np.max(np.abs(S - S_ref))", np.max(np.abs(S - S_ref)), 2e-5 * np.max(np.abs(S_ref)))
    q = g.get_states()
    meas("rel(q, q_ref)", rel(q, q_ref), 1e-4)
    meas("np.max(np.abs(ko.gram(q) - np.eye(nstates)))", np.max(np.abs(ko.gram(q) - np.eye(nstates))), 1e-4)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("m2max,nshell", [(2, 19), (5, 57), (9, 123)])
def test_rayleigh_ritz_degenerate_shells(ks, prec, m2max, nshell, meas):
    """Free electrons: the plane waves with |m|^2 <= m2max (shells of 1, 6, 12, 8, 6, 24, ...
    states), mixed by a random unitary.  Rayleigh-Ritz must return the exact shell energies and
    orthonormal eigenvectors even though the eigenvalues are exactly degenerate."""
    cell = inputs.small_cell(8.0, 24, 0, nshell, 19)
    ref = ko.Cell(cell)
    m2 = np.sum(ref.m ** 2, axis=1)
    picks = np.flatnonzero(m2 <= m2max)
    assert len(picks) == nshell
    c = np.zeros((nshell, ref.nG), complex)
    c[np.arange(nshell), picks] = 1.0
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(nshell, nshell)) + 1j * rng.normal(size=(nshell, nshell)))
    c = Q @ c
    g = ks.Grid(cell, prec=prec)
    g.set_states(c)
    eps = g.rayleigh_ritz()
    emax = max(1.0, np.max(np.abs(eps)))
    meas("degenerate shells, max |eps - |G|^2/2|", np.max(np.abs(eps - np.sort(0.5 * ref.g2[picks]))),
         1e-12 * emax if prec == "fp64" else 2e-5)
    q = g.get_states()
    tol = 1e-12 if prec == "fp64" else 1e-5
    meas("np.max(np.abs(ko.gram(q) - np.eye(nshell)))", np.max(np.abs(ko.gram(q) - np.eye(nshell))), tol)
    hq = ko.apply_h(ref, q)
    meas("np.max(np.abs(hq - eps[:, None] * q))", np.max(np.abs(hq - eps[:, None] * q)), (1e-12 * emax if prec == "fp64" else 1e-4))
    g.close()


@pytest.mark.parametrize("N,L,natoms", [(54, 12.0, 2), (8, 3.0, 0)])
def test_apply_h_plain_path_grids(ks, N, L, natoms, meas):
    """Grid sizes outside the fused kernels' list (54 = 2 * 27, the smallest grid 8) take the
    plain FP32 path: same operator, same tolerance.  (An 8^3 grid holding the 20 Ha sphere
    needs L < 4 bohr, smaller than a projector sphere's diameter, so that cell has no atoms.)"""
    cell = inputs.small_cell(L, N, natoms, 3, 41)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec="bf16x3")
    c = inputs.random_coeffs(41, 3, ref.nG)
    meas("rel(apply_dev(ks, g, c, 'bf16x3'), ko.apply_h(ref, c))", rel(apply_dev(ks, g, c, "bf16x3"), ko.apply_h(ref, c)), 2e-5)
    g.close()


def test_apply_h_block_only_8_byte_aligned(ks, meas):
    """States that start one state into a buffer with an odd |S| are only 8-byte aligned: the
    projections then take the register-fed overlap kernel (the TMA-fed one needs 16-byte
    aligned operands); same operator, same tolerance."""
    cell = inputs.small_cell(10.0, 24, 4, 5, 43)
    ref = ko.Cell(cell)
    assert ref.nG % 2 == 1
    g = ks.Grid(cell, prec="bf16x3")
    c = inputs.random_coeffs(43, 5, ref.nG)
    buf = torch.zeros((6, ref.nG), dtype=torch.complex64, device="cuda")
    buf[1:] = torch.from_numpy(c).to("cuda", torch.complex64)
    out = torch.zeros_like(buf)
    psi, h = buf[1:], out[1:]
    assert psi.data_ptr() % 16 == 8 and h.data_ptr() % 16 == 8
    g.apply_h(psi.data_ptr(), h.data_ptr(), 5)
    torch.cuda.synchronize()
    got = h.cpu().numpy().astype(np.complex128)
    meas("rel(H psi at 8-byte aligned rows, oracle)", rel(got, ko.apply_h(ref, c)), 2e-5)
    assert torch.all(out[0] == 0)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_apply_h_partial_block_and_empty(ks, prec, meas):
    """ks_apply_h on the first n of the handle's states (n = 0 is a no-op)."""
    cell = inputs.small_cell(10.0, 24, 3, 9, 42)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec=prec)
    c = inputs.random_coeffs(42, 4, ref.nG)
    tol = 1e-12 if prec == "fp64" else 2e-5
    meas("rel(apply_dev(ks, g, c, prec), ko.apply_h(ref, c))", rel(apply_dev(ks, g, c, prec), ko.apply_h(ref, c)), tol)
    psi = torch.zeros((1, ref.nG), dtype=CDT[prec], device="cuda")
    out = torch.full_like(psi, 7.0)
    g.apply_h(psi.data_ptr(), out.data_ptr(), 0)
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)                     # untouched
    g.close()


def test_zero_work_calls(ks):
    cell = inputs.small_cell(10.0, 24, 2, 4, 43)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec="bf16x3")
    c = inputs.random_coeffs(43, 4, ref.nG)
    g.set_states(c)
    before = g.get_states()
    assert g.block_iteration(0).shape == (4,)
    n, e = g.td_step(0.05, 0)
    assert n.shape == (0,) and e.shape == (0,)
    assert np.array_equal(g.get_states(), before)
    g.close()


def test_block_iteration_split_calls_bit_identical(ks):
    """The H psi a block iteration carries to the next call is exactly what one longer call
    uses, and new states discard it: split and fresh runs are bit-identical."""
    cell = inputs.small_cell(12.0, 32, 4, 10, 44, depth=-3.0)
    ref = ko.Cell(cell)
    c = inputs.random_coeffs(44, 10, ref.nG)
    c2 = inputs.random_coeffs(45, 10, ref.nG)
    a = ks.Grid(cell, prec="bf16x3")
    b = ks.Grid(cell, prec="bf16x3")
    a.set_states(c)
    b.set_states(c)
    a.block_iteration(3)
    ea = a.block_iteration(4)
    eb = b.block_iteration(7)
    assert np.array_equal(ea, eb)
    assert np.array_equal(a.get_states(), b.get_states())
    a.set_states(c2)
    b.close()
    b = ks.Grid(cell, prec="bf16x3")
    b.set_states(c2)
    assert np.array_equal(a.block_iteration(2), b.block_iteration(2))
    assert np.array_equal(a.get_states(), b.get_states())
    a.close()
    b.close()


def test_block_iteration_mixed_128_states(ks, meas):
    """128 states, the largest block whose Rayleigh-Ritz step runs in one CTA on the mixed
    path: eigenvalues against the oracle's, and the returned states in ascending order."""
    cell = inputs.small_cell(16.0, 48, 3, 128, 47, depth=-3.0)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec="bf16x3")
    c = inputs.random_coeffs(47, 128, ref.nG)
    g.set_states(c)
    eps = g.block_iteration(2)
    eps_ref, c_ref = ko.block_iteration(ref, c, 2)
    meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)), 1e-4 * max(1.0, np.max(np.abs(eps_ref))))
    # rows in ascending order of the (FP32) eigenvalues; the reported FP64 Rayleigh quotients
    # may swap only within the FP32 error
    assert np.all(np.diff(eps) >= -1e-5)
    g.close()


def test_block_iteration_degenerate_shells(ks, meas):
    """Free electrons, a block spanning the 19 plane waves with |m|^2 <= 2 mixed by a random
    unitary: one block iteration's Ritz values are the exact shell energies (1, 6 and 12-fold
    degenerate), and the states stay in the span (the SD step vanishes on exact eigenvectors)."""
    cell = inputs.small_cell(8.0, 24, 0, 19, 19)
    ref = ko.Cell(cell)
    m2 = np.sum(ref.m ** 2, axis=1)
    picks = np.flatnonzero(m2 <= 2)
    c = np.zeros((19, ref.nG), complex)
    c[np.arange(19), picks] = 1.0
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.normal(size=(19, 19)) + 1j * rng.normal(size=(19, 19)))
    g = ks.Grid(cell, prec="bf16x3")
    g.set_states(Q @ c)
    eps = g.block_iteration(1)
    assert np.allclose(eps, np.sort(0.5 * ref.g2[picks]), atol=2e-5)
    out = g.get_states()
    outside = np.delete(out, picks, axis=1)
    meas("np.max(np.abs(outside))", np.max(np.abs(outside)), 1e-5 * np.max(np.abs(out)))
    g.close()


def test_block_iteration_mixed_beyond_128_states(ks, meas):
    """150 states on the mixed path: the factor keeps the two-pass FP32 scheme (n <= 160) and
    the eigensolver falls back to FP64 Jacobi (n > 128)."""
    cell = inputs.small_cell(16.0, 48, 3, 150, 46, depth=-3.0)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec="bf16x3")
    c = inputs.random_coeffs(46, 150, ref.nG)
    g.set_states(c)
    eps = g.block_iteration(2)
    eps_ref, c_ref = ko.block_iteration(ref, c, 2)
    meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)), 1e-4 * max(1.0, np.max(np.abs(eps_ref))))
    q = g.get_states()
    s = ko.gram(q)
    # not orthonormal (the SD step follows the rotation), but Hermitian positive definite
    assert np.all(np.linalg.eigvalsh(0.5 * (s + s.conj().T)) > 0)
    g.close()


@pytest.mark.parametrize("n", [200, 256])
def test_mixed_subspace_129_to_256_states(ks, meas, n):
    """Blocks of 129-256 states on the mixed path: the FP32 Cholesky with its square array in
    global memory (n > 160) and the FP32 parallel Jacobi eigensolver (n > 128), finished by FP64
    refinement and FP64 Rayleigh quotients.  CholQR, Rayleigh-Ritz and two block iterations
    against the oracle at the mixed path's tolerances."""
    cell = inputs.small_cell(14.0, 32, 3, n, 70 + n, depth=-3.0)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec="bf16x3")
    c = inputs.random_coeffs(70 + n, n, ref.nG)
    g.set_states(c)
    S = g.orthonormalize(want_S=True)
    S_ref = ko.gram(c)
    meas("n=%d Gram S, max |d| / max |S|" % n, np.max(np.abs(S - S_ref)) / np.max(np.abs(S_ref)), 2e-5)
    q = g.get_states()
    meas("n=%d CholQR orthonormality" % n, np.max(np.abs(ko.gram(q) - np.eye(n))), 1e-4)
    eps = g.rayleigh_ritz()
    e_ref, _, _, _ = ko.rayleigh_ritz(q, ko.apply_h(ref, q))
    # FP32 H_sub entries carry ~1e-6 relative error of ||H||; an eigenvalue moves by at most the
    # 2-norm of the perturbation, ~sqrt(n) entry errors: the 12-state bound 2.5e-5 Ha scaled by
    # sqrt(n / 12) (measured 7.9e-6 at n = 12 and 4.0e-5 at n = 200, the same ratio)
    meas("n=%d Rayleigh-Ritz, max |d eps|" % n, np.max(np.abs(eps - e_ref)), 2.5e-5 * np.sqrt(n / 12.0))
    g.set_states(c)
    eps = g.block_iteration(2)
    eps_ref, _ = ko.block_iteration(ref, c, 2)
    meas("n=%d block iteration, max |d eps|" % n, np.max(np.abs(eps - eps_ref)),
         1e-4 * max(1.0, np.max(np.abs(eps_ref))))
    g.close()


# ------------------------------------------------------------------------------------------------
# Self-consistent field (Sec. "Ground-state solution"), linear mixing
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_scf_parity(ks, prec, meas):
    cell = inputs.small_cell(10.0, 24, 4, 8, 51, depth=-3.0)
    ref = ko.Cell(cell)
    c = inputs.random_coeffs(51, 8, ref.nG)
    eps_ref, res_ref, c_ref, _ = ko.scf(ref, c, 4, 2, 0.4)
    g = ks.Grid(cell, prec=prec)
    g.set_states(c)
    eps, res = g.scf(4, eig_iters=2, mix=0.4)
    assert eps.shape == eps_ref.shape and res.shape == res_ref.shape
    if prec == "fp64":
        meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)), 1e-12 * max(1.0, np.max(np.abs(eps_ref))))
        meas("np.max(np.abs(res - res_ref))", np.max(np.abs(res - res_ref)), 1e-12 * np.max(res_ref))
        meas("rel(g.get_states(), c_ref)", rel(g.get_states(), c_ref), 1e-12)
    else:
        meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)), 1e-4 * max(1.0, np.max(np.abs(eps_ref))))
        meas("np.max(np.abs(res - res_ref))", np.max(np.abs(res - res_ref)), 1e-3 * np.max(res_ref))
    # the states are orthonormal afterwards
    q = g.get_states()
    meas("np.max(np.abs(ko.gram(q) - np.eye(8)))", np.max(np.abs(ko.gram(q) - np.eye(8))), (1e-12 if prec == "fp64" else 1e-5))
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_scf_pulay_parity(ks, prec, meas):
    """Pulay mixing with a history of 3 pairs (so the ring of history slots wraps)."""
    cell = inputs.small_cell(10.0, 24, 4, 8, 58, depth=-3.0)
    ref = ko.Cell(cell)
    c = inputs.random_coeffs(58, 8, ref.nG)
    eps_ref, res_ref, _, _ = ko.scf(ref, c, 5, 2, 0.4, mixer="pulay", history=3)
    g = ks.Grid(cell, prec=prec)
    g.set_states(c)
    eps, res = g.scf(5, eig_iters=2, mix=0.4, mixer="pulay", history=3)
    if prec == "fp64":
        meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)), 1e-12 * max(1.0, np.max(np.abs(eps_ref))))
        meas("np.max(np.abs(res - res_ref))", np.max(np.abs(res - res_ref)), 1e-12 * np.max(res_ref))
    else:
        # the mixing coefficients come from differences of residuals, which amplifies the
        # single-precision error of the densities
        meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)), 1e-3 * max(1.0, np.max(np.abs(eps_ref))))
        meas("np.max(np.abs(res - res_ref))", np.max(np.abs(res - res_ref)), 1e-2 * np.max(res_ref))
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_scf_broyden_parity(ks, prec, meas):
    """Broyden mixing with a window of 3 pairs (the ring of history slots wraps), against the
    oracle's direct rank-one updates of the inverse Jacobian."""
    cell = inputs.small_cell(10.0, 24, 4, 8, 59, depth=-3.0)
    ref = ko.Cell(cell)
    c = inputs.random_coeffs(59, 8, ref.nG)
    eps_ref, res_ref, _, _ = ko.scf(ref, c, 6, 2, 0.4, mixer="broyden", history=3)
    g = ks.Grid(cell, prec=prec)
    g.set_states(c)
    eps, res = g.scf(6, eig_iters=2, mix=0.4, mixer="broyden", history=3)
    if prec == "fp64":
        meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)), 1e-12 * max(1.0, np.max(np.abs(eps_ref))))
        meas("np.max(np.abs(res - res_ref))", np.max(np.abs(res - res_ref)), 1e-12 * np.max(res_ref))
    else:
        # secant pairs are differences of densities and residuals, which amplifies the
        # single-precision error of the densities (as for Pulay mixing)
        meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)), 1e-3 * max(1.0, np.max(np.abs(eps_ref))))
        meas("np.max(np.abs(res - res_ref))", np.max(np.abs(res - res_ref)), 1e-2 * np.max(res_ref))
    g.close()


def test_scf_free_electron_fixed_point(ks):
    """Closed shells of free electrons: uniform density, so the SCF sits at its fixed point
    with Ritz values 1/2 |G|^2 + v_x(n0) (uniform-gas LDA exchange) and zero residual."""
    cell = inputs.small_cell(10.0, 24, 0, 7, 52)
    ref = ko.Cell(cell)
    picks = np.argsort(ref.g2)[:7]
    c = np.zeros((7, ref.nG), complex)
    c[np.arange(7), picks] = 1.0
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.normal(size=(7, 7)) + 1j * rng.normal(size=(7, 7)))
    rs = (3.0 / (4.0 * np.pi * 7.0 / ref.omega)) ** (1.0 / 3.0)
    vx = -0.610887 / rs
    for prec, tol in (("fp64", 1e-5), ("bf16x3", 3e-5)):
        g = ks.Grid(cell, prec=prec)
        g.set_states(Q @ c)
        eps, res = g.scf(2, eig_iters=1, mix=0.5)
        assert np.allclose(eps[-1], np.sort(0.5 * ref.g2[picks]) + vx, atol=tol)
        assert np.max(res) < (1e-12 if prec == "fp64" else 1e-5)
        g.close()


def test_scf_arguments_and_tolerance(ks):
    cell = inputs.small_cell(10.0, 24, 2, 4, 53)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec="bf16x3")
    g.set_states(inputs.random_coeffs(53, 4, ref.nG))
    for bad in (dict(eig_iters=0), dict(mix=0.0), dict(mix=1.5), dict(tol=-1.0), dict(mixer=3),
                dict(mixer="pulay", history=0), dict(mixer="pulay", history=9)):
        with pytest.raises(ks.KsError):
            g.scf(2, **bad)
    eps, res = g.scf(0)
    assert eps.shape == (0, 4) and res.shape == (0,)
    eps, res = g.scf(5, eig_iters=1, mix=0.5, tol=1e9)
    assert len(res) == 1
    g.close()


# ------------------------------------------------------------------------------------------------
# Delta kick and dipole (Sec. "Validation with other codes")
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_kick_and_dipole_parity(ks, prec, meas):
    cell = inputs.small_cell(10.0, 24, 3, 6, 56)
    ref = ko.Cell(cell)
    q, _ = ko.cholqr(inputs.random_coeffs(56, 6, ref.nG))
    kappa = (0.05, -0.03, 0.02)
    g = ks.Grid(cell, prec=prec)
    g.set_states(q)
    d0 = g.dipole()
    d0_ref = ko.dipole(ref, ko.density(ref, q))
    g.kick(kappa)
    got = g.get_states()
    kq = ko.kick(ref, q, kappa)
    if prec == "fp64":
        meas("rel(got, kq)", rel(got, kq), 1e-12)
        meas("np.max(np.abs(d0 - d0_ref))", np.max(np.abs(d0 - d0_ref)), 1e-12 * np.max(np.abs(d0_ref)))
    else:
        meas("rel(got, kq)", rel(got, kq), 2e-5)
        meas("np.max(np.abs(d0 - d0_ref))", np.max(np.abs(d0 - d0_ref)), 1e-5 * np.max(np.abs(d0_ref)))
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_td_dipole_after_kick_parity(ks, prec, meas):
    """Kick at t = 0, then ETRS steps with Hartree + exchange: the dipole at the start of
    every step against the oracle's."""
    cell = inputs.small_cell(10.0, 24, 3, 6, 57)
    ref = ko.Cell(cell)
    q, _ = ko.cholqr(inputs.random_coeffs(57, 6, ref.nG))
    kappa = (0.1, 0.0, 0.0)
    g = ks.Grid(cell, prec=prec)
    g.set_states(q)
    g.kick(kappa)
    norms, energies, dips = g.td_step(0.05, 4, "etrs", True, dipoles=True)
    _, n_ref, e_ref, d_ref = ko.td_run_dipole(ref, ko.kick(ref, q, kappa), 0.05, 4, "etrs", True)
    scale = np.max(np.abs(d_ref))
    if prec == "fp64":
        meas("np.max(np.abs(dips - d_ref))", np.max(np.abs(dips - d_ref)), 1e-12 * scale)
        meas("np.max(np.abs(norms - n_ref))", np.max(np.abs(norms - n_ref)), 1e-12 * n_ref[0])
    else:
        meas("np.max(np.abs(dips - d_ref))", np.max(np.abs(dips - d_ref)), 1e-5 * scale)
    # the dipole path adds no change to norms and energies
    g2 = ks.Grid(cell, prec=prec)
    g2.set_states(q)
    g2.kick(kappa)
    n2, e2 = g2.td_step(0.05, 4, "etrs", True)
    assert np.array_equal(n2, norms) and np.array_equal(e2, energies)
    g.close()
    g2.close()


# ------------------------------------------------------------------------------------------------
# Teter-preconditioned steepest descent (Sec. "Ground-state solution")
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_block_iteration_teter_parity(ks, prec, meas):
    cell = inputs.small_cell(12.0, 32, 4, 10, 59, depth=-3.0)
    ref = ko.Cell(cell)
    c = inputs.random_coeffs(59, 10, ref.nG)
    g = ks.Grid(cell, prec=prec)
    g.set_states(c)
    eps = g.block_iteration(6, precond="teter")
    eps_ref, c_ref = ko.block_iteration_teter(ref, c, 6)
    if prec == "fp64":
        meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)), 1e-12 * max(1.0, np.max(np.abs(eps_ref))))
        meas("rel(g.get_states(), c_ref)", rel(g.get_states(), c_ref), 1e-12)
    else:
        meas("np.max(np.abs(eps - eps_ref))", np.max(np.abs(eps - eps_ref)), 1e-4 * max(1.0, np.max(np.abs(eps_ref))))
    g.close()


def test_block_iteration_teter_free_electron_limit(ks):
    """No atoms: the preconditioned iteration reaches the G = 0 and |m| = 1 shells."""
    cell = inputs.small_cell(4.0, 12, 0, 7, 60)
    ref = ko.Cell(cell)
    c = inputs.random_coeffs(60, 7, ref.nG)
    for prec, tol in (("fp64", 1e-12), ("bf16x3", 2e-5)):
        g = ks.Grid(cell, prec=prec)
        g.set_states(c)
        eps = g.block_iteration(80, precond="teter")
        assert np.allclose(eps, np.sort(0.5 * ref.g2)[:7], atol=tol)
        g.close()


# ------------------------------------------------------------------------------------------------
# Forces from the orbital gradients (Sec. "Forces", Eq. 11)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_forces_parity(ks, prec, meas):
    cell = inputs.small_cell(10.0, 24, 3, 5, 63, depth=-3.0)
    occ = np.array([2.0, 2.0, 1.5, 1.0, 0.5])
    ref = ko.Cell(dict(cell, occ=occ))
    q, _ = ko.cholqr(inputs.random_coeffs(63, 5, ref.nG))
    q = ko.block_iteration(ref, q, 6)[1]
    g = ks.Grid(cell, prec=prec, occ=occ)
    g.set_states(q)
    F = g.forces()
    F_ref = ko.forces(ref, q)
    assert F.shape == (3, 3)
    scale = np.max(np.abs(F_ref))
    meas("np.max(np.abs(F - F_ref))", np.max(np.abs(F - F_ref)), (1e-12 if prec == "fp64" else 1e-4) * scale)
    g.close()


def test_forces_no_atoms(ks):
    cell = inputs.small_cell(10.0, 24, 0, 3, 64)
    ref = ko.Cell(cell)
    g = ks.Grid(cell, prec="bf16x3")
    g.set_states(inputs.random_coeffs(64, 3, ref.nG))
    assert g.forces().shape == (0, 3)
    g.close()


# ------------------------------------------------------------------------------------------------
# Moving atoms and Ehrenfest dynamics (Sec. "Real-time propagation")
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_set_positions_rebuilds_potential_and_projectors(ks, prec, meas):
    """After moving the atoms (one across the cell boundary, so that its projector sphere
    wraps), V_loc, H psi and the forces match an oracle cell built at the new positions."""
    cell = inputs.small_cell(10.0, 24, 3, 5, 65, depth=-3.0)
    moved = np.array(cell["pos"]) + np.array([[0.7, -0.4, 0.25], [-0.3, 0.9, -1.1], [0.05, 0.1, 0.2]])
    moved[0, 0] = 9.8                                                # next to the x = L face
    ref = ko.Cell(dict(cell, pos=moved))
    g = ks.Grid(cell, prec=prec)
    c = inputs.random_coeffs(65, 5, ref.nG)
    g.set_states(c)
    g.set_positions(moved)
    assert np.array_equal(g.positions(), moved)
    meas("np.max(np.abs(g.vloc() - ref.vloc))", np.max(np.abs(g.vloc() - ref.vloc)), 1e-13 * np.max(np.abs(ref.vloc)))
    got = apply_dev(ks, g, c, prec)
    expect = ko.apply_h(ref, c)
    for k in range(5):
        meas("rel(got[k], expect[k])", rel(got[k], expect[k]), TOL_H[prec])
    q = ko.block_iteration(ref, ko.cholqr(c)[0], 4)[1]
    g.set_states(q)
    F_ref = ko.forces(ref, q)
    meas("np.max(np.abs(g.forces() - F_ref))", np.max(np.abs(g.forces() - F_ref)), (1e-12 if prec == "fp64" else 1e-4) * np.max(np.abs(F_ref)))
    with pytest.raises(ks.KsError):
        g.set_positions(np.full((3, 3), np.nan))
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_ehrenfest_parity(ks, prec, meas):
    """Three Ehrenfest steps with Hartree and exchange against the oracle: positions,
    velocities, total energies and states."""
    desc = dict(L=8.0, N=24, ecut=20.0, pos=np.array([[2.0, 2.5, 3.0], [5.5, 4.0, 4.5]]), vloc_depth=-3.0,
                vloc_width=0.8, nproj=4, proj_sigma=0.5, proj_rc=2.0, proj_D=0.5, nstates=4)
    ref = ko.Cell(desc)
    c = ko.cholqr(ko.block_iteration(ref, inputs.random_coeffs(66, 4, ref.nG), 10)[1])[0]
    mass = np.array([20.0, 30.0])
    v0 = np.array([[0.05, 0.0, -0.03], [-0.03, 0.04, 0.0]])
    c_ref, P_ref, V_ref, E_ref = ko.ehrenfest_run(desc, c, 0.1, 3, mass, v0)
    g = ks.Grid(desc, prec=prec)
    g.set_states(c)
    P, V, E = g.ehrenfest(0.1, 3, mass, v0)
    dtol = 1e-12 if prec == "fp64" else 1e-5
    meas("np.max(np.abs(P - P_ref))", np.max(np.abs(P - P_ref)), dtol * np.max(np.abs(P_ref - desc["pos"])))
    meas("np.max(np.abs(V - V_ref[-1]))", np.max(np.abs(V - V_ref[-1])), (1e-12 if prec == "fp64" else 1e-4) * np.max(np.abs(V_ref[-1])))
    meas("np.max(np.abs(E - E_ref))", np.max(np.abs(E - E_ref)), (1e-12 if prec == "fp64" else 1e-4) * np.max(np.abs(E_ref)))
    meas("rel(g.get_states(), c_ref)", rel(g.get_states(), c_ref), (1e-12 if prec == "fp64" else 1e-4))
    assert np.array_equal(g.positions(), P[-1])
    g.close()


def test_ehrenfest_immobile_ions_match_td_step(ks, meas):
    """Masses so large that the ions stay put: the same norms, energies and states as the
    plain real-time steps (V_loc is recomputed on the device each step: equal to rounding)."""
    desc = dict(L=8.0, N=24, ecut=20.0, pos=np.array([[2.0, 2.5, 3.0], [5.5, 4.0, 4.5]]), vloc_depth=-3.0,
                vloc_width=0.8, nproj=4, proj_sigma=0.5, proj_rc=2.0, proj_D=0.5, nstates=4)
    ref = ko.Cell(desc)
    c = ko.cholqr(inputs.random_coeffs(67, 4, ref.nG))[0]
    a = ks.Grid(desc, prec="fp64")
    b = ks.Grid(desc, prec="fp64")
    a.set_states(c)
    b.set_states(c)
    P, V, E = a.ehrenfest(0.05, 3, [1e300, 1e300], np.zeros((2, 3)))
    _, e = b.td_step(0.05, 3)
    assert np.array_equal(P[-1], desc["pos"]) and np.max(np.abs(V)) < 1e-250
    meas("np.max(np.abs(E - e))", np.max(np.abs(E - e)), 1e-12 * np.max(np.abs(e)))
    meas("rel(a.get_states(), b.get_states())", rel(a.get_states(), b.get_states()), 1e-12)
    for bad in (dict(dt=0.0), dict(nsteps=-1), dict(mass=[1.0, -1.0]), dict(mass=[1.0, np.inf])):
        kw = dict(dt=0.05, nsteps=1, mass=[1.0, 1.0], vel=np.zeros((2, 3)))
        kw.update(bad)
        with pytest.raises(ks.KsError):
            a.ehrenfest(**kw)
    a.close()
    b.close()


def test_moved_atoms_and_forces_full_size_sampled(ks, meas):
    """The gs96 cell (96^3, 128 states, 64 atoms) with every atom displaced: H psi of sampled
    states after ks_set_positions, and the forces of one occupied state (occupations pick the
    state whose forces the oracle computes), against an oracle cell built at the new
    positions."""
    cell, _ = oracle_cell("gs96")
    rng = np.random.default_rng(cell["seed"] + 7)
    moved = np.asarray(cell["pos"]) + rng.normal(scale=0.3, size=np.shape(cell["pos"]))
    ref = ko.Cell(dict(cell, pos=moved))
    occ = np.zeros(cell["nstates"])
    occ[5] = 1.0
    g = ks.Grid(cell, prec="bf16x3", occ=occ)
    c = inputs.random_coeffs(cell["seed"], cell["nstates"], ref.nG)
    g.set_states(c)
    g.set_positions(moved)
    got = apply_dev(ks, g, c, "bf16x3")
    for k in (5, 127):
        e = ko.apply_h(ref, c[k:k + 1])[0]
        meas("rel(got[k], e)", rel(got[k], e), TOL_H["bf16x3"])
    g.set_states(c)
    F = g.forces()
    F_ref = ko.forces(ref, c[5:6])
    meas("np.max(np.abs(F - F_ref))", np.max(np.abs(F - F_ref)), 1e-4 * np.max(np.abs(F_ref)))
    g.close()
