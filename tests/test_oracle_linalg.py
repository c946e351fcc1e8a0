"""Pins for the oracle's density, CholQR, Rayleigh-Ritz and block iteration (CPU only)."""
import numpy as np

from oracle import ks_oracle as ko
from paper_2106_03872_gb300 import inputs


def make_cell(L=10.0, N=24, natoms=4, depth=-2.0, seed=11, ecut=20.0, D=0.5):
    pos = inputs.uniform_positions(seed, natoms, L)
    return ko.Cell(dict(L=L, N=N, ecut=ecut, pos=pos, vloc_depth=depth, vloc_width=0.8, nproj=4,
                        proj_sigma=0.5, proj_rc=2.0, proj_D=D))


def mgs(c):
    """Modified Gram-Schmidt on the rows of c."""
    q = c.astype(complex).copy()
    for i in range(q.shape[0]):
        for j in range(i):
            q[i] -= (np.vdot(q[j], q[i])) * q[j]
        q[i] /= np.linalg.norm(q[i])
    return q


def test_cholqr_orthonormal_and_unique():
    cell = make_cell()
    c = inputs.random_coeffs(1, 9, cell.nG)
    q, S = ko.cholqr(c)
    assert np.max(np.abs(ko.gram(q) - np.eye(9))) <= 1e-13
    assert np.max(np.abs(q - mgs(c))) <= 1e-12
    assert np.allclose(S, np.conj(S.T))


def test_density_integrates_to_occupations_and_plane_wave_uniform():
    cell = make_cell()
    c, _ = ko.cholqr(inputs.random_coeffs(2, 5, cell.nG))
    n = ko.density(cell, c)
    assert abs(cell.dV * n.sum() - 5.0) < 1e-12
    occ = np.array([2.0, 1.0, 0.5, 0.0, 1.0])
    assert abs(cell.dV * ko.density(cell, c, occ).sum() - occ.sum()) < 1e-12
    pw = np.zeros((1, cell.nG), complex)
    pw[0, 17] = 1.0
    assert np.max(np.abs(ko.density(cell, pw) - 1.0 / cell.omega)) < 1e-15


def test_rayleigh_ritz_recovers_exact_eigenvalues_of_invariant_subspace():
    cell = make_cell(natoms=0)
    picks = [0, 5, 40, 300, 2000]
    c = np.zeros((5, cell.nG), complex)
    for r, k in enumerate(picks):
        c[r, k] = 1.0
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5)))
    mixed = Q @ c
    eps, U, c2, hc2 = ko.rayleigh_ritz(mixed, ko.apply_h(cell, mixed))
    assert np.allclose(eps, np.sort(0.5 * cell.g2[picks]), atol=1e-12)
    assert np.allclose(hc2, eps[:, None] * c2, atol=1e-12)
    for j in range(5):                                   # phase convention
        i = np.argmax(np.abs(U[:, j]))
        assert abs(U[i, j].imag) < 1e-15 and U[i, j].real > 0


def test_block_iteration_free_electron_limit():
    """V_loc = 0, D = 0: the lowest 7 eigenvalues are the G = 0 and |m| = 1 shells."""
    cell = make_cell(L=4.0, N=12, natoms=0, ecut=20.0)
    c = inputs.random_coeffs(3, 7, cell.nG)
    eps, c = ko.block_iteration(cell, c, 250)
    shells = np.sort(0.5 * cell.g2)[:7]
    assert np.allclose(eps, shells, atol=1e-9)


def test_block_iteration_lowers_ritz_values():
    cell = make_cell(natoms=4, depth=-3.0)
    c = inputs.random_coeffs(5, 6, cell.nG)
    e1, c1 = ko.block_iteration(cell, c, 2)
    e2, _ = ko.block_iteration(cell, c1, 10)
    assert np.all(e2 <= e1 + 1e-12)


def test_scf_free_electron_closed_shell_is_a_fixed_point():
    """V_loc = 0, no projectors, the 7 plane waves of the G = 0 and |m| = 1 shells mixed by a
    random unitary: the density is uniform, n0 = 7 / Omega, so v_H = 0 and v_x is the
    uniform-gas value -0.610887 / r_s (textbook LDA exchange, r_s = (3 / (4 pi n0))^(1/3)).
    The SCF is at its fixed point: Ritz values 1/2 |G|^2 + v_x, density residual 0."""
    cell = make_cell(natoms=0)
    picks = np.argsort(cell.g2)[:7]
    assert np.allclose(np.sort(cell.g2[picks])[1:], cell.g2[picks].max())
    c = np.zeros((7, cell.nG), complex)
    c[np.arange(7), picks] = 1.0
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.normal(size=(7, 7)) + 1j * rng.normal(size=(7, 7)))
    eps, res, _, n_in = ko.scf(cell, Q @ c, 2, 1, 0.5)
    rs = (3.0 / (4.0 * np.pi * 7.0 / cell.omega)) ** (1.0 / 3.0)
    vx = -0.610887 / rs
    assert np.allclose(eps[-1], np.sort(0.5 * cell.g2[picks]) + vx, atol=1e-5)
    assert np.max(res) < 1e-12
    assert np.allclose(n_in, 7.0 / cell.omega, atol=1e-13)


def test_scf_residual_contracts_and_tolerance_stops():
    """From random states the residual is dominated by the unconverged eigenvectors at
    first; after a few iterations each SCF step shrinks it.  The tolerance stops the loop
    at the first iteration whose residual is below it, with the same history."""
    cell = make_cell(natoms=4, depth=-3.0)
    c = inputs.random_coeffs(9, 6, cell.nG)
    eps, res, c_out, _ = ko.scf(cell, c, 12, 5, 0.3)
    assert len(res) == 12
    assert np.all(np.diff(res[4:]) < 0)
    assert res[-1] < 0.6 * res[0]
    assert np.max(np.abs(ko.gram(c_out) - np.eye(6))) <= 1e-12
    eps2, res2, _, _ = ko.scf(cell, c, 12, 5, 0.3, tol=res[6] * 1.0000001)
    assert len(res2) == 7 and np.allclose(res2, res[:7]) and np.allclose(eps2, eps[:7])


def test_pulay_coefficients_closed_forms():
    """Two residuals R and -R: the combination 1/2 R + 1/2 (-R) = 0 is the minimiser.  Two
    orthogonal residuals of squared norms a and b: alpha = (b, a) / (a + b) (the weighted
    minimum of alpha_1^2 a + alpha_2^2 b on alpha_1 + alpha_2 = 1)."""
    A = np.array([[2.0, -2.0], [-2.0, 2.0]])
    assert np.allclose(ko.pulay_coefficients(A), [0.5, 0.5], atol=1e-6)
    a, b = 3.0, 0.5
    assert np.allclose(ko.pulay_coefficients(np.diag([a, b])), [b / (a + b), a / (a + b)], atol=1e-10)


def test_scf_pulay_with_one_pair_is_linear_and_converges_faster():
    """History 1 reduces Pulay mixing to linear mixing (alpha = 1); with history 4 the
    residual falls below linear mixing's after the same number of iterations."""
    cell = make_cell(natoms=4, depth=-3.0)
    c = inputs.random_coeffs(9, 6, cell.nG)
    e_lin, r_lin, _, _ = ko.scf(cell, c, 5, 5, 0.3)
    e_p1, r_p1, _, _ = ko.scf(cell, c, 5, 5, 0.3, mixer="pulay", history=1)
    assert np.allclose(r_p1, r_lin, rtol=1e-10) and np.allclose(e_p1, e_lin, atol=1e-10)
    _, r_lin12, _, _ = ko.scf(cell, c, 12, 5, 0.3)
    _, r_p4, _, _ = ko.scf(cell, c, 12, 5, 0.3, mixer="pulay", history=4)
    assert r_p4[-1] < r_lin12[-1]


def _secant_pairs(rng, d, m):
    return ([rng.standard_normal(d) for _ in range(m)], [rng.standard_normal(d) for _ in range(m)])


def test_broyden_update_secant_condition_and_invariance():
    """Broyden's second method: after the update with the pair (dx, dF), G dF = dx (the
    secant condition), and on every vector orthogonal to dF the new G acts as the previous
    one.  The two properties fix a rank-one update uniquely."""
    rng = np.random.default_rng(5)
    d, beta = 7, 0.3
    dx, dF = _secant_pairs(rng, d, 3)
    for m in (1, 2, 3):
        g = ko.broyden_apply(dx[:m], dF[:m], beta, dF[m - 1])
        assert np.allclose(g, dx[m - 1], rtol=0, atol=1e-12)
        v = rng.standard_normal(d)
        v -= dF[m - 1] * (np.dot(dF[m - 1], v) / np.dot(dF[m - 1], dF[m - 1]))
        prev = ko.broyden_apply(dx[:m - 1], dF[:m - 1], beta, v)
        assert np.allclose(ko.broyden_apply(dx[:m], dF[:m], beta, v), prev, rtol=0, atol=1e-12)
    # no pairs: linear mixing; a zero dF carries no update
    v = rng.standard_normal(d)
    assert np.array_equal(ko.broyden_apply([], [], beta, v), -beta * v)
    assert np.allclose(ko.broyden_apply([dx[0]], [np.zeros(d)], beta, v), -beta * v, atol=0)


def test_broyden_in_one_dimension_is_the_secant_method():
    """For a scalar equation f(x) = 0 the window of the last two pairs turns the Broyden step
    into the secant method x+ = x - f(x) (x - x_prev) / (f(x) - f(x_prev)); on 2 - x^3 (a
    decreasing residual, like a density residual) it converges superlinearly to 2^(1/3)."""
    f = lambda x: 2.0 - x ** 3
    beta = 0.1
    xs = [np.array([1.0])]
    xs.append(xs[0] - ko.broyden_apply([], [], beta, f(xs[0])))     # first step: linear
    assert np.isclose(xs[1][0], 1.1, rtol=0, atol=1e-15)
    for _ in range(8):
        x0, x1 = xs[-2], xs[-1]
        step = ko.broyden_apply([x1 - x0], [f(x1) - f(x0)], beta, f(x1))
        secant = f(x1) * (x1 - x0) / (f(x1) - f(x0))
        assert np.allclose(step, secant, rtol=1e-12, atol=0)
        xs.append(x1 - step)
        if abs(f(xs[-1])[0]) < 1e-14:
            break
    assert abs(xs[-1][0] - 2.0 ** (1.0 / 3.0)) < 1e-12
    assert len(xs) <= 10


def test_scf_broyden_with_one_pair_is_linear_and_converges_faster():
    """History 1 leaves no secant pair, so Broyden mixing is linear mixing; with history 4 the
    residual falls below linear mixing's after the same number of iterations."""
    cell = make_cell(natoms=4, depth=-3.0)
    c = inputs.random_coeffs(9, 6, cell.nG)
    e_lin, r_lin, _, _ = ko.scf(cell, c, 5, 5, 0.3)
    e_b1, r_b1, _, _ = ko.scf(cell, c, 5, 5, 0.3, mixer="broyden", history=1)
    assert np.allclose(r_b1, r_lin, rtol=1e-10) and np.allclose(e_b1, e_lin, atol=1e-10)
    _, r_lin12, _, _ = ko.scf(cell, c, 12, 5, 0.3)
    _, r_b4, _, _ = ko.scf(cell, c, 12, 5, 0.3, mixer="broyden", history=4)
    assert r_b4[-1] < r_lin12[-1]


def test_teter_block_iteration_free_electron_fixed_points_and_limit():
    """The preconditioner changes no fixed point: the free-electron limit still converges to
    the G = 0 and |m| = 1 shells."""
    cell = make_cell(L=4.0, N=12, natoms=0, ecut=20.0)
    c = inputs.random_coeffs(3, 7, cell.nG)
    eps, _ = ko.block_iteration_teter(cell, c, 80)
    assert np.allclose(eps, np.sort(0.5 * cell.g2)[:7], atol=1e-12)


def test_teter_preconditioning_converges_faster():
    """With atoms: after the same number of iterations the preconditioned Ritz values lie
    below the plain steepest-descent ones (Ritz values bound the eigenvalues from above)."""
    cell = make_cell(natoms=4, depth=-3.0)
    c = inputs.random_coeffs(5, 6, cell.nG)
    e_sd, _ = ko.block_iteration(cell, c, 15)
    e_pc, _ = ko.block_iteration_teter(cell, c, 15)
    assert np.sum(e_pc) < np.sum(e_sd) - 1e-3
    e_pc2, _ = ko.block_iteration_teter(cell, c, 30)
    assert np.all(e_pc2 <= e_pc + 1e-9)


def test_teter_factor_series_limits_and_exact_values():
    """K(x) of Teter, Payne and Allan, pinned by what its rational form fixes independently of
    the code: K(x) = 1 - (16/27) x^4 + O(x^5) near 0 (so its first three derivatives vanish
    there); x K(x) -> 1/2 as x -> infinity; and the exact values K(1/2) = 40/41, K(1) = 65/81,
    K(2) = 175/431 worked out by hand from 27 + 18x + 12x^2 + 8x^3 over the same plus 16x^4.
    A wrong coefficient anywhere fails one of them: the series fixes 27 and 16, the limit 8/16,
    the three exact values the x and x^2 terms."""
    for x in (1e-2, 2e-2):
        q = (ko.teter_factor(x) - 1.0) / x ** 4
        assert abs(q + 16.0 / 27.0) <= (16.0 / 27.0) * 1.0 * x          # next term is O(x)
    # finite differences at 0: K'(0) = K''(0) = K'''(0) = 0 (each estimate is O(h) from x^4)
    h = 1e-2
    k = [ko.teter_factor(j * h) for j in range(-2, 3)]
    d1 = (k[3] - k[1]) / (2 * h)
    d2 = (k[3] - 2 * k[2] + k[1]) / h ** 2
    d3 = (k[4] - 2 * k[3] + 2 * k[1] - k[0]) / (2 * h ** 3)
    assert abs(d1) < 1e-5 and abs(d2) < 1e-3 and abs(d3) < 0.1
    for x in (1e3, 1e5):
        assert abs(x * ko.teter_factor(x) - 0.5) <= 1.0 / x
    assert abs(ko.teter_factor(0.5) - 40.0 / 41.0) <= 1e-15
    assert abs(ko.teter_factor(1.0) - 65.0 / 81.0) <= 1e-15
    assert abs(ko.teter_factor(2.0) - 175.0 / 431.0) <= 1e-15
    assert ko.teter_factor(0.0) == 1.0
    xs = np.linspace(0.0, 50.0, 2001)
    ks = ko.teter_factor(xs)
    assert np.all(np.diff(ks) < 0) and np.all(ks > 0)


def _two_wave_state(cell, m1, m2):
    i1 = int(np.flatnonzero(np.all(cell.m == m1, axis=1))[0])
    i2 = int(np.flatnonzero(np.all(cell.m == m2, axis=1))[0])
    c = np.zeros((1, cell.nG), complex)
    c[0, i1] = c[0, i2] = 1.0 / np.sqrt(2.0)
    return c, i1, i2


def test_teter_step_hand_computed():
    """One preconditioned step of one free-electron state made of two plane waves (L = 2 pi, so
    |G|^2/2 = |m|^2/2; V_loc = 0; D = 0.5), worked out by hand:
    - waves m = 0 and (1,0,0): eps = 1/4, R = (-1/4, +1/4)/sqrt2, T = 1/4 is floored at
      (2 pi / L)^2 / 2 = 1/2, alpha = 1/(1/2 + 1/2) = 1, K(0) = 1 and K(1) = 65/81, so the new
      coefficients are (1 + 1/4)/sqrt2 and (1 - (65/81)/4)/sqrt2 = (259/324)/sqrt2;
    - waves (1,0,0) and (2,0,0): eps = 5/4, R = (-3/4, +3/4)/sqrt2, T = (1/2 + 2)/2 = 5/4,
      alpha = 1/(5/4 + 1/2) = 4/7, x = 2/5 and 8/5 with K = 22895/23151 and 74555/140091."""
    cell = make_cell(L=2.0 * np.pi, N=8, natoms=0, ecut=2.5)
    c, i1, i2 = _two_wave_state(cell, (0, 0, 0), (1, 0, 0))
    eps, out = ko.block_iteration_teter(cell, c, 1)
    assert abs(eps[0] - 0.25) <= 1e-14
    s = 1.0 / np.sqrt(2.0)
    assert abs(out[0, i1] - 1.25 * s) <= 1e-14
    assert abs(out[0, i2] - (259.0 / 324.0) * s) <= 1e-14
    assert np.max(np.abs(np.delete(out[0], [i1, i2]))) <= 1e-14
    c, i1, i2 = _two_wave_state(cell, (1, 0, 0), (2, 0, 0))
    eps, out = ko.block_iteration_teter(cell, c, 1)
    assert abs(eps[0] - 1.25) <= 1e-14
    a = 4.0 / 7.0
    assert abs(out[0, i1] - (1.0 + a * (22895.0 / 23151.0) * 0.75) * s) <= 1e-14
    assert abs(out[0, i2] - (1.0 - a * (74555.0 / 140091.0) * 0.75) * s) <= 1e-14
