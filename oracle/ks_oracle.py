"""Plain FP64 CPU oracle for the Kohn-Sham hot path (arXiv 2106.03872, "INQ").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA path (no kernels, headers, tables or helpers) and imports nothing from
the package; it is written for a reader checking it against the paper by eye,
not for speed.

What it computes, each function citing the paper passage it follows:

* own mixed-radix (2, 3) Cooley-Tukey FFT (the paper only says FFTs move between
  the real-space grid and the plane-wave basis, Sec. "DFT and TDDFT implementation");
* the plane-wave cutoff sphere, V_loc on the grid and the real-space projector
  spheres (Sec. "Pseudopotentials", Eq. 9);
* H psi = P_S (T + V + V_NL) P_S psi (Eq. 2, Sec. "Implementation of the KS Hamiltonian");
* the density n = sum_k f_k |phi_k|^2 (Eq. 1);
* Gram matrix, CholQR orthonormalisation and Rayleigh-Ritz rotation (Sec. "Ground-state solution");
* one steepest-descent block iteration (Sec. "Ground-state solution");
* periodic Poisson solve in Fourier space (Sec. "Poisson solver") and LDA Slater exchange;
* the total energy with eigenvalues replaced by expectation values (Eq. 5);
* the ETRS propagator with the 4th-order Taylor exponential and shared powers
  (Eqs. 6-8, Sec. "Real-time propagation");
* SCF density mixing (linear, Pulay, Broyden), Teter-preconditioned steepest descent, the
  delta kick and dipole, forces from the orbital gradients (Eq. 11) and Ehrenfest dynamics
  with velocity-Verlet ions.

Conventions where the paper is silent (each one a reading of it):
cubic cell of side L, grid N^3, r_j = h j, h = L/N; G = (2 pi / L) m with
m = j for j < N/2 else j - N; S = {G : |G|^2/2 <= E_cut} in grid-index order
(j_x, j_y, j_z) row-major, z fastest; psi(r_j) = Omega^{-1/2} sum_{G in S} c_G e^{i G.r_j};
c_G[f] = Omega^{1/2} N^{-3} sum_j e^{-i G.r_j} f(r_j).

Parity: every function here is pinned by ``tests/test_oracle_*.py`` except the
multi-iteration ground-state loop, whose converged eigenvalues have no external
truth beyond the free-electron limit ("parity unpinned" beyond that limit).
"""
import numpy as np

TWO_PI = 2.0 * np.pi


# ----------------------------------------------------------------------------------------------
# FFT: recursive decimation in time, radix 2 or 3, along the last axis.
# ----------------------------------------------------------------------------------------------
def fft_last_axis(x, sign):
    """Unnormalised DFT along the last axis: X[k] = sum_j x[j] exp(sign * 2 pi i j k / n).

    Decimation in time: split x into r interleaved subsequences x[q::r], transform each
    (length m = n/r), then X[k] = sum_q exp(sign 2 pi i q k / n) Y_q[k mod m].
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    if n == 1:
        return x.copy()
    if n % 2 == 0:
        r = 2
    elif n % 3 == 0:
        r = 3
    else:
        raise ValueError("oracle FFT supports lengths 2^a 3^b only, got %d" % n)
    m = n // r
    k = np.arange(n)
    out = np.zeros(x.shape, dtype=np.complex128)
    for q in range(r):
        yq = fft_last_axis(x[..., q::r], sign)           # [..., m]
        twiddle = np.exp(sign * 1j * TWO_PI * q * k / n)  # [n]
        out += twiddle * yq[..., k % m]
    return out


def fft_axis(x, axis, sign):
    return np.moveaxis(fft_last_axis(np.moveaxis(x, axis, -1), sign), -1, axis)


def fft3(x, sign):
    """Unnormalised 3D DFT over the last three axes, exponent sign ``sign``."""
    y = fft_axis(x, -1, sign)
    y = fft_axis(y, -2, sign)
    return fft_axis(y, -3, sign)


# ----------------------------------------------------------------------------------------------
# Geometry: cutoff sphere, local potential, projector spheres
# ----------------------------------------------------------------------------------------------
def integer_frequencies(N):
    """m_i = j_i for j_i < N/2 else j_i - N (FFT order)."""
    j = np.arange(N)
    return np.where(j < N / 2.0, j, j - N)


class Cell:
    """Everything the Hamiltonian needs for one periodic cubic cell.

    Built from the same plain dict that ``paper_2106_03872_gb300.inputs`` produces:
    L, N, ecut, pos [natoms,3], vloc_depth, vloc_width, nproj (1 or 4), proj_sigma,
    proj_rc, proj_D, optional occ [nstates].
    """

    def __init__(self, desc):
        self.L = float(desc["L"])
        self.N = int(desc["N"])
        self.ecut = float(desc["ecut"])
        self.pos = np.asarray(desc["pos"], float).reshape(-1, 3)
        self.natoms = len(self.pos)
        self.depth = float(desc["vloc_depth"])
        self.width = float(desc["vloc_width"])
        self.nproj = int(desc["nproj"])
        self.sigma_b = float(desc["proj_sigma"])
        self.rc = float(desc["proj_rc"])
        self.D = float(desc["proj_D"])
        self.occ = desc.get("occ")
        N, L = self.N, self.L
        self.h = L / N
        self.omega = L ** 3
        self.dV = self.omega / N ** 3
        self.build_sphere()
        self.vloc = self.local_potential()
        self.build_projectors()

    # -- Plane-wave basis: S = {G : |G|^2 / 2 <= E_cut} ------------------------------------
    def build_sphere(self):
        N = self.N
        m = integer_frequencies(N)
        mx, my, mz = np.meshgrid(m, m, m, indexing="ij")            # [jx, jy, jz]
        m2 = (mx ** 2 + my ** 2 + mz ** 2).ravel()
        g2_all = (TWO_PI / self.L) ** 2 * m2
        self.g2_full = g2_all.reshape(N, N, N)
        keep = 0.5 * g2_all <= self.ecut
        self.sphere_index = np.flatnonzero(keep)                    # row-major, z fastest
        self.m = np.stack([mx.ravel(), my.ravel(), mz.ravel()], axis=1)[self.sphere_index]
        self.g2 = g2_all[self.sphere_index]
        self.nG = len(self.sphere_index)

    def grid_points(self):
        j = np.arange(self.N) * self.h
        x, y, z = np.meshgrid(j, j, j, indexing="ij")
        return np.stack([x, y, z], axis=-1)                          # [N,N,N,3]

    # -- V_loc(r) = sum_a A exp(-|r - R_a - L n|^2 / (2 w^2)), 27 image shifts n -------------
    def local_potential(self):
        """Each Gaussian is evaluated in its separable form
        exp(-|d|^2/(2w^2)) = prod_axis exp(-d_axis^2/(2w^2))."""
        x = np.arange(self.N) * self.h
        v = np.zeros((self.N,) * 3)
        shifts = [np.array([a, b, c], float) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
        for R in self.pos:
            for s in shifts:
                C = R + self.L * s
                gx, gy, gz = (np.exp(-(x - C[k]) ** 2 / (2.0 * self.width ** 2)) for k in range(3))
                v += self.depth * gx[:, None, None] * gy[None, :, None] * gz[None, None, :]
        return v

    # -- KB projectors on the real-space sphere |r - R_I| < R_c (Eq. 9) ----------------------
    def build_projectors(self):
        """Per atom: flat grid indices inside the sphere (grid order) and beta [nproj, npts],
        s: exp(-d^2/(2 sigma^2)); p_alpha: d_alpha exp(-d^2/(2 sigma^2)); each normalised
        so that dV sum_j beta(r_j)^2 = 1.  d is the minimum-image displacement."""
        r = self.grid_points().reshape(-1, 3)
        self.proj_index, self.proj_beta = [], []
        for R in self.pos:
            d = r - R
            d -= self.L * np.round(d / self.L)
            d2 = np.sum(d * d, axis=1)
            inside = np.flatnonzero(d2 < self.rc ** 2)
            dd = d[inside]
            g = np.exp(-d2[inside] / (2.0 * self.sigma_b ** 2))
            rows = [g] if self.nproj == 1 else [g, dd[:, 0] * g, dd[:, 1] * g, dd[:, 2] * g]
            beta = np.array([b / np.sqrt(self.dV * np.sum(b * b)) for b in rows])
            self.proj_index.append(inside)
            self.proj_beta.append(beta)

    def occupations(self, nstates):
        if self.occ is None:
            return np.ones(nstates)
        return np.asarray(self.occ, float)[:nstates]

    def sd_step_length(self):
        """alpha = 1/(E_cut + (max V_loc - min V_loc) + D): bounds the steepest-descent
        update factor of every eigencomponent to [0, 1) (a reading; the paper gives no step)."""
        return 1.0 / (self.ecut + (self.vloc.max() - self.vloc.min()) + self.D)


# ----------------------------------------------------------------------------------------------
# Basis changes
# ----------------------------------------------------------------------------------------------
def to_real(cell, c):
    """psi(r_j) = Omega^{-1/2} sum_{G in S} c_G exp(i G.r_j); c [n, nG] -> [n, N, N, N]."""
    c = np.atleast_2d(c)
    N = cell.N
    grid = np.zeros((c.shape[0], N ** 3), dtype=np.complex128)
    grid[:, cell.sphere_index] = c
    return fft3(grid.reshape(-1, N, N, N), +1) / np.sqrt(cell.omega)


def to_coeff(cell, f):
    """c_G = Omega^{1/2} N^{-3} sum_j exp(-i G.r_j) f(r_j), kept on S; [n,N,N,N] -> [n, nG]."""
    N = cell.N
    F = fft3(np.asarray(f, dtype=np.complex128).reshape(-1, N, N, N), -1)
    return F.reshape(-1, N ** 3)[:, cell.sphere_index] * np.sqrt(cell.omega) / N ** 3


# ----------------------------------------------------------------------------------------------
# Hamiltonian application (Eq. 2; kinetic in Fourier space, local and nonlocal in real space)
# ----------------------------------------------------------------------------------------------
def nonlocal_projections(cell, psi_r):
    """p[k, I, l] = dV sum_{|r_j - R_I| < R_c} beta_Il(r_j) psi_k(r_j)  (the integral of Eq. 9)."""
    flat = psi_r.reshape(psi_r.shape[0], -1)
    p = np.zeros((flat.shape[0], cell.natoms, cell.nproj), dtype=np.complex128)
    for I in range(cell.natoms):
        vals = flat[:, cell.proj_index[I]]
        p[:, I, :] = cell.dV * vals @ cell.proj_beta[I].T
    return p


def apply_nonlocal(cell, psi_r):
    """V_NL psi(r) = sum_I sum_l D beta_Il(r) p_Il (Eq. 9 with KB coupling D), atoms in index order."""
    p = nonlocal_projections(cell, psi_r)
    out = np.zeros((psi_r.shape[0], cell.N ** 3), dtype=np.complex128)
    for I in range(cell.natoms):
        out[:, cell.proj_index[I]] += cell.D * p[:, I, :] @ cell.proj_beta[I]
    return out.reshape(psi_r.shape)


def apply_h(cell, c, v=None):
    """H c = P_S (T + V + V_NL) P_S c for a block c [n, nG].

    Steps as the paper describes them: transform to the real-space grid, apply the
    multiplicative potential v (default V_loc) and the nonlocal projectors there,
    transform back, keep G in S, and add the kinetic term |G|^2/2 (diagonal in
    Fourier space)."""
    c = np.atleast_2d(np.asarray(c, dtype=np.complex128))
    v = cell.vloc if v is None else v
    psi = to_real(cell, c)
    u = v[None] * psi + apply_nonlocal(cell, psi)
    return to_coeff(cell, u) + 0.5 * cell.g2[None, :] * c


# ----------------------------------------------------------------------------------------------
# Density (Eq. 1)
# ----------------------------------------------------------------------------------------------
def density(cell, c, occ=None):
    """n(r_j) = sum_k f_k |psi_k(r_j)|^2, shape [N, N, N] in grid order (x, y, z)."""
    c = np.atleast_2d(c)
    f = cell.occupations(c.shape[0]) if occ is None else np.asarray(occ, float)
    psi = to_real(cell, c)
    return np.einsum("k,kxyz->xyz", f, np.abs(psi) ** 2)


# ----------------------------------------------------------------------------------------------
# Rotations in state space (Sec. "Ground-state solution": orthogonalisation and subspace diagonalisation)
# ----------------------------------------------------------------------------------------------
def gram(a, b=None):
    """S_ij = sum_G conj(a_iG) b_jG  (S = Psi^H Psi for b = a)."""
    b = a if b is None else b
    return np.conj(a) @ b.T


def cholqr(c, S=None):
    """Orthonormalise the rows of c: S = L L^H, Psi <- Psi L^{-H} (rows: c <- conj(L^{-1}) c).
    S defaults to gram(c); a given S (e.g. one computed elsewhere in lower precision) is
    factored as is."""
    S = gram(c) if S is None else S
    L = np.linalg.cholesky(S)
    return np.conj(np.linalg.inv(L)) @ c, S


def fix_phases(U):
    """Make the largest-magnitude component of each column real and positive (lowest index on ties)."""
    U = U.copy()
    for j in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, j])))
        U[:, j] *= np.conj(U[i, j]) / abs(U[i, j])
    return U


def rayleigh_ritz(c, hc):
    """H_sub = Psi^H (H Psi), eigen-decomposed; returns (eps ascending, U, c U, (Hc) U)."""
    Hs = gram(c, hc)
    Hs = 0.5 * (Hs + np.conj(Hs.T))
    eps, U = np.linalg.eigh(Hs)
    U = fix_phases(U)
    return eps, U, U.T @ c, U.T @ hc


def block_iteration(cell, c, niter, v=None):
    """Steepest-descent block iteration (Sec. "Ground-state solution"), per iteration:
    CholQR -> H Psi -> Rayleigh-Ritz -> R = H Psi - Psi diag(eps) -> Psi <- Psi - alpha R.
    Returns (eps of the last Rayleigh-Ritz, final c)."""
    alpha = cell.sd_step_length()
    eps = None
    for _ in range(niter):
        c, _ = cholqr(c)
        hc = apply_h(cell, c, v)
        eps, _, c, hc = rayleigh_ritz(c, hc)
        c = c - alpha * (hc - eps[:, None] * c)
    return eps, c


def teter_factor(x):
    """Teter-Payne-Allan preconditioner (the paper's SD preconditioner, applied in Fourier
    space): K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4), with x the
    plane wave's kinetic energy over that of the residual vector it multiplies."""
    p = 27.0 + 18.0 * x + 12.0 * x ** 2 + 8.0 * x ** 3
    return p / (p + 16.0 * x ** 4)


def block_iteration_teter(cell, c, niter, v=None):
    """Preconditioned steepest descent (Sec. "Ground-state solution"), per iteration:
    CholQR -> H Psi -> Rayleigh-Ritz -> R = H Psi - Psi diag(eps) -> for each state i, with
    T_i = sum_G |G|^2/2 |R_iG|^2 / sum_G |R_iG|^2 the kinetic energy of its residual vector,
    floored at that of the smallest nonzero plane wave, (2 pi / L)^2 / 2 (a residual with
    weight at G = 0 only would give T_i = 0),
    c_iG <- c_iG - alpha_i K(|G|^2 / (2 T_i)) R_iG, alpha_i = 1 / (T_i + max V_loc - min V_loc + D)
    (a state with R_i = 0 is left as it is).  Returns (eps of the last Rayleigh-Ritz, final c)."""
    dv = float(cell.vloc.max() - cell.vloc.min())
    eps = None
    for _ in range(niter):
        c, _ = cholqr(c)
        hc = apply_h(cell, c, v)
        eps, _, c, hc = rayleigh_ritz(c, hc)
        R = hc - eps[:, None] * c
        r2 = np.real(np.sum(np.abs(R) ** 2, axis=1))
        tr = np.real(np.sum(0.5 * cell.g2[None, :] * np.abs(R) ** 2, axis=1))
        live = r2 > 0
        tmin = 0.5 * (2.0 * np.pi / cell.L) ** 2
        t = np.maximum(np.where(live, tr / np.where(live, r2, 1.0), tmin), tmin)
        alpha = np.where(live, 1.0 / (t + dv + cell.D), 0.0)
        K = teter_factor(0.5 * cell.g2[None, :] / t[:, None])
        c = c - alpha[:, None] * K * R
    return eps, c


# ----------------------------------------------------------------------------------------------
# Hartree (Sec. "Poisson solver", periodic) and LDA Slater exchange
# ----------------------------------------------------------------------------------------------
def hartree(cell, n):
    """v_H(G) = 4 pi n(G) / |G|^2 on the full grid, v_H(G=0) = 0 (neutralising background)."""
    N = cell.N
    nG = fft3(n.astype(np.complex128), -1) / N ** 3
    g2 = cell.g2_full
    vG = np.zeros_like(nG)
    nz = g2 > 0
    vG[nz] = 4.0 * np.pi * nG[nz] / g2[nz]
    return np.real(fft3(vG, +1))


def slater(n):
    """Dirac/Slater exchange: v_x = -(3 n / pi)^{1/3}, eps_x = -3/4 (3 n / pi)^{1/3}; n clamped at 0."""
    nn = np.maximum(n, 0.0)
    vx = -np.cbrt(3.0 * nn / np.pi)
    return vx, 0.75 * vx


def hxc_potential(cell, n):
    """V = V_loc + v_H[n] + v_x[n]; also returns the double-counting pieces for Eq. 5."""
    vh = hartree(cell, n)
    vx, ex = slater(n)
    dV = cell.dV
    parts = dict(eh=0.5 * dV * np.sum(n * vh), ex=dV * np.sum(n * ex), nvx=dV * np.sum(n * vx))
    return cell.vloc + vh + vx, parts


def pulay_coefficients(A):
    """alpha minimising || sum_i alpha_i R_i ||^2 subject to sum_i alpha_i = 1, from the Gram
    matrix A_ij = <R_i|R_j> (Pulay / DIIS): the bordered system [A 1; 1^T 0] [alpha; mu] =
    [0; 1], with A regularised by 1e-12 of its mean diagonal."""
    m = A.shape[0]
    reg = 1e-12 * max(np.trace(A) / m, 1e-300)
    B = np.zeros((m + 1, m + 1))
    B[:m, :m] = A + reg * np.eye(m)
    B[:m, m] = 1.0
    B[m, :m] = 1.0
    rhs = np.zeros(m + 1)
    rhs[m] = 1.0
    return np.linalg.solve(B, rhs)[:m]


def broyden_apply(dx, dF, beta, v):
    """G v for the approximate inverse Jacobian G of Broyden's second method (Broyden 1965,
    the method that updates the inverse directly; the paper names Broyden mixing as its
    default in Sec. "Ground-state solution").  G starts from -beta I and takes the secant
    pairs (dx_j, dF_j) in order, each a rank-one update
        G_{j+1} = G_j + (dx_j - G_j dF_j) dF_j^T / (dF_j^T dF_j),
    which makes G_{j+1} dF_j = dx_j and leaves G unchanged on vectors orthogonal to dF_j.
    Dot products are dV sums over the grid.  A pair with dF_j = 0 carries no information and
    is skipped."""
    us, ds = [], []
    for j in range(len(dF)):
        g = -beta * dF[j]                                 # G_j dF_j from the updates before j
        for u, d, f in zip(us, ds, dF[:j]):
            g = g + u * (float(np.sum(f * dF[j])) / d)
        dd = float(np.sum(dF[j] * dF[j]))
        us.append(dx[j] - g)
        ds.append(dd if dd > 0.0 else np.inf)
    out = -beta * v
    for u, d, f in zip(us, ds, dF):
        out = out + u * (float(np.sum(f * v)) / d)
    return out


def scf(cell, c, max_iter, eig_iters, mix, tol=0.0, mixer="linear", history=4):
    """Self-consistent field (Sec. "Ground-state solution"): each iteration solves the
    linear problem for the current input density with a few eigensolver iterations, forms
    the output density and mixes it into the input.

    The initial input density is that of the orthonormalised initial states (the paper
    starts from atomic densities of pseudopotential files, which this setting has none of).
    Per iteration: V = V_loc + v_H[n_in] + v_x[n_in]; eig_iters block iterations; CholQR;
    n_out = density; R = n_out - n_in, r = dV sum |R|; then
      linear: n_in <- n_in + mix R;
      pulay:  with the last `history` pairs (n_in_i, R_i) and alpha from pulay_coefficients
              of A_ij = dV sum R_i R_j, n_in <- sum_i alpha_i (n_in_i + mix R_i);
      broyden: the root of R(n_in) by Broyden's second method over the last `history` pairs:
              n_in <- n_in - G R with G from broyden_apply, started at -mix I and updated by
              the secant pairs (n_in_{i+1} - n_in_i, R_{i+1} - R_i) of the window in order
              (history 1 is linear mixing).
    Stops once r < tol.  Returns (Ritz values per iteration, residuals, states, final n_in)."""
    c, _ = cholqr(c)
    n_in = density(cell, c)
    eps_hist, res_hist = [], []
    hist_n, hist_r = [], []
    for _ in range(max_iter):
        v, _ = hxc_potential(cell, n_in)
        eps, c = block_iteration(cell, c, eig_iters, v)
        c, _ = cholqr(c)
        n_out = density(cell, c)
        R = n_out - n_in
        r = cell.dV * float(np.sum(np.abs(R)))
        eps_hist.append(eps)
        res_hist.append(r)
        if mixer == "linear":
            n_next = n_in + mix * R
        elif mixer == "broyden":
            hist_n.append(n_in)
            hist_r.append(R)
            hist_n, hist_r = hist_n[-history:], hist_r[-history:]
            dx = [b - a for a, b in zip(hist_n[:-1], hist_n[1:])]
            dF = [b - a for a, b in zip(hist_r[:-1], hist_r[1:])]
            n_next = n_in - broyden_apply(dx, dF, mix, R)
        else:
            hist_n.append(n_in)
            hist_r.append(R)
            hist_n, hist_r = hist_n[-history:], hist_r[-history:]
            A = np.array([[cell.dV * float(np.sum(a * b)) for b in hist_r] for a in hist_r])
            alpha = pulay_coefficients(A)
            n_next = sum(a * (n + mix * rr) for a, n, rr in zip(alpha, hist_n, hist_r))
        n_in = n_next
        if r < tol:
            break
    return np.array(eps_hist), np.array(res_hist), c, n_in


def total_energy(cell, c, hc, parts=None):
    """E = sum_k f_k <psi_k|H|psi_k> - 1/2 int n v_H + E_x - int n v_x (Eq. 5, eigenvalues
    replaced by expectation values).  Without Hartree/exchange only the first term remains."""
    f = cell.occupations(c.shape[0])
    band = float(np.sum(f * np.real(np.sum(np.conj(c) * hc, axis=1))))
    if parts is None:
        return band
    return band - parts["eh"] + parts["ex"] - parts["nvx"]


def total_norm(cell, c):
    f = cell.occupations(c.shape[0])
    return float(np.sum(f * np.sum(np.abs(c) ** 2, axis=1)))


# ----------------------------------------------------------------------------------------------
# Real-time propagation: ETRS with a 4th-order Taylor exponential, shared powers (Eqs. 6-8)
# ----------------------------------------------------------------------------------------------
TAYLOR_ORDER = 4


def taylor_coefficients(lam):
    """a_k = lam^k / k!, k = 0..4 (Eq. 8)."""
    a, out = 1.0 + 0j, []
    for k in range(TAYLOR_ORDER + 1):
        out.append(a)
        a = a * lam / (k + 1)
    return out


def potential_for(cell, c, hartree_xc):
    if not hartree_xc:
        return cell.vloc, None
    return hxc_potential(cell, density(cell, c))


def td_step(cell, c, dt, propagator="etrs", hartree_xc=True, next_cell=None):
    """One real-time step from t to t + dt; returns (c(t+dt), norm(t), energy(t)).

    ETRS (Eq. 6): phi(t+dt) = exp(-i dt/2 H(t+dt)) exp(-i dt/2 H(t)) phi(t), with
    H(t+dt) built from the density of the full step exp(-i dt H(t)) phi(t) (Eq. 7).
    The powers H(t)^k phi are computed once and combined with both coefficient sets
    lam = -i dt and lam = -i dt/2 (the shared-power saving).  'taylor' is the plain
    4th-order step phi <- sum_k (-i dt H(t))^k / k! phi.
    With moving ions, next_cell holds the ions at t + dt: H(t+dt) takes its local potential
    and projectors (the ionic potential evaluated at the time of the half step it acts in).
    """
    v_t, parts = potential_for(cell, c, hartree_xc)
    powers = [c]
    for _ in range(TAYLOR_ORDER):
        powers.append(apply_h(cell, powers[-1], v_t))
    norm_t = total_norm(cell, c)
    energy_t = total_energy(cell, c, powers[1], parts)
    full = sum(a * w for a, w in zip(taylor_coefficients(-1j * dt), powers))
    if propagator == "taylor":
        return full, norm_t, energy_t
    half = sum(a * w for a, w in zip(taylor_coefficients(-0.5j * dt), powers))
    cell2 = cell if next_cell is None else next_cell
    v_next, _ = potential_for(cell2, full, hartree_xc)
    out, w = half.copy(), half
    for a in taylor_coefficients(-0.5j * dt)[1:]:
        w = apply_h(cell2, w, v_next)
        out = out + a * w
    return out, norm_t, energy_t


def atom_potential(cell, R):
    """The local potential of one atom at R: A sum_{27 images} exp(-|r - R - L n|^2 / (2 w^2))."""
    x = np.arange(cell.N) * cell.h
    v = np.zeros((cell.N,) * 3)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            for cc in (-1, 0, 1):
                C = R + cell.L * np.array([a, b, cc], float)
                gx, gy, gz = (np.exp(-(x - C[k]) ** 2 / (2.0 * cell.width ** 2)) for k in range(3))
                v += cell.depth * gx[:, None, None] * gy[None, :, None] * gz[None, None, :]
    return v


def forces(cell, c):
    """Forces on the atoms from the orbital gradients (Eq. 11), F_I = -sum_k f_k
    [<grad phi_k| v_I |phi_k> + c.c.], v_I the local and KB nonlocal potential of atom I; the
    overall sign is that of -dE/dR_I (the printed Eqs. 10-11 carry the opposite one).
    Local part: -dV sum_j v_I(r_j) g(r_j), g = sum_k f_k 2 Re(conj(grad phi_k) phi_k) on the grid.
    Nonlocal part: -sum_k f_k sum_l 2 D Re(conj(q_Il) p_Il), p_Il = <beta_Il|phi_k> and
    q_Il = <beta_Il|grad phi_k> on the grid; grad phi from i G c_G.  Returns [natoms, 3]."""
    c = np.atleast_2d(c)
    f = cell.occupations(c.shape[0])
    psi = to_real(cell, c)
    G = 2.0 * np.pi / cell.L * cell.m
    grads = [to_real(cell, 1j * G[None, :, a] * c) for a in range(3)]
    p = nonlocal_projections(cell, psi)
    F = np.zeros((cell.natoms, 3))
    for a in range(3):
        g = np.einsum("k,kxyz->xyz", f, 2.0 * np.real(np.conj(grads[a]) * psi))
        for I, R in enumerate(cell.pos):
            F[I, a] -= cell.dV * np.sum(atom_potential(cell, R) * g)
        if cell.natoms:
            q = nonlocal_projections(cell, grads[a])
            F[:, a] -= np.einsum("k,kil->i", f, 2.0 * cell.D * np.real(np.conj(q) * p))
    return F


def kick(cell, c, kappa):
    """Delta kick (Sec. "Validation with other codes", a time-localised field at t = 0):
    psi(r) <- exp(i kappa . (r - L/2)) psi(r) on the grid, then back to the sphere S."""
    r = cell.grid_points()
    phase = np.exp(1j * np.tensordot(r - 0.5 * cell.L, np.asarray(kappa, float), axes=([3], [0])))
    return to_coeff(cell, phase[None] * to_real(cell, c))


def dipole(cell, n):
    """First moment of the density, d = dV sum_j (r_j - L/2) n(r_j)."""
    r = cell.grid_points()
    return cell.dV * np.tensordot(r - 0.5 * cell.L, n, axes=([0, 1, 2], [0, 1, 2]))


def td_run_dipole(cell, c, dt, nsteps, propagator="etrs", hartree_xc=True):
    """td_run that also returns the dipole of the density at the start of every step."""
    norms, energies, dips = [], [], []
    for _ in range(nsteps):
        dips.append(dipole(cell, density(cell, c)))
        c, nrm, e = td_step(cell, c, dt, propagator, hartree_xc)
        norms.append(nrm)
        energies.append(e)
    return c, np.array(norms), np.array(energies), np.array(dips)


def ehrenfest_run(desc, c, dt, nsteps, mass, vel, hartree_xc=True):
    """Ehrenfest dynamics (Sec. "Real-time propagation"): the electrons follow the ETRS step
    and the ions classical equations of motion under the forces of Eq. 11, integrated by
    velocity Verlet, with the ionic potential of H(t+dt) taken at the new positions:
      R(t+dt) = R(t) + v(t) dt + F(t) dt^2 / (2M);
      phi(t+dt) = ETRS step with H(t) at R(t) and H(t+dt) at R(t+dt);
      F(t+dt) = forces of phi(t+dt) at R(t+dt);  v(t+dt) = v(t) + (F(t) + F(t+dt)) dt / (2M).
    desc is the cell dict at the initial positions, mass [natoms] (electron masses), vel
    [natoms, 3] the initial velocities (bohr per atomic time unit).  Returns (c, positions
    [nsteps, natoms, 3] after each step, velocities [nsteps, natoms, 3] after each step,
    energies [nsteps]: electronic energy of Eq. 5 (as in td_step) plus the ionic kinetic energy
    sum 1/2 M v^2, both at the start of each step)."""
    M = np.asarray(mass, float)[:, None]
    v = np.array(vel, float).reshape(-1, 3)
    d = dict(desc)
    cell = Cell(d)
    F = forces(cell, c)
    pos_h, vel_h, e_h = [], [], []
    for _ in range(nsteps):
        kin = float(np.sum(0.5 * M * v * v))
        R1 = cell.pos + v * dt + F * dt * dt / (2.0 * M)
        d = dict(d, pos=R1)
        cell1 = Cell(d)
        c, _, e_el = td_step(cell, c, dt, "etrs", hartree_xc, next_cell=cell1)
        F1 = forces(cell1, c)
        v = v + (F + F1) * dt / (2.0 * M)
        cell, F = cell1, F1
        pos_h.append(cell.pos.copy())
        vel_h.append(v.copy())
        e_h.append(e_el + kin)
    return c, np.array(pos_h), np.array(vel_h), np.array(e_h)


def td_run(cell, c, dt, nsteps, propagator="etrs", hartree_xc=True):
    norms, energies = [], []
    for _ in range(nsteps):
        c, nrm, e = td_step(cell, c, dt, propagator, hartree_xc)
        norms.append(nrm)
        energies.append(e)
    return c, np.array(norms), np.array(energies)
