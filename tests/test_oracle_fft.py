"""Pins for the oracle's own FFT and basis changes (CPU only).

The oracle's FFT is checked against a brute-force 3D DFT (a direct sum over all
grid points with the full 3D phase, no separability), Parseval, the inverse
relation and numpy's library FFT.
"""
import numpy as np
import pytest

from oracle import ks_oracle as ko


def brute_dft3(x, sign):
    N = x.shape[-1]
    j = np.arange(N)
    J = np.stack(np.meshgrid(j, j, j, indexing="ij"), -1).reshape(-1, 3)
    phase = np.exp(sign * 2j * np.pi * (J @ J.T) / N)              # [k, j]
    return (phase @ x.reshape(-1)).reshape(N, N, N)


@pytest.mark.parametrize("N", [6, 8, 12])
@pytest.mark.parametrize("sign", [-1, +1])
def test_fft3_matches_bruteforce(N, sign):
    rng = np.random.default_rng(N)
    x = rng.normal(size=(N, N, N)) + 1j * rng.normal(size=(N, N, N))
    ref = brute_dft3(x, sign)
    got = ko.fft3(x, sign)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 9, 16, 24, 96, 128])
def test_fft_1d_matches_library(n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=(3, n)) + 1j * rng.normal(size=(3, n))
    assert np.allclose(ko.fft_last_axis(x, -1), np.fft.fft(x, axis=-1), rtol=0, atol=1e-12 * n)
    assert np.allclose(ko.fft_last_axis(x, +1), n * np.fft.ifft(x, axis=-1), rtol=0, atol=1e-12 * n)


def test_fft_rejects_other_radices():
    with pytest.raises(ValueError):
        ko.fft_last_axis(np.ones(5), -1)


@pytest.mark.parametrize("N", [8, 24])
def test_parseval_and_inverse(N):
    rng = np.random.default_rng(7)
    x = rng.normal(size=(2, N, N, N)) + 1j * rng.normal(size=(2, N, N, N))
    X = ko.fft3(x, -1)
    assert np.allclose(np.sum(np.abs(X) ** 2), N ** 3 * np.sum(np.abs(x) ** 2), rtol=1e-13)
    back = ko.fft3(X, +1) / N ** 3
    assert np.max(np.abs(back - x)) < 1e-13 * np.max(np.abs(x)) * 10


def free_cell(L=10.0, N=24, ecut=20.0):
    return ko.Cell(dict(L=L, N=N, ecut=ecut, pos=np.zeros((0, 3)), vloc_depth=0.0, vloc_width=0.8,
                        nproj=4, proj_sigma=0.5, proj_rc=2.0, proj_D=0.5))


def count_sphere_points(L, N, ecut):
    """Independent count of integer vectors m with (2 pi/L)^2 |m|^2 / 2 <= ecut and |m_i| < N/2
    (lattice points in a ball, by rows)."""
    bound = 2.0 * ecut * (L / (2 * np.pi)) ** 2
    mmax = int(np.floor(np.sqrt(bound)))
    assert mmax < N // 2
    total = 0
    for mx in range(-mmax, mmax + 1):
        for my in range(-mmax, mmax + 1):
            rest = bound - mx * mx - my * my
            if rest >= 0:
                total += 2 * int(np.floor(np.sqrt(rest) + 1e-12)) + 1
    return total


@pytest.mark.parametrize("L,N,expected", [(10.0, 24, 4337), (30.0, 96, 115313), (40.0, 128, 273425),
                                          (20.0, 64, None), (15.0, 48, 14363)])
def test_sphere_counts(L, N, expected):
    ref = count_sphere_points(L, N, 20.0)
    if expected is not None:
        assert ref == expected
    if N <= 64:
        cell = free_cell(L, N)
        assert cell.nG == ref
        assert np.all(np.diff(cell.sphere_index) > 0)        # canonical grid order
        assert np.all(0.5 * cell.g2 <= 20.0)


def test_plane_wave_real_space_and_roundtrip():
    cell = free_cell(10.0, 24)
    rng = np.random.default_rng(3)
    k = 1234
    c = np.zeros((1, cell.nG), complex)
    c[0, k] = 1.0
    psi = ko.to_real(cell, c)[0]
    G = 2 * np.pi / cell.L * cell.m[k]
    r = cell.grid_points()
    direct = np.exp(1j * (r @ G)) / np.sqrt(cell.omega)
    assert np.max(np.abs(psi - direct)) < 1e-13
    c = rng.normal(size=(3, cell.nG)) + 1j * rng.normal(size=(3, cell.nG))
    psi = ko.to_real(cell, c)
    assert np.allclose(cell.dV * np.sum(np.abs(psi) ** 2, axis=(1, 2, 3)), np.sum(np.abs(c) ** 2, axis=1),
                       rtol=1e-13)
    assert np.max(np.abs(ko.to_coeff(cell, psi) - c)) < 1e-13 * np.max(np.abs(c))
