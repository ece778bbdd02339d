"""Pins for the oracle's density of states from the retarded Green function (Eq. 41).

D(E) = -(2/pi) Im Tr(G(E + i eta) S).  Routes: Eq. (41) with dense inverses, the Lorentzian sum
over LAPACK eigenvalues, the open-chain closed-form spectrum, a one-orbital system by hand, and
the sum rule (the integral of each Lorentzian is known in closed form).
"""
import numpy as np

from synth import chain_nntb, lattice_system
from oracle.closed_form import chain_spectrum
from oracle.dense import generalized_eig, dos_eig, dos_inv


def test_single_orbital_by_hand():
    # H = [h], S = [s]: Tr(G S) = s / (z s - h) = 1 / (z - h/s)
    h, s, eta = -0.3, 1.7, 0.05
    E = np.array([-0.5, h / s, 0.4])
    d = dos_inv(np.array([[h]]), np.array([[s]]), E, eta)
    want = (2.0 / np.pi) * eta / ((E - h / s) ** 2 + eta ** 2)
    assert np.max(np.abs(d - want)) < 1e-13 * np.max(want)


def test_chain_closed_form():
    N, a, b, s = 30, 0.1, -0.8, 0.15
    Hd, Sd = chain_nntb(N, a, b, s).dense()
    eps, _ = chain_spectrum(N, a, b, s)
    E = np.linspace(-2.5, 2.5, 41)
    eta = 0.07
    d = dos_inv(Hd, Sd, E, eta)
    d_cf = dos_eig(eps, E, eta)
    assert np.max(np.abs(d - d_cf)) < 1e-11 * np.max(d_cf)
    assert np.all(d > 0)


def test_routes_agree_on_lattice():
    sysm = lattice_system((4, 3, 1), 2, "2d", 23)
    Hd, Sd = sysm.dense()
    eps, _ = generalized_eig(Hd, Sd)
    E = np.linspace(eps[0] - 0.3, eps[-1] + 0.3, 25)
    for eta in (0.01, 0.2):
        d1, d2 = dos_eig(eps, E, eta), dos_inv(Hd, Sd, E, eta)
        assert np.max(np.abs(d1 - d2)) < 1e-10 * np.max(d1)


def test_sum_rule():
    # integral over [lo, hi] = sum_nu (2/pi)(atan((hi - eps)/eta) - atan((lo - eps)/eta)) -> 2N
    sysm = lattice_system((3, 3, 1), 2, "2d", 24)
    Hd, Sd = sysm.dense()
    eps, _ = generalized_eig(Hd, Sd)
    eta, lo, hi = 0.1, eps[0] - 5.0, eps[-1] + 5.0
    E = np.linspace(lo, hi, 8001)
    d = dos_inv(Hd, Sd, E, eta)
    integral = np.sum(0.5 * (d[1:] + d[:-1]) * np.diff(E))
    exact = np.sum((2.0 / np.pi) * (np.arctan((hi - eps) / eta) - np.arctan((lo - eps) / eta)))
    assert abs(integral - exact) < 1e-4 * exact
    assert abs(exact - 2 * sysm.n) < 0.05 * sysm.n


def test_planted_mistake_trace_without_S():
    # Tr(G) in place of Tr(G S) is wrong when S != I: the closed form catches it
    N, a, b, s = 20, 0.0, -1.0, 0.2
    Hd, Sd = chain_nntb(N, a, b, s).dense()
    eps, _ = chain_spectrum(N, a, b, s)
    E, eta = np.linspace(-2, 2, 9), 0.1
    wrong = np.array([-(2.0 / np.pi) * np.imag(np.trace(np.linalg.inv((e + 1j * eta) * Sd - Hd))) for e in E])
    assert np.max(np.abs(wrong - dos_eig(eps, E, eta))) > 1e-2 * np.max(dos_eig(eps, E, eta))
