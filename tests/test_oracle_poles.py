"""Pins for the continued-fraction pole set (Eq. 7) of the oracle."""
import numpy as np
import pytest

from oracle.poles import cf_poles, fermi_from_poles, cf_fermi_truncated, fermi_exact, pole_weights


@pytest.mark.parametrize("M", [1, 2, 5, 10, 40, 80, 160])
def test_pole_form_equals_printed_fraction(M):
    # Eq. (7): the pole sum must reproduce the printed continued fraction truncated after
    # the denominator 4M-1, evaluated independently by backward recurrence.
    z, R = cf_poles(M)
    assert z.shape == (M,) and R.shape == (M,)
    x = np.concatenate([np.linspace(-60, 60, 4001), np.linspace(-2000, 2000, 4001)])
    a = fermi_from_poles(x, z, R)
    b = cf_fermi_truncated(x, 2 * M)
    assert np.max(np.abs(a - b)) < 1e-14


def test_matsubara_limit():
    # The lowest poles approach the Matsubara frequencies (2k-1) pi with residue -1
    # (the paper: "located on the imaginary axis like the Matsubara pole").
    z, R = cf_poles(80)
    k = np.arange(1, 6)
    assert np.allclose(z[:5], (2 * k - 1) * np.pi, rtol=0, atol=1e-12)
    assert np.allclose(R[:5], -1.0, rtol=0, atol=1e-12)
    assert np.all(R < 0) and np.all(np.diff(z) > 0)
    # and the density of poles thins out away from the real axis
    gaps = np.diff(z)
    assert gaps[-1] > 10 * gaps[0]


@pytest.mark.parametrize("M,xmax", [(40, 300.0), (80, 1000.0), (160, 1500.0)])
def test_fermi_exact_within_range(M, xmax):
    # Sec. II.B: a modest pole count is numerically exact in double precision.
    z, R = cf_poles(M)
    x = np.linspace(-xmax, xmax, 20001)
    assert np.max(np.abs(fermi_from_poles(x, z, R) - fermi_exact(x))) < 1e-13


def test_fermi_symmetry_and_half():
    z, R = cf_poles(40)
    x = np.linspace(0, 80, 801)
    fp = fermi_from_poles(x, z, R)
    fm = fermi_from_poles(-x, z, R)
    assert np.max(np.abs(fp + fm - 1.0)) < 1e-15
    assert abs(fermi_from_poles(np.array([0.0]), z, R)[0] - 0.5) < 1e-16


def test_pole_weights_sign():
    alpha, w = pole_weights(mu=-0.2, kT=0.01, M=10)
    assert np.all(alpha.real == -0.2)
    assert np.all(alpha.imag > 0)
    assert np.all(w > 0)          # w_p = -4 R_p / beta with R_p < 0


def test_hundred_poles_at_600_kelvin_are_exact():
    # Sec. II.B: 100 poles at 600 K reproduce the Fermi function to double precision over the
    # energies of a valence spectrum (here |E - mu| <= 1.5 Hartree)
    kT = 600.0 * 3.166811563e-6            # k_B in Hartree per kelvin
    z, R = cf_poles(100)
    x = np.linspace(-1.5, 1.5, 40001) / kT
    assert np.max(np.abs(fermi_from_poles(x, z, R) - fermi_exact(x))) < 1e-14


def test_pole_count_does_not_depend_on_size():
    # Sec. II.B: the truncation error of the M-pole expansion is set by the spectral range and kT,
    # not by the number of states: the same M serves a chain of 40 and of 400 sites
    from oracle.closed_form import chain_spectrum, chain_density
    from oracle.dense import occupation
    errs = {}
    for N in (40, 400):
        for M in (10, 20):
            kw = dict(N=N, a=0.0, b=-1.0, s=0.1, mu=0.05, kT=0.01)
            rM, _ = chain_density(occupation=lambda x, m, t, M=M: occupation(x, m, t, M), **kw)
            rX, _ = chain_density(occupation=lambda x, m, t: occupation(x, m, t, None), **kw)
            errs[(N, M)] = np.max(np.abs(rM - rX))
    for M in (10, 20):
        ratio = errs[(400, M)] / errs[(40, M)]
        assert 0.2 < ratio < 5.0, (M, errs)
    assert errs[(40, 20)] < errs[(40, 10)]
