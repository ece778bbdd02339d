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
