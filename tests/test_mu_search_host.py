"""The chemical-potential search logic (Sec. II.C.3) on the host, driven by the oracle.

ndsi_mu_search runs the same search as ndsi_find_mu over caller-supplied DeltaN(mu) and density
of states; here both come from the oracle's eigenvalues (Eq. 40 with the M-pole Fermi function,
Eq. 41's Lorentzian sum), so the root, the evaluation counts and the error paths are checked
without a GPU.
"""
import numpy as np
import pytest

from synth import config_system, lattice_system
from oracle.dense import generalized_eig, occupation, find_mu_eig, dos_eig
from tests.libtools import lib
from paper_1005_0088_gb300.ndsi import NDSI_ERR_INVALID


def _problem(sysm, kT, M):
    Hd, Sd = sysm.dense()
    eps, _ = generalized_eig(Hd, Sd)
    H, S = np.abs(Hd), np.abs(Sd)
    hd, sd = np.diag(Hd), np.diag(Sd)
    hr, sr = H.sum(1) - np.abs(hd), S.sum(1) - np.abs(sd)
    hlo, hhi = (hd - hr).min(), (hd + hr).max()
    slo, shi = (sd - sr).min(), (sd + sr).max()
    elo = hlo / (slo if hlo < 0 else shi)
    ehi = hhi / (slo if hhi > 0 else shi)
    ne = sysm.n_electrons
    calls = []

    def dn(mu):
        calls.append(mu)
        return float(np.sum(occupation(eps, mu, kT, M))) - ne

    return eps, elo, ehi, ne, dn, calls


@pytest.mark.parametrize("with_dos", [True, False])
def test_unbracketed_search_converges(with_dos):
    sysm = config_system("C1")
    kT, M = sysm.meta["kT"], sysm.meta["poles"]
    eps, elo, ehi, ne, dn, calls = _problem(sysm, kT, M)
    nd = lib()
    dos = (lambda E, eta: dos_eig(eps, E, eta)) if with_dos else None
    mu, d, evals = nd.ndsi_mu_search(dn, elo, ehi, kT, ne, dos=dos, n_grid=M + 1)
    print(f"C1 unbracketed, dos={with_dos}: {evals} evaluations")
    assert abs(d) < 1e-8
    assert abs(mu - find_mu_eig(eps, kT, ne, M)) < 1e-9
    assert evals == len(calls) + (1 if with_dos else 0)
    assert evals <= (10 if with_dos else 14)


def test_seeded_and_wrong_brackets():
    sysm = lattice_system((10, 10, 1), 3, "2d", 808)
    kT, M = 0.01, 40
    eps, elo, ehi, ne, dn, calls = _problem(sysm, kT, M)
    mu_ref = find_mu_eig(eps, kT, ne, M)
    nd = lib()
    mu, d, near = nd.ndsi_mu_search(dn, elo, ehi, kT, ne, mu_lo=mu_ref - 0.02, mu_hi=mu_ref + 0.03)
    assert abs(d) < 1e-8 and near <= 8
    mu, d, wide = nd.ndsi_mu_search(dn, elo, ehi, kT, ne, mu_lo=elo, mu_hi=ehi)
    assert abs(d) < 1e-8 and wide <= 16
    mu, d, wrong = nd.ndsi_mu_search(dn, elo, ehi, kT, ne, mu_lo=mu_ref + 0.2, mu_hi=mu_ref + 0.3)
    assert abs(d) < 1e-8 and abs(mu - mu_ref) < 1e-9
    print(f"near bracket {near}, spectral bounds {wide}, wrong bracket {wrong} evaluations")


def test_no_root_and_timeout():
    sysm = lattice_system((4, 4, 1), 2, "2d", 3)
    kT, M = 0.01, 20
    eps, elo, ehi, ne, dn, calls = _problem(sysm, kT, M)
    nd = lib()
    too_many = lambda mu: float(np.sum(occupation(eps, mu, kT, M))) - 3.0 * sysm.n   # noqa: E731
    with pytest.raises(nd.NdsiError) as e:
        nd.ndsi_mu_search(too_many, elo, ehi, kT, 3.0 * sysm.n)
    assert e.value.code == NDSI_ERR_INVALID
    with pytest.raises(nd.NdsiError) as e:
        nd.ndsi_mu_search(dn, elo, ehi, kT, ne, max_iter=2)
    mu, d, evals = e.value.result
    assert evals == 2 and np.isfinite(mu)


def test_callback_error_stops_search():
    nd = lib()

    def bad(mu):
        raise ValueError("evaluation failed")

    with pytest.raises(ValueError):
        nd.ndsi_mu_search(bad, -1.0, 1.0, 0.01, 1.0)


def test_batched_lockstep_matches_single_searches():
    # four systems searched in lockstep: every mu matches its own search, one callback per round
    systems = [lattice_system((6, 5, 1), 2, "2d", 90 + i) for i in range(3)] + [config_system("C1")]
    kTs = [0.01, 0.02, 0.005, 0.01]
    probs = [_problem(s, kT, 40) for s, kT in zip(systems, kTs)]
    nd = lib()
    eps = [p[0] for p in probs]
    elo = [p[1] for p in probs]
    ehi = [p[2] for p in probs]
    ne = [p[3] for p in probs]
    calls = []

    def delta_n(mu, active):
        calls.append(active.copy())
        return [float(np.sum(occupation(e, m, kT, 40))) - n for e, m, kT, n in zip(eps, mu, kTs, ne)]

    def dos(E, eta, active):
        return np.stack([dos_eig(e, E[i], eta[i]) for i, e in enumerate(eps)])

    mu, dn, evals, rounds = nd.ndsi_mu_search_batched(delta_n, elo, ehi, kTs, ne, dos=dos, n_grid=41)
    assert np.all(np.abs(dn) < 1e-8)
    for i in range(4):
        assert abs(mu[i] - find_mu_eig(eps[i], kTs[i], ne[i], 40)) < 1e-9
        single = nd.ndsi_mu_search(probs[i][4], elo[i], ehi[i], kTs[i], ne[i],
                                   dos=lambda E, eta, e=eps[i]: dos_eig(e, E, eta), n_grid=41)
        assert abs(single[0] - mu[i]) < 1e-12 and single[2] == evals[i]
    # rounds: the DOS round plus as many evaluation rounds as the slowest system needs
    assert rounds == max(evals)
    assert len(calls) == rounds - 1


def test_batched_errors_reach_every_system():
    nd = lib()

    def bad(mu, active):
        raise ValueError("sweep failed")

    with pytest.raises(ValueError):
        nd.ndsi_mu_search_batched(bad, [-1.0, -2.0], [1.0, 2.0], [0.01, 0.01], [1.0, 1.0])
