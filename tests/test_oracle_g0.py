"""Pins for the oracle's bare propagator and its interpolation.

- The K-space builder equals a Fock-space ED of the free CT-AUX H0 (hopping
  - (mu - U/2) n) on the 2x2 cluster, and the single-particle real-space form
  G0(tau) = -[e^{-tau h} (1 + e^{-beta h})^-1] on larger clusters.
- Linear interpolation reproduces grid nodes, is exact for linear data, and
  extends antiperiodically: g0(tau - beta) = -g0(tau).
"""
import numpy as np
import pytest

from oracle import ctaux, ed
from paper_1901_01047_gb300 import inputs
from tests.helpers import problem


def test_g0_builder_matches_free_ed_2x2():
    U, beta, mu, n_tau = 4.0, 3.0, 1.3, 48
    c, eps, kr, G0 = problem(4, 1.0, 0.0, U, beta, mu, n_tau)
    t = ed.hopping_from_dispersion(eps, kr, c.site_sub)
    E = ed.HubbardED(t, U, mu)
    taus = np.arange(1, n_tau) * beta / n_tau
    Ged = E.greens_translation_avg(beta, taus, c.site_sub, H=E.h0_shifted())
    assert np.abs(Ged - G0[0][:, 1:n_tau]).max() < 1e-13
    assert np.abs(G0[0] - G0[1]).max() == 0.0


@pytest.mark.parametrize("nc,tp", [(8, -0.15), (16, -0.15), (36, 0.0)])
def test_g0_builder_matches_single_particle_matrix_form(nc, tp):
    U, beta, mu, n_tau = 6.0, 5.0, 2.5, 16
    c, eps, kr, G0 = problem(nc, 1.0, tp, U, beta, mu, n_tau)
    t = ed.hopping_from_dispersion(eps, kr, c.site_sub)
    h = t - (mu - U / 2) * np.eye(nc)
    lam, V = np.linalg.eigh(h)
    for l in (0, 3, n_tau // 2, n_tau):
        tau = l * beta / n_tau
        w = np.exp(-tau * lam) / (1.0 + np.exp(-beta * lam))
        Gm = -(V * w) @ V.T
        for d in range(nc):
            x = [i for i in range(nc) if c.site_sub[i, 0] == d][0]
            assert abs(Gm[x, 0] - G0[0, d, l]) < 1e-13


def test_g0_paper_sign_and_boundaries():
    # G0(0+) - G0(beta-) = -1 on site (anticommutator), G0 < 0 on (0, beta) for the atom.
    U, beta, n_tau = 4.0, 2.0, 64
    for mu in (0.5, 2.0, 3.7):
        c, eps, kr, G0 = problem(1, 0.0, 0.0, U, beta, mu, n_tau)
        assert abs(G0[0, 0, 0] + G0[0, 0, n_tau] + 1.0) < 1e-14
        assert (G0 < 0).all()
    c, eps, kr, G0 = problem(16, 1.0, -0.15, 6.0, 20.0, 3.0, 128)
    assert np.abs(G0[0, 0, 0] + G0[0, 0, -1] + 1.0).max() < 1e-12


def test_interpolation_nodes_linearity_antiperiodicity():
    n_tau, beta = 32, 3.0
    rng = np.random.default_rng(0)
    row = rng.normal(size=n_tau + 1)
    for l in range(n_tau + 1):
        tau = l * beta / n_tau
        v = ctaux.g0_interp(row, n_tau, beta, tau if l < n_tau else beta * (1 - 1e-15))
        assert abs(v - row[l]) < 1e-12
    lin = 0.7 + 0.3 * np.arange(n_tau + 1) * beta / n_tau
    for tau in rng.uniform(0, beta, 50):
        assert abs(ctaux.g0_interp(lin, n_tau, beta, tau) - (0.7 + 0.3 * tau)) < 1e-12
        assert abs(ctaux.g0_interp(row, n_tau, beta, tau - beta) + ctaux.g0_interp(row, n_tau, beta, tau)) < 1e-12
    assert ctaux.g0_interp(row, n_tau, beta, 0.0) == row[0]


def test_cluster_geometry_group_structure():
    for nc in (1, 4, 8, 16, 36):
        c = inputs.cluster(nc)
        S = c.site_sub
        assert S.shape == (nc, nc)
        for i in range(nc):
            assert sorted(S[i]) == list(range(nc))
            assert S[i, i] == S[0, 0]
        # K . a in 2 pi Z for both superlattice vectors
        A = np.array(c.vecs, dtype=np.float64)
        ph = c.kpts @ A.T / (2 * np.pi)
        assert np.abs(ph - np.round(ph)).max() < 1e-9
