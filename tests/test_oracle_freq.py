"""Pins of the oracle's frequency-domain measurement of M (Sec. 2.3: the
Green's function is linear in M, whose Fourier coefficients are accumulated;
Eq. nfft evaluates them).  The oracle accumulates

    M(dr, i w_n) = 1/(beta Nc) sum_{i,j : r_i - r_j = dr} (e^{V_i} - 1) N_ij e^{i w_n (tau_i - tau_j)},

and, in the paper's sign, G(K, i w_n) = G0(K, i w_n) - G0(K, i w_n)^2 M(K, i w_n) with
M(K) = sum_dr e^{-i K.dr} M(dr).  Pinned by:
- U = 0: gamma = 0, so M = 0 exactly in every measurement;
- the Hubbard atom at mu = U/2: G0 = 1/(i w), G = i w / ((i w)^2 - U^2/4), hence
  M(i w) = (G0 - G) / G0^2 = i (U^2/4) w / (w^2 + U^2/4);
- the 2x2 cluster against exact diagonalisation (Lehmann sum).
The statistical checks compare many values at once (frequencies x real and
imaginary parts x spins), so each takes the mean of z^2 (about 1 for an
unbiased estimate with correct error bars) and bounds the largest |z| by 4.
"""
import numpy as np

from oracle import ctaux, ed
from tests.helpers import binned, problem


def _check_z(z):
    z = np.asarray(z).ravel()
    assert np.abs(z).max() < 4.0, z
    assert np.mean(z * z) < 2.0, z


def test_u0_frequency_measurement_vanishes():
    nc, beta, mu, n_tau = 4, 3.0, 0.4, 512
    c, eps, kr, G0 = problem(nc, 1.0, 0.0, 0.0, beta, mu, n_tau)
    w = ctaux.OracleWalker(nc, c.site_sub, 0.0, beta, 1.7, G0, warmup_sweeps=10, n_tau_meas=4, seed=11)
    w.enable_freq(16)
    w.sweep(300)
    assert w.counters()["k_sum"] > 0  # measurements at non-zero order happened
    M = w.M()
    assert M.shape == (2, nc, 16) and np.all(M == 0.0)


def test_atom_frequency_measurement_closed_form():
    U, beta, n_tau, nw = 4.0, 2.0, 4096, 12
    c, eps, kr, G0 = problem(1, 0.0, 0.0, U, beta, U / 2, n_tau)
    w = ctaux.OracleWalker(1, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=200, n_tau_meas=4, seed=3)
    w.enable_freq(nw)
    Mb = []
    for b in range(24):
        w.reset_accumulators()
        w.sweep(3000)
        g, ss, nm = w.G()
        Mb.append(w.M()[:, 0] / ss)
    Mb = np.array(Mb)
    wn = (2 * np.arange(nw) + 1) * np.pi / beta
    exact = 1j * (U * U / 4) * wn / (wn ** 2 + U * U / 4)
    z = []
    for sp in range(2):
        for part in (np.real, np.imag):
            m, e = binned(part(Mb[:, sp]))
            z.append((m - part(exact)) / np.maximum(e, 1e-12))
    _check_z(z)
    # the measured M is not trivially small: it carries the interaction
    assert np.abs(binned(np.imag(Mb[:, 0]))[0] - np.imag(exact)).max() < 0.05 * np.abs(np.imag(exact)).max()


def test_2x2_frequency_measurement_matches_ed():
    U, beta, mu, n_tau, nw = 4.0, 4.0, 1.0, 4096, 6
    c, eps, kr, G0 = problem(4, 1.0, 0.0, U, beta, mu, n_tau)
    t = ed.hopping_from_dispersion(eps, kr, c.site_sub)
    E = ed.HubbardED(t, U, mu)
    G_ed = E.greens_freq_K(beta, nw, c.site_sub, kr)             # [K, n]
    wn = (2 * np.arange(nw) + 1) * np.pi / beta
    xi = eps - (mu - U / 2)
    G0K = 1.0 / (1j * wn[None, :] - xi[:, None])                  # exact FT of the free propagator
    w = ctaux.OracleWalker(4, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=200, n_tau_meas=4, seed=1)
    w.enable_freq(nw)
    Gb = []
    for b in range(16):
        w.reset_accumulators()
        w.sweep(1500)
        g, ss, nm = w.G()
        MK = np.einsum("kd,sdn->skn", np.exp(-1j * kr), w.M()) / ss
        Gb.append(G0K[None] - G0K[None] ** 2 * MK)
    Gb = np.array(Gb)
    z = []
    for sp in range(2):
        for part in (np.real, np.imag):
            m, e = binned(part(Gb[:, sp]))
            z.append((m - part(G_ed)) / np.maximum(e, 1e-12))
    _check_z(z)


def test_ed_frequency_greens_against_closed_forms_and_its_time_domain():
    # The Lehmann sum of ED: (i) at U = 0 it is 1/(i w_n - xi_K) exactly; (ii) its
    # high-frequency tail is 1/(i w_n) (the anticommutator {c, c+} = 1); (iii)
    # it is the Fourier transform of the imaginary-time ED Green's function,
    # integrated here by Gauss-Legendre quadrature on (0, beta).
    c, eps, kr, G0 = problem(4, 1.0, 0.0, 0.0, 4.0, 1.0, 8)
    t = ed.hopping_from_dispersion(eps, kr, c.site_sub)
    beta, nw = 4.0, 6
    wn = (2 * np.arange(nw) + 1) * np.pi / beta
    G0_ed = ed.HubbardED(t, 0.0, 1.0).greens_freq_K(beta, nw, c.site_sub, kr)
    assert np.abs(G0_ed - 1.0 / (1j * wn[None, :] - (eps - 1.0)[:, None])).max() < 1e-12
    E = ed.HubbardED(t, 4.0, 1.0)
    far = E.greens_freq(beta, 3001)[:, :, -1]
    w_far = (2 * 3000 + 1) * np.pi / beta
    assert np.abs(1j * w_far * np.diag(far) - 1.0).max() < 10.0 / w_far
    assert np.abs(far - np.diag(np.diag(far))).max() < 10.0 / w_far ** 2  # off-diagonal tail starts at 1/w^2
    x, wq = np.polynomial.legendre.leggauss(120)
    taus = 0.5 * beta * (x + 1.0)
    Gt = E.greens(beta, taus)                                       # [nc, nc, q]
    Gw = E.greens_freq(beta, nw)
    quad = 0.5 * beta * np.einsum("xyq,q,qn->xyn", Gt, wq, np.exp(1j * np.outer(taus, wn)))
    assert np.abs(quad - Gw).max() < 1e-9
