"""Outer DCA loop on the GPU (dca_coarse_grain, dca_sigma_update,
dca_g0_table_from_freq) against the oracle's numpy loop on the same inputs,
and one full iteration around the walkers: run on the coarse-grained bath,
measure M in frequency, update Sigma, coarse-grain again and hand the new
table to the walkers.  FP64 both sides: agreement to 1e-12 (the table: to
1e-11, a sum over n_omega frequencies per point)."""
import numpy as np
import pytest

from oracle import ctaux
from oracle import dca_loop as dl
from paper_1901_01047_gb300 import inputs

pytestmark = pytest.mark.gpu


def _loop(nc, tp, mu, U, beta, n_fine, n_omega):
    from paper_1901_01047_gb300 import walker
    c = inputs.cluster(nc)
    kr = inputs.k_dot_r(c)
    lp = walker.DCALoop(nc, c.kpts, kr, dl.reciprocal_superlattice(c), 1.0, tp, mu, U, beta, n_fine, n_omega)
    return c, kr, lp


def _sigma(nc, beta, n_omega, seed):
    wn = dl.matsubara(beta, n_omega)
    rng = np.random.default_rng(seed)
    return rng.normal(size=(nc, 1)) * 0.5 - 1j * rng.uniform(0.5, 2.0, size=(nc, 1)) / (wn[None, :] + 1.0)


@pytest.mark.parametrize("nc,tp,n_fine", [(4, 0.0, 8), (16, -0.15, 4), (8, 0.0, 6), (1, 0.0, 16)])
def test_coarse_graining_and_table_match_the_oracle(nc, tp, n_fine):
    U, beta, mu, nw, n_tau = 5.0, 6.0, 2.1, 256, 1024
    c, kr, lp = _loop(nc, tp, mu, U, beta, n_fine, nw)
    sig = _sigma(nc, beta, nw, nc)
    Gbar, G0w, G0ws, xi = lp.coarse_grain(sig)
    Gbar_o = dl.coarse_grain(c, 1.0, tp, mu, beta, sig, n_fine)
    G0w_o = dl.cluster_exclusion(Gbar_o, sig)
    G0ws_o = dl.hartree_shift(G0w_o, U)
    xi_o = dl.patch_mean_dispersion(c, 1.0, tp, n_fine) - mu + U / 2
    assert np.abs(Gbar - Gbar_o).max() < 1e-12 * np.abs(Gbar_o).max()
    assert np.abs(G0w - G0w_o).max() < 1e-12 * np.abs(G0w_o).max()
    assert np.abs(G0ws - G0ws_o).max() < 1e-12 * np.abs(G0ws_o).max()
    assert np.abs(xi - xi_o).max() < 1e-13
    tab = lp.g0_table(G0ws, xi, n_tau)
    tab_o = dl.g0_table(G0ws_o, xi_o, kr, beta, n_tau)
    assert np.abs(tab - tab_o).max() < 1e-11


def test_sigma_update_matches_the_oracle():
    nc, U, beta, mu, nw = 4, 4.0, 5.0, 1.0, 64
    c, kr, lp = _loop(nc, 0.0, mu, U, beta, 4, nw)
    rng = np.random.default_rng(3)
    G0ws = dl.hartree_shift(dl.coarse_grain(c, 1.0, 0.0, mu, beta, np.zeros((nc, nw)), 4), U)
    M = rng.normal(size=(3, 2, nc, nw)) * 0.1 + 1j * rng.normal(size=(3, 2, nc, nw)) * 0.1
    ss = np.array([2.0, 3.5, 1.5])
    old = _sigma(nc, beta, nw, 5)
    new = lp.sigma_update(G0ws, M, ss, old, 0.6)
    MK = dl.M_of_K(M, kr).sum(axis=(0, 1)) / (2 * ss.sum())
    sig_qmc = dl.dyson_sigma(1.0 / (1.0 / G0ws + U / 2), dl.measured_G(G0ws, MK))
    ref = dl.mix(sig_qmc, old, 0.6)
    assert np.abs(new - ref).max() < 1e-12 * np.abs(ref).max()


def test_one_dca_iteration_around_the_walkers():
    # 2x2 cluster, U = 4, beta = 4, mu = 1: the first bath is the coarse-grained
    # lattice propagator (Sigma = 0), the walkers measure M(K, i w_n), the new
    # Sigma is causal (Im Sigma(K, i w_n) < 0 at the lowest frequency) and has
    # the Hartree value U <n_-sigma> = U n / 2 at high frequency, and the next
    # table is taken by the walkers, whose chains go on.
    import torch
    from paper_1901_01047_gb300 import walker
    nc, U, beta, mu, nw, n_tau, nf = 4, 4.0, 4.0, 1.0, 128, 1024, 8
    c, kr, lp = _loop(nc, 0.0, mu, U, beta, nf, nw)
    sig0 = np.zeros((nc, nw), np.complex128)
    Gbar, G0w, G0ws, xi = lp.coarse_grain(sig0)
    table = lp.g0_table(G0ws, xi, n_tau)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=table)
    gw = walker.Walkers([prob], n_walkers=8, k_sub=32, recompute_every=16, warmup_sweeps=50, n_tau_meas=32,
                        seed=4, n_omega_meas=nw, stream=torch.cuda.current_stream().cuda_stream)
    gw.sweep(50)
    gw.reset_measurements()
    gw.sweep(1500)
    M, ss, nm = gw.measure_M()
    assert all(s["status"] == 0 for s in gw.stats())
    sig1 = lp.sigma_update(G0ws, np.array(M), ss, sig0, 1.0)
    # the oracle's chain of formulas on the same measured M
    MK = dl.M_of_K(np.array(M), kr).sum(axis=(0, 1)) / (2 * ss.sum())
    ref = dl.dyson_sigma(1.0 / (1.0 / G0ws + U / 2), dl.measured_G(G0ws, MK))
    assert np.abs(sig1 - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.all(sig1[:, 0].imag < 0)
    # high-frequency Sigma -> U <n_-sigma>: the density from the measured G(tau) at tau -> beta
    G, ssg, _ = gw.measure_G()
    # -G(dr = 0, beta-) = <n_sigma>, from the last two midpoints of the tau grid extrapolated to beta
    g_last = np.mean([G[w][:, 0, -1].mean() / ssg[w] for w in range(8)])
    g_prev = np.mean([G[w][:, 0, -2].mean() / ssg[w] for w in range(8)])
    n_sigma = -(g_last + 0.5 * (g_last - g_prev))
    assert abs(np.mean(sig1[:, -8:].real) - U * n_sigma) < 0.15, (np.mean(sig1[:, -8:].real), U * n_sigma)
    Gbar1, G0w1, G0ws1, xi1 = lp.coarse_grain(sig1)
    table1 = lp.g0_table(G0ws1, xi1, n_tau)
    assert np.abs(table1 - table).max() > 1e-3  # the bath moved
    gw.update_G0(0, table1)
    gw.sweep(20)
    assert all(s["status"] == 0 for s in gw.stats())
    gw.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_update_G0_rebuilds_N_for_the_new_table(precision):
    # a new bare propagator changes N^-1 = e^V - g0 (e^V - 1): the walkers of
    # that problem get N rebuilt from scratch, with the configuration sign
    # from the new determinants; an unchanged table leaves N alone
    import torch
    from paper_1901_01047_gb300 import walker
    from tests.helpers import problem
    nc, U, beta = 4, 4.0, 4.0
    c, eps, kr, G0a = problem(nc, 1.0, 0.0, U, beta, 1.0, 1024)
    _, _, _, G0b = problem(nc, 1.0, 0.0, U, beta, 1.4, 1024)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0a)
    gw = walker.Walkers([prob], n_walkers=2, k_sub=16, recompute_every=8, warmup_sweeps=2, n_tau_meas=8, seed=3,
                        precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    gw.sweep(25)
    before = gw.state(0)
    gw.update_G0(0, G0a)  # the same table: nothing to rebuild
    same = gw.state(0)
    assert np.array_equal(same["N"][0], before["N"][0])
    gw.update_G0(0, G0b)
    after = gw.state(0)
    assert np.array_equal(after["site"], before["site"]) and np.array_equal(after["tau"], before["tau"])
    ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0b, warmup_sweeps=0, n_tau_meas=8, seed=3)
    ow.set_config(after["site"], after["tau"], after["s"])
    tol = 1e-10 if precision == "fp64" else 1e-5
    for sp in range(2):
        fresh, _ = ow.fresh_N(sp)
        assert np.abs(after["N"][sp] - fresh).max() < tol * np.abs(fresh).max()
    assert gw.stats()[0]["sign"] == ow.sign
    gw.sweep(10)
    assert all(s["status"] == 0 for s in gw.stats())
    gw.close()
