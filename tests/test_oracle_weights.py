"""Pins for the configuration weight and the rank-1 machinery of the oracle.

- prod_sigma det N_sigma^-1 (with N^-1 = e^V - g0 (e^V - 1), the reading of
  Eq. Zk) equals the brute-force time-ordered Fock-space trace
  <T prod_i exp(gamma s_i (n_{r_i up} - n_{r_i dn}))(tau_i)>_0 under the CT-AUX H0.
- The insert / remove ratios equal brute-force determinant ratios (LU).
- N after accepted moves equals the fresh inverse; insert-then-remove restores N.
"""
import numpy as np
import pytest

from oracle import ctaux, ed
from tests.helpers import problem


def _walker(nc, U, beta, mu, n_tau, tp=0.0, t=1.0, **kw):
    c, eps, kr, G0 = problem(nc, t, tp, U, beta, mu, n_tau)
    w = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, **kw)
    return c, eps, kr, G0, w


@pytest.mark.parametrize("nc,mu", [(1, 2.0), (1, 0.7), (4, 1.3), (4, 0.0)])
def test_weight_equals_time_ordered_trace(nc, mu):
    U, beta, n_tau = 4.0, 2.0, 64
    c, eps, kr, G0, w = _walker(nc, U, beta, mu, n_tau, init_config_size=0)
    t = ed.hopping_from_dispersion(eps, kr, c.site_sub)
    E = ed.HubbardED(t, U, mu)
    rng = np.random.default_rng(nc * 10 + int(mu * 10))
    for k in range(1, 6):
        site = rng.integers(0, nc, k)
        # vertex times on grid nodes: the linear interpolation is then exact
        tau = rng.choice(np.arange(n_tau), k, replace=False) * beta / n_tau
        s = rng.choice([-1, 1], k)
        det = np.prod([np.linalg.det(w.build_A(sp, site, tau, s)) for sp in range(2)])
        tr = E.aux_weight(beta, w.gamma, list(zip(site, tau, s)))
        assert abs(det / tr - 1.0) < 1e-11, (k, det, tr)


def test_gamma_decoupling_identity():
    # cosh(gamma) = 1 + U beta Nc / (2K)
    for nc, U, beta in [(1, 4.0, 2.0), (4, 4.0, 10.0), (16, 6.0, 20.0)]:
        c, eps, kr, G0 = problem(nc, 1.0, 0.0, U, beta, U / 2, 8)
        w = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, init_config_size=0)
        assert abs(np.cosh(w.gamma) - (1 + U * beta * nc / 2.0)) < 1e-9 * np.cosh(w.gamma)


def _dets(w, st):
    return np.array([np.linalg.det(w.build_A(sp, st["site"], st["tau"], st["s"])) for sp in range(2)])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rank1_ratios_and_updates_match_brute_force(seed):
    c, eps, kr, G0, w = _walker(4, 4.0, 3.0, 1.1, 256, init_config_size=9, seed=seed)
    rng = np.random.default_rng(seed)
    for step in range(12):
        st = w.state()
        d0 = _dets(w, st)
        if rng.random() < 0.5 or w.order < 2:
            site, tau, s = int(rng.integers(0, 4)), float(rng.uniform(0, 3.0)), int(rng.choice([-1, 1]))
            r = np.array(w.ratio_insert(site, tau, s))
            st2 = dict(site=np.r_[st["site"], site], tau=np.r_[st["tau"], tau], s=np.r_[st["s"], s])
            assert np.allclose(r, _dets(w, st2) / d0, rtol=1e-10, atol=0)
            w.try_insert(site, tau, s)
        else:
            p = int(rng.integers(0, w.order))
            r = np.array(w.ratio_remove(p))
            keep = [i for i in range(w.order) if i != p]
            st2 = dict(site=st["site"][keep], tau=st["tau"][keep], s=st["s"][keep])
            assert np.allclose(r, _dets(w, st2) / d0, rtol=1e-10, atol=0)
            w.try_remove(p)
        st = w.state()
        for sp in range(2):
            Nf, _ = w.fresh_N(sp)
            assert np.abs(Nf - st["N"][sp]).max() < 1e-10 * max(1.0, np.abs(Nf).max())


def test_insert_then_remove_restores_N():
    c, eps, kr, G0, w = _walker(4, 4.0, 3.0, 1.1, 256, init_config_size=7, seed=5)
    before = w.state()
    w.try_insert(2, 1.234, -1)
    w.try_remove(w.order - 1)
    after = w.state()
    for sp in range(2):
        assert np.abs(before["N"][sp] - after["N"][sp]).max() < 1e-12
    assert (before["site"] == after["site"]).all()


def test_rejected_move_leaves_state():
    c, eps, kr, G0, w = _walker(4, 4.0, 3.0, 1.1, 256, init_config_size=6, seed=6)
    before = w.state()
    w.try_insert(1, 0.5, 1, accept=False)
    w.try_remove(2, accept=False)
    after = w.state()
    for sp in range(2):
        assert (before["N"][sp] == after["N"][sp]).all()


def test_N_inverse_residual_after_long_run():
    c, eps, kr, G0, w = _walker(4, 4.0, 6.0, 0.9, 1024, init_config_size=10, seed=7, warmup_sweeps=5)
    w.sweep(300)
    st = w.state()
    for sp in range(2):
        A = w.build_A(sp, st["site"], st["tau"], st["s"])
        res = np.abs(A @ st["N"][sp] - np.eye(w.order)).max()
        assert res < 1e-9
