"""Pins of the oracle's auxiliary-spin flips and of the neglect rule (Sec. 2.3:
the third single-spin update, and "ignoring proposals of already chosen
spins" in a submatrix update).

- The flip ratio per spin equals the brute-force determinant ratio (LU) of
  A = N^-1 before and after the flip, and N after an accepted flip equals the
  fresh inverse, with the vertex still at its position and its spin negated;
  a flip followed by the flip back restores N.
- Flips keep detailed balance: with a third of the proposals flips, the
  Hubbard atom still meets its closed form and <k> identity, and the 2x2
  cluster its exact diagonalisation.
- The neglect rule with windows of one proposal never applies (nothing is
  changed twice in one proposal), so the chain is the exact one; with longer
  windows it rejects proposals and the chain departs.
"""
import json
import os

import numpy as np
import pytest

from oracle import ctaux, ed
from tests.helpers import binned, problem


def _dets(w, st):
    return np.array([np.linalg.det(w.build_A(sp, st["site"], st["tau"], st["s"])) for sp in range(2)])


@pytest.mark.parametrize("seed", [1, 2])
def test_flip_ratio_and_update_match_brute_force(seed):
    c, eps, kr, G0 = problem(4, 1.0, 0.0, 4.0, 3.0, 1.1, 256)
    w = ctaux.OracleWalker(4, c.site_sub, 4.0, 3.0, 1.0, G0, init_config_size=9, seed=seed)
    rng = np.random.default_rng(seed)
    for _ in range(6):
        st = w.state()
        d0 = _dets(w, st)
        p = int(rng.integers(0, st["site"].size))
        r = np.array(w.try_flip(p, accept=False))
        after = w.state()
        assert np.array_equal(after["s"], st["s"]) and np.abs(after["N"][0] - st["N"][0]).max() == 0
        st2 = dict(st, s=st["s"].copy())
        st2["s"][p] = -st2["s"][p]
        assert np.allclose(r, _dets(w, st2) / d0, rtol=1e-10, atol=0)
        w.try_flip(p, accept=True)
        now = w.state()
        assert np.array_equal(now["s"], st2["s"]) and np.array_equal(now["site"], st["site"])
        for sp in range(2):
            fresh = np.linalg.inv(w.build_A(sp, now["site"], now["tau"], now["s"]))
            assert np.abs(now["N"][sp] - fresh).max() < 1e-11 * np.abs(fresh).max()
    # flip and flip back
    st = w.state()
    w.try_flip(2, accept=True)
    w.try_flip(2, accept=True)
    back = w.state()
    assert np.array_equal(back["s"], st["s"])
    for sp in range(2):
        assert np.abs(back["N"][sp] - st["N"][sp]).max() < 1e-11 * np.abs(st["N"][sp]).max()


def test_atom_with_flips_meets_the_closed_form():
    U, beta, n_tau, ntm = 4.0, 2.0, 4096, 16
    c, eps, kr, G0 = problem(1, 0.0, 0.0, U, beta, U / 2, n_tau)
    w = ctaux.OracleWalker(1, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=200, n_tau_meas=ntm, seed=5,
                           flip_frac=1.0 / 3.0)
    Gb, kb = [], []
    for b in range(24):
        w.reset_accumulators()
        w.sweep(4000)
        g, ss, nm = w.G()
        Gb.append(g[:, 0] / ss)
        kb.append(w.counters()["k_sum"] / ss)
    Gb = np.array(Gb)
    taus = (np.arange(ntm) + 0.5) * beta / ntm
    exact = ed.atom_greens(U, beta, taus)
    z = np.concatenate([(binned(Gb[:, sp])[0] - exact) / binned(Gb[:, sp])[1] for sp in range(2)])
    assert np.abs(z).max() < 4.0 and np.mean(z * z) < 2.0, z
    m, e = binned(kb)
    k_exact = 1.0 + beta * (U / 2) * np.exp(beta * U / 2) / (1 + np.exp(beta * U / 2))
    assert abs(m - k_exact) < 3 * e, (m, e, k_exact)
    assert w.counters()["accepts"] > 0


def test_2x2_with_flips_matches_ed():
    U, beta, mu, n_tau, ntm = 4.0, 4.0, 1.0, 4096, 8
    c, eps, kr, G0 = problem(4, 1.0, 0.0, U, beta, mu, n_tau)
    t = ed.hopping_from_dispersion(eps, kr, c.site_sub)
    E = ed.HubbardED(t, U, mu)
    taus = (np.arange(ntm) + 0.5) * beta / ntm
    Gex = E.greens_translation_avg(beta, taus, c.site_sub)
    w = ctaux.OracleWalker(4, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=200, n_tau_meas=ntm, seed=2,
                           flip_frac=0.25)
    Gb = []
    for b in range(16):
        w.reset_accumulators()
        w.sweep(1500)
        g, ss, nm = w.G()
        Gb.append(g / ss)
    Gb = np.array(Gb)
    z = np.concatenate([((binned(Gb[:, sp])[0] - Gex) / binned(Gb[:, sp])[1]).ravel() for sp in range(2)])
    assert np.abs(z).max() < 4.0 and np.mean(z * z) < 2.0, z


def test_neglect_rule():
    c, eps, kr, G0 = problem(4, 1.0, 0.0, 4.0, 6.0, 1.0, 512)
    mk = lambda **kw: ctaux.OracleWalker(4, c.site_sub, 4.0, 6.0, 1.0, G0, warmup_sweeps=5, n_tau_meas=4, seed=8,
                                         flip_frac=0.2, **kw)
    a, b, d = mk(), mk(neglect_ks=1), mk(neglect_ks=32)
    for o in (a, b, d):
        o.enable_log(1 << 20)
        o.sweep(150)
    assert np.array_equal(a.log(), b.log()) and b.neglected == 0
    assert d.neglected > 0
    n = min(a.log().size, d.log().size)
    assert not np.array_equal(a.log()[:n], d.log()[:n])
