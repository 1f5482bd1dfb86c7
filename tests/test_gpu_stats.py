"""Statistical pins through the GPU path (FP64 walker).

- Hubbard atom (Nc=1, U=4, beta=2, mu=U/2, K=1, k_s=8, 1e4 sweeps): G(tau)
  against the closed form within 3 sigma; <k> against K - beta <H_int>.
- 2x2 Hubbard cluster (t=1, U=4, beta=10, density 0.9, k_s=32): G(dr, tau)
  and the signed <k> against exact diagonalisation over 256 independent
  walkers of one batch.

Away from half filling the weight has a sign, so every estimate is the ratio
sum(sign * O) / sum(sign); its error comes from a jackknife over bins (the
atom, whose chain decorrelates fast) or over independent walkers.
"""
import json
import os

import numpy as np
import pytest

from oracle import ed
from tests.helpers import problem

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _walkers(**kw):
    import torch
    from paper_1901_01047_gb300 import walker
    return walker.Walkers(stream=torch.cuda.current_stream().cuda_stream, **kw)


def jackknife_ratio(num, den):
    """Ratio sum(num) / sum(den) over the first axis and its jackknife error."""
    num = np.asarray(num, np.float64)
    den = np.asarray(den, np.float64)
    B = num.shape[0]
    tot = num.sum(0) / den.sum()
    shape = (B,) + (1,) * (num.ndim - 1)
    jk = (num.sum(0)[None] - num) / (den.sum() - den).reshape(shape)
    err = np.sqrt((B - 1) / B * ((jk - jk.mean(0)) ** 2).sum(0))
    return tot, err


def _bins(gw, n_bins, per_bin):
    Gs, Ks, Ss = [], [], []
    for _ in range(n_bins):
        gw.reset_measurements()
        gw.sweep(per_bin)
        G, ss, nm = gw.measure_G()
        Gs.append(G[0])
        Ks.append(gw.stats()[0]["k_sum"])
        Ss.append(ss[0])
    return np.array(Gs), np.array(Ks), np.array(Ss)


def test_atom_closed_form_full_run():
    U, beta, ntm = 4.0, 2.0, 32
    c, eps, kr, G0 = problem(1, 0.0, 0.0, U, beta, U / 2, 4096)
    gw = _walkers(problems=[dict(nc=1, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)], k_sub=8,
                  recompute_every=64, warmup_sweeps=20, n_tau_meas=ntm, seed=0)
    gw.sweep(20)
    G, K, S = _bins(gw, 20, 500)   # 1e4 measured sweeps
    assert np.all(S == 500)        # no sign problem at half filling
    taus = (np.arange(ntm) + 0.5) * beta / ntm
    exact = ed.atom_greens(U, beta, taus)
    for sp in range(2):
        m, e = jackknife_ratio(G[:, sp, 0], S)
        assert np.abs((m - exact) / e).max() < 3.0
    p1 = np.exp(beta * U / 2) / (1 + np.exp(beta * U / 2))
    m, e = jackknife_ratio(K, S)
    assert abs(m - (1 + beta * U / 2 * p1)) < 3 * e


def _ed_2x2(ntm):
    with open(os.path.join(GOLDEN, "hubbard_2x2_ed.json")) as f:
        gd = json.load(f)
    U, beta, mu = gd["U"], gd["beta"], gd["mu"]
    c, eps, kr, G0 = problem(4, 1.0, 0.0, U, beta, mu, 4096)
    t = ed.hopping_from_dispersion(eps, kr, c.site_sub)
    E = ed.HubbardED(t, U, mu)
    taus = (np.arange(ntm) + 0.5) * beta / ntm
    Gex = E.greens_translation_avg(beta, taus, c.site_sub)
    return gd, c, G0, Gex


def test_2x2_cluster_against_ed_256_walkers():
    # The isolated 2x2 cluster at beta = 10, density 0.9 tunnels slowly between
    # particle-number sectors: a single chain's autocorrelation time exceeds
    # 1e4 sweeps, so errors come from independent walkers of one batch.
    ntm = 16
    gd, c, G0, Gex = _ed_2x2(ntm)
    W = 256
    gw = _walkers(problems=[dict(nc=4, site_sub=c.site_sub, U=gd["U"], beta=gd["beta"], K=1.0, G0=G0)],
                  n_walkers=W, k_sub=32, recompute_every=64, warmup_sweeps=200, n_tau_meas=ntm, seed=0)
    gw.sweep(200)
    gw.reset_measurements()
    gw.sweep(2000)
    G, S, NM = gw.measure_G()
    G = np.array(G)
    K = np.array([s["k_sum"] for s in gw.stats()])
    m, e = jackknife_ratio(0.5 * (G[:, 0] + G[:, 1]), S)
    assert np.abs((m - Gex) / e).max() < 3.0
    m, e = jackknife_ratio(K, S)
    assert abs(m - gd["k_expected"]) < 3 * e
    assert 0.3 < S.sum() / NM.sum() < 0.8  # a sign problem is present
    assert all(s["status"] == 0 for s in gw.stats())
