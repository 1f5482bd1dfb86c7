"""Statistical pins through the GPU path (FP64 walker).

- Hubbard atom (Nc=1, U=4, beta=2, mu=U/2, K=1, k_s=8, 1e4 sweeps): G(tau)
  against the closed form within 3 sigma; <k> against K - beta <H_int>.
- 2x2 Hubbard cluster (t=1, U=4, beta=10, density 0.9, k_s=32, 1e5 sweeps):
  G(dr, tau) and <k> against exact diagonalisation within 3 sigma.
Error bars come from bins of consecutive sweeps.
"""
import json
import os

import numpy as np
import pytest

from oracle import ed
from tests.helpers import binned, problem

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _walkers(**kw):
    import torch
    from paper_1901_01047_gb300 import walker
    return walker.Walkers(stream=torch.cuda.current_stream().cuda_stream, **kw)


def _bins(gw, n_bins, per_bin):
    Gb, kb, sb = [], [], []
    for _ in range(n_bins):
        gw.reset_measurements()
        gw.sweep(per_bin)
        G, ss, nm = gw.measure_G()
        st = gw.stats()[0]
        Gb.append(G[0] / ss[0])
        kb.append(st["k_sum"] / nm[0])
        sb.append(ss[0] / nm[0])
    return np.array(Gb), np.array(kb), np.array(sb)


def test_atom_closed_form_full_run():
    U, beta, ntm = 4.0, 2.0, 32
    c, eps, kr, G0 = problem(1, 0.0, 0.0, U, beta, U / 2, 4096)
    gw = _walkers(problems=[dict(nc=1, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)], k_sub=8,
                  recompute_every=64, warmup_sweeps=20, n_tau_meas=ntm, seed=0)
    gw.sweep(20)
    Gb, kb, sb = _bins(gw, 20, 500)   # 1e4 measured sweeps
    taus = (np.arange(ntm) + 0.5) * beta / ntm
    exact = ed.atom_greens(U, beta, taus)
    for sp in range(2):
        m, e = binned(Gb[:, sp, 0])
        assert np.abs((m - exact) / e).max() < 3.0
    p1 = np.exp(beta * U / 2) / (1 + np.exp(beta * U / 2))
    m, e = binned(kb)
    assert abs(m - (1 + beta * U / 2 * p1)) < 3 * e
    assert np.all(sb == 1.0)


def test_2x2_cluster_against_ed_full_run():
    with open(os.path.join(GOLDEN, "hubbard_2x2_ed.json")) as f:
        gd = json.load(f)
    U, beta, mu, ntm = gd["U"], gd["beta"], gd["mu"], 16
    c, eps, kr, G0 = problem(4, 1.0, 0.0, U, beta, mu, 4096)
    t = ed.hopping_from_dispersion(eps, kr, c.site_sub)
    E = ed.HubbardED(t, U, mu)
    taus = (np.arange(ntm) + 0.5) * beta / ntm
    Gex = E.greens_translation_avg(beta, taus, c.site_sub)
    gw = _walkers(problems=[dict(nc=4, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)], k_sub=32,
                  recompute_every=64, warmup_sweeps=20, n_tau_meas=ntm, seed=0)
    gw.sweep(20)
    Gb, kb, sb = _bins(gw, 25, 4000)  # 1e5 measured sweeps
    for sp in range(2):
        m, e = binned(Gb[:, sp])
        assert np.abs((m - Gex) / e).max() < 3.0
    m, e = binned(kb)
    assert abs(m - gd["k_expected"]) < 3 * e
    st = gw.stats()[0]
    assert st["max_drift"] < 1e-10
