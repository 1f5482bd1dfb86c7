"""The two-particle measurement (particle-particle up-down channel, Sec. 2.5
Eq. bse_cluster; App. B four-point group) on the GPU against the oracle on
identical trajectories.

FP64 path: the accumulators A(s1, s2) = sum sign M_up(s1, s2) M_dn(q - s1,
q - s2) and D_sigma(s) = sum sign M_sigma(s, s) within 1e-10 of the oracle in
the norm form max|X_gpu - X_ora| / max|X_ora|, for the 2x2 cluster (frequency
and momentum transfer), the atom, and 16 sites with two walkers (point tiles
with ragged edges); U = 0 gives exactly zero.  Mixed path: the GPU replays the
oracle's decisions; the error is that of the FP32 N between recomputes and of
the FP32 products.  dca_g4_assemble against the oracle's assembly.
"""
import numpy as np
import pytest

from oracle import ctaux
from oracle import g4 as og4
from tests.helpers import problem

pytestmark = pytest.mark.gpu


def _walkers(**kw):
    import torch
    from paper_1901_01047_gb300 import walker
    return walker.Walkers(stream=torch.cuda.current_stream().cuda_stream, **kw)


def _pair(nc, tp, U, beta, mu, n_tau, k_sub, sweeps, n_w4, m4, q, precision="fp64", R=16, seed=0, warmup=10,
          walkers=1, recompute_at_measure=False):
    c, eps, kr, G0 = problem(nc, 1.0, tp, U, beta, mu, n_tau)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0, k_dot_r=kr, k_sub=c.k_sub)
    oracles, logs = [], []
    for wi in range(walkers):
        ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=warmup, n_tau_meas=8, seed=seed,
                                walker_id=wi)
        ow.enable_g4(n_w4, m4, kr, c.k_sub[q])
        ow.enable_log(1 << 22)
        ow.sweep(sweeps)
        oracles.append(ow)
        logs.append(ow.log())
    gw = _walkers(problems=[prob], n_walkers=walkers, k_sub=k_sub, recompute_every=R, warmup_sweeps=warmup,
                  n_tau_meas=8, seed=seed, precision=precision, log_capacity=1 << 22, n_w4=n_w4, w4_transfer=m4,
                  q4_transfer=q, recompute_at_measure=recompute_at_measure)
    for wi in range(walkers):
        gw.set_forced_decisions(wi, logs[wi])
    gw.sweep(sweeps)
    res, ssg, nmg = gw.measure_G4()
    out = []
    for wi in range(walkers):
        ow = oracles[wi]
        Ao, Do = ow.g4()
        g, sso, nmo = ow.G()
        assert nmg[wi] == nmo > 0 and ssg[wi] == sso
        Ag, Dg = res[wi]
        errA = np.abs(Ag - Ao).max() / max(np.abs(Ao).max(), 1e-300)
        errD = np.abs(Dg - Do).max() / max(np.abs(Do).max(), 1e-300)
        out.append(dict(errA=errA, errD=errD, A=Ag, D=Dg, Ao=Ao, Do=Do, ss=sso))
    st = gw.stats()
    gw.close()
    return out, st, (c, eps, kr)


@pytest.mark.parametrize("m4,q", [(0, 0), (1, 3)])
def test_g4_matches_the_oracle_fp64_2x2(m4, q):
    res, st, _ = _pair(4, 0.0, 4.0, 6.0, 1.0, 2048, k_sub=32, sweeps=150, n_w4=4, m4=m4, q=q)
    for r in res:
        assert r["errA"] < 1e-10 and r["errD"] < 1e-10, (r["errA"], r["errD"])
        assert np.abs(r["Ao"]).max() > 0


def test_g4_matches_the_oracle_fp64_atom_and_16_sites():
    res, _, _ = _pair(1, 0.0, 4.0, 2.0, 2.0, 2048, k_sub=8, sweeps=400, n_w4=8, m4=-2, q=0, warmup=20)
    assert res[0]["errA"] < 1e-10 and res[0]["errD"] < 1e-10, res[0]["errA"]
    # 16 sites, two walkers, S = 16 * 2 * 3 = 96 points: three 32-point tiles, a ragged 64-point tile
    res, _, _ = _pair(16, -0.15, 6.0, 4.0, 2.85, 2048, k_sub=64, sweeps=20, n_w4=3, m4=1, q=5, walkers=2)
    for r in res:
        assert r["errA"] < 1e-10 and r["errD"] < 1e-10, (r["errA"], r["errD"])


def test_g4_u0_is_exactly_zero_and_assembles_to_the_bubble():
    from paper_1901_01047_gb300 import walker
    nc, beta, mu, n_w4, m4, q = 4, 3.0, 0.4, 3, 1, 2
    c, eps, kr, G0 = problem(nc, 1.0, 0.0, 0.0, beta, mu, 512)
    gw = _walkers(problems=[dict(nc=nc, site_sub=c.site_sub, U=0.0, beta=beta, K=1.7, G0=G0, k_dot_r=kr,
                                 k_sub=c.k_sub)], n_walkers=2, k_sub=16, recompute_every=8, warmup_sweeps=5,
                  n_tau_meas=8, seed=1, n_w4=n_w4, w4_transfer=m4, q4_transfer=q)
    gw.sweep(60)
    res, ss, nm = gw.measure_G4()
    Ku, nu, Kd, nd = og4.points(nc, n_w4, m4, c.k_sub[q])
    g0 = lambda K, n: 1.0 / (1j * (2 * n + 1) * np.pi / beta - (eps[K] - mu))
    for wi in range(2):
        A, D = res[wi]
        assert nm[wi] > 0 and np.all(A == 0) and np.all(D == 0)
        G2 = walker.g4_assemble(A, D, ss[wi], g0(Ku, nu), g0(Kd, nd))
        assert np.allclose(G2, np.diag(g0(Ku, nu) * g0(Kd, nd)), rtol=1e-14, atol=0)
    gw.close()


def test_g4_assemble_matches_the_oracle():
    from paper_1901_01047_gb300 import walker
    res, _, (c, eps, kr) = _pair(4, 0.0, 4.0, 3.0, 1.1, 1024, k_sub=16, sweeps=80, n_w4=2, m4=1, q=1)
    r = res[0]
    Ku, nu, Kd, nd = og4.points(4, 2, 1, c.k_sub[1])
    g0 = lambda K, n: 1.0 / (1j * (2 * n + 1) * np.pi / 3.0 - (eps[K] - (1.1 - 2.0)))
    G2g = walker.g4_assemble(r["A"], r["D"], r["ss"], g0(Ku, nu), g0(Kd, nd))
    G2o = og4.assemble(r["Ao"], r["Do"], r["ss"], g0(Ku, nu), g0(Kd, nd))
    assert np.abs(G2g - G2o).max() < 1e-10 * np.abs(G2o).max()


def test_g4_mixed_replay_error():
    # same trajectory; the error of the FP32 N between recomputes (every 16
    # windows) and of the FP32 products, and with N recomputed before every
    # measurement
    res, _, _ = _pair(4, 0.0, 4.0, 6.0, 1.0, 2048, k_sub=32, sweeps=150, n_w4=4, m4=1, q=3, precision="mixed")
    print("mixed G4 replay error: A %.2e D %.2e" % (res[0]["errA"], res[0]["errD"]))
    assert res[0]["errA"] < 1e-4 and res[0]["errD"] < 1e-4
    res, _, _ = _pair(4, 0.0, 4.0, 6.0, 1.0, 2048, k_sub=32, sweeps=150, n_w4=4, m4=1, q=3, precision="mixed",
                      recompute_at_measure=True)
    print("mixed G4 replay error, N recomputed at every measurement: A %.2e D %.2e" % (res[0]["errA"], res[0]["errD"]))
    assert res[0]["errA"] < 1e-6 and res[0]["errD"] < 1e-6


def test_g4_checkpoint_round_trip():
    nc, U, beta, mu = 4, 4.0, 3.0, 1.1
    c, eps, kr, G0 = problem(nc, 1.0, 0.0, U, beta, mu, 512)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0, k_dot_r=kr, k_sub=c.k_sub)
    kw = dict(problems=[prob], n_walkers=2, k_sub=16, recompute_every=8, warmup_sweeps=5, n_tau_meas=8, seed=7,
              n_w4=2, w4_transfer=1, q4_transfer=2)
    a = _walkers(**kw)
    a.sweep(30)
    blob = a.save()
    a.sweep(20)
    ra, ssa, nma = a.measure_G4()
    b = _walkers(**kw)
    b.load(blob)
    b.sweep(20)
    rb, ssb, nmb = b.measure_G4()
    assert np.array_equal(nma, nmb) and np.array_equal(ssa, ssb)
    for wi in range(2):
        assert np.abs(ra[wi][0] - rb[wi][0]).max() <= 1e-10 * np.abs(ra[wi][0]).max()
        assert np.abs(ra[wi][1] - rb[wi][1]).max() <= 1e-10 * np.abs(ra[wi][1]).max()
    other = _walkers(**dict(kw, q4_transfer=1))
    with pytest.raises(Exception):
        other.load(blob)
    for h in (a, b, other):
        h.close()
