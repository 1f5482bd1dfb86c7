"""From-scratch N (`dca_fresh_N`) against the oracle's inverse of the same
configuration, for configurations sampled by the oracle's own chain."""
import numpy as np
import pytest

from oracle import ctaux
from tests.helpers import problem


def _sampled_config(nc, t, tp, U, beta, mu, n_tau, sweeps, seed):
    c, eps, kr, G0 = problem(nc, t, tp, U, beta, mu, n_tau)
    ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=sweeps, n_tau_meas=4, seed=seed)
    ow.sweep(sweeps)
    return c, G0, ow


@pytest.mark.gpu
@pytest.mark.parametrize("nc,tp,U,beta,mu,sweeps", [
    (1, 0.0, 4.0, 2.0, 2.0, 30),
    (4, 0.0, 4.0, 10.0, 0.9450480104035819, 60),
    (16, -0.15, 6.0, 2.0, 2.85, 15),
])
def test_fresh_N_matches_oracle(nc, tp, U, beta, mu, sweeps):
    from paper_1901_01047_gb300 import walker
    c, G0, ow = _sampled_config(nc, 1.0, tp, U, beta, mu, 1024, sweeps, seed=4)
    st = ow.state()
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)
    Nu, Nd, sg = walker.fresh_N(prob, st["site"], st["tau"], st["s"])
    assert sg == int(ow.sign)
    for sp, Ng in enumerate((Nu, Nd)):
        ref, osg = ow.fresh_N(sp)
        assert np.abs(Ng - ref).max() <= 1e-10 * np.abs(ref).max()
        A = ow.build_A(sp, st["site"], st["tau"], st["s"])
        assert np.abs(A @ Ng - np.eye(len(st["site"]))).max() < 1e-10


@pytest.mark.gpu
def test_fresh_N_empty_and_singleton():
    from paper_1901_01047_gb300 import walker
    c, eps, kr, G0 = problem(4, 1.0, 0.0, 4.0, 3.0, 1.0, 256)
    prob = dict(nc=4, site_sub=c.site_sub, U=4.0, beta=3.0, K=1.0, G0=G0)
    Nu, Nd, sg = walker.fresh_N(prob, [], [], [])
    assert Nu.shape == (0, 0) and sg == 1
    Nu, Nd, sg = walker.fresh_N(prob, [2], [1.0], [1])
    ow = ctaux.OracleWalker(4, c.site_sub, 4.0, 3.0, 1.0, G0, init_config_size=0)
    ow.set_config([2], [1.0], [1])
    assert abs(Nu[0, 0] - ow.fresh_N(0)[0][0, 0]) < 1e-14
    assert abs(Nd[0, 0] - ow.fresh_N(1)[0][0, 0]) < 1e-14


def test_fresh_N_rejects_bad_vertices():
    from paper_1901_01047_gb300 import build, walker
    build.build()
    c, eps, kr, G0 = problem(4, 1.0, 0.0, 4.0, 3.0, 1.0, 64)
    prob = dict(nc=4, site_sub=c.site_sub, U=4.0, beta=3.0, K=1.0, G0=G0)
    for site, tau, s in [([4], [0.5], [1]), ([0], [3.0], [1]), ([0], [-0.1], [1]), ([0], [0.5], [0])]:
        with pytest.raises(walker.WalkerError, match="ARG"):
            walker.fresh_N(prob, site, tau, s)


@pytest.mark.gpu
@pytest.mark.parametrize("n", [300, 700])
def test_fresh_N_large_random_configuration(n):
    # many rows per block of the 8-block cluster inverse.  Random vertices give
    # ill-conditioned A (entries of N over ~10 decades), so the check is the
    # residual A N - I against the oracle's own, plus a kappa-scaled agreement.
    from paper_1901_01047_gb300 import walker
    nc, U, beta = 16, 1.0, 5.0
    c, eps, kr, G0 = problem(nc, 1.0, -0.15, U, beta, 0.3, 1024)
    rng = np.random.default_rng(n)
    site = rng.integers(0, nc, n).astype(np.int32)
    tau = rng.uniform(0, beta, n)
    s = rng.choice([-1, 1], n).astype(np.int8)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)
    Nu, Nd, sg = walker.fresh_N(prob, site, tau, s)
    ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, init_config_size=0)
    ow.set_config(site, tau, s)
    assert sg == int(ow.sign)
    for sp, Ng in enumerate((Nu, Nd)):
        ref, _ = ow.fresh_N(sp)
        A = ow.build_A(sp, site, tau, s)
        res_g = np.abs(A @ Ng - np.eye(n)).max()
        res_o = np.abs(A @ ref - np.eye(n)).max()
        assert res_g <= 10 * res_o + 1e-12, (res_g, res_o)
        kappa = np.linalg.cond(A)
        assert np.abs(Ng - ref).max() <= 1e-15 * kappa * np.abs(ref).max()
