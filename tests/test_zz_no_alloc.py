"""The non-allocating from-scratch N (`dca_fresh_N_noalloc`).

Callers that cannot allocate device memory (processes whose device memory
belongs to another allocator, services with a fixed device footprint) use this
entry point; it must give the same N
and determinant sign as `dca_fresh_N`, call after call, although every call
reuses one fixed device array.  This file is collected last so that a run that
stops at the first failure has run every other test first; it also passes on
its own in a fresh process.
"""
import numpy as np
import pytest

from oracle import ctaux
from tests.helpers import problem

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def walker_mod():
    from paper_1901_01047_gb300 import build, walker
    build.build()
    walker.load()
    return walker


def _config(nc, tp, U, beta, mu, sweeps, seed):
    c, eps, kr, G0 = problem(nc, 1.0, tp, U, beta, mu, 1024)
    ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=sweeps, n_tau_meas=4, seed=seed)
    ow.sweep(sweeps)
    st = ow.state()
    return dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0), st


def _compare(walker_mod, prob, st):
    Na, Nb, sa = walker_mod.fresh_N(prob, st["site"], st["tau"], st["s"], fn="dca_fresh_N")
    Ma, Mb, sm = walker_mod.fresh_N(prob, st["site"], st["tau"], st["s"], fn="dca_fresh_N_noalloc")
    assert sm == sa
    for ref, got in ((Na, Ma), (Nb, Mb)):
        assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(walker_mod):
    # two different configurations in a row: the second call must not see the
    # first call's contents of the shared array
    prob1, st1 = _config(4, 0.0, 4.0, 10.0, 0.9450480104035819, 60, seed=4)
    prob2, st2 = _config(16, -0.15, 6.0, 2.0, 2.85, 15, seed=5)
    assert st1["site"].size != st2["site"].size
    _compare(walker_mod, prob1, st1)
    _compare(walker_mod, prob2, st2)
    _compare(walker_mod, prob1, st1)


def test_noalloc_at_its_largest_order_matches_the_oracle(walker_mod):
    # n = DCA_NOALLOC_MAX_ORDER exactly: every piece of the fixed array at its
    # largest size.  A random configuration, checked against the oracle's
    # inverse (residual and kappa-scaled agreement) and against the allocating
    # entry point, twice in a row.
    n, nc, U, beta = 256, 16, 1.0, 5.0
    c, eps, kr, G0 = problem(nc, 1.0, -0.15, U, beta, 0.3, 1024)
    rng = np.random.default_rng(256)
    site = rng.integers(0, nc, n).astype(np.int32)
    tau = rng.uniform(0, beta, n)
    s = rng.choice([-1, 1], n).astype(np.int8)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)
    ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, init_config_size=0)
    ow.set_config(site, tau, s)
    for _ in range(2):
        Nu, Nd, sg = walker_mod.fresh_N(prob, site, tau, s, fn="dca_fresh_N_noalloc")
        assert sg == int(ow.sign)
        for sp, Ng in enumerate((Nu, Nd)):
            ref, _ = ow.fresh_N(sp)
            A = ow.build_A(sp, site, tau, s)
            assert np.abs(A @ Ng - np.eye(n)).max() <= 10 * np.abs(A @ ref - np.eye(n)).max() + 1e-12
            assert np.abs(Ng - ref).max() <= 1e-15 * np.linalg.cond(A) * np.abs(ref).max()
        _compare(walker_mod, prob, dict(site=site, tau=tau, s=s))


def test_noalloc_rejects_sizes_beyond_its_array(walker_mod):
    prob, st = _config(4, 0.0, 4.0, 2.0, 1.0, 5, seed=1)
    n = 257
    rng = np.random.default_rng(0)
    site = rng.integers(0, 4, n)
    tau = np.sort(rng.uniform(0, 2.0, n))
    s = rng.choice([-1, 1], n)
    with pytest.raises(walker_mod.WalkerError, match="beyond the fixed scratch"):
        walker_mod.fresh_N(prob, site, tau, s, fn="dca_fresh_N_noalloc")
    # still usable afterwards
    _compare(walker_mod, prob, st)
