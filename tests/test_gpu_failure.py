"""Failure detection of the walker library, exercised without faulting the GPU.

Every failure here is made on the host or by a bounded wait that is given a
short bound: the window loop's iteration bound, the mbarrier wait bound of the
tensor-core kernels, a bare propagator whose entries overflow the arithmetic,
and a matrix capacity below the walker's natural order.  Each case checks the
error code, that the handle stays usable (stats, checkpoint, further sweeps),
and, where the chain goes on, that it is still the oracle's chain.
"""
import numpy as np
import pytest

from oracle import ctaux
from tests.helpers import problem

pytestmark = pytest.mark.gpu

TIMEOUT, NUMERIC, CAPACITY = -4, -5, -7


def _walkers(**kw):
    import torch
    from paper_1901_01047_gb300 import walker
    return walker.Walkers(stream=torch.cuda.current_stream().cuda_stream, **kw)


def _err():
    from paper_1901_01047_gb300 import walker
    return walker.WalkerError


def test_loop_iteration_bound_gives_timeout_and_the_chain_goes_on():
    nc, U, beta, mu = 4, 4.0, 6.0, 0.9450480104035819
    c, eps, kr, G0 = problem(nc, 1.0, 0.0, U, beta, mu, 2048)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)
    gw = _walkers(problems=[prob], n_walkers=2, k_sub=8, recompute_every=16, warmup_sweeps=3, n_tau_meas=8,
                  seed=21, log_capacity=1 << 20)
    gw.set_limits(max_windows=3)
    gw.sweep(40, sync=False)
    with pytest.raises(_err()) as e:
        gw.sync()
    assert e.value.code == TIMEOUT
    st = gw.stats()
    assert all(s["status"] == 0 for s in st) and all(s["windows"] == 3 for s in st)
    # the bound stopped the loop, not the chains: lift it and carry on
    gw.set_limits(0, 0)
    gw.sweep(5)
    sweeps = [s["sweeps"] for s in gw.stats()]
    for wi in range(2):
        log = gw.decision_log(wi)
        ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=3, n_tau_meas=8, seed=21,
                                walker_id=wi)
        ow.enable_log(1 << 20)
        ow.set_hints(log)
        ow.sweep(sweeps[wi])
        olog = ow.log()
        assert np.array_equal(log[:olog.size] & 1, olog & 1)
        gs, os_ = gw.state(wi), ow.state()
        assert np.array_equal(gs["site"], os_["site"])
        for sp in range(2):
            assert np.abs(gs["N"][sp] - os_["N"][sp]).max() <= 1e-10 * np.abs(os_["N"][sp]).max()
    gw.close()


def test_mbarrier_wait_bound_gives_timeout_and_a_checkpoint_restores_the_walkers():
    # Mixed precision on the tensor cores: with a wait bound of one SM clock
    # the first mbarrier wait that is not already complete gives up.  The
    # kernel stops the walkers it served with DCA_ERR_TIMEOUT, lets its copies
    # land, frees its tensor memory and returns; the context stays usable and a
    # checkpoint taken before brings the walkers back.
    nc, U, beta, mu = 16, 6.0, 4.0, 2.85
    c, eps, kr, G0 = problem(nc, 1.0, -0.15, U, beta, mu, 2048)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)
    gw = _walkers(problems=[prob], n_walkers=4, k_sub=32, recompute_every=0, recompute_sweeps=4,
                  warmup_sweeps=2, n_tau_meas=16, seed=5, precision="mixed", update_kernel="tcgen05")
    gw.sweep(3)
    ck = gw.save()
    gw.set_limits(wait_cycles=1)
    gw.sweep(2, sync=False)
    with pytest.raises(_err()) as e:
        gw.sync()
    assert e.value.code == TIMEOUT
    st = gw.stats()
    assert any(s["status"] == TIMEOUT for s in st)
    assert all(s["status"] in (0, TIMEOUT) for s in st)
    gw.set_limits(0, 0)
    gw.load(ck)
    assert all(s["status"] == 0 for s in gw.stats())
    gw.sweep(3)
    # the restored walkers follow the chains of an unbroken copy resumed from the same checkpoint
    ref = _walkers(problems=[prob], n_walkers=4, k_sub=32, recompute_every=0, recompute_sweeps=4,
                   warmup_sweeps=2, n_tau_meas=16, seed=5, precision="mixed", update_kernel="tcgen05")
    ref.load(ck)
    ref.sweep(3)
    for a, b in zip(gw.stats(), ref.stats()):
        assert a["status"] == 0 and a["proposals"] == b["proposals"] and a["order"] == b["order"]
    gw.close()
    ref.close()


def test_overflowing_bare_propagator_gives_numeric_error():
    # A propagator whose entries are finite but so large that the candidate
    # products overflow: the first non-finite ratio stops the walker with
    # DCA_ERR_NUMERIC instead of a silent NaN chain.
    nc, U, beta, mu = 4, 4.0, 4.0, 1.0
    c, eps, kr, G0 = problem(nc, 1.0, 0.0, U, beta, mu, 1024)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)
    for precision in ("fp64", "mixed"):
        gw = _walkers(problems=[prob], n_walkers=2, k_sub=16, recompute_every=8, warmup_sweeps=2, n_tau_meas=8,
                      seed=2, precision=precision)
        gw.sweep(3)
        gw.update_G0(0, G0 * 1e300)
        gw.sweep(3, sync=False)
        with pytest.raises(_err()) as e:
            gw.sync()
        assert e.value.code == NUMERIC, (precision, e.value.code)
        assert any(s["status"] == NUMERIC for s in gw.stats())
        gw.close()


def test_capacity_below_the_natural_order_gives_capacity_error():
    nc, U, beta, mu = 16, 6.0, 4.0, 2.85
    c, eps, kr, G0 = problem(nc, 1.0, -0.15, U, beta, mu, 1024)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)
    for precision in ("fp64", "mixed"):
        gw = _walkers(problems=[prob], n_walkers=2, k_sub=16, recompute_every=8, warmup_sweeps=2, n_tau_meas=8,
                      seed=3, precision=precision, capacity=64)
        assert gw.capacity(0) == 64
        gw.sweep(40, sync=False)
        with pytest.raises(_err()) as e:
            gw.sync()
        assert e.value.code == CAPACITY
        st = gw.stats()
        assert all(s["status"] == CAPACITY for s in st)
        assert all(s["order"] <= 64 for s in st)
        gw.close()


def test_non_finite_table_given_to_update_G0_is_rejected_on_the_device():
    nc, U, beta, mu = 4, 4.0, 4.0, 1.0
    c, eps, kr, G0 = problem(nc, 1.0, 0.0, U, beta, mu, 1024)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)
    gw = _walkers(problems=[prob], n_walkers=1, k_sub=16, recompute_every=8, warmup_sweeps=2, n_tau_meas=8, seed=2,
                  log_capacity=1 << 20)
    bad = G0.copy()
    bad[1, 2, 3] = np.nan
    gw.update_G0(0, bad)
    with pytest.raises(_err()) as e:
        gw.sync()
    assert e.value.code == -1
    # the old table stayed: the chain is the oracle's chain on the original G0
    gw.sweep(20)
    log = gw.decision_log(0)
    ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=2, n_tau_meas=8, seed=2)
    ow.enable_log(1 << 20)
    ow.set_hints(log)
    ow.sweep(20)
    assert np.array_equal(ow.log() & 1, log & 1)
    gw.close()


def test_update_G0_all_takes_the_finite_tables_and_rejects_the_others():
    # two problems; one call replaces both tables: problem 0 gets a new finite
    # table (another chemical potential), problem 1 a table with a NaN, which
    # is rejected while problem 0's is taken
    nc, U, beta = 4, 4.0, 4.0
    c, eps, kr, G0a = problem(nc, 1.0, 0.0, U, beta, 1.0, 1024)
    _, _, _, G0b = problem(nc, 1.0, 0.0, U, 3.0, 0.8, 1024)
    _, _, _, G0a_new = problem(nc, 1.0, 0.0, U, beta, 1.3, 1024)
    probs = [dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0a),
             dict(nc=nc, site_sub=c.site_sub, U=U, beta=3.0, K=1.0, G0=G0b)]
    gw = _walkers(problems=probs, n_walkers=2, k_sub=16, recompute_every=8, warmup_sweeps=2, n_tau_meas=8, seed=5,
                  log_capacity=1 << 20)
    bad = G0b.copy()
    bad[0, 1, 7] = np.inf
    gw.update_G0_all([G0a_new, bad])
    with pytest.raises(_err()) as e:
        gw.sync()
    assert e.value.code == -1
    gw.sweep(20)
    for wi, (b, g0) in enumerate(((beta, G0a_new), (3.0, G0b))):
        log = gw.decision_log(wi)
        ow = ctaux.OracleWalker(nc, c.site_sub, U, b, 1.0, g0, warmup_sweeps=2, n_tau_meas=8, seed=5, walker_id=wi)
        ow.enable_log(1 << 20)
        ow.set_hints(log)
        ow.sweep(20)
        assert np.array_equal(ow.log() & 1, log & 1), wi
        Go, sso, _ = ow.G()
        Gg, ssg, _ = gw.measure_G()
        assert np.abs(Gg[wi] - Go).max() < 1e-10 * np.abs(Go).max()
    # a finite pair of tables: no error
    gw.update_G0_all(np.concatenate([G0a.reshape(-1), G0b.reshape(-1)]))
    gw.sync()
    gw.close()
