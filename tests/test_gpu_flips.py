"""Auxiliary-spin flips and the neglect rule on the GPU against the oracle.

With flips (Sec. 2.3, the third single-spin update) the submatrix walker with
the abort rule still reaches the chain of single-spin updates: identical
decisions, vertex lists and spins, N and sum sign * G to 1e-10 (FP64).  The
neglect rule depends on the windows; the oracle replays the same windows of
k_s proposals, so the two still agree decision for decision.
"""
import numpy as np
import pytest

from oracle import ctaux
from tests.helpers import problem

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _pair(nc, tp, U, beta, mu, n_tau, k_sub, sweeps, flip, neglect=False, walkers=1, precision="fp64", R=16,
          warmup=10, ntm=16, seed=3, schedule="lockstep", replay=False, recompute_at_measure=False):
    import torch
    from paper_1901_01047_gb300 import walker
    c, eps, kr, G0 = problem(nc, 1.0, tp, U, beta, mu, n_tau)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)
    oracles = []
    for wi in range(walkers):
        ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=warmup, n_tau_meas=ntm, seed=seed,
                                walker_id=wi, flip_frac=flip, neglect_ks=k_sub if neglect else 0)
        ow.enable_log(1 << 22)
        oracles.append(ow)
    gw = walker.Walkers([prob], n_walkers=walkers, k_sub=k_sub, recompute_every=R, warmup_sweeps=warmup,
                        n_tau_meas=ntm, seed=seed, log_capacity=1 << 22, precision=precision, flip_fraction=flip,
                        duplicate_rule="neglect" if neglect else "abort", schedule=schedule,
                        recompute_at_measure=recompute_at_measure, stream=torch.cuda.current_stream().cuda_stream)
    if replay:
        for wi, ow in enumerate(oracles):
            ow.sweep(sweeps)
            gw.set_forced_decisions(wi, ow.log())
        gw.sweep(sweeps)
    else:
        gw.sweep(sweeps)
        for wi, ow in enumerate(oracles):
            ow.set_hints(gw.decision_log(wi))
            ow.sweep(sweeps)
    Gg, ssg, nmg = gw.measure_G()
    st = gw.stats()
    out = []
    for wi, ow in enumerate(oracles):
        gs, os_ = gw.state(wi), ow.state()
        glog, olog = gw.decision_log(wi), ow.log()
        assert glog.size == olog.size and np.array_equal(glog & 1, olog & 1)
        assert np.array_equal(gs["site"], os_["site"]) and np.array_equal(gs["s"], os_["s"])
        assert np.array_equal(gs["tau"], os_["tau"])
        Go, sso, nmo = ow.G()
        assert nmg[wi] == nmo
        errN = max(np.abs(gs["N"][sp] - os_["N"][sp]).max() / np.abs(os_["N"][sp]).max() for sp in range(2))
        errG = np.abs(Gg[wi] - Go).max() / np.abs(Go).max()
        out.append(dict(errN=errN, errG=errG, sign_equal=ssg[wi] == sso, neglected=st[wi]["neglected"],
                        oracle_neglected=ow.neglected, accepts=st[wi]["accepts"], aborts=st[wi]["aborts"]))
    gw.close()
    return out


@pytest.mark.parametrize("k_sub", [1, 16, 128])
def test_flips_fp64_parity(k_sub):
    res = _pair(4, 0.0, 4.0, 10.0, 0.9450480104035819, 4096, k_sub, 300, flip=1.0 / 3.0)
    for r in res:
        assert r["errN"] < TOL and r["errG"] < TOL and r["sign_equal"], r
        assert r["neglected"] == 0


def test_flips_fp64_parity_16_sites_batched():
    res = _pair(16, -0.15, 6.0, 4.0, 2.85, 2048, 64, 30, flip=0.25, walkers=3)
    for r in res:
        assert r["errN"] < TOL and r["errG"] < TOL and r["sign_equal"], r
    assert sum(r["aborts"] for r in res) > 0  # the duplicate rule fired on flipped or inserted spins


def test_neglect_rule_fp64_parity():
    res = _pair(4, 0.0, 4.0, 10.0, 0.9450480104035819, 4096, 32, 300, flip=0.2, neglect=True)
    for r in res:
        assert r["errN"] < TOL and r["errG"] < TOL and r["sign_equal"], r
        assert r["neglected"] == r["oracle_neglected"] > 0 and r["aborts"] == 0


def test_flips_mixed_replay():
    # A flip changes V by 2 gamma s (a = e^{-2V} - 1, up to e^{2 gamma} in size), so
    # the FP32 update terms of a window with flips are larger than with
    # insertions and removals alone: measured N 6.3e-4, G 3.3e-4 with a
    # recompute every 64 windows (bounds about three times that); with N
    # recomputed before every measurement G stays within 1e-6.
    res = _pair(16, -0.15, 6.0, 4.0, 2.85, 2048, 64, 40, flip=0.25, precision="mixed", replay=True, R=64)
    print("mixed replay with flips:", res)
    for r in res:
        assert r["errN"] < 2e-3 and r["errG"] < 1e-3, r
    res = _pair(16, -0.15, 6.0, 4.0, 2.85, 2048, 64, 40, flip=0.25, precision="mixed", replay=True, R=64,
                recompute_at_measure=True)
    print("mixed replay with flips, N recomputed at every measurement:", res)
    for r in res:
        assert r["errG"] < 1e-6, r


def _pair_update(nc, tp, U, beta, mu, n_tau, k_sub, sweeps, flip, walkers=1, precision="fp64", R=16, warmup=10,
                 ntm=16, seed=3, schedule="lockstep", replay=False):
    """The update rule against the oracle's plain chain of single-spin updates
    (no windows): a spin changed twice in a window is evaluated in place, so
    the chain is the same as with the abort rule, without aborts."""
    import torch
    from paper_1901_01047_gb300 import walker
    c, eps, kr, G0 = problem(nc, 1.0, tp, U, beta, mu, n_tau)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)
    oracles = []
    for wi in range(walkers):
        ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=warmup, n_tau_meas=ntm, seed=seed,
                                walker_id=wi, flip_frac=flip)
        ow.enable_log(1 << 22)
        oracles.append(ow)
    gw = walker.Walkers([prob], n_walkers=walkers, k_sub=k_sub, recompute_every=R, warmup_sweeps=warmup,
                        n_tau_meas=ntm, seed=seed, log_capacity=1 << 22, precision=precision, flip_fraction=flip,
                        duplicate_rule="update", schedule=schedule, stream=torch.cuda.current_stream().cuda_stream)
    if replay:
        for wi, ow in enumerate(oracles):
            ow.sweep(sweeps)
            gw.set_forced_decisions(wi, ow.log())
        gw.sweep(sweeps)
    else:
        gw.sweep(sweeps)
        for wi, ow in enumerate(oracles):
            ow.set_hints(gw.decision_log(wi))
            ow.sweep(sweeps)
    Gg, ssg, nmg = gw.measure_G()
    st = gw.stats()
    out = []
    for wi, ow in enumerate(oracles):
        gs, os_ = gw.state(wi), ow.state()
        glog, olog = gw.decision_log(wi), ow.log()
        assert glog.size == olog.size and np.array_equal(glog & 1, olog & 1)
        assert np.array_equal(gs["site"], os_["site"]) and np.array_equal(gs["s"], os_["s"])
        assert np.array_equal(gs["tau"], os_["tau"])
        Go, sso, nmo = ow.G()
        assert nmg[wi] == nmo
        errN = max(np.abs(gs["N"][sp] - os_["N"][sp]).max() / np.abs(os_["N"][sp]).max() for sp in range(2))
        errG = np.abs(Gg[wi] - Go).max() / max(np.abs(Go).max(), 1e-300)
        out.append(dict(errN=errN, errG=errG, sign_equal=ssg[wi] == sso, neglected=st[wi]["neglected"],
                        aborts=st[wi]["aborts"], windows=st[wi]["windows"], proposals=st[wi]["proposals"]))
    gw.close()
    return out


@pytest.mark.parametrize("k_sub", [16, 128])
def test_update_rule_fp64_parity(k_sub):
    # windows of 128 proposals on an expansion order of about 30: most windows
    # change some spin twice, and none ends early
    res = _pair_update(4, 0.0, 4.0, 10.0, 0.9450480104035819, 4096, k_sub, 300, flip=1.0 / 3.0)
    for r in res:
        assert r["errN"] < TOL and r["errG"] < TOL and r["sign_equal"], r
        assert r["aborts"] == 0 and r["neglected"] == 0, r


def test_update_rule_fp64_parity_16_sites_batched():
    for flip in (0.0, 0.25):
        res = _pair_update(16, -0.15, 6.0, 4.0, 2.85, 2048, 64, 30, flip=flip, walkers=3)
        for r in res:
            assert r["errN"] < TOL and r["errG"] < TOL and r["sign_equal"], r
            assert r["aborts"] == 0, r


def test_update_rule_mixed_replay():
    res = _pair_update(16, -0.15, 6.0, 4.0, 2.85, 2048, 64, 40, flip=0.25, precision="mixed", replay=True, R=64)
    print("mixed replay, update rule:", res)
    for r in res:
        assert r["errN"] < 2e-3 and r["errG"] < 1e-3 and r["aborts"] == 0, r
