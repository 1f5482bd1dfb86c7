"""The frequency-domain measurement (delayed NFFT, Sec. 2.3 Eq. nfft, and the
same sums as a dense contraction) against the oracle's plain non-uniform
Fourier sums on identical trajectories.

FP64 path: same decisions (the chain is the oracle's), and the accumulated
sum of sign * M(dr, i w_n) within 1e-10 of the oracle in the norm form
max|M_gpu - M_ora| / max|M_ora| (the Gaussian window of half-width 12 grid
points at oversampling 2 carries ~1e-12 of sum |c_ij| per frequency).  Mixed
path: the GPU replays the oracle's decisions and the error is that of its
FP32 N and FP32 spreading (window of half-width 8, ~1e-8).
"""
import numpy as np
import pytest

from oracle import ctaux
from tests.helpers import problem

pytestmark = pytest.mark.gpu


def _walkers(**kw):
    import torch
    from paper_1901_01047_gb300 import walker
    return walker.Walkers(stream=torch.cuda.current_stream().cuda_stream, **kw)


def _pair(nc, tp, U, beta, mu, n_tau, k_sub, sweeps, nw, precision="fp64", R=16, seed=0, warmup=10, walkers=1,
          recompute_at_measure=False, method="nfft"):
    c, eps, kr, G0 = problem(nc, 1.0, tp, U, beta, mu, n_tau)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)
    oracles, logs = [], []
    for wi in range(walkers):
        ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=warmup, n_tau_meas=8, seed=seed,
                                walker_id=wi)
        ow.enable_freq(nw)
        ow.enable_log(1 << 22)
        ow.sweep(sweeps)
        oracles.append(ow)
        logs.append(ow.log())
    gw = _walkers(problems=[prob], n_walkers=walkers, k_sub=k_sub, recompute_every=R, warmup_sweeps=warmup,
                  n_tau_meas=8, seed=seed, precision=precision, log_capacity=1 << 22, n_omega_meas=nw,
                  recompute_at_measure=recompute_at_measure, freq_method=method)
    for wi in range(walkers):
        gw.set_forced_decisions(wi, logs[wi])
    gw.sweep(sweeps)
    Mg, ssg, nmg = gw.measure_M()
    out = []
    for wi in range(walkers):
        ow = oracles[wi]
        Mo = ow.M()
        g, sso, nmo = ow.G()
        assert nmg[wi] == nmo > 0 and ssg[wi] == sso
        gs, os_ = gw.state(wi), ow.state()
        assert np.array_equal(gs["site"], os_["site"]) and np.array_equal(gs["tau"], os_["tau"])
        out.append(np.abs(Mg[wi] - Mo).max() / np.abs(Mo).max())
    st = gw.stats()
    gw.close()
    return out, st


@pytest.mark.parametrize("method", ["nfft", "dft"])
def test_frequency_measurement_matches_the_oracle_fp64_2x2(method):
    err, st = _pair(4, 0.0, 4.0, 10.0, 0.9450480104035819, 4096, k_sub=32, sweeps=300, nw=64, method=method)
    assert err[0] < 1e-10, err


@pytest.mark.parametrize("method", ["nfft", "dft"])
def test_frequency_measurement_matches_the_oracle_fp64_atom_and_16_sites(method):
    err, _ = _pair(1, 0.0, 4.0, 2.0, 2.0, 4096, k_sub=8, sweeps=2000, nw=16, warmup=20, method=method)
    assert err[0] < 1e-10, err
    # 16 sites, two walkers, 72 frequencies (a ragged frequency tile of the dense variant)
    err, _ = _pair(16, -0.15, 6.0, 4.0, 2.85, 2048, k_sub=64, sweeps=40, nw=72, walkers=2, method=method)
    assert max(err) < 1e-10, err


@pytest.mark.parametrize("method", ["nfft", "dft"])
def test_frequency_measurement_u0_is_exactly_zero(method):
    c, eps, kr, G0 = problem(4, 1.0, 0.0, 0.0, 3.0, 0.4, 512)
    gw = _walkers(problems=[dict(nc=4, site_sub=c.site_sub, U=0.0, beta=3.0, K=1.7, G0=G0)], n_walkers=2,
                  k_sub=16, recompute_every=8, warmup_sweeps=5, n_tau_meas=8, seed=1, n_omega_meas=16,
                  freq_method=method)
    gw.sweep(100)
    Mg, ss, nm = gw.measure_M()
    assert all(n > 0 for n in nm) and all(np.all(m == 0) for m in Mg)
    gw.close()


@pytest.mark.parametrize("method", ["nfft", "dft"])
def test_frequency_measurement_mixed_replay_error(method):
    # same trajectory; error of the FP32 N (recompute every 16 windows) and of
    # the FP32 arithmetic of the measurement (measured 1.1e-5, and 1.6e-7 with
    # N recomputed before every measurement, for the NFFT)
    err, st = _pair(4, 0.0, 4.0, 10.0, 0.9450480104035819, 4096, k_sub=32, sweeps=300, nw=64, precision="mixed",
                    method=method)
    print("mixed %s replay error:" % method, err)
    assert err[0] < 1e-4, err
    err, st = _pair(4, 0.0, 4.0, 10.0, 0.9450480104035819, 4096, k_sub=32, sweeps=300, nw=64, precision="mixed",
                    recompute_at_measure=True, method=method)
    print("mixed %s replay error, N recomputed at every measurement:" % method, err)
    assert err[0] < 1e-6, err


def test_measure_M_needs_the_frequency_measurement():
    from paper_1901_01047_gb300 import walker
    c, eps, kr, G0 = problem(4, 1.0, 0.0, 4.0, 3.0, 1.0, 256)
    gw = _walkers(problems=[dict(nc=4, site_sub=c.site_sub, U=4.0, beta=3.0, K=1.0, G0=G0)], n_walkers=1, k_sub=8,
                  recompute_every=8, warmup_sweeps=2, n_tau_meas=8, seed=1)
    gw.sweep(3)
    with pytest.raises(walker.WalkerError) as e:
        gw._check(gw._L.dca_walker_measure_M(gw._h, None, None, None))
    assert e.value.code == -6
    gw.close()
