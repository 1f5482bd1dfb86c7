"""Checkpoint and resume (dca_walker_save / dca_walker_load).

The Markov chain of a walker is fixed by its configuration, its sign, its
proposal counter (the Philox counter) and its sweep state; N is a function of
the configuration (Eq. Zk) and is rebuilt from scratch on load.  A resumed
FP64 run must therefore make the same decisions as the unbroken run, bit for
bit, and reach the same N and accumulated sign * G up to the rounding of the
rebuilt N (1e-10 in the norm form max|a - b| / max|b|).
"""
import numpy as np
import pytest

from oracle import ctaux
from tests.helpers import problem

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _walkers(**kw):
    import torch
    from paper_1901_01047_gb300 import walker
    return walker.Walkers(stream=torch.cuda.current_stream().cuda_stream, **kw)


def _setup(schedule="lockstep", precision="fp64", W=3):
    probs = []
    for beta in (4.0, 8.0):
        c, eps, kr, G0 = problem(4, 1.0, 0.0, 4.0, beta, 0.9450480104035819, 2048)
        probs.append(dict(nc=4, site_sub=c.site_sub, U=4.0, beta=beta, K=1.0, G0=G0))
    kw = dict(problems=probs, n_walkers=W, k_sub=16, recompute_every=8, warmup_sweeps=4, n_tau_meas=16, seed=13,
              log_capacity=1 << 20, schedule=schedule, precision=precision)
    return kw


def _compare_runs(a, b, W, q0):
    Ga, ssa, nma = a.measure_G()
    Gb, ssb, nmb = b.measure_G()
    sa, sb = a.stats(), b.stats()
    for wi in range(W):
        for key in ("proposals", "accepts", "sweeps", "measurements", "windows", "order"):
            assert sa[wi][key] == sb[wi][key], (wi, key, sa[wi][key], sb[wi][key])
        assert sa[wi]["sign"] == sb[wi]["sign"] and nma[wi] == nmb[wi] and ssa[wi] == ssb[wi]
        la, lb = a.decision_log(wi), b.decision_log(wi)
        assert la.size == lb.size
        assert np.array_equal(la[q0[wi]:] & 1, lb[q0[wi]:] & 1)
        ga, gb = a.state(wi), b.state(wi)
        assert np.array_equal(ga["site"], gb["site"]) and np.array_equal(ga["s"], gb["s"])
        assert np.array_equal(ga["tau"], gb["tau"])
        for sp in range(2):
            assert np.abs(ga["N"][sp] - gb["N"][sp]).max() <= TOL * np.abs(gb["N"][sp]).max()
        assert np.abs(Ga[wi] - Gb[wi]).max() <= TOL * max(np.abs(Gb[wi]).max(), 1e-300)


@pytest.mark.parametrize("schedule", ["lockstep", "pooled"])
def test_resume_equals_the_unbroken_run(schedule):
    # Under the pooled schedule the checkpoint is taken with walkers part-way
    # through a sweep; the sweep position is part of the state.
    W = 3
    kw = _setup(schedule, W=W)
    a = _walkers(**kw)
    a.sweep(7)
    ck = a.save()
    q0 = [s["proposals"] for s in a.stats()]  # no removal from an empty configuration here: q = proposals
    a.sweep(9)
    b = _walkers(**kw)
    b.load(ck)
    b.sweep(9)
    _compare_runs(a, b, W, q0)
    a.close()
    b.close()


def test_resumed_chain_is_the_oracle_chain():
    W = 2
    kw = _setup("lockstep", W=W)
    a = _walkers(**kw)
    a.sweep(6)
    ck = a.save()
    q0 = [s["proposals"] for s in a.stats()]
    a.close()
    b = _walkers(**kw)
    b.load(ck)
    b.sweep(10)
    st = b.stats()
    Gg, ssg, nmg = b.measure_G()
    for wi in range(W):
        pr = kw["problems"][wi % 2]
        ow = ctaux.OracleWalker(4, pr["site_sub"], pr["U"], pr["beta"], 1.0, pr["G0"], warmup_sweeps=4,
                                n_tau_meas=16, seed=13, walker_id=wi)
        ow.enable_log(1 << 20)
        ow.sweep(st[wi]["sweeps"])
        olog = ow.log()
        log = b.decision_log(wi)
        assert log.size == olog.size
        assert np.array_equal(log[q0[wi]:] & 1, olog[q0[wi]:] & 1)
        gs, os_ = b.state(wi), ow.state()
        assert np.array_equal(gs["site"], os_["site"]) and np.array_equal(gs["tau"], os_["tau"])
        for sp in range(2):
            assert np.abs(gs["N"][sp] - os_["N"][sp]).max() <= TOL * np.abs(os_["N"][sp]).max()
        Go, sso, nmo = ow.G()
        assert nmg[wi] == nmo and ssg[wi] == sso
        assert np.abs(Gg[wi] - Go).max() <= TOL * np.abs(Go).max()
    b.close()


def test_mixed_checkpoint_round_trip():
    W = 2
    kw = _setup("lockstep", precision="mixed", W=W)
    a = _walkers(**kw)
    a.sweep(8)
    before = [a.state(wi) for wi in range(W)]
    ck = a.save()
    b = _walkers(**kw)
    b.load(ck)
    for wi in range(W):
        s0, s1 = before[wi], b.state(wi)
        assert np.array_equal(s0["site"], s1["site"]) and np.array_equal(s0["tau"], s1["tau"])
        # the rebuilt N is the FP64 inverse rounded to FP32; the walker's own N
        # carries the drift since its last recompute (FP32 rounding amplified
        # by the conditioning of N^-1)
        for sp in range(2):
            assert np.abs(s0["N"][sp] - s1["N"][sp]).max() <= 1e-4 * np.abs(s1["N"][sp]).max()
    b.sweep(4)
    assert all(s["status"] == 0 for s in b.stats())
    a.close()
    b.close()


def test_load_rejects_a_mismatching_checkpoint_and_leaves_the_handle_usable():
    from paper_1901_01047_gb300 import walker
    kw = _setup("lockstep", W=3)
    a = _walkers(**kw)
    a.sweep(3)
    ck = a.save()
    kw2 = dict(kw, n_walkers=2)
    b = _walkers(**kw2)
    b.sweep(2)
    before = b.stats()
    with pytest.raises(walker.WalkerError) as e:
        b.load(ck)
    assert e.value.code == -1
    with pytest.raises(walker.WalkerError):
        a.load(ck[:-8])  # truncated
    bad = bytearray(ck)
    bad[0] ^= 0xFF       # not a checkpoint
    with pytest.raises(walker.WalkerError):
        a.load(bytes(bad))
    assert [s["proposals"] for s in b.stats()] == [s["proposals"] for s in before]
    b.sweep(2)
    a.sweep(2)
    assert all(s["status"] == 0 for s in a.stats() + b.stats())
    a.close()
    b.close()
