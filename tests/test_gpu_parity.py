"""GPU walker (FP64) against the oracle on identical seeded inputs.

The submatrix algorithm reaches exactly the chain of single-spin updates, so
for the same Philox stream both sides must take the same decisions (the
oracle adopts the GPU's decision only where | |R| - u | < 1e-10), end with the
same vertex list, and agree on N and on the accumulated sign * G to 1e-10 in
the norm form max|X_gpu - X_oracle| / max|X_oracle|.
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
    kw.setdefault("stream", torch.cuda.current_stream().cuda_stream)
    return walker.Walkers(**kw)


def run_pair(nc, t, tp, U, beta, mu, n_tau, k_sub, sweeps, seed=0, warmup=10, init=10, ntm=16, R=0,
             walkers=1, K=1.0, chunks=1, timed=False, R_sweeps=0):
    c, eps, kr, G0 = problem(nc, t, tp, U, beta, mu, n_tau)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=K, G0=G0)
    gw = _walkers(problems=[prob], n_walkers=walkers, k_sub=k_sub, recompute_every=R, warmup_sweeps=warmup,
                  n_tau_meas=ntm, init_config_size=init, seed=seed, log_capacity=1 << 23,
                  recompute_sweeps=R_sweeps)
    if timed:  # host-driven window loop with CUDA events instead of the graph loop
        from paper_1901_01047_gb300 import walker
        gw.set_timing(walker.GROUPS)
    for _ in range(chunks):
        gw.sweep(sweeps // chunks)
    Gg, ssg, nmg = gw.measure_G()
    st = gw.stats()
    results = []
    for wi in range(walkers):
        log = gw.decision_log(wi)
        ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, K, G0, warmup_sweeps=warmup, n_tau_meas=ntm, seed=seed,
                                walker_id=wi, init_config_size=init)
        ow.enable_log(1 << 23)
        ow.set_hints(log)
        ow.sweep(sweeps)
        results.append((gw.state(wi), ow.state(), log, ow.log(), Gg[wi], ssg[wi], nmg[wi], ow.G(), st[wi],
                        ow.counters()))
    gw.close()
    return results


def check(results):
    for gs, os_, glog, olog, Gg, ssg, nmg, (Go, sso, nmo), st, oc in results:
        assert glog.size == olog.size
        assert np.array_equal(glog & 1, olog & 1)
        assert st["proposals"] == oc["proposals"]
        assert np.array_equal(gs["site"], os_["site"])
        assert np.array_equal(gs["s"], os_["s"])
        assert np.array_equal(gs["tau"], os_["tau"])
        for sp in range(2):
            ref = os_["N"][sp]
            if ref.size:
                assert np.abs(gs["N"][sp] - ref).max() <= TOL * np.abs(ref).max()
        assert nmg == nmo and ssg == sso
        assert np.abs(Gg - Go).max() <= TOL * max(np.abs(Go).max(), 1e-300)
        assert st["status"] == 0


def test_atom_parity():
    # Hubbard atom Nc=1, U=4, beta=2, half filling, K=1, k_s=8, 4096-point G0
    res = run_pair(1, 0.0, 0.0, 4.0, 2.0, 2.0, 4096, k_sub=8, sweeps=3000, seed=0, warmup=20, ntm=64)
    check(res)


def test_2x2_parity_dense_run():
    # 2x2 cluster, t=1, U=4, beta=10, density 0.9 (mu from ED), k_s=32
    res = run_pair(4, 1.0, 0.0, 4.0, 10.0, 0.9450480104035819, 4096, k_sub=32, sweeps=400, seed=0, warmup=20,
                   ntm=32, R=16)
    check(res)
    st = res[0][8]
    assert st["recomputes"] > 0 and st["max_drift"] < 1e-10
    assert st["aborts"] > 0  # the duplicate-spin rule fired


def test_2x2_full_run_parity():
    # 2x2 cluster workload at full length: one walker, 1e5 sweeps after 20 warm-up
    # sweeps, k_s = 32, N recomputed every 64 submatrix updates.
    res = run_pair(4, 1.0, 0.0, 4.0, 10.0, 0.9450480104035819, 4096, k_sub=32, sweeps=100020, seed=0,
                   warmup=20, ntm=64, R=64)
    check(res)
    st = res[0][8]
    assert st["proposals"] > 3_000_000 and st["max_drift"] < 1e-9


def test_betts16_parity_at_order_1000():
    # 16-site cluster workload (t' = -0.15, U = 6, beta = 20, density 0.9,
    # k_s = 64, N recomputed every 64 submatrix updates), shortened to a few
    # sweeps.  It starts from 1000 random vertices, so the first sweeps run at
    # order ~1000 while the chain relaxes towards its equilibrium order (~760):
    # FP64 parity at the matrix sizes of the workload.  N^-1 is ill-conditioned
    # there (kappa ~ 1e7 and more), so two exact-in-FP64 algorithms (the
    # oracle's rank-1 updates, the GPU's rank-k updates and recomputes) agree
    # on N only to about kappa * 2^-53: the bound is max(1e-10, 50 kappa 2^-53),
    # and the GPU's N must be as close to the FP64 inverse of its final
    # configuration as the oracle's is.  The estimator multiplies N by
    # e^V - 1 (up to e^gamma ~ 1.9e3 here), so the accumulated G may differ
    # by up to e^gamma kappa 2^-53.  Decisions and vertices are exact.
    from paper_1901_01047_gb300 import inputs
    wl = inputs.WORKLOADS["betts16"]
    c, eps, kr, G0 = problem(16, 1.0, -0.15, 6.0, 20.0, wl.mu, 4096)
    res = run_pair(16, 1.0, -0.15, 6.0, 20.0, wl.mu, 4096, k_sub=64, sweeps=5, seed=0, warmup=2, init=1000,
                   ntm=64, R=64)
    gs, os_, glog, olog, Gg, ssg, nmg, (Go, sso, nmo), st, oc = res[0]
    assert glog.size == olog.size and np.array_equal(glog & 1, olog & 1)
    assert st["proposals"] == oc["proposals"] > 3000 and st["status"] == 0
    assert np.array_equal(gs["site"], os_["site"]) and np.array_equal(gs["s"], os_["s"])
    assert np.array_equal(gs["tau"], os_["tau"])
    assert nmg == nmo == 3 and ssg == sso and st["recomputes"] >= 1 and gs["site"].size > 700
    ow = ctaux.OracleWalker(16, c.site_sub, 6.0, 20.0, 1.0, G0, init_config_size=0)
    ow.set_config(gs["site"], gs["tau"], gs["s"])
    kappa = 0.0
    for sp in range(2):
        ref = os_["N"][sp]
        exact, _ = ow.fresh_N(sp)
        k_sp = np.linalg.cond(ref)
        kappa = max(kappa, k_sp)
        tol = max(TOL, 50 * k_sp * 2.0 ** -53)
        err = np.abs(gs["N"][sp] - ref).max() / np.abs(ref).max()
        e_gpu = np.abs(gs["N"][sp] - exact).max() / np.abs(exact).max()
        e_ora = np.abs(ref - exact).max() / np.abs(exact).max()
        print("order %d spin %d: kappa %.2e, |N_gpu - N_ora| %.2e (bound %.2e), to the exact inverse: GPU %.2e, "
              "oracle %.2e" % (gs["site"].size, sp, k_sp, err, tol, e_gpu, e_ora))
        assert err <= tol
        assert e_gpu <= 10 * e_ora + 1e-13
    errG = np.abs(Gg - Go).max() / np.abs(Go).max()
    e_gamma = np.exp(ow.gamma)
    print("accumulated G: %.2e (bound %.2e)" % (errG, e_gamma * kappa * 2.0 ** -53))
    assert errG <= max(TOL, e_gamma * kappa * 2.0 ** -53)


@pytest.mark.parametrize("k_sub", [1, 3, 16, 128])
def test_window_sizes_reach_the_same_chain(k_sub):
    res = run_pair(4, 1.0, 0.0, 4.0, 5.0, 1.2, 1024, k_sub=k_sub, sweeps=120, seed=3, warmup=5, ntm=8)
    check(res)


def test_host_driven_timed_loop_reaches_the_same_chain():
    res = run_pair(4, 1.0, 0.0, 4.0, 6.0, 1.1, 1024, k_sub=16, sweeps=150, seed=8, warmup=5, ntm=8, R=8,
                   walkers=3, chunks=3, timed=True)
    check(res)


def test_empty_initial_configuration_and_chunked_calls():
    res = run_pair(4, 1.0, -0.15, 3.0, 4.0, 0.8, 512, k_sub=16, sweeps=200, seed=5, warmup=0, init=0, ntm=8,
                   chunks=4)
    check(res)


def test_u0_keeps_N_identity_and_measures_G0():
    res = run_pair(4, 1.0, 0.0, 0.0, 3.0, 0.4, 512, k_sub=8, sweeps=300, seed=11, warmup=10, ntm=16, K=1.7)
    check(res)
    gs = res[0][0]
    for sp in range(2):
        assert np.array_equal(gs["N"][sp], np.eye(gs["site"].size))


def test_batched_walkers_match_their_own_oracles():
    res = run_pair(4, 1.0, 0.0, 4.0, 6.0, 1.0, 1024, k_sub=16, sweeps=80, seed=9, warmup=5, ntm=8, walkers=5,
                   R=8)
    check(res)
    logs = [r[2] for r in res]
    assert not np.array_equal(logs[0][:50], logs[1][:50])  # independent streams


def test_g0_builder_matches_oracle_builder():
    from paper_1901_01047_gb300 import inputs, walker
    from oracle import g0 as og0
    for nc, tp, U, beta, mu in [(1, 0.0, 4.0, 2.0, 2.0), (4, 0.0, 4.0, 10.0, 0.945), (16, -0.15, 6.0, 20.0, 2.85),
                                (36, 0.0, 7.0, 30.0, 3.49)]:
        c = inputs.cluster(nc)
        eps = inputs.square_dispersion(c.kpts, 1.0, tp)
        kr = inputs.k_dot_r(c)
        ref = og0.g0_table(eps, kr, mu, U, beta, 2048)
        got = walker.g0_isolated_cluster(eps, kr, mu, U, beta, 2048)
        assert np.abs(got - ref).max() < 1e-13


def test_batched_sweep_synchronised_recompute_keeps_parity():
    # Eight walkers recompute together after the first window of every third
    # sweep; in FP64 a recompute changes N only by rounding, so every chain
    # still matches the oracle (which never recomputes) decision for decision.
    res = run_pair(4, 1.0, 0.0, 4.0, 6.0, 0.9450480104035819, 2048, k_sub=16, sweeps=60, seed=5, warmup=6,
                   walkers=8, R_sweeps=3)
    check(res)
    for r in res:
        st = r[8]
        assert st["recomputes"] == (60 - 1) // 3, st["recomputes"]
        assert st["max_drift"] < 1e-9


def test_retuning_k_sub_between_sweeps_keeps_the_chain():
    # k_s only groups proposals into windows: changing it between sweeps (as
    # the autotuner does) leaves every decision and N unchanged.
    nc, U, beta, mu = 4, 4.0, 6.0, 0.9450480104035819
    c, eps, kr, G0 = problem(nc, 1.0, 0.0, U, beta, mu, 2048)
    prob = dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)
    gw = _walkers(problems=[prob], n_walkers=3, k_sub=16, recompute_every=8, warmup_sweeps=5, n_tau_meas=8,
                  seed=9, log_capacity=1 << 22)
    for ks in (16, 64, 3, 128, 32):
        gw.set_tuning(ks)
        gw.sweep(8)
    for wi in range(3):
        log = gw.decision_log(wi)
        ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=5, n_tau_meas=8, seed=9,
                                walker_id=wi)
        ow.enable_log(1 << 22)
        ow.set_hints(log)
        ow.sweep(40)
        assert np.array_equal(log & 1, ow.log() & 1)
        gs, os_ = gw.state(wi), ow.state()
        assert np.array_equal(gs["site"], os_["site"])
        for sp in range(2):
            ref = os_["N"][sp]
            assert np.abs(gs["N"][sp] - ref).max() <= TOL * np.abs(ref).max()
    gw.close()


def test_pooled_schedule_keeps_every_chain():
    # Pooled schedule: the walkers (beta = 3 and 8) share a budget of 6 sweeps
    # each and all take part in every window, so they complete different
    # numbers of sweeps.  Each chain is still its own Markov chain: its
    # decisions and its accumulated sign * G equal those of its oracle run for
    # the sweeps it completed.
    nc, U, mu, n_tau, ntm, warm, seed = 4, 4.0, 0.9450480104035819, 2048, 8, 3, 4
    c = None
    probs, setups = [], []
    for beta in (3.0, 8.0):
        c, eps, kr, G0 = problem(nc, 1.0, 0.0, U, beta, mu, n_tau)
        probs.append(dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0))
        setups.append((beta, G0))
    W = 4
    wp = np.arange(W, dtype=np.int32) % 2
    gw = _walkers(problems=probs, n_walkers=W, walker_problem=wp, k_sub=16, recompute_every=8,
                  warmup_sweeps=warm, n_tau_meas=ntm, seed=seed, log_capacity=1 << 22, schedule="pooled")
    gw.sweep(6)
    Gg, ssg, nmg = gw.measure_G()
    st = gw.stats()
    sweeps = [s["sweeps"] for s in st]
    assert sum(sweeps) >= 6 * W
    for wi in range(W):
        beta, G0 = setups[wp[wi]]
        log = gw.decision_log(wi)
        ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=warm, n_tau_meas=ntm, seed=seed,
                                walker_id=wi)
        ow.enable_log(1 << 22)
        ow.set_hints(log)
        ow.sweep(sweeps[wi])
        olog = ow.log()
        assert log.size >= olog.size
        assert np.array_equal(log[:olog.size] & 1, olog & 1)
        Go, sso, nmo = ow.G()
        assert nmg[wi] == nmo and ssg[wi] == sso
        assert np.abs(Gg[wi] - Go).max() <= TOL * max(np.abs(Go).max(), 1e-300)
        assert st[wi]["status"] == 0
    gw.close()
