"""The benchmarked configuration replayed against the oracle.

The throughput figures are taken on a batch of many walkers of uneven order
under the pooled schedule, mixed precision on the tensor cores, the batched
recompute every 8 sweeps, autotuned k_s and a spin changed twice in a
window applied in place, with the captured window split into four
concurrent branches (128 walkers or more).  Here that configuration
runs with a few of its walkers replaying the oracle's decisions (one walker
in each branch, the largest at order >= 1000), k_s switched from 64 to 128
part-way, and every replayed walker is compared with its own oracle chain:
the configuration exactly, N against the FP64 inverse of that configuration,
and the accumulated sign * G against the oracle's, both in the norm form
max|x - ref| / max|ref|.  The other walkers run free.

The error bounds are the mixed path's error budget (FP32 storage of N, 3xTF32
products rounded to TF32 in both split halves, FP32 measurement arithmetic),
measured on these workloads with head room for other trajectories.
"""
import threading

import numpy as np
import pytest

from oracle import ctaux
from tests.helpers import problem

pytestmark = pytest.mark.gpu

# Mixed-path bounds, about three times the largest errors measured on these
# chains (the error budget of the mixed path: FP32 storage of N and the drift
# of the 3xTF32 updates between recomputes).  Batch of orders up to ~1180,
# recompute every 8 sweeps: N 1.4e-4, G 3.4e-5.  36-site walkers (order
# ~700, recompute every 4 sweeps, a sign problem): N 1.8e-4, G 5.9e-4.  With
# N recomputed before every measurement, G is limited by the FP32
# measurement arithmetic: measured 5e-8 .. 3.1e-7 on both; the bound is the
# target of the mixed path, 1e-6.
TOL_N = 5e-4
TOL_G_BATCH = 1e-4
TOL_G_36 = 2e-3
TOL_G_FRESH = 1e-6


class _OracleRun(threading.Thread):
    """One oracle chain swept `sweeps` times, with a snapshot of its
    configuration, counters and G accumulators after every sweep (the oracle's
    C calls release the interpreter lock, so the chains run in parallel)."""

    def __init__(self, pr, seed, walker_id, warmup, ntm, init, sweeps):
        super().__init__(daemon=True)
        self.args = (pr, seed, walker_id, warmup, ntm, init, sweeps)
        self.snaps = []
        self.log = None
        self.error = None

    def run(self):
        try:
            pr, seed, walker_id, warmup, ntm, init, sweeps = self.args
            ow = ctaux.OracleWalker(pr["nc"], pr["site_sub"], pr["U"], pr["beta"], 1.0, pr["G0"],
                                    warmup_sweeps=warmup, n_tau_meas=ntm, seed=seed, walker_id=walker_id,
                                    init_config_size=init)
            ow.enable_log(1 << 26)
            self.snaps.append(self._snap(ow))
            for _ in range(sweeps):
                ow.sweep(1)
                self.snaps.append(self._snap(ow))
            self.log = ow.log()
            self.oracle = ow
        except Exception as e:  # reported by the test
            self.error = e

    @staticmethod
    def _snap(ow):
        st = ow.state()
        G, ss, nm = ow.G()
        return dict(site=st["site"], tau=st["tau"], s=st["s"], G=G, sign_sum=ss, n_meas=nm,
                    proposals=ow.counters()["proposals"], order=ow.order)


def _problem(nc, U, beta, n_tau=2048):
    c, eps, kr, G0 = problem(nc, 1.0, 0.0, U, beta, U / 2, n_tau)
    return dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)


def _exact_N(pr, st):
    ow = ctaux.OracleWalker(pr["nc"], pr["site_sub"], pr["U"], pr["beta"], 1.0, pr["G0"], init_config_size=0)
    ow.set_config(st["site"], st["tau"], st["s"])
    return ow.fresh_N(0)[0], ow.fresh_N(1)[0]


def _oracle_runs(probs, replay, warmup, ntm, init, oracle_sweeps, seed):
    runs = {}
    for wi in replay:
        runs[wi] = _OracleRun(probs[wi], seed, wi, warmup, ntm, init, oracle_sweeps[wi])
        runs[wi].start()
    for r in runs.values():
        r.join()
        assert r.error is None, r.error
    return runs


def _replay_batch(probs, runs, warmup, ntm, init, target_walker, target_sweeps, schedule, ks_switch,
                  recompute_sweeps, seed, recompute_at_measure=False):
    """Run the batch with the replayed walkers forced onto their oracle chains
    and compare them with the oracle at a common sweep boundary."""
    import torch
    from paper_1901_01047_gb300 import walker

    W = len(probs)
    replay = sorted(runs)
    gw = walker.Walkers(probs, n_walkers=W, walker_problem=np.arange(W), k_sub=64, recompute_every=0,
                        recompute_sweeps=recompute_sweeps, warmup_sweeps=warmup, n_tau_meas=ntm, precision="mixed",
                        update_kernel="tcgen05", init_config_size=init, seed=seed, schedule=schedule,
                        log_capacity=1 << 26, recompute_at_measure=recompute_at_measure,
                        duplicate_rule="update", stream=torch.cuda.current_stream().cuda_stream)
    for wi in replay:
        gw.set_forced_decisions(wi, runs[wi].log)
    max_order = {wi: 0 for wi in replay}
    switched = False
    calls = 0
    while True:
        st = gw.stats()
        for wi in replay:
            max_order[wi] = max(max_order[wi], st[wi]["order"])
        done = st[target_walker]["sweeps"]
        # stop at the target, or before any replayed walker outruns its oracle chain
        if done >= target_sweeps or any(st[wi]["sweeps"] + 3 >= len(runs[wi].snaps) for wi in replay):
            break
        if not switched and done >= ks_switch:
            gw.set_tuning(128)  # the autotuner's other candidate, on the same chains
            switched = True
        gw.sweep(1)
        calls += 1
        assert calls < 5000
    assert switched
    # bring every walker to a sweep boundary
    gw.set_schedule("lockstep")
    gw.sweep(1)
    st = gw.stats()
    Gg, ssg, nmg = gw.measure_G()
    out = []
    for wi in replay:
        run = runs[wi]
        m = st[wi]["sweeps"]
        assert st[wi]["status"] == 0
        assert m < len(run.snaps), (wi, m, len(run.snaps))
        assert st[wi]["proposals"] <= run.log.size  # every decision was the oracle's
        snap = run.snaps[m]
        gs = gw.state(wi)
        assert st[wi]["proposals"] == snap["proposals"]
        assert np.array_equal(gs["site"], snap["site"]) and np.array_equal(gs["s"], snap["s"])
        assert np.array_equal(gs["tau"], snap["tau"])
        assert nmg[wi] == snap["n_meas"] and ssg[wi] == snap["sign_sum"] and nmg[wi] > 0
        Nu, Nd = _exact_N(probs[wi], gs)
        errN = max(np.abs(gs["N"][0] - Nu).max() / np.abs(Nu).max(), np.abs(gs["N"][1] - Nd).max() / np.abs(Nd).max())
        errG = np.abs(Gg[wi] - snap["G"]).max() / np.abs(snap["G"]).max()
        out.append(dict(walker=wi, sweeps=m, order=st[wi]["order"], max_order=max_order[wi], errN=float(errN),
                        errG=float(errG), recomputes=st[wi]["recomputes"], measurements=int(nmg[wi])))
    # every walker's sign at the end and over its measurements
    signs = [bool(st[wi]["sign"] == 1.0 and ssg[wi] == nmg[wi]) for wi in range(W)]
    gw.close()
    return out, signs


def test_batched_pooled_four_branch_replay_at_bench_scale():
    # 128 walkers: four branches of 32.  Replayed walkers 5, 40, 77 and 127 (one
    # per branch, 127 the last walker of the last branch) with orders from a
    # few hundred to over a thousand; the free walkers take the bench's
    # parameter ranges (N_c 8 / 16, beta in [5, 25], U in [4, 7], half filling).
    # As in the bench, every walker starts from 10 vertices and warms up
    # (here 26 sweeps, with the batched recompute at sweeps 8, 16 and 24), then
    # measures.
    W, seed, warmup, ntm, init = 128, 7, 26, 64, 10
    rng = np.random.default_rng(2024)
    spec = {5: (8, 6.0, 20.0), 40: (16, 5.5, 12.0), 77: (8, 7.0, 25.0), 127: (16, 7.0, 25.0)}
    free = {wi: (8 if wi % 2 == 0 else 16, rng.uniform(4.0, 7.0), rng.uniform(5.0, 25.0)) for wi in range(W)}
    cache = {}

    def make_problem(wi):
        nc, U, beta = spec.get(wi, free[wi])
        key = (nc, round(U, 12), round(beta, 12))
        if key not in cache:
            cache[key] = _problem(nc, U, beta)
        return cache[key]

    probs = [make_problem(wi) for wi in range(W)]
    runs = _oracle_runs(probs, spec, warmup, ntm, init, {5: 90, 40: 75, 77: 65, 127: 34}, seed)
    kw = dict(warmup=warmup, ntm=ntm, init=init, target_walker=127, target_sweeps=30, schedule="pooled",
              ks_switch=28, recompute_sweeps=8, seed=seed)
    res, signs = _replay_batch(probs, runs, **kw)
    print("bench-scale replay:", res)
    big = [r for r in res if r["walker"] == 127][0]
    assert big["max_order"] >= 1000, big
    assert all(r["recomputes"] >= 3 and r["measurements"] >= 2 for r in res), res
    for r in res:
        assert r["errN"] < TOL_N and r["errG"] < TOL_G_BATCH, r
    # Half filling on bipartite clusters (t' = 0): no sign problem, so every
    # walker, free-running ones included, keeps sign +1 in every measurement.
    assert signs == [True] * W, [wi for wi, ok in enumerate(signs) if not ok]
    # the same chains with N recomputed before every measurement
    res, signs = _replay_batch(probs, runs, recompute_at_measure=True, **kw)
    print("bench-scale replay, N recomputed at every measurement:", res)
    for r in res:
        assert r["errG"] < TOL_G_FRESH, r
    assert signs == [True] * W


def test_betts36_walkers_replay_the_oracle():
    # 36-site walkers (config of the 2048-point measurement, shortened: beta = 8
    # instead of 30, so that the oracle replays them in seconds; measured on a
    # 64-point grid of the same phase-table kind).  32 walkers: two branches.
    W, seed, warmup, ntm, init = 32, 7, 5, 64, 500
    c, eps, kr, G0 = problem(36, 1.0, 0.0, 7.0, 8.0, 3.4878678207599574, 4096)
    pr = dict(nc=36, site_sub=c.site_sub, U=7.0, beta=8.0, K=1.0, G0=G0)
    probs = [pr] * W
    runs = _oracle_runs(probs, [3, 20], warmup, ntm, init, {3: 11, 20: 11}, seed)
    kw = dict(warmup=warmup, ntm=ntm, init=init, target_walker=3, target_sweeps=8, schedule="lockstep",
              ks_switch=3, recompute_sweeps=4, seed=seed)
    res, _ = _replay_batch(probs, runs, **kw)
    print("36-site replay:", res)
    for r in res:
        assert r["order"] >= 400, r
        assert r["errN"] < TOL_N and r["errG"] < TOL_G_36, r
    res, _ = _replay_batch(probs, runs, recompute_at_measure=True, **kw)
    print("36-site replay, N recomputed at every measurement:", res)
    for r in res:
        assert r["errG"] < TOL_G_FRESH, r
