"""Mixed precision (N stored in FP32, products in FP32; ratios, B^-1, the
update factors and the recompute in FP64) against the FP64 oracle.

Trajectories of two arithmetics part ways at the first flipped decision, so
the error is measured on an identical trajectory: the GPU walker replays the
oracle's decision log (forced decisions), and N and the accumulated sign * G
are compared at the end in the norm form max|X_gpu - X_ora| / max|X_ora|.
Without forcing, the free-running mixed walker must still agree with the
oracle's decisions for a long stretch.
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


def replay(nc, tp, U, beta, mu, k_sub, sweeps, R, seed=0, ntm=32, n_tau=4096, update_kernel="auto",
           return_state=False, recompute_method="auto", recompute_at_measure=False, precision="mixed", update_tile=0):
    c, eps, kr, G0 = problem(nc, 1.0, tp, U, beta, mu, n_tau)
    ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=10, n_tau_meas=ntm, seed=seed)
    ow.enable_log(1 << 24)
    ow.sweep(sweeps)
    log = ow.log()
    gw = _walkers(problems=[dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)], k_sub=k_sub,
                  recompute_every=R, warmup_sweeps=10, n_tau_meas=ntm, seed=seed, precision=precision,
                  log_capacity=1 << 24, update_kernel=update_kernel, recompute_method=recompute_method,
                  recompute_at_measure=recompute_at_measure)
    if update_tile:
        gw.set_update_tile(update_tile)
    gw.set_forced_decisions(0, log)
    gw.sweep(sweeps)
    gs, os_ = gw.state(0), ow.state()
    assert np.array_equal(gs["site"], os_["site"]) and np.array_equal(gs["s"], os_["s"])
    errN = max(np.abs(gs["N"][sp] - os_["N"][sp]).max() / np.abs(os_["N"][sp]).max() for sp in range(2))
    Gg, ssg, nmg = gw.measure_G()
    Go, sso, nmo = ow.G()
    assert nmg[0] == nmo and ssg[0] == sso
    errG = np.abs(Gg[0] - Go).max() / np.abs(Go).max()
    st = gw.stats()[0]
    gw.close()
    if return_state:
        return errN, errG, st, gs
    return errN, errG, st, log


# Bounds from measurement, with head room: the FP32 rounding is amplified by
# the conditioning of N^-1 (about 1e3 for the 2x2 cluster at beta = 10, 2e4
# for the 16-site case) and the result moves by a few times between builds
# that sum in another order.  Recomputing every 8 submatrix updates instead
# of 64 cuts the error several times.  The tensor-core path carries the
# N-sized products (update, both candidate products) in 3xTF32, about 22
# bits per product against 24 for FP32.
UPDATE_KERNELS = ["cuda_core", "tcgen05"]


@pytest.mark.parametrize("kern", UPDATE_KERNELS)
def test_mixed_replay_2x2_errors(kern):
    errN, errG, st, _ = replay(4, 0.0, 4.0, 10.0, 0.9450480104035819, 32, 2000, 64, update_kernel=kern)
    print("2x2 %s R=64: N %.2e G %.2e" % (kern, errN, errG))
    assert st["status"] == 0 and st["recomputes"] > 0
    assert errN < 1e-4, errN
    assert errG < 3e-4, errG
    errN8, errG8, st8, _ = replay(4, 0.0, 4.0, 10.0, 0.9450480104035819, 32, 2000, 8, update_kernel=kern)
    print("2x2 %s R=8: N %.2e G %.2e" % (kern, errN8, errG8))
    assert errG8 < 1e-4, errG8


@pytest.mark.parametrize("kern", UPDATE_KERNELS)
def test_mixed_replay_16_site_errors(kern):
    errN, errG, st, _ = replay(16, -0.15, 6.0, 4.0, 2.85, 64, 60, 64, ntm=16, n_tau=2048, update_kernel=kern)
    print("16 sites %s R=64: N %.2e G %.2e" % (kern, errN, errG))
    assert errN < 3e-4, errN
    assert errG < 5e-5, errG


def test_mixed_free_run_follows_the_oracle_for_a_long_stretch():
    nc, U, beta, mu = 4, 4.0, 10.0, 0.9450480104035819
    c, eps, kr, G0 = problem(nc, 1.0, 0.0, U, beta, mu, 4096)
    gw = _walkers(problems=[dict(nc=nc, site_sub=c.site_sub, U=U, beta=beta, K=1.0, G0=G0)], k_sub=32,
                  recompute_every=64, warmup_sweeps=10, n_tau_meas=8, seed=3, precision="mixed",
                  log_capacity=1 << 22)
    gw.sweep(300)
    glog = gw.decision_log(0)
    ow = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=10, n_tau_meas=8, seed=3)
    ow.enable_log(1 << 22)
    ow.sweep(300)
    olog = ow.log()
    n = min(glog.size, olog.size)
    mism = np.nonzero((glog[:n] & 1) != (olog[:n] & 1))[0]
    first = mism[0] if mism.size else n
    assert first > 2000, first


@pytest.mark.parametrize("k_sub,tile", [(16, 64), (16, 32), (48, 64), (64, 64), (64, 32), (96, 0), (128, 0)])
def test_tensor_core_update_matches_cuda_core_update(k_sub, tile):
    # Same forced trajectory, no recompute: the 3xTF32 tcgen05 update and the
    # FP32 CUDA-core update differ only by rounding.  k_sub covers the three
    # K extents of the tensor-core kernel (32, 64, 128), each also with a
    # window that fills it only in part (48, 96: the autotuner's other
    # sizes), tile both column tiles of N, and n spans several 128-row blocks
    # with a ragged tail.
    args = (16, -0.15, 6.0, 6.0, 2.85, k_sub, 30, 0)
    eN_c, eG_c, st_c, gs_c = replay(*args, ntm=16, n_tau=2048, update_kernel="cuda_core", return_state=True)
    eN_t, eG_t, st_t, gs_t = replay(*args, ntm=16, n_tau=2048, update_kernel="tcgen05", return_state=True,
                                    update_tile=tile)
    assert st_t["status"] == 0 and st_c["status"] == 0
    assert gs_t["N"][0].shape[0] > 128
    # Both drift from the FP64 oracle (no recompute).  3xTF32 keeps about 22
    # bits of every product against 24 for an FP32 FMA, so the tensor-core
    # path may drift several times more than the CUDA-core path, within the
    # mixed path's error budget; the two stay within the sum of their drifts
    # of each other.
    # (the floor is the mixed path's error budget of the 16-site replay test)
    print("k_s %d: tcgen05 N %.2e G %.2e, CUDA core N %.2e G %.2e" % (k_sub, eN_t, eG_t, eN_c, eG_c))
    assert eN_t <= 6 * eN_c + 1e-4 and eG_t <= 6 * eG_c + 2e-5, (eN_t, eN_c, eG_t, eG_c)
    for sp in range(2):
        a, b = gs_c["N"][sp], gs_t["N"][sp]
        assert np.abs(a - b).max() <= 2 * (eN_c + eN_t) * np.abs(a).max() + 1e-12


def test_mixed_batched_sweep_synchronised_recompute():
    # Uneven batch (two cluster sizes, several temperatures) with the batched
    # recompute schedule: every walker recomputes after the first window of
    # every second sweep, and the FP32 drift it removes stays small.
    import torch
    from paper_1901_01047_gb300 import walker
    probs = []
    for nc, beta in [(4, 4.0), (8, 3.0), (4, 8.0), (8, 5.0)]:
        c, eps, kr, G0 = problem(nc, 1.0, 0.0, 5.0, beta, 2.5, 2048)
        probs.append(dict(nc=nc, site_sub=c.site_sub, U=5.0, beta=beta, K=1.0, G0=G0))
    gw = walker.Walkers(probs, n_walkers=16, k_sub=32, recompute_every=0, recompute_sweeps=2, warmup_sweeps=4,
                        n_tau_meas=16, precision="mixed", seed=11, stream=torch.cuda.current_stream().cuda_stream)
    gw.sweep(21)
    for st in gw.stats():
        assert st["status"] == 0
        assert st["recomputes"] == 10, st["recomputes"]
        assert st["max_drift"] < 1e-3, st["max_drift"]
    gw.close()


@pytest.mark.parametrize("method", ["auto", "newton_df", "gj"])
def test_mixed_recompute_methods_restore_accuracy(method):
    # The Newton step (residual from digit planes on the tensor cores, or in
    # double-float on the CUDA cores; FP32 correction) and the Gauss-Jordan
    # inverse all bring N back to the FP32 level: recomputing every 8
    # submatrix updates keeps the error of N and G small on the 16-site case.
    errN, errG, st, _ = replay(16, -0.15, 6.0, 4.0, 2.85, 64, 60, 8, ntm=16, n_tau=2048, recompute_method=method)
    print("16 sites recompute %s every 8: N %.2e G %.2e drift %.2e" % (method, errN, errG, st["max_drift"]))
    assert st["status"] == 0 and st["recomputes"] >= 10
    assert errN < 1e-4, errN
    assert errG < 2e-5, errG
    assert st["max_drift"] < 1e-3


def test_autotuner_selects_a_candidate_and_leaves_walkers_on_it():
    import torch
    from paper_1901_01047_gb300 import autotune, walker
    probs = []
    for nc, beta in [(4, 6.0), (8, 4.0)]:
        c, eps, kr, G0 = problem(nc, 1.0, 0.0, 5.0, beta, 2.5, 1024)
        probs.append(dict(nc=nc, site_sub=c.site_sub, U=5.0, beta=beta, K=1.0, G0=G0))
    gw = walker.Walkers(probs, n_walkers=8, k_sub=32, recompute_every=0, recompute_sweeps=4, warmup_sweeps=2,
                        n_tau_meas=8, precision="mixed", seed=3, stream=torch.cuda.current_stream().cuda_stream)
    gw.sweep(6)
    res = autotune.tune(gw, "mixed", sweeps=1, settle=1)
    assert len(res["table"]) == len(autotune.KS_CANDIDATES) * len(autotune.KERNEL_CANDIDATES)
    assert res["k_sub"] in autotune.KS_CANDIDATES and res["update_kernel"] in autotune.KERNEL_CANDIDATES
    assert res["update_tile"] in autotune.TILE_CANDIDATES
    assert all(r["updates_per_s"] > 0 for r in res["table"])
    assert gw.k_sub == res["k_sub"]
    gw.sweep(2)
    assert all(s["status"] == 0 for s in gw.stats())
    gw.close()


def test_mixed_replay_error_at_the_batched_recompute_interval():
    # The batched bench recomputes every 8 sweeps, about 320 windows for its
    # largest walkers; the 16-site case recomputing every 320 windows states
    # the error reached there.
    errN, errG, st, _ = replay(16, -0.15, 6.0, 4.0, 2.85, 16, 200, 320, ntm=16, n_tau=2048)
    print("16 sites R=320: N %.2e G %.2e" % (errN, errG))
    assert st["status"] == 0 and st["recomputes"] >= 1
    assert errN < 2e-4, errN  # measured 2.5e-5
    assert errG < 3e-5, errG  # measured 4.3e-6


def test_mixed_replay_with_N_recomputed_at_every_measurement_meets_1e6():
    # The error of the mixed path is carried by N between recomputes; with N
    # recomputed before every measurement the accumulated G is within 1e-6 of
    # the FP64 oracle (measured 1.3e-7 on the 2x2 case and 5.6e-8 on 16 sites).
    errN, errG, st, _ = replay(4, 0.0, 4.0, 10.0, 0.9450480104035819, 32, 400, 64, recompute_at_measure=True)
    print("2x2 recompute at every measurement: N %.2e G %.2e" % (errN, errG))
    assert errG < 1e-6, errG
    errN, errG, st, _ = replay(16, -0.15, 6.0, 4.0, 2.85, 64, 60, 64, ntm=16, n_tau=2048, recompute_at_measure=True)
    print("16 sites recompute at every measurement: N %.2e G %.2e" % (errN, errG))
    assert errG < 1e-6, errG
    assert errN < 1e-6, errN  # N was just recomputed: its FP32 rounding


def test_tf32_single_product_replay_error():
    # One TF32 product per K step (about 11 bits): the error the 3xTF32 split
    # removes (measured 2.9e-3 on N and 2.1e-2 on G for this case)
    errN, errG, st, _ = replay(4, 0.0, 4.0, 10.0, 0.9450480104035819, 32, 400, 8, precision="tf32")
    print("2x2 TF32 R=8: N %.2e G %.2e" % (errN, errG))
    assert st["status"] == 0
    assert 1e-4 < errN < 5e-2 and errG < 0.1


@pytest.mark.parametrize("method", ["auto", "newton_df", "gj"])
def test_recompute_methods_bring_N_to_its_fp32_rounding(method):
    # N recomputed in the window that ends the last sweep: the state is the
    # recompute's result, within the FP32 rounding of N times its conditioning
    # for every method (the sliced residual's products are exact up to 2^-40
    # of the row and column maxima).  16 sites at order ~150 (two 128-column
    # and three 64-row tiles of the residual, a ragged K chunk) and the 2x2
    # cluster at beta = 10.
    for args, kw in [((16, -0.15, 6.0, 4.0, 2.85, 64, 60, 64), dict(ntm=16, n_tau=2048)),
                     ((4, 0.0, 4.0, 10.0, 0.9450480104035819, 32, 200, 64), {})]:
        errN, errG, st, gs = replay(*args, recompute_at_measure=True, recompute_method=method, return_state=True, **kw)
        print("recompute %s, order %d: N %.2e G %.2e" % (method, gs["site"].size, errN, errG))
        assert st["status"] == 0 and st["recomputes"] >= 10
        assert errN < 1e-6, errN
        assert errG < 1e-6, errG
