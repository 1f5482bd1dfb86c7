"""Pins of the oracle's outer DCA loop (Sec. 2.1), independent of the GPU.

- With Sigma = 0 and one point per patch the coarse-grained Gbar(K) is the free
  lattice propagator at K, 1/(i w_n + mu - eps_K), and the walker table built
  from it (Hartree shift, tail in closed form, Matsubara remainder) equals the
  isolated-cluster table of the oracle's analytic builder.
- With Sigma = 0 and many points per patch the table equals the patch average
  of the closed-form free propagators, up to the Matsubara truncation.
- The patches tile the Brillouin zone: the K-average of Gbar is the local
  lattice propagator summed directly over the same k mesh.
- Dyson round trip: a self-energy turned into the measured <G> (and <M>) and
  back by Eq. dyson_sigma is the same self-energy; mixing interpolates.
"""
import numpy as np

from oracle import dca_loop as dl
from oracle import g0 as og0
from paper_1901_01047_gb300 import inputs


def _setup(nc=4, t=1.0, tp=0.0):
    c = inputs.cluster(nc)
    return c, inputs.square_dispersion(c.kpts, t, tp), inputs.k_dot_r(c)


def test_one_point_patches_give_the_isolated_cluster_table():
    for nc, tp in ((4, 0.0), (16, -0.15), (8, 0.0)):
        c, eps, kr = _setup(nc, 1.0, tp)
        U, beta, mu, nw, n_tau = 5.0, 6.0, 2.1, 64, 512
        wn = dl.matsubara(beta, nw)
        Gbar = dl.coarse_grain(c, 1.0, tp, mu, beta, np.zeros((nc, nw)), n_fine=1)
        assert np.abs(Gbar - 1.0 / (1j * wn[None, :] + mu - eps[:, None])).max() < 1e-14
        G0w = dl.hartree_shift(dl.cluster_exclusion(Gbar, 0.0), U)
        xi = dl.patch_mean_dispersion(c, 1.0, tp, 1) - mu + U / 2
        table = dl.g0_table(G0w, xi, kr, beta, n_tau)
        ref = og0.g0_table(eps, kr, mu, U, beta, n_tau)
        assert np.abs(table - ref).max() < 1e-12


def test_patch_average_of_free_propagators():
    # U = 0 (no Hartree shift): calG0 = Gbar is the patch average of free
    # propagators, whose imaginary-time forms are known in closed form
    c, eps, kr = _setup(4)
    U, beta, mu, nw, n_tau, nf = 0.0, 4.0, 1.3, 2048, 64, 6
    Gbar = dl.coarse_grain(c, 1.0, 0.0, mu, beta, np.zeros((4, nw)), n_fine=nf)
    xi = dl.patch_mean_dispersion(c, 1.0, 0.0, nf) - mu + U / 2
    table = dl.g0_table(dl.hartree_shift(Gbar, U), xi, kr, beta, n_tau)
    tau = np.arange(n_tau + 1) * beta / n_tau
    kt = dl.patch_offsets(c, nf)
    ref = np.zeros((4, n_tau + 1))
    for K in range(4):
        xik = dl.dispersion(c.kpts[K][None, :] + kt, 1.0, 0.0) - mu + U / 2
        GK = dl.tail_tau(xik, beta, tau).mean(axis=0)
        ref += np.cos(kr[K])[:, None] * GK[None, :] / 4
    assert np.abs(table[0] - ref).max() < 2e-6
    assert np.abs(table[0] - og0.g0_table(eps, kr, mu, U, beta, n_tau)[0]).max() > 1e-3  # not the cluster G0


def test_patches_tile_the_brillouin_zone():
    for nc in (4, 8, 16):
        c, eps, kr = _setup(nc)
        beta, mu, nw, nf = 5.0, 0.3, 4, 4
        Gbar = dl.coarse_grain(c, 1.0, 0.0, mu, beta, np.zeros((nc, nw)), n_fine=nf)
        ks = (c.kpts[:, None, :] + dl.patch_offsets(c, nf)[None, :, :]).reshape(-1, 2)
        # the same points folded into [0, 2 pi)^2 are distinct lattice momenta
        folded = np.round(np.mod(ks, 2 * np.pi) * 1e9).astype(np.int64)
        assert len({tuple(p) for p in folded}) == ks.shape[0]
        wn = dl.matsubara(beta, nw)
        loc = np.mean(1.0 / (1j * wn[None, :] + mu - dl.dispersion(ks, 1.0, 0.0)[:, None]), axis=0)
        assert np.abs(Gbar.mean(axis=0) - loc).max() < 1e-14
        # the patch area is the Brillouin zone over Nc
        B = dl.reciprocal_superlattice(c)
        assert abs(abs(np.linalg.det(B)) * nc - (2 * np.pi) ** 2) < 1e-9


def test_dyson_round_trip_and_mixing():
    c, eps, kr = _setup(4)
    beta, mu, nw = 5.0, 0.8, 32
    wn = dl.matsubara(beta, nw)
    rng = np.random.default_rng(0)
    sig = (rng.normal(size=(4, 1)) - 1j * 2.0 / (wn[None, :] + 1.0)) * 0.7
    G0w = dl.cluster_exclusion(dl.coarse_grain(c, 1.0, 0.0, mu, beta, sig, 4), sig)
    G = 1.0 / (1.0 / G0w - sig)
    M = (G0w - G) / (G0w * G0w)
    assert np.abs(dl.dyson_sigma(G0w, dl.measured_G(G0w, M)) - sig).max() < 1e-12
    assert np.abs(dl.mix(sig, 0 * sig, 1.0) - sig).max() == 0
    assert np.abs(dl.mix(sig, 2 * sig, 0.25) - 1.75 * sig).max() < 1e-15
