"""Pins of the oracle's two-particle measurement (particle-particle up-down
channel, Sec. 2.5 Eq. bse_cluster; App. B four-point group), independent of
the GPU.

- U = 0: M = 0, so the accumulators vanish exactly and the assembled G2 is
  G0_up(K) G0_dn(q - K) delta_{K K'}, the paper's non-interacting G2^{0,pp}.
- The diagonal M_sigma(k, k) is the single-particle M(K, i w_n) of the
  frequency measurement (itself pinned to the atom's closed form and to ED),
  at positive and negative frequencies and at the shifted spin-down points.
- Per configuration, the two-point function G(k1, k2) built from M_sigma(k1,
  k2) equals the double Fourier transform of the time-domain Green's function
  of that configuration, G(x, y) = G0(x - y) - sum_ij G0(x - x_i) c_ij G0(x_j - y)
  (the form the tau-grid estimator uses, pinned by ED), evaluated by
  Gauss-Legendre quadrature with the closed-form free propagator: this fixes
  the signs of the phases, which index carries which frequency, the momentum
  convention and the 1/(beta Nc) normalisation.
- After one measurement the accumulators are sign * M_up o M_dn and sign *
  diag M_sigma, and the assembled G2 equals the product of the two
  per-configuration two-point functions.
"""
import numpy as np
import pytest

from oracle import ctaux
from oracle import g4 as og4
from tests.helpers import problem


def _walker(nc, U, beta, mu, n_w4, m4, q_idx, seed, nw=0, sweeps=0, warmup=5):
    c, eps, kr, G0 = problem(nc, 1.0, 0.0, U, beta, mu, 512)
    w = ctaux.OracleWalker(nc, c.site_sub, U, beta, 1.0, G0, warmup_sweeps=warmup, n_tau_meas=4, seed=seed)
    k_dn = c.k_sub[q_idx]  # index of Q - K
    w.enable_g4(n_w4, m4, kr, k_dn)
    if nw:
        w.enable_freq(nw)
    if sweeps:
        w.sweep(sweeps)
    return w, c, eps, kr, k_dn


def _g0_freq(eps, mu_eff, beta, K, n):
    """Closed-form free propagator 1/(i w_n - xi_K), paper sign."""
    wn = (2 * np.asarray(n) + 1) * np.pi / beta
    return 1.0 / (1j * wn - (eps[K] - mu_eff))


def test_u0_two_particle_function_is_the_bubble():
    nc, beta, mu, n_w4, m4, q = 4, 3.0, 0.4, 3, 1, 2
    w, c, eps, kr, k_dn = _walker(nc, 0.0, beta, mu, n_w4, m4, q, seed=1, sweeps=40)
    A, D = w.g4()
    assert np.all(A == 0) and np.all(D == 0)
    g, ss, nm = w.G()
    Ku, nu, Kd, nd = og4.points(nc, n_w4, m4, k_dn)
    G0u, G0d = _g0_freq(eps, mu, beta, Ku, nu), _g0_freq(eps, mu, beta, Kd, nd)
    G2 = og4.assemble(A, D, ss, G0u, G0d)
    assert np.allclose(G2, np.diag(G0u * G0d), rtol=1e-15, atol=0)
    # q - K for the points: momentum Q - K and frequency nu_m - w_n
    Q = c.kpts[q]
    dk = Q - c.kpts[Ku] - c.kpts[Kd]
    assert np.abs(np.exp(1j * dk) - 1).max() < 1e-12
    assert np.array_equal(nd + nu + 1, np.full_like(nu, m4))


@pytest.mark.parametrize("m4,q", [(0, 0), (2, 3)])
def test_diagonal_is_the_single_particle_measurement(m4, q):
    nc, U, beta, mu, n_w4 = 4, 4.0, 3.0, 1.1, 3
    nw = n_w4 + abs(m4) + 1
    w, c, eps, kr, k_dn = _walker(nc, U, beta, mu, n_w4, m4, q, seed=2, nw=nw, sweeps=60)
    A, D = w.g4()
    M = w.M()  # [2, nc(dr), nw]
    MK = np.einsum("kd,sdn->skn", np.exp(-1j * kr), M)  # M(K, i w_n), n >= 0
    Ku, nu, Kd, nd = og4.points(nc, n_w4, m4, k_dn)
    minus = c.k_sub[0]  # index of -K

    def single(sp, K, n):
        return MK[sp, K, n] if n >= 0 else np.conj(MK[sp, minus[K], -n - 1])

    ref_u = np.array([single(0, K, n) for K, n in zip(Ku, nu)])
    ref_d = np.array([single(1, K, n) for K, n in zip(Kd, nd)])
    scale = np.abs(ref_u).max()
    assert scale > 0
    assert np.abs(D[0] - ref_u).max() < 1e-12 * scale
    assert np.abs(D[1] - ref_d).max() < 1e-12 * np.abs(ref_d).max()


def _gl(a, b, n=64):
    x, wts = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * wts


def _g0_time(eps, mu_eff, beta, kr, r_index, tau):
    """Closed-form G0(r, tau) for tau in (-beta, beta) (paper sign), r a site index:
    (1/Nc) sum_K e^{i K.r} G0(K, tau), G0(K, tau) = -e^{-tau xi} / (1 + e^{-beta xi})."""
    tau = np.asarray(tau, np.float64)
    sgn = np.where(tau < 0, -1.0, 1.0)
    t = np.where(tau < 0, tau + beta, tau)
    xi = eps - mu_eff
    gK = -np.exp(-np.outer(t, xi)) / (1 + np.exp(-beta * xi))[None, :]  # [T, K]
    ph = np.exp(1j * kr[:, r_index])  # [K]
    return sgn * (gK @ ph).real / len(eps)


@pytest.mark.parametrize("sp", [0, 1])
def test_per_configuration_two_point_function_is_the_fourier_transform(sp):
    nc, U, beta, mu, n_w4, m4, q = 4, 4.0, 3.0, 1.1, 2, 1, 1
    w, c, eps, kr, k_dn = _walker(nc, U, beta, mu, n_w4, m4, q, seed=3, sweeps=30)
    st = w.state()
    k = st["site"].size
    assert k >= 3
    Msp = w.m2(sp)
    mu_eff = mu - U / 2
    sigma = 1 - 2 * sp
    cfac = (np.exp(sigma * w.gamma * st["s"].astype(np.float64)) - 1.0)[:, None] * st["N"][sp]
    Ku, nu, Kd, nd = og4.points(nc, n_w4, m4, k_dn)
    Kp, npnt = (Ku, nu) if sp == 0 else (Kd, nd)
    G0k = _g0_freq(eps, mu_eff, beta, Kp, npnt)
    S = Kp.size

    def transform(i, s, sgn):
        """int_0^beta dtau sum_r e^{sgn i (w tau - K.r)} G0(+-(r - r_i), +-(tau - tau_i)), split at tau_i:
        sgn = +1: G0(x - x_i) (left factor); sgn = -1: G0(x_i - x) (right factor)."""
        wn = (2 * npnt[s] + 1) * np.pi / beta
        tot = 0.0
        for a, b in ((0.0, st["tau"][i]), (st["tau"][i], beta)):
            tt, ww = _gl(a, b)
            for r in range(nc):
                if sgn > 0:
                    g = _g0_time(eps, mu_eff, beta, kr, c.site_sub[r, st["site"][i]], tt - st["tau"][i])
                else:
                    g = _g0_time(eps, mu_eff, beta, kr, c.site_sub[st["site"][i], r], st["tau"][i] - tt)
                tot = tot + np.sum(ww * g * np.exp(sgn * 1j * (wn * tt - kr[Kp[s], r])))
        return tot

    I = np.array([[transform(i, s, +1) for s in range(S)] for i in range(k)])  # [k, S]
    J = np.array([[transform(j, s, -1) for s in range(S)] for j in range(k)])  # [k, S]
    lhs = (I.T @ cfac @ J) / (beta * nc)  # the correction term of G(k1, k2), time-domain route
    rhs = G0k[:, None] * Msp * G0k[None, :]
    assert np.abs(rhs).max() > 1e-3
    assert np.abs(lhs - rhs).max() < 1e-11 * np.abs(rhs).max(), np.abs(lhs - rhs).max()
    # the factors themselves: int e^{i w tau - iK.r} G0(x - x_i) = e^{i (w tau_i - K.r_i)} G0(k)
    ph = np.exp(1j * (np.outer(st["tau"], (2 * npnt + 1) * np.pi / beta) - kr[Kp][:, st["site"]].T))
    assert np.abs(I - ph * G0k[None, :]).max() < 1e-12


def test_one_measurement_assembles_to_the_product_of_two_point_functions():
    nc, U, beta, mu, n_w4, m4, q = 4, 4.0, 3.0, 1.1, 2, 1, 3
    w, c, eps, kr, k_dn = _walker(nc, U, beta, mu, n_w4, m4, q, seed=4, sweeps=20)
    w.reset_accumulators()
    w.sweep(1)  # exactly one measurement, of the configuration the walker now holds
    A, D = w.g4()
    g, ss, nm = w.G()
    assert nm == 1 and abs(ss) == 1.0
    Mu, Md = w.m2(0), w.m2(1)
    assert np.abs(A - ss * Mu * Md).max() < 1e-14 * np.abs(A).max()
    assert np.array_equal(D[0], ss * np.diag(Mu)) and np.array_equal(D[1], ss * np.diag(Md))
    Ku, nu, Kd, nd = og4.points(nc, n_w4, m4, k_dn)
    mu_eff = mu - U / 2
    G0u, G0d = _g0_freq(eps, mu_eff, beta, Ku, nu), _g0_freq(eps, mu_eff, beta, Kd, nd)
    S = Ku.size
    Gu = np.diag(G0u) - G0u[:, None] * Mu * G0u[None, :]
    Gd = np.diag(G0d) - G0d[:, None] * Md * G0d[None, :]
    G2 = og4.assemble(A, D, ss, G0u, G0d)
    assert np.abs(G2 - Gu * Gd).max() < 1e-13 * np.abs(Gu * Gd).max()
    assert S == nc * 2 * n_w4
