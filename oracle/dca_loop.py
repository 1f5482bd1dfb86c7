"""Outer DCA self-consistency loop in plain numpy (TEST INFRASTRUCTURE ONLY).

Only tests/ may import this module; the product path never does.  It follows
the DCA paper's Sec. 2.1 step by step, in its notation, for the single-band
Hubbard model on the square lattice with a paramagnetic (spin-independent)
self-energy:

  Eq. sigma_dca          Sigma_DCA(k = K + k~, i w_n) = Sigma_c(K, i w_n)  (piecewise constant);
  Eq. G_coarsegrained    Gbar(K, i w_n) = (Nc / V_BZ) int_patch(K) dk [G0(k)^-1 - Sigma_DCA(k)]^-1,
                         G0(k, i w_n)^-1 = i w_n - eps_k + mu;
  Eq. cluster-exclusion  calG0(K, i w_n) = [Gbar^-1 + Sigma_c]^-1;
  Eq. dyson_sigma        Sigma(K, i w_n) = calG0^-1 - <G>^-1, with the measured
                         <G> = calG0 - calG0^2 <M(K, i w_n)> (Sec. 2.3, G linear in M);
  Eq. self-energy-mixing Sigma^(n) = alpha Sigma_QMC + (1 - alpha) Sigma^(n-1).

Readings where the paper is silent (the GPU library takes the same ones):
  - the patch of K is the cell of the reciprocal superlattice centred on K
    (for the square superlattices used here this is the Wigner-Seitz patch),
    integrated by the midpoint rule on n_fine x n_fine points;
  - the CT-AUX walker takes the bare propagator of H0 with the +U/2 shift of
    Eq. generalized_hubbard: calG0'^-1 = calG0^-1 - U/2;
  - the walker's table G0(r, tau_l), tau_l = l beta / n_tau (l = 0 read as 0+,
    l = n_tau as beta-), is G0(r, tau) = (1/Nc) sum_K cos(K.r) G0(K, tau) (the
    lattices here are inversion symmetric), G0(K, tau) = (1/beta) sum_n
    e^{-i w_n tau} G0(K, i w_n) with the tail 1/(i w_n - xi_K) summed in
    closed form, -e^{-tau xi} / (1 + e^{-beta xi}), and the remainder over
    |n| < n_omega; xi_K = (patch mean of eps) - mu + U/2 matches the first two
    high-frequency moments, so the remainder falls off as 1/w_n^3.
"""
import numpy as np


def matsubara(beta, n_omega):
    """Positive fermionic frequencies w_n = (2n + 1) pi / beta, n < n_omega."""
    return (2 * np.arange(n_omega) + 1) * np.pi / beta


def reciprocal_superlattice(cluster):
    """Rows b1, b2 with a_i . b_j = 2 pi delta_ij for the superlattice rows a_i."""
    A = np.array(cluster.vecs, dtype=np.float64)
    return 2.0 * np.pi * np.linalg.inv(A).T


def patch_offsets(cluster, n_fine):
    """Midpoints k~ of the n_fine x n_fine sub-cells of the patch centred on 0."""
    B = reciprocal_superlattice(cluster)
    u = (np.arange(n_fine) + 0.5) / n_fine - 0.5
    m1, m2 = np.meshgrid(u, u, indexing="ij")
    return m1.reshape(-1, 1) * B[0] + m2.reshape(-1, 1) * B[1]


def dispersion(k, t, tp):
    """eps_k = -2t (cos kx + cos ky) - 4t' cos kx cos ky."""
    cx, cy = np.cos(k[..., 0]), np.cos(k[..., 1])
    return -2.0 * t * (cx + cy) - 4.0 * tp * cx * cy


def coarse_grain(cluster, t, tp, mu, beta, sigma, n_fine):
    """Eqs. sigma_dca and G_coarsegrained: Gbar(K, i w_n) [nc, n_omega] for the
    cluster self-energy sigma [nc, n_omega]."""
    sigma = np.asarray(sigma, np.complex128)
    wn = matsubara(beta, sigma.shape[1])
    kt = patch_offsets(cluster, n_fine)
    Gbar = np.zeros_like(sigma)
    for K in range(cluster.nc):
        eps = dispersion(cluster.kpts[K][None, :] + kt, t, tp)          # [points]
        for n in range(wn.size):
            Gbar[K, n] = np.mean(1.0 / (1j * wn[n] + mu - eps - sigma[K, n]))
    return Gbar


def patch_mean_dispersion(cluster, t, tp, n_fine):
    kt = patch_offsets(cluster, n_fine)
    return np.array([np.mean(dispersion(cluster.kpts[K][None, :] + kt, t, tp)) for K in range(cluster.nc)])


def cluster_exclusion(Gbar, sigma):
    """Eq. cluster-exclusion: calG0 = [Gbar^-1 + Sigma]^-1."""
    return 1.0 / (1.0 / np.asarray(Gbar) + np.asarray(sigma))


def measured_G(G0w, MK):
    """<G> = calG0 - calG0^2 <M> (paper sign convention)."""
    return G0w - G0w * G0w * MK


def dyson_sigma(G0w, G):
    """Eq. dyson_sigma: Sigma = calG0^-1 - G^-1."""
    return 1.0 / np.asarray(G0w) - 1.0 / np.asarray(G)


def mix(sigma_qmc, sigma_old, alpha):
    """Eq. self-energy-mixing."""
    return alpha * np.asarray(sigma_qmc) + (1.0 - alpha) * np.asarray(sigma_old)


def M_of_K(M_dr, k_dot_r):
    """M(K) = sum_dr e^{-i K.dr} M(dr) for M_dr [..., nc_dr, n_omega]."""
    return np.einsum("kd,...dn->...kn", np.exp(-1j * np.asarray(k_dot_r)), M_dr)


def hartree_shift(G0w, U):
    """The CT-AUX bare propagator: calG0'^-1 = calG0^-1 - U/2."""
    return 1.0 / (1.0 / np.asarray(G0w) - 0.5 * U)


def tail_tau(xi, beta, tau):
    """(1/beta) sum_n e^{-i w_n tau} / (i w_n - xi) = -e^{-tau xi} / (1 + e^{-beta xi}), 0 < tau < beta."""
    xi = np.asarray(xi, np.float64)[:, None]
    tau = np.asarray(tau, np.float64)[None, :]
    return np.where(xi >= 0, -np.exp(-tau * xi) / (1.0 + np.exp(-beta * xi)),
                    -np.exp((beta - tau) * xi) / (np.exp(beta * xi) + 1.0))


def g0_table(G0w_shifted, xi, k_dot_r, beta, n_tau):
    """The walker's table [2][nc][n_tau + 1] (paper sign, both spins equal) from
    calG0'(K, i w_n) [nc, n_omega] and the tail parameter xi [nc]."""
    G0w = np.asarray(G0w_shifted, np.complex128)
    nc, nw = G0w.shape
    wn = matsubara(beta, nw)
    tau = np.arange(n_tau + 1) * beta / n_tau
    tau[0] = 0.0
    R = G0w - 1.0 / (1j * wn[None, :] - np.asarray(xi)[:, None])      # remainder
    GK = np.zeros((nc, n_tau + 1))
    for l in range(n_tau + 1):
        # G(K, tau) = tail + (2/beta) sum_{n >= 0} Re[e^{-i w_n tau} R(K, i w_n)]
        GK[:, l] = (2.0 / beta) * np.real(np.exp(-1j * wn * tau[l])[None, :] * R).sum(axis=1)
    t = tau.copy()
    t[0] = 0.0
    T = tail_tau(xi, beta, t)
    T[:, -1] = tail_tau(xi, beta, np.array([beta]))[:, 0]  # beta- (the closed form is continuous there)
    GK += T
    Gr = np.cos(np.asarray(k_dot_r)).T @ GK / nc                       # [nc_r, n_tau + 1]
    return np.stack([Gr, Gr])
