"""Bare propagator of an isolated cluster, tabulated on a tau grid (test infrastructure only).

The walker's input G0 is the bare cluster Green's function of the CT-AUX H0
of Eq. generalized_hubbard, which carries the shift + U/2 (n_up + n_dn), i.e.
an effective chemical potential mu - U/2.  For an isolated cluster (no DCA
bath) with dispersion eps_K at the Nc cluster momenta,

    G0(r, tau) = -(1/Nc) sum_K e^{i K.r} e^{-tau xi_K} / (1 + e^{-beta xi_K}),
    xi_K = eps_K - (mu - U/2),   0 < tau < beta,

in the paper's sign convention (negative on (0, beta)); sample l = 0 holds
G0(r, 0+) and sample l = n_tau holds G0(r, beta-).
"""
import numpy as np


def _fermi_weight(tau, xi, beta):
    """e^{-tau xi} / (1 + e^{-beta xi}) evaluated without overflow."""
    tau = np.asarray(tau, dtype=np.float64)[:, None]
    xi = np.asarray(xi, dtype=np.float64)[None, :]
    pos = xi >= 0
    out = np.empty(np.broadcast(tau, xi).shape)
    a = np.exp(-tau * np.where(pos, xi, 0.0)) / (1.0 + np.exp(-beta * np.where(pos, xi, 0.0)))
    b = np.exp((beta - tau) * np.where(pos, 0.0, xi)) / (np.exp(beta * np.where(pos, 0.0, xi)) + 1.0)
    out = np.where(pos, a, b)
    return out


def g0_table(eps_K, k_dot_r, mu, U, beta, n_tau):
    """Return G0[2][nc][n_tau+1] (paper convention) on tau_l = l beta / n_tau.

    eps_K: [nc] dispersion at the cluster momenta; k_dot_r: [nc_K, nc_r] K.r.
    """
    eps_K = np.asarray(eps_K, dtype=np.float64)
    nc = eps_K.size
    xi = eps_K - (mu - 0.5 * U)
    taus = np.arange(n_tau + 1, dtype=np.float64) * (beta / n_tau)
    w = _fermi_weight(taus, xi, beta)                       # [n_tau+1, nc_K]
    phase = np.cos(np.asarray(k_dot_r, dtype=np.float64))   # [nc_K, nc_r]; the cluster is inversion symmetric
    g = (w @ phase) / nc                                    # [n_tau+1, nc_r]
    G0 = -g.T                                               # [nc_r, n_tau+1]
    return np.ascontiguousarray(np.stack([G0, G0]))


def free_density(eps_K, mu, U, beta):
    """Density per site (both spins) of the CT-AUX H0 (effective mu - U/2)."""
    xi = np.asarray(eps_K, dtype=np.float64) - (mu - 0.5 * U)
    return 2.0 * np.mean(1.0 / (np.exp(np.clip(beta * xi, -700, 700)) + 1.0))
