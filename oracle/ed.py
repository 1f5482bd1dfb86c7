"""Exact diagonalisation of small Hubbard clusters (test infrastructure only).

This is the brute-force counterpart of the ED cluster solver the DCA++ paper
lists for validating QMC on small clusters (Sec. 3.1, "Cluster solver").
Everything is built in the full Fock space of 2 Nc spin-orbitals (Nc <= 4,
i.e. at most 256 states) with dense matrices:

    H = sum_{ij sigma} t_ij c+_{i sigma} c_{j sigma} - mu sum n + U sum_i n_{i up} n_{i dn}

(Eq. Hubbard plus a chemical potential; with H0 + H_int of
Eq. generalized_hubbard the +-U/2 shifts cancel).  The isolated-cluster
hopping is the Fourier transform of the cluster dispersion,
t_ij = (1/Nc) sum_K eps_K e^{i K (r_i - r_j)}, so that ED and the walker's
G0 describe the same Hamiltonian (for the periodic 2x2 cluster this doubles
the nearest-neighbour bond).

Mode index m = sigma * Nc + r (sigma = 0 up, 1 down); fermion signs follow
the Jordan-Wigner order of the mode index.
"""
import numpy as np


def annihilators(n_modes):
    dim = 1 << n_modes
    ops = []
    states = np.arange(dim)
    for m in range(n_modes):
        c = np.zeros((dim, dim))
        occ = (states >> m) & 1
        below = np.array([bin(s & ((1 << m) - 1)).count("1") for s in states])
        src = states[occ == 1]
        dst = src ^ (1 << m)
        c[dst, src] = (-1.0) ** below[occ == 1]
        ops.append(c)
    return ops


def hopping_from_dispersion(eps_K, k_dot_r_sites, site_sub):
    """t_ij = (1/Nc) sum_K eps_K cos(K . (r_i - r_j)) using the difference table."""
    eps_K = np.asarray(eps_K, np.float64)
    nc = eps_K.size
    t_dr = (np.cos(k_dot_r_sites).T @ eps_K) / nc       # [nc_r]
    return t_dr[np.asarray(site_sub)]


class HubbardED:
    def __init__(self, t_ij, U, mu):
        self.t = np.asarray(t_ij, np.float64)
        self.nc = self.t.shape[0]
        self.U = float(U)
        self.mu = float(mu)
        M = 2 * self.nc
        self.c = annihilators(M)
        dim = 1 << M
        self.n_op = [ci.T @ ci for ci in self.c]
        H0 = np.zeros((dim, dim))
        for s in range(2):
            for i in range(self.nc):
                for j in range(self.nc):
                    if self.t[i, j] != 0.0:
                        H0 += self.t[i, j] * self.c[s * self.nc + i].T @ self.c[s * self.nc + j]
        self.hop = H0
        self.ntot = sum(self.n_op)
        self.docc = sum(self.n_op[i] @ self.n_op[self.nc + i] for i in range(self.nc))
        self.H = H0 - self.mu * self.ntot + self.U * self.docc

    def thermal(self, beta, H=None):
        H = self.H if H is None else H
        E, V = np.linalg.eigh(H)
        E0 = E.min()
        w = np.exp(-beta * (E - E0))
        return E - E0, V, w / w.sum()

    def expect(self, op, beta):
        E, V, p = self.thermal(beta)
        d = np.einsum("im,ij,jm->m", V, op, V)
        return float(p @ d)

    def density(self, beta):
        """Density per site (both spins)."""
        return self.expect(self.ntot, beta) / self.nc

    def double_occupancy(self, beta):
        return self.expect(self.docc, beta) / self.nc

    def h_int(self, beta):
        """<H_int> with H_int = U sum_i [n_up n_dn - (n_up + n_dn)/2] (Eq. generalized_hubbard)."""
        return self.U * self.expect(self.docc - 0.5 * self.ntot, beta)

    def greens(self, beta, taus, H=None, spin=0):
        """G(x, y; tau) = -<T c_x(tau) c+_y(0)> for 0 < tau < beta, shape [nc, nc, len(taus)]."""
        E, V, _ = self.thermal(beta, H)
        Z = np.sum(np.exp(-beta * E))
        taus = np.asarray(taus, np.float64)
        ct = [V.T @ self.c[spin * self.nc + x] @ V for x in range(self.nc)]
        out = np.zeros((self.nc, self.nc, taus.size))
        for a, tau in enumerate(taus):
            em = np.exp(-(beta - tau) * E)     # weight of the left state m
            en = np.exp(-tau * E)              # weight of the right state n
            W = np.outer(em, en)               # W[m, n]
            for x in range(self.nc):
                A = ct[x] * W                  # A[m, n] (c_x)_{mn} w_mn
                for y in range(self.nc):
                    # Tr[e^{-(beta-tau)H} c_x e^{-tau H} c+_y] = sum_mn w_mn (c_x)_mn (c_y)_mn
                    out[x, y, a] = -np.sum(A * ct[y]) / Z
        return out

    def greens_translation_avg(self, beta, taus, site_sub, H=None, spin=0):
        """(1/Nc) sum_y G(y + dr, y; tau) indexed by the difference dr."""
        G = self.greens(beta, taus, H=H, spin=spin)
        nc = self.nc
        site_sub = np.asarray(site_sub)
        out = np.zeros((nc, G.shape[2]))
        for x in range(nc):
            for y in range(nc):
                out[site_sub[x, y]] += G[x, y]
        return out / nc

    def greens_freq(self, beta, n_omega, H=None, spin=0):
        """G(x, y; i w_n) = int_0^beta d tau e^{i w_n tau} G(x, y; tau) for the first n_omega
        positive fermionic frequencies w_n = (2n + 1) pi / beta, from the Lehmann sum
        (1/Z) sum_mn (c_x)_mn (c_y)_mn (e^{-beta E_n} + e^{-beta E_m}) / (i w_n + E_m - E_n),
        shape [nc, nc, n_omega] (complex)."""
        E, V, _ = self.thermal(beta, H)
        Z = np.sum(np.exp(-beta * E))
        w = (2 * np.arange(n_omega) + 1) * np.pi / beta
        ct = [V.T @ self.c[spin * self.nc + x] @ V for x in range(self.nc)]
        bw = np.exp(-beta * E)
        num = bw[None, :] + bw[:, None]           # [m, n]
        dE = E[:, None] - E[None, :]              # E_m - E_n
        out = np.zeros((self.nc, self.nc, n_omega), np.complex128)
        for k, wk in enumerate(w):
            D = num / (1j * wk + dE)
            for x in range(self.nc):
                A = ct[x] * D
                for y in range(self.nc):
                    out[x, y, k] = np.sum(A * ct[y]) / Z
        return out

    def greens_freq_K(self, beta, n_omega, site_sub, k_dot_r, H=None, spin=0):
        """G(K, i w_n) = sum_dr e^{-i K.dr} (1/Nc) sum_y G(y + dr, y; i w_n), [nc_K, n_omega]."""
        G = self.greens_freq(beta, n_omega, H=H, spin=spin)
        nc = self.nc
        site_sub = np.asarray(site_sub)
        Gdr = np.zeros((nc, n_omega), np.complex128)
        for x in range(nc):
            for y in range(nc):
                Gdr[site_sub[x, y]] += G[x, y]
        Gdr /= nc
        return np.exp(-1j * np.asarray(k_dot_r)) @ Gdr

    def h0_shifted(self):
        """CT-AUX H0 = hopping - (mu - U/2) n (Eq. generalized_hubbard, single band)."""
        return self.hop - (self.mu - 0.5 * self.U) * self.ntot

    def aux_weight(self, beta, gamma, verts):
        """<T prod_i exp(gamma s_i (n_{r_i up} - n_{r_i dn}))(tau_i)>_0 under H0 (shifted).

        verts: list of (site, tau, s).  Brute-force time-ordered trace."""
        H0 = self.h0_shifted()
        E, V = np.linalg.eigh(H0)
        E = E - E.min()
        def prop(dt):
            return (V * np.exp(-dt * E)) @ V.T
        order = sorted(verts, key=lambda v: v[1])
        nup = [np.diag(self.n_op[i]) for i in range(self.nc)]
        ndn = [np.diag(self.n_op[self.nc + i]) for i in range(self.nc)]
        dim = H0.shape[0]
        M = np.eye(dim)
        t_prev = 0.0
        for (r, tau, s) in order:
            M = prop(tau - t_prev) @ M
            M = np.diag(np.exp(gamma * s * (nup[r] - ndn[r]))) @ M
            t_prev = tau
        M = prop(beta - t_prev) @ M
        Z0 = np.sum(np.exp(-beta * E))
        return float(np.trace(M) / Z0)


def bisect_mu(t_ij, U, beta, target_density, lo=-10.0, hi=10.0, tol=1e-12):
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        n = HubbardED(t_ij, U, mid).density(beta)
        if n < target_density:
            lo = mid
        else:
            hi = mid
        if hi - lo < tol:
            break
    return 0.5 * (lo + hi)


def atom_greens(U, beta, taus):
    """Closed form for the Hubbard atom at mu = U/2 (standard convention):
    G(tau) = -[e^{-tau U/2} + e^{-(beta - tau) U/2}] / (2 (1 + e^{-beta U/2}))."""
    taus = np.asarray(taus, np.float64)
    return -(np.exp(-taus * U / 2) + np.exp(-(beta - taus) * U / 2)) / (2.0 * (1.0 + np.exp(-beta * U / 2)))
