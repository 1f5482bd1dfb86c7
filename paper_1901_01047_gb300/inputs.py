"""Seeded synthetic inputs shared by the GPU path, its tests and the oracle.

This module holds no CT-AUX arithmetic: only the geometry of square-lattice
DCA clusters (sites, the r_i - r_j table, cluster momenta and their
differences), the dispersion of
the single-band Hubbard model on the square lattice (t, t' as in the model
parameters of App. B), and the named workload parameter sets.

Cluster geometry.  A cluster is given by two superlattice vectors a1, a2 in
units of the square-lattice basis (App. B, "cluster").  Its sites are the
lattice points modulo the superlattice, so Nc = |det[a1; a2]|.  Cluster momenta
K satisfy K . a1, K . a2 in 2 pi Z.  The vectors of the 16- and 36-site
clusters are the square ones [[4,0],[0,4]] and [[6,0],[0,6]]; the 8-site
cluster is [[2,2],[2,-2]].
"""
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np


@dataclass
class Cluster:
    vecs: Tuple[Tuple[int, int], Tuple[int, int]]
    sites: np.ndarray        # [nc, 2] integer coordinates, reduced into the cell
    site_sub: np.ndarray     # [nc, nc] int32: index of (r_i - r_j) reduced into the cell
    kpts: np.ndarray         # [nc, 2] cluster momenta
    k_sub: np.ndarray        # [nc, nc] int32: index of (K_a - K_b) reduced modulo the reciprocal lattice

    @property
    def nc(self) -> int:
        return self.sites.shape[0]


def _reduce(pts: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Reduce integer points modulo the superlattice spanned by the rows of A."""
    Ainv = np.linalg.inv(A.astype(np.float64))
    f = pts.astype(np.float64) @ Ainv
    n = np.floor(f + 1e-9).astype(np.int64)
    return pts - n @ A


def make_cluster(vecs) -> Cluster:
    A = np.array(vecs, dtype=np.int64)
    nc = int(round(abs(np.linalg.det(A.astype(np.float64)))))
    if nc < 1:
        raise ValueError("degenerate cluster vectors")
    R = int(np.abs(A).sum()) + 1
    xs = np.arange(-R, R + 1)
    grid = np.array([(x, y) for x in xs for y in xs], dtype=np.int64)
    red = _reduce(grid, A)
    uniq = sorted(set(map(tuple, red.tolist())), key=lambda p: (p[1], p[0]))
    if len(uniq) != nc:
        raise ValueError("cluster reduction found %d sites, expected %d" % (len(uniq), nc))
    sites = np.array(uniq, dtype=np.int64)
    index = {p: i for i, p in enumerate(uniq)}
    diff = sites[:, None, :] - sites[None, :, :]
    dred = _reduce(diff.reshape(-1, 2), A).reshape(nc, nc, 2)
    site_sub = np.array([[index[tuple(dred[i, j])] for j in range(nc)] for i in range(nc)],
                        dtype=np.int32)
    # Cluster momenta: K = 2 pi A^-1 m for integer m, reduced modulo the
    # reciprocal lattice 2 pi Z^2.
    Ainv = np.linalg.inv(A.astype(np.float64))
    ks = set()
    for m0 in range(-nc, nc + 1):
        for m1 in range(-nc, nc + 1):
            k = Ainv @ np.array([m0, m1], dtype=np.float64)
            k = k - np.floor(k + 1e-9)
            ks.add((round(k[0] * nc) % nc, round(k[1] * nc) % nc))
    ks = sorted(ks)
    if len(ks) != nc:
        raise ValueError("found %d cluster momenta, expected %d" % (len(ks), nc))
    kpts = 2.0 * np.pi * np.array(ks, dtype=np.float64) / nc
    kindex = {p: i for i, p in enumerate(ks)}
    k_sub = np.array([[kindex[((ka[0] - kb[0]) % nc, (ka[1] - kb[1]) % nc)] for kb in ks] for ka in ks],
                     dtype=np.int32)
    return Cluster(vecs=tuple(map(tuple, A.tolist())), sites=sites, site_sub=site_sub, kpts=kpts, k_sub=k_sub)


def square_dispersion(kpts: np.ndarray, t: float, tp: float) -> np.ndarray:
    """eps_K = -2t (cos Kx + cos Ky) - 4t' cos Kx cos Ky (square lattice, App. B model group)."""
    cx, cy = np.cos(kpts[:, 0]), np.cos(kpts[:, 1])
    return -2.0 * t * (cx + cy) - 4.0 * tp * cx * cy


def k_dot_r(cluster: Cluster) -> np.ndarray:
    """[nc_K, nc_r] matrix of K . r for the cluster momenta and sites."""
    return cluster.kpts @ cluster.sites.T.astype(np.float64)


CLUSTER_VECS = {
    1: ((1, 0), (0, 1)),
    4: ((2, 0), (0, 2)),
    8: ((2, 2), (2, -2)),
    16: ((4, 0), (0, 4)),
    36: ((6, 0), (0, 6)),
}


def cluster(nc: int) -> Cluster:
    return make_cluster(CLUSTER_VECS[nc])


@dataclass
class Workload:
    """Named synthetic workload (the paper's Hubbard runs stand behind these shapes)."""
    name: str
    nc: int
    t: float
    tp: float
    U: float
    beta: float
    mu: float
    K: float = 1.0
    n_tau: int = 4096
    k_sub: int = 32
    walkers: int = 1
    sweeps: int = 10000
    warmup_sweeps: int = 20
    n_tau_meas: int = 256
    seed: int = 0
    init_config_size: int = 10
    recompute_every: int = 64
    recompute_sweeps: int = 0
    recompute_at_measure: bool = False  # mixed path: N recomputed before every measurement
    n_omega_meas: int = 0  # frequency measurement of M: positive Matsubara frequencies
    freq_method: str = "nfft"  # "nfft" (delayed NFFT) or "dft" (the same sums as a dense contraction)
    n_w4: int = 0  # two-particle measurement (pp up-down): fermionic frequencies per sign
    w4_transfer: int = 0  # its bosonic frequency transfer index
    q4_transfer: int = 0  # its momentum transfer (cluster momentum index)
    autotune: bool = False  # bench: choose k_s and the update kernel by the autotuner
    schedule: str = "lockstep"  # "pooled": the walkers share the sweep budget (all active every window)
    # a spin changed twice in one window: "update" applies it in place, "abort"
    # ends the window there (both give the chain of single-spin updates)
    duplicate_rule: str = "update"
    # recompute of N: "auto" (mixed: Newton step, residual from digit planes on
    # the tensor cores), "newton_df" (residual in double-float), "gj"
    recompute_method: str = "auto"
    precision: str = "fp64"
    # batched workloads: per-walker problems drawn from these ranges (seeded)
    nc_choices: Tuple[int, ...] = ()
    beta_range: Tuple[float, float] = (0.0, 0.0)
    U_range: Tuple[float, float] = (0.0, 0.0)
    extra: dict = field(default_factory=dict)

    def problem_params(self):
        """(list of per-problem dicts with nc, t, tp, U, beta, mu, K, n_tau; walker -> problem index)."""
        if not self.nc_choices:
            p = dict(nc=self.nc, t=self.t, tp=self.tp, U=self.U, beta=self.beta, mu=self.mu, K=self.K,
                     n_tau=self.n_tau)
            return [p], [0] * self.walkers
        rng = np.random.default_rng(self.seed + 12345)
        probs = []
        for w in range(self.walkers):
            nc = int(self.nc_choices[w % len(self.nc_choices)])
            beta = float(rng.uniform(*self.beta_range))
            U = float(rng.uniform(*self.U_range))
            probs.append(dict(nc=nc, t=self.t, tp=self.tp, U=U, beta=beta, mu=U / 2, K=self.K, n_tau=self.n_tau))
        return probs, list(range(self.walkers))


# Chemical potentials.  The atom is at half filling, mu = U/2.  The 2x2 value
# gives density 0.9 by exact diagonalisation; the 16- and 36-site values are
# U/2 + mu0 with mu0 giving the target density of the free isolated cluster.
# Both were produced by tests/golden/make_golden.py and are stored in
# tests/golden/hubbard_2x2_ed.json and tests/golden/free_cluster_mu.json.
WORKLOADS = {
    "atom_nc1": Workload(name="atom_nc1", nc=1, t=0.0, tp=0.0, U=4.0, beta=2.0, mu=2.0, K=1.0,
                         n_tau=4096, k_sub=8, sweeps=10000, n_tau_meas=256, seed=0),
    "hubbard_2x2": Workload(name="hubbard_2x2", nc=4, t=1.0, tp=0.0, U=4.0, beta=10.0,
                            mu=0.9450480104035819,
                            K=1.0, n_tau=4096, k_sub=32, sweeps=100000, n_tau_meas=256, seed=0),
    # 16-site square cluster, t' = -0.15, U = 6, beta = 20, density 0.9 (free-cluster mu)
    "betts16": Workload(name="betts16", nc=16, t=1.0, tp=-0.15, U=6.0, beta=20.0, mu=2.8528393768386398,
                        K=1.0, n_tau=4096, k_sub=64, sweeps=10000, warmup_sweeps=40, n_tau_meas=256,
                        recompute_every=64, precision="fp64"),
    "betts16_mixed": Workload(name="betts16_mixed", nc=16, t=1.0, tp=-0.15, U=6.0, beta=20.0,
                              mu=2.8528393768386398, K=1.0, n_tau=4096, k_sub=64, sweeps=10000,
                              warmup_sweeps=40, n_tau_meas=256, recompute_every=64, precision="mixed"),
    # 256 independent walkers, Nc in {8, 16}, beta ~ U[5, 25], U ~ U[4, 7], half filling;
    # N recomputed every 8 sweeps (the bench also times the schedule with N
    # recomputed before every measurement, which meets G error <= 1e-6)
    "batched256": Workload(name="batched256", nc=16, t=1.0, tp=0.0, U=5.5, beta=15.0, mu=2.75, K=1.0,
                           n_tau=2048, k_sub=64, walkers=256, warmup_sweeps=40, n_tau_meas=128,
                           recompute_every=0, recompute_sweeps=8, precision="mixed", nc_choices=(8, 16),
                           autotune=True, schedule="pooled", beta_range=(5.0, 25.0), U_range=(4.0, 7.0)),
    # the same batch with the frequency measurement of M on (128 frequencies): the
    # delayed NFFT, and the same sums as a dense contraction
    "batched256_freq": Workload(name="batched256_freq", nc=16, t=1.0, tp=0.0, U=5.5, beta=15.0, mu=2.75, K=1.0,
                                n_tau=2048, k_sub=64, walkers=256, warmup_sweeps=40, n_tau_meas=128,
                                recompute_every=0, recompute_sweeps=8, precision="mixed", n_omega_meas=128,
                                nc_choices=(8, 16), autotune=True, schedule="pooled", beta_range=(5.0, 25.0),
                                U_range=(4.0, 7.0)),
    "batched256_dft": Workload(name="batched256_dft", nc=16, t=1.0, tp=0.0, U=5.5, beta=15.0, mu=2.75, K=1.0,
                               n_tau=2048, k_sub=64, walkers=256, warmup_sweeps=40, n_tau_meas=128,
                               recompute_every=0, recompute_sweeps=8, precision="mixed", n_omega_meas=128,
                               freq_method="dft", nc_choices=(8, 16), autotune=True, schedule="pooled",
                               beta_range=(5.0, 25.0), U_range=(4.0, 7.0)),
    # the same batch with the two-particle measurement on: 8 fermionic frequencies
    # per sign (S = 128 or 256 points per spin), zero transfer
    "batched256_g4": Workload(name="batched256_g4", nc=16, t=1.0, tp=0.0, U=5.5, beta=15.0, mu=2.75, K=1.0,
                              n_tau=2048, k_sub=64, walkers=256, warmup_sweeps=40, n_tau_meas=128,
                              recompute_every=0, recompute_sweeps=8, precision="mixed", n_w4=8,
                              nc_choices=(8, 16), autotune=True, schedule="pooled", beta_range=(5.0, 25.0),
                              U_range=(4.0, 7.0)),
    # 36-site square cluster, U = 7, beta = 30, density 0.95, 32 walkers, G on 2048 tau points
    "betts36": Workload(name="betts36", nc=36, t=1.0, tp=0.0, U=7.0, beta=30.0, mu=3.4878678207599574, K=1.0,
                        n_tau=4096, k_sub=64, walkers=32, warmup_sweeps=40, n_tau_meas=2048,
                        recompute_every=0, recompute_sweeps=4, precision="mixed"),
}


def seeded_uniform(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    """Reproducible uniform draws for workload parameters (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return lo + (hi - lo) * rng.random(n)
