"""Shared test helpers: problem setup from the input generators plus the
oracle's G0 builder (never the GPU library), and binning statistics."""
import numpy as np

from oracle import g0 as og0
from paper_1901_01047_gb300 import inputs


def problem(nc, t, tp, U, beta, mu, n_tau):
    c = inputs.cluster(nc)
    eps = inputs.square_dispersion(c.kpts, t, tp)
    kr = inputs.k_dot_r(c)
    G0 = og0.g0_table(eps, kr, mu, U, beta, n_tau)
    return c, eps, kr, G0


def binned(values):
    """Mean and standard error over bins (rows)."""
    v = np.asarray(values, dtype=np.float64)
    return v.mean(0), v.std(0, ddof=1) / np.sqrt(v.shape[0])
