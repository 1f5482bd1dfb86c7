"""Write the stored inputs and expected values under tests/golden/.

Calls only the oracle (oracle/ed.py, oracle/g0.py) and the input generators.

- hubbard_2x2_ed.json: the chemical potential that gives density 0.9 for the
  2x2 Hubbard cluster (t=1, t'=0, U=4, beta=10) by ED bisection, with the ED
  density, <H_int> and <k> = K - beta <H_int> (K = 1) at that mu.
- free_cluster_mu.json: mu = U/2 + mu0 where mu0 gives the target density of
  the free isolated cluster at that beta (the stand-in used for clusters too
  large for ED), for the 16- and 36-site workloads.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ed, g0  # noqa: E402
from paper_1901_01047_gb300 import inputs  # noqa: E402


def bisect(f, target, lo, hi, it=200):
    for _ in range(it):
        mid = 0.5 * (lo + hi)
        if f(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def main():
    c = inputs.cluster(4)
    eps = inputs.square_dispersion(c.kpts, 1.0, 0.0)
    t = ed.hopping_from_dispersion(eps, inputs.k_dot_r(c), c.site_sub)
    U, beta = 4.0, 10.0
    mu = ed.bisect_mu(t, U, beta, 0.9)
    E = ed.HubbardED(t, U, mu)
    out = dict(nc=4, t=1.0, tp=0.0, U=U, beta=beta, target_density=0.9, mu=mu,
               density=E.density(beta), h_int=E.h_int(beta), k_expected=1.0 - beta * E.h_int(beta),
               double_occupancy=E.double_occupancy(beta))
    with open(os.path.join(HERE, "hubbard_2x2_ed.json"), "w") as f:
        json.dump(out, f, indent=1)
    free = {}
    for name, nc, tp, U, beta, dens in [("betts16", 16, -0.15, 6.0, 20.0, 0.9),
                                        ("betts36", 36, 0.0, 7.0, 30.0, 0.95)]:
        cl = inputs.cluster(nc)
        e = inputs.square_dispersion(cl.kpts, 1.0, tp)
        mu0 = bisect(lambda m: g0.free_density(e, m + U / 2, U, beta), dens, -10, 10)
        free[name] = dict(nc=nc, tp=tp, U=U, beta=beta, target_density=dens, mu=U / 2 + mu0,
                          free_density=g0.free_density(e, U / 2 + mu0, U, beta))
    with open(os.path.join(HERE, "free_cluster_mu.json"), "w") as f:
        json.dump(free, f, indent=1)


if __name__ == "__main__":
    main()
