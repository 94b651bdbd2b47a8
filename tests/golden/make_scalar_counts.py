"""Writes scalar_counts.txt and config_counts.txt: multiplications each scheme needs until its
scalar error bound max(beta, 1 - betabar) is at most 1e-9, on a spectrum
[0, 1] with the gap (width xi) centred on mu, from the oracle's scalar
schedules of Algorithm 1 (McWeeny, 2 products per iteration) and Algorithm 2
(P_{0,1} / P_{1,0}, 1 product per iteration), with scaling and without
(alpha = 1 / alpha = 0); config_counts.txt holds the same on the dense test
configurations' spectrum [-1, 1].  Calls only the oracle:

    python -m tests.golden.make_scalar_counts
"""
import os

from oracle import purify_oracle as O

TOL = 1e-9
HERE = os.path.dirname(os.path.abspath(__file__))


def counts(mu: float, xi: float):
    homo, lumo = mu - xi / 2, mu + xi / 2
    gamma = O.fixed_mu_gamma(0.0, 1.0, mu)
    b0 = O.fixed_mu_beta0(gamma, mu, homo, lumo)
    mcw = [2 * len(O.fixed_mu_schedule(b0, TOL, 10_000, scaled)[0]) for scaled in (False, True)]
    tb, tbb = O.tc_beta0(0.0, 1.0, homo, lumo)
    tc = [len(O.tc_schedule(tb, tbb, TOL, 10_000, scaled)) for scaled in (False, True)]
    return mcw[0], mcw[1], tc[0], tc[1]


def config_counts(gap: float, tol: float):
    """The same counts on the dense test configurations' spectrum: [-1, 1],
    mu = 0, gap edges -gap/2 and gap/2, to the bound tol."""
    homo, lumo = -gap / 2, gap / 2
    gamma = O.fixed_mu_gamma(-1.0, 1.0, 0.0)
    b0 = O.fixed_mu_beta0(gamma, 0.0, homo, lumo)
    mcw = [2 * len(O.fixed_mu_schedule(b0, tol, 10_000, scaled)[0]) for scaled in (False, True)]
    tb, tbb = O.tc_beta0(-1.0, 1.0, homo, lumo)
    tc = [len(O.tc_schedule(tb, tbb, tol, 10_000, scaled)) for scaled in (False, True)]
    return mcw[0], mcw[1], tc[0], tc[1]


def main() -> str:
    rows = ["# multiplications to max(beta, 1 - betabar) <= 1e-9, spectrum [0, 1]",
            "# columns: mu xi mcweeny_mono mcweeny_scaled tc_mono tc_scaled",
            "# (Algorithm 1 with alpha = 1 / Eq. 3's alpha; Algorithm 2 with alpha = 0 / its fold alpha)"]
    cases = [(0.5, 10.0 ** -k) for k in range(1, 7)] + [(mu, 0.01) for mu in (0.1, 0.25, 0.4, 0.6, 0.75, 0.9)]
    for mu, xi in cases:
        rows.append("%.2f %.0e %d %d %d %d" % ((mu, xi) + counts(mu, xi)))
    path = os.path.join(HERE, "scalar_counts.txt")
    with open(path, "w") as f:
        f.write("\n".join(rows) + "\n")
    rows = ["# multiplications to max(beta, 1 - betabar) <= tol, spectrum [-1, 1], mu = 0, gap edges -gap/2, gap/2",
            "# columns: gap tol mcweeny_mono mcweeny_scaled tc_mono tc_scaled"]
    for gap in (1e-1, 1e-2, 1e-3, 1e-4):
        for tol in (1e-12, 1e-9, 1e-6):
            rows.append("%.0e %.0e %d %d %d %d" % ((gap, tol) + config_counts(gap, tol)))
    with open(os.path.join(HERE, "config_counts.txt"), "w") as f:
        f.write("\n".join(rows) + "\n")
    return path


if __name__ == "__main__":
    print(main())
