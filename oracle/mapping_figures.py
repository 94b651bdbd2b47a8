"""Eigenvalue mappings of the paper's Fig. 1 and Fig. 2 (documentation).

For a spectrum [lambda_min, lambda_max] = [0, 1] with a gap of width 0.1 and
mu = lambda_min + 0.25 (lambda_max - lambda_min) (the figures' illustrative
case: bandwidth / gap = 10), plot lambda -> the eigenvalue of X_i that it maps
to, with and without scaling:

- Fig. 1: McWeeny based fixed-mu purification (Algorithm 1) after 1, 3 and 5
  iterations;
- Fig. 2: P_{0,1} & P_{1,0} based varying-mu purification (Algorithm 2) after
  1, 5 and 9 iterations.

The maps are the oracle's scalar recursions (functional calculus: the matrix
recursion acts on each eigenvalue).  Writes SVG (no plotting library needed):

    python -m oracle.mapping_figures [output directory, default docs/figures]
"""
from __future__ import annotations

import os
import sys

import numpy as np

from oracle import purify_oracle as O

LMIN, LMAX, MU, GAP = 0.0, 1.0, 0.25, 0.1
HOMO, LUMO = MU - GAP / 2, MU + GAP / 2


def fixed_mu_curves(iterations, n: int = 401):
    """lambda grid, and per requested iteration the images with scaling and
    with alpha = 1 (Algorithm 1)."""
    lam = np.linspace(LMIN, LMAX, n)
    gamma = O.fixed_mu_gamma(LMIN, LMAX, MU)
    beta0 = O.fixed_mu_beta0(gamma, MU, HOMO, LUMO)
    out = {}
    for scaled in (True, False):
        alphas, betas = O.fixed_mu_schedule(beta0, 0.0, max(iterations), scaled)
        x = (MU - lam) / gamma + 0.5
        for k, a in enumerate(alphas, start=1):
            xs = a * (x - 0.5) + 0.5
            x = O.P11(xs)
            if k in iterations:
                out[(k, scaled)] = (x.copy(), betas[k - 1], 1.0 - betas[k - 1])
    return lam, out


def tc_curves(iterations, n: int = 401):
    """The same for Algorithm 2 (branches and alpha from beta and beta-bar)."""
    lam = np.linspace(LMIN, LMAX, n)
    c0, c1 = O.tc_f0(LMIN, LMAX)
    b0, bb0 = O.tc_beta0(LMIN, LMAX, HOMO, LUMO)
    out = {}
    for scaled in (True, False):
        steps = O.tc_schedule(b0, bb0, 0.0, max(iterations), scaled)
        x = c0 + c1 * lam
        for k, (branch, a, b, bb) in enumerate(steps, start=1):
            x = O.tc_map(branch, a, x)
            if k in iterations:
                out[(k, scaled)] = (x.copy(), b, bb)
    return lam, out


def _panel(x0: float, y0: float, w: float, h: float, lam, curves, k: int) -> list[str]:
    """One panel: frame, gap band, mu, the scaled (solid) and unscaled
    (dashed) images after k iterations."""
    def px(v):
        return x0 + w * (v - LMIN) / (LMAX - LMIN)

    def py(v):
        return y0 + h * (1.05 - v) / 1.1

    s = [f'<rect x="{x0}" y="{y0}" width="{w}" height="{h}" fill="none" stroke="black"/>',
         f'<rect x="{px(HOMO):.1f}" y="{y0}" width="{px(LUMO) - px(HOMO):.1f}" height="{h}" '
         f'fill="#dddddd"/>',
         f'<line x1="{px(MU):.1f}" y1="{y0}" x2="{px(MU):.1f}" y2="{y0 + h}" stroke="#999999" '
         f'stroke-dasharray="2,2"/>']
    for v in (0.0, 1.0):
        s.append(f'<line x1="{x0}" y1="{py(v):.1f}" x2="{x0 + w}" y2="{py(v):.1f}" stroke="#cccccc"/>')
    for scaled, style in ((False, 'stroke="#888888" stroke-dasharray="5,3"'), (True, 'stroke="#1f4e9a"')):
        x, _, _ = curves[(k, scaled)]
        pts = " ".join(f"{px(a):.1f},{py(b):.1f}" for a, b in zip(lam, x))
        s.append(f'<polyline fill="none" stroke-width="1.5" {style} points="{pts}"/>')
    s.append(f'<text x="{x0 + w / 2}" y="{y0 + h + 16}" text-anchor="middle" font-size="12">'
             f"eigenvalue of F (iteration {k})</text>")
    return s


def write_svg(path: str, title: str, lam, curves, iterations) -> None:
    w, h, gap = 240, 200, 40
    width = 60 + len(iterations) * (w + gap)
    lines = [f'<svg xmlns="http://www.w3.org/2000/svg" width="{width}" height="{h + 90}" '
             f'font-family="sans-serif">',
             f'<text x="{width / 2}" y="18" text-anchor="middle" font-size="14">{title}</text>']
    for p, k in enumerate(iterations):
        lines += _panel(40 + p * (w + gap), 30, w, h, lam, curves, k)
    lines.append(f'<text x="40" y="{h + 80}" font-size="11">solid: with scaling; dashed: without; '
                 f'grey band: the gap; dotted: mu</text>')
    lines.append("</svg>")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def main(outdir: str = "docs/figures") -> list[str]:
    os.makedirs(outdir, exist_ok=True)
    lam, c1 = fixed_mu_curves((1, 3, 5))
    p1 = os.path.join(outdir, "mapping_fixed_mu_mcweeny.svg")
    write_svg(p1, "Fixed-mu McWeeny purification (Algorithm 1): eigenvalue of X_i", lam, c1, (1, 3, 5))
    lam, c2 = tc_curves((1, 5, 9))
    p2 = os.path.join(outdir, "mapping_varying_mu_p01_p10.svg")
    write_svg(p2, "Varying-mu P_{0,1} & P_{1,0} purification (Algorithm 2): eigenvalue of X_i", lam, c2,
              (1, 5, 9))
    return [p1, p2]


if __name__ == "__main__":
    for p in main(*sys.argv[1:2]):
        print(p)
