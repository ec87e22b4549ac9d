"""Error / parameter explorer: the curves of Figures 3, 5 and 7, from the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``error_table``  E(W, x0) of Eq. norm_bound for least-misfit kernels
  (Figure 3 plots E against W; Figures 5 and 7 against x0);
* ``tophat_curve`` E of the top hat (W_z = 1, the original W-stacking seen
  as gridding, Section 6.2) against z0, beside the quoted sqrt(pi/3) z0 (the
  first-order expansion gives (pi/3) z0, 2.3 % higher);
* ``layers``       w-layer counts of the original method (Eq. N_w) and the
  improved one (Eq. N_{w'}+W, with and without z offset) for a baseline set.

``python -m oracle.explore`` prints all three for the default grids.  The
fit is the oracle's ``lmfit.least_misfit``; E falls with W at every x0 of the
table up to W = 14.
"""
from __future__ import annotations

import math

from .geometry import layers_improved, layers_original
from .lmfit import error_bound, least_misfit, tophat_h, tophat_weights


def error_table(Ws=range(1, 15), x0s=(0.1, 0.15, 0.2, 0.25, 0.3, 0.35, 0.4)):
    """{(W, x0): E} for the least-misfit C and h of each pair (Section 3.3)."""
    return {(W, x0): least_misfit(W, x0).E for W in Ws for x0 in x0s}


def tophat_curve(z0s=(0.005, 0.01, 0.02, 0.05, 0.1, 0.2)):
    """[(z0, E_tophat, sqrt(pi/3) z0)]: E of C = top hat, h = 1/sinc (Section 6.2)."""
    return [(z0, error_bound(tophat_weights, tophat_h, 1, z0), math.sqrt(math.pi / 3.0) * z0) for z0 in z0s]


def layers(dn: float, dw: float, z0: float = 0.25, W: int = 7):
    """Layer counts for (n_max - n_min) = dn and (w_max - w_min) = dw wavelengths."""
    return {"original (Eq. N_w)": layers_original(dn, dw),
            "improved": layers_improved(dn, dw, z0, W, True),
            "improved, no z offset": layers_improved(dn, dw, z0, W, False)}


def main():
    x0s = (0.1, 0.15, 0.2, 0.25, 0.3, 0.35, 0.4)
    tab = error_table(range(1, 15), x0s)
    print("E(W, x0)   " + "  ".join(f"x0={x0:<6}" for x0 in x0s))
    for W in range(1, 15):
        print(f"W = {W:2d}    " + "  ".join(f"{tab[(W, x0)]:9.2e}" for x0 in x0s))
    print("\ntop hat: z0, E, sqrt(pi/3) z0")
    for z0, e, approx in tophat_curve():
        print(f"  {z0:6.3f}  {e:.4e}  {approx:.4e}")
    print("\nlayers for dn = 0.0646 (fov 0.5), dw = 2800 wavelengths:", layers(0.0646, 2800.0))


if __name__ == "__main__":
    main()
