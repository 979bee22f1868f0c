"""Write tests/golden/wide_smoothers.txt: the LFA-optimal symmetric 19- and
27-point 3D SPAI stencils, found by the oracle's numerical min-max over the
family's class weights (oracle.lfa.optimise_family).

Sec. 3.2 closes by noting that 19- and 27-point 3D stencils, optimised
heuristically, smooth better than M7, without giving their weights; these
are the values this min-max finds (a reading, not a paper value). The same
optimiser recovers Theorem 3.1's M9 and Theorem 3.2's M7 from scratch (the
CPU tests pin that). Run from the repository root:

    python tests/golden/make_wide_smoothers.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lfa  # noqa: E402


def main():
    lines = ["# LFA-optimal symmetric 3D SPAI stencils (numerical min-max, oracle.lfa.optimise_family)",
             "# written by tests/golden/make_wide_smoothers.py; class weights: centre, face, edge[, corner]",
             "# columns: family  quantity  values...",
             "# w = unfolded class weights (centre 1); omega = 2/(l0 + l1) (Eq. (2.7));",
             "# mu = (l1 - l0)/(l1 + l0) (Eq. (2.6)); c = omega * w (the folded weights of the sweep)"]
    for fam in ("nineteen", "twentyseven"):
        w, mu, om = lfa.optimise_family(fam)
        c = [om * x for x in w]
        lines.append(f"{fam} w {' '.join(repr(float(x)) for x in w)}")
        lines.append(f"{fam} omega {float(om)!r}")
        lines.append(f"{fam} mu {float(mu)!r}")
        lines.append(f"{fam} c {' '.join(repr(float(x)) for x in c)}")
    with open(os.path.join(ROOT, "tests", "golden", "wide_smoothers.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
