"""The SPAI smoothers of Sec. 3 as omega-folded stencil weights (oracle side).

TEST INFRASTRUCTURE (see the package docstring): only tests, smoke() and the
benchmark's CPU-baseline leg use this module.

A smoother u <- u + omega M_h (b_h - A_h u) (Sec. 2, Eq. (2.1)) whose M_h is a
symmetric stencil proportional to h^2 becomes, in the scaled form used by the
oracle (rh = h^2 (b - A u)),

    2D:  u <- u + c0 rh + c1 (edge sum of rh) + c2 (corner sum of rh)
    3D:  u <- u + c0 rh + c1 (face sum of rh)

with c_j = omega * (stencil weight of class j) / h^2. Each value below is
derived from the paper's exact rational / surd expression and rounded once
to the nearest double (Python's Fraction -> float conversion is correctly
rounded; sqrt(10) is carried to 60 significant digits first).
"""
from __future__ import annotations

from decimal import Decimal, getcontext
from fractions import Fraction as F

getcontext().prec = 60
_SQRT10 = F(Decimal(10).sqrt())


def _r(x: F) -> float:
    return float(x)


# --- exact relaxation parameters and stencils (paper passages) -------------

#: Theorem 3.1: omega_opt = (309 - 12 sqrt(10)) / 1720 for M9 = Upsilon(44,10,3)/24.
OMEGA_M9 = (F(309) - 12 * _SQRT10) / 1720
#: Theorem 3.1: mu_opt = (9 + 8 sqrt(10)) / 215.
MU_M9 = (F(9) + 8 * _SQRT10) / 215
#: Theorem 3.2: omega_opt = 20/73, mu_opt = 25/73 for M7 = T(8/5, 2/5).
OMEGA_M7 = F(20, 73)
MU_M7 = F(25, 73)

# (stencil weights in units of h^2: centre, edge, corner), omega
SMOOTHERS_2D = {
    # Sec. 3.1: weighted Jacobi M_J = h^2/4 I, omega = 4/5, mu = 3/5
    "jacobi": ((F(1, 4), F(0), F(0)), F(4, 5)),
    # Sec. 3.1: Tang-Wan M_5,TW = h^2/61 [3; 3 17 3; 3], omega = 1 (mu = 21/61)
    "tw5": ((F(17, 61), F(3, 61), F(0)), F(1)),
    # Sec. 3.1: best 5-point M_5 = 8h^2/41 [1; 1 6 1; 1], omega = 1/4, mu = 9/41
    "m5": ((F(48, 41), F(8, 41), F(0)), F(1, 4)),
    # Sec. 3.1: additive Vanka Upsilon(28,4,1)/96, omega = 24/25, mu = 7/25
    "vanka": ((F(28, 96), F(4, 96), F(1, 96)), F(24, 25)),
    # Sec. 3.1 / Theorem 3.1: M9 = Upsilon(44,10,3)/24
    "m9": ((F(44, 24), F(10, 24), F(3, 24)), OMEGA_M9),
}

# (stencil weights in units of h^2: centre, face), omega
SMOOTHERS_3D = {
    # Sec. 3.2: weighted Jacobi M_J = h^2/6 I, omega = 6/7, mu = 5/7
    "jacobi": ((F(1, 6), F(0)), F(6, 7)),
    # Sec. 3.2 / Theorem 3.2: M7 = T(8/5, 2/5) = h^2/10 {8 centre, 1 faces}
    "m7": ((F(8, 10), F(1, 10)), OMEGA_M7),
}


def exact_weights(d: int, name: str, omega: F | None = None):
    """omega * stencil weights as exact fractions (sqrt(10) to 60 digits)."""
    table = SMOOTHERS_2D if d == 2 else SMOOTHERS_3D
    w, om = table[name]
    om = om if omega is None else F(omega)
    return tuple(om * wj for wj in w)


def weights(d: int, name: str, omega=None) -> tuple:
    """Correctly rounded omega-folded weights (c0, c1[, c2]) as doubles."""
    return tuple(_r(x) for x in exact_weights(d, name, omega))


def default(d: int) -> tuple:
    """The paper's smoother for dimension d: M9 in 2D, M7 in 3D."""
    return weights(d, "m9" if d == 2 else "m7")
