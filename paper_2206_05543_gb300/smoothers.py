"""Stencil weights of the SPAI smoothers (He, Liu, Wang, arXiv:2206.05543, Sec. 3).

A smoother u <- u + omega M_h (b_h - A_h u) (Eq. (2.1)) with M_h a symmetric
stencil proportional to h^2 is passed to the library as h-free,
omega-folded weights c_j = omega * (stencil weight of class j) / h^2:

    2D: (centre, edge, corner)      3D: (centre, face[, edge, corner])

Each literal below is the double nearest to the exact value given beside it,
except M19 and M27, which are the values a numerical min-max of the
smoothing factor over their families gives (Sec. 3.2 names such stencils
but prints no weights).
"""
from __future__ import annotations

# 2D (Sec. 3.1)
M9 = (0.2889127276024975, 0.06566198354602215, 0.019698595063806647)
"""M9 = Upsilon(44, 10, 3)/24 with omega = (309 - 12 sqrt 10)/1720 (Theorem 3.1):
c = omega * (44, 10, 3) / 24; smoothing factor (9 + 8 sqrt 10)/215 ~ 0.1595."""
M5 = (12 / 41, 2 / 41)
"""M5 = 8h^2/41 [1; 1 6 1; 1] with omega = 1/4: c = (12/41, 2/41); mu = 9/41."""
VANKA = (7 / 25, 1 / 25, 1 / 100)
"""Additive Vanka Upsilon(28, 4, 1)/96 with omega = 24/25: c = (7/25, 1/25, 1/100); mu = 7/25."""
TANG_WAN = (17 / 61, 3 / 61)
"""M_5,TW = h^2/61 [3; 3 17 3; 3] with omega = 1: c = (17/61, 3/61); mu = 21/61."""
JACOBI_2D = (1 / 5,)
"""Weighted Jacobi h^2/4 with omega = 4/5: c0 = 1/5; mu = 3/5."""

# 3D (Sec. 3.2)
M7 = (16 / 73, 2 / 73)
"""M7 = T(8/5, 2/5) = h^2/10 {8 centre, 1 faces} with omega = 20/73 (Theorem 3.2):
c = (16/73, 2/73); smoothing factor 25/73 ~ 0.343."""
JACOBI_3D = (1 / 7,)
"""Weighted Jacobi h^2/6 with omega = 6/7: c0 = 1/7; mu = 5/7."""
M19 = (0.20341192950260992, 0.038265610500452976, 0.007552423125074582)
"""Symmetric 19-point stencil (centre, 6 faces, 12 edges) minimising the
smoothing factor over its family (Sec. 3.2, closing remark): unfolded class
weights (1, 0.188118811881, 0.0371287128712) with omega = 0.2034119295;
mu = 0.22663 (M7: 0.343)."""
M27 = (0.1965670905902807, 0.03973164596853401, 0.01150126593697686, 0.003659493706759684)
"""Symmetric 27-point stencil (centre, 6 faces, 12 edges, 8 corners)
minimising the smoothing factor over its family (Sec. 3.2, closing remark):
unfolded class weights (1, 0.2021276596, 0.0585106383, 0.0186170213) with
omega = 0.1965670906; mu = 0.19700 (M7: 0.343)."""

BY_NAME = {
    (2, "m9"): M9, (2, "m5"): M5, (2, "vanka"): VANKA, (2, "tw5"): TANG_WAN, (2, "jacobi"): JACOBI_2D,
    (3, "m7"): M7, (3, "jacobi"): JACOBI_3D, (3, "m19"): M19, (3, "m27"): M27,
}


def default(d: int) -> tuple:
    """The paper's smoother for dimension d: M9 (2D) or M7 (3D)."""
    return M9 if d == 2 else M7


def get(d: int, name: str) -> tuple:
    return BY_NAME[(d, name)]
