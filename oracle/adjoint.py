"""Reverse-mode derivative of K multigrid cycles (oracle side, FP64).

TEST INFRASTRUCTURE (see the package docstring).

Forward map (Sec. 4 cycle, scaled form of mg_oracle.c): u_K = K cycles of
V(nu1, nu2) from u_0 = 0 for right-hand side b and omega-folded weights c.
Loss (the adjoint workload): L = 1/2 ||u_K - u*||^2 with u* held constant.
This module returns dL/db and dL/dc_j for a given g = dL/du_K, by running the
forward once with every operator input recorded (a tape), then applying the
transpose of each operator in reverse order:

  sweep      u' = u + W rh, rh = bh - Ah u, W = sum_j c_j N_j
             (N_0 = I, N_1 = edge/face sum, N_2 = corner sum; Ah = h^2 A_h;
              all symmetric on the interior, Sec. 2 Eq. (2.1))
             gu  = g' - Ah (W g')      gbh += W g'     gc_j += <g', N_j rh>
  restrict   bh_c = 4 R (bh - Ah u)    gbh += 4 R^T g_c, gu -= Ah (4 R^T g_c)
  correct    u' = u + P e              gu = g',  ge = P^T g'
  solve      e = (h0^2 A_h0)^{-1} bh   gbh = (h0^2 A_h0)^{-1} ge  (symmetric)
  load       bh_0 = h^2 b              gb = h^2 gbh_0

with P = 2^d R^T, so 4 R^T g = (4 / 2^d) P g and P^T g = (2^d / 4) * (4 R g).
Every operator is one of the oracle's pinned C routines; the transposes use
the symmetry of Ah, N_j and the coarsest matrix. Only V cycles with nu1 >= 1
are supported (each level visit then starts from zero or from u_k).
"""
from __future__ import annotations

import numpy as np

from . import coarse_solve, prolong_add, residual_scaled, restrict, sweep


def _W(x, c):
    """W x = sum_j c_j N_j x (Dirichlet-truncated): a sweep from u = 0 with bh = x."""
    return sweep(np.zeros_like(x), x, c)


def _N(x, d, j):
    """N_j x with a unit weight vector."""
    e = [0.0, 0.0, 0.0][: (3 if d == 2 else 2)]
    e[j] = 1.0
    return sweep(np.zeros_like(x), x, e)


def _Ah(x):
    """Ah x = h^2 A_h x (scaled 5/7-point operator) = -(residual with bh = 0)."""
    return -residual_scaled(x, np.zeros_like(x))


def _Pt(g):
    """P^T g = 2^d R g."""
    d = g.ndim
    return (2 ** d / 4.0) * restrict(g)


def _4Rt(gc, n):
    """4 R^T g_c = (4 / 2^d) P g_c on a fine grid with n points per axis."""
    d = gc.ndim
    return (4.0 / 2 ** d) * prolong_add(gc, np.zeros((n,) * d))


class _Tape:
    def __init__(self):
        self.ops = []


def _visit(tape, u, bh, c, nu1, nu2, level):
    """Forward visit of one level (gamma = 1); returns the new u."""
    n = u.shape[0]
    if n == 3:
        tape.ops.append(("solve", level))
        return coarse_solve(bh)
    for _ in range(nu1):
        tape.ops.append(("sweep", level, u, bh))
        u = sweep(u, bh, c)
    tape.ops.append(("restrict", level, n))
    bc = restrict(residual_scaled(u, bh))
    e = _visit(tape, np.zeros_like(bc), bc, c, nu1, nu2, level + 1)
    tape.ops.append(("correct", level))
    u = prolong_add(e, u)
    for _ in range(nu2):
        tape.ops.append(("sweep", level, u, bh))
        u = sweep(u, bh, c)
    return u


def forward(b, c, K: int, nu1: int = 1, nu2: int = 1):
    """K V cycles from zero, with the tape; returns (u_K, tape)."""
    b = np.asarray(b, dtype=np.float64)
    N = b.shape[0] + 1
    bh = b / float(N) ** 2  # exact: N is a power of two
    u = np.zeros_like(b)
    tape = _Tape()
    for _ in range(K):
        tape.ops.append(("cycle",))
        u = _visit(tape, u, bh, c, nu1, nu2, 0)
    return u, tape


def vcycles_adjoint(b, c, K: int, g_uK, nu1: int = 1, nu2: int = 1):
    """(dL/db, dL/dc) for dL/du_K = g_uK after K V(nu1, nu2) cycles from 0."""
    if nu1 < 1:
        raise ValueError("the adjoint needs nu1 >= 1")
    b = np.asarray(b, dtype=np.float64)
    d, N = b.ndim, b.shape[0] + 1
    c = tuple(float(x) for x in c)
    ncoef = 3 if d == 2 else 2
    cc = (c + (0.0, 0.0, 0.0))[:ncoef]
    _, tape = forward(b, cc, K, nu1, nu2)
    gc = np.zeros(ncoef)
    # per level: gradient w.r.t. the level's current u and its bh
    gu = {0: np.array(g_uK, dtype=np.float64)}
    gbh = {0: np.zeros_like(b)}
    for op in reversed(tape.ops):
        kind = op[0]
        if kind == "cycle":
            continue
        lev = op[1]
        if kind == "sweep":
            _, _, u_in, bh = op
            g = gu[lev]
            rh = residual_scaled(u_in, bh)
            for j in range(ncoef):
                gc[j] += float(np.vdot(g, _N(rh, d, j)))
            t = _W(g, cc)
            gbh[lev] = gbh[lev] + t
            gu[lev] = g - _Ah(t)
        elif kind == "correct":
            # u' = u + P e: ge = P^T g', the level's gradient passes through
            gu[lev + 1] = _Pt(gu[lev])
            gbh[lev + 1] = np.zeros_like(gu[lev + 1])
        elif kind == "solve":
            gbh[lev] = gbh[lev] + coarse_solve(gu[lev])
            gu[lev] = np.zeros_like(gu[lev])  # the solve ignores its input
        elif kind == "restrict":
            n = op[2]
            gr = _4Rt(gbh[lev + 1], n)
            gbh[lev] = gbh[lev] + gr
            gu[lev] = gu[lev] - _Ah(gr)
    gb = gbh[0] / float(N) ** 2
    return gb, gc
