"""The hop operator M^4 = -1/2 Dhop M_phi evaluated at single (site, s) points.

Test infrastructure only (see oracle/__init__.py). Used to spot-check outputs
on lattices too large for the full-array oracle. It works directly on the
canonical layouts (gauge U[t][z][y][x][mu][a][b], half field
psi[s][t][z][y][xh][spin][colour]) and follows the same definitions as
dwf_operator (paper Sec. 2.2, eq. for D^w and M^4 = D^w M_phi).
"""
from __future__ import annotations

import numpy as np

from .dwf_operator import GAMMA, ID4, P_MINUS, P_PLUS, Action


def _half_index(coord):
    x, y, z, t = coord
    return (t, z, y, x // 2)


def _mphi_at(act: Action, half, coord, s: int, mf: float) -> np.ndarray:
    """(M_phi psi)(coord, s) = b psi_s + c (P_- psi_{s+1} + P_+ psi_{s-1})."""
    Ls = act.Ls
    h = _half_index(coord)
    v = act.b * half[(s,) + h]
    up = half[((s + 1) % Ls,) + h] * (-mf if s == Ls - 1 else 1.0)
    dn = half[((s - 1) % Ls,) + h] * (-mf if s == 0 else 1.0)
    return v + act.c * (P_MINUS @ up + P_PLUS @ dn)


def m4_at(act: Action, U, half_in, site, s: int, mf: float) -> np.ndarray:
    """(M^4 psi)(site, s) as a (4, 3) array; `half_in` lives on the parity
    opposite to `site`."""
    dims = act.dims
    acc = np.zeros((4, 3), dtype=np.complex128)
    for mu in range(4):
        for step in (+1, -1):
            nb = list(site)
            nb[mu] += step
            sign = 1.0
            if nb[mu] < 0 or nb[mu] >= dims[mu]:
                nb[mu] %= dims[mu]
                if act.antiperiodic and mu == 3:
                    sign = -1.0
            chi = _mphi_at(act, half_in, tuple(nb), s, mf) * sign
            x, y, z, t = site
            if step == +1:
                link = U[t, z, y, x, mu]
                proj = ID4 - GAMMA[mu]
            else:
                xb, yb, zb, tb = nb
                link = U[tb, zb, yb, xb, mu].conj().T
                proj = ID4 + GAMMA[mu]
            acc += proj @ (chi @ link.T)
    return -0.5 * acc
