"""FP64 oracle of the smoothed second-order total generalized variation (TGV)
regulariser of Stages 1 and 5 (Eq. 2, L_TGV), test infrastructure only.

Parity status: pinned by tests/test_oracle_pins.py (finite differences of the
energy in u and w; an independent sparse-matrix formulation; constant fields).

The paper names TGV without a discretisation.  Reading (the classical
second-order TGV of Bredies, Kunisch and Pock, with its two absolute values
smoothed so that Adam can descend it):

    J(u, w) = sum_i  alpha1 phi(D u[i] - w[i])  +  alpha0 phi_F(E(w)[i]),
    phi(v)   = sqrt(|v|^2 + eps^2)                          (3-vectors),
    phi_F(E) = sqrt(sum_ab E_ab^2 + eps^2)                  (3x3, all nine entries),
    E(w)_ab  = (D_a w_b + D_b w_a) / 2,

with w = (w_x, w_y, w_z) an auxiliary vector field on the voxel grid and D_a the
forward difference along axis a divided by the spacing, zero on the last
index (Neumann boundary).  Gradients, with q = alpha1 (D u - w) / phi and
P = alpha0 E / phi_F:

    dJ/du   = sum_a D_a^T q_a,
    dJ/dw_b = -q_b + sum_a D_a^T P_ab,

(D_a^T y)[j] = ([j_a >= 1] y[j - e_a] - [j_a <= n_a - 2] y[j]) / d_a.

Arrays are [nz][ny][nx] (x fastest); w is [3][nz][ny][nx] ordered (x, y, z).
"""
from __future__ import annotations

import math

import numpy as np

# array axis of each spatial direction (x, y, z) in a [nz][ny][nx] volume
_AX = (2, 1, 0)


def diff(v, a, d):
    """Forward difference along direction a (0 = x, 1 = y, 2 = z), zero on the last index."""
    ax = _AX[a]
    out = np.zeros_like(v, dtype=np.float64)
    hi = [slice(None)] * 3
    lo = [slice(None)] * 3
    hi[ax] = slice(1, None)
    lo[ax] = slice(0, -1)
    out[tuple(lo)] = (v[tuple(hi)] - v[tuple(lo)]) / d
    return out


def diff_t(y, a, d):
    """Transpose of diff: ([j_a >= 1] y[j - e_a] - [j_a <= n_a - 2] y[j]) / d."""
    ax = _AX[a]
    out = np.zeros_like(y, dtype=np.float64)
    dst = [slice(None)] * 3
    src = [slice(None)] * 3
    dst[ax] = slice(1, None)
    src[ax] = slice(0, -1)
    out[tuple(dst)] += y[tuple(src)]
    out[tuple(src)] -= y[tuple(src)]
    return out / d


def energy_and_grad(u, w, spacing, alpha1, alpha0, eps):
    """Returns (J, dJ/du [nz][ny][nx], dJ/dw [3][nz][ny][nx]) in FP64.
    spacing = (dx, dy, dz)."""
    u = np.asarray(u, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    d = [float(s) for s in spacing]
    r = np.stack([diff(u, a, d[a]) - w[a] for a in range(3)])          # D u - w
    phi1 = np.sqrt((r * r).sum(0) + eps * eps)
    E = np.empty((3, 3) + u.shape)
    Dw = [[diff(w[b], a, d[a]) for b in range(3)] for a in range(3)]   # Dw[a][b] = D_a w_b
    for a in range(3):
        for b in range(3):
            E[a, b] = 0.5 * (Dw[a][b] + Dw[b][a])
    phi2 = np.sqrt((E * E).sum((0, 1)) + eps * eps)
    J = alpha1 * math.fsum(phi1.ravel()) + alpha0 * math.fsum(phi2.ravel())
    q = alpha1 * r / phi1
    P = alpha0 * E / phi2
    gu = sum(diff_t(q[a], a, d[a]) for a in range(3))
    gw = np.stack([-q[b] + sum(diff_t(P[a, b], a, d[a]) for a in range(3)) for b in range(3)])
    return J, gu, gw
