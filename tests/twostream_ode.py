"""Independent reference for the pins: the two-stream differential equations
solved as a boundary-value problem with matrix exponentials.

This shares nothing with the oracle's closed forms.  With optical depth tau
increasing downward, mu = cos(theta*) > 0 and F_b = mu F* exp(-tau/mu) the
direct beam (Eq. B6 with mu* = -mu), the two streams obey

    dF_up/dtau =  g1 F_up - g2 F_dn - 2 pi (1 - w0) B - w0 g3 F_b / mu
    dF_dn/dtau =  g2 F_up - g1 F_dn + 2 pi (1 - w0) B + w0 g4 F_b / mu

with g1 + g2 = 2 E (1 - w0 g0), g1 - g2 = 2 (E - w0), g3 = 1/2 - g0 mu/(2 eps2),
g4 = 1 - g3.  For E = 1 these are the hemispheric-mean coefficients of
Toon et al. (1989), g1 = 2 - w0 (1 + g0), g2 = w0 (1 - g0); their exponential
rate and eigenvector ratio are the transmission exponent and coupling
coefficients of Eq. B2.  B(tau) is constant in an isothermal layer and linear
between the level values in a non-isothermal sub-layer.  Each sub-layer is
propagated exactly with expm of the 5x5 augmented generator acting on
(F_up, F_dn, B, dB/dtau, F_b); the levels are then tied together by the
boundary conditions F_dn = F_TOA at the top and F_up - F_dn = F_BOA + F_b at
the bottom (Eq. 10), and the dense linear system is solved directly.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

E_TAU32 = float(np.float32(1e-4))
W_SWITCH32 = float(np.float32(0.1))


def e_fit(w0, g0, improved=True, clamp=True):
    """Eq. 19, switched off for w0 <= 0.1 (threshold 0.1f), clamped at 1."""
    if not improved or not (w0 > W_SWITCH32):
        return 1.0
    E = (1.225 - 0.1582 * g0 - 0.1777 * w0 - 0.07465 * g0 ** 2 + 0.2351 * w0 * g0
         - 0.05582 * w0 ** 2)
    return max(E, 1.0) if clamp else E


def generator(w0, g0, E, mu, eps2):
    s, d = 2 * E * (1 - w0 * g0), 2 * (E - w0)
    g1, g2 = 0.5 * (s + d), 0.5 * (s - d)
    K = np.zeros((5, 5))
    K[0, :2] = [g1, -g2]
    K[1, :2] = [g2, -g1]
    K[0, 2] = -2 * np.pi * (1 - w0)
    K[1, 2] = 2 * np.pi * (1 - w0)
    K[2, 3] = 1.0
    if mu > 0:
        g3 = 0.5 - g0 * mu / (2 * eps2)
        g4 = 1.0 - g3
        K[0, 4] = -w0 * g3 / mu
        K[1, 4] = w0 * g4 / mu
        K[4, 4] = -1.0 / mu
    return K


def solve_column(dtau, w0, g0, Bc, Bi, mu, Fstar, F_BOA, *, isothermal=False,
                 improved=True, clamp=True, eps2=2 / 3, F_TOA=0.0):
    """Fluxes at levels, BOA first (matching the oracle's level order).

    dtau, w0, g0, Bc: per API layer (0 = TOA); Bi: per API interface.
    Inputs are used as given (pass float32-rounded values for parity)."""
    dtau = np.asarray(dtau, float); w0 = np.asarray(w0, float); g0 = np.asarray(g0, float)
    L = dtau.size
    subs = []
    for l in range(L):
        if isothermal:
            subs.append((dtau[l], w0[l], g0[l], Bc[l], Bc[l]))
        else:
            subs.append((0.5 * dtau[l], w0[l], g0[l], Bi[l], Bc[l]))
            subs.append((0.5 * dtau[l], w0[l], g0[l], Bc[l], Bi[l + 1]))
    n = len(subs)
    tau = np.concatenate([[0.0], np.cumsum([s[0] for s in subs])])
    Fb = mu * Fstar * np.exp(-tau / mu) if mu > 0 else np.zeros(n + 1)
    M = np.zeros((2 * (n + 1), 2 * (n + 1)))
    rhs = np.zeros(2 * (n + 1))
    # unknowns (TOA first): x[2k] = F_up at level k, x[2k+1] = F_dn
    M[0, 1] = 1.0
    rhs[0] = F_TOA
    for k, (dt, a, g, Bt, Bb) in enumerate(subs):
        E = e_fit(a, g, improved, clamp)
        if (not isothermal) and dt < E_TAU32:
            Bt = Bb = 0.5 * (Bt + Bb)
        Bp = 0.0 if isothermal else (Bb - Bt) / dt
        Phi = expm(generator(a, g, E, mu, eps2) * dt)
        r = 1 + 2 * k
        # [Fu, Fd]_{k+1} - Phi11 [Fu, Fd]_k = Phi12 [Bt, Bp, Fb_k]
        M[r:r + 2, 2 * (k + 1):2 * (k + 1) + 2] = np.eye(2)
        M[r:r + 2, 2 * k:2 * k + 2] = -Phi[:2, :2]
        rhs[r:r + 2] = Phi[:2, 2:] @ np.array([Bt, Bp, Fb[k]])
    M[-1, 2 * n] = 1.0
    M[-1, 2 * n + 1] = -1.0
    rhs[-1] = F_BOA + Fb[n]
    x = np.linalg.solve(M, rhs)
    up = x[0::2][::-1].copy()
    dn = x[1::2][::-1].copy()
    return up, dn, Fb[::-1].copy()
