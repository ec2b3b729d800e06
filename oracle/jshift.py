"""J-shifting interpolation (Section 2.5, Eq. J-shifting-interpolation). Test infrastructure only.

For J1 <= J <= J2 the probability at J is interpolated from the two computed J
values with energy shifts B [J(J+1) - J1(J1+1)] and B [J2(J2+1) - J(J+1)]:

  P_J(E) = w1 P_J1(E - B [J(J+1) - J1(J1+1)]) + w2 P_J2(E + B [J2(J2+1) - J(J+1)]).

Reading: the printed weights give (J - J1)/(J2 - J1) to the J1 term, which makes
P_J = P_J2 at J = J1; the standard linear weights w1 = (J2 - J)/(J2 - J1),
w2 = (J - J1)/(J2 - J1) are used (both are available through ``printed=True``).
B is fitted per interval by least squares so that the J2 curve shifted by
B [J2(J2+1) - J1(J1+1)] overlays the J1 curve.
"""
from __future__ import annotations

import numpy as np


def shifted(E, P, dE):
    """P(E - dE) by linear interpolation on the grid E (constant beyond the ends)."""
    return np.interp(E - dE, E, P, left=P[0], right=P[-1])


def fit_B(E, P1, P2, J1, J2, Bgrid=None):
    """B minimising sum_E (P_J1(E) - P_J2(E + B dJ))^2, dJ = J2(J2+1) - J1(J1+1)."""
    dJ = J2 * (J2 + 1) - J1 * (J1 + 1)
    if dJ == 0:
        return 0.0
    if Bgrid is None:
        span = (E[-1] - E[0]) / dJ
        Bgrid = np.linspace(0.0, span, 2001)
    errs = [np.sum((P1 - shifted(E, P2, -B * dJ)) ** 2) for B in Bgrid]
    return float(Bgrid[int(np.argmin(errs))])


def interpolate(E, P1, P2, J1, J2, J, B, printed=False):
    """J-shifting interpolation between the computed J1 and J2."""
    if J2 == J1:
        return P1.copy()
    w2 = (J - J1) / (J2 - J1)
    w1 = 1.0 - w2
    if printed:
        w1, w2 = w2, w1
    a = shifted(E, P1, B * (J * (J + 1) - J1 * (J1 + 1)))
    b = shifted(E, P2, -B * (J2 * (J2 + 1) - J * (J + 1)))
    return w1 * a + w2 * b
