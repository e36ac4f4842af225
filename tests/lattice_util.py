"""Small helpers shared by the tests: D2Q9 vectors and initial-state builders.

These build *initial states* only (e.g. a shear wave); no test uses them as the
expected answer. Expected answers come from closed forms, invariants, library
routines or the oracle.
"""
import math

import numpy as np

E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
WQ = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def equilibrium(rho, ux, uy):
    """Second-order D2Q9 equilibrium, used to set up smooth initial states."""
    eu = E[:, 0, None, None] * ux + E[:, 1, None, None] * uy
    uu = ux * ux + uy * uy
    return WQ[:, None, None] * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * uu)


def total_mass(f):
    return math.fsum(np.asarray(f, dtype=np.float64).ravel())


def total_momentum(f):
    f = np.asarray(f, dtype=np.float64)
    return np.array([math.fsum((f * E[:, 0, None, None]).ravel()),
                     math.fsum((f * E[:, 1, None, None]).ravel())])
