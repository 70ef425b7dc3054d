"""Exact OT values for small non-uniform instances, by the transport LP solved with scipy's HiGHS.

An independent exact p* (a library routine, not the oracle's arithmetic) for pins that the
certificate of Prop. 3 must bracket: L <= p* <= U.
"""
import numpy as np
from scipy.optimize import linprog
from scipy.sparse import identity, kron, vstack


def lp_pstar(a, b, C) -> float:
    """min <C, X> over X >= 0 with X 1 = a, X^T 1 = b (a, b normalised to the same mass).

    The n + m equalities have rank n + m - 1; the last one is dropped, since a total-mass mismatch of a
    few ulps otherwise makes HiGHS's presolve declare the full system infeasible.
    """
    C = np.asarray(C, np.float64)
    n, m = C.shape
    rows = kron(identity(n), np.ones((1, m)))
    cols = kron(np.ones((1, n)), identity(m))
    A_eq = vstack([rows, cols]).tocsr()[:-1]
    b_eq = np.concatenate([a, b])[:-1]
    res = linprog(C.ravel(), A_eq=A_eq, b_eq=b_eq, bounds=(0, None), method="highs")
    assert res.status == 0, res.message
    return float(res.fun)
