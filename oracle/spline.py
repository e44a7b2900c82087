"""Natural cubic spline with constant extension (oracle).

Sect. 6.2 states that all frame changes use cubic splines without naming the
end conditions; the reading used throughout is the natural spline (zero second
derivative at both ends) on the current height's reduced-frequency grid, and a
constant continuation by the end values outside the grid.  Pinned in tests
against scipy.interpolate.CubicSpline(bc_type='natural') and against exact
reproduction of polynomials of degree <= 1.
"""
import numpy as np


class NaturalSpline:
    """Linear map from node values y (shape (N, ...)) to spline values."""

    def __init__(self, u):
        u = np.asarray(u, dtype=np.float64)
        assert u.ndim == 1 and u.size >= 2 and np.all(np.diff(u) > 0)
        self.u = u
        n = u.size
        h = np.diff(u)
        self.h = h
        # Q maps node values to second derivatives M (M_0 = M_{n-1} = 0):
        # h_{i-1} M_{i-1} + 2 (h_{i-1} + h_i) M_i + h_i M_{i+1}
        #     = 6 [ (y_{i+1}-y_i)/h_i - (y_i-y_{i-1})/h_{i-1} ]
        Q = np.zeros((n, n))
        if n > 2:
            T = np.zeros((n - 2, n - 2))
            D = np.zeros((n - 2, n))
            for r, i in enumerate(range(1, n - 1)):
                T[r, r] = 2.0 * (h[i - 1] + h[i])
                if r > 0:
                    T[r, r - 1] = h[i - 1]
                if r < n - 3:
                    T[r, r + 1] = h[i]
                D[r, i + 1] += 6.0 / h[i]
                D[r, i] -= 6.0 / h[i] + 6.0 / h[i - 1]
                D[r, i - 1] += 6.0 / h[i - 1]
            Q[1:n - 1, :] = np.linalg.solve(T, D)
        self.Q = Q

    def basis(self, x):
        """Rows phi(x) with S[y](x) = phi(x) @ y, constant extension outside."""
        x = np.asarray(x, dtype=np.float64)
        u, h, Q = self.u, self.h, self.Q
        n = u.size
        out = np.zeros(x.shape + (n,))
        lo = x <= u[0]
        hi = x >= u[-1]
        mid = ~(lo | hi)
        out[lo, 0] = 1.0
        out[hi, n - 1] = 1.0
        xm = x[mid]
        k = np.clip(np.searchsorted(u, xm, side="right") - 1, 0, n - 2)
        t = (xm - u[k]) / h[k]
        rows = np.zeros((xm.size, n))
        idx = np.arange(xm.size)
        rows[idx, k] += 1.0 - t
        rows[idx, k + 1] += t
        c0 = (h[k] ** 2 / 6.0) * ((1.0 - t) ** 3 - (1.0 - t))
        c1 = (h[k] ** 2 / 6.0) * (t ** 3 - t)
        rows += c0[:, None] * Q[k, :] + c1[:, None] * Q[k + 1, :]
        out[mid] = rows
        return out

    def __call__(self, y, x):
        return self.basis(x) @ np.asarray(y)
