"""Truncated multivariate Taylor polynomials in d = 1 or 2 variables (plain forward-mode calculus).

Test infrastructure (the oracle), never imported by the product path.

A Taylor object holds, at every point of a batch, the coefficients c_a of
    f(y0 + h) = sum_{|a| <= K} c_a h^a        (a a multi-index, h^a = h1^a1 h2^a2)
so c_a = (d^a f)(y0) / a!.  Arithmetic is the truncated power-series arithmetic: sums add
coefficients, products convolve them (terms beyond total order K dropped), and a scalar function
phi of a series u = u0 + v (v without constant term) is sum_n phi^(n)(u0) / n! v^n, with v^n
again a truncated product.  Coefficients are numpy arrays (real or complex, so the caller can
differentiate the whole computation once more by a complex step).

It supplies the higher y-derivatives the derivative losses need (Methods, "Training Loss", the
d1 and d2 losses): the second-order Jet of jets.py stops at the Hessian.  Nothing here is
specific to the method.
"""
from __future__ import annotations

from math import factorial

import numpy as np


def multi_indices(d, K):
    """All multi-indices of total order <= K in d variables, by order then lexicographically."""
    out = []
    for n in range(K + 1):
        if d == 1:
            out.append((n,))
        else:
            for i in range(n, -1, -1):
                out.append((i, n - i))
    return out


class Taylor:
    __slots__ = ("c", "d", "K")

    def __init__(self, coeffs, d, K):
        self.c = dict(coeffs)   # multi-index -> array
        self.d = d
        self.K = K

    # -- constructors -------------------------------------------------------
    @staticmethod
    def variable(y, i, d, K):
        """The coordinate y_i expanded at y: value y, coefficient 1 on h_i."""
        c = {a: np.zeros_like(y) for a in multi_indices(d, K)}
        c[(0,) * d] = np.asarray(y) + 0.0
        if K >= 1:
            e = tuple(1 if k == i else 0 for k in range(d))
            c[e] = np.ones_like(y)
        return Taylor(c, d, K)

    @staticmethod
    def const(v, d, K, like=None):
        v = np.asarray(v) + 0.0
        if like is not None:
            v = v + np.zeros_like(like)
        c = {a: np.zeros_like(v) for a in multi_indices(d, K)}
        c[(0,) * d] = v
        return Taylor(c, d, K)

    # -- access -------------------------------------------------------------
    @property
    def v(self):
        return self.c[(0,) * self.d]

    def deriv(self, a):
        """The partial derivative d^a f at the expansion point: a! c_a."""
        m = 1
        for k in a:
            m *= factorial(k)
        return m * self.c[tuple(a)]

    def diff(self, i):
        """The series of d f / d y_i (one order lower)."""
        K = self.K - 1
        c = {}
        for a in multi_indices(self.d, K):
            b = tuple(a[k] + (1 if k == i else 0) for k in range(self.d))
            c[a] = (a[i] + 1) * self.c[b]
        return Taylor(c, self.d, K)

    # -- arithmetic -----------------------------------------------------------
    def _lift(self, o):
        if isinstance(o, Taylor):
            assert o.d == self.d
            if o.K == self.K:
                return o, self.K
            K = min(o.K, self.K)
            return o, K
        return Taylor.const(o, self.d, self.K, like=self.v), self.K

    def _trunc(self, K):
        if K == self.K:
            return self
        return Taylor({a: self.c[a] for a in multi_indices(self.d, K)}, self.d, K)

    def __add__(self, o):
        o, K = self._lift(o)
        a, b = self._trunc(K), o._trunc(K)
        return Taylor({m: a.c[m] + b.c[m] for m in multi_indices(self.d, K)}, self.d, K)

    __radd__ = __add__

    def __neg__(self):
        return Taylor({m: -x for m, x in self.c.items()}, self.d, self.K)

    def __sub__(self, o):
        return self + (-o if isinstance(o, Taylor) else -np.asarray(o))

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        if not isinstance(o, Taylor):
            o = np.asarray(o)
            return Taylor({m: x * o for m, x in self.c.items()}, self.d, self.K)
        K = min(self.K, o.K)
        a, b = self._trunc(K), o._trunc(K)
        idx = multi_indices(self.d, K)
        out = {m: 0.0 * a.v * b.v for m in idx}
        for p in idx:
            for q in idx:
                s = tuple(p[k] + q[k] for k in range(self.d))
                if sum(s) <= K:
                    out[s] = out[s] + a.c[p] * b.c[q]
        return Taylor(out, self.d, K)

    __rmul__ = __mul__

    def __truediv__(self, o):
        if isinstance(o, Taylor):
            return self * o.pow(-1.0)
        return self * (1.0 / np.asarray(o))

    def __rtruediv__(self, o):
        return self.pow(-1.0) * o

    def compose(self, derivs):
        """phi(self) for a scalar function phi given its derivatives phi^(n)(u0), n = 0..K."""
        u0 = self.v
        v = Taylor(dict(self.c), self.d, self.K)
        v.c[(0,) * self.d] = 0.0 * u0
        out = Taylor.const(derivs[0], self.d, self.K, like=u0)
        p = None
        for n in range(1, self.K + 1):
            p = v if p is None else p * v
            out = out + p * (derivs[n] / factorial(n))
        return out

    def pow(self, e):
        """self ** e for a constant exponent (falling factorials of e)."""
        x = self.v
        ds, f = [], 1.0
        for n in range(self.K + 1):
            ds.append(f * x ** (e - n))
            f = f * (e - n)
        return self.compose(ds)

    __pow__ = pow

    def sqrt(self):
        return self.pow(0.5)

    def exp(self):
        e = np.exp(self.v)
        return self.compose([e] * (self.K + 1))

    def tanh(self):
        # d/du of a polynomial P(t) in t = tanh u is P'(t) (1 - t^2): the derivatives are
        # polynomials in t, generated here rather than written out
        t = np.tanh(self.v)
        poly = np.array([0.0, 1.0])          # P_0(t) = t, coefficients by power
        ds = []
        for _ in range(self.K + 1):
            ds.append(np.polyval(poly[::-1], t))
            dp = np.polynomial.polynomial.polyder(poly)
            poly = np.polynomial.polynomial.polymul(dp, [1.0, 0.0, -1.0])
        return self.compose(ds)

    # -- vector-valued series (coefficients of shape (rows, n)), as the network needs ------------
    def ones_like(self):
        return Taylor.const(np.ones_like(self.v), self.d, self.K)

    def matvec(self, W, b=None):
        """Affine map W h + b on a series whose coefficients are (in, n) arrays: every
        coefficient maps through W, the bias enters the constant term only."""
        c = {m: W @ x for m, x in self.c.items()}
        if b is not None:
            z = (0,) * self.d
            c[z] = c[z] + b[:, None]
        return Taylor(c, self.d, self.K)

    def __getitem__(self, k):
        return Taylor({m: x[k] for m, x in self.c.items()}, self.d, self.K)

    @staticmethod
    def stack(series):
        s0 = series[0]
        return Taylor({m: np.stack([s.c[m] for s in series]) for m in s0.c}, s0.d, s0.K)

    @staticmethod
    def vconcat(a, b):
        """Rows of a on top of rows of b."""
        return Taylor({m: np.concatenate([a.c[m], b.c[m]]) for m in a.c}, a.d, a.K)

    def cos(self):
        c, s = np.cos(self.v), np.sin(self.v)
        cyc = [c, -s, -c, s]
        return self.compose([cyc[n % 4] for n in range(self.K + 1)])

    def sin(self):
        c, s = np.cos(self.v), np.sin(self.v)
        cyc = [s, c, -s, -c]
        return self.compose([cyc[n % 4] for n in range(self.K + 1)])
