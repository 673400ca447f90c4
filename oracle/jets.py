"""Second-order jets in d = 1 or 2 variables (plain forward-mode calculus).

A Jet carries a value and its first and second partial derivatives with
respect to the spatial coordinates y_1..y_d.  Every component is a numpy
array (real or complex: complex entries let the caller differentiate the
whole computation once more by the complex-step method).  The rules are the
product rule and the chain rule for a scalar function phi:
    (phi o f)_i  = phi'(f) f_i
    (phi o f)_ij = phi''(f) f_i f_j + phi'(f) f_ij
Nothing here is specific to the method; it only supplies derivatives of the
fields that the residual operators need.
"""
from __future__ import annotations

import numpy as np


class Jet:
    __slots__ = ("v", "g", "h", "d")

    def __init__(self, v, g, h):
        self.v = v
        self.g = list(g)
        self.h = [list(r) for r in h]
        self.d = len(self.g)

    # -- constructors -----------------------------------------------------
    @staticmethod
    def variable(y, i, d):
        """The coordinate y_i as a jet (d/dy_i = 1, everything else 0)."""
        y = np.asarray(y)
        z = np.zeros_like(y)
        g = [np.ones_like(y) if k == i else z for k in range(d)]
        h = [[z for _ in range(d)] for _ in range(d)]
        return Jet(y, g, h)

    @staticmethod
    def const(c, d):
        c = np.asarray(c)
        z = np.zeros_like(c)
        return Jet(c, [z] * d, [[z] * d for _ in range(d)])

    def _lift(self, o):
        return o if isinstance(o, Jet) else Jet.const(o, self.d)

    # -- arithmetic -------------------------------------------------------
    def __add__(self, o):
        if not isinstance(o, Jet):
            return Jet(self.v + o, self.g, self.h)
        return Jet(self.v + o.v, [a + b for a, b in zip(self.g, o.g)],
                   [[a + b for a, b in zip(r, s)] for r, s in zip(self.h, o.h)])

    __radd__ = __add__

    def __neg__(self):
        return Jet(-self.v, [-a for a in self.g], [[-a for a in r] for r in self.h])

    def __sub__(self, o):
        return self + (-self._lift(o))

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        if not isinstance(o, Jet):
            return Jet(self.v * o, [a * o for a in self.g], [[a * o for a in r] for r in self.h])
        d = self.d
        v = self.v * o.v
        g = [self.g[i] * o.v + self.v * o.g[i] for i in range(d)]
        h = [[self.h[i][j] * o.v + self.g[i] * o.g[j] + self.g[j] * o.g[i] + self.v * o.h[i][j]
              for j in range(d)] for i in range(d)]
        return Jet(v, g, h)

    __rmul__ = __mul__

    def __truediv__(self, o):
        return self * self._lift(o).pow(-1.0)

    def __rtruediv__(self, o):
        return self.pow(-1.0) * o

    def chain(self, f0, f1, f2):
        """Apply a scalar function given its value, first and second derivative at self.v."""
        d = self.d
        g = [f1 * self.g[i] for i in range(d)]
        h = [[f2 * self.g[i] * self.g[j] + f1 * self.h[i][j] for j in range(d)] for i in range(d)]
        return Jet(f0, g, h)

    def pow(self, p):
        """self ** p for a constant exponent p (p may be complex)."""
        x = self.v
        return self.chain(x ** p, p * x ** (p - 1.0), p * (p - 1.0) * x ** (p - 2.0))

    def __pow__(self, p):
        return self.pow(p)

    def sqrt(self):
        return self.pow(0.5)

    def tanh(self):
        t = np.tanh(self.v)
        t1 = 1.0 - t * t
        return self.chain(t, t1, -2.0 * t * t1)

    def exp(self):
        e = np.exp(self.v)
        return self.chain(e, e, e)

    def cos(self):
        c, sn = np.cos(self.v), np.sin(self.v)
        return self.chain(c, -sn, -c)

    def sin(self):
        c, sn = np.cos(self.v), np.sin(self.v)
        return self.chain(sn, c, -sn)

    def ones_like(self):
        return Jet.const(np.ones_like(self.v), self.d)

    @staticmethod
    def vconcat(a, b):
        """Rows of a on top of rows of b (components (rows, n))."""
        return Jet(np.concatenate([a.v, b.v]), [np.concatenate([x, y]) for x, y in zip(a.g, b.g)],
                   [[np.concatenate([x, y]) for x, y in zip(r, t)] for r, t in zip(a.h, b.h)])

    def matvec(self, W, b=None):
        """Affine map a = W h + b applied to a jet whose components are (in, n) arrays.
        The bias enters the value only; derivatives pass through W linearly."""
        v = W @ self.v
        if b is not None:
            v = v + b[:, None]
        return Jet(v, [W @ a for a in self.g], [[W @ a for a in r] for r in self.h])

    def __getitem__(self, k):
        return Jet(self.v[k], [a[k] for a in self.g], [[a[k] for a in r] for r in self.h])

    @staticmethod
    def stack(jets):
        d = jets[0].d
        return Jet(np.stack([j.v for j in jets]),
                   [np.stack([j.g[i] for j in jets]) for i in range(d)],
                   [[np.stack([j.h[i][k] for j in jets]) for k in range(d)] for i in range(d)])
