"""Scalar types the oracle's residual runs on: float, forward-mode dual numbers
and complex numbers (complex step).

The paper evaluates the Riemann-flux and ghost-state Jacobians exactly by
automatic differentiation (Sec. 4.4, after Eq. jac2).  The oracle follows
that: J v is the derivative part of the residual evaluated on ``Dual``
numbers (value, derivative).  The complex-step derivative
Im R(u + i h v) / h is a second, independent derivative used to pin the
dual-number result; for it |x| is continued as x sign(Re x).

The residual code calls only the helpers below, so one residual routine
serves all three scalar types.
"""
import numpy as np


class Dual:
    """Elementwise forward-mode dual number over numpy arrays."""

    __array_priority__ = 100.0

    def __init__(self, val, der):
        # float64, or complex128 when a complex step runs through dual numbers
        self.val = np.asarray(val, dtype=np.result_type(val, np.float64))
        self.der = np.asarray(der, dtype=np.result_type(der, np.float64))

    @staticmethod
    def _split(o):
        if isinstance(o, Dual):
            return o.val, o.der
        return o, 0.0

    def __add__(self, o):
        v, d = Dual._split(o)
        return Dual(self.val + v, self.der + d)

    __radd__ = __add__

    def __sub__(self, o):
        v, d = Dual._split(o)
        return Dual(self.val - v, self.der - d)

    def __rsub__(self, o):
        v, d = Dual._split(o)
        return Dual(v - self.val, d - self.der)

    def __neg__(self):
        return Dual(-self.val, -self.der)

    def __mul__(self, o):
        v, d = Dual._split(o)
        return Dual(self.val * v, self.der * v + self.val * d)

    __rmul__ = __mul__

    def __truediv__(self, o):
        v, d = Dual._split(o)
        q = self.val / v
        return Dual(q, (self.der - q * d) / v)

    def __rtruediv__(self, o):
        v, d = Dual._split(o)
        q = v / self.val
        return Dual(q, (d - q * self.der) / self.val)

    def __pow__(self, e):
        assert not isinstance(e, Dual)
        return Dual(self.val ** e, e * self.val ** (e - 1) * self.der)

    def __getitem__(self, idx):
        return Dual(self.val[idx], self.der[idx])

    @property
    def shape(self):
        return self.val.shape


def real(x):
    """The real (value) part, used for branch decisions."""
    if isinstance(x, Dual):
        return x.val
    return np.real(x)


def sqrt(x):
    if isinstance(x, Dual):
        s = np.sqrt(x.val)
        return Dual(s, 0.5 * x.der / s)
    return np.sqrt(x)


def absval(x):
    """|x| with derivative sign(x) (sign(0) = 0); complex continuation x sign(Re x)."""
    if isinstance(x, Dual):
        sg = np.sign(np.real(x.val))
        return Dual(x.val * sg, sg * x.der)
    if np.iscomplexobj(x):
        return x * np.sign(x.real)
    return np.abs(x)


def power(x, e):
    if isinstance(x, Dual):
        return x ** e
    return np.power(x, e)


def where(cond, a, b):
    """Elementwise select with a real boolean ``cond``."""
    if isinstance(a, Dual) or isinstance(b, Dual):
        av, ad = Dual._split(a)
        bv, bd = Dual._split(b)
        return Dual(np.where(cond, av, bv), np.where(cond, ad, bd))
    return np.where(cond, a, b)


def lin(fn, x):
    """Apply a linear map ``fn`` (e.g. an einsum with constant data) to x."""
    if isinstance(x, Dual):
        return Dual(fn(x.val), fn(x.der))
    return fn(x)


def stack(xs, axis=-1):
    if any(isinstance(x, Dual) for x in xs):
        vals = [Dual._split(x)[0] * np.ones_like(real(xs[0])) if not isinstance(x, Dual) else x.val for x in xs]
        ders = [np.zeros_like(real(xs[0])) if not isinstance(x, Dual) else x.der for x in xs]
        return Dual(np.stack(vals, axis=axis), np.stack(ders, axis=axis))
    return np.stack(xs, axis=axis)


def zeros_like_var(x, shape):
    """A zero array of ``shape`` with the scalar type of ``x``."""
    if isinstance(x, Dual):
        return Dual(np.zeros(shape, dtype=x.val.dtype), np.zeros(shape, dtype=np.result_type(x.val, x.der)))
    return np.zeros(shape, dtype=np.result_type(x, np.float64))


def add_at(target, idx, values):
    """np.add.at for all scalar types (target is modified and returned)."""
    if isinstance(target, Dual):
        vv, vd = Dual._split(values)
        np.add.at(target.val, idx, vv)
        np.add.at(target.der, idx, vd)
        return target
    np.add.at(target, idx, values)
    return target
