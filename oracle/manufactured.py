"""Fabricated (manufactured) solutions of Sec. 5 (oracle; test only).

All of the paper's fabricated fields have the form u = (f(x) g(t), 0, 0)
(static: u_x = 1.9 sin x - x; transient: u_x = sin(pi x / 2) sin(2 pi t) and
u_x = x^4 sin(2 pi t)).  For such a field F = diag(F11, 1, 1) with
F11 = 1 + f'(x) g(t), J = F11, and the neo-Hookean first Piola stress is
diagonal:

    P_xx = mu (F11 - 1/F11) + lambda ln(F11) / F11,   P_yy = P_zz = lambda ln F11.

Only P_xx varies along x, so Div P = (dP_xx/dF11 f''(x) g(t), 0, 0) with
dP_xx/dF11 = mu (1 + F11^-2) + lambda (1 - ln F11) F11^-2.  The body force per
unit reference volume is b = rho u_tt - Div P and the dead traction on a face
of outward normal N is P N.  These are closed forms, differentiated by hand.
"""
import numpy as np


class AxialField:
    def __init__(self, f, df, d2f, g=None, dg=None, d2g=None):
        self.f, self.df, self.d2f = f, df, d2f
        one = lambda t: 1.0
        zero = lambda t: 0.0
        self.g = g or one
        self.dg = dg or zero
        self.d2g = d2g or zero

    def displacement(self, X, t):
        out = np.zeros(X.shape)
        out[..., 0] = self.f(X[..., 0]) * self.g(t)
        return out

    def velocity(self, X, t):
        out = np.zeros(X.shape)
        out[..., 0] = self.f(X[..., 0]) * self.dg(t)
        return out

    def _F11(self, x, t):
        return 1.0 + self.df(x) * self.g(t)

    def stress(self, x, t, mu, lam):
        F = self._F11(x, t)
        lnF = np.log(F)
        Pxx = mu * (F - 1.0 / F) + lam * lnF / F
        Pyy = lam * lnF
        return Pxx, Pyy

    def body_force(self, mu, lam, rho):
        def b(X, t):
            x = X[..., 0]
            F = self._F11(x, t)
            dP = mu * (1.0 + F ** -2) + lam * (1.0 - np.log(F)) * F ** -2
            out = np.zeros(X.shape)
            out[..., 0] = rho * self.f(x) * self.d2g(t) - dP * self.d2f(x) * self.g(t)
            return out
        return b

    def traction(self, face, mu, lam):
        sign = -1.0 if face.endswith("min") else 1.0
        axis = "xyz".index(face[0])

        def t(X, tt):
            Pxx, Pyy = self.stress(X[..., 0], tt, mu, lam)
            out = np.zeros(X.shape)
            out[..., axis] = sign * (Pxx if axis == 0 else Pyy)
            return out
        return t


def static_field():
    """u_x = 1.9 sin x - x (Sec. 5.1)."""
    return AxialField(lambda x: 1.9 * np.sin(x) - x,
                      lambda x: 1.9 * np.cos(x) - 1.0,
                      lambda x: -1.9 * np.sin(x))


def sine_field():
    """u_x = sin(pi x / 2) sin(2 pi t) (Sec. 5.2, eq. large_field)."""
    w = 2.0 * np.pi
    k = 0.5 * np.pi
    return AxialField(lambda x: np.sin(k * x), lambda x: k * np.cos(k * x),
                      lambda x: -k * k * np.sin(k * x),
                      lambda t: np.sin(w * t), lambda t: w * np.cos(w * t),
                      lambda t: -w * w * np.sin(w * t))


def quartic_field():
    """u_x = x^4 sin(2 pi t) (Sec. 5.2, implicit)."""
    w = 2.0 * np.pi
    return AxialField(lambda x: x ** 4, lambda x: 4.0 * x ** 3, lambda x: 12.0 * x ** 2,
                      lambda t: np.sin(w * t), lambda t: w * np.cos(w * t),
                      lambda t: -w * w * np.sin(w * t))


def load_vector(disc, field, t, faces=("xmax", "ymin", "ymax", "zmin", "zmax")):
    """Body force plus face tractions of ``field`` at time t (global vector)."""
    f = disc.body_load(field.body_force(disc.mu, disc.lam, disc.rho), t)
    for face in faces:
        f = f + disc.traction_load(face, field.traction(face, disc.mu, disc.lam), t)
    return f
