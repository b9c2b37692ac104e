"""Independent uniform-grid finite-volume solver and exact-solution helpers for
the oracle pins.  It is the textbook FV scheme of Sec. 2 (Eq. 2) with the
explicit RK methods of Sec. 3 in Butcher form (Eqs. 8-9), written
vectorised over a uniform periodic 1D grid with numpy -- a different
formulation from the oracle's per-leaf compact-form loops."""
from __future__ import annotations

import numpy as np

# Butcher tableaux from Sec. 3: c1=0, c2=a21=1, b=(1/2,1/2) for RK2;
# c3=1/2, a31=a32=1/4, b=(1/6,1/6,2/3) for RK3
BUTCHER = {
    2: (np.array([[0, 0], [1, 0]], float), np.array([0.5, 0.5])),
    3: (np.array([[0, 0, 0], [1, 0, 0], [0.25, 0.25, 0]], float),
        np.array([1 / 6, 1 / 6, 2 / 3])),
}


def _minmod(a, b):
    return np.where(a * b <= 0, 0.0, np.where(np.abs(a) < np.abs(b), a, b))


def burgers_rhs(u, h):
    """-(F_{i+1/2} - F_{i-1/2})/h, MUSCL-minmod + Godunov, periodic."""
    um, up, upp = np.roll(u, 1), np.roll(u, -1), np.roll(u, -2)
    uL = u + 0.5 * _minmod(u - um, up - u)
    uR = up - 0.5 * _minmod(up - u, upp - up)
    fL, fR = 0.5 * uL ** 2, 0.5 * uR ** 2
    rare = np.where(uL > 0, fL, np.where(uR < 0, fR, 0.0))
    F = np.where(uL <= uR, rare, np.maximum(fL, fR))  # flux at i+1/2
    return -(F - np.roll(F, 1)) / h


def advection_rhs(u, h, a=1.0):
    F = a * (u + np.roll(u, -1)) / 2.0
    return -(F - np.roll(F, 1)) / h


def rk_solve(u0, rhs, dt, nsteps, order):
    A, b = BUTCHER[order]
    u = u0.copy()
    s = len(b)
    for _ in range(nsteps):
        K = []
        for i in range(s):
            ui = u + sum(A[i, j] * K[j] for j in range(i))
            K.append(dt * rhs(ui))
        u = u + sum(b[i] * K[i] for i in range(s))
    return u


def burgers_exact_sine(x, t, iters=60):
    """u = sin(2 pi (x - u t)) by Newton, valid before the shock (t < 1/(2 pi))."""
    u = np.sin(2 * np.pi * x)
    for _ in range(iters):
        g = u - np.sin(2 * np.pi * (x - u * t))
        dg = 1 + 2 * np.pi * t * np.cos(2 * np.pi * (x - u * t))
        u = u - g / dg
    return u


GL8_X, GL8_W = np.polynomial.legendre.leggauss(8)


def cell_average_1d(fun, n, lo=0.0, hi=1.0):
    h = (hi - lo) / n
    c = lo + (np.arange(n) + 0.5) * h
    return sum(0.5 * w * fun(c + 0.5 * h * x) for x, w in zip(GL8_X, GL8_W))


def poly_cell_average(coeffs, a, b):
    """exact mean of sum_k coeffs[k] x^k over [a, b]"""
    out = 0.0
    for k, ck in enumerate(coeffs):
        out = out + ck * (b ** (k + 1) - a ** (k + 1)) / ((k + 1) * (b - a))
    return out


def exact_riemann(left, right, gamma, xi):
    """Exact solution of the 1D Euler Riemann problem with states
    left = (rho, u, p), right = (rho, u, p), sampled at the similarity
    coordinates xi = (x - x0) / t.  Returns rho, u, p arrays.  The star
    pressure solves f_L(p) + f_R(p) + u_R - u_L = 0 (shock branch: Rankine-
    Hugoniot, rarefaction branch: isentropic), by Newton iteration from the
    two-rarefaction estimate; the waves are then sampled."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)

    def f(p, rk, pk, ck):
        if p > pk:  # shock
            A, B = 2.0 / ((g + 1.0) * rk), (g - 1.0) / (g + 1.0) * pk
            s = np.sqrt(A / (p + B))
            return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
        r = (p / pk) ** ((g - 1.0) / (2.0 * g))
        return 2.0 * ck / (g - 1.0) * (r - 1.0), 1.0 / (rk * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))

    z = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    for _ in range(100):
        fl, dl = f(p, rl, pl, cl)
        fr, dr = f(p, rr, pr, cr)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p = max(p - dp, 1e-14)
        if abs(dp) < 1e-15 * p:
            break
    fl, _ = f(p, rl, pl, cl)
    fr, _ = f(p, rr, pr, cr)
    us = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    gm = (g - 1.0) / (g + 1.0)
    out_r, out_u, out_p = np.empty_like(xi), np.empty_like(xi), np.empty_like(xi)
    for i, s in enumerate(np.asarray(xi, dtype=float)):
        if s <= us:  # left of the contact
            if p > pl:
                sl = ul - cl * np.sqrt((g + 1.0) / (2.0 * g) * p / pl + (g - 1.0) / (2.0 * g))
                v = (rl, ul, pl) if s <= sl else (rl * (p / pl + gm) / (gm * p / pl + 1.0), us, p)
            else:
                csl = cl * (p / pl) ** z
                if s <= ul - cl:
                    v = (rl, ul, pl)
                elif s >= us - csl:
                    v = (rl * (p / pl) ** (1.0 / g), us, p)
                else:
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    uu = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    v = (rl * (c / cl) ** (2.0 / (g - 1.0)), uu, pl * (c / cl) ** (2.0 * g / (g - 1.0)))
        else:  # right of the contact
            if p > pr:
                sr = ur + cr * np.sqrt((g + 1.0) / (2.0 * g) * p / pr + (g - 1.0) / (2.0 * g))
                v = (rr, ur, pr) if s >= sr else (rr * (p / pr + gm) / (gm * p / pr + 1.0), us, p)
            else:
                csr = cr * (p / pr) ** z
                if s >= ur + cr:
                    v = (rr, ur, pr)
                elif s <= us + csr:
                    v = (rr * (p / pr) ** (1.0 / g), us, p)
                else:
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    uu = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    v = (rr * (c / cr) ** (2.0 / (g - 1.0)), uu, pr * (c / cr) ** (2.0 * g / (g - 1.0)))
        out_r[i], out_u[i], out_p[i] = v
    return out_r, out_u, out_p


def _pad(u, axis, bc):
    """two ghost cells per side along axis: periodic wrap, Neumann even
    mirror, zero-Dirichlet odd mirror"""
    pw = [(0, 0)] * u.ndim
    pw[axis] = (2, 2)
    if bc == 0:
        return np.pad(u, pw, mode="wrap")
    g = np.pad(u, pw, mode="symmetric")
    if bc == 2:
        idx = [slice(None)] * u.ndim
        idx[axis] = slice(0, 2)
        g[tuple(idx)] *= -1.0
        idx[axis] = slice(-2, None)
        g[tuple(idx)] *= -1.0
    return g


def burgers_rhs_nd(u, h, bc):
    """-div F for u_t + sum_k (u^2/2)_{x_k} = 0 on a uniform grid of any
    dimension (array axes = directions), MUSCL-minmod + Godunov per direction,
    ghost cells per bc[axis]."""
    out = np.zeros_like(u)
    for ax in range(u.ndim):
        g = _pad(u, ax, bc[ax])
        n = u.shape[ax]

        def sl(a, b):
            idx = [slice(None)] * u.ndim
            idx[ax] = slice(a, b)
            return g[tuple(idx)]
        # faces f = 0..n between padded cells f+1 and f+2 (stencil f .. f+3)
        um, u0, u1, u2 = sl(0, n + 1), sl(1, n + 2), sl(2, n + 3), sl(3, n + 4)
        uL = u0 + 0.5 * _minmod(u0 - um, u1 - u0)
        uR = u1 - 0.5 * _minmod(u1 - u0, u2 - u1)
        fL, fR = 0.5 * uL ** 2, 0.5 * uR ** 2
        F = np.where(uL <= uR, np.where(uL > 0, fL, np.where(uR < 0, fR, 0.0)), np.maximum(fL, fR))
        idx_hi = [slice(None)] * u.ndim
        idx_lo = [slice(None)] * u.ndim
        idx_hi[ax] = slice(1, n + 1)
        idx_lo[ax] = slice(0, n)
        out -= (F[tuple(idx_hi)] - F[tuple(idx_lo)]) / h
    return out
