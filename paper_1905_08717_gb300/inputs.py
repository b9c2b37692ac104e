"""Seeded synthetic initial data shared by the CUDA path and the oracle.

This module only produces *inputs*: finest-level cell averages
(Sec. 2, definition of the cell average) of the analytic initial conditions
of the paper's test cases, plus the problem configurations that go with them.
It contains none of the multiresolution or time-stepping arithmetic.

Layout of every returned array: float64, shape (m, 2^L) in 1D,
(m, 2^L, 2^L) in 2D with index order [var, y, x] (x fastest in memory),
(m, 2^L, 2^L, 2^L) in 3D as [var, z, y, x].  Variables are conservative:
Burgers / advection / reaction-diffusion m = 1; Euler (rho, rho*u, rho*v[, rho*w], E).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

# equation ids (match the C-ABI enum)
EQ_ADVECTION = 0
EQ_BURGERS = 1
EQ_EULER = 2
EQ_REACTION_DIFFUSION = 3

BC_PERIODIC = 0
BC_NEUMANN = 1
BC_DIRICHLET0 = 2  # zero Dirichlet: odd-mirror ghost cells (scalar equations)

TIME_GTS = 0
TIME_LT = 1

ADAPT_NEVER = 0
ADAPT_MACRO = 1
ADAPT_EVERY = 2

FLUX_DEFAULT = 0
FLUX_AUSM_PLUS = 1

PREC_FP64 = 0
PREC_MIXED = 1   # FP32 state, fluxes and stage updates; registers and detail test FP64


@dataclass
class Problem:
    """A solver configuration (same fields as the C-ABI `mr_config`)."""

    dim: int
    equation: int
    max_level: int
    min_level: int
    eps: float
    eps_mode: int = 0          # 0 fixed, 1 level-scaled eps_l = 2^{d(l-L)} eps
    rk_order: int = 3
    time_mode: int = TIME_LT
    precision: int = 0
    adapt_mode: int = ADAPT_EVERY
    reflux: int = 1
    cfl: float = 0.5
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    bc: tuple = (BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)
    phys: tuple = (0.0,) * 8
    flux: int = 0              # 0 the equation's default flux, 1 AUSM+ (Euler)
    t_end: float = 0.0
    name: str = ""

    def nvars(self) -> int:
        return self.dim + 2 if self.equation == EQ_EULER else 1

    def replace(self, **kw) -> "Problem":
        d = asdict(self)
        d.update(kw)
        return Problem(**d)


# ---------------------------------------------------------------- quadrature
_GL4_X = np.array([-0.8611363115940526, -0.3399810435848563,
                   0.3399810435848563, 0.8611363115940526])
_GL4_W = np.array([0.3478548451374538, 0.6521451548625461,
                   0.6521451548625461, 0.3478548451374538])


def _cell_average_1d(fun, lo: float, hi: float, n: int) -> np.ndarray:
    """4-point Gauss-Legendre average of fun over each of n equal cells."""
    h = (hi - lo) / n
    centres = lo + (np.arange(n) + 0.5) * h
    acc = np.zeros(n)
    for xg, wg in zip(_GL4_X, _GL4_W):
        acc += 0.5 * wg * fun(centres + 0.5 * h * xg)
    return acc


def _cell_average_2d(fun, lo, hi, n: int, midpoint: bool = False) -> np.ndarray:
    """Tensor 4x4 Gauss-Legendre average over n x n cells, index [y, x]
    (midpoint: the value at the cell centre instead)."""
    hx = (hi[0] - lo[0]) / n
    hy = (hi[1] - lo[1]) / n
    cx = lo[0] + (np.arange(n) + 0.5) * hx
    cy = lo[1] + (np.arange(n) + 0.5) * hy
    if midpoint:
        return fun(cx[None, :], cy[:, None])
    acc = np.zeros((n, n))
    for xg, wx in zip(_GL4_X, _GL4_W):
        for yg, wy in zip(_GL4_X, _GL4_W):
            X = (cx + 0.5 * hx * xg)[None, :]
            Y = (cy + 0.5 * hy * yg)[:, None]
            acc += 0.25 * wx * wy * fun(X, Y)
    return acc


# ---------------------------------------------------------------- test cases
def burgers_1d(L: int = 10, eps: float = 1e-3, min_level: int = 2,
               rk_order: int = 3, time_mode: int = TIME_LT,
               t_end: float = 0.5) -> tuple[Problem, np.ndarray]:
    """1D inviscid Burgers, periodic [0,1], u0 = sin(2 pi x).

    Cell averages are exact: (cos 2 pi a - cos 2 pi b) / (2 pi h).
    """
    n = 1 << L
    h = 1.0 / n
    a = np.arange(n) * h
    b = a + h
    u = (np.cos(2 * np.pi * a) - np.cos(2 * np.pi * b)) / (2 * np.pi * h)
    p = Problem(dim=1, equation=EQ_BURGERS, max_level=L, min_level=min_level,
                eps=eps, eps_mode=1, rk_order=rk_order, time_mode=time_mode,
                cfl=0.5, bc=(BC_PERIODIC,) * 3, t_end=t_end,
                name=f"burgers1d_L{L}")
    return p, u[None, :].copy()


def burgers_2d(L: int = 7, eps: float = 1e-2, min_level: int = 2,
               rk_order: int = 3, time_mode: int = TIME_LT,
               t_end: float = 0.2, bc: int = BC_PERIODIC) -> tuple[Problem, np.ndarray]:
    """2D inviscid Burgers on [0,1]^2 with u0 = sin(2 pi x) sin(2 pi y), exact
    cell averages.  The paper's Sec. 5.1 case has u = 0 on the walls
    (bc=BC_DIRICHLET0, see burgers_2d_paper); periodic keeps mass exact."""
    n = 1 << L
    h = 1.0 / n
    a = np.arange(n) * h
    s = (np.cos(2 * np.pi * a) - np.cos(2 * np.pi * (a + h))) / (2 * np.pi * h)
    u = s[:, None] * s[None, :]
    p = Problem(dim=2, equation=EQ_BURGERS, max_level=L, min_level=min_level,
                eps=eps, eps_mode=0, rk_order=rk_order, time_mode=time_mode,
                cfl=0.5, bc=(bc,) * 3, t_end=t_end,
                name=f"burgers2d_L{L}")
    return p, u[None, :, :].copy()


def burgers_3d(L: int = 5, eps: float = 1e-2, min_level: int = 2, rk_order: int = 3,
               time_mode: int = TIME_LT, t_end: float = 0.1, bc: int = BC_PERIODIC) -> tuple[Problem, np.ndarray]:
    """3D inviscid Burgers u_t + sum_k (u^2/2)_{x_k} = 0 on [0,1]^3 with
    u0 = sin(2 pi x) sin(2 pi y) sin(2 pi z) (exact cell averages)."""
    n = 1 << L
    h = 1.0 / n
    a = np.arange(n) * h
    s = (np.cos(2 * np.pi * a) - np.cos(2 * np.pi * (a + h))) / (2 * np.pi * h)
    u = s[:, None, None] * s[None, :, None] * s[None, None, :]
    p = Problem(dim=3, equation=EQ_BURGERS, max_level=L, min_level=min_level, eps=eps, eps_mode=0,
                rk_order=rk_order, time_mode=time_mode, cfl=0.5, bc=(bc,) * 3, t_end=t_end,
                name=f"burgers3d_L{L}")
    return p, u[None].copy()


def burgers_2d_paper(L: int = 10, eps: float = 1e-3, min_level: int = 3, rk_order: int = 2,
                     time_mode: int = TIME_LT, t_end: float = 0.9) -> tuple[Problem, np.ndarray]:
    """The paper's 2D Burgers case (Sec. 5.1): sin(2 pi x) sin(2 pi y) on
    [0,1]^2, u = 0 on the walls, to t = 0.9 (its figure's final time), CFL 0.5.
    The paper's flux there is AUSM+; this build uses MUSCL-minmod + Godunov for
    Burgers."""
    p, q = burgers_2d(L=L, eps=eps, min_level=min_level, rk_order=rk_order,
                      time_mode=time_mode, t_end=t_end, bc=BC_DIRICHLET0)
    return p.replace(name=f"burgers2d_paper_L{L}"), q


# Lax-Liu configuration 6 (Table 8): quadrants 1..4 = [.5,1]x[.5,1], [0,.5]x[.5,1],
# [0,.5]x[0,.5], [.5,1]x[0,.5]; rows rho, p, u, v.
_LAXLIU6 = np.array([[1.00, 2.00, 1.00, 3.00],
                     [1.00, 1.00, 1.00, 1.00],
                     [0.75, 0.75, -0.75, -0.75],
                     [-0.50, 0.50, 0.50, -0.50]])


def quadrant_states(seed: int) -> np.ndarray:
    """(4 quadrants) x (rho, p, u, v).  seed 0 = the paper's Table 8 states."""
    if seed == 0:
        return _LAXLIU6.T.copy()
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 3.0, 4)
    pr = rng.uniform(0.5, 2.0, 4)
    u = rng.uniform(-0.75, 0.75, 4)
    v = rng.uniform(-0.75, 0.75, 4)
    return np.stack([rho, pr, u, v], axis=1)


def euler_2d_quadrants(L: int = 10, eps: float = 1e-3, seed: int = 0,
                       min_level: int = 3, rk_order: int = 3,
                       time_mode: int = TIME_LT, gamma: float = 1.4,
                       t_end: float = 0.25) -> tuple[Problem, np.ndarray]:
    """2D Euler four-quadrant Riemann problem on [0,1]^2, homogeneous Neumann.

    The quadrant interfaces x = 1/2, y = 1/2 are cell faces on every level >= 1,
    so the cell averages are the quadrant states exactly.
    """
    n = 1 << L
    st = quadrant_states(seed)
    xc = (np.arange(n) + 0.5) / n
    right = xc[None, :] > 0.5
    top = xc[:, None] > 0.5
    quad = np.where(top & right, 0, np.where(top & ~right, 1,
                    np.where(~top & ~right, 2, 3)))
    rho = st[quad, 0]
    pr = st[quad, 1]
    u = st[quad, 2]
    v = st[quad, 3]
    q = np.empty((4, n, n))
    q[0] = rho
    q[1] = rho * u
    q[2] = rho * v
    q[3] = pr / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    ph = (gamma,) + (0.0,) * 7
    p = Problem(dim=2, equation=EQ_EULER, max_level=L, min_level=min_level,
                eps=eps, eps_mode=0, rk_order=rk_order, time_mode=time_mode,
                cfl=0.5, bc=(BC_NEUMANN,) * 3, phys=ph, t_end=t_end,
                name=f"euler2d_quadrants_L{L}_seed{seed}")
    return p, q


def euler_1d_sod(L: int = 8, eps: float = 1e-3, min_level: int = 2,
                 rk_order: int = 3, time_mode: int = TIME_LT,
                 gamma: float = 1.4, t_end: float = 0.15) -> tuple[Problem, np.ndarray]:
    """1D Euler shock tube (rho,p,u) = (1,1,0) | (0.125,0.1,0) at x = 1/2, Neumann."""
    n = 1 << L
    xc = (np.arange(n) + 0.5) / n
    left = xc < 0.5
    rho = np.where(left, 1.0, 0.125)
    pr = np.where(left, 1.0, 0.1)
    q = np.empty((3, n))
    q[0] = rho
    q[1] = 0.0
    q[2] = pr / (gamma - 1.0)
    ph = (gamma,) + (0.0,) * 7
    p = Problem(dim=1, equation=EQ_EULER, max_level=L, min_level=min_level,
                eps=eps, eps_mode=0, rk_order=rk_order, time_mode=time_mode,
                cfl=0.5, bc=(BC_NEUMANN,) * 3, phys=ph, t_end=t_end,
                name=f"euler1d_sod_L{L}")
    return p, q


def euler_3d_blast(L: int = 8, eps: float = 1e-3, min_level: int = 3,
                   rk_order: int = 3, time_mode: int = TIME_LT,
                   precision: int = 1, gamma: float = 1.4, r0: float = 0.1,
                   p_in: float = 10.0, t_end: float = 0.1) -> tuple[Problem, np.ndarray]:
    """3D Euler blast on [0,1]^3, homogeneous Neumann: rho = 1, u = 0, p = 1,
    p = p_in inside the ball of radius r0 about the centre.  Cell averages of
    p are exact away from the sphere; cells the sphere cuts use the fraction
    of 4x4x4 midpoint sub-samples inside it."""
    n = 1 << L
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    d2 = ((c[None, None, :] - 0.5) ** 2 + (c[None, :, None] - 0.5) ** 2
          + (c[:, None, None] - 0.5) ** 2)
    half_diag = 0.5 * math.sqrt(3.0) * h
    r = np.sqrt(d2)
    frac = (r + half_diag <= r0).astype(np.float64)
    cut = np.argwhere((r - half_diag < r0) & (r + half_diag > r0))
    if len(cut):
        o = (np.arange(4) + 0.5) / 4 - 0.5
        OZ, OY, OX = (a.ravel()[None, :] for a in np.meshgrid(o, o, o, indexing="ij"))
        z, y, x = cut[:, 0:1], cut[:, 1:2], cut[:, 2:3]
        px = c[x] + OX * h - 0.5
        py = c[y] + OY * h - 0.5
        pz = c[z] + OZ * h - 0.5
        frac[cut[:, 0], cut[:, 1], cut[:, 2]] = np.mean(px * px + py * py + pz * pz < r0 * r0, axis=1)
    pr = 1.0 + (p_in - 1.0) * frac
    q = np.zeros((5, n, n, n))
    q[0] = 1.0
    q[4] = pr / (gamma - 1.0)
    ph = (gamma,) + (0.0,) * 7
    p = Problem(dim=3, equation=EQ_EULER, max_level=L, min_level=min_level,
                eps=eps, eps_mode=0, rk_order=rk_order, time_mode=time_mode,
                precision=precision, cfl=0.5, bc=(BC_NEUMANN,) * 3, phys=ph,
                t_end=t_end, name=f"euler3d_blast_L{L}")
    return p, q


def rd_bumps_2d(L: int = 8, eps: float = 1e-3, seed: int = 0,
                min_level: int = 3, rk_order: int = 2,
                time_mode: int = TIME_LT, D: float = 1e-3, k: float = 100.0,
                a: float = 0.3, t_end: float = 0.2, midpoint: bool = False) -> tuple[Problem, np.ndarray]:
    """2D bistable reaction-diffusion u_t = D lap u + k u(1-u)(u-a), Neumann,
    1..8 Gaussian bumps (centre U[.15,.85]^2, width U[.02,.06], amplitude 1),
    combined by max; cell averages by 4x4 Gauss-Legendre (midpoint: centre
    values, a cheaper input for large request streams)."""
    rng = np.random.default_rng(seed)
    nb = int(rng.integers(1, 9))
    cen = rng.uniform(0.15, 0.85, (nb, 2))
    wid = rng.uniform(0.02, 0.06, nb)

    def fun(X, Y):
        out = np.zeros(np.broadcast(X, Y).shape)
        for (cx, cy), w in zip(cen, wid):
            out = np.maximum(out, np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * w * w)))
        return out

    u = _cell_average_2d(fun, (0.0, 0.0), (1.0, 1.0), 1 << L, midpoint=midpoint)
    ph = (D, k, a) + (0.0,) * 5
    p = Problem(dim=2, equation=EQ_REACTION_DIFFUSION, max_level=L,
                min_level=min_level, eps=eps, eps_mode=0, rk_order=rk_order,
                time_mode=time_mode, cfl=0.5, bc=(BC_NEUMANN,) * 3, phys=ph,
                t_end=t_end, name=f"rd2d_L{L}_seed{seed}")
    return p, u[None, :, :].copy()


def rd_batch(n: int = 256, seed: int = 0, levels: tuple = (7, 10), eps_choices: tuple = (1e-3, 1e-4),
             t_end: float = 0.2) -> tuple[list, list]:
    """n independent 2D reaction-diffusion problems of uneven size: instance i
    has its own bumps (seed + i), finest level L ~ U{levels}, eps drawn from
    eps_choices, RK2 with LT/NERK, Neumann walls."""
    rng = np.random.default_rng(seed)
    Ls = rng.integers(levels[0], levels[1] + 1, n)
    es = rng.choice(np.asarray(eps_choices, dtype=np.float64), n)
    probs, qs = [], []
    for i in range(n):
        p, q = rd_bumps_2d(L=int(Ls[i]), eps=float(es[i]), seed=seed + i, t_end=t_end)
        probs.append(p.replace(name=f"rd2d_L{int(Ls[i])}_seed{seed + i}"))
        qs.append(q)
    return probs, qs


def serving_requests(n: int = 300, seed: int = 0, rate: float = 200.0) -> list:
    """A seeded stream of n requests arriving as a Poisson process of the given
    rate (per second): (arrival_s, problem, q0, t_end).  Kinds, equally
    likely: 1D Burgers (L ~ U{10..14}), 2D reaction-diffusion (L ~ U{8..10}),
    3D Euler blast (L ~ U{6..8}); eps ~ log-uniform [1e-4, 1e-2]; mixed
    precision; the coarsest level keeps a macro step at 2^7 fine steps or
    fewer.  t_end is set from a target of fine iterations at the initial CFL
    step, so that request sizes stay bounded."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    cache = {}  # Burgers and blast data depend on L only
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        kind = int(rng.integers(0, 3))
        eps = float(10.0 ** rng.uniform(-4.0, -2.0))
        if kind == 0:
            L = int(rng.integers(10, 15))
            if ("b", L) not in cache:
                cache[("b", L)] = burgers_1d(L=L, eps=eps, min_level=L - 7)
            p, q = cache[("b", L)]
            p = p.replace(eps=eps)
            its = int(rng.integers(32, 129))
            t_end = its * 0.5 / (1 << L)            # speed max |u| = 1
        elif kind == 1:
            L = int(rng.integers(8, 11))
            p, q = rd_bumps_2d(L=L, eps=eps, seed=seed + i, rk_order=2, midpoint=True)
            its = int(rng.integers(16, 65))
            dx = 1.0 / (1 << L)
            t_end = its * 0.5 * dx * dx / (4.0 * p.phys[0])  # diffusion limit
        else:
            L = int(rng.integers(6, 9))
            if ("e", L) not in cache:
                cache[("e", L)] = euler_3d_blast(L=L, eps=eps, min_level=L - 4)
            p, q = cache[("e", L)]
            p = p.replace(eps=eps)
            its = int(rng.integers(8, 25))
            t_end = its * 0.5 / (1 << L) / 4.0      # speed ~ 3.74
        p = p.replace(precision=PREC_MIXED, name=f"req{i}_{p.name}")
        out.append((t, p, q, float(t_end)))
    return out


def advection_gaussian_1d(L: int = 9, a: float = 1.0, rk_order: int = 3,
                          time_mode: int = TIME_LT,
                          t_end: float = 1.0) -> tuple[Problem, np.ndarray]:
    """Sec. 4.5 convergence case: q_t + q_x = 0 on periodic [0,1],
    q0 = exp(-100 (x - 1/4)^2), centred flux, no adaptation (fixed tree)."""
    u = _cell_average_1d(lambda x: np.exp(-100.0 * (x - 0.25) ** 2), 0.0, 1.0, 1 << L)
    ph = (a, 0.0, 0.0) + (0.0,) * 5
    p = Problem(dim=1, equation=EQ_ADVECTION, max_level=L, min_level=max(L - 3, 0),
                eps=0.0, eps_mode=0, rk_order=rk_order, time_mode=time_mode,
                adapt_mode=ADAPT_NEVER, cfl=0.5, bc=(BC_PERIODIC,) * 3,
                phys=ph, t_end=t_end, name=f"advection1d_L{L}")
    return p, u[None, :].copy()


def two_level_map_1d(L: int) -> np.ndarray:
    """Leaf level of every finest cell for the Sec. 4.5 fixed grid:
    level L on [0, 1/2), level L-1 on [1/2, 1)."""
    n = 1 << L
    m = np.full(n, L - 1, dtype=np.uint8)
    m[: n // 2] = L
    return m


def random_smooth_1d(L: int, seed: int) -> np.ndarray:
    """Smooth periodic random field (a few Fourier modes) for MR-operator tests."""
    rng = np.random.default_rng(seed)
    k = np.arange(1, 6)
    amp = rng.normal(size=5) / k ** 2
    ph = rng.uniform(0, 2 * np.pi, 5)
    n = 1 << L
    h = 1.0 / n
    a = np.arange(n) * h
    out = np.zeros(n)
    for kk, aa, pp in zip(k, amp, ph):
        w = 2 * np.pi * kk
        out += aa * (np.sin(w * (a + h) + pp) - np.sin(w * a + pp)) / (w * h)
    return out
