"""Seeded synthetic NMPC instances (inputs only; none of the method's arithmetic).

This module is the one piece shared by the CUDA path, its tests, the bench
and the oracle's callers.  It draws numbers and lays out instance
descriptions; it never evaluates the model, the KKT map or any solver step.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds.  Doubles in [0, 1) take the top 53 bits;
normals use the Box-Muller transform.

Workload shapes follow the heat-transfer problems the method is evaluated on
(Sec. 5 of the paper uses a 2D plate; the instances here are 1D/2D nonlinear
heat equations with point heat-source actuators):

* ``heat1d_single``  1D, M=32, dt=1e-4, N=20, actuators at x=0.25, 0.75
* ``heat2d_single``  2D 64x64, dt=2e-5, N=50, 8 actuators on a 2x4 grid
* ``heat1d_ragged_batch``  1024 1D instances with M, N, n_u, R drawn per seed
* ``heat2d_large_batch``   64 2D 256x256 instances, N=100, 16 actuators

Grid convention: interior cells only (Dirichlet-zero ring outside), cell
(iy, ix) at coordinates ((ix+1)/(mx+1), (iy+1)/(my+1)), stored row-major,
flat index iy*mx + ix.  A "point actuator at p" acts on the interior cell
nearest to p (ties to the lower index) as a heat source: that cell's
temperature equation gains ``act_gain * u_a``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First ``n`` outputs of SplitMix64 started from state ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """``n`` doubles in [0, 1) from the top 53 bits of SplitMix64(seed)."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int) -> np.ndarray:
    """``n`` standard normals by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


@dataclasses.dataclass
class Instance:
    """One NMPC instance: grid, horizon, actuators, weights, x0 and reference.

    ``x0`` and ``ref`` are flat (my*mx,) float64 arrays on the interior grid.
    ``act`` holds flat cell indices of the actuator (heat source) cells and
    ``act_gain`` the heating rate of such a cell per unit input.
    Diffusivity k(w) = k0 * (1 + k1 * w).  Weights: stage cost
    h/2 (q |x - ref|^2 + r |u|^2), terminal cost h/2 qf |x_N - ref|^2.
    """

    dim: int
    mx: int
    my: int
    horizon: int
    h: float
    act: np.ndarray
    q: float
    r: float
    qf: float
    gamma: float
    k0: float
    k1: float
    x0: np.ndarray
    ref: np.ndarray
    act_gain: float = 32.0
    name: str = ""

    @property
    def ng(self) -> int:
        return self.mx * self.my

    @property
    def n_u(self) -> int:
        return int(len(self.act))


def nearest_cell(p: float, m: int) -> int:
    """0-based interior cell nearest to coordinate p on m cells of [0,1]."""
    # cell j (0-based) sits at (j+1)/(m+1); ties go to the lower index
    t = p * (m + 1) - 1.0
    j = int(math.floor(t))
    if t - j > 0.5:
        j += 1
    return min(max(j, 0), m - 1)


def _coords_1d(m: int) -> np.ndarray:
    return np.arange(1, m + 1, dtype=np.float64) / (m + 1)


def _sine_field(mx: int, my: int, seed: int, modes: int = 4, std: float = 0.1) -> np.ndarray:
    a = normal(seed, modes * modes).reshape(modes, modes) * std
    xs, ys = _coords_1d(mx), _coords_1d(my)
    f = np.zeros((my, mx))
    for p in range(1, modes + 1):
        sx = np.sin(p * np.pi * xs)
        for q in range(1, modes + 1):
            f += a[p - 1, q - 1] * np.outer(np.sin(q * np.pi * ys), sx)
    return f.reshape(-1)


def _gauss_bump(mx: int, my: int, cx: float = 0.5, cy: float = 0.5,
                amp: float = 1.0, width: float = 0.15) -> np.ndarray:
    xs, ys = _coords_1d(mx), _coords_1d(my)
    d2 = (xs[None, :] - cx) ** 2 + (ys[:, None] - cy) ** 2
    return (amp * np.exp(-d2 / (2.0 * width * width))).reshape(-1)


def _act_grid(mx: int, my: int, nx_act: int, ny_act: int) -> np.ndarray:
    cells = []
    for r in range(ny_act):
        iy = nearest_cell((r + 0.5) / ny_act, my)
        for c in range(nx_act):
            ix = nearest_cell((c + 0.5) / nx_act, mx)
            cells.append(iy * mx + ix)
    return np.asarray(cells, dtype=np.int32)


def default_gamma(h: float, r: float) -> float:
    """Regularization weight used when a workload does not fix one: gamma = h R,
    the ratio of the paper's experiment (gamma = 0.5 with h = 5 s, R = 0.1)."""
    return h * r


def heat1d(m: int, horizon: int, n_u: int, r: float, seed: int, h: float = 1e-4,
           act_pos: Optional[List[float]] = None, gamma: Optional[float] = None,
           k1: float = 0.5, name: str = "") -> Instance:
    """1D instance: x0 ~ U[0,1] per cell (SplitMix64(seed)), ref 0.8 sin(pi x)."""
    if act_pos is None:
        act_pos = [(a + 0.5) / n_u for a in range(n_u)]
    act = np.asarray([nearest_cell(p, m) for p in act_pos], dtype=np.int32)
    x0 = uniform01(seed, m)
    ref = 0.8 * np.sin(np.pi * _coords_1d(m))
    return Instance(dim=1, mx=m, my=1, horizon=horizon, h=h, act=act, q=1.0, r=r,
                    qf=10.0, gamma=default_gamma(h, r) if gamma is None else gamma,
                    k0=0.1, k1=k1, x0=x0, ref=ref, name=name)


def heat2d(mx: int, my: int, horizon: int, nx_act: int, ny_act: int, seed: int,
           h: float = 2e-5, r: float = 0.01, gamma: Optional[float] = None,
           ref_center=(0.5, 0.5), ref_amp: float = 1.0, k1: float = 0.5,
           name: str = "") -> Instance:
    """2D instance: 16-mode sine initial field (a_pq ~ N(0, 0.1^2), seed),
    Gaussian-bump reference (sigma 0.15), actuators on a regular grid."""
    act = _act_grid(mx, my, nx_act, ny_act)
    x0 = _sine_field(mx, my, seed)
    ref = _gauss_bump(mx, my, ref_center[0], ref_center[1], ref_amp)
    return Instance(dim=2, mx=mx, my=my, horizon=horizon, h=h, act=act, q=1.0, r=r,
                    qf=10.0, gamma=default_gamma(h, r) if gamma is None else gamma,
                    k0=0.1, k1=k1, x0=x0, ref=ref, name=name)


def heat1d_single() -> Instance:
    """1D, M=32, dt=1e-4, N=20, actuators at x=0.25 and 0.75, x0 ~ U[0,1] seed 0."""
    return heat1d(32, 20, 2, 0.01, seed=0, act_pos=[0.25, 0.75], name="heat1d_M32_N20")


def heat2d_single(seed: int = 1) -> Instance:
    """2D 64x64, dt=2e-5, N=50, 8 actuators (2 rows x 4 columns), seed 1."""
    return heat2d(64, 64, 50, 4, 2, seed=seed, name="heat2d_64x64_N50")


def heat1d_ragged_batch(n: int = 1024, base_seed: int = 3000) -> List[Instance]:
    """Ragged 1D batch: instance b uses seed base_seed+b to draw
    M ~ U{32..256}, N ~ U{10..60}, n_u ~ U{1..4}, R = 10^U[-3,-1];
    its x0 comes from seed (base_seed+b) << 20."""
    out = []
    for b in range(n):
        s = base_seed + b
        d = uniform01(s, 4)
        m = 32 + int(d[0] * 225)
        horizon = 10 + int(d[1] * 51)
        n_u = 1 + int(d[2] * 4)
        r = 10.0 ** (-3.0 + 2.0 * d[3])
        out.append(heat1d(m, horizon, n_u, r, seed=s << 20, name=f"heat1d_b{b}"))
    return out


def heat2d_large_batch(n: int = 64, base_seed: int = 5000, m: int = 256,
                       horizon: int = 100) -> List[Instance]:
    """Large 2D batch: 256x256, N=100, 16 actuators (4x4), dt=2e-5; instance b
    has sine initial field seed base_seed+b and a bump reference whose centre
    ~ U[0.3,0.7]^2 and amplitude ~ U[0.5,1.5] come from seed base_seed+b+10^6."""
    out = []
    for b in range(n):
        d = uniform01(base_seed + b + 1_000_000, 3)
        out.append(heat2d(m, m, horizon, 4, 4, seed=base_seed + b,
                          ref_center=(0.3 + 0.4 * d[0], 0.3 + 0.4 * d[1]),
                          ref_amp=0.5 + d[2], name=f"heat2d_{m}_b{b}"))
    return out


def tiny1d(m: int = 8, horizon: int = 4, n_u: int = 1, seed: int = 7, h: float = 1e-3,
           k1: float = 0.5, gamma: Optional[float] = None) -> Instance:
    """Small 1D instance for dense cross-checks (Newton, full KKT LU, Riccati)."""
    return heat1d(m, horizon, n_u, 0.01, seed=seed, h=h, k1=k1, gamma=gamma,
                  name=f"tiny1d_M{m}_N{horizon}")


def tiny2d(mx: int = 6, my: int = 6, horizon: int = 3, seed: int = 11, h: float = 1e-3,
           k1: float = 0.5, gamma: Optional[float] = None) -> Instance:
    """Small 2D instance (2x2 actuators) for dense cross-checks."""
    return heat2d(mx, my, horizon, 2, 2, seed=seed, h=h, k1=k1, gamma=gamma,
                  name=f"tiny2d_{mx}x{my}_N{horizon}")


def heat2d_learning_instance(seed: int) -> Instance:
    """The 2D 64x64, N=50 problem with a seeded smooth initial field (seed) and
    a Gaussian-bump reference whose centre ~ U[0.3, 0.7]^2 and amplitude ~
    U[0.5, 1.5] come from seed + 77_777_777 (training and test sets of the
    learned warm start use disjoint seed ranges)."""
    d = uniform01(seed + 77_777_777, 3)
    return heat2d(64, 64, 50, 4, 2, seed=seed, ref_center=(0.3 + 0.4 * d[0], 0.3 + 0.4 * d[1]),
                  ref_amp=0.5 + d[2], name=f"heat2d_learn_{seed}")


# ---------------------------------------------------------------------------
# Pinned-actuator problems: the copper plate of the paper's experiment
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class PlateInstance:
    """A pinned-actuator instance: the temperatures of the grid points in
    ``act`` are the inputs (they are not states).  ``x0`` and ``x_ref`` hold
    the state points (grid order, actuator points left out), ``u_ref`` the
    actuator points.  Model w_t = Lap(k0 (w + k1 w^2 / 2)) - beta (w - t_amb)
    - gamma_r (w^4 - t_amb^4); bounds u_lo <= u <= u_hi with barrier weight
    tau (0: no bounds)."""

    dim: int
    m: int
    bc: str
    horizon: int
    h: float
    act: np.ndarray
    k0: float
    k1: float
    beta: float
    t_amb: float
    gamma_r: float
    q: float
    r: float
    qf: float
    gamma: float
    tau: float
    u_lo: float
    u_hi: float
    x0: np.ndarray
    x_ref: np.ndarray
    u_ref: np.ndarray
    name: str = ""

    @property
    def ng(self) -> int:
        return self.m ** self.dim

    @property
    def ns(self) -> int:
        return self.ng - len(self.act)


# Table 1 of the paper (copper plate) and Table 2 (NMPC settings)
PLATE_RHO, PLATE_CP, PLATE_TZ, PLATE_K = 8960.0, 386.0, 0.01, 400.0
PLATE_HC, PLATE_TA, PLATE_EPS, PLATE_SIGMA = 1.0, 300.0, 0.5, 5.67e-8


def plate_reference(m: int, shape: str, t_amb: float = PLATE_TA) -> np.ndarray:
    """Stand-ins for the paper's reference fields (its figure is not
    available): "slope", t_amb + 50 + 300 x, and "V", t_amb + 50 + 300 |2x - 1|,
    over the m x m grid points of [0, 1]^2 (x the horizontal axis)."""
    xs = np.linspace(0.0, 1.0, m)
    prof = xs if shape == "slope" else np.abs(2.0 * xs - 1.0)
    field = np.tile(t_amb + 50.0 + 300.0 * prof, (m, 1))
    return field.reshape(-1)


def plate_instance(m: int = 13, horizon: int = 20, T: float = 100.0, shape: str = "slope",
                   x0_field: Optional[np.ndarray] = None, act_idx=(1, 4, 8, 11),
                   tau: float = 100.0, gamma: float = 0.5, name: str = "") -> PlateInstance:
    """The paper's plate: m x m points with zero-Neumann boundaries, actuators
    at the grid points act_idx x act_idx (16 for the default 13 x 13 grid:
    169 - 16 = 153 states), inputs in [t_amb, t_amb + 400] K, T = 100 s,
    N = 20 (h = 5 s), Q = I, R = 0.1 I, tau = 100, gamma = 0.5; the state
    starts at the ambient temperature unless x0_field (m x m) is given."""
    rc = PLATE_RHO * PLATE_CP
    if not all(0 <= a < m for a in act_idx):
        raise ValueError("actuator indices outside the grid")
    act = np.asarray([iy * m + ix for iy in act_idx for ix in act_idx], dtype=np.int32)
    is_act = np.zeros(m * m, dtype=bool)
    is_act[act] = True
    full_ref = plate_reference(m, shape)
    full_x0 = np.full(m * m, PLATE_TA) if x0_field is None else np.asarray(x0_field, float)
    return PlateInstance(dim=2, m=m, bc="neumann", horizon=horizon, h=T / horizon, act=act,
                         k0=PLATE_K / rc, k1=0.0, beta=2.0 * PLATE_HC / (rc * PLATE_TZ),
                         t_amb=PLATE_TA, gamma_r=2.0 * PLATE_EPS * PLATE_SIGMA / (rc * PLATE_TZ),
                         q=1.0, r=0.1, qf=0.0, gamma=gamma, tau=tau, u_lo=PLATE_TA,
                         u_hi=PLATE_TA + 400.0, x0=full_x0[~is_act].copy(),
                         x_ref=full_ref[~is_act].copy(), u_ref=full_ref[is_act].copy(),
                         name=name or f"plate_{m}x{m}_N{horizon}_{shape}")


def plate_batch(n: int, base_seed: int = 9000, m: int = 13, horizon: int = 20,
                act_idx=(1, 4, 8, 11)) -> List[PlateInstance]:
    """n plates whose initial temperature fields are t_amb plus a seeded smooth
    perturbation (16 cosine modes, amplitudes N(0, 10^2) K) and whose
    reference is the slope or the V field (alternating)."""
    out = []
    xs = np.linspace(0.0, 1.0, m)
    for b in range(n):
        a = normal(base_seed + b, 16).reshape(4, 4) * 10.0
        f = np.full((m, m), PLATE_TA)
        for p_ in range(4):
            for q_ in range(4):
                f += a[p_, q_] * np.outer(np.cos(q_ * np.pi * xs), np.cos(p_ * np.pi * xs))
        out.append(plate_instance(m, horizon, shape="slope" if b % 2 == 0 else "V",
                                  x0_field=f.reshape(-1), act_idx=act_idx, name=f"plate_b{b}"))
    return out


def pinned_heat1d(m: int = 32, horizon: int = 20, h: float = 1e-4, seed: int = 0,
                  act_pos=(0.25, 0.75), r: float = 0.01,
                  gamma: Optional[float] = None) -> PlateInstance:
    """The 1D heat workload (M = 32 interior cells, Dirichlet ring, k(w) =
    0.1 (1 + 0.5 w), N = 20, h = 1e-4, reference 0.8 sin(pi x), R = 0.01,
    terminal weight 10) with the other reading of its actuators: the cells
    nearest x = 0.25 and 0.75 pinned to the inputs (no bounds)."""
    act = np.asarray([nearest_cell(p_, m) for p_ in act_pos], dtype=np.int32)
    is_act = np.zeros(m, dtype=bool)
    is_act[act] = True
    x0 = uniform01(seed, m)
    ref = 0.8 * np.sin(np.pi * _coords_1d(m))
    return PlateInstance(dim=1, m=m, bc="dirichlet", horizon=horizon, h=h, act=act, k0=0.1,
                         k1=0.5, beta=0.0, t_amb=0.0, gamma_r=0.0, q=1.0, r=r, qf=10.0,
                         gamma=default_gamma(h, r) if gamma is None else gamma, tau=0.0,
                         u_lo=-np.inf, u_hi=np.inf, x0=x0[~is_act].copy(),
                         x_ref=ref[~is_act].copy(), u_ref=np.zeros(len(act)),
                         name="pinned_heat1d_M32_N20")


@dataclasses.dataclass
class WaveInstance:
    """A second-order-in-time instance: a w_tt + b w_t = c Lap w - kappa w^3
    + sum_a gain u_a delta_a on a grid of m (dim 1) or m x m (dim 2) points,
    point forces at the cells ``act``.  ``x0`` holds the initial (W, V) with
    V = dW/dt (all W first), ``w_ref`` the displacement reference, ``u_ref``
    the input reference."""

    dim: int
    m: int
    bc: str
    horizon: int
    h: float
    act: np.ndarray
    a: float
    b: float
    c: float
    kappa: float
    gain: float
    q: float
    qv: float
    r: float
    qf: float
    gamma: float
    x0: np.ndarray
    w_ref: np.ndarray
    u_ref: np.ndarray
    name: str = ""

    @property
    def ng(self) -> int:
        return self.m ** self.dim


def wave_instance(dim: int = 1, m: int = 64, horizon: int = 20, T: float = 0.06, seed: int = 0,
                  n_act: int = 2, a: float = 1.0, b: float = 1.0, c: float = 1.0,
                  kappa: float = 10.0, gain: float = 10.0, r: float = 1e-2, qv: float = 0.1, qf: float = 10.0,
                  gamma: Optional[float] = None, bc: str = "dirichlet",
                  name: str = "") -> WaveInstance:
    """A damped string (dim 1) or membrane (dim 2) with a cubic stiffening
    term, interior grid, zero Dirichlet ring (``bc="neumann"``: free edges,
    boundary points included).  Actuators: n_act (1D) or n_act x n_act (2D)
    point forces at the cells nearest the centres (k + 1/2) / n_act, force
    ``gain`` per unit input on the cell.  gamma defaults to h r (the ratio of
    the paper's experiment).  Initial displacement a
    smooth random field (4 sine modes per axis, std 0.1) at rest; reference a
    Gaussian bump of height 0.2 and width 0.15 in the middle."""
    coords = _coords_1d(m) if bc == "dirichlet" else np.linspace(0.0, 1.0, m)
    near = lambda p_: int(np.argmin(np.abs(coords - p_)))
    cents = [(k + 0.5) / n_act for k in range(n_act)]
    if dim == 1:
        act = np.asarray([near(p_) for p_ in cents], dtype=np.int32)
        W0 = np.zeros(m)
        a_ = normal(seed, 4) * 0.1
        for k in range(4):
            W0 += a_[k] * np.sin((k + 1) * np.pi * coords)
        ref = 0.2 * np.exp(-(coords - 0.5) ** 2 / (2 * 0.15 ** 2))
    else:
        act = np.asarray([near(py) * m + near(px) for py in cents for px in cents], dtype=np.int32)
        a_ = normal(seed, 16).reshape(4, 4) * 0.1
        W0 = np.zeros((m, m))
        for p_ in range(4):
            for q_ in range(4):
                W0 += a_[p_, q_] * np.outer(np.sin((q_ + 1) * np.pi * coords),
                                            np.sin((p_ + 1) * np.pi * coords))
        W0 = W0.reshape(-1)
        d2 = (coords[None, :] - 0.5) ** 2 + (coords[:, None] - 0.5) ** 2
        ref = (0.2 * np.exp(-d2 / (2 * 0.15 ** 2))).reshape(-1)
    if len(set(act.tolist())) != len(act):
        raise ValueError("two actuators on one cell")
    h = T / horizon
    return WaveInstance(dim=dim, m=m, bc=bc, horizon=horizon, h=h, act=act, a=a, b=b, c=c,
                        kappa=kappa, gain=gain, q=1.0, qv=qv, r=r, qf=qf,
                        gamma=default_gamma(h, r) if gamma is None else gamma,
                        x0=np.concatenate([W0, np.zeros_like(W0)]), w_ref=ref,
                        u_ref=np.zeros(len(act)),
                        name=name or f"wave{dim}d_m{m}_N{horizon}_s{seed}")
