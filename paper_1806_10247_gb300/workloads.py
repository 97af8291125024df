"""Seeded synthetic workloads shaped like the paper's benchmark problems.

This module only draws parameters and tabulates input shapes (numpy, on the
host).  It holds none of the lattice Boltzmann arithmetic, so both the CUDA
path and the CPU oracle can take their inputs from it.

Conventions shared with the library: lattice units (dx = dt = 1); a force or
source is F(x, t) = a(t) * P(x) with a separable shape
P_c(x, y, z) = (px_c[x] * py_c[y]) * pz_c[z], each table of length 1 (constant
along that axis) or the axis extent; shear relaxation omega = 1/tau with
nu = (tau - 1/2)/3 (Sec. 6 preamble); diffusivity D = (tau_phi - 1/2)/3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

D2Q9, D3Q27, D2Q5, D3Q15 = 1, 2, 3, 4
SEED = 10247


def tau_from_nu(nu: float) -> float:
    return 3.0 * nu + 0.5


@dataclass
class Workload:
    """One lattice problem: geometry, relaxation, initial state and forcing."""

    name: str
    lattice: int
    shape: tuple                      # (nx, ny, nz)
    wall: tuple                       # per axis: 1 = halfway bounce-back walls
    omega: tuple                      # 9 relaxation rates, numbered as in the library header
    rho0: np.ndarray | float = 1.0    # initial density (flow) or scalar (D2Q5)
    u0: np.ndarray | tuple = (0.0, 0.0, 0.0)  # initial velocity (flow) or advecting velocity (D2Q5)
    tables: list | None = None        # per component (px, py, pz)
    envelope: object = None           # a(t), or None for a == 1
    steps: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return int(self.shape[0] * self.shape[1] * self.shape[2])


def d2q9_omega(tau: float, w3: float = 1.0, w6: float = 1.0, w7: float = 1.0, w8: float = 1.0):
    """omega_3..omega_8 of Eq. 23 at their array positions 3..8 (Sec. 6: omega_4 = omega_5 = 1/tau)."""
    return (0.0, 0.0, 0.0, w3, 1.0 / tau, 1.0 / tau, w6, w7, w8)


def d2q5_omega(tau_phi: float, w3: float = 1.0, w4: float = 1.0):
    """omega_1^phi..omega_4^phi of Eq. 41 at positions 1..4 (omega_1 = omega_2 = 1/tau_phi)."""
    return (0.0, 1.0 / tau_phi, 1.0 / tau_phi, w3, w4, 0.0, 0.0, 0.0, 0.0)


def d3q27_omega(tau: float, bulk: float = 1.0, high=(1.0, 1.0, 1.0, 1.0)):
    """D3Q27 rates: [1] trace (bulk), [2] shear = 1/tau, [3..6] orders 3..6."""
    return (0.0, bulk, 1.0 / tau, high[0], high[1], high[2], high[3], 0.0, 0.0)


def d3q15_omega(tau: float, bulk: float = 1.0, third: float = 1.0, fourth: float = 1.0):
    """D3Q15 rates (Appendix A, Eq. 6A): [1] omega_9 (trace), [2] omega_4..8 = 1/tau,
    [3] omega_10..13, [4] omega_14."""
    return (0.0, bulk, 1.0 / tau, third, fourth, 0.0, 0.0, 0.0, 0.0)


def poiseuille(ny: int = 33, nx: int = 3, tau: float = 0.8, Fx: float = 1e-6) -> Workload:
    """Body-force driven channel: x periodic, walls at y = -1/2 and ny - 1/2 (Sec. 6.1)."""
    return Workload(
        name=f"poiseuille_d2q9_{nx}x{ny}", lattice=D2Q9, shape=(nx, ny, 1), wall=(0, 1, 0),
        omega=d2q9_omega(tau), rho0=1.0, u0=(0.0, 0.0, 0.0),
        tables=[(np.array([Fx]), np.array([1.0]), np.array([1.0])),
                (np.array([0.0]), np.array([1.0]), np.array([1.0]))],
        steps=10000, meta={"tau": tau, "Fx": Fx, "nu": (tau - 0.5) / 3.0})


@dataclass
class CDECase:
    """Manufactured-source scalar problem on a periodic N x N grid (one sweep member)."""

    N: int
    D: float
    A: float
    ux: float
    uy: float
    lam: float
    T: int


def cde_sweep_params(seed: int = SEED, sizes=(32, 64, 128, 256, 512), T32: int = 400):
    """Parameters of the diffusive-scaling refinement sweep of the scalar problem.

    D ~ U[0.01, 0.1] and A ~ U[1e-4, 1e-3] are drawn once from the seed; the
    advecting velocity (0.01, 0.01) and A scale as 32/N and (32/N)^2, the
    envelope rate is lambda = D (2 pi / N)^2 and the run length T_N = T32 (N/32)^2."""
    rng = np.random.default_rng(seed)
    D = float(rng.uniform(0.01, 0.1))
    A = float(rng.uniform(1e-4, 1e-3))
    out = []
    for N in sizes:
        s = 32.0 / N
        k = 2.0 * math.pi / N
        out.append(CDECase(N=N, D=D, A=A * s * s, ux=0.01 * s, uy=0.01 * s, lam=D * k * k,
                           T=int(round(T32 / (s * s)))))
    return out


def cde_closed_form(c: CDECase, t: float) -> np.ndarray:
    """Exact solution psi = phi - phi0 of the convection-diffusion equation
    (Sec. 5, Eq. 33) on the periodic N x N square for the manufactured source
    S = A sin(kx) sin(ky) e^{-lambda t}, uniform velocity and psi(0) = 0, as an
    [N][N] array (y, x).  Per Fourier mode kappa:
    psi_hat(t) = S_hat (e^{-lambda t} - e^{-sigma t}) / (sigma - lambda),
    sigma = i kappa.u + D |kappa|^2; sin(kx) sin(ky) = (cos k(x-y) - cos k(x+y))/2."""
    N = c.N
    k = 2.0 * math.pi / N
    x = np.arange(N)[None, :]
    y = np.arange(N)[:, None]
    out = np.zeros((N, N))
    for sgn, kap in ((+1, (k, -k)), (-1, (k, k))):
        sigma = 1j * (kap[0] * c.ux + kap[1] * c.uy) + c.D * (kap[0] ** 2 + kap[1] ** 2)
        R = (math.exp(-c.lam * t) - np.exp(-sigma * t)) / (sigma - c.lam)
        out += sgn * 0.5 * c.A * np.real(R * np.exp(1j * (kap[0] * x + kap[1] * y)))
    return out


def poiseuille_parabola(ny: int, tau: float, Fx: float) -> np.ndarray:
    """Analytic channel profile with walls at y = -1/2 and ny - 1/2 (Sec. 6.1)."""
    nu = (tau - 0.5) / 3.0
    y = np.arange(ny, dtype=np.float64)
    return Fx / (2.0 * nu) * (y + 0.5) * (ny - 0.5 - y)


def cde_workload(c: CDECase, phi0: float = 1.0) -> Workload:
    N = c.N
    x = np.arange(N, dtype=np.float64)
    px = c.A * np.sin(2.0 * math.pi * x / N)
    py = np.sin(2.0 * math.pi * x / N)
    lam = c.lam
    tau_phi = 3.0 * c.D + 0.5
    return Workload(
        name=f"cde_d2q5_{N}x{N}", lattice=D2Q5, shape=(N, N, 1), wall=(0, 0, 0),
        omega=d2q5_omega(tau_phi), rho0=phi0, u0=(c.ux, c.uy, 0.0),
        tables=[(px, py, np.array([1.0]))], envelope=lambda t, lam=lam: math.exp(-lam * t),
        steps=c.T, meta={"D": c.D, "A": c.A, "lam": lam, "tau_phi": tau_phi})


def kolmogorov(n: int = 256, F0: float = 1e-5, nu: float = 0.02, noise: float = 1e-4,
               seed: int = SEED, shape=None) -> Workload:
    """Periodic 3D Kolmogorov flow: F_x = F0 sin(2 pi y / Ly), rho = 1, seeded velocity noise."""
    nx, ny, nz = shape if shape is not None else (n, n, n)
    rng = np.random.default_rng(seed)
    u0 = noise * rng.standard_normal((3, nx * ny * nz))
    y = np.arange(ny, dtype=np.float64)
    py = F0 * np.sin(2.0 * math.pi * y / ny)
    one = np.array([1.0])
    zero = np.array([0.0])
    return Workload(
        name=f"kolmogorov_d3q27_{nx}x{ny}x{nz}", lattice=D3Q27, shape=(nx, ny, nz), wall=(0, 0, 0),
        omega=d3q27_omega(tau_from_nu(nu)), rho0=1.0, u0=u0,
        tables=[(one, py, one), (zero, one, one), (zero, one, one)], steps=1000,
        meta={"F0": F0, "nu": nu})


def duct(n: int = 128, nx: int = 3, F0: float = 1e-6, nu: float = 0.05, seed: int = SEED) -> Workload:
    """Square duct: x periodic, halfway bounce-back walls in y and z,
    F_x = F0 (1 + 0.5 sin(2 pi z / Lz))."""
    z = np.arange(n, dtype=np.float64)
    pz = F0 * (1.0 + 0.5 * np.sin(2.0 * math.pi * z / n))
    one = np.array([1.0])
    zero = np.array([0.0])
    return Workload(
        name=f"duct_d3q27_{nx}x{n}x{n}", lattice=D3Q27, shape=(nx, n, n), wall=(0, 1, 1),
        omega=d3q27_omega(tau_from_nu(nu)), rho0=1.0, u0=(0.0, 0.0, 0.0),
        tables=[(one, one, pz), (zero, one, one), (zero, one, one)], steps=1000,
        meta={"F0": F0, "nu": nu})


def hartmann(ny: int = 33, nx: int = 3, Ha: float = 3.0, tau: float = 0.8, Fb: float = 1e-6) -> Workload:
    """Hartmann flow (Sec. 6.2): channel with halfway bounce-back walls at
    y = -1/2 and ny - 1/2 (half-width L = ny/2), driven by F_b and retarded by
    the Lorentz force of a transverse field; the total force is
    F_x(y) = F_b Ha cosh(Ha y'/L) / sinh(Ha), y' = y + 1/2 - L (a per-y table)."""
    L = ny / 2.0
    yc = np.arange(ny, dtype=np.float64) + 0.5 - L
    py = Fb * Ha * np.cosh(Ha * yc / L) / math.sinh(Ha)
    one = np.array([1.0])
    return Workload(
        name=f"hartmann_d2q9_{nx}x{ny}_Ha{Ha:g}", lattice=D2Q9, shape=(nx, ny, 1), wall=(0, 1, 0),
        omega=d2q9_omega(tau), rho0=1.0, u0=(0.0, 0.0, 0.0),
        tables=[(one, py, one), (np.array([0.0]), one, one)],
        meta={"Ha": Ha, "Fb": Fb, "tau": tau, "nu": (tau - 0.5) / 3.0, "L": L})


def hartmann_profile(w: Workload) -> np.ndarray:
    """Analytic Hartmann velocity u_x(y) = F_b L^2 coth(Ha) / (Ha nu) [1 - cosh(Ha y'/L)/cosh(Ha)]
    (Sec. 6.2 with eta = B0^2 L^2 / (Ha^2 nu))."""
    m = w.meta
    L, Ha, nu = m["L"], m["Ha"], m["nu"]
    yc = np.arange(w.shape[1], dtype=np.float64) + 0.5 - L
    return m["Fb"] * L * L / (Ha * nu) / math.tanh(Ha) * (1.0 - np.cosh(Ha * yc / L) / math.cosh(Ha))


def womersley(ny: int = 32, nx: int = 3, tau: float = 1.0, period: int = 2000, Fm: float = 1e-5) -> Workload:
    """Womersley flow (Sec. 6.3): channel with halfway bounce-back walls driven
    by F_x = F_m cos(2 pi t / T) (a constant shape with a time envelope)."""
    om = 2.0 * math.pi / period
    one = np.array([1.0])
    return Workload(
        name=f"womersley_d2q9_{nx}x{ny}_T{period}", lattice=D2Q9, shape=(nx, ny, 1), wall=(0, 1, 0),
        omega=d2q9_omega(tau), rho0=1.0, u0=(0.0, 0.0, 0.0),
        tables=[(np.array([Fm]), one, one), (np.array([0.0]), one, one)],
        envelope=lambda t, om=om: math.cos(om * t),
        meta={"Fm": Fm, "period": period, "tau": tau, "nu": (tau - 0.5) / 3.0, "L": ny / 2.0,
              "Wo": ny / 2.0 * math.sqrt(om / ((tau - 0.5) / 3.0))})


def womersley_profile(w: Workload, t: float) -> np.ndarray:
    """Periodic-state solution of u_t = nu u_yy + F_m cos(omega t), u(+-L) = 0:
    u = Re{ F_m/(i omega) [1 - cosh(k y')/cosh(k L)] e^{i omega t} }, k = sqrt(i omega / nu)
    (the solution Sec. 6.3 prints, written with k instead of gamma = i k L)."""
    m = w.meta
    om = 2.0 * math.pi / m["period"]
    L = m["L"]
    k = np.sqrt(1j * om / m["nu"])
    yc = np.arange(w.shape[1], dtype=np.float64) + 0.5 - L
    U = m["Fm"] / (1j * om) * (1.0 - np.cosh(k * yc) / np.cosh(k * L))
    return np.real(U * np.exp(1j * om * t))


def four_rolls(N: int = 48, u0: float = 0.01, nu96: float = 0.0011 * 96 / (2.0 * math.pi)) -> Workload:
    """Four-rolls mill (Sec. 6.5): periodic N x N lattice covering [0, 2 pi)^2,
    F_x = 2 nu k^2 u0 sin(kx) sin(ky), F_y = 2 nu k^2 u0 cos(kx) cos(ky),
    k = 2 pi / N, whose steady solution is u = u0 (sin kx sin ky, cos kx cos ky).
    Convective scaling: u0 fixed in lattice units, nu = nu96 N / 96 (nu = 0.0011 in
    units where the domain is 2 pi wide), so tau_N = 1/2 + 3 nu."""
    nu = nu96 * N / 96.0
    tau = 0.5 + 3.0 * nu
    k = 2.0 * math.pi / N
    x = np.arange(N, dtype=np.float64)
    A = 2.0 * nu * k * k * u0
    one = np.array([1.0])
    X, Y = np.meshgrid(x, x, indexing="xy")
    start = np.stack([(u0 * np.sin(k * X) * np.sin(k * Y)).reshape(-1), (u0 * np.cos(k * X) * np.cos(k * Y)).reshape(-1)])
    return Workload(
        name=f"four_rolls_d2q9_{N}x{N}", lattice=D2Q9, shape=(N, N, 1), wall=(0, 0, 0),
        omega=d2q9_omega(tau), rho0=1.0, u0=start,
        tables=[(A * np.sin(k * x), np.sin(k * x), one), (A * np.cos(k * x), np.cos(k * x), one)],
        meta={"u0": u0, "nu": nu, "tau": tau, "k": k})


def four_rolls_velocity(w: Workload) -> np.ndarray:
    """Analytic steady velocity [2][N] of the four-rolls mill, node order x fastest
    (also the workload's initial velocity)."""
    return np.array(w.u0, copy=True)


def batched_sweep(count: int = 2048, seed: int = SEED, nx_range=(32, 512), ny_range=(32, 256)):
    """Parameter sweep of many small, unevenly sized 2D lattices.

    `count` force-driven D2Q9 channels (x periodic, halfway bounce-back walls in
    y) with nx ~ U{32..512}, ny ~ U{32..256}, tau ~ U[0.55, 1.5] and a uniform
    force F_x log-uniform in [1e-7, 1e-4], redrawn until the channel's
    centreline speed F ny^2 / (8 nu) stays at or below Mach 0.3 (0.3 c_s,
    c_s = 1/sqrt(3)); plus `count` periodic D2Q5 scalar lattices of the same
    sizes with tau_phi = tau, advecting velocity (0.01, 0.01) and a constant
    source A sin(2 pi x/nx) sin(2 pi y/ny), A log-uniform in [1e-7, 1e-4].
    Returns (channels, scalars)."""
    rng = np.random.default_rng([seed, 4])
    u_max = 0.3 / math.sqrt(3.0)
    channels, scalars = [], []
    one = np.array([1.0])
    for k in range(count):
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        tau = float(rng.uniform(0.55, 1.5))
        nu = (tau - 0.5) / 3.0
        while True:
            F = float(10.0 ** rng.uniform(-7.0, -4.0))
            if F * ny * ny / (8.0 * nu) <= u_max:
                break
        A = float(10.0 ** rng.uniform(-7.0, -4.0))
        channels.append(Workload(
            name=f"channel_d2q9_{nx}x{ny}_{k}", lattice=D2Q9, shape=(nx, ny, 1), wall=(0, 1, 0),
            omega=d2q9_omega(tau), rho0=1.0, u0=(0.0, 0.0, 0.0),
            tables=[(np.array([F]), one, one), (np.array([0.0]), one, one)],
            meta={"tau": tau, "Fx": F, "nu": nu}))
        x = np.arange(nx, dtype=np.float64)
        y = np.arange(ny, dtype=np.float64)
        scalars.append(Workload(
            name=f"scalar_d2q5_{nx}x{ny}_{k}", lattice=D2Q5, shape=(nx, ny, 1), wall=(0, 0, 0),
            omega=d2q5_omega(tau), rho0=1.0, u0=(0.01, 0.01, 0.0),
            tables=[(A * np.sin(2.0 * math.pi * x / nx), np.sin(2.0 * math.pi * y / ny), one)],
            meta={"tau_phi": tau, "A": A, "D": nu}))
    return channels, scalars


def duct15(n: int = 45, nx: int = 3, tau: float = 0.76, F0: float = 1e-7) -> Workload:
    """The paper's D3Q15 demonstration: a square duct (x periodic, halfway
    bounce-back walls in y and z) of n x n nodes driven by a constant F_x
    (Sec. 6.4 with Appendix A; 3 x 45 x 45, tau = 0.76, F = 1e-7)."""
    one = np.array([1.0])
    zero = np.array([0.0])
    return Workload(
        name=f"duct_d3q15_{nx}x{n}x{n}", lattice=D3Q15, shape=(nx, n, n), wall=(0, 1, 1),
        omega=d3q15_omega(tau), rho0=1.0, u0=(0.0, 0.0, 0.0),
        tables=[(np.array([F0]), one, one), (zero, one, one), (zero, one, one)], steps=1000,
        meta={"F0": F0, "nu": (tau - 0.5) / 3.0, "tau": tau})


def random_populations(q: int, N: int, weights, seed: int, amp: float = 0.05) -> np.ndarray:
    """Positive populations near a rest state, for collision-level tests."""
    rng = np.random.default_rng(seed)
    w = np.asarray(weights, np.float64)[:, None]
    return np.ascontiguousarray(w * (1.0 + amp * rng.standard_normal((q, N))))
