"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only draws numbers and shapes them into the arrays a caller hands
to the solver; it holds none of the projection method's arithmetic.

* ``splitmix64``: the published SplitMix64 generator (Steele, Lea & Flood,
  OOPSLA 2014), evaluated counter-style on (seed, linear index), so any element
  can be reproduced alone. Uniforms take its top 53 bits.
* ``normal_noise``: Box-Muller on consecutive uniform pairs.
* ``chi_field``: the random effective-temperature initial condition of the
  paper's section 4.4, Eq. (47): white noise convolved with exp(-|r|^2/l_c^2),
  normalised so every cell is N(mean, std^2). The sum is cut off at
  ``cutoff * l_c`` cells per axis (the paper's cutoff factor, 5), x and y wrap
  periodically, and z is padded with a shell of independent noise (the
  paper's ghost set V').  The Gaussian is separable, so the 3-D sum is three
  1-D passes.
* ``rhs_field``: uniform [-1, 1) right-hand side on interior corner nodes.

Array layouts match the library: velocity-like (3, nz+1, ny, nx), cell
scalars (nz, ny, nx), x fastest, float64.
"""
from __future__ import annotations

import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 output for state ``seed + (idx+1)*golden`` (uint64, wraps)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniforms in [0, 1) from the top 53 bits of splitmix64."""
    idx = np.arange(offset, offset + n, dtype=np.uint64)
    return (splitmix64(seed, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal_noise(seed: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller on uniform pairs (u1, u2)."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1-u1 in (0, 1]
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(2.0 * math.pi * u2)
    out[1::2] = r * np.sin(2.0 * math.pi * u2)
    return out[:n]


def gaussian_taps(lc_cells: float, cutoff: float = 5.0) -> np.ndarray:
    """1-D taps exp(-d^2/l_c^2) for |d| <= ceil(cutoff*l_c) (cell units)."""
    c = int(math.ceil(cutoff * lc_cells))
    d = np.arange(-c, c + 1, dtype=np.float64)
    return np.exp(-(d * d) / (lc_cells * lc_cells))


def chi_field(seed: int, nx: int, ny: int, nz: int, mean: float, std: float,
              lc_cells: float, cutoff: float = 5.0) -> np.ndarray:
    """Random chi^0 of section 4.4, Eq. (47); returns (nz, ny, nx) float64."""
    g = gaussian_taps(lc_cells, cutoff)
    c = (g.size - 1) // 2
    nzp = nz + 2 * c
    w = normal_noise(seed, nzp * ny * nx).reshape(nzp, ny, nx)
    from scipy.ndimage import correlate1d
    # x and y: periodic wrap; z: the padded shell supplies the out-of-range terms
    w = correlate1d(w, g, axis=2, mode="wrap")
    w = correlate1d(w, g, axis=1, mode="wrap")
    out = correlate1d(w, g, axis=0, mode="constant")[c:c + nz]
    # N = sqrt(sum over the cutoff box of exp(-2|r|^2/l_c^2)) = (sum g_d^2)^(3/2)
    norm = float(np.sum(g * g)) ** 1.5
    return mean + std * out / norm


def rhs_field(seed: int, nx: int, ny: int, nz: int) -> np.ndarray:
    """Uniform [-1, 1) on interior corner nodes, zero on the wall planes."""
    u = uniform01(seed, 3 * (nz + 1) * ny * nx).reshape(3, nz + 1, ny, nx)
    b = 2.0 * u - 1.0
    b[:, 0] = 0.0
    b[:, nz] = 0.0
    return b


# ---------------------------------------------------------------------------
# Table 1 of the paper (material parameters) and workload recipes
# ---------------------------------------------------------------------------

K_BOLTZMANN = 1.380649e-23  # J/K (exact SI value)

TABLE1 = dict(
    K=122e9,          # bulk modulus, Pa
    mu=37.4e9,        # shear modulus, Pa
    rho=6125.0,       # density, kg/m^3
    sY=0.85e9,        # yield stress, Pa
    tau0=1e-13,       # molecular vibration timescale, s
    eps0=0.3,         # typical local strain
    c0=0.4,           # effective heat capacity
    Delta_K=8000.0,   # activation barrier / k_B, K
    Omega=300e-30,    # activation volume, m^3 (300 cubic angstrom)
    T=400.0,          # bath temperature, K
    chi_inf=900.0,    # steady-state effective temperature, K
    ez_K=21000.0,     # STZ formation energy / k_B, K
)


def lame_lambda(K: float, mu: float) -> float:
    """Lame's first parameter from bulk and shear moduli (lambda = K - 2 mu / 3)."""
    return K - 2.0 * mu / 3.0


def stz_values(l: float) -> dict:
    """STZ parameter values of Table 1 plus the diffusion length l (m)."""
    t = TABLE1
    return dict(tau0=t["tau0"], eps0=t["eps0"], c0=t["c0"], Delta_K=t["Delta_K"],
                Omega=t["Omega"], T=t["T"], chi_inf=t["chi_inf"], ez_K=t["ez_K"],
                sY=t["sY"], l=l, kB=K_BOLTZMANN)


def shear_time_unit(L: float = 0.01) -> float:
    """t_s = L / c_s with c_s = sqrt(mu/rho) (section 4)."""
    return L / (TABLE1["mu"] / TABLE1["rho"]) ** 0.5


class Workload:
    """Synthetic simple-shear or disc workload on an n^3-cell grid.

    Geometry: x, y in [-L, L) with L = 1 cm, so h = 2L/n; height n h.
    Time step dt = 200 t_s (section 4.3).  ``strain`` is the engineering
    wall-to-wall shear strain reached after ``steps`` steps (2 U t / H).
    ``preload`` is an initial uniform sigma_xz (Pa); with preload = 0 the
    state starts unstressed.  ``chi`` follows Eq. (47) with the given mean,
    std and correlation length (cells).
    """

    def __init__(self, n, steps, strain=0.02, preload=0.0, chi_mean=600.0, chi_std=30.0,
                 lc_cells=4.0, seed=2, kind=0, l_cells=1.0, nz=None, dt_ts=200.0):
        self.nx = self.ny = n
        self.nz = n if nz is None else nz
        self.L = 0.01
        self.h = 2.0 * self.L / n
        self.H = self.nz * self.h
        self.ts = shear_time_unit(self.L)
        self.dt = dt_ts * self.ts
        self.steps = steps
        self.lam = lame_lambda(TABLE1["K"], TABLE1["mu"])
        self.mu = TABLE1["mu"]
        self.stz = stz_values(l_cells * self.h)
        self.kind = kind
        self.U_B = strain * self.H / (2.0 * steps * self.dt)
        self.t_ramp = self.ts
        self.omega = 0.0
        self.R = 1.0 / 3.0
        self.lambda_w = 16.0 * math.log(10.0) / (1.0 - self.R ** 2) ** 2
        self.preload = preload
        self.chi_recipe = (seed, chi_mean, chi_std, lc_cells)

    def bc_values(self) -> dict:
        return dict(kind=self.kind, U_B=self.U_B, t_ramp=self.t_ramp, omega=self.omega,
                    R=self.R, lambda_w=self.lambda_w)

    def initial_state(self):
        """(v, sigma, chi, t0) as float64 numpy arrays.

        With a preload the walls start at full speed (t0 = t_ramp) and v is the
        matching linear shear profile; otherwise v = 0 and t0 = 0.
        """
        nx, ny, nz = self.nx, self.ny, self.nz
        v = np.zeros((3, nz + 1, ny, nx))
        sig = np.zeros((6, nz, ny, nx))
        t0 = 0.0
        if self.preload != 0.0:
            sig[4] = self.preload
            if self.kind == 0:
                t0 = self.t_ramp
                zk = (np.arange(nz + 1) - nz / 2.0) * self.h
                v[0] = (2.0 * self.U_B / self.H * zk)[:, None, None]
        seed, m, s, lc = self.chi_recipe
        chi = chi_field(seed, nx, ny, nz, m, s, lc)
        return v, sig, chi, t0
