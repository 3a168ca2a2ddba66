"""Seeded synthetic initial conditions for the COLATUS workloads.

This module only draws and lays out input data; it holds none of the
integrator's or the force sum's arithmetic.  It is shared by the tests (which
feed the same arrays to the CUDA library and to the oracle), the benchmark and
the smoke check.  All draws use NumPy's PCG64 (``np.random.default_rng``).

The paper's own initial conditions (glass + Zel'dovich displacements of an
Eisenstein-Hu spectrum, Sec. II and Fig. 1) need a power-spectrum pipeline that
is outside the hot path; these recipes stand in for them with the same sizes
(up to 32^3 particles in a unit box) and structure (a perturbed uniform grid
with growing-mode-like velocities, or clustered Plummer spheres).

The only cosmology-dependent numbers here are input-recipe constants: the
growing-mode velocity factor H(a) f(a) of the perturbed-grid velocities and
the flat-LCDM closed-form age used to pick a uniform step size.
"""
import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# flat LCDM of the workloads: Omega_M = 0.3, Omega_L = 0.7, H0 = 1 (code units)
LCDM = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
A_START = 1.0 / 51.0


@dataclass
class ICs:
    """One realisation: positions x [N,3], velocities v [N,3], masses m [N]
    (all float64 holding float32-representable values), softening eps and the
    recipe's name.  ``q`` is the unperturbed lattice point (perturbed grids)."""
    x: np.ndarray
    v: np.ndarray
    m: np.ndarray
    eps: float
    name: str
    q: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return len(self.m)


def f32(a) -> np.ndarray:
    """Round to float32 and widen back to float64 exactly, so both sides of a
    parity test see the identical values."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def lcdm_age(a: float, Omega_M: float = 0.3, Omega_L: float = 0.7, H0: float = 1.0) -> float:
    """Closed-form cosmic time of a flat LCDM universe at scale factor a
    (t = 0 at a = 0): t = 2 asinh(sqrt(Omega_L/Omega_M) a^{3/2}) / (3 H0 sqrt(Omega_L))."""
    return 2.0 * math.asinh(math.sqrt(Omega_L / Omega_M) * a ** 1.5) / (3.0 * H0 * math.sqrt(Omega_L))


def lcdm_tau(nsteps: int, a0: float = A_START, a1: float = 1.0) -> float:
    """Uniform step size that takes a flat LCDM universe from a0 to a1 in nsteps."""
    return (lcdm_age(a1) - lcdm_age(a0)) / nsteps


def growing_mode_factor(a: float, Omega_M: float = 0.3, Omega_L: float = 0.7,
                        H0: float = 1.0) -> float:
    """H(a) f(a) with f = Omega_M(a)^0.55 for flat LCDM: the factor that turns
    a lattice displacement into a growing-mode peculiar velocity."""
    e2 = Omega_M * a ** -3 + Omega_L
    om_a = Omega_M * a ** -3 / e2
    return H0 * math.sqrt(e2) * om_a ** 0.55


# Mean comoving matter density of the flat LCDM background with G = H0 = 1:
# Omega_M * 3 H0^2 / (8 pi G).  The paper's boxes hold their galaxies "in the
# critical density"; total mass 1 in the unit box (m = 1/N) is ~28x denser.
CRITICAL_MATTER_DENSITY = 0.3 * 3.0 / (8.0 * math.pi)


def perturbed_grid(n: int, sigma: float, eps_spacing: float, seed: int,
                   zeldovich: bool = False, a_start: float = A_START, count: Optional[int] = None,
                   name: str = "perturbed_grid", total_mass: float = 1.0) -> ICs:
    """Lattice q = (i + 1/2)/n per axis in the unit box, displaced by Gaussian
    noise of standard deviation sigma/n; m = total_mass/N, eps = eps_spacing/n.

    count < n^3 keeps the first ``count`` lattice points of a seeded
    permutation (uneven-N ensembles).  zeldovich=True gives v = H f (x - q)."""
    rng = np.random.default_rng(seed)
    g = (np.arange(n) + 0.5) / n
    q = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    if count is not None:
        perm = rng.permutation(len(q))[:count]
        q = q[np.sort(perm)]
    N = len(q)
    x = f32(q + rng.normal(0.0, sigma / n, size=q.shape))
    if zeldovich:
        v = f32(growing_mode_factor(a_start) * (x - q))
    else:
        v = np.zeros_like(x)
    m = f32(np.full(N, total_mass / N))
    spacing = 1.0 / n if count is None else N ** (-1.0 / 3.0)
    return ICs(x=x, v=v, m=m, eps=float(np.float32(eps_spacing * spacing)), name=name, q=q,
               meta=dict(n=n, sigma=sigma, seed=seed))


def uniform(N: int, seed: int, eps: float = 1e-3) -> ICs:
    """N equal masses (1/N) uniform in [0,1)^3, at rest."""
    rng = np.random.default_rng(seed)
    x = f32(rng.random((N, 3)))
    m = f32(np.full(N, 1.0 / N))
    return ICs(x=x, v=np.zeros_like(x), m=m, eps=eps, name="uniform", meta=dict(seed=seed))


def plummer_clusters(N: int, seed: int, nclusters: int = 20, b: float = 0.02,
                     rmax_b: float = 10.0, mass_sigma: float = 0.5, eps: float = 1e-3) -> ICs:
    """nclusters Plummer spheres (scale radius b, truncated at rmax_b * b) with
    centres uniform in [0.1, 0.9]^3, N/nclusters bodies each (remainder to the
    first), isotropic directions, lognormal(0, mass_sigma) masses normalised
    to a total of 1, at rest."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.1, 0.9, size=(nclusters, 3))
    counts = np.full(nclusters, N // nclusters)
    counts[0] += N - counts.sum()
    pts = []
    for c, k in zip(centres, counts):
        r = np.empty(0)
        while r.size < k:
            u = rng.random(2 * k)
            u = u[u > 0]
            rr = b / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
            r = np.concatenate([r, rr[rr <= rmax_b * b]])
        r = r[:k]
        d = rng.normal(size=(k, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pts.append(c + r[:, None] * d)
    x = f32(np.concatenate(pts))
    m = rng.lognormal(0.0, mass_sigma, size=N)
    m = f32(m / m.sum())
    return ICs(x=x, v=np.zeros_like(x), m=m, eps=eps, name="plummer_clusters",
               meta=dict(seed=seed, nclusters=nclusters, b=b))


def tracers(N: int, ntr: int, seed: int) -> np.ndarray:
    """ntr distinct particle indices drawn without replacement (sorted)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(N, size=min(ntr, N), replace=False)).astype(np.int64)


# ---------------------------------------------------------------- workloads
def grid16(seed: int = 1, critical: bool = False) -> ICs:
    """N = 16^3 = 4096, sigma = 0.05 spacing, v = 0, eps = 0.01 spacing,
    m = 1/N (critical=True: the box at the background matter density)."""
    return perturbed_grid(16, 0.05, 0.01, seed, zeldovich=False, name="grid16",
                          total_mass=CRITICAL_MATTER_DENSITY if critical else 1.0)


def grid32(seed: int = 2, critical: bool = False) -> ICs:
    """N = 32^3 = 32768, sigma = 0.1 spacing, growing-mode velocities,
    eps = 0.02 spacing (the paper's 32^3 run size), m = 1/N (critical=True:
    the box at the background matter density)."""
    return perturbed_grid(32, 0.1, 0.02, seed, zeldovich=True, name="grid32",
                          total_mass=CRITICAL_MATTER_DENSITY if critical else 1.0)


def grid8(seed: int = 4) -> ICs:
    """N = 8^3 = 512 with the grid32 recipe (adjoint finite-difference checks)."""
    return perturbed_grid(8, 0.1, 0.02, seed, zeldovich=True, name="grid8")


def ensemble(R: int = 64, seed: int = 5, nmin: int = 1024, nmax: int = 32768,
             critical: bool = False):
    """R realisations with N_r = round(nmin (nmax/nmin)^U), U uniform (log-
    uniform N), each a perturbed grid of side ceil(N_r^{1/3}) keeping N_r
    lattice points, sigma = 0.1 and eps = 0.02 local spacing, growing-mode
    velocities; seeds derived from ``seed``.  critical=True gives each
    realisation the background matter density as its total mass (the same
    positions and velocities)."""
    rng = np.random.default_rng(seed)
    Ns = np.rint(nmin * (nmax / nmin) ** rng.random(R)).astype(np.int64)
    out = []
    for r, Nr in enumerate(Ns):
        n = int(math.ceil(round(Nr ** (1.0 / 3.0), 9)))
        while n ** 3 < Nr:
            n += 1
        out.append(perturbed_grid(n, 0.1, 0.02, seed * 1000 + r, zeldovich=True,
                                  count=int(Nr), name=f"ensemble[{r}]",
                                  total_mass=CRITICAL_MATTER_DENSITY if critical else 1.0))
    return out
