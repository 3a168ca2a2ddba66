"""FP64 oracle: the plain definitions of COLATUS's hot path (arXiv 1208.3444).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Readings of the paper taken here (each is also listed in the design notes):

* Eq. 1 force orientation: attractive, F_k = G sum_{j!=k} m_j (x_j-x_k)/s^3.
  The printed Eq. 1 right-hand side points away from the other bodies.
* The a^-3 factor of Eq. 1 / Eq. 4 is applied once, in the kick coefficient.
* Isolated boundaries, no background subtraction (Eq. 1 taken literally).
* Eq. 2 drives a(t) through da/dt = a H(a), integrated by classical RK4 with
  a fixed number of sub-steps per half step; t = 0 at a_start, tau uniform.
* DKD (Eqs. 3-5): H and a in Eq. 4 are taken at t^{n+1/2}.
* KDK: the trapezoidal drag of Eq. 4 applied over a half step h = tau/2,
  v' (1 + H h) = v (1 - H h) + h F / a^3, at t^n for the first half kick and
  at t^{n+1} for the second.
"""
import ctypes
import math
from typing import NamedTuple, Optional

import numpy as np

from . import build as _build

__all__ = [
    "Cosmology", "FriedmannError", "E2", "hubble", "friedmann_rhs",
    "friedmann_advance", "forces", "forces_pairwise", "potential", "vjp", "jvp",
    "kick_coefficients", "schedule", "run", "diagnostics", "layzer_irvine",
    "adjoint_run", "tangent_run", "ftle", "num_threads", "set_threads", "PINS",
    "deformation_force", "deformation_vjp", "deformation_jvp", "total_force",
    "velocity_spectrum", "friedmann_integrals", "canonical_coefficients",
    "ewald_forces", "ewald_jvp", "ewald_vjp",
]

# Parity pin of every oracle function: which non-oracle fact each one is
# tested against in tests/test_oracle_*.py.
PINS = {
    "hubble": "closed-form E(a) special cases (EdS, Milne, de Sitter, radiation)",
    "friedmann_advance": "closed-form a(t): EdS, flat LCDM sinh form, Milne, "
                         "radiation, de Sitter; RK4 fourth-order convergence",
    "forces_pairwise": "two-body point-mass law, regular ring and tetrahedron "
                       "closed forms, momentum and Newton-3, FD of potential",
    "forces": "equals pairwise within rounding; mpmath brute force on N<=12",
    "potential": "two-body closed form; its FD gradient is the force",
    "vjp": "central finite differences of the force (x and m)",
    "jvp": "central finite differences of the force; <lam, J u> duality",
    "run": "Kepler circular orbit period, drag-only v ~ a^-2 with order-2 "
           "convergence, discrete momentum/angular-momentum scaling, "
           "time reversibility, Layzer-Irvine tau^2 convergence",
    "adjoint_run": "central finite differences of a trajectory loss",
    "tangent_run": "finite differences of trajectories; adjoint duality",
    "ftle": "central differences of two oracle trajectories; the exact discrete solution "
            "of the KDK leapfrog for a coincident pair (a harmonic relative coordinate)",
    "diagnostics": "rigid rotation L = a^2 I omega and K = omega.L/2 (inertia tensor by hand); "
                   "boosts (P += a^2 M u, L about the centre of mass unchanged); translations "
                   "(COM += s, L += s x P); mirror symmetry; two-body Plummer energy; powers of a",
    "deformation_force": "equals the Eq. 1 pull of an extra body of mass C psi / G fixed at "
                         "x_psi (the paper's own description); single-body closed form",
    "deformation_vjp/jvp": "central finite differences of deformation_force",
    "friedmann_integrals": "closed-form int dt/a and int dt/a^2 for EdS, de Sitter and a static "
                           "universe; fourth-order convergence; a(t) bitwise friedmann_advance's",
    "run (canonical)": "H0 = 0 reduces to the drag KDK; drag-only canonical momentum a^2 v "
                       "conserved exactly; the one-step map is symplectic in (x, a^2 v) while "
                       "the drag KDK's is not; second-order convergence to the drag KDK's limit",
    "ewald_forces": "independent of the splitting parameter alpha; zero on a perfect lattice "
                    "and between bodies half a box apart; periodic in every body's position "
                    "and translation invariant; Newton's third law; at separations << L "
                    "the isolated Plummer force plus the background term (4 pi/3V) m d",
    "ewald_jvp": "central finite differences of ewald_forces in x and m; independent of "
                 "the splitting parameter alpha; zero row sum of the mass-weighted Jacobian "
                 "(translation); the isolated Jacobian plus (4 pi/3V) m I at separations << L",
    "ewald_vjp": "duality <lam, J u> = <J^T lam, u> with ewald_jvp in x and m; central "
                 "finite differences of lam . ewald_forces; alpha independence; sum of "
                 "dL/dx is zero (translation invariance)",
    "adjoint_run / tangent_run (box)": "central finite differences of a periodic trajectory "
                                       "loss; adjoint-tangent duality",
    "velocity_spectrum": "pure sinusoid closed form (peak height, Hann side lobes 1/4), "
                         "Parseval identity with and without the window, numpy.fft.rfft, "
                         "constant series",
}


class Cosmology(NamedTuple):
    """Density parameters and Hubble constant of Eq. 2 (code units)."""
    Omega_R: float
    Omega_M: float
    Omega_K: float
    Omega_L: float
    H0: float


class FriedmannError(ValueError):
    """H^2 < 0 (the Eq. 2 radicand went negative, e.g. recollapse)."""


# ---------------------------------------------------------------- C library
_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)


def _load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build())
        i64, dbl = ctypes.c_int64, ctypes.c_double
        L.colatus_oracle_forces_pairwise.argtypes = [i64, _dp, _dp, dbl, dbl, _dp]
        L.colatus_oracle_forces_rows.argtypes = [i64, _dp, _dp, dbl, dbl, _ip, i64, _dp]
        L.colatus_oracle_potential_rows.argtypes = [i64, _dp, _dp, dbl, dbl, _ip, i64, _dp]
        L.colatus_oracle_vjp_rows.argtypes = [i64, _dp, _dp, _dp, dbl, dbl, _ip, i64, _dp, _dp]
        L.colatus_oracle_jvp_rows.argtypes = [i64, _dp, _dp, _dp, _dp, dbl, dbl, _ip, i64, _dp]
        L.colatus_oracle_ewald_real_rows.argtypes = [i64, _dp, _dp, dbl, dbl, dbl, dbl, i64, _ip,
                                                     i64, _dp]
        L.colatus_oracle_ewald_real_jvp_rows.argtypes = [i64, _dp, _dp, _dp, _dp, dbl, dbl, dbl, dbl,
                                                         i64, _ip, i64, _dp]
        L.colatus_oracle_ewald_real_vjp_rows.argtypes = [i64, _dp, _dp, _dp, dbl, dbl, dbl, dbl, i64,
                                                         _ip, i64, _dp, _dp]
        L.colatus_oracle_threads.restype = ctypes.c_int
        L.colatus_oracle_set_threads.argtypes = [ctypes.c_int]
        L.colatus_oracle_set_threads.restype = None
        for f in (L.colatus_oracle_forces_pairwise, L.colatus_oracle_forces_rows,
                  L.colatus_oracle_potential_rows, L.colatus_oracle_vjp_rows,
                  L.colatus_oracle_jvp_rows, L.colatus_oracle_ewald_real_rows,
                  L.colatus_oracle_ewald_real_jvp_rows, L.colatus_oracle_ewald_real_vjp_rows):
            f.restype = None
        _lib = L
    return _lib


def num_threads() -> int:
    """OpenMP threads the row-parallel pair loops use."""
    return int(_load().colatus_oracle_threads())


def set_threads(n: int) -> None:
    """Run the row-parallel pair loops on n threads from now on."""
    _load().colatus_oracle_set_threads(int(n))


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def _rows(n, rows):
    if rows is None:
        rows = np.arange(n, dtype=np.int64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= n):
        raise IndexError("row index out of range")
    return rows


# ----------------------------------------------------------------- Eq. 2
def E2(a: float, c: Cosmology) -> float:
    """Radicand of Eq. 2: Omega_R a^-4 + Omega_M a^-3 + Omega_K a^-2 + Omega_L."""
    return c.Omega_R * a ** -4 + c.Omega_M * a ** -3 + c.Omega_K * a ** -2 + c.Omega_L


def hubble(a: float, c: Cosmology) -> float:
    """H(a) = H0 sqrt(E2(a)) (Eq. 2).  Raises FriedmannError if E2 < 0."""
    e2 = E2(a, c)
    if not e2 >= 0.0:
        raise FriedmannError(f"H^2 < 0 at a={a!r}")
    return c.H0 * math.sqrt(e2)


def friedmann_rhs(a: float, c: Cosmology) -> float:
    """da/dt = a H(a) (Eq. 2 with H = a-dot / a)."""
    return a * hubble(a, c)


def friedmann_advance(a: float, dt: float, c: Cosmology, nsub: int) -> float:
    """Advance a(t) by dt with nsub classical RK4 sub-steps of da/dt = a H(a)."""
    h = dt / nsub
    for _ in range(nsub):
        k1 = friedmann_rhs(a, c)
        k2 = friedmann_rhs(a + 0.5 * h * k1, c)
        k3 = friedmann_rhs(a + 0.5 * h * k2, c)
        k4 = friedmann_rhs(a + h * k3, c)
        a = a + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return a


# ------------------------------------------------------------ Eq. 1 sums
def forces_pairwise(x, m, eps: float, G: float = 1.0) -> np.ndarray:
    """Raw attractive force F (Eq. 1 without a^-3), one pass over pairs j<k."""
    x, m = _d(x).reshape(-1, 3), _d(m).reshape(-1)
    out = np.empty_like(x)
    _load().colatus_oracle_forces_pairwise(len(m), _ptr(x), _ptr(m), float(eps), float(G), _ptr(out))
    return out


def forces(x, m, eps: float, G: float = 1.0, rows=None) -> np.ndarray:
    """Raw attractive force F (Eq. 1 without a^-3) on the given target rows,
    each summed over all sources j != k in index order."""
    x, m = _d(x).reshape(-1, 3), _d(m).reshape(-1)
    rows = _rows(len(m), rows)
    out = np.empty((len(rows), 3))
    _load().colatus_oracle_forces_rows(len(m), _ptr(x), _ptr(m), float(eps), float(G),
                                       _ptr(rows, _ip), len(rows), _ptr(out))
    return out


def potential(x, m, eps: float, G: float = 1.0, rows=None) -> np.ndarray:
    """phi_k = -G sum_{j!=k} m_j / s_kj, the potential of the Eq. 1 force."""
    x, m = _d(x).reshape(-1, 3), _d(m).reshape(-1)
    rows = _rows(len(m), rows)
    out = np.empty(len(rows))
    _load().colatus_oracle_potential_rows(len(m), _ptr(x), _ptr(m), float(eps), float(G),
                                          _ptr(rows, _ip), len(rows), _ptr(out))
    return out


def vjp(x, m, lam, eps: float, G: float = 1.0, rows=None):
    """(dL/dx, dL/dm) of L = sum_k lam_k . F_k(x, m) on the given rows."""
    x, m, lam = _d(x).reshape(-1, 3), _d(m).reshape(-1), _d(lam).reshape(-1, 3)
    rows = _rows(len(m), rows)
    gx, gm = np.empty((len(rows), 3)), np.empty(len(rows))
    _load().colatus_oracle_vjp_rows(len(m), _ptr(x), _ptr(m), _ptr(lam), float(eps), float(G),
                                    _ptr(rows, _ip), len(rows), _ptr(gx), _ptr(gm))
    return gx, gm


def jvp(x, m, dx, eps: float, G: float = 1.0, dm=None, rows=None) -> np.ndarray:
    """Directional derivative of F along (dx, dm) on the given rows."""
    x, m, dx = _d(x).reshape(-1, 3), _d(m).reshape(-1), _d(dx).reshape(-1, 3)
    rows = _rows(len(m), rows)
    keep = None if dm is None else _d(dm).reshape(-1)
    dmp = None if keep is None else _ptr(keep)
    out = np.empty((len(rows), 3))
    _load().colatus_oracle_jvp_rows(len(m), _ptr(x), _ptr(m), _ptr(dx), dmp, float(eps), float(G),
                                    _ptr(rows, _ip), len(rows), _ptr(out))
    return out


# --------------------------------------------------- Eq. 6 deformation term
def deformation_force(x, Cpsi: float, xpsi, eps: float) -> np.ndarray:
    """The deformation term of Eq. 6 in the attractive reading of R1:
    C psi (x_psi - x_k) / (|x_k - x_psi|^2 + eps^2)^{3/2} for every body k, the
    pull of a fixed point "mass" C psi at x_psi (no G factor)."""
    d = np.asarray(xpsi, dtype=np.float64)[None, :] - _d(x).reshape(-1, 3)
    s2 = np.sum(d * d, axis=1) + eps * eps
    return Cpsi * d / (s2 * np.sqrt(s2))[:, None]


def _defo_J_apply(x, Cpsi, xpsi, eps, w):
    """-C psi J(d_k) w_k with d_k = x_psi - x_k, J(d) = I/s^3 - 3 d d^T / s^5:
    the derivative of deformation_force along w (J is symmetric)."""
    d = np.asarray(xpsi, dtype=np.float64)[None, :] - _d(x).reshape(-1, 3)
    w = _d(w).reshape(-1, 3)
    s2 = np.sum(d * d, axis=1) + eps * eps
    inv3 = 1.0 / (s2 * np.sqrt(s2))
    inv5 = inv3 / s2
    dw = np.sum(d * w, axis=1)
    return -Cpsi * (w * inv3[:, None] - 3.0 * d * (dw * inv5)[:, None])


def deformation_vjp(x, Cpsi: float, xpsi, eps: float, lam) -> np.ndarray:
    """d(sum_k lam_k . deformation_force_k)/dx."""
    return _defo_J_apply(x, Cpsi, xpsi, eps, lam)


def deformation_jvp(x, Cpsi: float, xpsi, eps: float, dx) -> np.ndarray:
    """Directional derivative of deformation_force along dx."""
    return _defo_J_apply(x, Cpsi, xpsi, eps, dx)


def total_force(x, m, eps: float, G: float, defo=None, box=None) -> np.ndarray:
    """F of Eq. 1 (attractive), plus the Eq. 6 deformation term when
    defo = (C psi, x_psi) is given; box = L makes the boundaries periodic
    (``ewald_forces``)."""
    F = forces(x, m, eps, G) if box is None else ewald_forces(x, m, eps, box, G)
    if defo is not None:
        F = F + deformation_force(x, defo[0], defo[1], eps)
    return F


# ------------------------------------------------- Eqs. 3-5 and KDK variant
def friedmann_integrals(a: float, dt: float, c: Cosmology, nsub: int):
    """Advance a(t) by dt as friedmann_advance does and integrate the drift and
    kick factors of the canonical leapfrog (the symplectic reformulation of
    Sec. II, after Quinn et al.): returns (a(t+dt), int dt/a, int dt/a^2).
    RK4 on the system (a, I1, I2)' = (a H(a), 1/a, 1/a^2) with nsub sub-steps,
    so a(t) is the same sequence as friedmann_advance's."""
    h = dt / nsub
    I1 = I2 = 0.0
    for _ in range(nsub):
        s1 = a
        k1 = friedmann_rhs(s1, c)
        s2 = a + 0.5 * h * k1
        k2 = friedmann_rhs(s2, c)
        s3 = a + 0.5 * h * k2
        k3 = friedmann_rhs(s3, c)
        s4 = a + h * k3
        k4 = friedmann_rhs(s4, c)
        I1 += (h / 6.0) * (1.0 / s1 + 2.0 / s2 + 2.0 / s3 + 1.0 / s4)
        I2 += (h / 6.0) * (1.0 / s1 ** 2 + 2.0 / s2 ** 2 + 2.0 / s3 ** 2 + 1.0 / s4 ** 2)
        a = a + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return a, I1, I2


def canonical_coefficients(a0: float, a1: float, K1: float, K2: float, D: float, tau: float):
    """The canonical kick-drift-kick (p = a^2 v per unit mass, dp/dt = G F / a,
    dx/dt = p / a^2; drift x += p int dt/a^2, kick p += G F int dt/a) written
    in the velocity form of ``run``'s KDK, with vh the mean drift velocity
    (x^{n+1} = x^n + tau vh):
        vh      = (D/tau) a0^2 v^n + (D/tau) K1 G F(x^n)
        v^{n+1} = tau/(D a1^2) vh  + K2/a1^2 G F(x^{n+1})
    K1, K2 = int dt/a over the two half steps, D = int dt/a^2 over the step.
    Returns (c1, d1, c2, d2) without G (G is applied like the drag kick's)."""
    return D / tau * a0 * a0, D / tau * K1, tau / (D * a1 * a1), K2 / (a1 * a1)


def kick_coefficients(a: float, H: float, h: float):
    """Trapezoidal Hubble-drag kick over a span h (Eq. 4 with tau -> h):
    v' = c v + d F with c = (1 - H h)/(1 + H h), d = h / (a^3 (1 + H h))."""
    return (1.0 - H * h) / (1.0 + H * h), h / (a ** 3 * (1.0 + H * h))


def schedule(cosmo: Cosmology, a_start: float, tau: float, nsteps: int,
             scheme: str = "kdk", nsub: int = 8):
    """Per-step scale factors and kick coefficients.

    a is advanced from t^n to t^{n+1/2} and on to t^{n+1} with nsub RK4
    sub-steps per half step.  Returns a dict of arrays: a (nsteps+1 values at
    integer steps), a_half, and the coefficients: DKD -> c, d (at t^{n+1/2});
    KDK -> c1, d1 (at t^n, span tau/2) and c2, d2 (at t^{n+1}, span tau/2);
    canonical -> c1, d1, c2, d2 of canonical_coefficients, plus K1, K2, D.
    """
    a_int = np.empty(nsteps + 1)
    a_half = np.empty(nsteps)
    a_int[0] = a_start
    a = a_start
    K1 = np.empty(nsteps)
    K2 = np.empty(nsteps)
    D = np.empty(nsteps)
    for n in range(nsteps):
        if scheme == "canonical":
            a_half[n], K1[n], Da = friedmann_integrals(a, 0.5 * tau, cosmo, nsub)
            a, K2[n], Db = friedmann_integrals(a_half[n], 0.5 * tau, cosmo, nsub)
            D[n] = Da + Db
        else:
            a_half[n] = friedmann_advance(a, 0.5 * tau, cosmo, nsub)
            a = friedmann_advance(a_half[n], 0.5 * tau, cosmo, nsub)
        a_int[n + 1] = a
    out = {"a": a_int, "a_half": a_half, "t": tau * np.arange(nsteps + 1)}
    if scheme == "canonical":
        cc = [canonical_coefficients(a_int[n], a_int[n + 1], K1[n], K2[n], D[n], tau)
              for n in range(nsteps)]
        for k, name in enumerate(("c1", "d1", "c2", "d2")):
            out[name] = np.array([q[k] for q in cc])
        out["K1"], out["K2"], out["D"] = K1, K2, D
    elif scheme == "dkd":
        cd = [kick_coefficients(ah, hubble(ah, cosmo), tau) for ah in a_half]
        out["c"] = np.array([p[0] for p in cd])
        out["d"] = np.array([p[1] for p in cd])
    elif scheme == "kdk":
        k1 = [kick_coefficients(an, hubble(an, cosmo), 0.5 * tau) for an in a_int[:-1]]
        k2 = [kick_coefficients(an, hubble(an, cosmo), 0.5 * tau) for an in a_int[1:]]
        out["c1"] = np.array([p[0] for p in k1])
        out["d1"] = np.array([p[1] for p in k1])
        out["c2"] = np.array([p[0] for p in k2])
        out["d2"] = np.array([p[1] for p in k2])
    else:
        raise ValueError("scheme must be 'dkd', 'kdk' or 'canonical'")
    return out


def run(x, v, m, eps: float, G: float, cosmo: Cosmology, a_start: float,
        tau: float, nsteps: int, scheme: str = "kdk", nsub: int = 8,
        tracers=None, keep_states: bool = False, diag_every: int = 0, defo=None, box=None):
    """Integrate Eq. 1 with the Hubble-drag leapfrog for nsteps.

    DKD follows Eqs. 3-5 literally:
        x^{n+1/2} = x^n + (tau/2) v^n
        v^{n+1}   = c v^n + d F(x^{n+1/2})         (c, d at t^{n+1/2})
        x^{n+1}   = x^{n+1/2} + (tau/2) v^{n+1}
    KDK (the configurations' "kick-drift-kick"):
        v^{n+1/2} = c1 v^n + d1 F(x^n)             (c1, d1 at t^n)
        x^{n+1}   = x^n + tau v^{n+1/2}
        v^{n+1}   = c2 v^{n+1/2} + d2 F(x^{n+1})   (c2, d2 at t^{n+1})
    F is the raw Eq. 1 force; a^-3 sits in d.  Returns a dict with the final
    x, v, the schedule, tracer records [nsteps, ntr, 6] (x, v after each step),
    optional per-step states and diagnostics every diag_every steps.
    defo = (C psi, x_psi) adds the Eq. 6 deformation term to F; box = L
    makes the boundaries periodic (positions are not wrapped).
    """
    x = _d(x).reshape(-1, 3).copy()
    v = _d(v).reshape(-1, 3).copy()
    m = _d(m).reshape(-1)
    sch = schedule(cosmo, a_start, tau, nsteps, scheme, nsub)
    tr = None if tracers is None else np.asarray(tracers, dtype=np.int64)
    rec = np.empty((nsteps, 0 if tr is None else len(tr), 6))
    states = [] if keep_states else None
    diags = []
    if diag_every:
        diags.append((0, diagnostics(x, v, m, sch["a"][0], eps, G, cosmo)))
    F = total_force(x, m, eps, G, defo, box) if scheme != "dkd" else None
    for n in range(nsteps):
        if keep_states:
            states.append((x.copy(), v.copy()))
        if scheme == "dkd":
            xh = x + 0.5 * tau * v
            v = sch["c"][n] * v + sch["d"][n] * total_force(xh, m, eps, G, defo, box)
            x = xh + 0.5 * tau * v
        else:
            vh = sch["c1"][n] * v + sch["d1"][n] * F
            x = x + tau * vh
            F = total_force(x, m, eps, G, defo, box)
            v = sch["c2"][n] * vh + sch["d2"][n] * F
        if tr is not None:
            rec[n, :, :3] = x[tr]
            rec[n, :, 3:] = v[tr]
        if diag_every and (n + 1) % diag_every == 0:
            diags.append((n + 1, diagnostics(x, v, m, sch["a"][n + 1], eps, G, cosmo)))
    out = {"x": x, "v": v, "schedule": sch, "tracers": rec, "diagnostics": diags}
    if keep_states:
        states.append((x.copy(), v.copy()))
        out["states"] = states
    return out


# ------------------------------------------------------------- diagnostics
def diagnostics(x, v, m, a: float, eps: float, G: float, cosmo: Optional[Cosmology] = None):
    """Energies and moments of the comoving system at scale factor a.

    With p = m a^2 v the canonical momentum of the paper's Hamiltonian
    section, the literal Eq. 1 dynamics has Hamiltonian K + W with
        K = (1/2) sum m a^2 |v|^2,   W = W_x / a,
        W_x = (1/2) sum_k m_k phi_k  (softened pair potential energy),
    P = sum m a^2 v (conserved), L = sum m a^2 x cross v (conserved),
    COM = sum m x / sum m.
    """
    x, v, m = _d(x).reshape(-1, 3), _d(v).reshape(-1, 3), _d(m).reshape(-1)
    phi = potential(x, m, eps, G)
    K = 0.5 * a * a * float(np.sum(m * np.sum(v * v, axis=1)))
    Wx = 0.5 * float(np.sum(m * phi))
    d = {
        "K": K, "W": Wx / a, "Wx": Wx,
        "P": a * a * np.sum(m[:, None] * v, axis=0),
        "L": a * a * np.sum(m[:, None] * np.cross(x, v), axis=0),
        "COM": np.sum(m[:, None] * x, axis=0) / np.sum(m),
        "a": a,
    }
    if cosmo is not None:
        d["H"] = hubble(a, cosmo)
    return d


def layzer_irvine(diags, t):
    """Residual of the Layzer-Irvine equation d(K+W)/dt = -H (2K + W).

    diags: list of diagnostics dicts (with H) at times t (same length).  The
    integral of H (2K + W) is taken by the trapezoid rule over the samples.
    Returns (E + I - E_0) / |W_0| at each sample.
    """
    E = np.array([d["K"] + d["W"] for d in diags])
    g = np.array([d["H"] * (2.0 * d["K"] + d["W"]) for d in diags])
    t = np.asarray(t, dtype=np.float64)
    I = np.concatenate([[0.0], np.cumsum(0.5 * (g[1:] + g[:-1]) * np.diff(t))])
    return (E + I - E[0]) / abs(diags[0]["W"])


# ---------------------------------------------------- discrete adjoint
def adjoint_run(x0, v0, m, eps: float, G: float, cosmo: Cosmology, a_start: float,
                tau: float, nsteps: int, gx_T, gv_T, gm_T=None,
                scheme: str = "kdk", nsub: int = 8, defo=None, box=None):
    """Exact transpose of the discrete leapfrog of ``run``.

    Given dLoss/dx^N, dLoss/dv^N (and an explicit dLoss/dm), returns
    (dLoss/dx^0, dLoss/dv^0, dLoss/dm) of the same FP64 trajectory.  The
    scale factor does not depend on the particles, so c, d carry no gradient.
    Every state of the forward pass is stored (no checkpointing).  box = L:
    periodic boundaries (``ewald_forces`` and ``ewald_vjp``).
    """
    m = _d(m).reshape(-1)
    fw = run(x0, v0, m, eps, G, cosmo, a_start, tau, nsteps, scheme, nsub, keep_states=True,
             defo=defo, box=box)

    def vjp_total(xx, w):
        if box is not None:
            return ewald_vjp(xx, m, w, eps, box, G)
        gx_, gm_ = vjp(xx, m, w, eps, G)
        if defo is not None:
            gx_ = gx_ + deformation_vjp(xx, defo[0], defo[1], eps, w)
        return gx_, gm_

    sch, states = fw["schedule"], fw["states"]
    lx = _d(gx_T).reshape(-1, 3).copy()
    lv = _d(gv_T).reshape(-1, 3).copy()
    gm = np.zeros_like(m) if gm_T is None else _d(gm_T).reshape(-1).copy()
    for n in reversed(range(nsteps)):
        x, v = states[n]
        if scheme == "dkd":
            xh = x + 0.5 * tau * v
            # x^{n+1} = xh + (tau/2) v^{n+1}
            lxh = lx
            lv = lv + 0.5 * tau * lx
            # v^{n+1} = c v^n + d F(xh)
            w = sch["d"][n] * lv
            gx_, gm_ = vjp_total(xh, w)
            lxh = lxh + gx_
            gm = gm + gm_
            lv = sch["c"][n] * lv
            # xh = x^n + (tau/2) v^n
            lx = lxh
            lv = lv + 0.5 * tau * lxh
        else:
            vh = sch["c1"][n] * v + sch["d1"][n] * total_force(x, m, eps, G, defo, box)
            x1 = x + tau * vh
            # v^{n+1} = c2 vh + d2 F(x^{n+1})
            lvh = sch["c2"][n] * lv
            w = sch["d2"][n] * lv
            gx_, gm_ = vjp_total(x1, w)
            lx1 = lx + gx_
            gm = gm + gm_
            # x^{n+1} = x^n + tau vh
            lvh = lvh + tau * lx1
            lx = lx1
            # vh = c1 v^n + d1 F(x^n)
            w = sch["d1"][n] * lvh
            gx_, gm_ = vjp_total(x, w)
            lx = lx + gx_
            gm = gm + gm_
            lv = sch["c1"][n] * lvh
    return lx, lv, gm


# --------------------------------------------------------- tangent model
def tangent_run(x0, v0, m, eps: float, G: float, cosmo: Cosmology, a_start: float,
                tau: float, nsteps: int, dx0, dv0, scheme: str = "kdk", nsub: int = 8,
                dm=None, defo=None, box=None):
    """Linearisation of ``run`` along (dx0, dv0[, dm]): returns the final
    tangent (dx, dv) and the per-step tangent states [nsteps+1] of (dx, dv).
    box = L: periodic boundaries (``ewald_forces`` and ``ewald_jvp``)."""
    m = _d(m).reshape(-1)
    x = _d(x0).reshape(-1, 3).copy()
    v = _d(v0).reshape(-1, 3).copy()
    dx = _d(dx0).reshape(-1, 3).copy()
    dv = _d(dv0).reshape(-1, 3).copy()
    sch = schedule(cosmo, a_start, tau, nsteps, scheme, nsub)
    hist = [(dx.copy(), dv.copy())]

    def fj(xx, ddx):
        F_ = total_force(xx, m, eps, G, defo, box)
        if box is not None:
            return F_, ewald_jvp(xx, m, ddx, eps, box, G, dm=dm)
        dF_ = jvp(xx, m, ddx, eps, G, dm=dm)
        if defo is not None:
            dF_ = dF_ + deformation_jvp(xx, defo[0], defo[1], eps, ddx)
        return F_, dF_

    for n in range(nsteps):
        if scheme == "dkd":
            xh = x + 0.5 * tau * v
            dxh = dx + 0.5 * tau * dv
            F, dF = fj(xh, dxh)
            v = sch["c"][n] * v + sch["d"][n] * F
            dv = sch["c"][n] * dv + sch["d"][n] * dF
            x = xh + 0.5 * tau * v
            dx = dxh + 0.5 * tau * dv
        else:
            F, dF = fj(x, dx)
            vh = sch["c1"][n] * v + sch["d1"][n] * F
            dvh = sch["c1"][n] * dv + sch["d1"][n] * dF
            x = x + tau * vh
            dx = dx + tau * dvh
            F, dF = fj(x, dx)
            v = sch["c2"][n] * vh + sch["d2"][n] * F
            dv = sch["c2"][n] * dvh + sch["d2"][n] * dF
        hist.append((dx.copy(), dv.copy()))
    return dx, dv, hist


def ftle(x0, v0, m, eps: float, G: float, cosmo: Cosmology, a_start: float,
         tau: float, nsteps: int, tracer: int, direction=(1.0, 0.0, 0.0),
         scheme: str = "kdk", nsub: int = 8, box=None) -> np.ndarray:
    """Finite-time Lyapunov growth of one tracer's own phase-space perturbation.

    The tangent is seeded with a unit position perturbation on the tracer only
    (the rest of the system starts unperturbed but responds).  Returns, for
    n = 1..nsteps, ln(|(dx_i, dv_i)(t^n)| / |(dx_i, dv_i)(0)|) / t^n.
    """
    n_ = len(_d(m).reshape(-1))
    dx0 = np.zeros((n_, 3))
    dx0[tracer] = np.asarray(direction, dtype=np.float64) / np.linalg.norm(direction)
    _, _, hist = tangent_run(x0, v0, m, eps, G, cosmo, a_start, tau, nsteps,
                             dx0, np.zeros((n_, 3)), scheme, nsub, box=box)
    g0 = math.sqrt(float(np.sum(hist[0][0][tracer] ** 2) + np.sum(hist[0][1][tracer] ** 2)))
    out = np.empty(nsteps)
    for n in range(1, nsteps + 1):
        dxn, dvn = hist[n]
        g = math.sqrt(float(np.sum(dxn[tracer] ** 2) + np.sum(dvn[tracer] ** 2)))
        out[n - 1] = math.log(g / g0) / (n * tau)
    return out


# --------------------------------------- tracer velocity energy spectrum
def velocity_spectrum(v, dt: float, window: str = "rect", detrend: bool = True) -> np.ndarray:
    """One-sided energy spectrum of each tracer's velocity record (Sec. I and
    Sec. IV: the velocity of single bodies at every step, and its energy power
    spectrum, for chaotic-advection analysis).

    v: [T, ntr, 3] velocities at uniform spacing dt.  With u = v - mean(v)
    (detrend) or u = v, w the rectangular or periodic Hann window
    w_n = (1 - cos(2 pi n / T)) / 2 and U = (1/T) sum_n w_n^2,

        E_k(f_j) = c_j dt / (T U) * (1/2) sum_c |sum_n w_n u_{n,k,c} e^{-2 pi i j n / T}|^2

    for j = 0 .. floor(T/2), f_j = j / (T dt), c_j = 2 except c_0 = 1 and
    c_{T/2} = 1 (T even).  Then sum_j E_k(f_j) / (T dt) is the window-weighted
    mean of (1/2)|u|^2, i.e. the specific kinetic energy of the fluctuation
    (Parseval).  Returns E [ntr, floor(T/2)+1].  The DFT is the explicit sum
    (a matrix product with the exponential table), in double precision.
    """
    v = np.asarray(v, dtype=np.float64)
    T = v.shape[0]
    u = v - v.mean(axis=0, keepdims=True) if detrend else v.copy()
    n = np.arange(T)
    if window == "hann":
        w = 0.5 * (1.0 - np.cos(2.0 * np.pi * n / T))
    elif window == "rect":
        w = np.ones(T)
    else:
        raise ValueError(window)
    U = float(np.sum(w * w)) / T
    nf = T // 2 + 1
    j = np.arange(nf)
    # reduce j n mod T before forming the angle, so the table is exact to rounding
    ang = 2.0 * np.pi * ((j[:, None] * n[None, :]) % T) / T
    Ereal = np.cos(ang) @ (w[:, None, None] * u).reshape(T, -1)
    Eimag = -np.sin(ang) @ (w[:, None, None] * u).reshape(T, -1)
    power = (Ereal ** 2 + Eimag ** 2).reshape(nf, v.shape[1], 3).sum(axis=2)
    c = np.full(nf, 2.0)
    c[0] = 1.0
    if T % 2 == 0:
        c[-1] = 1.0
    return (0.5 * c[:, None] * dt / (T * U) * power).T


# ------------------------------------------------- periodic boundaries (Ewald)
def ewald_forces(x, m, eps: float, L: float, G: float = 1.0, alpha=None, nreal: int = 1,
                 nk=None, rows=None) -> np.ndarray:
    """Raw attractive force (Eq. 1 without a^-3) in a periodic box of side L
    (Sec. II states periodic boundaries for a homogeneous distribution): the
    pull of every image of every body, with the uniform mean density removed
    (the k = 0 mode left out, so a homogeneous box feels no force), and the
    nearest image Plummer-softened with eps instead of Newtonian.

    Ewald's split with parameter alpha: the real-space sum over images within
    nreal boxes of the nearest one (C loops) plus the reciprocal sum over
    k = 2 pi n / L, 0 < |n_c| <= nk:
        a_L(x_k) = -(4 pi G / L^3) sum_k exp(-k^2/(4 alpha^2)) / k^2
                     * k * sum_j m_j sin(k . (x_k - x_j)).
    Defaults (alpha L = 6, nreal = 1: the first image left out is 1.5 L away,
    erfc(9) ~ 4e-37; nk from exp(-(pi nk/(alpha L))^2) < 1e-18) converge both
    sums to double rounding.  The result does not depend on alpha."""
    x, m = _d(x).reshape(-1, 3), _d(m).reshape(-1)
    rows = _rows(len(m), rows)
    alpha = 6.0 / L if alpha is None else float(alpha)
    if nk is None:
        # exp(-pi^2 n^2 / (alpha L)^2) below 1e-18
        nk = int(math.ceil(alpha * L / math.pi * math.sqrt(18.0 * math.log(10.0))))
    out = np.empty((len(rows), 3))
    _load().colatus_oracle_ewald_real_rows(len(m), _ptr(x), _ptr(m), float(eps), float(G), float(L),
                                           alpha, int(nreal), _ptr(rows, _ip), len(rows), _ptr(out))
    r = np.arange(-nk, nk + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    n = n[np.any(n != 0, axis=1)]
    V = L ** 3
    xt = x[rows]
    for c0 in range(0, len(n), 2048):
        k = 2.0 * np.pi / L * n[c0:c0 + 2048]                      # [K, 3]
        k2 = np.sum(k * k, axis=1)
        w = 4.0 * np.pi * G / V * np.exp(-k2 / (4.0 * alpha * alpha)) / k2
        rho = np.exp(1j * (k @ x.T)) @ m                            # sum_j m_j e^{i k.x_j}
        s = np.imag(np.exp(1j * (k @ xt.T)) * np.conj(rho)[:, None])  # sum_j m_j sin(k.(x_t - x_j))
        out -= (w[:, None] * s).T @ k
    return out


def _ewald_defaults(L, alpha, nk):
    alpha = 6.0 / L if alpha is None else float(alpha)
    if nk is None:
        nk = int(math.ceil(alpha * L / math.pi * math.sqrt(18.0 * math.log(10.0))))
    return alpha, nk


def _kvectors(L, nk):
    r = np.arange(-nk, nk + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    return n[np.any(n != 0, axis=1)]


def ewald_jvp(x, m, dx, eps: float, L: float, G: float = 1.0, alpha=None, nreal: int = 1,
              nk=None, rows=None, dm=None) -> np.ndarray:
    """Directional derivative of ``ewald_forces`` along (dx, dm).

    The periodic force is F_k = G sum_j m_j Phi(x_j - x_k) with Phi odd; its
    derivative is G sum_j [m_j J(d_kj) (dx_j - dx_k) + dm_j Phi(d_kj)], J the
    Jacobian of Phi.  Real space: C loops over the same images as the force
    (colatus_oracle_ewald_real_jvp_rows).  Reciprocal space, differentiating
    the k-sum of ``ewald_forces`` term by term:
        (4 pi G / L^3) sum_k A(k) k sum_j [ m_j cos(k.(x_j - x_k)) k.(dx_j - dx_k)
                                            + dm_j sin(k.(x_j - x_k)) ],
    A(k) = exp(-k^2/(4 alpha^2)) / k^2."""
    x, m, dx = _d(x).reshape(-1, 3), _d(m).reshape(-1), _d(dx).reshape(-1, 3)
    rows = _rows(len(m), rows)
    alpha, nk = _ewald_defaults(L, alpha, nk)
    keep = None if dm is None else _d(dm).reshape(-1)
    out = np.empty((len(rows), 3))
    _load().colatus_oracle_ewald_real_jvp_rows(len(m), _ptr(x), _ptr(m), _ptr(dx),
                                               None if keep is None else _ptr(keep), float(eps),
                                               float(G), float(L), alpha, int(nreal),
                                               _ptr(rows, _ip), len(rows), _ptr(out))
    n = _kvectors(L, nk)
    V = L ** 3
    xt, dxt = x[rows], dx[rows]
    for c0 in range(0, len(n), 2048):
        k = 2.0 * np.pi / L * n[c0:c0 + 2048]                       # [K, 3]
        k2 = np.sum(k * k, axis=1)
        A = 4.0 * np.pi * G / V * np.exp(-k2 / (4.0 * alpha * alpha)) / k2
        cj, sj = np.cos(k @ x.T), np.sin(k @ x.T)                    # [K, N]
        ct, st = np.cos(k @ xt.T), np.sin(k @ xt.T)                  # [K, R]
        kdx = k @ dx.T                                               # k . dx_j
        P = (cj * kdx) @ m                                           # sum_j m_j (k.dx_j) cos
        Q = (sj * kdx) @ m                                           # sum_j m_j (k.dx_j) sin
        C, S = cj @ m, sj @ m
        # sum_j m_j cos(k.(x_j - x_t)) k.dx_j = cos_t P + sin_t Q
        # sum_j m_j cos(k.(x_j - x_t)) k.dx_t = (k.dx_t) (cos_t C + sin_t S)
        term = ct * P[:, None] + st * Q[:, None] - (k @ dxt.T) * (ct * C[:, None] + st * S[:, None])
        if keep is not None:
            Cd, Sd = cj @ keep, sj @ keep
            # sum_j dm_j sin(k.(x_j - x_t)) = cos_t Sd - sin_t Cd
            term = term + ct * Sd[:, None] - st * Cd[:, None]
        out += (A[:, None] * term).T @ k
    return out


def ewald_vjp(x, m, lam, eps: float, L: float, G: float = 1.0, alpha=None, nreal: int = 1,
              nk=None, rows=None):
    """(dL/dx, dL/dm) of L = sum_k lam_k . F_k for the periodic force of
    ``ewald_forces``: with F_k = G sum_j m_j Phi(x_j - x_k),
        dL/dx_i = G sum_j J(d_ij) (m_i lam_j - m_j lam_i),
        dL/dm_i = -G sum_j lam_j . Phi(d_ij).
    Real space by C loops (colatus_oracle_ewald_real_vjp_rows); reciprocal
    space from the k-sum, with cos/sin(k.(x_j - x_i)) expanded per k."""
    x, m, lam = _d(x).reshape(-1, 3), _d(m).reshape(-1), _d(lam).reshape(-1, 3)
    rows = _rows(len(m), rows)
    alpha, nk = _ewald_defaults(L, alpha, nk)
    gx, gm = np.empty((len(rows), 3)), np.empty(len(rows))
    _load().colatus_oracle_ewald_real_vjp_rows(len(m), _ptr(x), _ptr(m), _ptr(lam), float(eps),
                                               float(G), float(L), alpha, int(nreal),
                                               _ptr(rows, _ip), len(rows), _ptr(gx), _ptr(gm))
    n = _kvectors(L, nk)
    V = L ** 3
    xt, lt, mt = x[rows], lam[rows], m[rows]
    for c0 in range(0, len(n), 2048):
        k = 2.0 * np.pi / L * n[c0:c0 + 2048]
        k2 = np.sum(k * k, axis=1)
        A = 4.0 * np.pi * G / V * np.exp(-k2 / (4.0 * alpha * alpha)) / k2
        cj, sj = np.cos(k @ x.T), np.sin(k @ x.T)
        ct, st = np.cos(k @ xt.T), np.sin(k @ xt.T)
        kl = k @ lam.T                                               # k . lam_j
        Pw, Qw = np.sum(cj * kl, axis=1), np.sum(sj * kl, axis=1)
        C, S = cj @ m, sj @ m
        # sum_j cos(k.(x_j - x_i)) [m_i k.lam_j - m_j k.lam_i]
        term = (mt[None, :] * (ct * Pw[:, None] + st * Qw[:, None])
                - (k @ lt.T) * (ct * C[:, None] + st * S[:, None]))
        gx += (A[:, None] * term).T @ k
        # -sum_j k.lam_j sin(k.(x_j - x_i)) = -(cos_i Qw - sin_i Pw)
        gm -= A @ (ct * Qw[:, None] - st * Pw[:, None])
    return gx, gm

