"""Flory-Huggins thermodynamics the paper compares its simulations against.

TEST INFRASTRUCTURE ONLY (part of the oracle package).

Sec. 4 of the paper validates the lattice Boltzmann update by comparing the
coexisting (binodal) compositions of phase-separated binary and ternary
mixtures to those obtained by minimising the Flory-Huggins free energy
(Eq. lgf).  Per unit mer density and in units of theta, that free energy is

    f(phi) = sum_s (phi^s / m^s) ln phi^s + 1/2 sum_{s,t} chi^{st} phi^s phi^t

up to terms linear in phi, which do not change coexistence.  Coexisting
phases share the exchange chemical potentials d f / d phi^s - d f / d phi^N
and the grand potential f - sum_s phi^s d f/d phi^s (the common tangent
plane), i.e. they are the contact points of a facet of the lower convex hull
of f over the composition simplex.

Two independent routes are provided so that each pins the other: a Newton
solve of the tangent conditions, and a brute-force lower convex hull of f
sampled on a fine grid.
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np
from scipy import optimize


def free_energy(phi, chi, m) -> np.ndarray:
    """f(phi) per unit mer density, theta = 1.  phi has shape (..., N)."""
    phi = np.asarray(phi, dtype=np.float64)
    chi = np.asarray(chi, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        ent = np.where(phi > 0, phi / m * np.log(np.where(phi > 0, phi, 1.0)), 0.0)
    return ent.sum(-1) + 0.5 * np.einsum("...s,st,...t->...", phi, chi, phi)


def dfdphi(phi, chi, m) -> np.ndarray:
    """Partial derivatives d f / d phi^s treating every phi^s as independent."""
    phi = np.asarray(phi, dtype=np.float64)
    return (np.log(phi) + 1.0) / np.asarray(m) + phi @ np.asarray(chi)


def exchange_potentials(phi, chi, m) -> np.ndarray:
    """d f/d phi^s - d f/d phi^{N-1} for s = 0..N-2 (the simplex has N-1 free coordinates)."""
    g = dfdphi(phi, chi, m)
    return g[..., :-1] - g[..., -1:]


def grand_potential(phi, chi, m) -> np.ndarray:
    phi = np.asarray(phi, dtype=np.float64)
    ex = exchange_potentials(phi, chi, m)
    return free_energy(phi, chi, m) - (phi[..., :-1] * ex).sum(-1)


# ------------------------------------------------------------------ binary

def critical_binary(mA: float, mB: float) -> Tuple[float, float]:
    """Critical point (phi_A, chi) of the binary Flory-Huggins mixture.

    f''(phi) = 1/(mA phi) + 1/(mB (1-phi)) - 2 chi and f''' = 0 give
    phi_c = sqrt(mB) / (sqrt(mA) + sqrt(mB)), chi_c = (1/sqrt(mA) + 1/sqrt(mB))^2 / 2.
    """
    a, b = math.sqrt(mA), math.sqrt(mB)
    return b / (a + b), 0.5 * (1.0 / a + 1.0 / b) ** 2


def _binary_vec(x, chi, mA, mB):
    return np.array([x, 1.0 - x])


def binodal_binary(chi: float, mA: float = 1.0, mB: float = 1.0) -> Tuple[float, float]:
    """Coexisting phi_A of the two phases (low, high) from the common tangent.

    Newton (scipy) on: equal exchange potential and equal grand potential,
    started from the brute-force hull.
    """
    C = np.array([[0.0, chi], [chi, 0.0]])
    m = np.array([mA, mB])
    lo, hi = hull_binary(chi, mA, mB)

    def eqs(v):
        p1 = np.array([v[0], 1 - v[0]])
        p2 = np.array([v[1], 1 - v[1]])
        return [exchange_potentials(p1, C, m)[0] - exchange_potentials(p2, C, m)[0],
                grand_potential(p1, C, m) - grand_potential(p2, C, m)]

    sol = optimize.root(eqs, [lo, hi], method="hybr", tol=1e-15)
    a, b = sorted(sol.x)
    if np.max(np.abs(eqs(sol.x))) > 1e-12 or not (0 < a < b < 1):
        raise RuntimeError(f"binary binodal failed for chi={chi}: {sol.message}")
    return float(a), float(b)


def hull_binary(chi: float, mA: float = 1.0, mB: float = 1.0, n: int = 200001):
    """Brute-force coexistence: the widest gap of the lower convex hull of f(phi_A)."""
    x = np.linspace(1e-9, 1 - 1e-9, n)
    C = np.array([[0.0, chi], [chi, 0.0]])
    f = free_energy(np.stack([x, 1 - x], -1), C, np.array([mA, mB]))
    # monotone-chain lower hull
    hull = []
    for k in range(n):
        while len(hull) >= 2:
            i, j = hull[-2], hull[-1]
            if (x[j] - x[i]) * (f[k] - f[i]) - (f[j] - f[i]) * (x[k] - x[i]) <= 0:
                hull.pop()
            else:
                break
        hull.append(k)
    hull = np.array(hull)
    gaps = np.diff(x[hull])
    g = int(np.argmax(gaps))
    return float(x[hull[g]]), float(x[hull[g + 1]])


def symmetric_binary_binodal(chi: float) -> float:
    """For mA = mB = 1 the high branch solves ln(phi/(1-phi)) = chi (2 phi - 1)."""
    return optimize.brentq(lambda p: math.log(p / (1 - p)) - chi * (2 * p - 1), 0.5 + 1e-12,
                           1 - 1e-15, xtol=1e-16)


def spinodal_chi_binary(phi: float, mA: float = 1.0, mB: float = 1.0) -> float:
    """chi at which f''(phi) = 0: (1/(mA phi) + 1/(mB (1-phi))) / 2."""
    return 0.5 * (1.0 / (mA * phi) + 1.0 / (mB * (1.0 - phi)))


# ----------------------------------------------------------------- ternary

def simplex_grid(n: int) -> np.ndarray:
    """All compositions (i, j, n-i-j)/n with strictly positive entries."""
    pts = [(i, j, n - i - j) for i in range(1, n) for j in range(1, n - i)]
    return np.array(pts, dtype=np.float64) / n


def hull_ternary(chi, m, phibar, n: int = 300):
    """Brute-force: the lower-hull facet of f over the simplex whose projection
    contains phibar.  Returns its three vertices (3 x 3 compositions).  In a
    two-phase region two vertices lie near one phase and one near the other (or
    the facet is a sliver along the tie line); in a three-phase region the
    vertices approximate the three phases."""
    from scipy.spatial import ConvexHull
    P = simplex_grid(n)
    f = free_energy(P, chi, m)
    pts = np.column_stack([P[:, 0], P[:, 1], f])
    hull = ConvexHull(pts)
    best = None
    pb = np.asarray(phibar, dtype=np.float64)
    for simplex, eq in zip(hull.simplices, hull.equations):
        if eq[2] >= 0:  # keep the lower facets only
            continue
        tri = P[simplex]
        # barycentric coordinates of phibar in the projected triangle
        T = np.array([[tri[0, 0] - tri[2, 0], tri[1, 0] - tri[2, 0]],
                      [tri[0, 1] - tri[2, 1], tri[1, 1] - tri[2, 1]]])
        if abs(np.linalg.det(T)) < 1e-300:
            continue
        l12 = np.linalg.solve(T, pb[:2] - tri[2, :2])
        lam = np.array([l12[0], l12[1], 1 - l12.sum()])
        if lam.min() >= -1e-12:
            area = abs(np.linalg.det(T))
            if best is None or area > best[0]:
                best = (area, tri, lam)
    if best is None:
        raise RuntimeError("phibar outside the sampled simplex")
    return best[1], best[2]


def tie_line(chi, m, phibar, guess=None):
    """The two coexisting phases whose tie line passes through phibar (N = 3).

    Unknowns: phase compositions p1, p2 (first two coordinates each) and the
    lever fraction t (phibar = t p1 + (1 - t) p2).  Equations: equal exchange
    potentials (2), equal grand potential (1), lever rule (2).
    """
    chi = np.asarray(chi, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    pb = np.asarray(phibar, dtype=np.float64)
    if guess is None:
        tri, lam = hull_ternary(chi, m, pb)
        # split the facet's vertices into two clusters: the far-apart pair
        d = [np.linalg.norm(tri[a] - tri[b]) for a, b in ((0, 1), (0, 2), (1, 2))]
        a, b = [(0, 1), (0, 2), (1, 2)][int(np.argmax(d))]
        p1, p2 = tri[a], tri[b]
        t0 = float(np.clip(np.dot(pb - p2, p1 - p2) / np.dot(p1 - p2, p1 - p2), 0.05, 0.95))
        guess = np.array([p1[0], p1[1], p2[0], p2[1], t0])

    def full(a, b):
        return np.array([a, b, 1.0 - a - b])

    def eqs(v):
        q1, q2 = full(v[0], v[1]), full(v[2], v[3])
        if q1.min() <= 0 or q2.min() <= 0:
            return np.full(5, 1e3)
        e1, e2 = exchange_potentials(q1, chi, m), exchange_potentials(q2, chi, m)
        lever = v[4] * q1 + (1 - v[4]) * q2 - pb
        return np.array([e1[0] - e2[0], e1[1] - e2[1],
                         grand_potential(q1, chi, m) - grand_potential(q2, chi, m),
                         lever[0], lever[1]])

    sol = optimize.root(eqs, guess, method="hybr", tol=1e-14)
    if np.max(np.abs(eqs(sol.x))) > 1e-11:
        raise RuntimeError(f"tie line failed: {sol.message}")
    q1, q2 = full(sol.x[0], sol.x[1]), full(sol.x[2], sol.x[3])
    return q1, q2


def symmetric_three_phase(chi: float) -> Tuple[float, float]:
    """Symmetric ternary (uniform chi, m = 1): phases (a,b,b), (b,a,b), (b,b,a) with
    a + 2b = 1 and equal exchange potentials, ln(a/b) = chi (a - b).  Returns (a, b)."""
    g = lambda b: math.log((1 - 2 * b) / b) - chi * (1 - 3 * b)
    b = optimize.brentq(g, 1e-14, 1.0 / 3.0 - 1e-9, xtol=1e-16)
    return 1 - 2 * b, b


def spinodal_det(phi, chi, m) -> float:
    """Determinant of the Hessian of f on the simplex (free coordinates 0..N-2)."""
    phi = np.asarray(phi, dtype=np.float64)
    N = phi.size
    H = np.diag(1.0 / (np.asarray(m) * phi)) + np.asarray(chi)
    # restrict to the tangent space of sum phi = 1
    B = np.zeros((N, N - 1))
    for k in range(N - 1):
        B[k, k] = 1.0
        B[N - 1, k] = -1.0
    return float(np.linalg.det(B.T @ H @ B))


def critical_ternary(chi, m, guess) -> np.ndarray:
    """A critical point of a ternary mixture (N = 3) near `guess`.

    Two conditions on the composition phi: the Hessian of f restricted to the simplex is
    singular (the spinodal, det = 0), and the third derivative of f along its null
    direction v vanishes (the two coexisting phases merge there).  f's third derivatives
    are diagonal, d^3 f / d phi^s^3 = -1 / (m^s phi^s^2), so the second condition reads
    sum_s v_s^3 / (m^s phi_s^2) = 0 with v = (w_0, w_1, -w_0 - w_1), w the null vector of
    the 2 x 2 restricted Hessian."""
    chi = np.asarray(chi, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    B = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, -1.0]])

    def eqs(x):
        phi = np.array([x[0], x[1], 1.0 - x[0] - x[1]])
        if phi.min() <= 0:
            return np.full(2, 1e3)
        H = B.T @ (np.diag(1.0 / (m * phi)) + chi) @ B
        # null direction of the singular 2 x 2 matrix (the row with the larger entries)
        w = np.array([-H[0, 1], H[0, 0]]) if abs(H[0, 0]) + abs(H[0, 1]) >= abs(H[1, 0]) + abs(H[1, 1]) \
            else np.array([H[1, 1], -H[1, 0]])
        v = B @ (w / np.linalg.norm(w))
        return np.array([np.linalg.det(H), np.sum(v ** 3 / (m * phi ** 2))])

    sol = optimize.root(eqs, np.asarray(guess, dtype=np.float64)[:2], method="hybr", tol=1e-14)
    if np.max(np.abs(eqs(sol.x))) > 1e-10:
        raise RuntimeError(f"critical point failed: {sol.message}")
    return np.array([sol.x[0], sol.x[1], 1.0 - sol.x[0] - sol.x[1]])
