"""Seeded synthetic inputs for the multicomponent lattice Boltzmann update.

This module only draws numbers and lays out initial fields; it holds none of
the method's arithmetic (no moments, potentials, equilibria or collisions), so
both the CUDA path and the FP64 CPU oracle can be fed from it.

Random numbers come from one portable counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): state_k = seed + k * 0x9E3779B97F4A7C15, followed by the
published three-step xor-shift/multiply finaliser.  A uniform double is the
top 53 bits of the output times 2**-53; Gaussian numbers use the Box-Muller
transform.  Every stream is identified by (seed, stream id), so the same seed
gives the same fields on any machine.

The workloads follow the paper's problem statement (Sec. 3, Eq. for the
per-component LBE; Sec. 4, Flory-Huggins free energy): N components on a
periodic D2Q9 lattice, one relaxation time, a symmetric interaction matrix
chi with zero diagonal (Sec. 4 sets the self interaction to zero), unit
polymerisation, total density 1 and zero initial velocity unless stated.

Fields are float64 arrays: rho has shape (N, ny, nx) (component, row, column;
x fastest), u has shape (2, ny, nx).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n outputs of SplitMix64 started at state seed + stream * 2**32."""
    with np.errstate(over="ignore"):
        base = np.uint64((int(seed) + (int(stream) << 32)) & 0xFFFFFFFFFFFFFFFF)
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = base + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1)."""
    return (splitmix64(seed, n, stream) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n standard normal doubles (Box-Muller on two uniform streams)."""
    u1 = uniform(seed, n, 2 * stream + 1000)
    u2 = uniform(seed, n, 2 * stream + 1001)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


@dataclass
class Problem:
    """One simulation: parameters of the paper's problem statement plus initial fields.

    chi is the symmetric N x N Flory-Huggins interaction matrix (Sec. 4),
    m the polymerisations, theta the Flory-Huggins temperature, kappa the
    gradient (interfacial) coefficient, tau the relaxation time of the BGK
    collision, force the body acceleration g.
    """
    name: str
    ncomp: int
    nx: int
    ny: int
    tau: float
    chi: np.ndarray
    m: np.ndarray
    theta: float
    kappa: float
    force: tuple
    rho: np.ndarray            # (N, ny, nx); (N, nz, ny, nx) on D3Q19
    u: np.ndarray              # (2, ny, nx); (3, nz, ny, nx) on D3Q19
    steps: int = 0
    precision: str = "fp32"
    meta: dict = field(default_factory=dict)
    forcing_velocity: int = 0      # 0: Eq. ff3 as printed, 1: barycentric reading
    lattice: str = "d2q9"          # or "d1q3" (ny = 1) or "d3q19"
    force_form: int = 0            # 0: Eq. definef as printed, 1: Gibbs-Duhem total (kappa = 0)
    nz: int = 1                    # layers (D3Q19)
    walls: int = 0                 # 1: solid walls in y (D2Q9)

    @property
    def sites(self) -> int:
        return self.nx * self.ny * self.nz


def uniform_chi(n: int, value: float) -> np.ndarray:
    """Pair interaction `value` between every two distinct components, zero diagonal."""
    chi = np.full((n, n), float(value))
    np.fill_diagonal(chi, 0.0)
    return chi


def chi_critical_pair(ma: float = 1.0, mb: float = 1.0) -> float:
    """Critical Flory-Huggins interaction of a binary pair with polymerisations ma, mb:
    (1/sqrt(ma) + 1/sqrt(mb))^2 / 2, i.e. 2 for two monomers.

    This is the *reading* used to turn "k x critical" into a number for every
    workload: k times the critical interaction of a pair of components.  (The
    equimolar-spinodal reading chi_c = N would put the five-component pairs up to
    chi = 7.5, far beyond the largest chi the paper runs, and there the method
    diverges within a few hundred steps.)
    """
    return 0.5 * (1.0 / math.sqrt(ma) + 1.0 / math.sqrt(mb)) ** 2


def _mass_neutral(noise: np.ndarray) -> np.ndarray:
    """Subtract the across-component mean so the component noises sum to zero per site."""
    return noise - noise.mean(axis=0, keepdims=True)


def _problem(name, ncomp, nx, ny, tau, chi, phi, *, m=None, theta=1.0 / 3.0, kappa=0.0,
             force=(0.0, 0.0), rho_total=1.0, steps=0, precision="fp32", meta=None) -> Problem:
    phi = np.asarray(phi, dtype=np.float64).reshape(ncomp, ny, nx)
    rho = np.ascontiguousarray(phi * rho_total)
    u = np.zeros((2, ny, nx), dtype=np.float64)
    m = np.ones(ncomp) if m is None else np.asarray(m, dtype=np.float64)
    return Problem(name=name, ncomp=ncomp, nx=nx, ny=ny, tau=float(tau),
                   chi=np.asarray(chi, dtype=np.float64), m=m, theta=float(theta),
                   kappa=float(kappa), force=tuple(float(g) for g in force), rho=rho, u=u,
                   steps=steps, precision=precision, meta=dict(meta or {}))


def binary_noise(nx=64, ny=64, *, chi=2.2, tau=1.0, kappa=0.01, amp=0.01, seed=1,
                 steps=1000, precision="fp64", name="binary_64x64") -> Problem:
    """Binary mixture, phi_A = 0.5 + U(-amp, amp), total density 1, zero velocity.

    Defaults: 64 x 64, chi_AB = 2.2 (1.1 x the critical 2), kappa = 0.01, tau = 1.
    """
    s = nx * ny
    phia = 0.5 + amp * (2.0 * uniform(seed, s) - 1.0)
    phi = np.stack([phia, 1.0 - phia]).reshape(2, ny, nx)
    return _problem(name, 2, nx, ny, tau, uniform_chi(2, chi), phi, kappa=kappa, steps=steps,
                    precision=precision)


def ternary_gauss(nx=256, ny=256, *, chi=2.4, tau=0.8, kappa=0.01, sigma=0.005, seed=2,
                  steps=5000, precision="fp32", name="ternary_256x256") -> Problem:
    """Ternary mixture, phi = 1/3 + N(0, sigma^2) made mass neutral per site.

    Defaults: 256 x 256, chi_ij = 2.4 (1.2 x the pair critical 2), tau = 0.8.
    """
    s = nx * ny
    noise = np.stack([sigma * gaussian(seed, s, k) for k in range(3)])
    phi = (1.0 / 3.0 + _mass_neutral(noise)).reshape(3, ny, nx)
    return _problem(name, 3, nx, ny, tau, uniform_chi(3, chi), phi, kappa=kappa, steps=steps,
                    precision=precision)


def ternary_droplets(nx=256, ny=256, *, chi=2.4, tau=0.8, kappa=0.01, sigma=0.005, seed=12,
                     ndrop=6, steps=100, precision="fp32", name="ternary_droplets") -> Problem:
    """The ternary workload's parameters (chi_ij = 2.4, tau = 0.8, kappa = 0.01) started
    phase separated: `ndrop` discs rich in component 0, phi = (0.8, 0.15, 0.05), in a
    matrix rich in component 1, (0.15, 0.8, 0.05), with tanh edges of width 2 and
    Gaussian noise sigma made mass neutral; disc centres and radii (8..24) drawn from
    the seed, periodic images included.  (At chi = 2.4 the A-B pair coexists near
    0.17 / 0.83, so the discs stay: a state with interfaces everywhere.)
    """
    s = nx * ny
    r = uniform(seed, 3 * ndrop, 5).reshape(ndrop, 3)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    inside = np.zeros((ny, nx))
    for k in range(ndrop):
        cx, cy, rad = r[k, 0] * nx, r[k, 1] * ny, 8.0 + 16.0 * r[k, 2]
        dx = np.minimum(np.abs(x - cx), nx - np.abs(x - cx))
        dy = np.minimum(np.abs(y - cy), ny - np.abs(y - cy))
        w = 0.5 * (1.0 - np.tanh((np.sqrt(dx * dx + dy * dy) - rad) / 2.0))
        inside = np.maximum(inside, w)
    a, b = np.array([0.8, 0.15, 0.05]), np.array([0.15, 0.8, 0.05])
    phi = a[:, None, None] * inside[None] + b[:, None, None] * (1.0 - inside[None])
    noise = np.stack([sigma * gaussian(seed, s, k) for k in range(3)]).reshape(3, ny, nx)
    phi = phi + _mass_neutral(noise)
    return _problem(name, 3, nx, ny, tau, uniform_chi(3, chi), phi, kappa=kappa, steps=steps,
                    precision=precision)


def random_chi(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Symmetric matrix chi_ij = chi_c * U[lo, hi] for i != j (chi_c the monomer pair
    critical value 2), zero diagonal."""
    r = uniform(seed, n * n, 77)
    chi = np.zeros((n, n))
    k = 0
    for i in range(n):
        for j in range(i + 1, n):
            v = chi_critical_pair() * (lo + (hi - lo) * r[k])
            chi[i, j] = chi[j, i] = v
            k += 1
    return chi


def multi_uniform(nx=2048, ny=2048, *, ncomp=5, tau=1.0, kappa=0.01, amp=0.01, seed=3,
                  steps=2000, precision="fp32", name="n5_2048x2048") -> Problem:
    """N-component mixture with a random symmetric chi in [0.8, 1.5] x critical.

    Defaults: N = 5 on 2048 x 2048, phi = 1/N + U(-amp, amp) mass neutral, tau = 1.
    """
    s = nx * ny
    noise = np.stack([amp * (2.0 * uniform(seed, s, k) - 1.0) for k in range(ncomp)])
    phi = (1.0 / ncomp + _mass_neutral(noise)).reshape(ncomp, ny, nx)
    return _problem(name, ncomp, nx, ny, tau, random_chi(ncomp, 0.8, 1.5, seed), phi,
                    kappa=kappa, steps=steps, precision=precision)


def multi_spinodal(nx=256, ny=256, *, ncomp=5, tau=1.0, kappa=0.01, amp=0.01, seed=3,
                   steps=2000, precision="fp32", name="n5_spinodal") -> Problem:
    """The N-component workload's interactions (random symmetric chi in [0.8, 1.5] x
    critical, same seed) with a mean composition inside the spinodal: the pair with the
    largest chi at 0.4 each, the other components sharing 0.2, plus mass-neutral uniform
    noise of amplitude `amp`.  (At the equimolar composition that chi set is stable; here
    the pair's composition mode grows and the mixture separates into two phases.)
    """
    chi = random_chi(ncomp, 0.8, 1.5, seed)
    a, b = np.unravel_index(np.argmax(chi), chi.shape)
    phi0 = np.full(ncomp, 0.2 / (ncomp - 2))
    phi0[a] = phi0[b] = 0.4
    s = nx * ny
    noise = np.stack([amp * (2.0 * uniform(seed + 17, s, k) - 1.0) for k in range(ncomp)])
    phi = (phi0[:, None] + _mass_neutral(noise)).reshape(ncomp, ny, nx)
    return _problem(name, ncomp, nx, ny, tau, chi, phi, kappa=kappa, steps=steps,
                    precision=precision, meta={"pair": (int(a), int(b))})


def slab(nx=8192, ny=2048, *, tau=1.0 / 0.9, kappa=0.01, amp=0.01, seed=5, steps=20000,
         precision="fp32", name="slab_8192x2048") -> Problem:
    """Polymer (P) / solvent (S) mixture 0.3/0.7 on the left half against pure
    non-solvent (NS) on the right; periodic in both directions.

    Component order (P, S, NS).  chi_{P,NS} = 3, chi_{P,S} = 0.5, chi_{S,NS} = 0.2
    (the paper's ternary parameter set, Sec. 4, mapped A->P, B->NS, C->S).  In the
    two columns on each side of both contacts the two states are blended with
    weight s = 1/2 + U(-amp, amp).
    """
    left = np.array([0.3, 0.7, 0.0])
    right = np.array([0.0, 0.0, 1.0])
    half = nx // 2
    wleft = np.zeros((ny, nx))
    wleft[:, :half] = 1.0
    r = uniform(seed, ny * 8).reshape(ny, 8)
    cols = [half - 2, half - 1, half, half + 1, nx - 2, nx - 1, 0, 1]
    for k, c in enumerate(cols):
        wleft[:, c % nx] = 0.5 + amp * (2.0 * r[:, k] - 1.0)
    phi = left[:, None, None] * wleft[None] + right[:, None, None] * (1.0 - wleft[None])
    chi = np.zeros((3, 3))
    P, S, NS = 0, 1, 2
    chi[P, NS] = chi[NS, P] = 3.0
    chi[P, S] = chi[S, P] = 0.5
    chi[S, NS] = chi[NS, S] = 0.2
    return _problem(name, 3, nx, ny, tau, chi, phi, kappa=kappa, steps=steps,
                    precision=precision)


def ternary3d(n=256, *, tau=1.0 / 0.9, kappa=0.01, amp=0.01, seed=6, steps=1000,
              precision="fp32", name="ternary3d_256") -> Problem:
    """Three components on an n^3 D3Q19 lattice with the paper's ternary chi set
    (chi_AB = 3, chi_AC = 0.5, chi_BC = 0.2, Sec. 4) at the mean composition
    (0.4, 0.4, 0.2), inside the A-B spinodal, plus mass-neutral uniform noise of amplitude
    `amp`: the mixture separates into A-rich and B-rich domains in three dimensions."""
    chi = np.zeros((3, 3))
    chi[0, 1] = chi[1, 0] = 3.0
    chi[0, 2] = chi[2, 0] = 0.5
    chi[1, 2] = chi[2, 1] = 0.2
    s = n * n * n
    noise = np.stack([amp * (2.0 * uniform(seed, s, k) - 1.0) for k in range(3)])
    phi = (np.array([0.4, 0.4, 0.2])[:, None] + _mass_neutral(noise)).reshape(3, n, n, n)
    return Problem(name=name, ncomp=3, nx=n, ny=n, tau=float(tau), chi=chi, m=np.ones(3),
                   theta=1.0 / 3.0, kappa=float(kappa), force=(0.0, 0.0, 0.0),
                   rho=np.ascontiguousarray(phi), u=np.zeros((3, n, n, n)), steps=steps,
                   precision=precision, lattice="d3q19", nz=n)


def flat_interface(phi0, *, chi, nx=128, ny=1, m=None, tau=1.0 / 0.9, kappa=0.0, amp=0.1,
                   rho_total=1.0, steps=50000, precision="fp64", name="flat") -> Problem:
    """Sinusoidal perturbation of a homogeneous mixture (Sec. 4): amplitude `amp`,
    wavelength the lattice size, added to component 0 and subtracted from
    component 1; any further components stay constant.  y-invariant.
    """
    phi0 = np.asarray(phi0, dtype=np.float64)
    n = phi0.size
    x = np.arange(nx)
    d = amp * np.sin(2.0 * math.pi * x / nx)
    phi = np.empty((n, ny, nx))
    for k in range(n):
        phi[k] = phi0[k]
    phi[0] += d[None, :]
    phi[1] -= d[None, :]
    return _problem(name, n, nx, ny, tau, chi, phi, m=m, kappa=kappa, rho_total=rho_total,
                    steps=steps, precision=precision)


def batch(count=512, *, seed=4, lo=32, hi=512, steps=1000, precision="fp32") -> List[Problem]:
    """Independent binary/ternary instances of uneven size.

    N uniform in {2, 3}; nx, ny independent uniform integers in [lo, hi];
    chi = s * chi_c with s ~ U[0.9, 1.6] (chi_c = 2, the pair critical value);
    tau ~ U[0.6, 1.5]; kappa = 0.01;
    initial fields as the binary (uniform noise 0.01) and ternary (Gaussian
    noise 0.005) recipes, each instance with its own seed.
    """
    r = uniform(seed, count * 5, 9).reshape(count, 5)
    out = []
    for k in range(count):
        n = 2 if r[k, 0] < 0.5 else 3
        nx = lo + int(r[k, 1] * (hi - lo + 1))
        ny = lo + int(r[k, 2] * (hi - lo + 1))
        s = 0.9 + 0.7 * r[k, 3]
        tau = 0.6 + 0.9 * r[k, 4]
        chi = s * chi_critical_pair()
        iseed = seed * 100003 + k
        if n == 2:
            p = binary_noise(nx, ny, chi=chi, tau=tau, kappa=0.01, seed=iseed, steps=steps,
                             precision=precision, name=f"batch{k}")
        else:
            p = ternary_gauss(nx, ny, chi=chi, tau=tau, kappa=0.01, seed=iseed, steps=steps,
                              precision=precision, name=f"batch{k}")
        out.append(p)
    return out


def random_state(ncomp, nx, ny, *, seed, amp=0.05, umax=0.05) -> tuple:
    """Generic positive densities and small velocities for parity cases.

    rho^sigma = (1 + amp * U(-1, 1)) / N, u = umax * U(-1, 1) per component of u.
    """
    s = nx * ny
    rho = np.stack([(1.0 + amp * (2.0 * uniform(seed, s, k) - 1.0)) / ncomp
                    for k in range(ncomp)]).reshape(ncomp, ny, nx)
    u = np.stack([umax * (2.0 * uniform(seed, s, 50 + k) - 1.0) for k in range(2)]).reshape(2, ny, nx)
    return np.ascontiguousarray(rho), np.ascontiguousarray(u)
