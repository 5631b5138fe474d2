"""Report: the paper's Sec. 4 binodal sweeps run by the FP64 oracle (CPU), against the
Flory-Huggins theory of oracle.thermo.  Not a test; it prints the tables that the build's
design notes quote and takes a few minutes on all host cores.

    python tests/paper_sweeps.py [--only binary|polymer|ternary]

Every run is a y-invariant flat interface (one row; the D2Q9 update then equals the
paper's D1Q3 lattice), started as two slabs at the theory's coexisting compositions, with
kappa = 0 as in the paper:
  * monomer binary, chi = 2.05 ... 3.0 at 1/tau = 0.7 and 0.9, 64 sites, 40 000 steps;
  * polymer binary m = (10, 1), chi = 0.9 ... 1.3, 1/tau = 0.9, 128 sites, 50 000 steps;
  * ternary chi_AB = 3, chi_AC = 0.5, chi_BC = 0.2, mean compositions on the line from the
    printed critical point toward (0.5, 0.5, 0) (monomer, and polymer m = (10, 1, 1)),
    1/tau = 0.9, 128 sites, 200 000 steps.
A run whose densities stop being finite is reported as diverging.  For the polymer binary the
total-density step between the phases is printed too (the paper reports < 1e-5).
"""
import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import Oracle, thermo  # noqa: E402


def slab_run(hi, lo, chi, m, steps, nx=128, itau=0.9):
    x = np.arange(nx)
    inside = (x >= nx // 4) & (x < 3 * nx // 4)
    phi = np.where(inside[None, :], np.asarray(hi)[:, None], np.asarray(lo)[:, None])
    o = Oracle(len(m), nx, 1, 1 / itau, chi, m=np.asarray(m, float))
    o.init(phi[:, None, :], np.zeros((2, 1, nx)))
    o.run(steps)
    r = o.moments()["rho"][:, 0, :]
    if not np.all(np.isfinite(r)):
        return None
    tot = r.sum(0)
    ph = r / tot
    mid, ends = slice(nx // 2 - 4, nx // 2 + 4), np.r_[0:4, nx - 4:nx]
    rich, poor = ph[:, mid].mean(1), ph[:, ends].mean(1)
    step = abs(tot[mid].mean() - tot[ends].mean()) / tot.mean()   # total density between phases
    return rich, poor, step


def binary():
    print("| chi | binodal phi_A (poor / rich) | rich plateau, 1/tau = 0.7 | 1/tau = 0.9 |")
    print("|---|---|---|---|")
    for chi_v in (2.05, 2.1, 2.2, 2.3, 2.4, 2.5, 2.6, 2.7, 2.8, 3.0):
        lo, hi = thermo.binodal_binary(chi_v)
        C = np.array([[0.0, chi_v], [chi_v, 0.0]])
        row = []
        for itau in (0.7, 0.9):
            r = slab_run([hi, 1 - hi], [lo, 1 - lo], C, [1, 1], 40000, nx=64, itau=itau)
            row.append("diverges" if r is None else f"{r[0][0]:.4f} ({r[0][0] - hi:+.4f})")
        print(f"| {chi_v} | {lo:.4f} / {hi:.4f} | {row[0]} | {row[1]} |", flush=True)


def polymer():
    print("| chi (m = (10, 1)) | binodal phi_A (poor / rich) | plateau errors (poor / rich) | drho/rho between phases |")
    print("|---|---|---|---|")
    for chi_v in (0.9, 0.94, 1.0, 1.1, 1.2, 1.3):
        lo, hi = thermo.binodal_binary(chi_v, 10.0, 1.0)
        C = np.array([[0.0, chi_v], [chi_v, 0.0]])
        r = slab_run([hi, 1 - hi], [lo, 1 - lo], C, [10, 1], 50000)
        res = "diverges | -" if r is None else f"{r[1][0] - lo:+.4f} / {r[0][0] - hi:+.4f} | {r[2]:.1e}"
        print(f"| {chi_v} | {lo:.4f} / {hi:.4f} | {res} |", flush=True)


def ternary():
    C3 = np.zeros((3, 3))
    C3[0, 1] = C3[1, 0] = 3.0
    C3[0, 2] = C3[2, 0] = 0.5
    C3[1, 2] = C3[2, 1] = 0.2
    end = np.array([0.5, 0.5, 0.0])
    for tag, m, pc in (("monomer", [1, 1, 1], [0.32, 0.32, 0.36]),
                       ("polymer m = (10, 1, 1)", [10, 1, 1], [0.14, 0.11, 0.75])):
        print(f"| s ({tag}) | max error of the rich plateau |")
        print("|---|---|")
        for s in np.arange(0.1, 1.0, 0.1):
            pb = np.asarray(pc) + s * (end - np.asarray(pc))
            try:
                q1, q2 = thermo.tie_line(C3, np.asarray(m, float), pb)
            except Exception:
                print(f"| {s:.1f} | no tie line |")
                continue
            hi, lo = (q1, q2) if q1[0] > q2[0] else (q2, q1)
            r = slab_run(hi, lo, C3, m, 200000)
            print(f"| {s:.1f} | " + ("diverges" if r is None else f"{np.abs(r[0] - hi).max():.4f}") + " |",
                  flush=True)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", choices=["binary", "polymer", "ternary"])
    a = ap.parse_args()
    for name, fn in (("binary", binary), ("polymer", polymer), ("ternary", ternary)):
        if a.only in (None, name):
            fn()
