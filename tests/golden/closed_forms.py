"""Writes tests/golden/closed_forms.json: closed-form values that pin the oracle.

Everything here follows from the Lennard-Jones 12-6 pair potential
u(r) = 4 eps ((sigma/r)^12 - (sigma/r)^6) and geometry alone, evaluated in
40-digit decimal arithmetic.  It does not call the oracle or the CUDA path.
The paper names LJ molecules (§3) but prints no formula, so none of these
numbers is printed in it; each entry states its derivation.

  * two molecules: u(r) and the radial force f(r) = -du/dr
  * three molecules: equilateral triangle of side sigma, and three molecules
    on a line at the potential minimum spacing
  * perfect FCC at reduced density 0.8: lattice-shell sums for U/N and the
    pair virial sum_pairs r f(r) / N, and the number of pairs per molecule
  * N_c(x): cubes of a uniform cubic mesh with a corner within x w of a corner
    of the central cube (§2.4), counted over integer offsets
  * the k = 5 non-double-counting DIL loop order (App. A.1 table)
"""
import json
import os
from decimal import Decimal as D, getcontext

getcontext().prec = 40


def u(r):
    return 4 * (r ** -12 - r ** -6)


def f(r):
    return 24 * (2 * r ** -13 - r ** -7)


def cbrt(x):
    return x ** (D(1) / D(3))


def main():
    two = D(2) ** (D(1) / D(6))
    out = {"two_molecule": [], "source": __doc__.strip().splitlines()[0]}
    for name, r in (("minimum 2^(1/6)", two), ("sigma", D(1)), ("2.5", D("2.5")), ("3.0", D(3))):
        out["two_molecule"].append(dict(r=float(r), f=float(f(r)), u=float(u(r)), what=name))
    out["equilateral_side_1"] = dict(net_force=float(24 * D(3).sqrt()), U=0.0,
                                     why="each pair f(1) = 24 repulsive; two pairs at 60 degrees")
    r2 = 2 * two
    out["collinear_minimum"] = dict(spacing=float(two), U=float(-2 + u(r2)), end_force=float(f(r2)),
                                    why="neighbours sit at the minimum (f = 0); the end pair is 2^(7/6) apart")
    a = cbrt(D(4) / D("0.8"))
    shells = [(1, 12), (2, 6), (3, 24), (4, 12), (5, 24), (6, 8)]   # r^2 = (a^2/2) s, multiplicity
    fcc = {}
    for rc in (D("2.5"), D(3)):
        U = V = D(0)
        npair = 0
        for s, m in shells:
            r = (a * a / 2 * s).sqrt()
            if r < rc:
                U += D(m) * u(r) / 2
                V += D(m) * r * f(r) / 2
                npair += m
        fcc[str(rc)] = dict(U_per_N=float(U), virial_rf_per_N=float(V), pairs_per_N=npair // 2)
    out["fcc_rho08"] = dict(a=float(a), shells="r^2=(a^2/2)s, s=1..6, multiplicities 12,6,24,12,24,8",
                            **fcc)
    def n_c(x):
        n = 0
        R = 4
        for i in range(-R, R + 1):
            for j in range(-R, R + 1):
                for k in range(-R, R + 1):
                    g = sum(max(abs(t) - 1, 0) ** 2 for t in (i, j, k))
                    n += g < x * x
        return n
    out["N_c"] = {str(x): n_c(x) for x in (0.5, 0.877, 1.0965, 1.5, 2.2)}
    out["dil_k5"] = {str(i): list(range(i + 1, 5)) for i in range(5)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_forms.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
