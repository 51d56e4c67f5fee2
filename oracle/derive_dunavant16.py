"""Derive the 16-point, degree-8 fully symmetric triangle rule (Dunavant 1985).

Test infrastructure: this script writes nothing that the CUDA path reads; it
prints the rule so that the oracle's table (and, independently typed, the
kernel's table) can be checked against the moment equations.

The rule has the orbit structure 1 + 3*3 + 6: a centroid point, three
(a, a, 1-2a) orbits and one (a, b, 1-a-b) orbit, i.e. 10 unknowns.  A fully
symmetric rule is exact for all polynomials of degree <= 8 iff it is exact for
the 10 symmetric invariants e2^i e3^j (2i + 3j <= 8), with e2 = sum l_i l_j and
e3 = l1 l2 l3 in barycentric coordinates.  The exact averages over the
triangle follow from  mean(l1^a l2^b l3^c) = 2 a! b! c! / (a+b+c+2)!.

Newton's method in 50-digit arithmetic, started from the published 15-digit
values, converges to the rule to full double precision.

Run:  python oracle/derive_dunavant16.py
"""
import itertools

import mpmath as mp

mp.mp.dps = 50

INVARIANTS = [(i, j) for i in range(5) for j in range(3) if 2 * i + 3 * j <= 8]


def exact_mean(i, j):
    # expand e2^i e3^j into monomials in (l1, l2, l3) and average each
    total = mp.mpf(0)
    e2_terms = [(1, 1, 0), (0, 1, 1), (1, 0, 1)]
    for combo in itertools.product(range(3), repeat=i):
        ex = [j, j, j]
        for t in combo:
            for k in range(3):
                ex[k] += e2_terms[t][k]
        a, b, c = ex
        total += 2 * mp.factorial(a) * mp.factorial(b) * mp.factorial(c) / mp.factorial(a + b + c + 2)
    return total


def orbit_points(params):
    w0, a1, w1, a2, w2, a3, w3, a4, b4, w4 = params
    pts = [((mp.mpf(1) / 3,) * 3, w0)]
    for a, w in ((a1, w1), (a2, w2), (a3, w3)):
        c = 1 - 2 * a
        for p in ((a, a, c), (a, c, a), (c, a, a)):
            pts.append((p, w))
    c4 = 1 - a4 - b4
    for p in set(itertools.permutations((0, 1, 2))):
        lam = [a4, b4, c4]
        pts.append(((lam[p[0]], lam[p[1]], lam[p[2]]), w4))
    return pts


def residual(params):
    pts = orbit_points(params)
    res = []
    for (i, j) in INVARIANTS:
        s = mp.mpf(0)
        for (l1, l2, l3), w in pts:
            e2 = l1 * l2 + l2 * l3 + l3 * l1
            e3 = l1 * l2 * l3
            s += w * e2 ** i * e3 ** j
        res.append(s - exact_mean(i, j))
    return res


START = [0.144315607677787, 0.459292588292723, 0.095091634267285,
         0.170569307751760, 0.103217370534718, 0.050547228317031,
         0.032458497623198, 0.008394777409958, 0.263112829634638,
         0.027230314174435]


def derive():
    x = mp.matrix([mp.mpf(v) for v in START])
    for _ in range(30):
        f = mp.matrix(residual(list(x)))
        jac = mp.matrix(len(INVARIANTS), len(x))
        for k in range(len(x)):
            h = mp.mpf(10) ** -30
            xp = x.copy()
            xp[k] += h
            fp = mp.matrix(residual(list(xp)))
            for r in range(len(INVARIANTS)):
                jac[r, k] = (fp[r] - f[r]) / h
        dx = mp.lu_solve(jac, -f)
        x += dx
        if mp.norm(dx) < mp.mpf(10) ** -40:
            break
    return list(x)


if __name__ == "__main__":
    sol = derive()
    names = ["w0", "a1", "w1", "a2", "w2", "a3", "w3", "a4", "b4", "w4"]
    for n, v in zip(names, sol):
        print(f"{n} = {mp.nstr(v, 25)}")
    print("max residual:", mp.nstr(max(abs(r) for r in residual(sol)), 5))
