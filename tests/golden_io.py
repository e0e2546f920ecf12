"""Readers for the small text fixtures under tests/golden/."""
from __future__ import annotations

import os
from fractions import Fraction

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                yield [c.strip() for c in line.split("|")]


def ksg_hand_cases():
    out = []
    for name, k, x, y, eps, nx, ny, mi in _rows("ksg_hand.txt"):
        out.append(dict(name=name, k=int(k), x=[float(t) for t in x.split()],
                        y=[float(t) for t in y.split()], eps=[float(t) for t in eps.split()],
                        nx=[int(t) for t in nx.split()], ny=[int(t) for t in ny.split()],
                        mi=Fraction(mi)))
    return out


def ksg2_hand_cases():
    out = []
    for name, k, x, y, ex, ey, nx, ny, mi in _rows("ksg2_hand.txt"):
        f = lambda t: [float(u) for u in t.split()]
        i = lambda t: [int(u) for u in t.split()]
        out.append(dict(name=name, k=int(k), x=f(x), y=f(y), ex=f(ex), ey=f(ey), nx=i(nx),
                        ny=i(ny), mi=Fraction(mi)))
    return out


def pearson_hand_cases():
    out = []
    for x, y, num, den_sq in _rows("pearson_hand.txt"):
        out.append(dict(x=[float(t) for t in x.split()], y=[float(t) for t in y.split()],
                        r=float(num) / float(den_sq) ** 0.5))
    return out
