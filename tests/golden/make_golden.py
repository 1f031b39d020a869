"""Writes the closed-form fixtures in this directory.

Each value is derived from geometry alone (no oracle call):
* two_charges.json  - Eq. 3 (Sec. 3.1): F_ij = r q_i q_j / (4 pi r^3), r = x_i - x_j.
* cube_corners.json - eight unit charges on a unit cube (Eq. 3 units): each
  corner sees 3 neighbours at distance 1, 3 at sqrt(2), 1 at sqrt(3).
Run: python tests/golden/make_golden.py
"""
import json
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def two_charges():
    x = [[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]]
    q = [1.0, 2.0]
    c = 1.0 / (4.0 * math.pi)
    pot = [c * q[1] / 1.0, c * q[0] / 1.0]
    # F_01 = (x0 - x1) q0 q1 / (4 pi r^3) with r = 1
    f0 = [-(c * q[0] * q[1]), 0.0, 0.0]
    f1 = [c * q[0] * q[1], 0.0, 0.0]
    return {"cite": "Eq. 3, Sec. 3.1", "x": x, "q": q, "pot": pot, "force": [f0, f1]}


def cube_corners():
    x = [[i, j, k] for i in (0.0, 1.0) for j in (0.0, 1.0) for k in (0.0, 1.0)]
    c = 1.0 / (4.0 * math.pi)
    pot = c * (3.0 + 3.0 / math.sqrt(2.0) + 1.0 / math.sqrt(3.0))
    # per-axis pull of the outward diagonal: edges 1, faces 2 * (1 / (2 sqrt 2)), body 1 / (3 sqrt 3)
    comp = c * (1.0 + 1.0 / math.sqrt(2.0) + 1.0 / (3.0 * math.sqrt(3.0)))
    return {"cite": "Eq. 3, Sec. 3.1", "x": x, "pot_each": pot, "force_mag": comp * math.sqrt(3.0)}


if __name__ == "__main__":
    for name, fn in (("two_charges.json", two_charges), ("cube_corners.json", cube_corners)):
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(fn(), f, indent=1)
            f.write("\n")
