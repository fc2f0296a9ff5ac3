"""Writes the oracle regression fixtures of this directory (calls only the
FP64 oracle and the seeded input generators).

Each fixture freezes the oracle's output for a small case: receiver, path
count, receiver flags, then per frequency the field (re, im of E_x, E_y,
E_z).  tests/test_oracle_golden.py checks that the oracle still reproduces
them, so that any later change to the oracle's arithmetic shows up and has
to be justified (and the fixtures rewritten with this script).

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_2310_10578_gb300 import scenes  # noqa: E402


def cases():
    """(name, citation, scene) of every fixture."""
    ring = scenes.sphere_ring(n_rx=4096)
    ring = ring.subset(np.arange(0, 4096, 128), ring.name)
    room = scenes.room(n_cyl=6, nx=8, ny=6, freqs=(2.4e9, 28e9), seed=5)
    walls = (5.31, 0.48)
    ext = scenes.room(n_cyl=6, nx=8, ny=6, freqs=(2.4e9, 28e9), seed=5,
                      face_eps=[(4.0, 0.2), None, walls, walls, walls, walls])
    ext.max_enc = 1
    ext.wall_creep = True
    office = scenes.office(n_rooms=(2, 2), n_furn=40, n_cyl=6, n_sph=3, n_tx=1, nx=8, ny=6, freqs=(5.8e9,))
    office.candidates = oracle.candidates(office, 4096, 3)
    return [
        ("sphere_ring", "PEC sphere, direct + GO reflection + first creeping rays (Eqs. 1-4, Sec. IV.A setting)", ring),
        ("room", "PEC room with 6 cylinders, planar reflections <= 2 (Eq. 3) and body paths (Eqs. 3-4)", room),
        ("room_extended", "the same room with dielectric faces, one extra turn and wall -> creeping paths", ext),
        ("office_small", "small office, orders 1-3 from the 4096-ray candidate list, BVH-free brute force", office),
    ]


def render(name, cite, sc):
    r = oracle.evaluate(sc)
    lines = ["# %s -- FP64 oracle output; %s" % (name, cite),
             "# scene: %s" % sc.name,
             "# written by tests/golden/make_golden.py (oracle/ only)",
             "# columns: receiver, path count, flags, then per frequency re/im of E_x, E_y, E_z"]
    for i in range(sc.n_rx):
        row = ["%d" % i, "%d" % r.counts[i], "%d" % r.flags[i]]
        for f in range(len(sc.freqs)):
            for q in range(3):
                row.append("%.17e" % r.E[f, q, i].real)
                row.append("%.17e" % r.E[f, q, i].imag)
        lines.append(" ".join(row))
    return "\n".join(lines) + "\n"


def main():
    for name, cite, sc in cases():
        with open(os.path.join(HERE, name + ".txt"), "w") as fh:
            fh.write(render(name, cite, sc))
        print("wrote", name)


if __name__ == "__main__":
    main()
