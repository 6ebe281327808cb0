"""Readers for tests/golden (plain text, '#' comments)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


def table1():
    r = rows("table1_angles.txt")
    return [float(x[1]) for x in r], [float(x[2]) for x in r]


def table2():
    return {int(x[0]): (float(x[1]), float(x[2])) for x in rows("table2_energies.txt")}


def philox_kat():
    return [([int(v, 16) for v in x[:4]], [int(v, 16) for v in x[4:6]],
             [int(v, 16) for v in x[6:10]]) for x in rows("philox_kat.txt")]


def gaussian_cz():
    return {x[0]: float(x[1]) for x in rows("gaussian_cz.txt")}
