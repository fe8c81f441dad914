"""Readers for the paper-transcribed fixtures in tests/golden/."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line


def frac(s: str) -> float:
    return float(Fraction(s))


def jump1d():
    """{k: coefficient vector over (a_{i-1}, a_i, a_{i+1}, a_{i+2}, m_{i-1}, ..., m_{i+2})}."""
    out = {}
    for line in _lines("jump1d.txt"):
        r = line.split()
        k, den = int(r[0]), float(r[1])
        out[k] = np.array([float(x) for x in r[2:]]) / den
    return out


def jump2d():
    """{(k, 'A'|'B'|'C'): 4x3 array}, rows s = -1..2, columns l = -1..1."""
    out, key, rows = {}, None, []
    for line in _lines("jump2d_ABC.txt"):
        if line.startswith("k="):
            if key:
                out[key] = np.array(rows)
            kk, name = line.split()
            key, rows = (int(kk[2:]), name), []
        else:
            rows.append([frac(x) for x in line.split()])
    out[key] = np.array(rows)
    return out


def fourier_D():
    """{(k, l): 2x2 array}."""
    out = {}
    for line in _lines("fourier_Dk.txt"):
        r = line.split()
        out[(int(r[0]), int(r[1]))] = np.array([frac(x) for x in r[2:]]).reshape(2, 2)
    return out


def fourier_modes():
    spur, phys, cfl = {}, {}, {}
    for line in _lines("fourier_modes.txt"):
        r = line.split()
        if r[0] == "spurious":
            spur[int(r[1])] = frac(r[2])
        elif r[0] == "physical":
            phys[int(r[1])] = (int(r[2]), complex(frac(r[3]), frac(r[4])))
        elif r[0] == "cfl":
            cfl[int(r[1])] = float(r[2])
    return spur, phys, cfl


def app_a():
    out = []
    for line in _lines("app_a_example.txt"):
        r = line.split()
        out.append(([frac(x) for x in r[:4]], r[4], float(r[5])))
    return out


def accuracy():
    """{(table, N): [FAM3, FAM4, FAM5, FAM6]}."""
    out = {}
    for line in _lines("accuracy.txt"):
        r = line.split()
        out[(r[0], int(r[1]))] = [float(x) for x in r[2:]]
    return out
