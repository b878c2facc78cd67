"""Distance-ratio accuracy experiment of Sec. 4 (Figs. 8 and 9), run on the
oracle: random unit-cube elements, a random field-point direction from the
centroid at a fixed distance ratio DR = D / L, the average relative error of
each cubature rule against the GL2 reference (Sec. 2), with the paper's error
definitions (Sec. 2): err(phi) = |phi - phi_GL2| / |phi_GL2| and
err(E) = sum_j |E_j - E_j,GL2| / |E_GL2|.

TEST INFRASTRUCTURE: calls only the oracle and the seeded generators.

Run as a script to print the error table and the rule-band limits that meet
a target:  python -m oracle.dr_experiment [--target 2e-15] [--elements 1000]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

import synth
from . import METHOD_GL2, METHOD_RULE, element_batch, element_geometry


def errors(type_: int, dr: float, n_el: int = 1000, seed: int = 0):
    """Mean err(phi) and err(E) for the five rules of one element type at one
    distance ratio; returns (5, 2)."""
    verts = synth.random_elements(type_, n_el, seed)
    dirs = synth.random_directions(n_el, seed)
    P = np.zeros((n_el, 3))
    for i in range(n_el):
        g = element_geometry(type_, verts[i])
        P[i] = g["centroid"] + dr * g["L"] * dirs[i]
    types = np.full(n_el, type_, np.int32)
    ref, _ = element_batch(types, verts, P, METHOD_GL2, 16)
    out = np.zeros((5, 2))
    for r in range(5):
        cub, _ = element_batch(types, verts, P, METHOD_RULE, r)
        ephi = np.abs(cub[:, 0] - ref[:, 0]) / np.abs(ref[:, 0])
        eE = np.abs(cub[:, 1:] - ref[:, 1:]).sum(1) / np.linalg.norm(ref[:, 1:], axis=1)
        out[r] = ephi.mean(), eE.mean()
    return out


def table(type_: int, drs, n_el: int = 1000, seed: int = 0) -> np.ndarray:
    """(len(drs), 5, 2) mean errors."""
    return np.stack([errors(type_, float(d), n_el, seed + 17 * i) for i, d in enumerate(drs)])


def limits_from_table(drs, tab, target: float, which: int, near: float = 3.0) -> list[float]:
    """Smallest DR from which each rule stays at or below `target`
    (which = 0: phi, 1: E, 2: both); returned as the ascending band limits
    [near, lim33, lim19/17, lim12, lim7] with each limit at least the one
    below it."""
    drs = np.asarray(drs)
    lim = []
    for r in range(5):
        e = tab[:, r, :2].max(1) if which == 2 else tab[:, r, which]
        ok = e <= target
        # smallest DR such that every DR above it is ok
        idx = len(drs)
        for k in range(len(drs) - 1, -1, -1):
            if not ok[k]:
                break
            idx = k
        lim.append(float(drs[idx]) if idx < len(drs) else float("inf"))
    # rule r = 0 (4 points) ... 4 (33 points); bands ascending by DR
    out = [near, max(near, lim[3]), lim[2], lim[1], lim[0]]
    for k in range(1, 5):
        out[k] = max(out[k], out[k - 1])
    out[1] = max(out[1], near)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--target", type=float, default=2e-15)
    ap.add_argument("--elements", type=int, default=1000)
    ap.add_argument("--points", type=int, default=60)
    ap.add_argument("--seed", type=int, default=11)
    a = ap.parse_args()
    drs = np.geomspace(2.0, 10000.0, a.points)
    res = {}
    for t, name in ((0, "triangle"), (1, "rectangle")):
        tab = table(t, drs, a.elements, a.seed)
        print(f"# {name}: mean err(phi) | mean err(E) per rule (N = {'4 7 12 19 33' if t == 0 else '4 7 12 17 33'})")
        for i, d in enumerate(drs):
            print(f"DR {d:9.2f}  " + "  ".join(f"{tab[i, r, 0]:.1e}|{tab[i, r, 1]:.1e}" for r in range(5)))
        res[name] = {"phi": limits_from_table(drs, tab, a.target, 0), "E": limits_from_table(drs, tab, a.target, 1),
                     "both": limits_from_table(drs, tab, a.target, 2)}
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
