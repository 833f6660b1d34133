"""Helpers for comparing the CUDA path (through the C ABI) with the CPU oracle."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O


def direction_map():
    """perm[i_gpu] = i_oracle for the same velocity vector."""
    from paper_2403_05443_gb300 import lbsph as L
    cg, _ = L.lb_lattice()
    co, _ = O.lattice()
    idx = {tuple(v): k for k, v in enumerate(co.tolist())}
    return np.array([idx[tuple(v)] for v in cg.tolist()])


def oracle_df_gpu_layout(sim: O.Sim, rho0=1.0):
    """Oracle pre-collision deviations in the GPU layout [19][nz][ny][nx] (fluid
    nodes; solid nodes 0)."""
    f = sim.f()                                      # [nz,ny,nx,19]
    _, w = O.lattice()
    own = sim.owner()
    df = f - w[None, None, None, :] * rho0
    df[own != 0] = 0.0
    perm = direction_map()
    return np.ascontiguousarray(np.moveaxis(df[..., perm], -1, 0))


def normwise(a, ref, floor=1e-9):
    """max |a - ref| / max(max |ref|, floor): the relative error of a field.  The
    floor keeps a quiescent box (deviations of 1e-17 from FP64 round-off in the
    oracle) from dividing by zero."""
    den = max(float(np.abs(ref).max()), floor)
    return float(np.abs(np.asarray(a, np.float64) - ref).max() / den)


def gpu_links_as_set(sim, box=0, p=0):
    from paper_2403_05443_gb300 import lbsph as L
    node, d = sim.links(box, p)
    c, _ = L.lb_lattice()
    return {(int(n), tuple(int(v) for v in c[b])) for n, b in zip(node, d)}


def oracle_links_as_set(sim: O.Sim, p=0):
    node, cv = sim.links(p)
    return {(int(n), tuple(int(v) for v in c)) for n, c in zip(node, cv)}
