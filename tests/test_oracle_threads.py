"""The oracle's host threads change no result: its parallel loops write disjoint outputs with
the same operations in the same order as one thread (no GPU)."""
import os

import numpy as np

import oracle as mb
from paper_1407_5600_gb300 import workloads as wl


def _run_all():
    spec, s = wl.dense_suspension(n=16, a=2.2, phi=0.3, seed=9, mc_sweeps=1)
    g = mb.Grid(16, 16, 16, dt=0.05, mean_mode=0, advection=1)
    v0 = wl.random_field(g.shape, 5, scale=1e-3)
    out = list(mb.step(g, 2, s.pos, v0, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut,
                       body=s.body, kT=1e-3, seed=3))
    out += list(mb.stokes_step(mb.Grid(16, 16, 16, dt=0.05, mean_mode=1), 2, s.pos, s.pid,
                               s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut, body=s.body))
    out.append(mb.pair_forces_subset(g, s.pos, s.pid, 100.0, 2.5, np.arange(0, s.n_blobs, 7)))
    out.append(mb.dft3(v0[0] + 1j * v0[1]))
    return out


def test_thread_count_changes_no_bit():
    before = mb.set_threads(0)
    try:
        mb.set_threads(1)
        one = _run_all()
        mb.set_threads(max(4, os.cpu_count() or 4))
        many = _run_all()
    finally:
        mb.set_threads(before)
    for a, b in zip(one, many):
        assert np.array_equal(a, b)
