"""Pins of the oracle's directional estimator (Sec. 4.1, Eq. 9-10)."""
import json
import os

import numpy as np

import oracle as O
from synth import meshes as M
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_fig1a_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "fig1a_lout.json")))
    r = [c[0] for c in g["crossings"]]
    s = [c[1] for c in g["crossings"]]
    assert O.l_out(g["r_e"], r, s, g["chi_o"]) == g["l_out"]
    # the same ray seen from outside the solid: no crossing before p_e and an
    # outside start leave the whole segment outside
    assert O.l_out(3.0, [], [], 0) == 3.0


def _box(c, R, half):
    return np.concatenate([c, R[0], R[1], half])


def test_empty_box_gives_its_volume():
    m = M.icosphere(2, radius=0.3)
    rng = np.random.Generator(np.random.PCG64(2))
    R = pins.random_rotation(rng)
    half = np.array([0.4, 0.25, 0.15])
    est = O.directional_outer_volume(m.verts, m.tris, _box([3.0, 0.0, 0.0], R, half), m=24)
    assert abs(est - 8 * half.prod()) <= 0.02 * 8 * half.prod()


def test_box_inside_solid_is_zero():
    m = M.icosphere(3, radius=1.0)
    est = O.directional_outer_volume(m.verts, m.tris, _box([0.05, 0.0, -0.05], np.eye(3), [0.3, 0.2, 0.25]), m=12)
    assert abs(est) < 1e-12


def test_sphere_in_its_bounding_cube():
    m = M.icosphere(3, radius=1.0)
    V = m.verts.astype(np.float64)
    F = m.tris.astype(np.int64)
    poly = abs(pins.polyhedron_volume(V, F))
    ext = V.max(0) - V.min(0)
    est = O.directional_outer_volume(m.verts, m.tris, _box((V.max(0) + V.min(0)) / 2, np.eye(3), ext / 2), m=24)
    exact = ext.prod() - poly
    assert abs(est - exact) <= 0.03 * exact
