"""Pins for the oracle's diffraction filters (Sec. III-D): the field of view around the emitter's forward
axis, the incidence constraint on the candidate triangle's normal and the line of sight to the emitter.

A floor quad (z = 0, normal +z) and a small box; the emitter 1 m above the origin.  Every candidate is
placed so that the answer is clear from the geometry, far from any threshold (angles in degrees between
the direction from the emitter to the candidate and the forward axis, and between the direction from the
candidate to the emitter and the floor's normal):
  A (2, 0.5):   29 deg off the forward axis +x, 64 deg from the normal, clear line of sight
  B (-2, 0.5):  behind the emitter (151 deg off +x), otherwise as A
  C (10, 1):    8 deg off +x, 84 deg from the normal (grazing: beyond 80, within 85)
  D (2, -0.5):  as A, but the box sits on the segment to the emitter
  E (1, 1.5):   61 deg off +x, 43 deg off +y, 61 deg from the normal, clear
  F (0.3, 3):   85 deg off +x, 19 deg off +y, 72 deg from the normal, clear.
A filter that reversed the direction of the field of view, dropped the incidence constraint or the line
of sight, or ignored the emitter's orientation fails one of the cases below."""
import math

import numpy as np

import oracle
import synth

EMITTER = np.array([0.0, 0.0, 1.0], np.float32)
POINTS = {"A": (2.0, 0.5), "B": (-2.0, 0.5), "C": (10.0, 1.0), "D": (2.0, -0.5), "E": (1.0, 1.5), "F": (0.3, 3.0)}


def _scene():
    fv = np.array([[-20, -20, 0], [20, -20, 0], [20, 20, 0], [-20, 20, 0]], np.float32)
    ft = np.array([[0, 1, 2], [0, 2, 3]], np.int32)  # triangle 0: y <= x, triangle 1: y >= x
    bv, bt, _ = synth._box_tris((0.8, -0.45, 0.3), (1.2, -0.05, 0.7))  # holds (1, -0.25, 0.5), D's midpoint
    return oracle.Scene(np.concatenate([fv, bv]), np.concatenate([ft, bt + 4]))


def _keep(q, **kw):
    sc = _scene()
    names = list(POINTS)
    cp = np.array([[x, y, 0.0] for x, y in POINTS.values()], np.float32)
    ct = np.array([0 if y <= x else 1 for x, y in POINTS.values()], np.int32)
    k = oracle.diffraction_filter(sc, EMITTER, np.asarray(q, np.float32), ct, cp, **kw)
    return {n: bool(v) for n, v in zip(names, k)}


IDENT = (1.0, 0.0, 0.0, 0.0)
TO_Y = (math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4))  # +x turned to +y


def test_field_of_view_incidence_and_line_of_sight():
    k = _keep(IDENT, fov_half=math.radians(45.0))
    assert k == {"A": True, "B": False, "C": False, "D": False, "E": False, "F": False}


def test_field_of_view_off():
    k = _keep(IDENT)  # half-angle pi: every direction
    assert k == {"A": True, "B": True, "C": False, "D": False, "E": True, "F": True}


def test_wider_incidence_limit_admits_the_grazing_candidate():
    k = _keep(IDENT, theta_inc_deg=85.0)
    assert k["C"] and not k["D"]


def test_forward_axis_follows_the_emitter_orientation():
    k = _keep(TO_Y, fov_half=math.radians(30.0))
    assert k["F"] and not k["A"] and not k["B"] and not k["C"] and not k["E"]
