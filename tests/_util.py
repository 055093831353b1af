"""Shared comparison helpers for the parity tests."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# FP32 storage and arithmetic against the FP64 oracle: relative L2 error per
# field after 100 steps, and particle positions in lattice units.
FIELD_RTOL = 1e-5
POS_ATOL = 1e-6


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    num = np.linalg.norm((a - b).ravel())
    if den == 0.0:
        return num
    return num / den


def velocity_rel_l2(sim_fields, orc_fields):
    a = np.stack(sim_fields)
    b = np.stack(orc_fields)
    return rel_l2(a, b)


def build_library():
    from paper_1502_01159_gb300 import build
    return build.build()
