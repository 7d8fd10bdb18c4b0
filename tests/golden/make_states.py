"""Prints the post-shock boundary states stored in ``workloads.py``.

Calls only the oracle (Rankine-Hugoniot relations at gamma = 2):
    python tests/golden/make_states.py
"""
import math
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

from oracle import exact  # noqa: E402

r, u, v, p = exact.oblique_shock(1.0, 2.9 * math.sqrt(2.0), 0.0, 1.0, math.radians(30.0))
print("REFLECT_M29_TOP = (%r, %r, %r, %r)" % (r, u, v, p / r))
r, u, v, p = exact.moving_shock(1.0, 1.0, 1.22, (-1.0, 0.0))
print("bubble post-shock (rho, u, v, p) = (%r, %r, %r, %r)" % (r, u, v, p))
