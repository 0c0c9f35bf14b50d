"""FP64 CPU oracle of the reconstruction path — TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously correct restatement of what the
paper's method computes (Sec. 2.3-2.5): normal splat (Eqs. 23-25), divergence
right-hand side (Eqs. 22, 26), Poisson solve (Eqs. 15, 20-21), iso-value
(Eq. 27), marching cubes (Eq. 28), exact signed distance (Eqs. 29-34),
gradient normals (Sec. 2.4, below Eq. 32), query interpolation and the
adjoint chain (Eqs. 35-39).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline
may import it.  The CUDA library never calls it and shares no code, table or
constant generator with it; the only thing both sides use is the input
generator package ``synth``.

Floating point is FP64 throughout; float32 inputs are promoted to double.
Array layout: grids are numpy arrays indexed [z, y, x] (x fastest, matching a
C-order res^3 buffer); per-point integer cell coordinates are (x, y, z).
"""
from .pipeline import Reconstruction, reconstruct, query, backward  # noqa: F401
