"""FP64 CPU oracle for the collision-aware local-global soft-robot loop.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
``cpu_baseline`` / reference leg of the benchmark may import this package.
The product path (the CUDA library and its Python binding) never calls it and
shares no code with it; the two meet only in the seeded input generator.

What it computes, step by step (paper: Fang, Tian, Weightman, Wang,
"Collision-Aware Fast Simulation for Soft Robots by Optimization-Based
Geometric Computing"):

* ``mesh``      -- element quantities: centering N (Eq. 1), rest shapes, volumes,
                   boundary faces and surface vertices (Sec. II-A).
* ``local``     -- local projection: rotation by SVD (Sec. II-A), chamber target
                   (Sec. III-A.1), body blend + volume scaling (Eq. 6, Eq. 7).
* ``collision`` -- brute-force collision definition (Sec. II-B, Eq. 3, Eq. 4)
                   with exact orientation predicates.
* ``springs``   -- virtual-spring targets and release (Sec. II-C, Eq. 5,
                   Sec. III-A.3 release condition).
* ``global_step`` -- the least-squares global step of Eq. 8, solved exactly.
* ``loop``      -- the inner while-loop of Algorithm 1 run for n iterations.
* ``adjoint``   -- reverse-mode derivative of the unrolled loop w.r.t. the
                   chamber volume ratios.
* ``remesh``    -- the remesh trigger of Sec. III-C (volume change and
                   distortion of chamber elements) and Algorithm 1's outer
                   loop of progressive actuation (without remeshing).
* ``anderson``  -- Anderson acceleration of the loop (Sec. III-B) with an
                   energy safeguard.

Parity pins: every function is pinned by tests under ``tests/`` against
closed forms, invariants, brute force or library routines; functions without
such a pin say "parity unpinned" in their docstring.
"""
from . import mesh, local, collision, springs, global_step, loop, remesh, anderson  # noqa: F401
# ``oracle.adjoint`` needs PyTorch and is imported on demand.
