"""FP64 CPU oracle for the soft-shadow hot path.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package.  It is
independent of the CUDA path: it imports nothing from ``paper_2005_06671_gb300``
and shares no source with it.

* ``oracle.cref`` -- ctypes binding of ``shadow_oracle.c`` (C, FP64, OpenMP):
  brute force over every sample of every ray, the analytic gradient at the
  argmin, and the maximum mipmap.
  ``view_oracle.c`` adds the first terrain hit of a camera's view rays (the
  polar scene's ray origins); ``greedy_oracle.c`` restates the paper's greedy
  Algorithm 1 (an approximation, reproduced to measure its error);
  ``shade_oracle.c`` the Lambertian shading of the lit fractions.
* ``oracle.mini`` -- an independent NumPy restatement for tiny inputs, used to
  cross-check the C code.

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
(closed forms, Monte-Carlo disc area, brute-force block maxima, finite
differences, and the C-vs-NumPy cross-check); none is "parity unpinned".
"""
from .cref import (build_oracle, disc_light, shadow, shadow_svec, sun_vector, sample_uv,
                   ray_costs, sin_elev, grad, maxmip, num_threads, library_path, view_hits,
                   greedy, shade)

__all__ = ["build_oracle", "disc_light", "shadow", "shadow_svec", "sun_vector", "sample_uv",
           "ray_costs", "sin_elev", "grad",
           "maxmip", "num_threads", "library_path", "view_hits", "greedy", "shade"]
