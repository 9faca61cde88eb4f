"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package holds input generation only (terrain, sun directions, ray origins).
It contains none of the shadow method's arithmetic, imports neither the CUDA
package nor the oracle, and is the one module both sides may use.
"""
from .terrain import fbm, add_craters, lunar_tile, sun_list, random_origins
from .configs import (CONFIGS, MOON_RADIUS_M, SUN_ANGULAR_RADIUS_RAD, config,
                      make_instance, batched_instances, bump_target, camera,
                      POLAR_CAMERA, EARTH_LIGHT)

__all__ = ["fbm", "add_craters", "lunar_tile", "sun_list", "random_origins",
           "CONFIGS", "MOON_RADIUS_M", "SUN_ANGULAR_RADIUS_RAD", "config",
           "make_instance", "batched_instances", "bump_target", "camera", "POLAR_CAMERA",
           "EARTH_LIGHT"]
