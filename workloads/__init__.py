"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the benchmark.

This package only *makes inputs*: triangle soups shaped like the paper's geometries and initial
flow fields.  It holds none of the method's arithmetic (no classification, no stencils, no solver)
so that the oracle and the CUDA path stay independent of each other.
"""
from .soups import (icosphere, axis_box, dirty_sphere, cube_and_plate, vehicle_assembly,
                    fan_disk, random_soup, prism_2d, taylor_green_body)
from .configs import CONFIGS, Config, get_config, initial_fields, taylor_green, taylor_green_velocity

__all__ = ["icosphere", "axis_box", "dirty_sphere", "cube_and_plate", "vehicle_assembly",
           "fan_disk", "random_soup", "CONFIGS", "Config", "get_config", "initial_fields",
           "taylor_green", "prism_2d", "taylor_green_body", "taylor_green_velocity"]
