"""Seeded synthetic inputs for the motion-focus path.

This package is shared by the FP64 oracle tests, the GPU parity tests and the
benchmark.  It generates inputs only -- walker camera trajectories, a box
scene and its ray-cast z-depth -- and holds none of the motion-focus method's
own arithmetic (no pose inversion for camera centres, no differencing, no
projection of motion directions, no Gaussian maps).

The paper's own inputs come from a handheld-phone dataset (Section 2.1,
Table 1) run through a depth/pose foundation model (Section 2.2); neither is
available, so these generators stand in for them with the shapes, rates and
motion statistics that the paper describes (walking at 30 fps, head sway,
turns, 320x240 .. 3840x2160 frames).
"""
from .rng import Xoshiro256ss, splitmix64  # noqa: F401
from .walker import WalkerSpec, walk  # noqa: F401
from .scene import Box, make_scene, render_depth  # noqa: F401
from .workloads import (  # noqa: F401
    StreamWorkload,
    small_stream,
    hd_stream,
    mixed_streams,
)
