"""FP64 CPU oracle of the motion-focus path -- TEST INFRASTRUCTURE ONLY.

Importable only from ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py``.  The product library never loads
it, and it shares no code with the CUDA path.
"""
from .motion_focus import *  # noqa: F401,F403
from .motion_focus import (  # noqa: F401
    OracleStream, Params, FramePoints, ls_weights, ls_weights_exact, camera_centre,
    anchor_transform, compensated_intrinsics, frame_points, focus_map, guided_depth,
    map_argmax, focus_pixel, is_rigid, rot_y, to4x4,
)
