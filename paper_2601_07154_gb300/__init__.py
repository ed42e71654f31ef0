"""GB300 (sm_103a) motion-focus maps for egocentric video streams.

Implements the data-parallel path of "Motion Focus Recognition in
Fast-Moving Egocentric Video" (arXiv 2601.07154): gravity-locked anchoring
of sliding pose batches (Section 2.2), motion points from camera poses
(Eqs. 1-6), the motion-focus map (Eq. 7) and the motion-guided depth map.
The work runs in hand-written CUDA kernels inside ``libmf.so``; this package
is its ctypes binding (``_mf``) plus a torch-facing wrapper (``stream``).
"""
from . import _mf  # noqa: F401  (raises ImportError if libmf.so is missing)
from ._mf import *  # noqa: F401,F403
from .stream import MotionFocusEngine, MotionFocusServer, MotionFocusStream  # noqa: F401
