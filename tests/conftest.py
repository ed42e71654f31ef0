import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """The largest GPU-vs-oracle coordinate (pixels) and map errors of the session."""
    parity = sys.modules.get("tests.parity")
    if parity is None:
        return
    rec = {k: {"max_du_px": v[0], "max_dv_px": v[1], "points": v[2]}
           for k, v in parity.COORD_ERR.items() if v[2]}
    if rec:
        terminalreporter.write_line("COORD_ERROR " + json.dumps(rec))
    maps = {k: {"max_rel": v[0], "max_abs": v[1], "pixels": v[2]} for k, v in parity.MAP_ERR.items() if v[2]}
    if maps:
        terminalreporter.write_line("MAP_ERROR " + json.dumps(maps))
