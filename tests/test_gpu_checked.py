"""The checked debug library (MF_CHECKED=1): the same renders through it and
through the release library, each in a fresh process.  With every index in
range, the checked library reports no caught access (every wait returns
MF_OK) and its outputs equal the release library's bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_catches_nothing_and_changes_nothing(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_mf_build", os.path.join(ROOT, "paper_2601_07154_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    b.build(checked=True)
    runs = {}
    for name, flag in (("release", None), ("checked", "1")):
        env = dict(os.environ)
        env.pop("MF_CHECKED", None)
        if flag:
            env["MF_CHECKED"] = flag
        path = str(tmp_path / f"{name}.npz")
        subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_run.py"), path],
                       cwd=ROOT, env=env, check=True, timeout=600)
        runs[name] = np.load(path)
    assert str(runs["release"]["lib"]) == "libmf.so"
    assert str(runs["checked"]["lib"]) == "libmf_checked.so"
    keys = [k for k in runs["release"].files if k != "lib"]
    assert len(keys) > 10
    for k in keys:
        assert np.array_equal(runs["release"][k], runs["checked"][k], equal_nan=True), k
    assert any(runs["release"][k].any() for k in keys if k.endswith("_M"))
