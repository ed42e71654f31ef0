"""Pointer classification of the C ABI (host side, no GPU): device memory of
another GPU than the one a stream, engine or allocation-free call works on is
refused before any launch, since its kernels would fault reading it.  A box
with one GPU cannot produce such a pointer, so the rule itself is compiled
here from its header and checked against every memory type."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2601_07154_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "mf_ptr_kind.h"
int main() {
  // (memory type, attribute device, work device) -> kind
  const int cases[][4] = {
      {0, -2, 0, mf::kPtrHost},        // unregistered host memory
      {1, 0, 0, mf::kPtrHost},         // page-locked host memory
      {2, 0, 0, mf::kPtrDevice},       // this GPU
      {2, 1, 0, mf::kPtrOtherDevice},  // another GPU
      {2, 0, 3, mf::kPtrOtherDevice},
      {3, 1, 0, mf::kPtrDevice},       // managed memory (any device)
  };
  int bad = 0;
  for (const auto& c : cases)
    if (mf::classify_pointer(c[0], c[1], c[2]) != c[3]) {
      std::printf("case %d %d %d -> %d\n", c[0], c[1], c[2], mf::classify_pointer(c[0], c[1], c[2]));
      bad = 1;
    }
  return bad;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_other_gpu_memory_is_refused(tmp_path):
    src = tmp_path / "kind.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "kind"
    subprocess.run(["g++", "-std=c++17", "-I", HDR, str(src), "-o", str(exe)], check=True)
    assert subprocess.run([str(exe)]).returncode == 0
