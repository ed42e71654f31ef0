"""Builds libmf.so (CUDA kernels + C ABI) in-tree for sm_103a with nvcc.

Translation units compile in parallel into ``_build/`` and link into
``libmf.so`` beside this file.  ``build(checked=True)`` builds the checked
debug library instead (``-DMF_CHECKED``: every global access of the map
kernels is tested against its plane, and one outside is reported and
skipped) into ``_build_checked/`` and ``libmf_checked.so``; the binding
loads it when MF_CHECKED=1 is set.  A unit is rebuilt only when it or a header is
newer than its object.  Host code uses no architecture-specific intrinsics,
so the same sources build on x86_64 and aarch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["mf_map_kernel.cu", "mf_map_n8.cu", "mf_map_n16.cu", "mf_map_n32.cu", "mf_map_tc.cu", "mf_pose_kernels.cu", "mf_stream.cpp", "mf_noalloc.cu",
           "mf_engine.cpp", "mf_engine_kernels.cu", "mf_server.cpp", "mf_probe.cpp", "mf_fault.cpp", "mf_align.cu"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "mf.h"))
    return hs


def build(verbose=False, force=False, checked=False):
    build_dir = BUILD + "_checked" if checked else BUILD
    lib = os.path.join(HERE, "libmf_checked.so") if checked else LIB
    defs = ["-DMF_CHECKED"] if checked else []
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    newest_header = max(os.path.getmtime(h) for h in _headers())
    procs, objs = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(build_dir, src + ".o")
        objs.append(obj)
        if (not force and os.path.exists(obj)
                and os.path.getmtime(obj) >= max(os.path.getmtime(path), newest_header)):
            continue
        cmd = [nvcc, *ARCH, *defs, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", os.path.join(ROOT, "include"), "-c", path, "-o", obj]
        if src.endswith(".cpp"):
            cmd[1:1] = ["-x", "cu"]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append(src)
            sys.stderr.write(out.decode(errors="replace"))
        elif verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    if procs or not os.path.exists(lib):
        cuda_lib = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", lib + ".tmp", *objs,
               "-Xlinker", "-rpath," + cuda_lib]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv, checked="--checked" in sys.argv)
