"""Compile libctrex.so (sm_103a) in-tree with nvcc: one process per .cu file,
run in parallel, then a single shared-library link."""

import glob
import os
import platform
import struct
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build", platform.machine())
LIB = os.path.join(HERE, "libctrex.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    cand = os.environ.get("NVCC") or os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


_MACHINE = {"x86_64": 62, "AMD64": 62, "aarch64": 183, "arm64": 183}


def _native(path):
    """True if the ELF file at path was built for this machine."""
    try:
        with open(path, "rb") as f:
            head = f.read(20)
        return head[:4] == b"\x7fELF" and struct.unpack("<H", head[18:20])[0] == _MACHINE.get(platform.machine())
    except OSError:
        return False


def _stale(target, deps):
    if not os.path.exists(target) or not _native(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(extra_flags=(), verbose=False, lib=None, build_dir=None) -> str:
    """Build libctrex.so (or ``lib``, with objects in ``build_dir``) with the
    given extra nvcc flags."""
    global LIB, BUILD
    lib_path, build_path = LIB, BUILD
    if lib is not None:
        LIB, BUILD = lib, build_dir or os.path.join(os.path.dirname(lib), "_objs")
    try:
        return _build(extra_flags, verbose)
    finally:
        LIB, BUILD = lib_path, build_path


def _build(extra_flags, verbose) -> str:
    os.makedirs(BUILD, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))
    objs, procs = [], []
    for src in sources:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if _stale(obj, [src, __file__] + headers):
            cmd = [nvcc()] + ARCH + FLAGS + list(extra_flags) + ["-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd))
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(f"{s}:\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    if _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB
