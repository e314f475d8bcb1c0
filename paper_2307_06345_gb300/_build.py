"""In-tree build of the CUDA library ``libcstone.so`` for sm_103a (nvcc, no CMake).

Each ``csrc/*.cu`` translation unit is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and the objects are linked into one
shared library next to this file. The runtime is linked dynamically, so inside a process that
already loaded PyTorch the library shares PyTorch's CUDA runtime.

Tile shapes are compile-time knobs; ``tuning.json`` (written by ``autotune.py`` on the target GPU)
holds the chosen values, which become ``-D`` definitions of every translation unit.
"""
from __future__ import annotations

import concurrent.futures
import glob
import json
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libcstone.so")
OBJDIR = os.path.join(HERE, "_build")
TUNING = os.path.join(HERE, "tuning.json")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# knob name in tuning.json -> preprocessor definition
KNOBS = {("sort", "threads"): "CSTONE_SORT_THREADS", ("sort", "items"): "CSTONE_SORT_ITEMS",
         ("sort", "min_blocks"): "CSTONE_SORT_MIN_BLOCKS", ("leaves", "items"): "CSTONE_LEAVES_ITEMS"}


def tuned_knobs() -> dict:
    """{definition: value} from tuning.json (empty when the file is absent)."""
    if not os.path.exists(TUNING):
        return {}
    with open(TUNING) as f:
        t = json.load(f)
    out = {}
    for (group, key), name in KNOBS.items():
        v = t.get("choice", {}).get(group, {}).get(key)
        if v is not None:
            out[name] = int(v)
    return out


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcstone.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


# Translation units that do not depend on the key length; every other one is compiled twice, for
# 63-bit keys (entry points cstone_*) and with CSTONE_KEY32 for 30-bit keys (cstone30_*).
KEY_INDEPENDENT = {"status.cu", "decompose.cu"}


def _units():
    """(source, object name, extra definitions) of every object of the library."""
    out = []
    for src in _sources():
        base = os.path.basename(src)[:-3]
        out.append((src, base + ".o", {}))
        if os.path.basename(src) not in KEY_INDEPENDENT:
            out.append((src, base + "30.o", {"CSTONE_KEY32": 1}))
    return out


def _deps():
    deps = _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(INCLUDE, "cstone.h")]
    return deps + ([TUNING] if os.path.exists(TUNING) else [])


def is_stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in _deps())


def _flags(knobs: dict):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I", INCLUDE,
                   "-I", CSRC, "--expt-relaxed-constexpr", "-DCSTONE_BUILD"] + [f"-D{k}={v}" for k, v in knobs.items()]


def _compile(units, objdir: str, knobs: dict, verbose: bool = False):
    os.makedirs(objdir, exist_ok=True)
    cc = nvcc()

    def compile_one(unit):
        src, name, extra = unit
        obj = os.path.join(objdir, name)
        cmd = [cc] + _flags({**knobs, **extra}) + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(12, os.cpu_count() or 2)) as ex:
        return list(ex.map(compile_one, units))


def _link(objs, out: str):
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
        "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not is_stale():
        return LIB
    objs = _compile(_units(), OBJDIR, tuned_knobs(), verbose)
    return _link(objs, LIB)


def build_variant(knobs: dict, out: str, objdir: str) -> str:
    """A copy of the library with the given knob definitions (on top of the tuned ones), for the
    autotuner. Only the 63-bit-key objects of the translation units the knobs affect are rebuilt; the
    others are the main build's objects."""
    build()
    merged = dict(tuned_knobs())
    merged.update(knobs)
    touched = {"sort.cu"} if any(k.startswith("CSTONE_SORT") for k in knobs) else set()
    if any(k.startswith("CSTONE_LEAVES") for k in knobs):
        touched.add("leaves.cu")
    units = [u for u in _units() if os.path.basename(u[0]) in touched and not u[2]]  # 63-bit keys only
    new_objs = {os.path.basename(o): o for o in _compile(units, objdir, merged)}
    objs = [new_objs.get(name, os.path.join(OBJDIR, name)) for _, name, _ in _units()]
    return _link(objs, out)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
