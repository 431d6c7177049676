"""Build liblb.so in-tree for sm_103a.

The kernels are instantiated per (velocity set, storage type) in small
generated translation units so that nvcc can compile them in parallel; the
host sources (C-ABI, quadrature builder) are compiled alongside, and the
objects are linked into ``paper_0908_4520_gb300/liblb.so`` against the shared
CUDA runtime.  Rebuilds only what changed.

Supported build options (environment variables):

* ``LB_EXTRA_NVCC``: extra nvcc flags for every unit, e.g. the launch-shape
  overrides of ``csrc/lb_kernels.cuh`` (``-DLB_TMA_K=9``, ``-DLB_TMA_BAND=0``,
  ``-DLB_TMA_WIDE_SMEM=...``; each macro there states its default and what was
  measured for it);
* ``LB_BUILD_TAG``: build into ``_build_<tag>/`` and ``liblb_<tag>.so`` instead,
  so that a library built with other options sits beside the default one
  (the binding loads it when ``LB_LIB_PATH`` names it);
* ``LB_UNITS``: a comma list of the generated units to compile (``gh6_f32``,
  ``d2q37_f32``, ...), for a quick build of one set and storage; a library
  built this way rejects the other sets with ``LB_ERR_UNSUPPORTED``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
GEN = os.path.join(BUILD, "gen")
LIB = os.path.join(PKG, "liblb.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-diag-suppress", "177",
              "-I", INCLUDE, "-I", CSRC] + os.environ.get("LB_EXTRA_NVCC", "").split()
# a tagged build goes to its own folder and library name
if os.environ.get("LB_BUILD_TAG"):
    BUILD = os.path.join(PKG, "_build_" + os.environ["LB_BUILD_TAG"])
    GEN = os.path.join(BUILD, "gen")
    LIB = os.path.join(PKG, f"liblb_{os.environ['LB_BUILD_TAG']}.so")

# (generated name, velocity-set class, lb_quadrature enumerator)
_SETS16 = [("gh4", "GH4", "LB_D2Q16_GH"), ("gh6", "GH6", "LB_D2Q36_GH"), ("gh8", "GH8", "LB_D2Q64_GH")]
_SETS = [("d2q37", "D2Q37", "LB_D2Q37"), ("d2q9", "D2Q9", "LB_D2Q9"), ("d2q16i", "D2Q16I", "LB_D2Q16_INT"),
         ("d2q17", "D2Q17", "LB_D2Q17"), ("d2q21", "D2Q21", "LB_D2Q21"), ("d2q25", "D2Q25", "LB_D2Q25")]
# storage tag -> (storage type, arithmetic type, lb_precision enumerator)
_STORES = {"f32": ("float", "float", "LB_F32"), "f64": ("double", "double", "LB_F64"),
           "bf16": ("__nv_bfloat16", "float", "LB_BF16"), "f16": ("__half", "float", "LB_F16")}


def _units():
    """All (set, storage) units, or the subset named in LB_UNITS (comma list)."""
    units = []
    for name, cls, q in _SETS16:
        for st in ("f32", "f64", "bf16", "f16"):
            units.append((f"{name}_{st}", cls, q, *_STORES[st]))
    for name, cls, q in _SETS:
        for st in ("f32", "f64"):
            units.append((f"{name}_{st}", cls, q, *_STORES[st]))
    only = os.environ.get("LB_UNITS")
    if only:
        keep = set(only.split(","))
        units = [u for u in units if u[0] in keep]
    return units


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _digest(src, extra=()):
    """Hash of one object's inputs: its source, every header, the flags."""
    h = hashlib.sha256()
    h.update(" ".join(extra).encode())
    for f in [src] + sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                            + [os.path.join(INCLUDE, "lb.h")]):
        with open(f, "rb") as fh:
            h.update(f.encode() + fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()


def _write_if_changed(path, text):
    if os.path.exists(path):
        with open(path) as fh:
            if fh.read() == text:
                return
    with open(path, "w") as fh:
        fh.write(text)


def _compile(src, obj, extra=()):
    stamp = obj + ".sha"
    dig = _digest(src, extra)
    if os.path.exists(obj) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read() == dig:
                return obj, False
    cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
    with open(stamp, "w") as fh:
        fh.write(dig)
    return obj, True


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    os.makedirs(GEN, exist_ok=True)
    if force:
        for o in glob.glob(os.path.join(BUILD, "*.sha")):
            os.remove(o)
    jobs = jobs or max(1, min(32, os.cpu_count() or 1))
    tasks = []
    for tag, cls, qenum, st, rt, penum in _units():
        src = os.path.join(GEN, f"k_{tag}.cu")
        _write_if_changed(src, (
            f"// generated by builder.py: kernels of the {cls} set with {st} storage\n"
            "#include \"lb_kernels.cuh\"\n\n"
            "namespace lbk {\n"
            "namespace {\n"
            f"cudaError_t launch_unit(const Launch& L) {{ return launch_order<lbvs::{cls}, {st}, {rt}>(L); }}\n"
            f"const bool registered = register_launcher({qenum}, {penum}, &launch_unit);\n"
            "}  // namespace\n"
            "}  // namespace lbk\n"))
        tasks.append((src, os.path.join(BUILD, f"k_{tag}.o")))
    for f in ("lb_api.cpp", "quadrature.cpp", "fp32_identities.cpp", "lb_batch.cpp", "lb_server.cpp", "lb_dvm.cu"):
        tasks.append((os.path.join(CSRC, f), os.path.join(BUILD, os.path.splitext(f)[0] + ".o"), ()))
    tasks = [t if len(t) == 3 else (t[0], t[1], ()) for t in tasks]
    # the multi-instance kernel, once per storage type
    for tag, st in (("f32", "float"), ("f16", "__half"), ("bf16", "__nv_bfloat16")):
        tasks.append((os.path.join(CSRC, "lb_batch_kernels.cu"), os.path.join(BUILD, f"batch_{tag}.o"),
                      (f"-DLB_BATCH_STORAGE={st}", f"-DLB_BATCH_ENTRY(x)=batch_##x##_{tag}")))
    # the allocation-free single solve (runs the multi-instance kernel)
    tasks.append((os.path.join(CSRC, "lb_static.cu"), os.path.join(BUILD, "lb_static.o"), ()))
    # largest units first
    tasks.sort(key=lambda t: ("batch" not in t[1], "gh8" not in t[0], "gh6" not in t[0], "d2q37" not in t[0]))
    changed = False
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = [ex.submit(_compile, s, o, x) for s, o, x in tasks]
        for f in cf.as_completed(futs):
            o, did = f.result()
            changed |= did
            if verbose and did:
                print("built", os.path.basename(o), flush=True)
    if changed or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *[o for _, o, _x in tasks], "-cudart", "shared",
               "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
