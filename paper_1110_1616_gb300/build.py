"""Builds libamrmhd.so in-tree for sm_103a (nvcc for the CUDA units, g++ for
the host hierarchy builder, compiled in parallel)."""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libamrmhd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
UNITS = [
    ("api.cu", ["-Xcompiler", "-fopenmp"]),
    # FP32 division and square root without IEEE rounding (FP64 code is unaffected)
    ("kernels_fast.cu", ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]),
    ("kernels_strict.cu", ["--fmad=false"]),
    # the same mixed-precision kernels as kernels_fast.cu, so the same flags
    ("noalloc.cu", ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]),
    # no FMA contraction: the adjoint re-evaluates the forward's formulas (with
    # dual numbers) and must take the same branches as the strict FP64 forward
    ("adjoint.cu", ["--fmad=false"]),
    ("regrid_api.cu", []),
    ("partition.cu", []),
    ("maps_dev.cu", []),
    ("regrid_dev.cu", []),
    ("boxes_dev.cu", []),
]
HOST_UNITS = ["hierarchy.cpp", "regrid.cpp"]
HEADERS = ["hierarchy.hpp", "kernels.hpp", "kernels_impl.cuh", "kernels_fused.cuh", "mhd_device.cuh", "ctx.hpp",
           "adjoint_local.cuh", "fp_bits.cuh",
           "regrid.hpp"]


def _sources():
    s = [os.path.join(CSRC, u) for u, _ in UNITS] + [os.path.join(CSRC, u) for u in HOST_UNITS]
    s += [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "amrmhd.h")]
    return s


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force=False, verbose=False):
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    jobs = []
    for unit, extra in UNITS:
        obj = os.path.join(OUT, unit.replace(".cu", ".o"))
        cmd = [NVCC, "-std=c++17", *ARCH, "-O3", "-lineinfo", "-Xcompiler", "-fPIC", *extra, "-c",
               os.path.join(CSRC, unit), "-o", obj]
        jobs.append((cmd, obj))
    for unit in HOST_UNITS:
        hobj = os.path.join(OUT, unit.replace(".cpp", ".o"))
        jobs.append((["g++", "-std=c++17", "-O2", "-fPIC", "-fopenmp", "-c", os.path.join(CSRC, unit), "-o", hobj],
                     hobj))
    with cf.ThreadPoolExecutor(len(jobs)) as ex:
        futs = [ex.submit(subprocess.run, cmd, capture_output=True, text=True) for cmd, _ in jobs]
        for (cmd, _), f in zip(jobs, futs):
            r = f.result()
            if r.returncode != 0:
                raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
            if verbose:
                print(r.stdout + r.stderr)
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp] + [o for _, o in jobs] + ["-lgomp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
