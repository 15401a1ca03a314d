"""Build the in-tree CUDA library libfwi.so for sm_103a (B300).

The step kernels are instantiated per grid size in translation units of their own
(csrc/inst_*.cu compiled once per size), so the objects compile in parallel; they are
then linked into one shared library.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfwi.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]

# (object name, source, defines): the library's translation units
UNITS = [("fwi", "fwi.cu", []), ("lbfgs", "lbfgs.cu", []), ("resample", "resample.cu", [])]
UNITS += [(f"plane2_{n}", "inst_plane2.cu", [f"-DFWI_N={n}"]) for n in (32, 64, 96, 128, 135, 160)]
UNITS += [(f"zpass2_{n}", "inst_zpass2.cu", [f"-DFWI_N={n}"]) for n in (32, 48, 64, 80, 96, 128, 135, 256)]
UNITS += [(f"split2_{n}", "inst_split2.cu", [f"-DFWI_N={n}"]) for n in (243, 256, 480)]
UNITS += [(f"zpass_{e}_{n}", "inst_zpass.cu", [f"-DFWI_E={e}", f"-DFWI_N={n}"])
          for e, n in [(8, 32), (8, 48), (8, 64), (8, 80), (8, 96), (8, 128), (8, 0), (16, 0)]]
UNITS += [(f"plane_{e}_{n}", "inst_plane.cu", [f"-DFWI_E={e}", f"-DFWI_N={n}"])
          for e, n in [(8, 32), (8, 64), (8, 96), (8, 128), (8, 160), (8, 0), (16, 0)]]
UNITS += [(f"split_{e}", "inst_split.cu", [f"-DFWI_E={e}"]) for e in (8, 16)]


def _newest_dep():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "fwi.h"))
    return max(os.path.getmtime(d) for d in deps)


def _stale(target, newer_than):
    return not os.path.exists(target) or os.path.getmtime(target) < newer_than


def build(force: bool = False, verbose: bool = False, jobs: int = 0) -> str:
    """Compile csrc into paper_2102_00755_b300/libfwi.so with nvcc (no GPU needed)."""
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ, exist_ok=True)
    hdr = _newest_dep()
    todo = []
    objs = []
    for name, src, defs in UNITS:
        o = os.path.join(OBJ, name + ".o")
        objs.append(o)
        s = os.path.join(CSRC, src)
        if force or _stale(o, max(hdr, os.path.getmtime(s))):
            todo.append([nvcc, *ARCH, *FLAGS, *defs, "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)

    if todo:
        with concurrent.futures.ThreadPoolExecutor(jobs or os.cpu_count() or 1) as ex:
            for f in [ex.submit(run, c) for c in todo]:
                f.result()
    if force or todo or _stale(LIB, max(os.path.getmtime(o) for o in objs)):
        run([nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *objs])
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
