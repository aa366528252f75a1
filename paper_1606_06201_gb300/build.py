"""Build the CUDA library libtopo_gb300.so in-tree for sm_103a (nvcc, no cmake).

Every translation unit is compiled in parallel to an object with -fPIC, then linked into one
shared library next to this file.  ``python -m paper_1606_06201_gb300.build`` runs it;
``--bounds-check`` builds the debug variant with index checks (-DTOPO_BOUNDS_CHECK) as
libtopo_gb300_bc.so (load it by setting TOPO_LIBRARY to its path before importing the binding).
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtopo_gb300.so")
LIB_BC = os.path.join(HERE, "libtopo_gb300_bc.so")
SOURCES = ["kernels_fe.cu", "kernels_q1.cu", "kernels_q1w.cu", "kernels_hex.cu", "kernels_rap.cu", "kernels_pcg.cu",
           "kernels_ip.cu",
           "solver.cu", "ipoc.cu", "static_scratch.cu",
           "element.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _compile(src, extra, build_dir=BUILD):
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    if src.endswith(".cu"):
        cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", "-c", path, "-o", obj, *extra]
    else:
        cmd = [nvcc(), "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-c", path, "-o", obj, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return obj, r.stderr


def build(verbose=False, extra=(), bounds_check=False):
    build_dir, lib = (BUILD + "_bc", LIB_BC) if bounds_check else (BUILD, LIB)
    extra = list(extra) + (["-DTOPO_BOUNDS_CHECK"] if bounds_check else [])
    os.makedirs(build_dir, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, build_dir), SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, err in results:
            if err.strip():
                sys.stderr.write(err)
    cmd = [nvcc(), *ARCH, "-shared", "-o", lib, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return lib


if __name__ == "__main__":
    args = sys.argv[1:]
    bc = "--bounds-check" in args
    print(build(verbose=True, extra=[a for a in args if a != "--bounds-check"], bounds_check=bc))
