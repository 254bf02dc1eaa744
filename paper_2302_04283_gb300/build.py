"""Build librad.so in-tree for sm_103a with nvcc (one -gencode, parallel TUs)."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librad.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]

SOURCES = ["angles.cpp", "capi.cu", "geom.cu", "step.cu",
           "stage_f32_flat.cu", "stage_f32_flat164.cu", "stage_f32_flat164x.cu", "stage_f32_ang.cu", "stage_f32_ang164.cu",
           "stage_f32_ang364.cu", "stage_f32_ang644.cu", "stage_f32_angplm.cu", "stage_f32_angmapr.cu",
           "stage_f64_flat.cu", "stage_f64_ang.cu", "stage_f64_angplm.cu", "stage_f64_angmapr.cu",
           "moments.cu", "moments_tc.cu", "adjoint.cu", "adjoint_tadj_f32_flat.cu", "adjoint_tadj_f32_ang.cu",
           "adjoint_tadj_f64_flat.cu", "adjoint_tadj_f64_ang.cu",
           "adjoint_tadj_f32_angplm.cu", "adjoint_tadj_f64_angplm.cu",
           "adjoint_tadj_f32_angmapr.cu", "adjoint_tadj_f64_angmapr.cu", "noalloc.cu", "host_stream.cu", "raddom.cu", "peak.cu", "halo.cu", "frequency.cu", "gas.cu"]


def _compile(src, extra):
    obj = os.path.join(BUILD, src + ".o")
    cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd = [NVCC] + FLAGS + ["-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, r


def build(verbose=False, extra=()):
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 2)) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra)), SOURCES))
    objs = []
    for src, obj, r in results:
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("nvcc failed on " + src)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        objs.append(obj)
    tmp = LIB + ".tmp"
    r = subprocess.run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    extra = sys.argv[1:]
    print(build(verbose=True, extra=extra))
