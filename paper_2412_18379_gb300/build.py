"""Build libcnnsns.so in-tree (paper_2412_18379_gb300/_build/) for sm_103a.

CUDA sources go through nvcc with one -gencode (compute_103a -> sm_103a);
host C++ through g++ with -ffp-contract=off (the mesh preprocessing computes
the inverse-affine matrices whose rounding the walk depends on). Translation
units compile in parallel; the link is nvcc -shared.
"""

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libcnnsns.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc"),
              shutil.which("nvcc") or ""):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def _cuda_inc():
    return os.path.join(os.path.dirname(os.path.dirname(_nvcc())), "include")


# per-file nvcc flags: the walk keeps every FP64 rounding explicit
CU_FLAGS = {
    "walk.cu": ["--fmad=false"],
    "search.cu": ["--fmad=false"],
    "classifier.cu": ["--fmad=false"],
}


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    hdr = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdr += [os.path.join(INC, f) for f in os.listdir(INC) if f.endswith(".h")]
    return cu, cpp, hdr


def _compile(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(force=False, verbose=False, ptxas_v=False):
    os.makedirs(OUT, exist_ok=True)
    cu, cpp, hdr = _sources()
    srcs = [os.path.join(CSRC, f) for f in cu + cpp]
    deps = srcs + hdr + [__file__]
    if (not force and os.path.exists(LIB)
            and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in deps)):
        return LIB
    nvcc = _nvcc()
    jobs = []
    objs = []
    for f in cu:
        o = os.path.join(OUT, f + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", INC, "-I", CSRC, *CU_FLAGS.get(f, []), "-c", os.path.join(CSRC, f),
               "-o", o]
        if ptxas_v:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append(cmd)
        objs.append(o)
    for f in cpp:
        o = os.path.join(OUT, f + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
               "-Wall", "-I", INC, "-I", CSRC, "-I", _cuda_inc(), "-c",
               os.path.join(CSRC, f), "-o", o]
        jobs.append(cmd)
        objs.append(o)
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        outs = list(ex.map(_compile, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = LIB + ".%d.tmp" % os.getpid()
    _compile([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, ptxas_v="-v" in sys.argv))
