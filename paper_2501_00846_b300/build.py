"""Build the CUDA library (sm_103a) in-tree: paper_2501_00846_b300/libtslb_b300.so."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
SOURCES = ["lbm_api.cu", "step_split.cu", "step_fused2.cu", "step_unfused.cu", "step_lbm16.cu", "observables.cu",
           "observables_noalloc.cu", "ensemble.cu", "closure.cu", "step_mom.cu"]
LIB = os.path.join(HERE, "libtslb_b300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_flags(extra=()):
    return ["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
            "-I", os.path.join(ROOT, "include"), *extra]


def build(verbose: bool = False, extra=()) -> str:
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    objs = [os.path.join(bdir, src.replace(".cu", ".o")) for src in SOURCES]

    def compile_one(src, obj):
        cmd = nvcc_flags(extra) + (["-Xptxas=-v"] if verbose else []) + ["-c", os.path.join(CSRC, src), "-o", obj]
        subprocess.run(cmd, check=True)

    # translation units compile independently: one nvcc process each, a few at a time
    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 1)) as pool:
        for f in [pool.submit(compile_one, s, o) for s, o in zip(SOURCES, objs)]:
            f.result()
    tmp = LIB + ".tmp"
    subprocess.run(["nvcc", *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
