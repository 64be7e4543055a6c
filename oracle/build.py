"""Build step of the oracle's C library (test infrastructure; see oracle/__init__.py)."""
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "liboracle.so")


def build() -> str:
    """Compile tslb_oracle.c with plain IEEE FP64 semantics (no fast-math) and OpenMP."""
    src = os.path.join(_HERE, "tslb_oracle.c")
    out = library_path()
    tmp = out + ".tmp"
    cmd = ["gcc", "-O3", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build())
