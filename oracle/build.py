"""Compile the FP64 C oracle into ``oracle/_build/liblboracle.so``.

TEST INFRASTRUCTURE: the oracle is only built and loaded by the test suite,
the smoke check and the benchmark's CPU-baseline leg.

The build uses plain ``gcc -O2`` with OpenMP when the compiler supports it
(the OpenMP loops run over sites or z-planes and hold no reductions, so the
result does not depend on the thread count), and falls back to a serial
build otherwise. No ``-march=native``: the same source builds on x86_64 and
aarch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lb_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblboracle.so")


def build_oracle(force: bool = False) -> str:
    """Build the oracle shared library if it is missing or stale; return its path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
