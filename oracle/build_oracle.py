"""Compile the CPU oracle (test infrastructure) into two shared libraries.

liboracle_f64.so  the reference arithmetic (double)
liboracle_f32.so  the same source at single precision (-DORACLE_FP32)

Plain gcc, no FMA contraction (-ffp-contract=off) and no fast-math, so each
floating-point operation is one IEEE-rounded operation on x86-64 and aarch64.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bsd_oracle.c")
TARGETS = {
    "liboracle_f64.so": [],
    "liboracle_f32.so": ["-DORACLE_FP32"],
}
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wno-unused-function"]


def compile_library(src: str, out: str, single: bool = False) -> None:
    """Compile one build of an oracle source file (double, or single with
    single=True) into the shared library `out`."""
    cmd = ["gcc", *CFLAGS, *(["-DORACLE_FP32"] if single else []), "-o", out, src, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)


def _needs(out: str) -> bool:
    return not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC)


def build(force: bool = False) -> None:
    def one(item):
        name, extra = item
        out = os.path.join(HERE, name)
        if not force and not _needs(out):
            return
        tmp = out + f".tmp{os.getpid()}"
        compile_library(SRC, tmp, single=bool(extra))
        os.replace(tmp, out)

    with ThreadPoolExecutor(len(TARGETS)) as ex:
        list(ex.map(one, TARGETS.items()))


if __name__ == "__main__":
    build(force="--force" in sys.argv)
