"""Compile the CPU oracle (test infrastructure only) into oracle/_build/.

The oracle is plain C11, built with -O2 -ffp-contract=off and no fast-math
so that every float operation is rounded once, in source order.  Only the
tests, the smoke check and the benchmark's CPU-baseline leg load it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vg_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libvg_oracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
          "-Wall", "-Wextra", "-Werror"]


def build(src=SRC, out=LIB, extra_flags=(), force=False):
    """Build the oracle shared library (or a variant of it) and return its path.

    Rebuilds when the source or header is newer than the library, or when
    force is set.  extra_flags are appended to the compiler command.
    """
    os.makedirs(os.path.dirname(out), exist_ok=True)
    hdr = os.path.join(os.path.dirname(src), "vg_oracle.h")
    deps = [src, hdr if os.path.exists(hdr) else os.path.join(HERE, "vg_oracle.h")]
    if (not force and os.path.exists(out)
            and all(os.path.getmtime(out) >= os.path.getmtime(d) for d in deps)):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = (["gcc"] + CFLAGS + list(extra_flags)
           + ["-I", os.path.dirname(src), "-shared", "-o", tmp, src, "-lm"])
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
