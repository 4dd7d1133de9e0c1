"""Build the binary128 Boys-function oracle (test infrastructure only).

Compiles ``boys_oracle.c`` with the host C compiler into
``oracle/_build/liboracle.so``.  On x86-64 the quad type is ``__float128``
and libquadmath is linked; on AArch64 ``long double`` is binary128 and libm
suffices.  OpenMP parallelises the batch entry points.
"""
import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "boys_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False, src: str = SRC, lib: str = LIB) -> str:
    """Compile the oracle if the library is missing or older than its source.

    ``src``/``lib`` let a test compile a modified copy of the source (a
    planted mistake) to a scratch location; the product never calls this.
    """
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(src)):
        return lib
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    cc = os.environ.get("CC", "gcc")
    cmd = [cc, "-O2", "-fPIC", "-shared", "-fopenmp", "-Wall", "-Wextra",
           "-o", lib + ".tmp", src]
    if platform.machine() in ("x86_64", "AMD64", "i686"):
        cmd.append("-lquadmath")
    cmd.append("-lm")
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
