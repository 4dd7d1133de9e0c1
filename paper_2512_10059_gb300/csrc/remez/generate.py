"""Regenerate ``csrc/boys_coeffs_fp32.h`` with the rational Remez generator.

    python paper_2512_10059_gb300/csrc/remez/generate.py [--check KFIRST KLAST]

Compiles ``boys_remez.cpp`` with the host C++ compiler (OpenMP over kmax)
and runs it; the result depends on the ``long double`` format, so the
committed header was produced on x86-64 (64-bit extended significand).
``--check`` only prints the generator's output for a kmax range to stdout.
"""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "boys_remez.cpp")
HEADER = os.path.join(os.path.dirname(HERE), "boys_coeffs_fp32.h")


def compile_generator(out_dir: str) -> str:
    exe = os.path.join(out_dir, "boys_remez")
    subprocess.run([os.environ.get("CXX", "g++"), "-O2", "-fopenmp", "-o", exe, SRC], check=True)
    return exe


def run(kfirst=None, klast=None) -> str:
    with tempfile.TemporaryDirectory() as d:
        exe = compile_generator(d)
        args = [exe] + ([str(kfirst), str(klast)] if kfirst is not None else [])
        r = subprocess.run(args, check=True, capture_output=True, text=True)
        return r.stdout


if __name__ == "__main__":
    if len(sys.argv) == 4 and sys.argv[1] == "--check":
        sys.stdout.write(run(int(sys.argv[2]), int(sys.argv[3])))
    else:
        text = run()
        with open(HEADER, "w") as fh:
            fh.write(text)
        print(HEADER)
