"""Measured ceilings of the MTTKRP data path (gather rows per clock from
L1 / L2 / HBM, vector-atomic rows per second, de-linearization keys per
clock) on the current GPU:

    python -m paper_2102_10245_gb300.probe [--out FILE]

compiles ``ceilings.cu`` with nvcc for sm_103a into ``_build/`` and prints one
JSON line per measurement."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def build():
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    exe = os.path.join(out, "ceilings")
    src = os.path.join(HERE, "ceilings.cu")
    if not os.path.exists(exe) or os.path.getmtime(exe) < os.path.getmtime(src):
        subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-lineinfo",
                        "-o", exe, src], check=True)
    return exe


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    exe = build()
    res = subprocess.run([exe], capture_output=True, text=True, check=False)
    if "--out" in argv:
        with open(argv[argv.index("--out") + 1], "w") as f:
            f.write(res.stdout)
    sys.stdout.write(res.stdout)
    return res.returncode


if __name__ == "__main__":
    sys.exit(main())
