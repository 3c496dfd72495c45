"""Compile and run ceilings.cu (sm_103a); prints one JSON line with the
register-only rates of the modular multiply-accumulate and the NTT
butterfly on this GPU."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    exe = os.path.join(HERE, "_ceilings")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "ceilings.cu")], check=True)
    return subprocess.run([exe]).returncode


if __name__ == "__main__":
    sys.exit(main())
