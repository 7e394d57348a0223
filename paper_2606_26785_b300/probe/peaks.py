"""Build and run the arithmetic-rate probe (peaks.cu) on the current GPU and
print its JSON line: FP64 FMA, FP64 tensor-core MMA and FP32 FMA rates in
TFLOP/s.  The benchmark's FP64 and FP32 roofline peaks are these figures.

    python -m paper_2606_26785_b300.probe.peaks
"""
import subprocess
import sys
import tempfile
from pathlib import Path

HERE = Path(__file__).resolve().parent


def main():
    with tempfile.TemporaryDirectory() as d:
        exe = Path(d) / "peaks"
        subprocess.run(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                        str(HERE / "peaks.cu"), "-o", str(exe)], check=True)
        r = subprocess.run([str(exe)], capture_output=True, text=True)
        sys.stdout.write(r.stdout)
        sys.stderr.write(r.stderr)
        return r.returncode


if __name__ == "__main__":
    sys.exit(main())
