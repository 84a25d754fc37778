"""FP64 / FP32 FMA and streaming-read probe (``python -m paper_2403_09198_gb300.probe``).

Compiles ``fp64_probe.cu`` for sm_103a into ``_build/`` and runs it.  Its
output gives the FP64 FMA rate per SM per clock from which the benchmark derives
the FP64 roofline peak.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def run() -> str:
    build = os.path.join(os.path.dirname(HERE), "_build")
    os.makedirs(build, exist_ok=True)
    exe = os.path.join(build, "fp64_probe")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "fp64_probe.cu")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return out
