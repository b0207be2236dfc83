"""Build the oracle's C part (the FP32 replay) with the host compiler.

-ffp-contract=off keeps every multiply and add separately rounded unless the source calls
fmaf explicitly: the replay's rounding sequence is part of spec R. No -march flags, so the
same source gives the same results on x86_64 and aarch64.
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "replay32.c")
OUT = os.path.join(_HERE, "_replay32.so")


def build_replay(force: bool = False) -> str:
    if force or not os.path.exists(OUT) or os.path.getmtime(OUT) < os.path.getmtime(SRC):
        tmp = OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build_replay(force=True))
