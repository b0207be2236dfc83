"""Build the oracle's C parts with the host compiler.

replay32.c (the FP32 replay): -ffp-contract=off keeps every multiply and add separately
rounded unless the source calls fmaf explicitly: the replay's rounding sequence is part of
spec R. pic64.c (the FP64 mover and deposit as loops): the same flag, and OpenMP when the
compiler has it (built without it otherwise: the loops then run on one thread). No -march
flags, so the same source gives the same results on x86_64 and aarch64.
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "replay32.c")
OUT = os.path.join(_HERE, "_replay32.so")
SRC64 = os.path.join(_HERE, "pic64.c")
OUT64 = os.path.join(_HERE, "_pic64.so")


def _compile(src, out, extra, force):
    if force or not os.path.exists(out) or os.path.getmtime(out) < max(os.path.getmtime(src), os.path.getmtime(__file__)):
        tmp = out + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
        try:
            subprocess.check_call(base + extra, stderr=subprocess.DEVNULL if extra else None)
        except subprocess.CalledProcessError:
            if not extra:
                raise
            subprocess.check_call(base)
        os.replace(tmp, out)
    return out


def build_replay(force: bool = False) -> str:
    return _compile(SRC, OUT, [], force)


def build_pic64(force: bool = False) -> str:
    return _compile(SRC64, OUT64, ["-fopenmp"], force)


def build_all(force: bool = False):
    return build_replay(force), build_pic64(force)


if __name__ == "__main__":
    print(build_all(force=True))
