"""Compile the FP64 oracle (plain C, gcc) into oracle/_build/liboracle.so.

Test infrastructure only. Flags keep the arithmetic plain: no fast-math and no
floating-point contraction, so x86-64 and aarch64 builds round identically.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "prdpt_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def _compile(src: str, out: str) -> None:
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-D_GNU_SOURCE", src, "-o", out, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    _compile(SRC, tmp)
    os.replace(tmp, LIB)
    return LIB


def build_modified(replace: dict, out_dir: str) -> str:
    """Compile a copy of the oracle's source with each key of `replace` (an exact line or
    fragment that must occur once) replaced by its value, into out_dir. Tests use it to
    plant a mistake and check that a pin fails on it."""
    text = open(SRC).read()
    for old, new in replace.items():
        if text.count(old) != 1:
            raise ValueError(f"fragment to replace occurs {text.count(old)} times: {old!r}")
        text = text.replace(old, new)
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "oracle_modified.c")
    with open(src, "w") as f:
        f.write(text)
    out = os.path.join(out_dir, "liboracle_modified.so")
    _compile(src, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
