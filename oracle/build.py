"""Build the FP64 CPU oracle (plain C, gcc, OpenMP) into oracle/_build/.

Test infrastructure: building the checker is not using it.  Flags keep IEEE
semantics (no fast-math, no FMA contraction) so results agree across the x86
development host and the Arm GPU host.
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "_build", "liboracle.so")


def build_oracle(force: bool = False) -> str:
    src = os.path.join(_HERE, "fgs4d_oracle.c")
    out = library_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-Wall", "-Wextra",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def sanitized_library_path() -> str:
    return os.path.join(_HERE, "_build", "liboracle_san.so")


def build_oracle_sanitized(force: bool = False) -> str:
    """The same library built with AddressSanitizer and UndefinedBehavior-
    Sanitizer (every finding aborts), for the sanitizer test; loaded instead
    of the plain build when FGS4D_ORACLE_SANITIZED=1 (the process must
    preload libasan, as the interpreter is not instrumented)."""
    src = os.path.join(_HERE, "fgs4d_oracle.c")
    out = sanitized_library_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O1", "-g", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-Wall", "-Wextra",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(force=True))
