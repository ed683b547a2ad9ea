"""Compile the C oracle (test infrastructure) into oracle/_build/libref.so."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build", "libref.so")


def build(force=False, verbose=False):
    src = os.path.join(HERE, "ref.c")
    if (not force and os.path.exists(OUT)
            and os.path.getmtime(OUT) >= os.path.getmtime(src)):
        return OUT
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    tmp = OUT + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, src]
    # OpenMP only spreads the timed plain loop over the host's cores; without
    # it the oracle builds single-threaded
    for cmd in (base + ["-fopenmp", "-lm"], base + ["-lm"]):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        if subprocess.run(cmd, capture_output=not verbose).returncode == 0:
            break
    else:
        raise RuntimeError("could not compile %s" % src)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True, verbose=True))
