"""Build step for the FP64 CPU oracle (test infrastructure).

Compiles ``dugks_oracle.c`` twice with the system C compiler: once on ``double``
(``liboracle.so``) and once on ``double _Complex`` (``liboracle_cs.so``, the complex-step
derivative build). FMA contraction is switched off so both the x86 and the Arm host round
every operation the same way.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dugks_oracle.c")
LIBS = {
    "liboracle.so": [],
    "liboracle_cs.so": ["-DORACLE_COMPLEX_STEP"],
}
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def lib_path(name="liboracle.so"):
    return os.path.join(HERE, name)


def build(force=False, verbose=False):
    """Compile both oracle libraries if missing or older than the source."""
    cc = os.environ.get("CC", "gcc")
    for name, extra in LIBS.items():
        out = lib_path(name)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
            continue
        tmp = out + ".tmp%d" % os.getpid()
        cmd = [cc] + CFLAGS + extra + ["-o", tmp, SRC, "-lm"]
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return [lib_path(n) for n in LIBS]


if __name__ == "__main__":
    build(force=True, verbose=True)
