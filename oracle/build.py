"""Compile the C oracle (``ac_oracle.c``) into ``oracle/_build/liboracle.so``.

Test infrastructure only.  Built with ``-O2 -ffp-contract=off`` and without
fast-math so that every operation is one separately rounded binary64 operation.
"""
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ac_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()


def library_path():
    return _LIB


def build_oracle(force=False):
    """Build the oracle library if it is missing or older than its source."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
        return _LIB
