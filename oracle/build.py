"""Build step for the oracle's shared library (plain C, gcc)."""
import os
import subprocess
import tempfile
from pathlib import Path

HERE = Path(__file__).resolve().parent
LIB = HERE / "lib" / "liboracle.so"
SRC = HERE / "cb_oracle.c"


def build_oracle(force: bool = False) -> Path:
    """Compile cb_oracle.c into lib/liboracle.so if missing or out of date."""
    if not force and LIB.exists() and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    LIB.parent.mkdir(parents=True, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=str(LIB.parent))
    os.close(fd)
    try:
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, str(SRC)],
                       check=True, capture_output=True, text=True)
        os.replace(tmp, LIB)
    except subprocess.CalledProcessError as exc:
        os.unlink(tmp)
        raise RuntimeError(f"oracle build failed:\n{exc.stderr}") from exc
    return LIB
