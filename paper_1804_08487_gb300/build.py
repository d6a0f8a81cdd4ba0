"""Native build steps for the package.

``build_cuda`` compiles every ``csrc/*.cu`` for sm_103a into ``lib/libcb.so``;
``build_synth`` compiles the host-side input generator into ``lib/libcbsynth.so``.
Both build in-tree and only rebuild when a source is newer than the library.
"""
import os
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
LIBDIR = PKG / "lib"
INCLUDE = ROOT / "include"
NVCC_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale(target: Path, sources) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(s).stat().st_mtime > t for s in sources)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(map(str, cmd))}\n{r.stdout}\n{r.stderr}")
    return r


def _atomic_build(target: Path, make):
    target.parent.mkdir(parents=True, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=target.suffix, dir=str(target.parent))
    os.close(fd)
    try:
        make(tmp)
        os.replace(tmp, target)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)


def build_synth(force: bool = False) -> Path:
    out = LIBDIR / "libcbsynth.so"
    src = CSRC / "synth.c"
    if force or _stale(out, [src]):
        _atomic_build(out, lambda tmp: _run(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
             "-o", tmp, str(src)]))
    return out


def cuda_sources():
    return sorted(CSRC.glob("*.cu"))


def cuda_headers():
    return sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))


def build_cuda(force: bool = False, verbose_ptxas: bool = False) -> Path:
    """Compile the CUDA library for sm_103a (one object per .cu, in parallel)."""
    out = LIBDIR / "libcb.so"
    srcs = cuda_sources()
    if not srcs:
        raise RuntimeError("no CUDA sources")
    if not (force or verbose_ptxas or _stale(out, srcs + cuda_headers())):
        return out
    objdir = LIBDIR / "obj"
    objdir.mkdir(parents=True, exist_ok=True)
    flags = NVCC_ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                         "-I", str(INCLUDE), "-I", str(CSRC), "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = objdir / (src.stem + ".o")
        r = _run(["nvcc", "-c", str(src), "-o", str(obj)] + flags)
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose_ptxas:
        for _, err in results:
            print(err)
    objs = [str(o) for o, _ in results]
    _atomic_build(out, lambda tmp: _run(["nvcc", "-shared"] + NVCC_ARCH + ["-o", tmp] + objs + ["-lpthread"]))
    return out


def build_all(force: bool = False):
    return build_synth(force), build_cuda(force)
