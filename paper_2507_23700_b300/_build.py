"""Build libarbx.so (the CUDA kernels and the C ABI) in-tree for sm_103a.

    python paper_2507_23700_b300/_build.py [--force] [--verbose] [--checked]

Each translation unit under csrc/ is compiled with nvcc in parallel into
_build/, then linked into paper_2507_23700_b300/libarbx.so against the shared
CUDA runtime (the same libcudart.so.13 that PyTorch loads).  -fmad=false keeps
every float multiply and add separately rounded (the exactness contract).
--checked builds the bounds-checked variant (-DARBX_CHECKED=1) into
_build_checked/ and libarbx_checked.so; the package loads it when the
environment has ARBX_CHECKED=1.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
BUILD = PKG / "_build"
LIB = PKG / "libarbx.so"
BUILD_CHECKED = PKG / "_build_checked"
LIB_CHECKED = PKG / "libarbx_checked.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC,-O2",
              "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[Path]:
    return sorted(CSRC.glob("*.cu"))


def headers() -> list[Path]:
    return sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))


def _stale(target: Path, deps: list[Path]) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          checked: bool = False) -> Path:
    bdir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    bdir.mkdir(exist_ok=True)
    cc = nvcc()
    hdrs = headers()
    flags = NVCC_FLAGS + (["-DARBX_CHECKED=1"] if checked else []) + list(extra_flags or []) \
        + os.environ.get("ARBX_EXTRA_NVCC", "").split()
    # objects built with other flags are rebuilt
    stamp = bdir / "flags.txt"
    line = " ".join([cc, *ARCH, *flags])
    if not stamp.exists() or stamp.read_text() != line:
        force = True
        stamp.write_text(line)
    jobs = []
    objs = []
    for src in sources():
        obj = bdir / (src.stem + ".o")
        objs.append(obj)
        if force or _stale(obj, [src, *hdrs, Path(__file__)]):
            jobs.append([cc, *ARCH, *flags, "-c", str(src), "-o", str(obj)])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for j, f in zip(jobs, futs):
                r = f.result()
                if verbose or r.returncode != 0:
                    sys.stderr.write(" ".join(j) + "\n" + r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed for {j[-3]}")
    if force or jobs or _stale(lib, objs):
        tmp = lib.with_suffix(f".{os.getpid()}.tmp")
        cmd = [cc, *ARCH, "-shared", "-cudart", "shared", *[str(o) for o in objs], "-o", str(tmp),
               "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib)
    return lib


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true", help="print registers/spills per kernel")
    ap.add_argument("--checked", action="store_true", help="build the bounds-checked libarbx_checked.so")
    a = ap.parse_args()
    extra = ["-Xptxas", "-v"] if a.ptxas_info else None
    print(build(force=a.force or a.ptxas_info, verbose=a.verbose or a.ptxas_info, extra_flags=extra,
                checked=a.checked))


if __name__ == "__main__":
    main()
