"""Build libprad.so (sm_103a) in-tree with nvcc: one object per .cu, in
parallel, then a shared-library link.  Output: paper_1409_5574_gb300/_build/."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libprad.so")
ROOT = os.path.dirname(HERE)

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
    "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


# The kernel translation unit the run-time specialisation compiles with
# NVRTC (spec.cu), then the headers it includes, by their include names.
SPEC_SOURCES = [os.path.join(CSRC, "push_emit.cu"), os.path.join(CSRC, "prad_internal.h"),
                os.path.join(CSRC, "mlp_device.cuh"), os.path.join(CSRC, "rtc_prelude.h"),
                os.path.join(ROOT, "include", "prad.h")]


def _write_spec_sources(out: str) -> str:
    """Embed SPEC_SOURCES as raw string literals; rewritten only on change."""
    names, texts = [], []
    for path in SPEC_SOURCES:
        with open(path) as f:
            text = f.read()
        assert ")PRADSRC" not in text
        names.append(os.path.basename(path))
        texts.append(text)
    body = "static const char* const kSpecSrcName[] = {%s};\n" % ", ".join(
        '"%s"' % n for n in names)
    body += "static const char* const kSpecSrc[] = {\n%s};\n" % ",\n".join(
        'R"PRADSRC(%s)PRADSRC"' % t for t in texts)
    inc = os.path.join(out, "prad_spec_sources.inc")
    old = None
    if os.path.exists(inc):
        with open(inc) as f:
            old = f.read()
    if old != body:
        with open(inc, "w") as f:
            f.write(body)
    return inc


def _spec_flags(nvcc: str, out: str) -> list:
    """spec.cu: the generated sources and where NVRTC and the CUDA headers are."""
    path = nvcc if os.path.isabs(nvcc) else (shutil.which(nvcc) or nvcc)
    home = os.path.dirname(os.path.dirname(os.path.realpath(path)))
    return ["-I", out, '-DPRAD_CUDA_INCLUDE="%s"' % os.path.join(home, "include"),
            '-DPRAD_CUDA_LIBDIR="%s"' % os.path.join(home, "lib64")]


def sources() -> list:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(target: str, deps: list) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra_flags: list | None = None,
          out_dir: str | None = None) -> str:
    """Compile (incrementally) and link; returns the library path.
    ``extra_flags`` / ``out_dir`` build a variant elsewhere (e.g. -D tuning
    macros) without touching the default library."""
    out = out_dir or OUT
    lib = os.path.join(out, "libprad.so")
    os.makedirs(out, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "prad.h"))
    flags = NVCC_FLAGS + (extra_flags or [])
    nvcc = _nvcc()
    spec_inc = _write_spec_sources(out)
    jobs = []
    for src in sources():
        obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
        deps, f = [src] + headers, flags
        if os.path.basename(src) == "spec.cu":
            deps, f = deps + [spec_inc], flags + _spec_flags(nvcc, out)
        if _stale(obj, deps) or extra_flags:
            jobs.append([nvcc] + f + ["-c", src, "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(out, os.path.basename(s)[:-3] + ".o") for s in sources()]
    if _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        # static cudart: the library loads without a CUDA runtime on the
        # loader path and shares the device's primary context with torch
        run([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a",
             "-cudart", "static", "-o", tmp] + objs + ["-ldl"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
