"""In-tree build of libgoo.so (CUDA C++ for sm_103a) with nvcc.

Every translation unit under csrc/ is compiled in parallel into _build/, then linked into
paper_1710_08826_gb300/libgoo.so.  A unit is rebuilt when it or any header is newer than
its object file.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgoo.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgoo.so")
    return path


def _cuda_lib_dir(nvcc):
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


# Headers that the run-time specialised event kernel is compiled from (jit.cu, NVRTC).
JIT_HEADERS = [os.path.join(INCLUDE, "goo.h"), os.path.join(CSRC, "common.cuh"), os.path.join(CSRC, "model.cuh"),
               os.path.join(CSRC, "sop_kernels.cuh")]
_DELIM = "goo_jit_src"


def _write_jit_sources():
    """_build/jit_sources.inc: the JIT headers as C++ raw string literals (rewritten only when
    their content changes)."""
    parts = ["// generated by buildlib.py from " + ", ".join(os.path.basename(h) for h in JIT_HEADERS) + "\n"]
    parts.append("static const char* const kJitHeaderNames[] = {" +
                 ", ".join('"%s"' % os.path.basename(h) for h in JIT_HEADERS) + "};\n")
    parts.append("static const char* const kJitHeaderSources[] = {\n")
    for h in JIT_HEADERS:
        text = open(h).read()
        if ")" + _DELIM + '"' in text:
            raise RuntimeError(f"{h} contains the raw-string delimiter")
        parts.append('R"' + _DELIM + "(" + text + ")" + _DELIM + '",\n')
    parts.append("};\n")
    out = os.path.join(BUILD, "jit_sources.inc")
    new = "".join(parts)
    if not os.path.exists(out) or open(out).read() != new:
        with open(out, "w") as f:
            f.write(new)


def build(verbose=False, force=False, jobs=None):
    """Compile and link libgoo.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    _write_jit_sources()
    newest_header = max((os.path.getmtime(h) for h in _headers()), default=0.0)
    cuda_include = os.path.join(os.path.dirname(_cuda_lib_dir(nvcc)), "include")
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + BUILD,
                    '-DGOO_CUDA_INCLUDE="%s"' % cuda_include, "-Xptxas", "-warn-spills"]

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        if (not force and os.path.exists(obj)
                and os.path.getmtime(obj) >= max(os.path.getmtime(src), newest_header)):
            return obj, False
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj, True

    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=jobs or min(8, len(srcs))) as ex:
        results = list(ex.map(compile_one, srcs))
    objs = [o for o, _ in results]
    relink = force or not os.path.exists(LIB) or any(changed for _, changed in results) or \
        os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs)
    if relink:
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB] + objs + [
            "-cudart", "shared", "-lnvrtc", "-Xlinker", "-rpath," + _cuda_lib_dir(nvcc)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of libgoo.so failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
