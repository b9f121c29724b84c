"""Build libsmg.so in-tree: host setup with g++, kernels with nvcc for sm_103a.

Translation units compile in parallel; the library links the CUDA runtime
statically.  Rebuilds only when a source or header is newer than the library.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libsmg.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _sources():
    host = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    cuda = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    deps = host + cuda + glob.glob(os.path.join(CSRC, "*.h*")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    deps += glob.glob(os.path.join(INC, "*.h"))
    return host, cuda, deps


def build(force=False, verbose=False):
    host, cuda, deps = _sources()
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    jobs, objs = [], []
    for src in host:
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-pthread", "-ffp-contract=off", "-Wall", "-Wextra",
               "-I", INC, "-I", "/usr/local/cuda/include", "-c", src, "-o", obj]
        jobs.append((cmd, src))
        objs.append(obj)
    for src in cuda:
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        cmd = [NVCC, "-std=c++17", "-O3", ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-ffp-contract=off", "-I", INC, "-c", src, "-o", obj]
        jobs.append((cmd, src))
        objs.append(obj)
    procs = [(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), src)
             for cmd, src in jobs]
    failed = []
    for p, src in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((src, text))
        elif verbose and text.strip():
            print(text)
    if failed:
        msg = "\n".join("%s:\n%s" % f for f in failed)
        raise RuntimeError("libsmg build failed\n" + msg)
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.run([NVCC, "-shared", ARCH, "-o", tmp] + objs + ["-lpthread"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
