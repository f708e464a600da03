"""Build liblscan.so in-tree with nvcc for sm_103a (no GPU needed).

Each .cu under csrc/ compiles to an object in parallel; the objects link into
paper_1604_04815_gb300/_build/liblscan.so with the CUDA runtime linked
statically.  Only x86/Arm-neutral host flags are used, so the same command
builds on the x86 development machine and on the Arm GPU host.
"""
import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblscan.so")
# the benchmark's comparator (CUB's device scan), a library of its own
CMP_SRC = os.path.join(HERE, "compare", "cub_scan.cu")
CMP_LIB = os.path.join(OUT, "libcubcmp.so")
# ... and the multi-threaded host scan (plain C, gcc)
CPU_SRC = os.path.join(HERE, "compare", "cpu_scan.c")
CPU_LIB = os.path.join(OUT, "libcpuscan.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-O2", "--expt-relaxed-constexpr",
              "-I", os.path.join(ROOT, "include")]


def _nvcc():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build "
                       "liblscan.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(CSRC, "*.h")) +
                  [os.path.join(ROOT, "include", "lscan.h")])


def _stamp():
    h = hashlib.sha256()
    for f in _sources() + _headers() + [CMP_SRC, CPU_SRC, os.path.abspath(__file__)]:
        with open(f, "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()


def build(force=False, jobs=None, verbose=False):
    """Compile csrc/*.cu and link liblscan.so; returns the library path."""
    os.makedirs(OUT, exist_ok=True)
    stamp_file = os.path.join(OUT, "stamp.txt")
    stamp = _stamp()
    if (not force and os.path.exists(LIB) and os.path.exists(stamp_file)
            and open(stamp_file).read() == stamp):
        return LIB
    nvcc = _nvcc()
    objs = []
    cmds = []
    for src in _sources():
        obj = os.path.join(OUT, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmds.append([nvcc] + ARCH + NVCC_FLAGS + ["-c", src, "-o", obj])
    cmp_obj = os.path.join(OUT, "cub_scan.o")
    cmp_cmd = [nvcc] + ARCH + NVCC_FLAGS + ["-c", CMP_SRC, "-o", cmp_obj]
    jobs = jobs or max(1, min(len(cmds) + 1, os.cpu_count() or 4))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" +
                               r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return cmd[-1]

    with cf.ThreadPoolExecutor(jobs) as ex:
        cmp_job = ex.submit(run, cmp_cmd) if os.path.exists(CMP_SRC) else None
        list(ex.map(run, cmds))
        cmp_err = None
        if cmp_job is not None:
            try:
                cmp_job.result()
            except RuntimeError as e:  # the comparator is optional
                cmp_err = e
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    # the comparator library: bench.py reports its section as unavailable
    # when it did not build
    if cmp_job is not None and cmp_err is None:
        tmp = CMP_LIB + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp, cmp_obj],
                           capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, CMP_LIB)
    elif cmp_err is not None and verbose:
        print(f"comparator not built: {cmp_err}", file=sys.stderr)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc and os.path.exists(CPU_SRC):
        tmp = CPU_LIB + f".tmp{os.getpid()}"
        r = subprocess.run([cc, "-O3", "-fPIC", "-shared", "-pthread", "-o", tmp, CPU_SRC],
                           capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, CPU_LIB)
        elif verbose:
            print("host comparator not built:\n" + r.stderr, file=sys.stderr)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
