"""Build step for libjacc.so (sm_103a kernels + host runtime), in-tree.

Compiles every translation unit in parallel with nvcc / g++ and links
paper_2110_14340_gb300/_build/libjacc.so.  Rebuilds only what changed.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
KDIR = os.path.join(CSRC, "kernels")
HDIR = os.path.join(CSRC, "host")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libjacc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")

KERNEL_HEADERS = [os.path.join(KDIR, f) for f in ("jacc_device.cuh", "jacc_params.h", "tiles.h", "batched.h", "mlp.h")]
HOST_HEADERS = [os.path.join(HDIR, "jacc_internal.h"), os.path.join(ROOT, "include", "jacc.h")]


def _mtime(paths):
    return max(os.path.getmtime(p) for p in paths)


def _stale(out, deps):
    return not os.path.exists(out) or os.path.getmtime(out) < _mtime(deps)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _embed():
    out = os.path.join(BUILD, "jacc_embedded_src.inc")
    srcs = [os.path.join(KDIR, "jacc_device.cuh"), os.path.join(KDIR, "jacc_params.h")]
    if not _stale(out, srcs + [__file__]):
        return out
    dev = open(srcs[0]).read()
    par = open(srcs[1]).read()
    for t in (dev, par):
        assert ")JACCSRC\"" not in t
    with open(out + ".tmp", "w") as f:
        f.write('static const char kDeviceSource[] = R"JACCSRC(' + dev + ')JACCSRC";\n')
        f.write('static const char kParamsSource[] = R"JACCSRC(' + par + ')JACCSRC";\n')
    os.replace(out + ".tmp", out)
    return out


def _jobs():
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + KDIR, "-I" + BUILD]
    cu_flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v"] + inc
    jobs = []
    for st in (5, 7, 27):
        for dt in (32, 64):
            obj = os.path.join(BUILD, f"inst_{st}_{dt}.o")
            jobs.append((obj, KERNEL_HEADERS + [os.path.join(KDIR, "inst.cu")],
                         [NVCC] + cu_flags + [f"-DJACC_INST_STENCIL={st}", f"-DJACC_INST_DTYPE={dt}", "-c",
                                              os.path.join(KDIR, "inst.cu"), "-o", obj]))
    for name in ("aux.cu", "static_scratch.cu", "batched.cu", "mlp.cu", "jacobi_cluster.cu", "until.cu", "var19.cu",
                 "box27_tb2.cu"):
        obj = os.path.join(BUILD, name.replace(".cu", ".o"))
        jobs.append((obj, KERNEL_HEADERS + HOST_HEADERS + [os.path.join(KDIR, name)],
                     [NVCC] + cu_flags + ["-c", os.path.join(KDIR, name), "-o", obj]))
    cxx = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-Wextra", "-I/usr/local/cuda/include"] + inc
    for name in sorted(os.listdir(HDIR)):
        if name.endswith(".cpp"):
            obj = os.path.join(BUILD, name.replace(".cpp", ".o"))
            deps = HOST_HEADERS + [os.path.join(HDIR, name), os.path.join(KDIR, "jacc_params.h"),
                                   os.path.join(KDIR, "tiles.h")]
            if name == "sources.cpp":
                deps.append(os.path.join(BUILD, "jacc_embedded_src.inc"))
            jobs.append((obj, deps, cxx + ["-c", os.path.join(HDIR, name), "-o", obj]))
    return jobs


def build(force=False, verbose=False):
    """Compile and link libjacc.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    _embed()
    jobs = _jobs()
    todo = [j for j in jobs if force or _stale(j[0], j[1])]
    logs = {}
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            futs = {ex.submit(_run, cmd): obj for obj, _, cmd in todo}
            for f in cf.as_completed(futs):
                logs[futs[f]] = f.result()
    objs = [j[0] for j in jobs]
    if force or todo or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        _run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lnvrtc"])
        os.replace(tmp, LIB)
    if verbose:
        for obj, log in sorted(logs.items()):
            print(f"== {os.path.basename(obj)}\n{log}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
