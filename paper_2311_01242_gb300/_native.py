"""Build and load libvqe (the CUDA library behind include/vqe.h).

The library is compiled in-tree for sm_103a with nvcc and loaded with ctypes.
There is no fallback: if the shared library is missing or cannot be loaded,
every entry point raises.
"""
import ctypes
import os
import shutil
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_SRC_DIR = os.path.join(_HERE, "csrc")
_BUILD_DIR = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD_DIR, "libvqe.so")
HEADER = os.path.join(_ROOT, "include", "vqe.h")

SOURCES = ["vqe_kernels.cu", "vqe_batch.cu", "vqe_host.cpp", "vqe_static.cu", "vqe_mlp.cu", "vqe_probe.cu",
           "vqe_aux.cu", "vqe_pool.cu", "vqe_phi.cu"]
DEPS = SOURCES + ["vqe_internal.h", "vqe_device.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC"]

_lock = threading.Lock()
_lib = None


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvqe")
    return p


def _stale():
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(_SRC_DIR, f) for f in DEPS] + [HEADER]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile libvqe for sm_103a (sources compiled in parallel, then linked).

    Safe to call from several processes at once: a file lock serialises builds.
    """
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(_BUILD_DIR, exist_ok=True)
    import fcntl
    with open(os.path.join(_BUILD_DIR, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        try:
            if not force and not _stale():
                return LIB_PATH
            return _build_locked(verbose)
        finally:
            fcntl.flock(lk, fcntl.LOCK_UN)


def _build_locked(verbose):
    nvcc = _nvcc()
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(_BUILD_DIR, src + ".o")
        cmd = [nvcc] + CFLAGS + ["-c", os.path.join(_SRC_DIR, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + out.decode(errors="replace"))
    tmp = LIB_PATH + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


c_i32, c_i64, c_u64, c_dbl, c_vp, c_sz = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                           ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t)
P = ctypes.POINTER

PROTOTYPES = {
    "vqe_version": (ctypes.c_int, []),
    "vqe_set_flags": (ctypes.c_int, [ctypes.c_int]),
    "vqe_last_error": (ctypes.c_char_p, []),
    "vqe_jordan_wigner": (ctypes.c_int, [ctypes.c_int, c_vp, c_vp, c_dbl, c_dbl, c_i64, c_vp, c_vp, c_vp,
                                         P(c_i64)]),
    "vqe_fold_frozen": (ctypes.c_int, [ctypes.c_int, c_vp, c_vp, c_dbl, ctypes.c_int, c_vp, ctypes.c_int, c_vp,
                                       c_vp, c_vp, P(c_dbl)]),
    "vqe_hcb_hamiltonian": (ctypes.c_int, [ctypes.c_int, c_vp, c_vp, c_dbl, c_dbl, c_i64, c_vp, c_vp, c_vp,
                                           P(c_i64)]),
    "vqe_create_hamiltonian": (ctypes.c_int, [ctypes.c_int, c_i64, c_vp, c_vp, c_vp, c_dbl, P(c_vp)]),
    "vqe_hamiltonian_info": (ctypes.c_int, [c_vp, P(ctypes.c_int), P(c_i64), P(c_i64), P(ctypes.c_int)]),
    "vqe_hamiltonian_terms": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp]),
    "vqe_set_coefs": (ctypes.c_int, [c_vp, c_vp, c_vp]),
    "vqe_destroy_hamiltonian": (None, [c_vp]),
    "vqe_create_ansatz": (ctypes.c_int, [ctypes.c_int, c_u64, c_i32, c_vp, P(c_vp)]),
    "vqe_create_ansatz_hcb": (ctypes.c_int, [ctypes.c_int, c_u64, c_i32, c_vp, P(c_vp)]),
    "vqe_ansatz_info": (ctypes.c_int, [c_vp, P(ctypes.c_int), P(c_i32), P(c_i64), P(c_i64)]),
    "vqe_destroy_ansatz": (None, [c_vp]),
    "vqe_workspace_bytes": (c_sz, [c_vp, c_vp, ctypes.c_int]),
    "vqe_energy": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "vqe_energy_grad": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "vqe_state": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "vqe_apply_hamiltonian": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "vqe_apply_hamiltonian_sector": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "vqe_pool_workspace_bytes": (c_sz, [c_vp, c_vp, c_vp]),
    "vqe_pool_gradients": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "vqe_create_batch": (ctypes.c_int, [ctypes.c_int, c_vp, c_vp, P(c_vp)]),
    "vqe_batch_max_params": (c_i32, [c_vp]),
    "vqe_batch_workspace_bytes": (c_sz, [c_vp, ctypes.c_int]),
    "vqe_batch_energy_grad": (ctypes.c_int, [c_vp, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_sz, c_vp]),
    "vqe_batch_host_workspace_bytes": (c_sz, [c_vp, ctypes.c_int]),
    "vqe_batch_energy_grad_host": (ctypes.c_int, [c_vp, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_sz, c_vp]),
    "vqe_batch_set_tuning": (ctypes.c_int, [c_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "vqe_batch_get_tuning": (ctypes.c_int, [c_vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int), P(c_i64)]),
    "vqe_batch_set_wait": (ctypes.c_int, [c_vp, c_i64, c_i32]),
    "vqe_batch_status": (ctypes.c_int, [c_vp, c_vp, c_sz, c_vp]),
    "vqe_destroy_batch": (None, [c_vp]),
    "vqe_batched_workspace_bytes": (c_sz, [ctypes.c_int, c_vp, c_vp, ctypes.c_int]),
    "vqe_energy_batched": (ctypes.c_int, [ctypes.c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "vqe_energy_grad_batched": (ctypes.c_int, [ctypes.c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "vqe_work_estimate": (ctypes.c_int, [c_vp, c_vp, ctypes.c_int, P(c_dbl), P(c_dbl)]),
    "vqe_work_counts": (ctypes.c_int, [c_vp, c_vp, P(c_i64), P(c_i64), P(c_dbl)]),
    "vqe_energy_grad_noalloc": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "vqe_probe_fp64": (ctypes.c_int, [P(c_dbl), P(c_dbl), P(c_dbl), P(ctypes.c_int), P(ctypes.c_int), P(c_sz),
                                      P(ctypes.c_int)]),
    "vqe_mlp_param_count": (c_i64, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "vqe_mlp_workspace_bytes": (c_sz, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "vqe_mlp_to_bf16": (ctypes.c_int, [c_i64, c_vp, c_vp, c_vp]),
    "vqe_mlp_forward": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_vp, c_vp, c_vp,
                                       c_vp, c_vp, c_sz, c_vp]),
    "vqe_mlp_loss_grad": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_vp, c_vp, c_vp,
                                         c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "vqe_mlp_adam": (ctypes.c_int, [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, c_vp, c_vp]),
}


def load(path=None):
    """Load (building first if needed) and return the ctypes library."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if path is None and _stale():
            build()
        if not os.path.exists(p):
            raise RuntimeError(f"libvqe not built: {p} is missing")
        lib = ctypes.CDLL(p)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def declared_symbols():
    """Function names declared in include/vqe.h."""
    import re
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(vqe_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))
