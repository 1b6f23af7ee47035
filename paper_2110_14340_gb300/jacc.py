"""Python binding of libjacc.so (ctypes).  Argument marshalling only.

Every computation happens in the library's CUDA kernels; this module turns
torch tensors into device pointers and Python values into the C structs of
include/jacc.h.  If the library is missing, `lib()` raises: there is no
fallback path.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libjacc.so")

MAX_DIMS = 8
MAX_LOOPS = 8
NUM_TILES = 24

OK = 0
ERR_INVALID_ARG, ERR_OUT_OF_BOUNDS, ERR_OVERFLOW, ERR_CUDA = -1, -2, -3, -4
ERR_COMPILE, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_NOMEM = -5, -6, -7, -8
STATUS_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OUT_OF_BOUNDS", -3: "OVERFLOW", -4: "CUDA", -5: "COMPILE",
                -6: "TIMEOUT", -7: "UNSUPPORTED", -8: "NOMEM"}

STENCIL_5PT, STENCIL_7PT, STENCIL_27PT, STENCIL_19PT = 5, 7, 27, 19
F32, F64 = 32, 64
DIRICHLET, PERIODIC = 0, 1
ARITH_AUTO, ARITH_NATIVE = 0, 1
SPEC_JIT = 1
SPEC_CLUSTER = 2
SWEEP_GRAPH = 1


class JaccError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"jacc status {status} ({STATUS_NAMES.get(status, '?')}): {msg}")
        self.status = status


class Loop(C.Structure):
    _fields_ = [("lo", C.c_int64), ("hi", C.c_int64), ("step", C.c_int64)]


class Ref(C.Structure):
    _fields_ = [("array_id", C.c_int32), ("ndim", C.c_int32), ("is_write", C.c_int32), ("reserved", C.c_int32),
                ("coef", (C.c_int64 * MAX_LOOPS) * MAX_DIMS), ("off", C.c_int64 * MAX_DIMS)]


class Array(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("reserved", C.c_int32), ("extent", C.c_int64 * MAX_DIMS)]


class Region(C.Structure):
    _fields_ = [("has_read", C.c_int32), ("has_write", C.c_int32),
                ("rlo", C.c_int64 * MAX_DIMS), ("rhi", C.c_int64 * MAX_DIMS),
                ("wlo", C.c_int64 * MAX_DIMS), ("whi", C.c_int64 * MAX_DIMS),
                ("rlin_lo", C.c_int64), ("rlin_hi", C.c_int64), ("wlin_lo", C.c_int64), ("wlin_hi", C.c_int64)]


class KernelDesc(C.Structure):
    _fields_ = [("stencil", C.c_int32), ("dtype", C.c_int32), ("boundary", C.c_int32), ("tile_id", C.c_int32),
                ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64), ("coeffs", C.c_double * 4),
                ("arith", C.c_int32), ("flags", C.c_uint32), ("tblock", C.c_int32), ("reserved", C.c_int32)]


class KernelInfo(C.Structure):
    _fields_ = [("tile_id", C.c_int32), ("jit", C.c_int32), ("fixed_point", C.c_int32), ("tblock", C.c_int32),
                ("block", C.c_int32 * 3), ("grid", C.c_int32 * 3), ("compile_ms", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("u0", C.c_void_p), ("u1", C.c_void_p)]


class BatchConfig(C.Structure):
    _fields_ = [("item_points", C.c_int32), ("ctas_per_sm", C.c_int32), ("order", C.c_int32),
                ("timeout_ms", C.c_int32), ("test_stall_ticket", C.c_int64), ("group_bytes", C.c_int64),
                ("march", C.c_int32), ("test_stall_row", C.c_int32)]


class TuneTable(C.Structure):
    _fields_ = [("stencil", C.c_int32), ("dtype", C.c_int32), ("side", C.c_double),
                ("ms", C.c_double * NUM_TILES), ("valid", C.c_int32 * NUM_TILES)]


class CostModelEval(C.Structure):
    _fields_ = [("pick", C.c_int32), ("fallback", C.c_int32), ("gap", C.c_double), ("regret", C.c_double),
                ("regret_topk", C.c_double), ("search_ms_topk", C.c_double)]


class BatchTile(C.Structure):
    _fields_ = [("rows", C.c_int32), ("cols", C.c_int32), ("nitems", C.c_int32), ("group", C.c_int32)]


class TuneResult(C.Structure):
    _fields_ = [("ms", C.c_double * NUM_TILES), ("valid", C.c_int32 * NUM_TILES), ("best_tile", C.c_int32),
                ("reserved", C.c_int32), ("best_ms", C.c_double)]


class LoopAffine(C.Structure):
    _fields_ = [("lo", C.c_int64), ("hi", C.c_int64), ("lo_coef", C.c_int64 * MAX_LOOPS),
                ("hi_coef", C.c_int64 * MAX_LOOPS)]


class Box(C.Structure):
    _fields_ = [("array_id", C.c_int32), ("is_write", C.c_int32), ("exact", C.c_int32), ("reserved", C.c_int32),
                ("lo", C.c_int64 * MAX_DIMS), ("hi", C.c_int64 * MAX_DIMS)]


class Tile(C.Structure):
    _fields_ = [("bx", C.c_int32), ("by", C.c_int32), ("vec16", C.c_int32), ("zc", C.c_int32)]


# Every symbol include/jacc.h declares, with its argument and result types.
P = C.c_void_p
SIGNATURES = {
    "jacc_last_error": ([], C.c_char_p),
    "jacc_version": ([], C.c_char_p),
    "jacc_region_analyze": ([C.c_int32, P, C.c_int32, P, C.c_int32, P, P], C.c_int32),
    "jacc_region_analyze_affine": ([C.c_int32, P, C.c_int32, P, C.c_int32, P, P], C.c_int32),
    "jacc_region_boxes": ([C.c_int32, P, C.c_int32, P, C.c_int32, P, P, C.c_int32, P], C.c_int32),
    "jacc_region_boxes_affine": ([C.c_int32, P, C.c_int32, P, C.c_int32, P, P, C.c_int32, P], C.c_int32),
    "jacc_specialize": ([P, P], C.c_int32),
    "jacc_kernel_info": ([P, P], C.c_int32),
    "jacc_release": ([P], C.c_int32),
    "jacc_kernel_status": ([P, P], C.c_int32),
    "jacc_kernel_set_wait": ([P, C.c_int32, C.c_int32], C.c_int32),
    "jacc_tile_info": ([C.c_int32, P], C.c_int32),
    "jacc_launch": ([P, P, P, P, C.c_size_t], C.c_int32),
    "jacc_launch_static": ([P, P, P, P, C.c_size_t], C.c_int32),
    "jacc_sweep": ([P, P, P, C.c_int32, P, C.c_uint32, C.c_size_t, P], C.c_int32),
    "jacc_sweep_host": ([P, P, P, P, P, C.c_int32, P, P, C.c_uint32, C.c_size_t, C.c_size_t, C.c_size_t, P],
                        C.c_int32),
    "jacc_sweep_until": ([P, P, P, C.c_int32, C.c_double, P, P, C.c_size_t], C.c_int32),
    "jacc_sweep_coeffs": ([P, P, P, C.c_int32, P, C.c_int32, P, C.c_uint32, C.c_size_t, P], C.c_int32),
    "jacc_sched_create": ([C.c_int32, C.c_uint32, C.c_size_t, P], C.c_int32),
    "jacc_sched_sweep": ([P, P, P, P, C.c_int32, P, P], C.c_int32),
    "jacc_sched_copy": ([P, P, P, C.c_uint64, P], C.c_int32),
    "jacc_sched_nest_begin": ([P, C.c_int32, P, C.c_int32, P, C.c_int32, P, P, P, P, P], C.c_int32),
    "jacc_sched_nest_begin_affine": ([P, C.c_int32, P, C.c_int32, P, C.c_int32, P, P, P, P, P], C.c_int32),
    "jacc_sched_nest_end": ([P, C.c_int32], C.c_int32),
    "jacc_sched_task_info": ([P, C.c_int32, P, C.c_int32, P, P], C.c_int32),
    "jacc_sched_join": ([P, C.c_size_t], C.c_int32),
    "jacc_sched_live_events": ([P, P, P], C.c_int32),
    "jacc_sched_release": ([P], C.c_int32),
    "jacc_shutdown": ([], C.c_int32),
    "jacc_batch_create": ([C.c_int32, P, P, P], C.c_int32),
    "jacc_batch_configure": ([P, P], C.c_int32),
    "jacc_batch_get_config": ([P, P], C.c_int32),
    "jacc_batch_set_tiles": ([P, C.c_int32, P], C.c_int32),
    "jacc_batch_get_tiles": ([P, C.c_int32, P], C.c_int32),
    "jacc_batch_sweep": ([P, C.c_int32, P, C.c_uint32, C.c_size_t, P], C.c_int32),
    "jacc_batch_status": ([P, C.c_size_t], C.c_int32),
    "jacc_batch_tune": ([P, C.c_int32, C.c_size_t, P, P], C.c_int32),
    "jacc_batch_release": ([P], C.c_int32),
    "jacc_autotune": ([P, P, P, C.c_int32, C.c_int32, C.c_size_t, P], C.c_int32),
    "jacc_autotune_tiles": ([P, P, P, C.c_int32, C.c_int32, C.c_size_t, P, C.c_int32, P], C.c_int32),
    "jacc_autotune_forget": ([], C.c_int32),
    "jacc_costmodel_features": ([C.c_int32, C.c_double, C.c_int32, C.c_int32, P], C.c_int32),
    "jacc_costmodel_create": ([P, C.c_uint64, P], C.c_int32),
    "jacc_costmodel_set_params": ([P, P], C.c_int32),
    "jacc_costmodel_get_params": ([P, P], C.c_int32),
    "jacc_costmodel_loss_grad": ([P, P, P, C.c_int32, P, P, C.c_size_t], C.c_int32),
    "jacc_costmodel_train": ([P, P, P, C.c_int32, C.c_int32, C.c_float, C.c_size_t, P], C.c_int32),
    "jacc_costmodel_predict": ([P, P, C.c_int32, P, C.c_size_t], C.c_int32),
    "jacc_costmodel_pick": ([P, P, P, C.c_int32, P, P, P, C.c_size_t], C.c_int32),
    "jacc_costmodel_set_range": ([P, C.c_double, C.c_double, C.c_double], C.c_int32),
    "jacc_costmodel_choose": ([P, P, P, P, C.c_size_t, P, P], C.c_int32),
    "jacc_costmodel_choose_topk": ([P, P, P, P, C.c_size_t, C.c_int32, P], C.c_int32),
    "jacc_costmodel_fit_tables": ([P, C.c_int32, P, C.c_int32, C.c_float, C.c_size_t, P], C.c_int32),
    "jacc_costmodel_evaluate": ([P, C.c_int32, P, C.c_double, C.c_int32, C.c_size_t, P], C.c_int32),
    "jacc_costmodel_fixed_tile": ([C.c_int32, P, P], C.c_int32),
    "jacc_costmodel_regret": ([C.c_int32, P, P, P], C.c_int32),
    "jacc_costmodel_margin": ([P, C.c_int32, P, C.c_double, C.c_size_t, P], C.c_int32),
    "jacc_costmodel_save": ([P, C.c_char_p], C.c_int32),
    "jacc_costmodel_load": ([P, C.c_char_p], C.c_int32),
    "jacc_costmodel_release": ([P], C.c_int32),
}

_lib = None


def lib():
    """Load libjacc.so (built by paper_2110_14340_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libjacc.so not built ({LIB_PATH}); run paper_2110_14340_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(st):
    if st != OK:
        raise JaccError(st, lib().jacc_last_error().decode())


def version():
    return lib().jacc_version().decode()


# ----------------------------------------------------------------------------- region analysis

def _nest(loops, refs, arrays):
    """ctypes arrays for a loop nest: loops [(lo, hi, step)], refs [dict(array, coef, off, write)],
    arrays [extents]."""
    L = (Loop * max(1, len(loops)))()
    for k, (lo, hi, st) in enumerate(loops):
        L[k].lo, L[k].hi, L[k].step = lo, hi, st
    R = (Ref * max(1, len(refs)))()
    for r, ref in enumerate(refs):
        R[r].array_id = ref["array"]
        R[r].ndim = len(ref["off"])
        R[r].is_write = 1 if ref.get("write") else 0
        for d, row in enumerate(ref["coef"]):
            for k, c in enumerate(row):
                R[r].coef[d][k] = c
        for d, o in enumerate(ref["off"]):
            R[r].off[d] = o
    A = (Array * max(1, len(arrays)))()
    for a, ext in enumerate(arrays):
        A[a].ndim = len(ext)
        for d, e in enumerate(ext):
            A[a].extent[d] = e
    return L, R, A


def region_analyze(loops, refs, arrays):
    """Same argument format as the oracle's region_analyze; returns (status, [dict per array])."""
    L, R, A = _nest(loops, refs, arrays)
    O = (Region * max(1, len(arrays)))()
    st = lib().jacc_region_analyze(len(loops), C.cast(L, P), len(refs), C.cast(R, P), len(arrays), C.cast(A, P),
                                   C.cast(O, P))
    out = []
    for a, ext in enumerate(arrays):
        nd = len(ext)
        o = O[a]
        out.append(dict(has_read=bool(o.has_read), has_write=bool(o.has_write),
                        rlo=list(o.rlo[:nd]), rhi=list(o.rhi[:nd]), wlo=list(o.wlo[:nd]), whi=list(o.whi[:nd]),
                        rlin=(o.rlin_lo, o.rlin_hi), wlin=(o.wlin_lo, o.wlin_hi)))
    return st, out


def _region_list(O, arrays):
    out = []
    for a, ext in enumerate(arrays):
        nd = len(ext)
        o = O[a]
        out.append(dict(has_read=bool(o.has_read), has_write=bool(o.has_write),
                        rlo=list(o.rlo[:nd]), rhi=list(o.rhi[:nd]), wlo=list(o.wlo[:nd]), whi=list(o.whi[:nd]),
                        rlin=(o.rlin_lo, o.rlin_hi), wlin=(o.wlin_lo, o.wlin_hi)))
    return out


def _affine_loops(loops):
    L = (LoopAffine * max(1, len(loops)))()
    for k, (lo, hi, lc, hc) in enumerate(loops):
        L[k].lo, L[k].hi = lo, hi
        for m, c in enumerate(lc):
            L[k].lo_coef[m] = c
        for m, c in enumerate(hc):
            L[k].hi_coef[m] = c
    return L


def region_analyze_affine(loops, refs, arrays):
    """Triangular nests: loops [(lo, hi, lo_coef[], hi_coef[])], step 1; returns (status, [dict per array])."""
    L = _affine_loops(loops)
    _, R, A = _nest([(0, 0, 1)] * len(loops), refs, arrays)
    O = (Region * max(1, len(arrays)))()
    st = lib().jacc_region_analyze_affine(len(loops), C.cast(L, P), len(refs), C.cast(R, P), len(arrays),
                                          C.cast(A, P), C.cast(O, P))
    return st, _region_list(O, arrays)


def region_boxes_affine(loops, refs, arrays, max_boxes=256):
    """region_boxes for an affine nest: loops [(lo, hi, lo_coef[], hi_coef[])], step 1."""
    L = _affine_loops(loops)
    _, R, A = _nest([(0, 0, 1)] * len(loops), refs, arrays)
    B = (Box * max(1, max_boxes))()
    n = C.c_int32(0)
    st = lib().jacc_region_boxes_affine(len(loops), C.cast(L, P), len(refs), C.cast(R, P), len(arrays),
                                        C.cast(A, P), C.cast(B, P), max_boxes, C.byref(n))
    return st, _boxes_list(B, n, max_boxes, arrays)


def region_boxes(loops, refs, arrays, max_boxes=256):
    """Touched sets as a union of boxes; returns (status, [dict(array, write, exact, lo, hi)])."""
    L, R, A = _nest(loops, refs, arrays)
    B = (Box * max(1, max_boxes))()
    n = C.c_int32(0)
    st = lib().jacc_region_boxes(len(loops), C.cast(L, P), len(refs), C.cast(R, P), len(arrays), C.cast(A, P),
                                 C.cast(B, P), max_boxes, C.byref(n))
    return st, _boxes_list(B, n, max_boxes, arrays)


def _boxes_list(B, n, max_boxes, arrays):
    out = []
    for i in range(min(n.value, max_boxes)):
        b = B[i]
        nd = len(arrays[b.array_id])
        out.append(dict(array=b.array_id, write=bool(b.is_write), exact=bool(b.exact), lo=list(b.lo[:nd]),
                        hi=list(b.hi[:nd])))
    return out


# ----------------------------------------------------------------------------- kernels

def tile_info(tile_id):
    t = Tile()
    _check(lib().jacc_tile_info(tile_id, C.byref(t)))
    return dict(bx=t.bx, by=t.by, vec16=bool(t.vec16), zc=t.zc)


class Desc:
    """A kernel descriptor (jacc_kernel_desc) and the field shape it implies."""

    def __init__(self, stencil, dtype, nx, ny, nz=1, coeffs=(0.0, 0.0, 0.0, 0.0), tile_id=-1, jit=False,
                 arith=ARITH_AUTO, boundary=None, tblock=0, cluster=False):
        d = KernelDesc()
        d.stencil = stencil
        d.dtype = dtype
        d.boundary = (PERIODIC if stencil == STENCIL_27PT else DIRICHLET) if boundary is None else boundary
        d.tile_id = tile_id
        d.nx, d.ny, d.nz = nx, ny, nz
        cs = list(coeffs) + [0.0] * (4 - len(coeffs))
        for j in range(4):
            d.coeffs[j] = float(cs[j])
        d.arith = arith
        d.flags = (SPEC_JIT if jit else 0) | (SPEC_CLUSTER if cluster else 0)
        d.tblock = tblock
        self.desc = d
        self.shape = (ny, nx) if stencil == STENCIL_5PT else (nz, ny, nx)


class Kernel(Desc):
    """A specialised stencil kernel (owns one reference to the library handle)."""

    def __init__(self, *args, **kw):
        super().__init__(*args, **kw)
        h = C.c_void_p()
        _check(lib().jacc_specialize(C.byref(self.desc), C.byref(h)))
        self.handle = h

    def info(self):
        i = KernelInfo()
        _check(lib().jacc_kernel_info(self.handle, C.byref(i)))
        return dict(tile_id=i.tile_id, jit=bool(i.jit), fixed_point=bool(i.fixed_point), tblock=i.tblock,
                    block=tuple(i.block), grid=tuple(i.grid), compile_ms=i.compile_ms)

    def status(self):
        """Read and clear the device status word (0 or TIMEOUT); synchronises."""
        v = C.c_int32()
        _check(lib().jacc_kernel_status(self.handle, C.byref(v)))
        return v.value

    def set_wait(self, timeout_ms=0, stall_plane=-1):
        """Limit of each bounded device wait (0: default) and the stall test hook."""
        _check(lib().jacc_kernel_set_wait(self.handle, int(timeout_ms), int(stall_plane)))

    def release(self):
        if self.handle:
            _check(lib().jacc_release(self.handle))
            self.handle = None

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.jacc_release(self.handle)
        except Exception:
            pass


def specialize(*args, **kw):
    return Kernel(*args, **kw)


def _field(k, t, name):
    import torch
    want = torch.float64 if k.desc.dtype == F64 else torch.float32
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != want or not t.is_contiguous() or tuple(t.shape) != k.shape:
        raise ValueError(f"{name} must be a contiguous {want} tensor of shape {k.shape}")
    return t.data_ptr()


def _resid(r):
    import torch
    if r is None:
        return None
    if not isinstance(r, torch.Tensor) or not r.is_cuda or r.dtype != torch.float64 or not r.is_contiguous():
        raise ValueError("resid must be a contiguous CUDA float64 tensor")
    return r.data_ptr()


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def launch(k, u_in, u_out, resid=None, stream=None):
    """One sweep u_in -> u_out; resid (1 double) receives the reduction."""
    if resid is not None and resid.numel() < 1:
        raise ValueError("resid needs one element")
    _check(lib().jacc_launch(k.handle, _field(k, u_in, "u_in"), _field(k, u_out, "u_out"), _resid(resid),
                             _stream(stream)))


def sweep(k, u0, u1, nsweeps, resid=None, graph=True, stream=None):
    """nsweeps ping-pong sweeps; returns 0 if the result is in u0, 1 if in u1."""
    if resid is not None and resid.numel() < nsweeps:
        raise ValueError("resid needs nsweeps elements")
    fb = C.c_int32(-1)
    _check(lib().jacc_sweep(k.handle, _field(k, u0, "u0"), _field(k, u1, "u1"), nsweeps, _resid(resid),
                            SWEEP_GRAPH if graph else 0, _stream(stream), C.byref(fb)))
    return fb.value


def _host_field(k, t, name):
    import torch
    want = torch.float64 if k.desc.dtype == F64 else torch.float32
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name} must be a CPU tensor")
    if t.dtype != want or not t.is_contiguous() or tuple(t.shape) != k.shape:
        raise ValueError(f"{name} must be a contiguous {want} tensor of shape {k.shape}")
    return t.data_ptr()


def sweep_host(k, u_host, result_host, u0, u1, nsweeps, resid=None, resid_host=None, graph=True, stream=None,
               wait_event=None, done_event=None):
    """jacc_sweep_host: copy u_host (CPU tensor; pinned for asynchronous copies) into
    u0, run the sequence, copy the result field into result_host (and the residuals
    into resid_host, a CPU float64 tensor, which needs resid).  The sweeps wait for
    wait_event and done_event is recorded after them (torch.cuda.Event, optional).
    Returns 0 if the device result is in u0, 1 if in u1.  The host tensors must stay
    alive until the stream has run the copies."""
    import torch
    if resid is not None and resid.numel() < nsweeps:
        raise ValueError("resid needs nsweeps elements")
    rh = None
    if resid_host is not None:
        if (not isinstance(resid_host, torch.Tensor) or resid_host.is_cuda or resid_host.dtype != torch.float64
                or not resid_host.is_contiguous() or resid_host.numel() < nsweeps):
            raise ValueError("resid_host must be a contiguous CPU float64 tensor of nsweeps elements")
        rh = resid_host.data_ptr()
    fb = C.c_int32(-1)
    _check(lib().jacc_sweep_host(k.handle, _host_field(k, u_host, "u_host"), _host_field(k, result_host, "result_host"),
                                 _field(k, u0, "u0"), _field(k, u1, "u1"), nsweeps, _resid(resid), rh,
                                 SWEEP_GRAPH if graph else 0, _stream(stream), _event(wait_event),
                                 _event(done_event, create=True), C.byref(fb)))
    return fb.value


def _event(e, create=False):
    """A torch.cuda.Event as the cudaEvent_t integer (0 for None).  torch creates an
    event on its first record: one never recorded is nothing to wait for, and one
    the library is to record is created here first."""
    if e is None:
        return 0
    if e.cuda_event == 0:
        if not create:
            return 0
        e.record()
    return e.cuda_event


def sweep_coeffs(k, u0, u1, nsweeps, fields, resid=None, graph=True, stream=None):
    """Sweeps of a 19-point variable-coefficient kernel with its 12 coefficient fields
    (a0 a1 a2 a3 b0 b1 b2 c0 c1 c2 wrk1 bnd: contiguous CUDA float32 tensors of the field's
    shape).  Returns 0 if the result is in u0, 1 if in u1."""
    import torch
    if len(fields) != 12:
        raise ValueError("twelve coefficient fields")
    for f in fields:
        if (not isinstance(f, torch.Tensor) or not f.is_cuda or f.dtype != torch.float32 or not f.is_contiguous()
                or tuple(f.shape) != tuple(k.shape)):
            raise ValueError("coefficient fields must be contiguous CUDA float32 tensors of the field's shape")
    if resid is not None and resid.numel() < nsweeps:
        raise ValueError("resid needs nsweeps elements")
    table = (C.c_void_p * 12)(*[f.data_ptr() for f in fields])
    fb = C.c_int32(-1)
    _check(lib().jacc_sweep_coeffs(k.handle, _field(k, u0, "u0"), _field(k, u1, "u1"), nsweeps, table, 12,
                                   _resid(resid), SWEEP_GRAPH if graph else 0, _stream(stream), C.byref(fb)))
    return fb.value


def sweep_until(k, u0, u1, max_sweeps, tol, resid, status, stream=None):
    """Sweeps until a residual <= tol or max_sweeps; device-side loop (no host wait).

    resid: CUDA float64 tensor of >= max_sweeps elements; status: CUDA int32
    tensor of >= 2 elements, receiving (sweeps run, result buffer 0/1)."""
    import torch
    if resid.numel() < max_sweeps:
        raise ValueError("resid needs max_sweeps elements")
    if not (isinstance(status, torch.Tensor) and status.is_cuda and status.dtype == torch.int32
            and status.is_contiguous() and status.numel() >= 2):
        raise ValueError("status must be a contiguous CUDA int32 tensor of >= 2 elements")
    _check(lib().jacc_sweep_until(k.handle, _field(k, u0, "u0"), _field(k, u1, "u1"), int(max_sweeps), float(tol),
                                  _resid(resid), status.data_ptr(), _stream(stream)))


def shutdown():
    if _lib is not None:
        _check(_lib.jacc_shutdown())


# ----------------------------------------------------------------------------- async scheduler

SCHED_DRY_RUN = 1


class Sched:
    """Region-driven asynchronous scheduler over a pool of streams (dry_run: no CUDA call)."""

    def __init__(self, nstreams=8, dry_run=False, origin=None):
        h = C.c_void_p()
        _check(lib().jacc_sched_create(int(nstreams), SCHED_DRY_RUN if dry_run else 0,
                                       0 if dry_run else _stream(origin), C.byref(h)))
        self.handle = h

    def sweep(self, k, u0, u1, nsweeps, resid=None):
        t = C.c_int32(-1)
        _check(lib().jacc_sched_sweep(self.handle, k.handle, _field(k, u0, "u0"), _field(k, u1, "u1"), nsweeps,
                                      _resid(resid), C.byref(t)))
        return t.value

    def copy(self, dst, src, nbytes):
        """dst, src: device addresses (ints) or CUDA tensors."""
        d = dst.data_ptr() if hasattr(dst, "data_ptr") else int(dst)
        c = src.data_ptr() if hasattr(src, "data_ptr") else int(src)
        t = C.c_int32(-1)
        _check(lib().jacc_sched_copy(self.handle, C.c_void_p(d), C.c_void_p(c), C.c_uint64(int(nbytes)),
                                     C.byref(t)))
        return t.value

    def nest_begin(self, loops, refs, arrays, bases, elem_bytes):
        """A task described by its loop nest; returns (task id, stream handle as int)."""
        L, R, A = _nest(loops, refs, arrays)
        B = (C.c_uint64 * max(1, len(arrays)))(*[int(b) for b in bases])
        E = (C.c_int32 * max(1, len(arrays)))(*[int(e) for e in elem_bytes])
        t = C.c_int32(-1)
        st = C.c_size_t(0)
        _check(lib().jacc_sched_nest_begin(self.handle, len(loops), C.cast(L, P), len(refs), C.cast(R, P),
                                           len(arrays), C.cast(A, P), C.cast(B, P), C.cast(E, P), C.byref(t),
                                           C.byref(st)))
        return t.value, st.value

    def nest_begin_affine(self, loops, refs, arrays, bases, elem_bytes):
        """nest_begin for an affine nest: loops [(lo, hi, lo_coef[], hi_coef[])], step 1."""
        L = _affine_loops(loops)
        _, R, A = _nest([(0, 0, 1)] * len(loops), refs, arrays)
        B = (C.c_uint64 * max(1, len(arrays)))(*[int(b) for b in bases])
        E = (C.c_int32 * max(1, len(arrays)))(*[int(e) for e in elem_bytes])
        t = C.c_int32(-1)
        st = C.c_size_t(0)
        _check(lib().jacc_sched_nest_begin_affine(self.handle, len(loops), C.cast(L, P), len(refs), C.cast(R, P),
                                                  len(arrays), C.cast(A, P), C.cast(B, P), C.cast(E, P), C.byref(t),
                                                  C.byref(st)))
        return t.value, st.value

    def nest_end(self, task):
        _check(lib().jacc_sched_nest_end(self.handle, int(task)))

    def info(self, task, max_deps=4096):
        d = (C.c_int32 * max_deps)()
        n = C.c_int32(0)
        s = C.c_int32(-1)
        _check(lib().jacc_sched_task_info(self.handle, int(task), d, max_deps, C.byref(n), C.byref(s)))
        return list(d[:min(n.value, max_deps)]), s.value

    def live_events(self):
        """(tasks still holding a completion event, tasks submitted), after retiring completed ones."""
        e = C.c_int64(0)
        n = C.c_int64(0)
        _check(lib().jacc_sched_live_events(self.handle, C.byref(e), C.byref(n)))
        return e.value, n.value

    def join(self, stream=None):
        _check(lib().jacc_sched_join(self.handle, _stream(stream)))

    def release(self):
        if self.handle:
            _check(lib().jacc_sched_release(self.handle))
            self.handle = None


# ----------------------------------------------------------------------------- batched sweeps

def _cfg_dict(c):
    return dict(item_points=c.item_points, ctas_per_sm=c.ctas_per_sm, order=c.order, timeout_ms=c.timeout_ms,
                test_stall_ticket=c.test_stall_ticket, group_bytes=c.group_bytes, march=c.march,
                test_stall_row=c.test_stall_row)


def _cfg_struct(item_points=0, ctas_per_sm=0, order=0, timeout_ms=0, test_stall_ticket=-1, group_bytes=0, march=0,
                test_stall_row=0):
    c = BatchConfig()
    c.item_points, c.ctas_per_sm, c.order = item_points, ctas_per_sm, order
    c.timeout_ms, c.test_stall_ticket = timeout_ms, test_stall_ticket
    c.group_bytes, c.march, c.test_stall_row = group_bytes, march, test_stall_row
    return c


class Batch:
    """Many 2D 5-point FP64 grids swept in one persistent launch.

    fields: list of (u0, u1) CUDA float64 tensor pairs of shape (ny, nx)."""

    def __init__(self, fields, **cfg):
        import torch
        n = len(fields)
        G = (Grid * n)()
        for g, (a, b) in enumerate(fields):
            for t in (a, b):
                if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or \
                        not t.is_contiguous() or t.dim() != 2:
                    raise ValueError("batch fields must be contiguous 2D CUDA float64 tensors")
            if a.shape != b.shape:
                raise ValueError("u0 and u1 of a grid must have the same shape")
            G[g].ny, G[g].nx = a.shape
            G[g].u0, G[g].u1 = a.data_ptr(), b.data_ptr()
        self.n = n
        self.fields = list(fields)
        h = C.c_void_p()
        c = _cfg_struct(**cfg) if cfg else None
        _check(lib().jacc_batch_create(n, C.cast(G, P), C.byref(c) if c is not None else None, C.byref(h)))
        self.handle = h

    def configure(self, **cfg):
        _check(lib().jacc_batch_configure(self.handle, C.byref(_cfg_struct(**cfg))))

    def config(self):
        c = BatchConfig()
        _check(lib().jacc_batch_get_config(self.handle, C.byref(c)))
        return _cfg_dict(c)

    def sweep(self, nsweeps, resid=None, graph=True, stream=None):
        if resid is not None and resid.numel() < self.n * nsweeps:
            raise ValueError("resid needs ngrids * nsweeps elements")
        fb = C.c_int32(-1)
        _check(lib().jacc_batch_sweep(self.handle, nsweeps, _resid(resid), SWEEP_GRAPH if graph else 0,
                                      _stream(stream), C.byref(fb)))
        return fb.value

    def status(self, stream=None):
        """JACC_OK or the status of the last run (raises JaccError on a timeout)."""
        _check(lib().jacc_batch_status(self.handle, _stream(stream)))

    def tiles(self):
        """Per grid: dict(rows, cols, nitems, group)."""
        T = (BatchTile * self.n)()
        _check(lib().jacc_batch_get_tiles(self.handle, self.n, C.cast(T, P)))
        return [dict(rows=t.rows, cols=t.cols, nitems=t.nitems, group=t.group) for t in T]

    def set_tiles(self, tiles):
        """tiles: per grid (rows, cols); 0 = the default for item_points."""
        if len(tiles) != self.n:
            raise ValueError("one tile per grid")
        T = (BatchTile * self.n)()
        for g, (r, c) in enumerate(tiles):
            T[g].rows, T[g].cols = int(r), int(c)
        _check(lib().jacc_batch_set_tiles(self.handle, self.n, C.cast(T, P)))

    def tune(self, probe_sweeps=20, stream=None):
        c = BatchConfig()
        ms = C.c_double()
        _check(lib().jacc_batch_tune(self.handle, probe_sweeps, _stream(stream), C.byref(c), C.byref(ms)))
        return _cfg_dict(c), ms.value

    def release(self):
        if self.handle:
            _check(lib().jacc_batch_release(self.handle))
            self.handle = None

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.jacc_batch_release(self.handle)
        except Exception:
            pass


# ----------------------------------------------------------------------------- autotuner

def autotune(k_args, u0, u1, sweeps_per_rep=2, reps=3, stream=None):
    """Exhaustive tile search for the descriptor Kernel(**k_args) (tile_id ignored).

    Returns dict(ms=[24 floats, inf if invalid], valid=[24 bools], best_tile, best_ms)."""
    k = Desc(**dict(k_args, tile_id=-1))
    r = TuneResult()
    _check(lib().jacc_autotune(C.byref(k.desc), _field(k, u0, "u0"), _field(k, u1, "u1"), sweeps_per_rep, reps,
                               _stream(stream), C.byref(r)))
    return dict(ms=list(r.ms), valid=[bool(v) for v in r.valid], best_tile=r.best_tile, best_ms=r.best_ms)


def autotune_tiles(k_args, u0, u1, tiles, sweeps_per_rep=2, reps=3, stream=None):
    """autotune restricted to the tile ids in `tiles`; same result dict (untimed tiles invalid)."""
    k = Desc(**dict(k_args, tile_id=-1))
    r = TuneResult()
    arr = (C.c_int32 * len(tiles))(*[int(t) for t in tiles])
    _check(lib().jacc_autotune_tiles(C.byref(k.desc), _field(k, u0, "u0"), _field(k, u1, "u1"), sweeps_per_rep, reps,
                                     _stream(stream), arr, len(tiles), C.byref(r)))
    return dict(ms=list(r.ms), valid=[bool(v) for v in r.valid], best_tile=r.best_tile, best_ms=r.best_ms)


def autotune_forget():
    _check(lib().jacc_autotune_forget())


# ----------------------------------------------------------------------------- learned cost model

MLP_NPARAM = 8705


def features(stencil, side, dtype, tile):
    out = (C.c_float * 4)()
    _check(lib().jacc_costmodel_features(stencil, float(side), dtype, tile, out))
    return list(out)


def tune_tables(tables):
    """ctypes array of jacc_tune_table rows from dicts (stencil, dtype, side, ms[24], valid[24])."""
    T = (TuneTable * max(1, len(tables)))()
    for i, q in enumerate(tables):
        T[i].stencil, T[i].dtype, T[i].side = int(q["stencil"]), int(q["dtype"]), float(q["side"])
        for t in range(NUM_TILES):
            v = bool(q["valid"][t])
            T[i].valid[t] = 1 if v else 0
            T[i].ms[t] = float(q["ms"][t]) if v else 0.0
    return T


def fixed_tile(tables):
    """The best single tile over the tables (the method without the model)."""
    T = tune_tables(tables)
    t = C.c_int32(-1)
    _check(lib().jacc_costmodel_fixed_tile(len(tables), C.cast(T, P), C.byref(t)))
    return t.value


def regret(tables, picks):
    """Per query: ms[pick] / best ms - 1, by the library."""
    T = tune_tables(tables)
    pk = (C.c_int32 * max(1, len(tables)))(*[int(p) for p in picks])
    out = (C.c_double * max(1, len(tables)))()
    _check(lib().jacc_costmodel_regret(len(tables), C.cast(T, P), C.cast(pk, P), C.cast(out, P)))
    return list(out[:len(tables)])


def _f32(t, n=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA float32 tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} needs {n} elements")
    return t.data_ptr()


class CostModel:
    """The MLP cost model; parameters live on the device."""

    def __init__(self, init_params=None, seed=5):
        import numpy as np
        h = C.c_void_p()
        if init_params is not None:
            p = np.ascontiguousarray(init_params, dtype=np.float32)
            assert p.size == MLP_NPARAM
            _check(lib().jacc_costmodel_create(p.ctypes.data_as(P), seed, C.byref(h)))
        else:
            _check(lib().jacc_costmodel_create(None, seed, C.byref(h)))
        self.handle = h

    def params(self):
        import numpy as np
        p = np.empty(MLP_NPARAM, dtype=np.float32)
        _check(lib().jacc_costmodel_get_params(self.handle, p.ctypes.data_as(P)))
        return p

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().jacc_costmodel_set_params(self.handle, p.ctypes.data_as(P)))

    def loss_grad(self, x, y, stream=None):
        import torch
        n = y.numel()
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        _check(lib().jacc_costmodel_loss_grad(self.handle, _f32(x, 4 * n, "x"), _f32(y, n, "y"), n, g.data_ptr(),
                                              loss.data_ptr(), _stream(stream)))
        return loss, g

    def train(self, x, y, epochs, lr=1e-3, stream=None):
        import torch
        n = y.numel()
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        _check(lib().jacc_costmodel_train(self.handle, _f32(x, 4 * n, "x"), _f32(y, n, "y"), n, epochs, lr,
                                          _stream(stream), loss.data_ptr()))
        return loss

    def predict(self, x, stream=None):
        import torch
        n = x.numel() // 4
        y = torch.empty(n, dtype=torch.float32, device=x.device)
        _check(lib().jacc_costmodel_predict(self.handle, _f32(x, 4 * n, "x"), n, y.data_ptr(), _stream(stream)))
        return y

    def pick(self, feats, valid, stream=None):
        """feats [nq, 24, 4] float32, valid [nq, 24] int32 (CUDA) -> (pred, pick, gap)."""
        import torch
        nq = feats.shape[0]
        pred = torch.empty(nq * NUM_TILES, dtype=torch.float32, device=feats.device)
        pick = torch.empty(nq, dtype=torch.int32, device=feats.device)
        gap = torch.empty(nq, dtype=torch.float32, device=feats.device)
        if valid.dtype != torch.int32 or not valid.is_cuda or not valid.is_contiguous():
            raise ValueError("valid must be a contiguous CUDA int32 tensor")
        _check(lib().jacc_costmodel_pick(self.handle, _f32(feats, nq * NUM_TILES * 4, "feats"), valid.data_ptr(), nq,
                                         pred.data_ptr(), pick.data_ptr(), gap.data_ptr(), _stream(stream)))
        return pred.view(nq, NUM_TILES), pick, gap

    def set_range(self, side_lo, side_hi, margin):
        _check(lib().jacc_costmodel_set_range(self.handle, side_lo, side_hi, margin))

    def choose(self, k_args, u0=None, u1=None, stream=None):
        """(tile, used_fallback) for the descriptor Kernel(**k_args)."""
        k = Desc(**dict(k_args, tile_id=-1))
        p0 = _field(k, u0, "u0") if u0 is not None else None
        p1 = _field(k, u1, "u1") if u1 is not None else None
        t = C.c_int32(-1)
        fb = C.c_int32(0)
        _check(lib().jacc_costmodel_choose(self.handle, C.byref(k.desc), p0, p1, _stream(stream), C.byref(t),
                                           C.byref(fb)))
        return t.value, bool(fb.value)

    def choose_topk(self, k_args, u0, u1, k, stream=None):
        """The fastest of the model's k best-predicted tiles, timed on u0/u1."""
        d = Desc(**dict(k_args, tile_id=-1))
        t = C.c_int32(-1)
        _check(lib().jacc_costmodel_choose_topk(self.handle, C.byref(d.desc), _field(d, u0, "u0"),
                                                _field(d, u1, "u1"), _stream(stream), int(k), C.byref(t)))
        return t.value

    def fit_tables(self, tables, epochs, lr=1e-3, stream=None):
        """Train on autotuner tables (list of dict(stencil, dtype, side, ms[24], valid[24])); returns the final MSE."""
        T = tune_tables(tables)
        mse = C.c_double(0.0)
        _check(lib().jacc_costmodel_fit_tables(self.handle, len(tables), C.cast(T, P), int(epochs), float(lr),
                                               _stream(stream), C.byref(mse)))
        return mse.value

    def evaluate(self, tables, margin=0.0, topk=1, stream=None):
        """Per query: dict(pick, fallback, gap, regret, regret_topk, search_ms_topk)."""
        T = tune_tables(tables)
        E = (CostModelEval * len(tables))()
        _check(lib().jacc_costmodel_evaluate(self.handle, len(tables), C.cast(T, P), float(margin), int(topk),
                                             _stream(stream), C.cast(E, P)))
        return [dict(pick=e.pick, fallback=bool(e.fallback), gap=e.gap, regret=e.regret, regret_topk=e.regret_topk,
                     search_ms_topk=e.search_ms_topk) for e in E]

    def margin(self, tables, fraction, stream=None):
        """The decision margin at which at most `fraction` of these queries fall back."""
        T = tune_tables(tables)
        m = C.c_double(0.0)
        _check(lib().jacc_costmodel_margin(self.handle, len(tables), C.cast(T, P), float(fraction), _stream(stream),
                                           C.byref(m)))
        return m.value

    def save(self, path):
        _check(lib().jacc_costmodel_save(self.handle, path.encode()))

    def load(self, path):
        _check(lib().jacc_costmodel_load(self.handle, path.encode()))

    def release(self):
        if self.handle:
            _check(lib().jacc_costmodel_release(self.handle))
            self.handle = None

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.jacc_costmodel_release(self.handle)
        except Exception:
            pass
