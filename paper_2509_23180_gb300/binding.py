"""Thin Python binding of the C ABI in include/fpg.h (argument marshalling only).

Every step of the solve runs in the CUDA library libfpg.so; this module only
turns torch tensors (device memory, streams) into the plain pointers and sizes
the C functions take.  If the library is missing the import fails loudly: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfpg.so")

GEOMETRY = {"L": 0, "T": 1, "cross": 2, "chain": 3, "lattice": 4}
BOUNDARY = {"dirichlet": 0, "neumann_sides": 1}
RECT = {"dirichlet": 0, "neumann": 1, "periodic": 2}
SCHUR = {"reduced": 0, "literal": 1}
STATUS = {0: "FPG_OK", 1: "FPG_EINVAL", 2: "FPG_ENOMEM", 3: "FPG_ECUDA", 4: "FPG_ENOCONV",
          5: "FPG_ETIMEOUT", 6: "FPG_EUNSUPPORTED", 7: "FPG_EBUDGET"}
FPG_OK, FPG_EINVAL, FPG_ENOMEM, FPG_ECUDA, FPG_ENOCONV = 0, 1, 2, 3, 4
FPG_ETIMEOUT, FPG_EUNSUPPORTED, FPG_EBUDGET = 5, 6, 7
OPT_ARNOLDI_CLUSTER = 1
OPT_CUDA_GRAPHS = 2
OPT_PRECOND = 3
OPT_FUSED_FASTSOLVE = 4
OPT_ARNOLDI_CSZ = 5
OPT_ARNOLDI_THREADS = 6
OPT_DST_ENGINE = 7
OPT_SCHUR_TRANSFORM = 8
OPT_ARM_REFINE = 9
OPT_DST_BULK = 10
OPT_WAIT_LIMIT = 11
OPT_CLUSTER_FASTSOLVE = 12
OPT_DST_PAIRS = 13
OPT_THOMAS_WARPS = 14
OPT_THOMAS_PRODUCTS = 15
PRECOND = {"fft": 0, "none": 1, "jacobi": 2}
PHASES = ("precond", "schur", "arnoldi", "givens", "cycle_end", "setup_finish", "residual",
          "dst_forward", "thomas", "dst_inverse", "fast_solve_fused")
# fpg_fast_solve_path -> kernel names of the a1 phases
FAST_SOLVE_KERNELS = {
    0: {"dst_forward": "k_fft_forward", "thomas": "k_thomas_reg", "dst_inverse": "k_fft_inverse"},
    1: {"dst_forward": "k_dst_lines_fwd", "thomas": "k_thomas_reg", "dst_inverse": "k_dst_lines_inv"},
    2: {"dst_forward": "k_dense_forward", "thomas": "k_thomas_reg", "dst_inverse": "k_dense_inverse"},
    3: {"fast_solve_fused": "k_fast_solve_fused"},
    4: {},
    7: {"fast_solve_fused": "k_fast_solve_cluster"},
}


class DomainDesc(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int32), ("n", ctypes.c_int32), ("kappa", ctypes.c_double),
                ("nrhs", ctypes.c_int32), ("restart", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("max_iters", ctypes.c_int32), ("precond_precision", ctypes.c_int32),
                ("schur_mode", ctypes.c_int32), ("boundary", ctypes.c_int32), ("chain", ctypes.c_int32),
                ("lattice", ctypes.c_uint64)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("residual", ctypes.c_double), ("schur_residual", ctypes.c_double)]


class BatchDescC(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_domains", ctypes.c_int32), ("max_per_key", ctypes.c_int32),
                ("max_busy", ctypes.c_int32)]


class BatchStats(ctypes.Structure):
    _fields_ = [("resident", ctypes.c_int32), ("busy", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("open_tickets", ctypes.c_int32), ("pool_used", ctypes.c_int64), ("created", ctypes.c_int64),
                ("evicted", ctypes.c_int64)]


class TuneResult(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int32), ("mt", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("precond_ms", ctypes.c_double), ("arnoldi_ms", ctypes.c_double)]


class FpgError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        super().__init__(f"{where}: {STATUS.get(status, status)} {detail}".strip())
        self.status = status


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double
_SIGS = {
    "fpg_status_string": ([_I32], ctypes.c_char_p),
    "fpg_last_cuda_error": ([], ctypes.c_char_p),
    "fpg_version": ([], ctypes.c_char_p),
    "fpg_unknowns": ([_P, ctypes.POINTER(_I64)], _I32),
    "fpg_workspace_bytes": ([_P, ctypes.POINTER(ctypes.c_size_t)], _I32),
    "fpg_create_domain": ([_P, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)], _I32),
    "fpg_set_rhs": ([_P, _P, _I32], _I32),
    "fpg_set_rhs_host": ([_P, _P, _I32], _I32),
    "fpg_solve": ([_P, _P, _P], _I32),
    "fpg_solve_resume": ([_P, _P, _P], _I32),
    "fpg_solve_async": ([_P, _P], _I32),
    "fpg_solve_finish": ([_P, _P], _I32),
    "fpg_solve_host": ([_P, _P, _P, _P], _I32),
    "fpg_destroy_domain": ([_P], None),
    "fpg_solve_many": ([_P, _I32, _P, _P], _I32),
    "fpg_apply_precond": ([_P, _P, _P, _I32], _I32),
    "fpg_block_solve": ([_P, _I32, _P, _P, _I32], _I32),
    "fpg_apply_schur": ([_P, _P, _I32, _P, _I32], _I32),
    "fpg_arnoldi_mgs": ([_P, _P, _I32, _P, _P, _I64, _I32], _I32),
    "fpg_givens": ([_P, _P, _P, _P, _P, _P, _I32, _I32, _I32], _I32),
    "fpg_global_residual": ([_P, _P, _P, _P, _I32], _I32),
    "fpg_apply_global": ([_P, _P, _P, _I32], _I32),
    "fpg_set_option": ([_P, _I32, _I32], _I32),
    "fpg_set_stream": ([_P, _P], _I32),
    "fpg_autotune": ([_P, _P], _I32),
    "fpg_set_profiling": ([_P, _I32], _I32),
    "fpg_phase_stats": ([_P, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_D)], _I32),
    "fpg_launch_count": ([_P, ctypes.POINTER(_I64)], _I32),
    "fpg_fast_solve_path": ([_P, ctypes.POINTER(_I32)], _I32),
    "fpg_arnoldi_shape": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                           ctypes.POINTER(_I32)], _I32),
    "fpg_convert": ([_P, _I32, _P, _I32, _I64, _P], _I32),
    "fpg_neumann_workspace_bytes": ([_I32, _I32, _I32, ctypes.POINTER(ctypes.c_size_t)], _I32),
    "fpg_neumann_solve": ([_I32, _I32, _D, _D, _P, _P, _I32, _P, ctypes.c_size_t, _P], _I32),
    "fpg_rect_plan_bytes": ([_I32, _I32, _I32, _I32, ctypes.POINTER(ctypes.c_size_t)], _I32),
    "fpg_rect_plan_create": ([_I32, _I32, _I32, _D, _D, _I32, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)], _I32),
    "fpg_rect_solve": ([_P, _P, _P, _I32], _I32),
    "fpg_rect_plan_destroy": ([_P], None),
    "fpg_batch_create": ([_P, _P, ctypes.c_size_t, ctypes.POINTER(_P)], _I32),
    "fpg_batch_admit": ([_P, _P, _P, _P, ctypes.POINTER(_I64)], _I32),
    "fpg_batch_step": ([_P, _P, _I32, ctypes.POINTER(_I32)], _I32),
    "fpg_batch_poll": ([_P, _I64, ctypes.POINTER(_I32), _P], _I32),
    "fpg_batch_stats": ([_P, _P], _I32),
    "fpg_batch_destroy": ([_P], None),
    "fpg_set_history": ([_P, _P, _I32], _I32),
    "fpg_box_plan_bytes": ([_I32, _I32, _I32, _I32, ctypes.POINTER(ctypes.c_size_t)], _I32),
    "fpg_box_plan_create": ([_I32, _I32, _I32, _D, _D, _I32, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)], _I32),
    "fpg_box_solve": ([_P, _P, _P, _I32], _I32),
    "fpg_box_plan_destroy": ([_P], None),
    "fpg_periodic_workspace_bytes": ([_I32, _I32, _I32, ctypes.POINTER(ctypes.c_size_t)], _I32),
    "fpg_periodic_solve": ([_I32, _I32, _D, _D, _P, _P, _I32, _P, ctypes.c_size_t, _P], _I32),
    "fpg_probe_fma_peak": ([_I32, ctypes.POINTER(_D)], _I32),
    "fpg_fast_solve_noalloc": ([_I32, _D, _P, _P, _I32, _P], _I32),
}
EXPORTED = tuple(_SIGS)

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libfpg.so (built by paper_2509_23180_gb300.build) and declare its ABI."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2509_23180_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(status: int, where: str) -> int:
    if status not in (FPG_OK,):
        lib = load()
        detail = lib.fpg_last_cuda_error().decode() if status == FPG_ECUDA else ""
        raise FpgError(status, where, detail)
    return status


def make_desc(geometry="cross", n=64, kappa=0.0, nrhs=1, restart=30, rtol=1e-10, max_iters=None,
              precond_precision=64, schur_mode="reduced", boundary="dirichlet", chain=0,
              lattice=0) -> DomainDesc:
    if max_iters is None:
        max_iters = 50 * restart
    return DomainDesc(GEOMETRY[geometry] if isinstance(geometry, str) else int(geometry), int(n), float(kappa),
                      int(nrhs), int(restart), float(rtol), int(max_iters), int(precond_precision),
                      SCHUR[schur_mode] if isinstance(schur_mode, str) else int(schur_mode),
                      BOUNDARY[boundary] if isinstance(boundary, str) else int(boundary), int(chain),
                      int(lattice))


def unknowns(desc: DomainDesc) -> int:
    out = _I64()
    _check(load().fpg_unknowns(ctypes.byref(desc), ctypes.byref(out)), "fpg_unknowns")
    return int(out.value)


def workspace_bytes(desc: DomainDesc) -> int:
    out = ctypes.c_size_t()
    _check(load().fpg_workspace_bytes(ctypes.byref(desc), ctypes.byref(out)), "fpg_workspace_bytes")
    return int(out.value)


def _ptr(t) -> int:
    return t.data_ptr()


class Domain:
    """A domain handle with its caller-owned device workspace (a torch uint8 tensor)."""

    def __init__(self, desc: DomainDesc, stream=None, device="cuda"):
        import torch
        self.lib = load()
        self.desc = desc
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.nbytes = workspace_bytes(desc)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.N = unknowns(desc)
        self.nc = {3: ((2 * desc.chain - 1) * (desc.n + 1) - 1) * desc.n, 4: None}.get(desc.geometry, desc.n * desc.n)
        h = _P()
        _check(self.lib.fpg_create_domain(ctypes.byref(desc), _ptr(self.workspace), self.nbytes,
                                          self.stream.cuda_stream, ctypes.byref(h)), "fpg_create_domain")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fpg_destroy_domain(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- solve -----------------------------------------------------------
    def set_rhs(self, f, index: int = -1):
        _check(self.lib.fpg_set_rhs(self.handle, _ptr(f), index), "fpg_set_rhs")

    def set_rhs_host(self, f_host, index: int = -1):
        _check(self.lib.fpg_set_rhs_host(self.handle, _ptr(f_host), index), "fpg_set_rhs_host")

    def _infos(self):
        return (SolveInfo * self.desc.nrhs)()

    @staticmethod
    def _info_list(arr):
        return [{"iterations": i.iterations, "restarts": i.restarts, "status": i.status,
                 "residual": i.residual, "schur_residual": i.schur_residual} for i in arr]

    def solve(self, p, check: bool = True):
        infos = self._infos()
        st = self.lib.fpg_solve(self.handle, _ptr(p), infos)
        if check and st != FPG_ENOCONV:
            _check(st, "fpg_solve")
        return st, self._info_list(infos)

    def solve_resume(self, p, check: bool = True):
        """fpg_solve_resume: continue from the iterates already in p (checkpoint / resume)."""
        infos = self._infos()
        st = self.lib.fpg_solve_resume(self.handle, _ptr(p), infos)
        if check and st not in (FPG_OK, FPG_ENOCONV):
            _check(st, "fpg_solve_resume")
        return st, self._info_list(infos)

    def solve_async(self, p):
        _check(self.lib.fpg_solve_async(self.handle, _ptr(p)), "fpg_solve_async")

    def solve_finish(self):
        infos = self._infos()
        st = self.lib.fpg_solve_finish(self.handle, infos)
        if st != FPG_ENOCONV:
            _check(st, "fpg_solve_finish")
        return st, self._info_list(infos)

    def solve_host(self, f_host, p_host):
        infos = self._infos()
        st = self.lib.fpg_solve_host(self.handle, _ptr(f_host), _ptr(p_host), infos)
        if st != FPG_ENOCONV:
            _check(st, "fpg_solve_host")
        return st, self._info_list(infos)

    # -- operators ------------------------------------------------------
    def apply_precond(self, v, z, nvec: int):
        _check(self.lib.fpg_apply_precond(self.handle, _ptr(v), _ptr(z), nvec), "fpg_apply_precond")

    def block_solve(self, block: int, v, z, nvec: int):
        _check(self.lib.fpg_block_solve(self.handle, block, _ptr(v), _ptr(z), nvec), "fpg_block_solve")

    def apply_schur(self, z, zprec: int, w, nvec: int):
        _check(self.lib.fpg_apply_schur(self.handle, _ptr(z), zprec, _ptr(w), nvec), "fpg_apply_schur")

    def arnoldi_mgs(self, V, j: int, w, h, length: int, nvec: int):
        _check(self.lib.fpg_arnoldi_mgs(self.handle, _ptr(V), j, _ptr(w), _ptr(h), length, nvec),
               "fpg_arnoldi_mgs")

    def givens(self, Hcol, cs, sn, g, res, j: int, m: int, nvec: int):
        _check(self.lib.fpg_givens(self.handle, _ptr(Hcol), _ptr(cs), _ptr(sn), _ptr(g), _ptr(res), j, m, nvec),
               "fpg_givens")

    def global_residual(self, f, p, nvec: int):
        out = (ctypes.c_double * nvec)()
        _check(self.lib.fpg_global_residual(self.handle, _ptr(f), _ptr(p), out, nvec), "fpg_global_residual")
        return list(out)

    def apply_global(self, p, y, nvec: int):
        _check(self.lib.fpg_apply_global(self.handle, _ptr(p), _ptr(y), nvec), "fpg_apply_global")

    def autotune(self) -> dict:
        """fpg_autotune: time the launch shapes of the hot kernels, keep the fastest."""
        r = TuneResult()
        _check(self.lib.fpg_autotune(self.handle, ctypes.byref(r)), "fpg_autotune")
        return {"q": r.q, "mt": r.mt, "cluster": r.cluster, "threads": r.threads, "precond_ms": r.precond_ms, "arnoldi_ms": r.arnoldi_ms}

    def set_stream(self, stream):
        """fpg_set_stream: later calls run on this torch stream."""
        self.stream = stream
        _check(self.lib.fpg_set_stream(self.handle, stream.cuda_stream), "fpg_set_stream")

    def set_option(self, option: int, value: int):
        _check(self.lib.fpg_set_option(self.handle, option, value), "fpg_set_option")

    # -- measurement -----------------------------------------------------
    def set_profiling(self, on: bool):
        _check(self.lib.fpg_set_profiling(self.handle, 1 if on else 0), "fpg_set_profiling")

    def phase_stats(self):
        out = {}
        for i, name in enumerate(PHASES):
            ln, ms = _I64(), _D()
            _check(self.lib.fpg_phase_stats(self.handle, i, ctypes.byref(ln), ctypes.byref(ms)), "fpg_phase_stats")
            out[name] = {"launches": int(ln.value), "ms": float(ms.value)}
        return out

    def set_history(self, buf):
        """fpg_set_history: buf a CUDA float64 tensor (nrhs, len), or None to stop."""
        if buf is None:
            _check(self.lib.fpg_set_history(self.handle, None, 0), "fpg_set_history")
        else:
            _check(self.lib.fpg_set_history(self.handle, _ptr(buf), buf.shape[-1]), "fpg_set_history")
        self._hist = buf  # keep the buffer alive while the library writes it

    def fast_solve_path(self) -> int:
        """fpg_fast_solve_path: which kernels the preconditioner runs (see FAST_SOLVE_KERNELS)."""
        out = _I32()
        _check(self.lib.fpg_fast_solve_path(self.handle, ctypes.byref(out)), "fpg_fast_solve_path")
        return int(out.value)

    def arnoldi_shape(self) -> dict:
        """fpg_arnoldi_shape: kernel form (1 register cluster, 2 cluster with w in HBM,
        0 multi-launch MGS), CTAs per right-hand side, threads per CTA, CTAs per launch."""
        k, c, t, n = _I32(), _I32(), _I32(), _I32()
        _check(self.lib.fpg_arnoldi_shape(self.handle, ctypes.byref(k), ctypes.byref(c), ctypes.byref(t),
                                          ctypes.byref(n)), "fpg_arnoldi_shape")
        return {"kind": int(k.value), "cluster": int(c.value), "threads": int(t.value), "ctas": int(n.value)}

    def launch_count(self) -> int:
        out = _I64()
        _check(self.lib.fpg_launch_count(self.handle, ctypes.byref(out)), "fpg_launch_count")
        return int(out.value)


def convert(src, dst, stream=None):
    """fpg_convert: FP64 <-> FP32 with the library's integer-pipe conversion
    (src and dst are CUDA tensors of the same length)."""
    import torch
    lib = load()
    prec = {torch.float64: 64, torch.float32: 32}
    st = stream if stream is not None else torch.cuda.current_stream(src.device)
    _check(lib.fpg_convert(_ptr(src), prec[src.dtype], _ptr(dst), prec[dst.dtype], src.numel(), st.cuda_stream),
           "fpg_convert")


def neumann_solve(v, z, nt: int, ns: int, h: float, kappa: float, stream=None):
    """fpg_neumann_solve on nvec = v.shape[0] Neumann rectangles (CUDA float64
    tensors of shape (nvec, nt * ns)); the workspace is a torch uint8 tensor."""
    import torch
    lib = load()
    nvec = v.shape[0]
    nb = ctypes.c_size_t()
    _check(lib.fpg_neumann_workspace_bytes(nt, ns, nvec, ctypes.byref(nb)), "fpg_neumann_workspace_bytes")
    ws = torch.empty(nb.value, dtype=torch.uint8, device=v.device)
    st = stream if stream is not None else torch.cuda.current_stream(v.device)
    _check(lib.fpg_neumann_solve(nt, ns, h, kappa, _ptr(v), _ptr(z), nvec, _ptr(ws), nb.value, st.cuda_stream),
           "fpg_neumann_solve")
    return ws


def solve_many(domains, ps):
    """fpg_solve_many over Domain objects and their solution tensors; returns
    (status, [infos per domain])."""
    lib = load()
    n = len(domains)
    hs = (_P * n)(*[d.handle for d in domains])
    pp = (_P * n)(*[p.data_ptr() for p in ps])
    arrs = [d._infos() for d in domains]
    ip = (_P * n)(*[ctypes.cast(a, _P) for a in arrs])
    st = lib.fpg_solve_many(hs, n, pp, ip)
    if st not in (FPG_OK, FPG_ENOCONV):
        _check(st, "fpg_solve_many")
    return st, [Domain._info_list(a) for a in arrs]


def probe_fma_peak(precision: int = 64) -> float:
    """FLOP/s of FMA on this GPU, measured by the library's own probe kernel."""
    out = _D()
    _check(load().fpg_probe_fma_peak(precision, ctypes.byref(out)), "fpg_probe_fma_peak")
    return float(out.value)


def periodic_solve(v, z, nt: int, ns: int, h: float, kappa: float, stream=None):
    """fpg_periodic_solve on nvec = v.shape[0] periodic rectangles (CUDA float64
    tensors of shape (nvec, nt * ns)); the workspace is a torch uint8 tensor."""
    import torch
    lib = load()
    nvec = v.shape[0]
    nb = ctypes.c_size_t()
    _check(lib.fpg_periodic_workspace_bytes(nt, ns, nvec, ctypes.byref(nb)), "fpg_periodic_workspace_bytes")
    ws = torch.empty(nb.value, dtype=torch.uint8, device=v.device)
    st = stream if stream is not None else torch.cuda.current_stream(v.device)
    _check(lib.fpg_periodic_solve(nt, ns, h, kappa, _ptr(v), _ptr(z), nvec, _ptr(ws), nb.value, st.cuda_stream),
           "fpg_periodic_solve")
    return ws


class RectPlan:
    """A rectangle fast-solve plan (fpg_rect_plan_*) with its device workspace."""

    def __init__(self, kind, nt: int, ns: int, h: float, kappa: float, nvec: int, stream=None, device="cuda"):
        import torch
        self.lib = load()
        self.kind = RECT[kind] if isinstance(kind, str) else int(kind)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        nb = ctypes.c_size_t()
        _check(self.lib.fpg_rect_plan_bytes(self.kind, nt, ns, nvec, ctypes.byref(nb)), "fpg_rect_plan_bytes")
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=device)
        h_ = _P()
        _check(self.lib.fpg_rect_plan_create(self.kind, nt, ns, h, kappa, nvec, _ptr(self.workspace), nb.value,
                                             self.stream.cuda_stream, ctypes.byref(h_)), "fpg_rect_plan_create")
        self.handle = h_

    def solve(self, v, z, nvec: int):
        _check(self.lib.fpg_rect_solve(self.handle, _ptr(v), _ptr(z), nvec), "fpg_rect_solve")

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fpg_rect_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


class BoxPlan:
    """A 3-D box fast-solve plan (fpg_box_plan_*) with its device workspace."""

    def __init__(self, nx: int, ny: int, nz: int, h: float, kappa: float, nvec: int, stream=None, device="cuda"):
        import torch
        self.lib = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        nb = ctypes.c_size_t()
        _check(self.lib.fpg_box_plan_bytes(nx, ny, nz, nvec, ctypes.byref(nb)), "fpg_box_plan_bytes")
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=device)
        h_ = _P()
        _check(self.lib.fpg_box_plan_create(nx, ny, nz, h, kappa, nvec, _ptr(self.workspace), nb.value,
                                            self.stream.cuda_stream, ctypes.byref(h_)), "fpg_box_plan_create")
        self.handle = h_

    def solve(self, v, z, nvec: int):
        _check(self.lib.fpg_box_solve(self.handle, _ptr(v), _ptr(z), nvec), "fpg_box_solve")

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fpg_box_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


class Batch:
    """The library's batch runtime (fpg_batch_*): continuous batching of requests
    over resident domains carved from one device pool (a torch uint8 tensor)."""

    report_cap = 256  # finished tickets one step() reports; poll() finds any beyond them

    def __init__(self, pool_bytes: int, slots: int = 8, max_domains: int = 64, max_per_key: int = 2, max_busy: int = 0,
                 device="cuda"):
        import torch
        self.lib = load()
        self.slots = slots
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=device)
        d = BatchDescC(slots, max_domains, max_per_key, max_busy)
        h = _P()
        _check(self.lib.fpg_batch_create(ctypes.byref(d), _ptr(self.pool), int(pool_bytes), ctypes.byref(h)),
               "fpg_batch_create")
        self.handle = h

    def admit(self, desc: DomainDesc, f, p) -> int:
        """f, p: CUDA float64 tensors (desc.nrhs, unknowns); f must be final (the
        caller synchronises the stream that produced it); both stay referenced by
        the caller until poll() reports the ticket done."""
        t = _I64()
        _check(self.lib.fpg_batch_admit(self.handle, ctypes.byref(desc), _ptr(f), _ptr(p), ctypes.byref(t)),
               "fpg_batch_admit")
        return int(t.value)

    def step(self) -> list:
        """Advance the runtime; returns the tickets that finished in this step."""
        cap = self.report_cap
        buf = (_I64 * cap)()
        c = _I32()
        _check(self.lib.fpg_batch_step(self.handle, buf, cap, ctypes.byref(c)), "fpg_batch_step")
        return list(buf[:min(cap, c.value)])

    def poll(self, ticket: int, nrhs: int):
        """None while running; else the list of per-RHS info dicts (the ticket is released).
        The library writes one entry per right-hand side of the request, at most
        `slots`, so the array is sized by slots whatever nrhs the caller names."""
        done = _I32()
        arr = (SolveInfo * max(1, self.slots, nrhs))()
        _check(self.lib.fpg_batch_poll(self.handle, ticket, ctypes.byref(done), arr), "fpg_batch_poll")
        if not done.value:
            return None
        return Domain._info_list(arr[:nrhs])

    def stats(self) -> dict:
        s = BatchStats()
        _check(self.lib.fpg_batch_stats(self.handle, ctypes.byref(s)), "fpg_batch_stats")
        return {k: getattr(s, k) for k, _ in BatchStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fpg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()
