"""Python binding of libhom, the GB300 library for FFT-based homogenisation with filtered
material properties (Gélébart & Ouaki, arXiv 1412.3228).

This module only marshals arguments: every step of the computation runs in the CUDA kernels of
libhom.so (built in-tree by `_build_lib.build()`).  PyTorch provides device memory and streams.
The functions carry the C ABI's names (include/hom.h):

    hom_filter_build(cells, phases)          -> Material   (section 2, eqs. 3, 4, 5)
    hom_solve(material, E, c0, ...)          -> dict       (section 2, eqs. 1-a, 1-b, 2)
    hom_effective_stiffness(E, mean_sigma)   -> ndarray    (C_eff from mean stresses)

There is no CPU fallback: if the library or a CUDA device is missing the calls raise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhom.so")

# constants of include/hom.h
HOM_OK = 0
HOM_ERR_NOT_CONVERGED = 3
HOM_ERR_DIVERGED = 4
HOM_ERR_CAPACITY = 8
HOM_ERR_NOT_IMPL = 9
HOM_ERR_BOUNDS = 10
HOM_FP32, HOM_FP64 = 0, 1
HOM_CRIT_E, HOM_CRIT_EN = 0, 1
HOM_PASSES_AUTO, HOM_PASSES_GENERIC = 0, 1
HOM_GREEN_CONTINUOUS, HOM_GREEN_ROTATED = 0, 1
HOM_SCHEME_BASIC, HOM_SCHEME_EYRE_MILTON = 0, 1
HOM_STATUS = {0: "converged", 1: "max_iter", 2: "diverged", 3: "stalled", -1: "active"}
HOM_MIXED_BIT = 0x80000000
HOM_NKERNEL = 8
KERNEL_NAMES = ["filter", "row", "yfwd", "green", "yinv", "control", "output", "init"]

EXPORTED = ["hom_filter_build", "hom_solve", "hom_solve_noalloc", "hom_solve_cg", "hom_solve_backward",
            "hom_effective_stiffness", "hom_fourier_extrapolate", "hom_autotune_report", "hom_last_error", "hom_release",
            "hom_version", "hom_build_flags"]


class HomError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libhom error %d: %s" % (code, msg))
        self.code = code


class hom_primitive(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("phase", ctypes.c_int32), ("axis", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("centre", ctypes.c_double * 3), ("radius", ctypes.c_double)]


class hom_cell(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int32), ("matrix_phase", ctypes.c_int32),
                ("rule", ctypes.c_int32), ("radius_px", ctypes.c_double), ("subgrid", ctypes.c_int32),
                ("nprim", ctypes.c_int32), ("prims", ctypes.POINTER(hom_primitive))]


class hom_phase(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("mu", ctypes.c_double)]


class hom_material(ctypes.Structure):
    _fields_ = [("label", ctypes.c_void_p), ("mixed_c64", ctypes.c_void_p), ("mixed_c32", ctypes.c_void_p),
                ("mixed_phases", ctypes.c_void_p), ("mixed_frac", ctypes.c_void_p),
                ("mixed_normal", ctypes.c_void_p), ("mixed_voxel", ctypes.c_void_p),
                ("mixed_capacity", ctypes.c_int64), ("phase_c64", ctypes.c_void_p),
                ("phase_c32", ctypes.c_void_p), ("nphase", ctypes.c_int32), ("dim", ctypes.c_int32),
                ("mixed_count", ctypes.c_int64)]


class hom_solve_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("criterion", ctypes.c_int32), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("diverge_window", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("max_radix", ctypes.c_int32), ("green", ctypes.c_int32), ("tune", ctypes.c_int32),
                ("stall_window", ctypes.c_int32), ("refine", ctypes.c_int32), ("refine_inner", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("warm_start", ctypes.c_int32)]


class hom_kernel_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * HOM_NKERNEL), ("ms", ctypes.c_double * HOM_NKERNEL),
                ("bytes", ctypes.c_double * HOM_NKERNEL), ("voxel_iterations", ctypes.c_double)]


class hom_result(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("mean_sigma", ctypes.c_void_p),
                ("iterations", ctypes.c_void_p), ("status", ctypes.c_void_p), ("err", ctypes.c_void_p),
                ("err_n", ctypes.c_void_p), ("stats", ctypes.POINTER(hom_kernel_stats)), ("err_c", ctypes.c_void_p),
                ("history", ctypes.c_void_p)]


_lib_handle = None


def lib() -> ctypes.CDLL:
    """The loaded libhom.so (raises if it was not built)."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhom.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        h = ctypes.CDLL(LIB_PATH)
        h.hom_filter_build.argtypes = [ctypes.POINTER(hom_cell), ctypes.c_int32, ctypes.POINTER(hom_phase),
                                       ctypes.c_int32, ctypes.POINTER(hom_material), ctypes.c_void_p]
        h.hom_solve.argtypes = [ctypes.POINTER(hom_cell), ctypes.c_int32, ctypes.POINTER(hom_material),
                                ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(hom_solve_opts), ctypes.POINTER(hom_result), ctypes.c_void_p]
        h.hom_solve_noalloc.argtypes = h.hom_solve.argtypes
        h.hom_solve_cg.argtypes = [ctypes.POINTER(hom_cell), ctypes.c_int32, ctypes.POINTER(hom_material),
                                   ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.POINTER(hom_solve_opts),
                                   ctypes.POINTER(hom_result), ctypes.c_void_p]
        h.hom_solve_backward.argtypes = [ctypes.POINTER(hom_cell), ctypes.c_int32, ctypes.POINTER(hom_material),
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                         ctypes.POINTER(hom_solve_opts), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.POINTER(hom_result), ctypes.c_void_p]
        h.hom_effective_stiffness.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                              ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
        h.hom_fourier_extrapolate.argtypes = [ctypes.POINTER(hom_cell), ctypes.c_int32, ctypes.POINTER(hom_material),
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.c_void_p]
        h.hom_autotune_report.argtypes = [ctypes.c_char_p, ctypes.c_int32]
        h.hom_autotune_report.restype = ctypes.c_int32
        h.hom_last_error.restype = ctypes.c_char_p
        h.hom_version.restype = ctypes.c_int32
        h.hom_build_flags.restype = ctypes.c_int32
        _lib_handle = h
    return _lib_handle


def use_debug_library() -> str:
    """Load the bounds-checked build of the library (-DHOM_DEBUG, built on first use) instead of the
    release one.  Call before the first call into the library; returns its path."""
    global LIB_PATH
    if _lib_handle is not None:
        raise RuntimeError("libhom.so is already loaded in this process")
    from . import _build_lib
    LIB_PATH = _build_lib.build(debug=True)
    return LIB_PATH


def _check(code: int, allow=(HOM_OK,)) -> int:
    if code not in allow:
        raise HomError(code, lib().hom_last_error().decode())
    return code


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def ns_of(dim: int) -> int:
    return 6 if dim == 2 else 21


def nc_of(dim: int) -> int:
    return 3 if dim == 2 else 6


# ---------------------------------------------------------------------------------------------
# marshalling of the seeded inputs (hom_inputs.Cell / Primitive or any object with the same
# attributes)

@dataclasses.dataclass
class _CellArray:
    cells: ctypes.Array
    keep: list
    dims: List[int]
    ns: List[int]


def _marshal_cells(cells) -> _CellArray:
    arr = (hom_cell * len(cells))()
    keep = []
    for i, c in enumerate(cells):
        prims = (hom_primitive * max(1, len(c.prims)))()
        for j, p in enumerate(c.prims):
            prims[j].kind = p.kind
            prims[j].phase = p.phase
            prims[j].axis = getattr(p, "axis", 0)
            prims[j].reserved = 0
            for d in range(3):
                prims[j].centre[d] = float(p.centre[d])
            prims[j].radius = float(p.radius)
        keep.append(prims)
        arr[i].dim = c.dim
        arr[i].n = c.n
        arr[i].matrix_phase = c.matrix_phase
        arr[i].rule = c.rule
        arr[i].radius_px = float(c.radius_px)
        arr[i].subgrid = int(c.subgrid)
        arr[i].nprim = len(c.prims)
        arr[i].prims = ctypes.cast(prims, ctypes.POINTER(hom_primitive))
    return _CellArray(arr, keep, [c.dim for c in cells], [c.n for c in cells])


@dataclasses.dataclass
class Material:
    """Filtered stiffness of a batch of cells (device tensors owned by this object)."""
    cells: list
    dim: int
    label: torch.Tensor          # int32 view of the uint32 labels, [sum n^dim]
    mixed_c64: torch.Tensor
    mixed_c32: torch.Tensor
    mixed_phases: torch.Tensor
    mixed_frac: torch.Tensor
    mixed_normal: torch.Tensor
    mixed_voxel: torch.Tensor
    phase_c64: torch.Tensor
    phase_c32: torch.Tensor
    mixed_count: int
    struct: hom_material
    marshalled: _CellArray

    def voxel_offsets(self) -> List[int]:
        off, out = 0, []
        for c in self.cells:
            out.append(off)
            off += c.n ** c.dim
        return out


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def hom_filter_build(cells: Sequence, phases: Sequence[Tuple[float, float]], device=None, stream=None,
                     capacity: Optional[int] = None) -> Material:
    """Filtered stiffness of every voxel (section 2, eqs. 3-5); see include/hom.h."""
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    cells = list(cells)
    dim = cells[0].dim
    nvox = sum(c.n ** c.dim for c in cells)
    ns = ns_of(dim)
    nphase = len(phases)
    ph = (hom_phase * nphase)()
    for i, (lam, mu) in enumerate(phases):
        ph[i].lambda_ = float(lam)
        ph[i].mu = float(mu)
    mc = _marshal_cells(cells)
    label = torch.empty(nvox, dtype=torch.int32, device=device)
    phase_c64 = torch.empty(nphase * ns, dtype=torch.float64, device=device)
    phase_c32 = torch.empty(nphase * ns, dtype=torch.float32, device=device)
    cap = capacity if capacity is not None else max(1024, nvox // 16)
    for _attempt in range(2):
        mixed = dict(
            mixed_c64=torch.empty(cap * ns, dtype=torch.float64, device=device),
            mixed_c32=torch.empty(cap * ns, dtype=torch.float32, device=device),
            mixed_phases=torch.empty(cap * 2, dtype=torch.int32, device=device),
            mixed_frac=torch.empty(cap, dtype=torch.float64, device=device),
            mixed_normal=torch.empty(cap * 3, dtype=torch.float64, device=device),
            mixed_voxel=torch.empty(cap, dtype=torch.int64, device=device))
        st = hom_material(label=_ptr(label), mixed_c64=_ptr(mixed["mixed_c64"]), mixed_c32=_ptr(mixed["mixed_c32"]),
                          mixed_phases=_ptr(mixed["mixed_phases"]), mixed_frac=_ptr(mixed["mixed_frac"]),
                          mixed_normal=_ptr(mixed["mixed_normal"]), mixed_voxel=_ptr(mixed["mixed_voxel"]),
                          mixed_capacity=cap, phase_c64=_ptr(phase_c64), phase_c32=_ptr(phase_c32),
                          nphase=nphase, dim=dim, mixed_count=0)
        with torch.cuda.device(device):
            code = lib().hom_filter_build(mc.cells, len(cells), ph, nphase, ctypes.byref(st), _stream_handle(stream))
        if code == HOM_ERR_CAPACITY:
            cap = int(st.mixed_count)
            continue
        _check(code)
        return Material(cells, dim, label, phase_c64=phase_c64, phase_c32=phase_c32,
                        mixed_count=int(st.mixed_count), struct=st, marshalled=mc, **mixed)
    raise HomError(HOM_ERR_CAPACITY, "mixed table did not fit after resizing")


def hom_solve_noalloc(material: Material, E, c0, **kw) -> dict:
    """hom_solve through the no-allocation entry point (fixed 64 MiB device scratch inside the
    library; no graphs, no kernel statistics).  The output tensors are still allocated here, by
    the caller side."""
    return hom_solve(material, E, c0, _entry="hom_solve_noalloc", **kw)


def hom_solve(material: Material, E, c0, *, L: Optional[int] = None, precision: int = HOM_FP64,
              criterion: int = HOM_CRIT_E, tol: float = 1e-8, max_iter: int = 1000, fields: bool = True,
              host_fields: bool = False, check_every: int = 0, diverge_window: int = 0, use_graph: bool = False,
              passes: int = HOM_PASSES_AUTO, max_radix: int = 0, green: int = HOM_GREEN_CONTINUOUS,
              tune: bool = False, stall_window: int = 0, refine: int = 0, refine_inner: int = 0,
              scheme: int = HOM_SCHEME_BASIC, eps0: Optional[torch.Tensor] = None, history: bool = False,
              stats: bool = False, stream=None,
              allow_not_converged: bool = True, _entry: str = "hom_solve") -> dict:
    """Basic fixed-point scheme for every cell x load case (section 2, eqs. 1-a, 1-b, 2), or the
    Eyre-Milton scheme with scheme=HOM_SCHEME_EYRE_MILTON.

    E: [ncells, L, nc] (or [L, nc], shared by every cell) Mandel macroscopic strains.
    c0: [ncells, 2] (or [2]) Lamé constants of the reference medium.
    Returns a dict with eps / sigma fields ([sum over cells of L*nc*n^dim], flat, cell-major),
    mean_sigma [ncells, L, nc], iterations / status / err / err_n / err_c [ncells, L] and the
    kernel statistics when stats=True.
    eps0: warm start, a device tensor laid out like the returned eps (field precision); the solve
    reads it through the returned eps buffer, which starts as a copy of it.
    history=True adds "history" [ncells, L, max_iter + 1]: the stopping quantity of every
    iterate (NaN where not written)."""
    cells = material.cells
    ncells = len(cells)
    dim = material.dim
    nc = nc_of(dim)
    E = np.asarray(E, dtype=np.float64)
    if E.ndim == 2:
        E = np.broadcast_to(E, (ncells,) + E.shape)
    L = E.shape[1]
    E = np.ascontiguousarray(E)
    c0 = np.ascontiguousarray(np.broadcast_to(np.asarray(c0, dtype=np.float64), (ncells, 2)))
    device = material.label.device
    ftype = torch.float32 if precision == HOM_FP32 else torch.float64
    nfield = sum(L * nc * c.n ** c.dim for c in cells)
    eps = sig = None
    if eps0 is not None:
        fields = True
        host_fields = False
    if fields:
        if host_fields:
            eps = torch.empty(nfield, dtype=ftype, pin_memory=True)
            sig = torch.empty(nfield, dtype=ftype, pin_memory=True)
        else:
            eps = torch.empty(nfield, dtype=ftype, device=device)
            sig = torch.empty(nfield, dtype=ftype, device=device)
            if eps0 is not None:
                if eps0.numel() != nfield or eps0.dtype != ftype:
                    raise ValueError("eps0 must hold %d values of %s" % (nfield, ftype))
                eps.copy_(eps0.reshape(-1))
    mean_sigma = np.zeros((ncells, L, nc))
    iters = np.zeros((ncells, L), dtype=np.int32)
    status = np.zeros((ncells, L), dtype=np.int32)
    err = np.zeros((ncells, L))
    err_n = np.zeros((ncells, L))
    err_c = np.zeros((ncells, L))
    hist = np.full((ncells, L, int(max_iter) + 1), np.nan) if history else None
    st = hom_kernel_stats() if stats else None
    res = hom_result(eps=_ptr(eps), sigma=_ptr(sig), mean_sigma=mean_sigma.ctypes.data,
                     iterations=iters.ctypes.data, status=status.ctypes.data, err=err.ctypes.data,
                     err_n=err_n.ctypes.data, stats=ctypes.pointer(st) if st is not None else None,
                     err_c=err_c.ctypes.data, history=hist.ctypes.data if hist is not None else None)
    opts = hom_solve_opts(precision=precision, criterion=criterion, tol=float(tol), max_iter=int(max_iter),
                          check_every=int(check_every), diverge_window=int(diverge_window),
                          use_graph=int(bool(use_graph)), passes=int(passes), max_radix=int(max_radix),
                          green=int(green), tune=int(bool(tune)), stall_window=int(stall_window),
                          refine=int(refine), refine_inner=int(refine_inner), scheme=int(scheme),
                          warm_start=int(eps0 is not None))
    with torch.cuda.device(device):
        if _entry == "hom_solve_cg":
            code = lib().hom_solve_cg(material.marshalled.cells, ncells, ctypes.byref(material.struct),
                                      E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), L, ctypes.byref(opts),
                                      ctypes.byref(res), _stream_handle(stream))
        else:
            code = getattr(lib(), _entry)(material.marshalled.cells, ncells, ctypes.byref(material.struct),
                                          E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), L,
                                          c0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(opts),
                                          ctypes.byref(res), _stream_handle(stream))
    allowed = (HOM_OK, HOM_ERR_NOT_CONVERGED, HOM_ERR_DIVERGED) if allow_not_converged else (HOM_OK,)
    _check(code, allowed)
    out = dict(eps=eps, sigma=sig, mean_sigma=mean_sigma, iterations=iters, status=status, err=err,
               err_n=err_n, err_c=err_c, code=code, E=E, L=L)
    if hist is not None:
        out["history"] = hist
    if st is not None:
        out["stats"] = {KERNEL_NAMES[k]: dict(launches=int(st.launches[k]), ms=float(st.ms[k]),
                                              bytes=float(st.bytes[k])) for k in range(HOM_NKERNEL)}
        out["voxel_iterations"] = float(st.voxel_iterations)
    return out


def hom_solve_cg(material: Material, E, **kw) -> dict:
    """Conjugate-gradient solve of the same discrete problem (reference medium c0 = identity, the
    projection G); see include/hom.h.  Keyword arguments as hom_solve (criterion and diverge_window
    are ignored; err and err_n both hold e_G, which lies between e_n and sqrt(2) e_n)."""
    return hom_solve(material, E, [0.0, 0.5], _entry="hom_solve_cg", **kw)


def hom_solve_backward(material: Material, forward: dict, c0, *, dL_dC=None, dL_dsigma: Optional[torch.Tensor] = None,
                       want_ctilde: bool = True, want_frac: bool = True, precision: int = HOM_FP64,
                       criterion: int = HOM_CRIT_E, tol: float = 1e-10, max_iter: int = 2000,
                       passes: int = HOM_PASSES_AUTO, green: int = HOM_GREEN_CONTINUOUS, stream=None) -> dict:
    """Adjoint derivative of L(C_eff, sigma) (see include/hom.h).  `forward` is the dict returned by
    hom_solve (with device fields); dL_dC is [ncells, nc, nc] (host), dL_dsigma a device tensor laid
    out like forward['sigma'].  Returns dctilde [sum voxels, ns] (device), dphase [nphase, 2],
    dfrac [mixed_count] (device) and the adjoint solve's iterations / status."""
    cells = material.cells
    ncells = len(cells)
    dim = material.dim
    nc = nc_of(dim)
    L = forward["L"]
    c0 = np.ascontiguousarray(np.broadcast_to(np.asarray(c0, dtype=np.float64), (ncells, 2)))
    device = material.label.device
    ftype = torch.float32 if precision == HOM_FP32 else torch.float64
    eps = forward["eps"]
    if eps is None or not eps.is_cuda or eps.dtype != ftype:
        raise ValueError("forward eps fields must be device tensors of the solve precision")
    nvox = sum(c.n ** c.dim for c in cells)
    dct = torch.empty(nvox * ns_of(dim), dtype=ftype, device=device) if want_ctilde else None
    dfr = torch.zeros(max(1, material.mixed_count), dtype=torch.float64, device=device) if want_frac else None
    dph = np.zeros((material.struct.nphase, 2))
    G = None
    if dL_dC is not None:
        G = np.ascontiguousarray(np.asarray(dL_dC, dtype=np.float64).reshape(ncells, nc, nc))
    if dL_dsigma is not None and (not dL_dsigma.is_cuda or dL_dsigma.dtype != ftype):
        raise ValueError("dL_dsigma must be a device tensor of the solve precision")
    iters = np.zeros((ncells, L), dtype=np.int32)
    status = np.zeros((ncells, L), dtype=np.int32)
    err = np.zeros((ncells, L))
    err_n = np.zeros((ncells, L))
    info = hom_result(iterations=iters.ctypes.data, status=status.ctypes.data, err=err.ctypes.data,
                      err_n=err_n.ctypes.data)
    opts = hom_solve_opts(precision=precision, criterion=criterion, tol=float(tol), max_iter=int(max_iter),
                          check_every=0, diverge_window=0, use_graph=0, passes=int(passes), max_radix=0,
                          green=int(green), tune=0, stall_window=0, refine=0, refine_inner=0)
    with torch.cuda.device(device):
        code = lib().hom_solve_backward(material.marshalled.cells, ncells, ctypes.byref(material.struct),
                                        c0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), L, ctypes.byref(opts),
                                        ctypes.c_void_p(eps.data_ptr()),
                                        None if G is None else ctypes.c_void_p(G.ctypes.data),
                                        None if dL_dsigma is None else ctypes.c_void_p(dL_dsigma.data_ptr()),
                                        None if dct is None else ctypes.c_void_p(dct.data_ptr()),
                                        ctypes.c_void_p(dph.ctypes.data),
                                        None if dfr is None else ctypes.c_void_p(dfr.data_ptr()),
                                        ctypes.byref(info), _stream_handle(stream))
    _check(code, (HOM_OK, HOM_ERR_NOT_CONVERGED))
    return dict(dctilde=dct, dphase=dph, dfrac=None if dfr is None else dfr[:material.mixed_count],
                adjoint_iterations=iters, adjoint_status=status, adjoint_err=err, adjoint_err_n=err_n, code=code)


class HomSolve(torch.autograd.Function):
    """C_eff (and the local stress fields) of a batch of cells as a differentiable function of the
    phase Lame constants.  Forward: hom_filter_build + hom_solve with the nc unit Mandel loads +
    hom_effective_stiffness.  Backward: hom_solve_backward (adjoint solve, no iterate history).

        C, sigma = HomSolve.apply(phase_lame, cells, c0, settings)
    phase_lame: float64 tensor [nphase, 2] (lambda, mu); c0: [ncells, 2] reference media (held fixed:
    the converged discrete solution does not depend on c0); settings: dict of hom_solve keywords.
    Returns C [ncells, nc, nc] (float64, CPU) and sigma (device, layout of hom_solve's fields)."""

    @staticmethod
    def forward(ctx, phase_lame, cells, c0, settings):
        ctx.set_materialize_grads(False)
        phases = [tuple(map(float, row)) for row in phase_lame.detach().cpu().tolist()]
        mat = hom_filter_build(cells, phases)
        dim = mat.dim
        E = np.eye(nc_of(dim))
        res = hom_solve(mat, E, c0, fields=True, **settings)
        C = hom_effective_stiffness(E, res["mean_sigma"], dim)
        ctx.mat, ctx.res, ctx.c0, ctx.settings = mat, res, c0, settings
        return torch.from_numpy(C), res["sigma"]

    @staticmethod
    def backward(ctx, gC, gsigma):
        st = ctx.settings
        g = hom_solve_backward(ctx.mat, ctx.res, ctx.c0,
                               dL_dC=None if gC is None else gC.detach().cpu().numpy(),
                               dL_dsigma=None if gsigma is None else gsigma.detach().contiguous(),
                               want_ctilde=False, want_frac=False, precision=st.get("precision", HOM_FP64),
                               criterion=st.get("criterion", HOM_CRIT_E), tol=st.get("tol", 1e-10),
                               max_iter=st.get("max_iter", 2000))
        return torch.from_numpy(g["dphase"]), None, None, None


def hom_autotune_report() -> str:
    """The autotuner's record: one line per batch shape, with the candidate timings and the choice."""
    n = lib().hom_autotune_report(None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    lib().hom_autotune_report(buf, n + 1)
    return buf.value.decode()


def hom_effective_stiffness(E, mean_sigma, dim: int) -> np.ndarray:
    """C_eff [ncells, nc, nc] from nc linearly independent load cases per cell."""
    nc = nc_of(dim)
    S = np.ascontiguousarray(np.asarray(mean_sigma, dtype=np.float64).reshape(-1, nc, nc))
    ncells = S.shape[0]
    E = np.asarray(E, dtype=np.float64)
    if E.ndim == 2:
        E = np.broadcast_to(E, (ncells, nc, nc))
    E = np.ascontiguousarray(E)
    C = np.zeros((ncells, nc, nc))
    _check(lib().hom_effective_stiffness(ncells, dim, E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         ctypes.c_void_p(S.ctypes.data),
                                         C.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return C


def packed_index(i: int, j: int, dim: int) -> int:
    """Position of stiffness entry (i, j) (Mandel indices) in the packed upper triangle."""
    nc = nc_of(dim)
    i, j = min(i, j), max(i, j)
    return i * nc - i * (i - 1) // 2 + (j - i)


def hom_fourier_extrapolate(material: Material, cell: int, m: int, comp: int = 0, out: Optional[torch.Tensor] = None,
                            stream=None) -> torch.Tensor:
    """Truncated Fourier series of packed component `comp` of c~ for one cell of the material,
    evaluated at the voxel centres of an m^dim grid (section 6, Fig. 4); see include/hom.h.
    Returns a float64 tensor [(m,) m, m] on the material's device (or fills `out`, host or device)."""
    dim = material.dim
    if out is None:
        out = torch.empty((m,) * dim, dtype=torch.float64, device=material.label.device)
    if out.dtype != torch.float64 or not out.is_contiguous() or out.numel() != m ** dim:
        raise ValueError("out must be a contiguous float64 tensor of m^dim elements")
    with torch.cuda.device(material.label.device):
        _check(lib().hom_fourier_extrapolate(material.marshalled.cells, len(material.cells),
                                             ctypes.byref(material.struct), int(cell), int(comp), int(m),
                                             out.data_ptr(), _stream_handle(stream)))
    return out


def field_views(result: dict, cells, dim: int) -> List[torch.Tensor]:
    """Split a flat field (result['eps'] or result['sigma']) per cell into [L, nc, (n,) n, n]."""
    nc = nc_of(dim)
    L = result["L"]
    views, off = {}, 0
    out = {"eps": [], "sigma": []}
    for key in ("eps", "sigma"):
        f = result[key]
        off = 0
        for c in cells:
            size = L * nc * c.n ** c.dim
            out[key].append(None if f is None else f[off:off + size].view((L, nc) + (c.n,) * c.dim))
            off += size
    return out
