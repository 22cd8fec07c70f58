"""Python binding of libdmp (include/dmp.h).

Argument marshalling only: tensors are passed to the C ABI as raw device
pointers, workspaces are allocated as torch byte tensors, and every step of the
computation runs in libdmp's CUDA kernels. There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.
"""

from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdmp.so")

MODES = {"fp64": 0, "int8": 1, "bf16": 2, "e4m3": 3}
METHODS = {"pm": 0, "trs4": 1, "sp2": 2}
EXECUTORS = {"auto": 0, "imma": 1, "tc": 2}
BETA = {"int8": 7, "bf16": 8, "e4m3": 5}

OK, NOT_CONVERGED, STALLED, C_OUT_OF_RANGE = 0, 1, 2, 3
ERR_INVALID_ARG, ERR_NONFINITE, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_WORKSPACE = -1, -2, -3, -4, -5, -6


class DmpError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {status_str(code)} ({code})")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("slices", ctypes.c_int32), ("executor", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("checkpoint_every", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("tol", ctypes.c_double), ("energy_tol", ctypes.c_double),
                ("refine_slices", ctypes.c_int32), ("method", ctypes.c_int32),
                ("late_slices", ctypes.c_int32), ("late_idem", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("slices_used", ctypes.c_int32),
                ("executor_used", ctypes.c_int32), ("energy", ctypes.c_double),
                ("band_energy", ctypes.c_double), ("idem", ctypes.c_double), ("trace", ctypes.c_double),
                ("c_last", ctypes.c_double), ("h_min", ctypes.c_double), ("h_max", ctypes.c_double),
                ("energy_unrefined", ctypes.c_double), ("refined", ctypes.c_int32), ("late_iters", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class FoeParams(ctypes.Structure):
    _fields_ = [("kT", ctypes.c_double), ("mu", ctypes.c_double), ("n_occ", ctypes.c_int64),
                ("n_terms", ctypes.c_int32), ("scheme", ctypes.c_int32), ("e_min", ctypes.c_double),
                ("e_max", ctypes.c_double)]


class FoeInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_terms", ctypes.c_int32), ("products", ctypes.c_int32),
                ("slices_used", ctypes.c_int32), ("mu", ctypes.c_double), ("trace", ctypes.c_double),
                ("energy", ctypes.c_double), ("band_energy", ctypes.c_double), ("e_min", ctypes.c_double),
                ("e_max", ctypes.c_double), ("tail", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


FOE_MAX_TERMS = 16384
FOE_SCHEMES = {"recurrence": 0, "ps": 1}

_lib = None

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_szp = ctypes.POINTER(ctypes.c_size_t)

# exported symbol -> (restype, argtypes); the test suite checks this list against include/dmp.h
SIGNATURES = {
    "dmp_workspace_size": (ctypes.c_int, [_i64, ctypes.POINTER(Opts), _szp]),
    "dmp_tape_size": (ctypes.c_int, [_i64, ctypes.POINTER(Opts), _szp]),
    "dm_purify": (ctypes.c_int, [_vp, _i64, _i64, _i64, ctypes.POINTER(Opts), _vp, _i64,
                                 ctypes.POINTER(Info), _vp, _sz, _vp, _sz, _vp]),
    "dmp_host_workspace_size": (ctypes.c_int, [_i64, ctypes.POINTER(Opts), _szp]),
    "dm_purify_host": (ctypes.c_int, [_vp, _i64, _i64, _i64, ctypes.POINTER(Opts), _vp, _i64,
                                      ctypes.POINTER(Info), _vp, _sz, _vp]),
    "ozaki_gemm_workspace_size": (ctypes.c_int, [_i64, _i64, _i64, _i32, _i32, _i32, _szp]),
    "ozaki_gemm": (ctypes.c_int, [_i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _i32, _i32, _i32,
                                  _vp, _sz, _vp]),
    "ozaki_gemm_noalloc": (ctypes.c_int, [_i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _i32, _i32, _i32,
                                          _vp]),
    "ozaki_level_sums": (ctypes.c_int, [_i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i32, _i32, _i32,
                                        _vp, _sz, _vp]),
    "ozaki_split": (ctypes.c_int, [_i64, _i64, _vp, _i64, _i32, _i32, _i32, _vp, _vp, _vp, _sz, _vp]),
    "dmp_batched_workspace_size": (ctypes.c_int, [_i32, ctypes.POINTER(_i64), ctypes.POINTER(Opts), _szp]),
    "dm_purify_batched": (ctypes.c_int, [_i32, ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                         ctypes.POINTER(_vp), ctypes.POINTER(Opts), ctypes.POINTER(Info), _vp,
                                         _sz, _vp]),
    "dmp_backward_workspace_size": (ctypes.c_int, [_i64, ctypes.POINTER(Opts), _szp]),
    "dm_purify_backward": (ctypes.c_int, [_vp, _i64, _i64, ctypes.POINTER(Opts), _vp, _sz, _vp, _vp, _vp,
                                          _sz, _vp]),
    "dm_foe_workspace_size": (ctypes.c_int, [_i64, ctypes.POINTER(FoeParams), ctypes.POINTER(Opts), _szp]),
    "dm_foe": (ctypes.c_int, [_vp, _i64, _i64, ctypes.POINTER(FoeParams), ctypes.POINTER(Opts), _vp, _i64,
                              ctypes.POINTER(FoeInfo), _vp, _sz, _vp]),
    "dmp_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "dmp_profile_reset": (ctypes.c_int, []),
    "dmp_profile_read": (ctypes.c_int, [_i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "dmp_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "dmp_launch_count": (ctypes.c_longlong, []),
    "dmp_version": (ctypes.c_char_p, []),
    "dmp_set_tc_pairing": (ctypes.c_int, [ctypes.c_int]),
    "dmp_test_stall_next_product": (ctypes.c_int, [_i32]),
    "dmp_set_tc_split_tiles": (ctypes.c_int, [ctypes.c_int]),
    "dmp_set_batched_tile": (ctypes.c_int, [ctypes.c_int]),
}


def lib() -> ctypes.CDLL:
    """Load libdmp.so (built by paper_2407_13299_gb300.build) once."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libdmp.so not built ({LIB_PATH}); run paper_2407_13299_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_str(code: int) -> str:
    try:
        return lib().dmp_status_str(int(code)).decode()
    except ImportError:
        return str(code)


def launch_count() -> int:
    """Kernels launched by libdmp in this process so far."""
    return int(lib().dmp_launch_count())


def set_tc_pairing(enable: bool) -> bool:
    """Run tcgen05 beta = 7 products on CTA pairs (2-SM MMA, the default) or on
    single CTAs (dmp_set_tc_pairing). Returns the previous setting."""
    return bool(lib().dmp_set_tc_pairing(1 if enable else 0))


def set_tc_split_tiles(enable: bool) -> bool:
    """Split the last partial wave of tcgen05 product tiles into chunk units
    shared by every CTA (dmp_set_tc_split_tiles; on by default). Returns the
    previous setting."""
    return bool(lib().dmp_set_tc_split_tiles(1 if enable else 0))


def set_batched_tile(tile: int) -> int:
    """Force the tile shape of dm_purify_batched's grouped product (128, 256:
    single-CTA tiles of 128 x tile; 512: CTA pairs on 256 x 256 tiles) or let
    the autotuner pick it (0, the default). Returns the previous setting
    (dmp_set_batched_tile)."""
    return _check(int(lib().dmp_set_batched_tile(int(tile))), "dmp_set_batched_tile", allow_status=True)


def test_stall_next_product(wait_limit_us: int) -> None:
    """Test hook (dmp_test_stall_next_product): the next tcgen05 product launch
    withholds its first operand stage and bounds its waits by wait_limit_us, so
    its call returns DMP_ERR_TIMEOUT through the kernel's abort path."""
    _check(lib().dmp_test_stall_next_product(int(wait_limit_us)), "dmp_test_stall_next_product")


PROF_PRODUCT, PROF_SPLIT, PROF_MEASURE, PROF_INIT, PROF_OTHER = 0, 1, 2, 3, 4


def profile_enable(on: bool = True) -> None:
    """Bracket every libdmp launch with CUDA events on its stream (dmp_profile_*)."""
    lib().dmp_profile_enable(1 if on else 0)


def profile_reset() -> None:
    lib().dmp_profile_reset()


def profile_read(kind: int):
    """(total device ms, launches) of one kernel class since the last reset."""
    ms = ctypes.c_double(0.0)
    cnt = ctypes.c_longlong(0)
    _check(lib().dmp_profile_read(int(kind), ctypes.byref(ms), ctypes.byref(cnt)), "dmp_profile_read")
    return ms.value, cnt.value


def _check(code: int, where: str, allow_status: bool = False) -> int:
    if code < 0 or (code > 0 and not allow_status):
        raise DmpError(code, where)
    return code


def _stream_ptr(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
            raise TypeError("expected a float64 CUDA tensor")


FLAG_BOUNDS_CONSTANT, FLAG_FP32_STORAGE, FLAG_BATCHED_STREAM = 1, 2, 4


def make_opts(mode="int8", slices=7, executor="auto", tol=1e-10, energy_tol=0.0, max_iter=100,
              checkpoint_every=8, refine=0, method="pm", fp32_storage=False, late_slices=0,
              late_idem=0.0) -> Opts:
    """refine: 0 none, -1 a McWeeny refinement step with FP64 products, s_r > 0
    one with Ozaki products of s_r slices (see dm_purify). method: "pm"
    (canonical purification), "trs4" or "sp2" (DMP_METHOD_*). fp32_storage:
    every stored matrix rounded to an FP32 value (DMP_FLAG_FP32_STORAGE).
    late_slices, late_idem: the late-slice schedule (passes after an iterate
    with ||P^2 - P||_F < late_idem use late_slices slices; 0: off)."""
    return Opts(MODES[mode], int(slices) if mode != "fp64" else 0, EXECUTORS[executor], int(max_iter),
                int(checkpoint_every), FLAG_FP32_STORAGE if fp32_storage else 0, float(tol), float(energy_tol),
                int(refine), METHODS[method], int(late_slices), float(late_idem))


def workspace(nbytes: int, device=None) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def purify_workspace_bytes(n: int, opts: Opts) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().dmp_workspace_size(n, ctypes.byref(opts), ctypes.byref(b)), "dmp_workspace_size")
    return b.value


def tape_bytes(n: int, opts: Opts) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().dmp_tape_size(n, ctypes.byref(opts), ctypes.byref(b)), "dmp_tape_size")
    return b.value


def purify(H: torch.Tensor, n_occ: int, mode="int8", slices=7, executor="auto", tol=1e-10,
           energy_tol=0.0, max_iter=100, P=None, ws=None, tape=None, stream=None, checkpoint_every=8, refine=0,
           method="pm", fp32_storage=False, late_slices=0, late_idem=0.0):
    """dm_purify on a float64 CUDA tensor H. Returns (P, info dict).

    `ws`, `P` and `tape` may be passed preallocated (see purify_workspace_bytes,
    tape_bytes) so that repeated calls allocate nothing. `refine` adds the
    McWeeny refinement step, `method` picks canonical purification, TRS4 or
    SP2, `fp32_storage` rounds every stored matrix to an FP32 value,
    `late_slices` / `late_idem` set the late-slice schedule (make_opts).
    """
    _require_cuda(H)
    n = H.shape[0]
    opts = make_opts(mode, slices, executor, tol, energy_tol, max_iter, checkpoint_every, refine, method,
                     fp32_storage, late_slices, late_idem)
    if P is None:
        P = torch.empty_like(H)
    if ws is None:
        ws = workspace(purify_workspace_bytes(n, opts), H.device)
    info = Info()
    tp = tape.data_ptr() if tape is not None else None
    tb = tape.numel() if tape is not None else 0
    code = lib().dm_purify(H.data_ptr(), n, H.stride(0), int(n_occ), ctypes.byref(opts), P.data_ptr(),
                           P.stride(0), ctypes.byref(info), ws.data_ptr(), ws.numel(), tp, tb,
                           _stream_ptr(stream))
    _check(code, "dm_purify", allow_status=True)
    return P, info.as_dict()


def host_workspace_bytes(n: int, opts: Opts) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().dmp_host_workspace_size(n, ctypes.byref(opts), ctypes.byref(b)), "dmp_host_workspace_size")
    return b.value


def purify_host(H_host: torch.Tensor, n_occ: int, out: torch.Tensor | None = None, ws=None, stream=None,
                mode="int8", slices=7, executor="auto", tol=1e-10, energy_tol=0.0, max_iter=100, refine=0,
                method="pm", fp32_storage=False, late_slices=0, late_idem=0.0):
    """dm_purify_host: H and P in host memory, both copies made by the library
    on its stream (one cudaMemcpy2DAsync each way). `H_host` is a float64 CPU
    tensor (pinned memory keeps the copies at full link speed); `out`, a host
    tensor of the same shape, receives P (allocated, pinned like H_host, when
    not given). `ws` is a device workspace of host_workspace_bytes bytes.
    Returns (P on the host, info dict)."""
    if not (isinstance(H_host, torch.Tensor) and not H_host.is_cuda and H_host.dtype == torch.float64):
        raise TypeError("expected a float64 host tensor")
    if H_host.dim() != 2 or H_host.stride(1) != 1:
        raise ValueError("H_host must be a row-major matrix")
    n = H_host.shape[0]
    opts = make_opts(mode, slices, executor, tol, energy_tol, max_iter, 8, refine, method, fp32_storage,
                     late_slices, late_idem)
    if out is None:
        out = torch.empty((n, n), dtype=torch.float64, pin_memory=H_host.is_pinned())
    if out.is_cuda or out.dtype != torch.float64 or out.stride(1) != 1 or tuple(out.shape) != (n, n):
        raise ValueError("out must be an n x n row-major float64 host tensor")
    if ws is None:
        ws = workspace(host_workspace_bytes(n, opts))
    info = Info()
    code = lib().dm_purify_host(H_host.data_ptr(), n, H_host.stride(0), int(n_occ), ctypes.byref(opts),
                                out.data_ptr(), out.stride(0), ctypes.byref(info), ws.data_ptr(), ws.numel(),
                                _stream_ptr(stream))
    _check(code, "dm_purify_host", allow_status=True)
    return out, info.as_dict()


def foe_params(kT: float, n_terms: int, mu: float | None = None, n_occ: int | None = None, bounds=None,
               scheme="recurrence") -> FoeParams:
    lo, hi = (0.0, 0.0) if bounds is None else (float(bounds[0]), float(bounds[1]))
    return FoeParams(float(kT), 0.0 if mu is None else float(mu), 0 if n_occ is None else int(n_occ),
                     int(n_terms), FOE_SCHEMES[scheme], lo, hi)


def foe_workspace_bytes(n: int, params: FoeParams, opts: Opts) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().dm_foe_workspace_size(n, ctypes.byref(params), ctypes.byref(opts), ctypes.byref(b)),
           "dm_foe_workspace_size")
    return b.value


def foe(H: torch.Tensor, kT: float, n_terms: int, mu: float | None = None, n_occ: int | None = None,
        bounds=None, mode="int8", slices=7, executor="auto", scheme="recurrence", P=None, ws=None, stream=None):
    """dm_foe: the Chebyshev Fermi-operator expansion P = f(H) at electronic
    temperature kT on a float64 CUDA tensor H. Give mu (grand-canonical) or
    n_occ (mu solved so that tr(P) = n_occ). `bounds` = (e_min, e_max) is a
    spectral enclosure to scale H by (default: the Gershgorin bounds).
    `scheme`: "recurrence" (M - 2 products per pass) or "ps" (the
    Paterson-Stockmeyer evaluation, about 2 sqrt(M) products). Returns
    (P, info dict)."""
    _require_cuda(H)
    if (mu is None) == (n_occ is None):
        raise ValueError("give exactly one of mu and n_occ")
    n = H.shape[0]
    opts = make_opts(mode, slices, executor)
    params = foe_params(kT, n_terms, mu, n_occ, bounds, scheme)
    if P is None:
        P = torch.empty_like(H)
    if ws is None:
        ws = workspace(foe_workspace_bytes(n, params, opts), H.device)
    info = FoeInfo()
    code = lib().dm_foe(H.data_ptr(), n, H.stride(0), ctypes.byref(params), ctypes.byref(opts), P.data_ptr(),
                        P.stride(0), ctypes.byref(info), ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    _check(code, "dm_foe")
    return P, info.as_dict()


def gemm_workspace_bytes(m, n, k, mode="int8", slices=7, executor="auto") -> int:
    b = ctypes.c_size_t(0)
    _check(lib().ozaki_gemm_workspace_size(m, n, k, MODES[mode], slices, EXECUTORS[executor],
                                           ctypes.byref(b)), "ozaki_gemm_workspace_size")
    return b.value


def ozaki_gemm(A: torch.Tensor, B: torch.Tensor, mode="int8", slices=7, executor="auto", C=None, ws=None,
               stream=None) -> torch.Tensor:
    _require_cuda(A, B)
    m, k = A.shape
    k2, n = B.shape
    if k2 != k:
        raise ValueError("shape mismatch")
    if C is None:
        C = torch.empty((m, n), dtype=torch.float64, device=A.device)
    if ws is None:
        ws = workspace(gemm_workspace_bytes(m, n, k, mode, slices, executor), A.device)
    code = lib().ozaki_gemm(m, n, k, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), C.data_ptr(),
                            C.stride(0), MODES[mode], slices, EXECUTORS[executor], ws.data_ptr(), ws.numel(),
                            _stream_ptr(stream))
    _check(code, "ozaki_gemm")
    return C


def ozaki_level_sums(A: torch.Tensor, B: torch.Tensor, mode="int8", slices=7, executor="auto",
                     stream=None) -> torch.Tensor:
    """Exact integer level sums S[L-2] = sum_{i+j=L} A_i B_j, int32 (s, m, n)."""
    _require_cuda(A, B)
    m, k = A.shape
    n = B.shape[1]
    S = torch.zeros((slices, m, n), dtype=torch.int32, device=A.device)
    ws = workspace(gemm_workspace_bytes(m, n, k, mode, slices, executor), A.device)
    code = lib().ozaki_level_sums(m, n, k, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), S.data_ptr(),
                                  MODES[mode], slices, EXECUTORS[executor], ws.data_ptr(), ws.numel(),
                                  _stream_ptr(stream))
    _check(code, "ozaki_level_sums")
    return S


def ozaki_split(A: torch.Tensor, mode="int8", slices=7, executor="auto", stream=None):
    """(row exponents int32 (m,), digit planes (s, m, k)): int8 for the IMMA
    executor, bfloat16 for the tcgen05 executor, raw E4M3 bytes (uint8) for
    mode "e4m3"."""
    _require_cuda(A)
    m, k = A.shape
    ex = executor if executor != "auto" else ("imma" if mode == "int8" else "tc")
    dt = torch.uint8 if mode == "e4m3" else (torch.int8 if ex == "imma" else torch.bfloat16)
    exps = torch.empty(m, dtype=torch.int32, device=A.device)
    digits = torch.empty((slices, m, k), dtype=dt, device=A.device)
    ws = workspace(gemm_workspace_bytes(m, 1, k, mode, slices, ex), A.device)
    code = lib().ozaki_split(m, k, A.data_ptr(), A.stride(0), MODES[mode], slices, EXECUTORS[ex], exps.data_ptr(),
                             digits.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    _check(code, "ozaki_split")
    return exps, digits


def backward_workspace_bytes(n: int, opts: Opts) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().dmp_backward_workspace_size(n, ctypes.byref(opts), ctypes.byref(b)), "dmp_backward_workspace_size")
    return b.value


def purify_backward(H: torch.Tensor, n_occ: int, tape: torch.Tensor, G: torch.Tensor, mode="int8", slices=7,
                    executor="auto", tol=1e-10, energy_tol=0.0, max_iter=100, checkpoint_every=8,
                    bounds_constant=False, ws=None, stream=None) -> torch.Tensor:
    """dm_purify_backward: dL/dH (symmetric) from G = dL/dP for the purification
    that `purify(..., tape=tape)` ran with the same options."""
    _require_cuda(H, G)
    n = H.shape[0]
    opts = make_opts(mode, slices, executor, tol, energy_tol, max_iter, checkpoint_every)
    opts.flags = FLAG_BOUNDS_CONSTANT if bounds_constant else 0
    H = H.contiguous()
    G = G.contiguous()
    out = torch.empty_like(H)
    if ws is None:
        ws = workspace(backward_workspace_bytes(n, opts), H.device)
    code = lib().dm_purify_backward(H.data_ptr(), n, int(n_occ), ctypes.byref(opts), tape.data_ptr(), tape.numel(),
                                    G.data_ptr(), out.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    _check(code, "dm_purify_backward")
    return out


class PurifyFunction(torch.autograd.Function):
    """P = purify(H) with a hand-written backward (dm_purify_backward).

    The forward keeps the adjoint tape (checkpoints every `checkpoint_every`
    iterates); the backward returns the gradient for symmetric H."""

    @staticmethod
    def forward(ctx, H, n_occ, mode, slices, executor, tol, max_iter, checkpoint_every, bounds_constant):
        H = H.contiguous()
        n = H.shape[0]
        opts = make_opts(mode, slices, executor, tol, 0.0, max_iter, checkpoint_every)
        tape = torch.empty(tape_bytes(n, opts), dtype=torch.uint8, device=H.device)
        P, info = purify(H, n_occ, mode=mode, slices=slices, executor=executor, tol=tol, max_iter=max_iter,
                         tape=tape, checkpoint_every=checkpoint_every)
        ctx.save_for_backward(H)
        ctx.tape = tape
        ctx.cfg = (n_occ, mode, slices, executor, tol, max_iter, checkpoint_every, bounds_constant)
        ctx.info = info
        return P

    @staticmethod
    def backward(ctx, gP):
        (H,) = ctx.saved_tensors
        n_occ, mode, slices, executor, tol, max_iter, every, bc = ctx.cfg
        dH = purify_backward(H, n_occ, ctx.tape, gP.to(torch.float64), mode=mode, slices=slices, executor=executor,
                             tol=tol, max_iter=max_iter, checkpoint_every=every, bounds_constant=bc)
        return dH, None, None, None, None, None, None, None, None


def purify_autograd(H, n_occ, mode="int8", slices=7, executor="auto", tol=1e-10, max_iter=100, checkpoint_every=8,
                    bounds_constant=False):
    """Differentiable purification: P = purify(H), backward through dm_purify_backward."""
    return PurifyFunction.apply(H, n_occ, mode, slices, executor, tol, max_iter, checkpoint_every, bounds_constant)


def batched_workspace_bytes(ns, opts: Opts) -> int:
    arr = (ctypes.c_int64 * len(ns))(*[int(x) for x in ns])
    b = ctypes.c_size_t(0)
    _check(lib().dmp_batched_workspace_size(len(ns), arr, ctypes.byref(opts), ctypes.byref(b)),
           "dmp_batched_workspace_size")
    return b.value


def purify_batched(Hs, n_occs, mode="int8", slices=0, executor="tc", tol=1e-10, energy_tol=0.0, max_iter=100,
                   Ps=None, ws=None, stream=None, raise_on_error=True, stream_launches=False, refine=0):
    """dm_purify_batched over a list of float64 CUDA tensors (each n x n,
    contiguous). slices=0 lets the library's autotuner pick s. refine=r > 0
    adds the r-slice refinement step to every member (opts.refine_slices).
    stream_launches=True runs the iterations as plain stream launches instead
    of one graph launch (DMP_FLAG_BATCHED_STREAM: same results, visible to
    profilers and to dmp_profile_*). Returns (list of P, list of info dicts,
    return code)."""
    for H in Hs:
        _require_cuda(H)
    B = len(Hs)
    opts = make_opts(mode, slices if slices else 7, executor, tol, energy_tol, max_iter)
    opts.slices = int(slices)
    opts.flags = FLAG_BATCHED_STREAM if stream_launches else 0
    opts.refine_slices = int(refine)
    ns = [int(H.shape[0]) for H in Hs]
    Hs = [H.contiguous() for H in Hs]
    if Ps is None:
        Ps = [torch.empty_like(H) for H in Hs]
    if ws is None:
        ws = workspace(batched_workspace_bytes(ns, opts), Hs[0].device)
    Hp = (ctypes.c_void_p * B)(*[H.data_ptr() for H in Hs])
    Pp = (ctypes.c_void_p * B)(*[P.data_ptr() for P in Ps])
    na = (ctypes.c_int64 * B)(*ns)
    oa = (ctypes.c_int64 * B)(*[int(x) for x in n_occs])
    infos = (Info * B)()
    code = lib().dm_purify_batched(B, Hp, na, oa, Pp, ctypes.byref(opts), infos, ws.data_ptr(), ws.numel(),
                                   _stream_ptr(stream))
    if raise_on_error:
        _check(code, "dm_purify_batched", allow_status=True)
    return Ps, [infos[i].as_dict() for i in range(B)], code
