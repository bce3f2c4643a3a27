"""Python binding of the C ABI in ``include/mbbp.h`` (ctypes).

Argument marshalling only: every step of the decoder runs in ``libmbbp.so``.
The functions keep the C names.  Host arrays are numpy arrays; device buffers
are CUDA torch tensors (torch provides the memory and the current stream).
Packed bit vectors (uint32 words in the ABI) are held in int32 tensors,
uint16 outputs in int16 tensors and uint64 counters in int64 tensors, with
the same bits.

There is no CPU fallback: importing this module raises if the library has
not been built, and every non-OK status raises ``MBBPError``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmbbp.so")

RULE_NMS = 0
RULE_SP = 1
SCHEDULE_FLOODING = 0
SCHEDULE_SERIAL = 1
DECISION_FWS = 0
DECISION_LMS = 1
NOISE_BSC = 0
NOISE_DEPOLARIZING = 1
PROBE_FADD = 0
PROBE_FMNMX = 1
PROBE_LOP3 = 2
PROBE_SMEM = 3
MAX_R = 64
LMAX = 1.0e4
SP_MAX = 16.635532

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = C.CDLL(LIB_PATH)


class MBBPError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.mbbp_last_error().decode()
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


class CodeIO(C.Structure):
    """mbbp_code_io: one code's device buffers in a mixed batch."""
    _fields_ = [("batch", C.c_int), ("syndromes", C.c_void_p), ("llr", C.c_void_p),
                ("llr_stride", C.c_int), ("e_hat", C.c_void_p), ("conv", C.c_void_p),
                ("iters_run", C.c_void_p), ("success", C.c_void_p), ("selected", C.c_void_p)]


class Options(C.Structure):
    """mbbp_options: check rule, alpha, schedule and decision rule."""
    _fields_ = [("rule", C.c_int), ("alpha", C.c_float), ("schedule", C.c_int), ("decision", C.c_int)]


_i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
_vp = C.c_void_p
_sig = {
    "mbbp_last_error": (C.c_char_p, []),
    "mbbp_version": (C.c_char_p, []),
    "mbbp_permutation": (C.c_int, [C.c_uint64, C.c_int, C.c_int, _i32p]),
    "mbbp_subtrees": (C.c_int, [_u8p, C.c_int, C.c_int, _i32p, _i32p, _vp, _vp]),
    "mbbp_collect_subtrees": (C.c_int, [_u8p, C.c_int, C.c_int, C.c_int, C.c_uint64, _i32p, _i32p]),
    "mbbp_build_bases": (C.c_int, [_u8p, C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(_vp)]),
    "mbbp_build_bases_from_sets": (C.c_int, [_u8p, C.c_int, C.c_int, C.c_int, _i32p, _i32p,
                                             C.POINTER(_vp)]),
    "mbbp_random_sets": (C.c_int, [C.c_int, C.c_int, _i32p, C.c_uint64, _i32p, _i32p]),
    "mbbp_bases_info": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "mbbp_bases_layers": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    "mbbp_bases_free": (None, [_vp]),
    "mbbp_sample_errors": (C.c_int, [C.c_int, C.c_int, C.c_uint64, C.c_uint64, C.c_double, C.c_int,
                                     _vp, _vp, _vp]),
    "mbbp_syndrome": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    "mbbp_decode_workspace_size": (C.c_size_t, [_vp, C.c_int]),
    "mbbp_decode": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, C.c_int, C.c_float, C.c_int,
                              _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "mbbp_decode_ex": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, C.c_int, C.POINTER(Options),
                                 _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "mbbp_decode_trace": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, C.c_int, C.POINTER(Options),
                                    _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "mbbp_decode_noalloc": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, C.c_int, C.c_float, C.c_int,
                                      _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "mbbp_plan_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(_vp)]),
    "mbbp_plan_free": (None, [_vp]),
    "mbbp_plan_workspace_size": (C.c_size_t, [_vp, _i32p]),
    "mbbp_decode_mixed": (C.c_int, [_vp, C.POINTER(CodeIO), C.c_int, C.c_float, C.c_int, _vp,
                                    C.c_size_t, _vp]),
    "mbbp_plan_autotune": (C.c_int, [_vp, C.POINTER(CodeIO), C.c_int, C.c_float, C.c_int, _vp,
                                     C.c_size_t, _vp, C.POINTER(C.c_float)]),
    "mbbp_plan_info": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "mbbp_wms_workspace_size": (C.c_size_t, [_vp, C.c_int, C.c_int, C.c_int]),
    "mbbp_wms_forward": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp, C.c_int, _vp,
                                   C.c_float, C.c_int, _vp, _vp, _vp, C.c_size_t, _vp]),
    "mbbp_wms_backward": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp, C.c_int, _vp,
                                    C.c_float, C.c_int, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "mbbp_wms_decode_workspace_size": (C.c_size_t, [_vp, C.c_int, C.c_int]),
    "mbbp_wms_decode": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp,
                                  _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "mbbp_adam_step": (C.c_int, [_vp, _vp, _vp, _vp, C.c_size_t, C.c_float, C.c_float, C.c_float,
                                 C.c_float, C.c_int, C.c_float, C.c_float, _vp]),
    "mbbp_logicals_build": (C.c_int, [_u8p, C.c_int, _u8p, C.c_int, C.c_int, C.POINTER(_vp)]),
    "mbbp_logicals_info": (C.c_int, [_vp, _vp, _vp]),
    "mbbp_judge": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp]),
    "mbbp_logicals_free": (None, [_vp]),
    "mbbp_probe": (C.c_int, [C.c_int, C.c_int, _vp, C.POINTER(C.c_double), _vp]),
}
for _name, (_res, _args) in _sig.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

EXPORTED = tuple(_sig)


def _check(status: int, where: str) -> None:
    if status != 0:
        raise MBBPError(status, where)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.uint8)


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dptr(t, dtype=None, name="buffer"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _out(t, dtype, name, numel, device):
    """_dptr plus the checks the kernels rely on: at least `numel` elements
    and the handle's device (an undersized or foreign buffer would be read or
    written out of bounds)."""
    if t is None:
        return None
    ptr = _dptr(t, dtype, name)
    if t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements, got {t.numel()}")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the handle on cuda:{device}")
    return ptr


def _llr_checked(llr, n, batch, device):
    """Pointer and stride of a channel-LLR tensor: [n] (shared) or
    [batch, stride >= n] (per shot)."""
    import torch
    if llr.dim() == 1:
        return _out(llr, torch.float32, "llr", n, device), 0
    stride = llr.shape[-1]
    if stride < n:
        raise ValueError(f"llr rows must hold at least n = {n} values, got {stride}")
    return _out(llr, torch.float32, "llr", batch * stride, device), stride


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _current_device():
    try:
        import torch
        return torch.cuda.current_device() if torch.cuda.is_available() else None
    except Exception:  # pragma: no cover
        return None


def mbbp_version() -> str:
    return _lib.mbbp_version().decode()


def mbbp_last_error() -> str:
    return _lib.mbbp_last_error().decode()


# ----------------------------------------------------------------- host only

def mbbp_permutation(seed: int, j: int, m: int) -> np.ndarray:
    perm = np.zeros(m, np.int32)
    _check(_lib.mbbp_permutation(seed, j, m, perm), "mbbp_permutation")
    return perm


def mbbp_subtrees(H, perm):
    """Algorithm 2: (check_sets 1-based, acceptance order, number of subtrees)."""
    H = _u8(H)
    m, n = H.shape
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    cs = np.zeros(m, np.int32)
    order = np.zeros(m, np.int32)
    ns = C.c_int32(0)
    _check(_lib.mbbp_subtrees(H, m, n, perm, cs, _np_ptr(order), C.cast(C.pointer(ns), C.c_void_p)),
           "mbbp_subtrees")
    return cs, order, int(ns.value)


def mbbp_collect_subtrees(H, R: int, seed: int):
    """The R subtrees used as representations (row arrays in acceptance order)."""
    H = _u8(H)
    m, n = H.shape
    ptr = np.zeros(R + 1, np.int32)
    rows = np.zeros(max(R * m, 1), np.int32)
    _check(_lib.mbbp_collect_subtrees(H, m, n, R, seed, ptr, rows), "mbbp_collect_subtrees")
    return [rows[ptr[t]:ptr[t + 1]].copy() for t in range(R)]


class Bases:
    """Owner of an ``mbbp_bases`` handle (freed with the object)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)
        info = mbbp_bases_info(self)
        self.m, self.n, self.R = info["m"], info["n"], info["R"]
        self.rows, self.edges, self.sets = info["rows"], info["edges"], info["sets"]
        self.words = (self.n + 31) // 32
        self.device = _current_device()  # the device its tables were copied to

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _lib.mbbp_bases_free(h)
            self.handle = C.c_void_p(None)


def mbbp_build_bases(H, R: int, seed: int) -> Bases:
    H = _u8(H)
    m, n = H.shape
    out = C.c_void_p()
    _check(_lib.mbbp_build_bases(H, m, n, R, seed, C.byref(out)), "mbbp_build_bases")
    return Bases(out.value)


def mbbp_build_bases_from_sets(H, sets) -> Bases:
    H = _u8(H)
    m, n = H.shape
    R = len(sets)
    ptr = np.zeros(R + 1, np.int32)
    for t, s in enumerate(sets):
        ptr[t + 1] = ptr[t] + len(s)
    rows = np.ascontiguousarray(
        np.concatenate([np.asarray(s, np.int32) for s in sets]) if ptr[-1] else np.zeros(1, np.int32),
        dtype=np.int32)
    out = C.c_void_p()
    _check(_lib.mbbp_build_bases_from_sets(H, m, n, R, ptr, rows, C.byref(out)),
           "mbbp_build_bases_from_sets")
    return Bases(out.value)


def mbbp_bases_info(B: Bases) -> dict:
    m, n, R = C.c_int32(), C.c_int32(), C.c_int32()
    _check(_lib.mbbp_bases_info(B.handle, C.cast(C.pointer(m), _vp), C.cast(C.pointer(n), _vp),
                                C.cast(C.pointer(R), _vp), None, None, None, None), "mbbp_bases_info")
    R_ = R.value
    rows = np.zeros(R_, np.int32)
    edges = np.zeros(R_, np.int32)
    ptr = np.zeros(R_ + 1, np.int32)
    _check(_lib.mbbp_bases_info(B.handle, None, None, None, _np_ptr(rows), _np_ptr(edges),
                                _np_ptr(ptr), None), "mbbp_bases_info")
    srows = np.zeros(max(int(ptr[-1]), 1), np.int32)
    _check(_lib.mbbp_bases_info(B.handle, None, None, None, None, None, None, _np_ptr(srows)),
           "mbbp_bases_info")
    sets = [srows[ptr[t]:ptr[t + 1]].copy() for t in range(R_)]
    return {"m": m.value, "n": n.value, "R": R_, "rows": rows, "edges": edges, "sets": sets}


def mbbp_random_sets(m: int, sizes, seed: int) -> list:
    """Random augmentation sets (Table II): list of int32 row arrays."""
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    R = len(sizes)
    ptr = np.zeros(R + 1, np.int32)
    rows = np.zeros(max(int(np.minimum(sizes, m).sum()), 1), np.int32)
    _check(_lib.mbbp_random_sets(m, R, sizes, seed, ptr, rows), "mbbp_random_sets")
    return [rows[ptr[t]:ptr[t + 1]].copy() for t in range(R)]


def mbbp_bases_layers(B: Bases, t: int) -> list:
    """Layers of the serial schedule of representation t: list of row arrays."""
    nl = C.c_int32()
    _check(_lib.mbbp_bases_layers(B.handle, t, None, None, C.cast(C.pointer(nl), _vp)), "mbbp_bases_layers")
    info = mbbp_bases_info(B)
    order = np.zeros(int(info["rows"][t]), np.int32)
    ptr = np.zeros(nl.value + 1, np.int32)
    _check(_lib.mbbp_bases_layers(B.handle, t, _np_ptr(order), _np_ptr(ptr), None), "mbbp_bases_layers")
    return [order[ptr[L]:ptr[L + 1]].copy() for L in range(nl.value)]


# ----------------------------------------------------------------- device

def mbbp_sample_errors(n: int, batch: int, first_shot: int, seed: int, p: float, noise: int,
                       ex, ez=None, stream=None) -> None:
    """ex / ez: int32 CUDA tensors of batch * ceil(n/32) words."""
    import torch
    words = batch * ((n + 31) // 32)
    _check(_lib.mbbp_sample_errors(n, batch, first_shot, seed, float(p), noise,
                                   _out(ex, torch.int32, "ex", words, None), _out(ez, torch.int32, "ez", words, None),
                                   _stream(stream)), "mbbp_sample_errors")


def mbbp_syndrome(B: Bases, e, s, stream=None) -> None:
    """e: int32 [batch, W] packed errors; s: uint8 [batch, m]."""
    import torch
    batch = s.shape[0] if s.dim() > 1 else s.numel() // B.m
    _check(_lib.mbbp_syndrome(B.handle, batch, _out(e, torch.int32, "e", batch * B.words, B.device),
                              _out(s, torch.uint8, "s", batch * B.m, B.device), _stream(stream)), "mbbp_syndrome")


def mbbp_decode_workspace_size(B: Bases, batch: int) -> int:
    return int(_lib.mbbp_decode_workspace_size(B.handle, batch))


def _decode_io(B: Bases, syndromes, llr, e_hat, conv, success, iters_run, selected, posterior):
    """Checked pointers of mbbp_decode's device arguments (shared by the
    three decode entry points): batch, syndromes, llr, stride, then the
    outputs in ABI order."""
    import torch
    batch = syndromes.shape[0]
    if syndromes.numel() != batch * B.m:
        raise ValueError("syndromes must be [batch, m]")
    dev, n, R = B.device, B.n, B.R
    llr_p, stride = _llr_checked(llr, n, batch, dev)
    return (batch, _out(syndromes, torch.uint8, "syndromes", batch * B.m, dev), llr_p, stride,
            _out(e_hat, torch.uint8, "e_hat", batch * n, dev), _out(conv, torch.uint8, "conv", batch * R, dev),
            _out(iters_run, torch.int16, "iters_run", batch * R, dev),
            _out(success, torch.uint8, "success", batch, dev), _out(selected, torch.int16, "selected", batch, dev),
            _out(posterior, torch.float32, "posterior", batch * R * n, dev))


def mbbp_decode(B: Bases, syndromes, llr, iters: int, alpha: float, rule: int, e_hat, conv,
                success, workspace, iters_run=None, selected=None, posterior=None,
                stream=None) -> None:
    """Algorithm 1 on a batch; see mbbp.h for every argument."""
    import torch
    batch, sp, lp, stride, ep, cp, ip, okp, selp, pp = _decode_io(B, syndromes, llr, e_hat, conv, success,
                                                                  iters_run, selected, posterior)
    _check(_lib.mbbp_decode(
        B.handle, batch, sp, lp, stride, iters, float(alpha), rule, ep, cp, ip, okp, selp, pp,
        _out(workspace, torch.uint8, "workspace", 0, B.device), workspace.numel(), _stream(stream)),
        "mbbp_decode")


def mbbp_decode_ex(B: Bases, syndromes, llr, iters: int, opt: Options, e_hat, conv, success, workspace,
                   iters_run=None, selected=None, posterior=None, stream=None) -> None:
    """mbbp_decode with a schedule and a decision rule (Options)."""
    import torch
    batch, sp, lp, stride, ep, cp, ip, okp, selp, pp = _decode_io(B, syndromes, llr, e_hat, conv, success,
                                                                  iters_run, selected, posterior)
    _check(_lib.mbbp_decode_ex(
        B.handle, batch, sp, lp, stride, iters, C.byref(opt), ep, cp, ip, okp, selp, pp,
        _out(workspace, torch.uint8, "workspace", 0, B.device), workspace.numel(), _stream(stream)),
        "mbbp_decode_ex")


def mbbp_decode_trace(B: Bases, syndromes, llr, iters: int, opt: Options, e_hat, conv, success, c2v, workspace,
                      iters_run=None, selected=None, posterior=None, stream=None) -> None:
    """mbbp_decode_ex (flooding) that also writes the last iteration's check
    messages of every (shot, representation) to c2v, float32 [batch, R, E]
    with E the largest edge count (edges row by row, columns ascending)."""
    import torch
    batch, sp, lp, stride, ep, cp, ip, okp, selp, pp = _decode_io(B, syndromes, llr, e_hat, conv, success,
                                                                  iters_run, selected, posterior)
    cvp = _out(c2v, torch.float32, "c2v", batch * B.R * int(B.edges.max()), B.device)
    _check(_lib.mbbp_decode_trace(
        B.handle, batch, sp, lp, stride, iters, C.byref(opt), ep, cp, ip, okp, selp, pp, cvp,
        _out(workspace, torch.uint8, "workspace", 0, B.device), workspace.numel(), _stream(stream)),
        "mbbp_decode_trace")


def mbbp_decode_noalloc(B: Bases, syndromes, llr, iters: int, alpha: float, rule: int, e_hat, conv,
                        success, iters_run=None, selected=None, posterior=None, stream=None) -> None:
    """mbbp_decode without a workspace, for callers that cannot allocate
    device memory: the scratch is the library's fixed array (see mbbp.h for
    its size limit and for why overlapping calls race)."""
    batch, sp, lp, stride, ep, cp, ip, okp, selp, pp = _decode_io(B, syndromes, llr, e_hat, conv, success,
                                                                  iters_run, selected, posterior)
    _check(_lib.mbbp_decode_noalloc(
        B.handle, batch, sp, lp, stride, iters, float(alpha), rule, ep, cp, ip, okp, selp, pp,
        _stream(stream)), "mbbp_decode_noalloc")


class Plan:
    """Owner of an ``mbbp_plan`` (keeps its code handles alive)."""

    def __init__(self, codes):
        self.codes = list(codes)
        arr = (C.c_void_p * len(self.codes))(*[c.handle.value for c in self.codes])
        out = C.c_void_p()
        _check(_lib.mbbp_plan_create(arr, len(self.codes), C.byref(out)), "mbbp_plan_create")
        self.handle = out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _lib.mbbp_plan_free(h)
            self.handle = C.c_void_p(None)


def mbbp_plan_create(codes) -> Plan:
    return Plan(codes)


def mbbp_plan_workspace_size(P: Plan, batches) -> int:
    return int(_lib.mbbp_plan_workspace_size(P.handle, np.ascontiguousarray(batches, dtype=np.int32)))


def mbbp_plan_info(P: Plan) -> dict:
    nc = len(P.codes)
    warps = C.c_int32()
    chunk, kind, order = (np.zeros(nc, np.int32) for _ in range(3))
    _check(_lib.mbbp_plan_info(P.handle, C.cast(C.pointer(warps), _vp), _np_ptr(chunk), _np_ptr(kind),
                               _np_ptr(order)), "mbbp_plan_info")
    return {"warps": warps.value, "chunk": chunk.tolist(), "kind": kind.tolist(), "order": order.tolist()}


def _code_io(P: Plan, ios):
    if len(ios) != len(P.codes):
        raise ValueError(f"the plan has {len(P.codes)} codes, got {len(ios)} inputs")
    arr = (CodeIO * len(ios))()
    for i, (B, x) in enumerate(zip(P.codes, ios)):
        batch, sp, lp, stride, ep, cp, ip, okp, selp, _ = _decode_io(
            B, x["syndromes"], x["llr"], x["e_hat"], x["conv"], x["success"], x.get("iters"), x.get("selected"),
            None)
        arr[i] = CodeIO(batch, sp, lp, stride, ep, cp, ip, okp, selp)
    return arr


def mbbp_decode_mixed(P: Plan, ios, iters: int, alpha: float, rule: int, workspace, stream=None) -> None:
    """ios: one dict per code of the plan with CUDA tensors syndromes, llr,
    e_hat, conv, success and optionally iters (int16) and selected."""
    import torch
    arr = _code_io(P, ios)
    _check(_lib.mbbp_decode_mixed(P.handle, arr, iters, float(alpha), rule,
                                  _dptr(workspace, torch.uint8, "workspace"), workspace.numel(), _stream(stream)),
           "mbbp_decode_mixed")


def mbbp_plan_autotune(P: Plan, ios, iters: int, alpha: float, rule: int, workspace, stream=None) -> float:
    import torch
    arr = _code_io(P, ios)
    best = C.c_float(0.0)
    _check(_lib.mbbp_plan_autotune(P.handle, arr, iters, float(alpha), rule,
                                   _dptr(workspace, torch.uint8, "workspace"), workspace.numel(),
                                   _stream(stream), C.byref(best)), "mbbp_plan_autotune")
    return best.value


def mixed_buffers(P: Plan, syndromes, llrs) -> tuple[list, object]:
    """Allocate per-code outputs (torch, on the syndromes' device) and the
    workspace for mbbp_decode_mixed; returns (ios, workspace)."""
    import torch
    ios = []
    for B, s, l in zip(P.codes, syndromes, llrs):
        b, dev = s.shape[0], s.device
        ios.append({"syndromes": s, "llr": l,
                    "e_hat": torch.empty((b, B.n), dtype=torch.uint8, device=dev),
                    "conv": torch.empty((b, B.R), dtype=torch.uint8, device=dev),
                    "iters": torch.empty((b, B.R), dtype=torch.int16, device=dev),
                    "success": torch.empty((b,), dtype=torch.uint8, device=dev),
                    "selected": torch.empty((b,), dtype=torch.int16, device=dev)})
    ws = torch.empty(mbbp_plan_workspace_size(P, [s.shape[0] for s in syndromes]), dtype=torch.uint8,
                     device=syndromes[0].device)
    return ios, ws


# ----------------------------------------------------------- weighted min-sum

def wms_params(B: Bases, T: int, alpha: float = 0.625, device="cuda"):
    """(w, g) initialised to normalized min-sum: w = alpha, g = 0, shape
    [R, T, E] with E the largest edge count of the representations."""
    import torch
    E = int(B.edges.max())
    w = torch.full((B.R, T, E), float(alpha), dtype=torch.float32, device=device)
    g = torch.zeros((B.R, T, E), dtype=torch.float32, device=device)
    return w, g


def mbbp_wms_workspace_size(B: Bases, batch: int, T: int, ckpt: int) -> int:
    return int(_lib.mbbp_wms_workspace_size(B.handle, batch, T, ckpt))


def _wms_io(B, syndromes, llr, T, w, g, etrue):
    """Checked pointers shared by the WMS entry points: batch, syndromes,
    llr, stride, w, g, etrue."""
    import torch
    batch = syndromes.shape[0]
    if syndromes.numel() != batch * B.m:
        raise ValueError("syndromes must be [batch, m]")
    dev = B.device
    wn = B.R * T * int(B.edges.max())
    llr_p, stride = _llr_checked(llr, B.n, batch, dev)
    return (batch, _out(syndromes, torch.uint8, "syndromes", batch * B.m, dev), llr_p, stride,
            _out(w, torch.float32, "w", wn, dev), _out(g, torch.float32, "g", wn, dev),
            _out(etrue, torch.int32, "etrue", batch * B.words, dev))


def mbbp_wms_forward(B, syndromes, llr, T, w, g, ckpt, etrue, scale, posterior, loss, workspace,
                     all_iters=False, stream=None) -> None:
    import torch
    batch, sp, lp, stride, wp, gp, ep = _wms_io(B, syndromes, llr, T, w, g, etrue)
    dev = B.device
    _check(_lib.mbbp_wms_forward(
        B.handle, batch, sp, lp, stride, T, wp, gp, ckpt, ep, float(scale), int(all_iters),
        _out(posterior, torch.float32, "posterior", batch * B.R * B.n, dev),
        _out(loss, torch.float32, "loss", batch * B.R, dev), _out(workspace, torch.uint8, "workspace", 0, dev),
        workspace.numel(), _stream(stream)), "mbbp_wms_forward")


def mbbp_wms_backward(B, syndromes, llr, T, w, g, ckpt, etrue, scale, posterior, gw, gg, workspace,
                      all_iters=False, stream=None) -> None:
    import torch
    batch, sp, lp, stride, wp, gp, ep = _wms_io(B, syndromes, llr, T, w, g, etrue)
    dev = B.device
    wn = B.R * T * int(B.edges.max())
    _check(_lib.mbbp_wms_backward(
        B.handle, batch, sp, lp, stride, T, wp, gp, ckpt, ep, float(scale), int(all_iters),
        _out(posterior, torch.float32, "posterior", batch * B.R * B.n, dev),
        _out(gw, torch.float32, "gw", wn, dev), _out(gg, torch.float32, "gg", wn, dev),
        _out(workspace, torch.uint8, "workspace", 0, dev), workspace.numel(), _stream(stream)), "mbbp_wms_backward")


def mbbp_wms_decode_workspace_size(B: Bases, batch: int, T: int) -> int:
    return int(_lib.mbbp_wms_decode_workspace_size(B.handle, batch, T))


def mbbp_wms_decode(B, syndromes, llr, iters, T, w, g, e_hat, conv, success, workspace, iters_run=None,
                    selected=None, stream=None) -> None:
    import torch
    batch, sp, lp, stride, wp, gp, _ = _wms_io(B, syndromes, llr, T, w, g, None)
    _, _, _, _, ep, cp, ip, okp, selp, _ = _decode_io(B, syndromes, llr, e_hat, conv, success, iters_run, selected,
                                                      None)
    _check(_lib.mbbp_wms_decode(
        B.handle, batch, sp, lp, stride, iters, T, wp, gp, ep, cp, ip, okp, selp,
        _out(workspace, torch.uint8, "workspace", 0, B.device), workspace.numel(), _stream(stream)),
        "mbbp_wms_decode")


def mbbp_adam_step(params, grad, m, v, lr, beta1, beta2, eps, step, lo, hi, stream=None) -> None:
    import torch
    cnt, dev = params.numel(), params.device.index
    _check(_lib.mbbp_adam_step(_dptr(params, torch.float32, "params"), _out(grad, torch.float32, "grad", cnt, dev),
                               _out(m, torch.float32, "m", cnt, dev), _out(v, torch.float32, "v", cnt, dev), cnt,
                               float(lr), float(beta1), float(beta2), float(eps), int(step), float(lo), float(hi),
                               _stream(stream)), "mbbp_adam_step")


def wms_decode(B, syndromes, llr, iters, w, g) -> dict:
    """Allocate outputs and run mbbp_wms_decode (T = w.shape[1])."""
    import torch
    dev = syndromes.device
    batch = syndromes.shape[0]
    out = {"e_hat": torch.empty((batch, B.n), dtype=torch.uint8, device=dev),
           "conv": torch.empty((batch, B.R), dtype=torch.uint8, device=dev),
           "iters": torch.empty((batch, B.R), dtype=torch.int16, device=dev),
           "success": torch.empty((batch,), dtype=torch.uint8, device=dev),
           "selected": torch.empty((batch,), dtype=torch.int16, device=dev)}
    ws = torch.empty(mbbp_wms_decode_workspace_size(B, batch, w.shape[1]), dtype=torch.uint8, device=dev)
    mbbp_wms_decode(B, syndromes, llr, iters, w.shape[1], w, g, out["e_hat"], out["conv"], out["success"], ws,
                    iters_run=out["iters"], selected=out["selected"])
    return out


def _wms_function():
    import torch

    class WMSLoss(torch.autograd.Function):
        """Summed WMS loss of a batch; backward is the hand-written adjoint
        kernel (mbbp_wms_backward) with checkpoints every `ckpt` iterations."""

        @staticmethod
        def forward(ctx, w, g, B, syndromes, llr, etrue, ckpt, scale, all_iters):
            T = w.shape[1]
            batch = syndromes.shape[0]
            post = torch.empty((batch, B.R, B.n), dtype=torch.float32, device=w.device)
            loss = torch.empty((batch, B.R), dtype=torch.float32, device=w.device)
            ws = torch.empty(mbbp_wms_workspace_size(B, batch, T, ckpt), dtype=torch.uint8, device=w.device)
            mbbp_wms_forward(B, syndromes, llr, T, w, g, ckpt, etrue, scale, post, loss, ws, all_iters=all_iters)
            ctx.B, ctx.ckpt, ctx.scale, ctx.all_iters = B, ckpt, scale, all_iters
            ctx.save_for_backward(w, g, syndromes, llr, etrue, post, ws)
            return loss.sum()

        @staticmethod
        def backward(ctx, grad_out):
            w, g, syndromes, llr, etrue, post, ws = ctx.saved_tensors
            gw = torch.zeros_like(w)
            gg = torch.zeros_like(g)
            mbbp_wms_backward(ctx.B, syndromes, llr, w.shape[1], w, g, ctx.ckpt, etrue, ctx.scale, post, gw, gg, ws,
                              all_iters=ctx.all_iters)
            return gw * grad_out, gg * grad_out, None, None, None, None, None, None, None

    return WMSLoss


_WMS_FN = None


def wms_loss(w, g, B, syndromes, llr, etrue, ckpt: int = 5, scale: float | None = None, all_iters: bool = False):
    """Differentiable WMS loss (mean BCE over shots, representations and
    variables unless ``scale`` is given; with ``all_iters`` also over the
    iterations).  etrue: bit-packed true errors (int32 words)."""
    global _WMS_FN
    if _WMS_FN is None:
        _WMS_FN = _wms_function()
    if scale is None:
        scale = 1.0 / (syndromes.shape[0] * B.R * B.n)
    return _WMS_FN.apply(w, g, B, syndromes, llr, etrue, ckpt, scale, all_iters)


class Logicals:
    """Owner of an ``mbbp_logicals`` handle."""

    def __init__(self, handle: int, n: int):
        self.handle = C.c_void_p(handle)
        self.n = n
        self.device = _current_device()
        k = C.c_int32()
        _check(_lib.mbbp_logicals_info(self.handle, C.cast(C.pointer(k), _vp), None), "mbbp_logicals_info")
        self.k = k.value

    def ops(self) -> np.ndarray:
        out = np.zeros((max(self.k, 1), self.n), np.uint8)
        _check(_lib.mbbp_logicals_info(self.handle, None, _np_ptr(out)), "mbbp_logicals_info")
        return out[: self.k]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _lib.mbbp_logicals_free(h)
            self.handle = C.c_void_p(None)


def mbbp_logicals_build(H, H_other) -> Logicals:
    H, Ho = _u8(H), _u8(H_other)
    out = C.c_void_p()
    _check(_lib.mbbp_logicals_build(H, H.shape[0], Ho, Ho.shape[0], H.shape[1], C.byref(out)),
           "mbbp_logicals_build")
    return Logicals(out.value, H.shape[1])


def mbbp_judge(L: Logicals, e, e_hat, fail=None, counts=None, stream=None) -> None:
    import torch
    batch = e_hat.shape[0]
    n, dev = L.n, L.device
    if e_hat.numel() != batch * n:
        raise ValueError("e_hat must be [batch, n]")
    _check(_lib.mbbp_judge(L.handle, batch, _out(e, torch.int32, "e", batch * ((n + 31) // 32), dev),
                           _out(e_hat, torch.uint8, "e_hat", batch * n, dev), _out(fail, torch.uint8, "fail", batch, dev),
                           _out(counts, torch.int64, "counts", 3, dev), _stream(stream)), "mbbp_judge")


# ----------------------------------------------------------------- helpers

def decode(B: Bases, syndromes, llr, iters: int, alpha: float, rule: int = RULE_NMS,
           want_posterior: bool = False, stream=None, schedule: int = SCHEDULE_FLOODING,
           decision: int = DECISION_FWS, want_c2v: bool = False) -> dict:
    """Allocate the outputs with torch and call ``mbbp_decode`` (or
    ``mbbp_decode_ex`` for the serial schedule or the LMS decision).

    Returns a dict of CUDA tensors: e_hat [batch, n], conv [batch, R],
    iters [batch, R] (int16 holding uint16), success [batch], selected
    [batch], cand [batch, R, W] (int32 words; a view of the workspace) and
    posterior [batch, R, n] if requested, and with want_c2v the last
    iteration's check messages c2v [batch, R, E] (mbbp_decode_trace)."""
    import torch
    dev = syndromes.device
    batch = syndromes.shape[0]
    out = {
        "e_hat": torch.empty((batch, B.n), dtype=torch.uint8, device=dev),
        "conv": torch.empty((batch, B.R), dtype=torch.uint8, device=dev),
        "iters": torch.empty((batch, B.R), dtype=torch.int16, device=dev),
        "success": torch.empty((batch,), dtype=torch.uint8, device=dev),
        "selected": torch.empty((batch,), dtype=torch.int16, device=dev),
    }
    ws_bytes = mbbp_decode_workspace_size(B, batch)
    ws = torch.empty((ws_bytes,), dtype=torch.uint8, device=dev)
    post = (torch.empty((batch, B.R, B.n), dtype=torch.float32, device=dev)
            if want_posterior else None)
    if want_c2v:
        out["c2v"] = torch.zeros((batch, B.R, int(B.edges.max())), dtype=torch.float32, device=dev)
        opt = Options(rule, float(alpha), schedule, decision)
        mbbp_decode_trace(B, syndromes, llr, iters, opt, out["e_hat"], out["conv"], out["success"], out["c2v"], ws,
                          iters_run=out["iters"], selected=out["selected"], posterior=post, stream=stream)
    elif schedule == SCHEDULE_FLOODING and decision == DECISION_FWS:
        mbbp_decode(B, syndromes, llr, iters, alpha, rule, out["e_hat"], out["conv"], out["success"], ws,
                    iters_run=out["iters"], selected=out["selected"], posterior=post, stream=stream)
    else:
        opt = Options(rule, float(alpha), schedule, decision)
        mbbp_decode_ex(B, syndromes, llr, iters, opt, out["e_hat"], out["conv"], out["success"], ws,
                       iters_run=out["iters"], selected=out["selected"], posterior=post, stream=stream)
    out["cand"] = ws[: batch * B.R * B.words * 4].view(torch.int32).view(batch, B.R, B.words)
    out["workspace"] = ws
    if want_posterior:
        out["posterior"] = post
    return out


def unpack_words(words, n: int) -> np.ndarray:
    """int32 words [..., W] (numpy or tensor) -> uint8 bits [..., n]."""
    if hasattr(words, "cpu"):
        words = words.cpu().numpy()
    w = np.ascontiguousarray(words).view(np.uint32)
    bits = ((w[..., :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8)
    return bits.reshape(w.shape[:-1] + (w.shape[-1] * 32,))[..., :n]


def pack_bits(bits) -> np.ndarray:
    """uint8 bits [..., n] -> int32 words [..., ceil(n/32)]."""
    bits = np.asarray(bits, np.uint8)
    n = bits.shape[-1]
    W = (n + 31) // 32
    pad = np.zeros(bits.shape[:-1] + (W * 32,), np.uint8)
    pad[..., :n] = bits
    w = (pad.reshape(bits.shape[:-1] + (W, 32)).astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(-1)
    return w.astype(np.uint32).view(np.int32)


# ---------------------------------------------------------------- probes

def mbbp_probe(kind: int, rounds: int, sink, stream=None) -> float:
    """Enqueue one throughput-probe launch; returns its work (lane operations,
    or shared-memory bytes for PROBE_SMEM).  sink: CUDA float32 tensor [1]."""
    import torch
    work = C.c_double(0.0)
    _check(_lib.mbbp_probe(kind, rounds, _dptr(sink, torch.float32, "sink"), C.byref(work), _stream(stream)),
           "mbbp_probe")
    return work.value
