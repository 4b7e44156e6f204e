"""Thin Python binding of libfock (include/fock.h): same names, argument
marshalling only.  Every computation runs in the CUDA library; there is no
Python or CPU fallback, and a missing library raises at first use.

Device buffers are torch CUDA tensors (their data pointers are passed to the
C ABI); `stream` defaults to torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

FOCK_OK = 0
FOCK_ERR_ARG = -1
FOCK_ERR_OVERFLOW = -2
FOCK_ERR_INVALID_CONFIG = -3
FOCK_ERR_RANGE = -4
FOCK_ERR_NOMEM = -5
FOCK_ERR_NOT_HERMITIAN = -6
FOCK_ERR_ALIAS = -7
FOCK_ERR_CUDA = -8
FOCK_ERR_NOCONV = -9
FOCK_ERR_UNSUPPORTED = -10
FOCK_ERR_TIMEOUT = -11
FOCK_ERR_NOT_BUILT = -12
FOCK_ERR_DEVICE = -13
FOCK_ERR_SCRATCH_LIMIT = -14
FOCK_ERR_NOT_CONSERVING = -15
FOCK_NOALLOC_SCRATCH_BYTES = 64 << 20

FOCK_MAP_SINGLE = 1
FOCK_MAP_DOUBLE = 2

FOCK_PREC_F64 = 0
FOCK_PREC_F64_NATIVE = 1
FOCK_PREC_F32_MIXED = 2

FOCK_ARM_AUTO = 0
FOCK_ARM_HASH = 1
FOCK_ARM_MAPS = 2

FOCK_PATH_AUTO = 0
FOCK_PATH_TWOPHASE_TC = 1
FOCK_PATH_TWOPHASE = 2
FOCK_PATH_NN = 3
FOCK_PATH_DENSE = 4
FOCK_PATH_SPARSE = 5
FOCK_PATH_LIST = 6
FOCK_PATH_TWOPHASE_BLOCK = 7
FOCK_FORM_DENSE = 1
FOCK_FORM_PAIR_WEIGHT = 2
FOCK_FORM_PAIR_MOMENTUM = 4
FOCK_FORM_NEAREST_NEIGHBOUR = 8
PATH_NAMES = {1: "twophase_tc", 2: "twophase", 3: "nn", 4: "dense", 5: "sparse", 6: "list", 7: "twophase_block"}

# Every extern "C" symbol declared in include/fock.h.
EXPORTS = (
    "fock_strerror", "fock_version",
    "fock_space_create", "fock_space_destroy", "fock_space_size", "fock_rank", "fock_unrank",
    "fock_build_jump_maps", "fock_jump_map_get", "fock_jump_maps_free",
    "fock_hamiltonian_create", "fock_hamiltonian_destroy", "fock_hamiltonian_terms",
    "fock_hamiltonian_is_real", "fock_hamiltonian_forms",
    "fock_apply_path", "fock_apply_set_path", "fock_autotune",
    "fock_apply_set_events", "fock_apply_workspace_size", "fock_apply_H", "fock_apply_check", "fock_debug_set_wait_polls",
    "fock_apply_H_host", "fock_apply_H_noalloc",
    "fock_lanczos_ground", "fock_sil_step", "fock_density_matrices",
    "fock_sector_create", "fock_sector_destroy", "fock_sector_size", "fock_sector_rank", "fock_sector_unrank",
    "fock_sector_terms", "fock_sector_workspace_size", "fock_sector_apply_H", "fock_sector_lanczos_ground",
    "fock_batch_create", "fock_batch_destroy", "fock_batch_offsets", "fock_batch_own_apply", "fock_batch_terms", "fock_batch_apply",
    "fock_batch_autotune", "fock_batch_lanczos_ground",
)


class FockTuning(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("arm", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("from_cache", ctypes.c_int32), ("ms", ctypes.c_double)]


class FockError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {fock_strerror(status)} ({status})")


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libfock.so (built by ``_build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"libfock is not built ({p}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(p)
    vp, i32, i64, sz, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
    P = ctypes.POINTER
    lib.fock_strerror.restype = ctypes.c_char_p
    lib.fock_strerror.argtypes = [ctypes.c_int]
    lib.fock_version.restype = ctypes.c_int
    sigs = {
        "fock_space_create": [i32, i32, P(vp)],
        "fock_space_destroy": [vp],
        "fock_space_size": [vp, P(i64)],
        "fock_rank": [vp, vp, i64, vp, vp],
        "fock_unrank": [vp, vp, i64, vp, vp],
        "fock_build_jump_maps": [vp, ctypes.c_int, ctypes.c_int, P(sz), vp],
        "fock_jump_map_get": [vp, ctypes.c_int, P(vp), P(i64), P(i64)],
        "fock_jump_maps_free": [vp],
        "fock_hamiltonian_create": [vp, vp, vp, dbl, P(vp)],
        "fock_hamiltonian_destroy": [vp],
        "fock_hamiltonian_terms": [vp, P(i64)],
        "fock_hamiltonian_is_real": [vp, P(ctypes.c_int)],
        "fock_hamiltonian_forms": [vp, P(ctypes.c_int32)],
        "fock_apply_path": [vp, vp, i32, ctypes.c_int, ctypes.c_int, sz, P(i32)],
        "fock_apply_set_path": [vp, i32, ctypes.c_int, ctypes.c_int, ctypes.c_int],
        "fock_autotune": [vp, vp, i32, ctypes.c_int, ctypes.c_char_p, P(FockTuning), vp],
        "fock_apply_set_events": [vp, vp, vp],
        "fock_apply_workspace_size": [vp, vp, i32, ctypes.c_int, P(sz)],
        "fock_apply_H": [vp, vp, vp, vp, i32, ctypes.c_int, ctypes.c_int, vp, sz, vp],
        "fock_apply_H_host": [vp, vp, vp, vp, i32, ctypes.c_int, ctypes.c_int, vp],
        "fock_apply_H_noalloc": [vp, vp, vp, vp, i32, ctypes.c_int, vp],
        "fock_apply_check": [vp, vp, vp, ctypes.c_int, vp],
        "fock_debug_set_wait_polls": [i64],
        "fock_lanczos_ground": [vp, vp, i32, i32, dbl, ctypes.c_uint64, ctypes.c_int, vp,
                                P(dbl), P(dbl), vp, P(i32), vp],
        "fock_density_matrices": [vp, vp, vp, vp, vp],
        "fock_sil_step": [vp, vp, vp, dbl, i32, dbl, ctypes.c_int, P(i32), P(dbl), vp],
    }
    sigs.update({
        "fock_sector_create": [vp, i64, P(vp)],
        "fock_sector_destroy": [vp],
        "fock_sector_size": [vp, P(i64)],
        "fock_sector_rank": [vp, vp, i64, vp, vp],
        "fock_sector_unrank": [vp, vp, i64, vp, vp],
        "fock_sector_terms": [vp, vp, P(i64)],
        "fock_sector_workspace_size": [vp, i32, ctypes.c_int, P(sz)],
        "fock_sector_apply_H": [vp, vp, vp, vp, i32, ctypes.c_int, vp, sz, vp],
        "fock_sector_lanczos_ground": [vp, vp, i32, i32, dbl, ctypes.c_uint64, ctypes.c_int, vp,
                                       P(dbl), P(dbl), vp, P(i32), vp],
    })
    sigs.update({
        "fock_batch_create": [i32, vp, vp, vp, vp, dbl, P(vp)],
        "fock_batch_destroy": [vp],
        "fock_batch_offsets": [vp, vp],
        "fock_batch_terms": [vp, P(i64)],
        "fock_batch_own_apply": [vp, vp],
        "fock_batch_apply": [vp, vp, vp, ctypes.c_int, vp],
        "fock_batch_autotune": [vp, vp, vp, ctypes.c_int, ctypes.c_char_p, P(i32), P(i32), vp],
        "fock_batch_lanczos_ground": [vp, i32, i32, dbl, ctypes.c_uint64, vp, vp, vp, vp],
    })
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = args
    _lib = lib
    return lib


def fock_strerror(status: int) -> str:
    return load().fock_strerror(int(status)).decode()


def fock_version() -> int:
    return int(load().fock_version())


def _check(st: int, where: str, allow=()):
    if st != FOCK_OK and st not in allow:
        raise FockError(st, where)
    return st


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


# --------------------------------------------------------------------------
# space, hash, maps
# --------------------------------------------------------------------------
def fock_space_create(N: int, M: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().fock_space_create(int(N), int(M), ctypes.byref(h)), "fock_space_create")
    return h


def fock_space_destroy(sp) -> None:
    load().fock_space_destroy(sp)


def fock_space_size(sp) -> int:
    n = ctypes.c_int64()
    _check(load().fock_space_size(sp, ctypes.byref(n)), "fock_space_size")
    return n.value


def fock_rank(sp, occ, idx=None, stream=None, check: bool = True):
    """occ: int32 CUDA tensor [count, M]; returns (int64 indices, status)."""
    import torch
    count = occ.shape[0]
    if idx is None:
        idx = torch.empty(count, dtype=torch.int64, device=occ.device)
    st = load().fock_rank(sp, _dptr(occ), count, _dptr(idx), _stream(stream))
    if check:
        _check(st, "fock_rank")
    return idx, st


def fock_unrank(sp, idx, M: int, occ=None, stream=None, check: bool = True):
    """idx: int64 CUDA tensor [count]; returns (int32 occupations [count, M], status)."""
    import torch
    count = idx.shape[0]
    if occ is None:
        occ = torch.empty((count, M), dtype=torch.int32, device=idx.device)
    st = load().fock_unrank(sp, _dptr(idx), count, _dptr(occ), _stream(stream))
    if check:
        _check(st, "fock_unrank")
    return occ, st


def fock_build_jump_maps(sp, which: int, dry_run: bool = False, stream=None) -> int:
    b = ctypes.c_size_t()
    _check(load().fock_build_jump_maps(sp, int(which), int(bool(dry_run)), ctypes.byref(b),
                                       _stream(stream) if not dry_run else None),
           "fock_build_jump_maps")
    return b.value


class _DeviceArray:
    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (ptr, False), "version": 2, "strides": None}


def fock_jump_map_get(sp, which: int):
    """View [slots, N_c] of a built map as an int32 torch tensor (owned by the
    space; treat it as read-only)."""
    import torch
    p, slots, stride = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().fock_jump_map_get(sp, int(which), ctypes.byref(p), ctypes.byref(slots),
                                    ctypes.byref(stride)), "fock_jump_map_get")
    return torch.as_tensor(_DeviceArray(p.value, (slots.value, stride.value), "<i4"), device="cuda")


def fock_jump_maps_free(sp) -> None:
    _check(load().fock_jump_maps_free(sp), "fock_jump_maps_free")


# --------------------------------------------------------------------------
# Hamiltonian and apply
# --------------------------------------------------------------------------
def fock_hamiltonian_create(sp, h, W=None, tol: float = 1e-12):
    M = int(round(np.asarray(h).size ** 0.5))
    hh = np.ascontiguousarray(np.asarray(h, dtype=np.complex128).reshape(M, M))
    WW = None if W is None else np.ascontiguousarray(np.asarray(W, dtype=np.complex128).reshape(-1))
    out = ctypes.c_void_p()
    _check(load().fock_hamiltonian_create(
        sp, hh.ctypes.data_as(ctypes.c_void_p),
        None if WW is None else WW.ctypes.data_as(ctypes.c_void_p), float(tol), ctypes.byref(out)),
        "fock_hamiltonian_create")
    return out


def fock_hamiltonian_destroy(ham) -> None:
    load().fock_hamiltonian_destroy(ham)


def fock_hamiltonian_terms(ham) -> int:
    n = ctypes.c_int64()
    _check(load().fock_hamiltonian_terms(ham, ctypes.byref(n)), "fock_hamiltonian_terms")
    return n.value


def fock_hamiltonian_is_real(ham) -> bool:
    r = ctypes.c_int()
    _check(load().fock_hamiltonian_is_real(ham, ctypes.byref(r)), "fock_hamiltonian_is_real")
    return bool(r.value)


def fock_hamiltonian_forms(ham) -> int:
    """FOCK_FORM_* bits of the operator's structure."""
    r = ctypes.c_int32()
    _check(load().fock_hamiltonian_forms(ham, ctypes.byref(r)), "fock_hamiltonian_forms")
    return r.value


def fock_apply_path(sp, ham, nrhs: int = 1, precision: int = FOCK_PREC_F64, arm: int = FOCK_ARM_AUTO,
                    workspace_bytes: int | None = None) -> int:
    """FOCK_PATH_* an apply with these options takes (default: the preferred workspace)."""
    if workspace_bytes is None:
        workspace_bytes = fock_apply_workspace_size(sp, ham, nrhs, precision)
    p = ctypes.c_int32()
    _check(load().fock_apply_path(sp, ham, int(nrhs), int(precision), int(arm), int(workspace_bytes),
                                  ctypes.byref(p)), "fock_apply_path")
    return p.value


def fock_apply_set_path(ham, nrhs: int, precision: int, path: int, arm: int = FOCK_ARM_HASH) -> None:
    _check(load().fock_apply_set_path(ham, int(nrhs), int(precision), int(path),
                                      int(FOCK_ARM_AUTO if path == FOCK_PATH_AUTO else arm)),
           "fock_apply_set_path")


def fock_autotune(sp, ham, nrhs: int = 1, precision: int = FOCK_PREC_F64, cache_path: str | None = None,
                  stream=None) -> FockTuning:
    t = FockTuning()
    _check(load().fock_autotune(sp, ham, int(nrhs), int(precision),
                                None if cache_path is None else cache_path.encode(), ctypes.byref(t),
                                _stream(stream)), "fock_autotune")
    return t


def fock_apply_set_events(ham, start_event=None, stop_event=None) -> None:
    """Record torch.cuda.Event objects around the main kernel of later applies."""
    a = None if start_event is None else ctypes.c_void_p(start_event.cuda_event)
    b = None if stop_event is None else ctypes.c_void_p(stop_event.cuda_event)
    _check(load().fock_apply_set_events(ham, a, b), "fock_apply_set_events")


def fock_apply_workspace_size(sp, ham, nrhs: int, precision: int) -> int:
    b = ctypes.c_size_t()
    _check(load().fock_apply_workspace_size(sp, ham, int(nrhs), int(precision), ctypes.byref(b)),
           "fock_apply_workspace_size")
    return b.value


def fock_apply_H(sp, ham, C, sigma=None, nrhs: int = 1, precision: int = FOCK_PREC_F64,
                 arm: int = FOCK_ARM_AUTO, workspace=None, stream=None):
    """sigma = H C.  C: CUDA tensor [N_c] or [N_c, nrhs], complex128 (FOCK_PREC_F64*)
    or complex64 (FOCK_PREC_F32_MIXED).  Returns sigma (allocated if None)."""
    import torch
    if sigma is None:
        sigma = torch.empty_like(C)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load().fock_apply_H(sp, ham, _dptr(C), _dptr(sigma), int(nrhs), int(precision), int(arm),
                               _dptr(workspace), ws_bytes, _stream(stream)), "fock_apply_H")
    return sigma


def fock_apply_check(sp, ham, workspace=None, noalloc: bool = False, stream=None) -> int:
    """Status of the last apply that ran the tensor-core phase 1 with this
    workspace (None: the Hamiltonian's own; noalloc: the fixed array):
    FOCK_OK or FOCK_ERR_TIMEOUT.  Waits on the stream."""
    st = load().fock_apply_check(sp, ham, _dptr(workspace), int(bool(noalloc)), _stream(stream))
    _check(st, "fock_apply_check", allow=(FOCK_ERR_TIMEOUT,))
    return st


def fock_debug_set_wait_polls(polls: int) -> None:
    """Test hook: poll budget of phase 1's bounded waits (< 0: default, 0: give up at once)."""
    _check(load().fock_debug_set_wait_polls(int(polls)), "fock_debug_set_wait_polls")


def fock_apply_H_host(sp, ham, C_host, sigma_host, nrhs: int = 1, precision: int = FOCK_PREC_F64,
                      arm: int = FOCK_ARM_AUTO, stream=None):
    """Host-buffer variant: C_host and sigma_host are CPU tensors (pinned for speed)."""
    _check(load().fock_apply_H_host(sp, ham, ctypes.c_void_p(C_host.data_ptr()),
                                    ctypes.c_void_p(sigma_host.data_ptr()), int(nrhs), int(precision),
                                    int(arm), _stream(stream)), "fock_apply_H_host")
    return sigma_host


def fock_apply_H_noalloc(sp, ham, C, sigma=None, nrhs: int = 1, arm: int = FOCK_ARM_AUTO,
                         stream=None, check: bool = True):
    """FP64-class sigma = H C with the library's fixed scratch instead of an
    allocation (for callers whose device memory is managed elsewhere).
    Returns (sigma, status)."""
    import torch
    if sigma is None:
        sigma = torch.empty_like(C)
    st = load().fock_apply_H_noalloc(sp, ham, _dptr(C), _dptr(sigma), int(nrhs), int(arm),
                                     _stream(stream))
    if check:
        _check(st, "fock_apply_H_noalloc")
    return sigma, st


def fock_lanczos_ground(sp, ham, max_iter: int = 300, restart_len: int = 30, tol: float = 1e-12,
                        seed: int = 1, precision: int = FOCK_PREC_F64, start=None, want_vector=False,
                        stream=None):
    """Returns (E0, residual, iterations, vector-or-None, status)."""
    import torch
    E0, res, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    vec = None
    if want_vector:
        vec = torch.empty(fock_space_size(sp), dtype=torch.complex128, device="cuda")
    st = load().fock_lanczos_ground(sp, ham, int(max_iter), int(restart_len), float(tol),
                                    ctypes.c_uint64(int(seed)), int(precision), _dptr(start),
                                    ctypes.byref(E0), ctypes.byref(res), _dptr(vec), ctypes.byref(it),
                                    _stream(stream))
    _check(st, "fock_lanczos_ground", allow=(FOCK_ERR_NOCONV,))
    return E0.value, res.value, it.value, vec, st


def fock_sil_step(sp, ham, C, dt: float, max_krylov: int = 30, tol: float = 1e-12,
                  precision: int = FOCK_PREC_F64, stream=None):
    """C <- exp(-i H dt) C in place (complex128 CUDA vector); returns
    (krylov dimension, error estimate, status)."""
    m, err = ctypes.c_int32(), ctypes.c_double()
    st = load().fock_sil_step(sp, ham, _dptr(C), float(dt), int(max_krylov), float(tol), int(precision),
                              ctypes.byref(m), ctypes.byref(err), _stream(stream))
    _check(st, "fock_sil_step", allow=(FOCK_ERR_NOCONV,))
    return m.value, err.value, st


def fock_density_matrices(sp, C, M: int, want_rho2: bool = True, stream=None):
    """(rho1 [M, M], rho2 [M, M, M, M] or None) of the complex128 CUDA vector C
    as numpy complex128 arrays: rho1[k, l] = <C|a^dag_k a_l|C>,
    rho2[k, l, q, s] = <C|a^dag_k a^dag_l a_q a_s|C>."""
    import numpy as np
    r1 = np.zeros((M, M), dtype=np.complex128)
    r2 = np.zeros((M, M, M, M), dtype=np.complex128) if want_rho2 else None
    _check(load().fock_density_matrices(sp, _dptr(C), r1.ctypes.data,
                                        None if r2 is None else r2.ctypes.data, _stream(stream)),
           "fock_density_matrices")
    return r1, r2


# --------------------------------------------------------------------------
# convenience wrappers (own the handles)
# --------------------------------------------------------------------------
class Space:
    def __init__(self, N: int, M: int):
        self.N, self.M = int(N), int(M)
        self.handle = fock_space_create(N, M)
        self.nc = fock_space_size(self.handle)

    def close(self):
        if self.handle:
            fock_space_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hamiltonian:
    def __init__(self, space: Space, h, W=None, tol: float = 1e-12):
        self.space = space
        self.handle = fock_hamiltonian_create(space.handle, h, W, tol)
        self.terms = fock_hamiltonian_terms(self.handle)
        self.real = fock_hamiltonian_is_real(self.handle)
        self.forms = fock_hamiltonian_forms(self.handle)

    def apply(self, C, sigma=None, nrhs=1, precision=FOCK_PREC_F64, arm=FOCK_ARM_AUTO, workspace=None):
        return fock_apply_H(self.space.handle, self.handle, C, sigma, nrhs, precision, arm, workspace)

    def close(self):
        if self.handle:
            fock_hamiltonian_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# sectors of fixed total orbital weight (total momentum)
# --------------------------------------------------------------------------
def fock_sector_create(sp, Q: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().fock_sector_create(sp, int(Q), ctypes.byref(h)), "fock_sector_create")
    return h


def fock_sector_destroy(sec) -> None:
    load().fock_sector_destroy(sec)


def fock_sector_size(sec) -> int:
    n = ctypes.c_int64()
    _check(load().fock_sector_size(sec, ctypes.byref(n)), "fock_sector_size")
    return n.value


def fock_sector_rank(sec, occ, idx=None, stream=None, check: bool = True):
    """occ: int32 CUDA tensor [count, M]; returns (int64 sector indices, status)."""
    import torch
    if idx is None:
        idx = torch.empty(occ.shape[0], dtype=torch.int64, device=occ.device)
    st = load().fock_sector_rank(sec, _dptr(occ), occ.shape[0], _dptr(idx), _stream(stream))
    if check:
        _check(st, "fock_sector_rank")
    return idx, st


def fock_sector_unrank(sec, idx, M: int, occ=None, stream=None, check: bool = True):
    """idx: int64 CUDA tensor [count]; returns (int32 occupations [count, M], status)."""
    import torch
    if occ is None:
        occ = torch.empty((idx.shape[0], M), dtype=torch.int32, device=idx.device)
    st = load().fock_sector_unrank(sec, _dptr(idx), idx.shape[0], _dptr(occ), _stream(stream))
    if check:
        _check(st, "fock_sector_unrank")
    return occ, st


def fock_sector_terms(sec, ham) -> int:
    n = ctypes.c_int64()
    _check(load().fock_sector_terms(sec, ham, ctypes.byref(n)), "fock_sector_terms")
    return n.value


def fock_sector_workspace_size(sec, nrhs: int, precision: int) -> int:
    b = ctypes.c_size_t()
    _check(load().fock_sector_workspace_size(sec, int(nrhs), int(precision), ctypes.byref(b)),
           "fock_sector_workspace_size")
    return b.value


def fock_sector_apply_H(sec, ham, C, sigma=None, nrhs: int = 1, precision: int = FOCK_PREC_F64,
                        workspace=None, stream=None):
    """sigma = H C within the sector (C: CUDA tensor [N_sec] or [N_sec, nrhs])."""
    import torch
    if sigma is None:
        sigma = torch.empty_like(C)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load().fock_sector_apply_H(sec, ham, _dptr(C), _dptr(sigma), int(nrhs), int(precision),
                                      _dptr(workspace), ws_bytes, _stream(stream)), "fock_sector_apply_H")
    return sigma


def fock_sector_lanczos_ground(sec, ham, max_iter: int = 300, restart_len: int = 30, tol: float = 1e-12,
                               seed: int = 1, precision: int = FOCK_PREC_F64, start=None,
                               want_vector=False, stream=None):
    """Returns (E0, residual, iterations, vector-or-None, status)."""
    import torch
    E0, res, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    vec = None
    if want_vector:
        vec = torch.empty(fock_sector_size(sec), dtype=torch.complex128, device="cuda")
    st = load().fock_sector_lanczos_ground(sec, ham, int(max_iter), int(restart_len), float(tol),
                                           ctypes.c_uint64(int(seed)), int(precision), _dptr(start),
                                           ctypes.byref(E0), ctypes.byref(res), _dptr(vec), ctypes.byref(it),
                                           _stream(stream))
    _check(st, "fock_sector_lanczos_ground", allow=(FOCK_ERR_NOCONV,))
    return E0.value, res.value, it.value, vec, st


class Sector:
    """The configurations of `space` with sum_i i n_i = Q."""

    def __init__(self, space: Space, Q: int):
        self.space, self.Q = space, int(Q)
        self.handle = fock_sector_create(space.handle, Q)
        self.size = fock_sector_size(self.handle)

    def apply(self, ham: Hamiltonian, C, sigma=None, nrhs=1, precision=FOCK_PREC_F64, workspace=None):
        return fock_sector_apply_H(self.handle, ham.handle, C, sigma, nrhs, precision, workspace)

    def close(self):
        if self.handle:
            fock_sector_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# uneven batches
# --------------------------------------------------------------------------
class Batch:
    """Independent problems [(N, M, h, W), ...] applied and solved together."""

    def __init__(self, problems, tol: float = 1e-12):
        self.count = len(problems)
        Ns = np.array([p[0] for p in problems], dtype=np.int32)
        Ms = np.array([p[1] for p in problems], dtype=np.int32)
        self._h = [np.ascontiguousarray(np.asarray(p[2], dtype=np.complex128).reshape(-1)) for p in problems]
        self._W = [None if p[3] is None else np.ascontiguousarray(np.asarray(p[3], dtype=np.complex128).reshape(-1))
                   for p in problems]
        hp = (ctypes.c_void_p * self.count)(*[a.ctypes.data for a in self._h])
        Wp = (ctypes.c_void_p * self.count)(*[None if a is None else a.ctypes.data for a in self._W])
        self.handle = ctypes.c_void_p()
        _check(load().fock_batch_create(self.count, Ns.ctypes.data_as(ctypes.c_void_p),
                                        Ms.ctypes.data_as(ctypes.c_void_p), hp, Wp, float(tol),
                                        ctypes.byref(self.handle)), "fock_batch_create")
        off = np.zeros(self.count + 1, dtype=np.int64)
        _check(load().fock_batch_offsets(self.handle, off.ctypes.data_as(ctypes.c_void_p)), "fock_batch_offsets")
        self.offsets = off
        self.total = int(off[-1])
        t = ctypes.c_int64()
        _check(load().fock_batch_terms(self.handle, ctypes.byref(t)), "fock_batch_terms")
        self.terms = t.value
        own = np.zeros(self.count, dtype=np.int32)
        _check(load().fock_batch_own_apply(self.handle, own.ctypes.data_as(ctypes.c_void_p)), "fock_batch_own_apply")
        self.own = own.astype(bool)     # instances with an apply of their own

    def apply(self, C, sigma=None, precision=FOCK_PREC_F64, stream=None):
        import torch
        if sigma is None:
            sigma = torch.empty_like(C)
        _check(load().fock_batch_apply(self.handle, _dptr(C), _dptr(sigma), int(precision), _stream(stream)),
               "fock_batch_apply")
        return sigma

    def autotune(self, C, sigma, precision=FOCK_PREC_F64, cache_path=None, stream=None):
        t, b = ctypes.c_int32(), ctypes.c_int32()
        _check(load().fock_batch_autotune(self.handle, _dptr(C), _dptr(sigma), int(precision),
                                          None if cache_path is None else str(cache_path).encode(),
                                          ctypes.byref(t), ctypes.byref(b), _stream(stream)), "fock_batch_autotune")
        return t.value, b.value

    def lanczos_ground(self, max_iter=300, restart_len=12, tol=1e-10, seed=1, stream=None):
        E = np.zeros(self.count)
        R = np.zeros(self.count)
        it = np.zeros(self.count, dtype=np.int32)
        st = load().fock_batch_lanczos_ground(self.handle, int(max_iter), int(restart_len), float(tol),
                                              ctypes.c_uint64(int(seed)), E.ctypes.data_as(ctypes.c_void_p),
                                              R.ctypes.data_as(ctypes.c_void_p), it.ctypes.data_as(ctypes.c_void_p),
                                              _stream(stream))
        _check(st, "fock_batch_lanczos_ground", allow=(FOCK_ERR_NOCONV,))
        return E, R, it, st

    def close(self):
        if self.handle:
            load().fock_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
