"""Thin Python binding of the C ABI (argument marshalling only).

Every function here has the name of the C entry point it calls and passes
device pointers of torch tensors (or host numpy arrays where the C ABI takes
host memory).  All arithmetic of the method runs in the CUDA library; when
the library is missing, :func:`_capi.load` raises and nothing falls back.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _capi
from ._capi import (IFCI_BF16, IFCI_ERR_NOT_CONVERGED, IFCI_FP32, IFCI_FP64, IFCI_FP64E, IFCI_OK, IFCI_SCREENED,  # noqa: F401
                    IFCI_TF32)

PRECISIONS = {"fp64": IFCI_FP64, "fp32": IFCI_FP32, "tf32": IFCI_TF32, "bf16": IFCI_BF16, "fp64e": IFCI_FP64E}


class IfciError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ifci error {code}: {msg}")
        self.code = code


def _lib():
    return _capi.load()


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t: Optional[torch.Tensor]) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


class Handle:
    """Owns an ``ifci_handle_t`` (device binding and workspace)."""

    def __init__(self, workspace_bytes: int = 0, device: int = 0):
        self._h = ctypes.c_void_p()
        rc = _lib().ifci_handle_create(ctypes.byref(self._h), workspace_bytes, device)
        if rc != IFCI_OK:
            raise IfciError(rc, f"ifci_handle_create(device={device}) failed")
        self.device = device

    @property
    def ptr(self):
        return self._h

    def check(self, rc: int, allow=()):
        if rc != IFCI_OK and rc not in allow:
            msg = _lib().ifci_last_error_string(self._h).decode(errors="replace")
            raise IfciError(rc, msg)
        return rc

    def launches(self) -> int:
        return int(_lib().ifci_kernel_launches(self._h))

    def workspace_bytes(self) -> int:
        return int(_lib().ifci_workspace_bytes(self._h))

    def profile_enable(self, on: bool = True):
        self.check(_lib().ifci_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """{class: (milliseconds, launches)} of the per-kernel-class event timing."""
        out = {}
        for name, k in _capi.PROFILE_KINDS.items():
            ms, n = ctypes.c_double(), ctypes.c_longlong()
            self.check(_lib().ifci_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    def close(self):
        if self._h:
            _lib().ifci_handle_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- strings

def ifci_string_counts(norb: int, nelec_spin: int):
    ns, ne = ctypes.c_int(), ctypes.c_int()
    rc = _lib().ifci_string_counts(norb, nelec_spin, ctypes.byref(ns), ctypes.byref(ne))
    if rc != IFCI_OK:
        raise IfciError(rc, f"ifci_string_counts({norb}, {nelec_spin})")
    return ns.value, ne.value


@dataclass
class StringTables:
    norb: int
    nelec_spin: int
    nstr: int
    nexc: int
    strings: torch.Tensor       # int64 view of uint64 masks
    exc: torch.Tensor           # int32
    cstruct: _capi.Strings = field(default=None, repr=False)

    def as_c(self):
        if self.cstruct is None:
            self.cstruct = _capi.Strings(self.norb, self.nelec_spin, self.nstr, self.nexc,
                                         self.strings.data_ptr(), self.exc.data_ptr())
        return ctypes.byref(self.cstruct)


def ifci_build_strings(handle: Handle, norb: int, nelec_spin: int, stream=None, device=None) -> StringTables:
    nstr, nexc = ifci_string_counts(norb, nelec_spin)
    dev = device or torch.device("cuda", handle.device)
    strings = torch.empty(nstr, dtype=torch.int64, device=dev)
    exc = torch.empty(nstr * nexc, dtype=torch.int32, device=dev)
    handle.check(_lib().ifci_build_strings(handle.ptr, norb, nelec_spin, _ptr(strings), _ptr(exc), _stream(stream)))
    return StringTables(norb, nelec_spin, nstr, nexc, strings, exc)


# ---------------------------------------------------------------- one CI space

def ifci_sigma(handle: Handle, tables: StringTables, h1: torch.Tensor, eri: torch.Tensor, c: torch.Tensor,
               sigma: Optional[torch.Tensor] = None, precision: int = IFCI_FP64, stream=None,
               spin_symmetric: bool = False) -> torch.Tensor:
    """sigma = H c.  ``spin_symmetric``: the caller asserts c[Ia][Ib] = c[Ib][Ia];
    the tensor-core precisions then take the alpha-only gather."""
    if sigma is None:
        sigma = torch.empty_like(c)
    prec = int(precision) | (_capi.IFCI_SIGMA_SPIN_SYMMETRIC if spin_symmetric else 0)
    handle.check(_lib().ifci_sigma(handle.ptr, tables.as_c(), _ptr(h1), _ptr(eri), _ptr(c), _ptr(sigma),
                                   prec, _stream(stream)))
    return sigma


def ifci_sigma_noalloc(tables: StringTables, h1: torch.Tensor, eri: torch.Tensor, c: torch.Tensor,
                       sigma: torch.Tensor, stream=None) -> int:
    """FP64 sigma into a caller-provided ``sigma`` with no device allocation by
    the library (fixed scratch array).  Returns the C status code."""
    return int(_lib().ifci_sigma_noalloc(tables.as_c(), _ptr(h1), _ptr(eri), _ptr(c), _ptr(sigma),
                                         _stream(stream)))


def ifci_sigma_noalloc_max_bytes() -> int:
    return int(_lib().ifci_sigma_noalloc_max_bytes())


def ifci_wait_selftest(handle: Handle, limit_cycles: int, stream=None) -> int:
    """Runs out one bounded device wait on purpose; returns the C status
    (IFCI_ERR_TIMEOUT expected)."""
    return int(_lib().ifci_wait_selftest(handle.ptr, int(limit_cycles), _stream(stream)))


def ifci_h_elements(handle: Handle, tables: StringTables, h1: torch.Tensor, eri: torch.Tensor,
                    bra: torch.Tensor, ket: torch.Tensor, stream=None) -> torch.Tensor:
    """<I|H|J> for int64 determinant index pairs (device tensors)."""
    bra = bra.to(torch.int64).contiguous()
    ket = ket.to(torch.int64).contiguous()
    out = torch.empty(bra.numel(), dtype=torch.float64, device=bra.device)
    handle.check(_lib().ifci_h_elements(handle.ptr, tables.as_c(), _ptr(h1), _ptr(eri), int(bra.numel()),
                                        _ptr(bra), _ptr(ket), _ptr(out), _stream(stream)))
    return out


def ifci_hdiag(handle: Handle, tables: StringTables, h1: torch.Tensor, eri: torch.Tensor,
               hd: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    if hd is None:
        hd = torch.empty(tables.nstr * tables.nstr, dtype=torch.float64, device=h1.device)
    handle.check(_lib().ifci_hdiag(handle.ptr, tables.as_c(), _ptr(h1), _ptr(eri), _ptr(hd), _stream(stream)))
    return hd


# ---------------------------------------------------------------- systems

class SystemArrays:
    """Marshals an iFCI system (bodies + integrals) into ``ifci_system_t``.

    h: (norb, norb) float64, eri: (npair, npair) float64 packed (pq|rs); both
    either CUDA tensors or host numpy arrays (``on_host``).
    """

    def __init__(self, body_offset: Sequence[int], h, eri):
        self.body_offset = np.ascontiguousarray(body_offset, dtype=np.int32)
        self.nbody = len(self.body_offset) - 1
        self.norb = int(self.body_offset[-1])
        self.on_host = not (isinstance(h, torch.Tensor) and h.is_cuda)
        if self.on_host:
            self.h = np.ascontiguousarray(h, dtype=np.float64)
            self.eri = np.ascontiguousarray(eri, dtype=np.float64)
            hp, ep = self.h.ctypes.data, self.eri.ctypes.data
        else:
            self.h = h.contiguous()
            self.eri = eri.contiguous()
            assert self.h.dtype == torch.float64 and self.eri.dtype == torch.float64
            hp, ep = self.h.data_ptr(), self.eri.data_ptr()
        npair = self.norb * (self.norb + 1) // 2
        assert tuple(self.h.shape) == (self.norb, self.norb) and tuple(self.eri.shape) == (npair, npair)
        self.c = _capi.System(self.nbody, self.body_offset.ctypes.data_as(_capi.c_int_p), self.norb, hp, ep,
                              1 if self.on_host else 0)

    def as_c(self):
        return ctypes.byref(self.c)


def ifci_frozen_core(handle: Handle, system: SystemArrays, bodies: Sequence[int], stream=None):
    """(h1 (nA, nA), eri_x (npA, npA), e_core) of the CI problem of body set ``bodies``."""
    bodies = sorted(bodies)
    nA = sum(int(system.body_offset[b + 1] - system.body_offset[b]) for b in bodies)
    npA = nA * (nA + 1) // 2
    dev = torch.device("cuda", handle.device)
    h1 = torch.empty((nA, nA), dtype=torch.float64, device=dev)
    eri = torch.empty((npA, npA), dtype=torch.float64, device=dev)
    ec = ctypes.c_double()
    arr = (ctypes.c_int * len(bodies))(*bodies)
    handle.check(_lib().ifci_frozen_core(handle.ptr, system.as_c(), len(bodies), arr, _ptr(h1), _ptr(eri),
                                         ctypes.byref(ec), _stream(stream)))
    return h1, eri, ec.value


# ---------------------------------------------------------------- Davidson / increments

def davidson_opts(precision=IFCI_FP64, **kw) -> _capi.DavidsonOpts:
    o = _capi.DavidsonOpts()
    _lib().ifci_davidson_default_opts(ctypes.byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    for k, v in kw.items():
        if k == "hi_precision" and isinstance(v, str):
            v = PRECISIONS[v]
        setattr(o, k, v)
    return o


@dataclass
class CIProblem:
    norb: int
    nelec_spin: int
    h1: torch.Tensor
    eri: torch.Tensor
    e_core: float = 0.0
    c_out: Optional[torch.Tensor] = None


def ifci_davidson_batched(handle: Handle, problems: List[CIProblem], opts=None, stream=None, allow_unconverged=False):
    n = len(problems)
    arr = (_capi.Problem * max(n, 1))()
    for i, p in enumerate(problems):
        arr[i] = _capi.Problem(p.norb, p.nelec_spin, p.h1.data_ptr(), p.eri.data_ptr(), float(p.e_core),
                               p.c_out.data_ptr() if p.c_out is not None else None)
    e = np.zeros(n)
    it = np.zeros(n, dtype=np.int32)
    st = np.zeros(n, dtype=np.int32)
    o = opts or davidson_opts()
    rc = _lib().ifci_davidson_batched(handle.ptr, n, arr, ctypes.byref(o), e.ctypes.data_as(_capi.c_double_p),
                                      it.ctypes.data_as(_capi.c_int_p), st.ctypes.data_as(_capi.c_int_p),
                                      _stream(stream))
    handle.check(rc, allow=(IFCI_ERR_NOT_CONVERGED,) if allow_unconverged else ())
    return e, it, st


def ifci_hbci_batched(handle: Handle, problems: List[CIProblem], start_dets, eps1: float = 1e-3, eps2: float = 1e-6,
                      max_rounds: int = 50, opts=None, stream=None, allow_unconverged=False):
    """Heat-bath selected CI + EN-PT2 per problem (include/ifci.h).  Returns a
    dict of e_var, e_pt2, e_hbci (= e_var + e_pt2), nsel, rounds, status."""
    n = len(problems)
    arr = (_capi.Problem * max(n, 1))()
    for i, p in enumerate(problems):
        arr[i] = _capi.Problem(p.norb, p.nelec_spin, p.h1.data_ptr(), p.eri.data_ptr(), float(p.e_core),
                               p.c_out.data_ptr() if p.c_out is not None else None)
    start = np.ascontiguousarray(np.asarray(start_dets, dtype=np.int64).reshape(-1))
    if start.size != n:
        raise ValueError("one start determinant per problem")
    ev, e2 = np.zeros(n), np.zeros(n)
    nsel = np.zeros(n, dtype=np.int64)
    rounds = np.zeros(n, dtype=np.int32)
    st = np.zeros(n, dtype=np.int32)
    o = opts or davidson_opts(IFCI_FP64E)
    hb = _capi.HbciOpts(float(eps1), float(eps2), int(max_rounds))
    rc = _lib().ifci_hbci_batched(handle.ptr, n, arr, start.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                  ctypes.byref(o), ctypes.byref(hb), ev.ctypes.data_as(_capi.c_double_p),
                                  e2.ctypes.data_as(_capi.c_double_p),
                                  nsel.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                  rounds.ctypes.data_as(_capi.c_int_p), st.ctypes.data_as(_capi.c_int_p),
                                  _stream(stream))
    handle.check(rc, allow=(IFCI_ERR_NOT_CONVERGED,) if allow_unconverged else ())
    return {"e_var": ev, "e_pt2": e2, "e_hbci": ev + e2, "nsel": nsel, "rounds": rounds, "status": st}


def reference_determinant(body_sizes, X) -> int:
    """Index I = Ia * nstr + Ia of the determinant with every bonding orbital of
    the body set X doubly occupied (each body's first orbital; X's orbitals in
    body order, strings ranked by increasing bit mask)."""
    import math
    X = sorted(X)
    bonding, off = [], 0
    for b in X:
        bonding.append(off)
        off += int(body_sizes[b])
    m = len(X)
    ra = sum(math.comb(p, k + 1) for k, p in enumerate(bonding))
    nstr = math.comb(off, m)
    return ra * nstr + ra


def ifci_num_subsets(nbody: int, max_order: int) -> int:
    c = ctypes.c_longlong()
    rc = _lib().ifci_num_subsets(nbody, max_order, ctypes.byref(c))
    if rc != IFCI_OK:
        raise IfciError(rc, "ifci_num_subsets")
    return c.value


def body_subsets(nbody: int, max_order: int):
    """Order of every per-set array: by size, then lexicographic (mirrors the C enumeration)."""
    import itertools
    out = []
    for k in range(1, max_order + 1):
        out.extend(itertools.combinations(range(nbody), k))
    return out


def ifci_increments(handle: Handle, system: SystemArrays, max_order: int, opts=None, stream=None,
                    allow_unconverged=False):
    ns = ifci_num_subsets(system.nbody, max_order)
    e0, tot = ctypes.c_double(), ctypes.c_double()
    ex = np.zeros(ns)
    eps = np.zeros(ns)
    st = np.zeros(ns, dtype=np.int32)
    it = np.zeros(ns, dtype=np.int32)
    o = opts or davidson_opts()
    rc = _lib().ifci_increments(handle.ptr, system.as_c(), max_order, ctypes.byref(o), ctypes.byref(e0),
                                ex.ctypes.data_as(_capi.c_double_p), eps.ctypes.data_as(_capi.c_double_p),
                                ctypes.byref(tot), it.ctypes.data_as(_capi.c_int_p),
                                st.ctypes.data_as(_capi.c_int_p), _stream(stream))
    handle.check(rc, allow=(IFCI_ERR_NOT_CONVERGED,) if allow_unconverged else ())
    return {"e0": e0.value, "e_x": ex, "eps": eps, "e_total": tot.value, "iters": it, "status": st}


def ifci_rdm_backward(handle: Handle, system: SystemArrays, max_order: int, grad_out: float = 1.0, opts=None,
                      recompute_vectors: bool = False, stream=None):
    dev = torch.device("cuda", handle.device)
    n = system.norb
    npair = n * (n + 1) // 2
    dh = torch.empty((n, n), dtype=torch.float64, device=dev)
    deri = torch.empty((npair, npair), dtype=torch.float64, device=dev)
    o = opts or davidson_opts()
    handle.check(_lib().ifci_rdm_backward(handle.ptr, system.as_c(), max_order, ctypes.byref(o), float(grad_out),
                                          _ptr(dh), _ptr(deri), 1 if recompute_vectors else 0, _stream(stream)))
    return dh, deri


# ---------------------------------------------------------------- autograd

class IfciEnergy(torch.autograd.Function):
    """E_iFCI(h, V) with its gradient from ifci_rdm_backward.

    forward(h (norb, norb) CUDA float64, V (npair, npair) CUDA float64, body_offset,
    max_order, handle, opts) -> 0-d float64 tensor on h's device.  The
    backward reuses the CI vectors the forward call kept in the handle; the
    gradient with respect to the symmetric parameter V[A][B] = V[B][A] is the
    sum of the two returned entries (see ifci_rdm_backward).
    """

    @staticmethod
    def forward(ctx, h, V, body_offset, max_order, handle, opts=None):
        sysd = SystemArrays(body_offset, h.detach(), V.detach())
        out = ifci_increments(handle, sysd, max_order, opts)
        ctx.state = (sysd, max_order, handle, opts)
        return torch.tensor(out["e_total"], dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(ctx, grad):
        sysd, max_order, handle, opts = ctx.state
        dh, dV = ifci_rdm_backward(handle, sysd, max_order, float(grad), opts, recompute_vectors=False)
        return dh, dV, None, None, None, None


def ifci_energy(h, V, body_offset, max_order, handle, opts=None):
    """Differentiable E_iFCI (see IfciEnergy)."""
    return IfciEnergy.apply(h, V, body_offset, max_order, handle, opts)
