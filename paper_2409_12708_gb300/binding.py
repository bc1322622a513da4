"""Python binding of the C ABI in include/thc.h (ctypes; argument marshalling only).

Every numerical step runs inside libthc.so's CUDA kernels.  PyTorch supplies
device memory (its caching allocator is handed to the library as the
thc_allocator callbacks), the current CUDA stream, and the tensors that hold
site tensors.  There is no CPU fallback: if the library is missing, importing
this module raises.

An MPS is a list of L CUDA tensors, site i of shape [chi_i, 4, chi_{i+1}]
(float64 or complex128 for path "fp64", float32 or complex64 for paths "fp32"
and "tf32"; "tf32" runs the compression's contractions on the tensor cores).
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libthc.so")

MAX_SITES = 64
OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EBREAKDOWN, EUNSUPPORTED = range(8)
F64, F32, C64, C128 = range(4)
PATH_FP64, PATH_FP32, PATH_TF32 = 0, 1, 2
_PATHS = {"fp64": PATH_FP64, "fp32": PATH_FP32, "tf32": PATH_TF32}
_DT = {PATH_FP64: (F64, torch.float64), PATH_FP32: (F32, torch.float32), PATH_TF32: (F32, torch.float32)}
_TORCH_OF = {F64: torch.float64, F32: torch.float32, C64: torch.complex64, C128: torch.complex128}
_TYPESTR = {F64: "<f8", F32: "<f4", C64: "<c8", C128: "<c16"}


class ThcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"thc status {status}: {msg}")
        self.status = status


class thc_mps(C.Structure):
    _fields_ = [("L", C.c_int), ("d", C.c_int), ("dtype", C.c_int),
                ("bond", C.c_int * (MAX_SITES + 1)), ("site", C.c_void_p * MAX_SITES),
                ("owner", C.c_void_p)]


class thc_hamiltonian(C.Structure):
    _fields_ = [("L", C.c_int), ("N", C.c_int), ("t", C.c_void_p), ("chi", C.c_void_p),
                ("zeta", C.c_void_p)]


class thc_opts(C.Structure):
    _fields_ = [("D_max", C.c_int), ("tol", C.c_double), ("path", C.c_int),
                ("term_begin", C.c_long), ("term_end", C.c_long), ("batch", C.c_int),
                ("chunk", C.c_int), ("merge_spin", C.c_int)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class thc_allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", C.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    sig = {
        "thc_apply_H": [P(thc_hamiltonian), P(thc_mps), P(thc_opts), P(thc_mps), P(thc_allocator), C.c_void_p],
        "thc_layer_apply": [P(thc_mps), C.c_void_p, C.c_int, C.c_int, P(thc_opts), P(thc_mps),
                            P(thc_allocator), C.c_void_p],
        "thc_compress": [P(thc_mps), P(thc_opts), P(thc_mps), P(thc_allocator), C.c_void_p],
        "mps_inner": [P(thc_mps), P(thc_mps), P(C.c_double), P(C.c_double), C.c_void_p],
        "mps_add_compress": [C.c_int, P(C.c_double), P(C.c_double), P(P(thc_mps)), P(thc_opts),
                             P(thc_mps), P(thc_allocator), C.c_void_p],
        "krylov_lanczos_ground": [P(thc_hamiltonian), P(thc_mps), C.c_int, P(thc_opts), P(C.c_double),
                                  P(C.c_double), P(thc_mps), P(thc_allocator), C.c_void_p],
        "krylov_lanczos_restarted": [P(thc_hamiltonian), P(thc_mps), C.c_int, C.c_int, C.c_int,
                                     P(P(thc_mps)), P(thc_opts), P(C.c_double), P(thc_mps), P(thc_allocator),
                                     C.c_void_p],
        "krylov_expm_apply": [P(thc_hamiltonian), P(thc_mps), C.c_double, C.c_int, P(thc_opts),
                              P(thc_mps), P(C.c_double), P(thc_allocator), C.c_void_p],
        "thc_kinetic_factors": [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
        "mps_inner_noalloc": [P(thc_mps), P(thc_mps), P(C.c_double), C.c_void_p],
        "thc_apply_H_batched": [C.c_int, P(P(thc_hamiltonian)), P(P(thc_mps)), P(thc_opts), P(thc_mps),
                                P(thc_allocator), C.c_void_p],
        "thc_expect_grad": [P(thc_hamiltonian), P(thc_mps), P(thc_mps), P(thc_opts), P(C.c_double), C.c_void_p,
                            C.c_void_p, C.c_void_p, P(thc_mps), P(thc_allocator), C.c_void_p],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.thc_mps_free.argtypes = [P(thc_mps), P(thc_allocator), C.c_void_p]
    lib.thc_mps_free.restype = None
    lib.thc_last_error.restype = C.c_char_p
    lib.thc_build_info.restype = C.c_char_p
    lib.thc_kernel_launches.restype = C.c_ulonglong
    lib.thc_profile_enable.argtypes = [C.c_int]
    lib.thc_profile_enable.restype = None
    lib.thc_profile_read.argtypes = [C.c_char_p, C.c_int]
    lib.thc_profile_read.restype = C.c_int
    return lib


LIB = _load()

# the declared entry points of include/thc.h (checked by the CPU tests)
EXPORTED = ("thc_apply_H", "thc_layer_apply", "thc_compress", "mps_inner", "mps_add_compress",
            "krylov_lanczos_ground", "krylov_expm_apply", "thc_kinetic_factors", "thc_mps_free",
            "thc_last_error", "thc_build_info", "thc_kernel_launches", "thc_profile_enable",
            "thc_profile_read", "mps_inner_noalloc", "krylov_lanczos_restarted", "thc_expect_grad",
            "thc_apply_H_batched")


# --------------------------------------------------------------------- allocator
def _torch_alloc(size, stream, ctx):
    try:
        return torch.cuda.caching_allocator_alloc(int(size), stream=int(stream or 0))
    except Exception:  # out of memory: the library turns NULL into THC_ENOMEM
        return None


def _torch_free(ptr, stream, ctx):
    if ptr:
        torch.cuda.caching_allocator_delete(ptr)


_ALLOC_CB = _ALLOC_FN(_torch_alloc)
_FREE_CB = _FREE_FN(_torch_free)
TORCH_ALLOCATOR = thc_allocator(_ALLOC_CB, _FREE_CB, None)


def make_allocator(alloc, free):
    """A thc_allocator from two Python callables: alloc(bytes, stream) -> int
    device pointer or None (failure), free(ptr, stream).  The returned object
    keeps its C callbacks alive."""
    a = _ALLOC_FN(lambda size, stream, ctx: alloc(int(size), stream))
    f = _FREE_FN(lambda ptr, stream, ctx: free(ptr, stream))
    out = thc_allocator(a, f, None)
    out._keep = (a, f)
    return out


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(status):
    if status != OK:
        raise ThcError(status, LIB.thc_last_error().decode())


# --------------------------------------------------------------------- marshalling
_CODE_OF = {torch.float64: F64, torch.float32: F32, torch.complex64: C64, torch.complex128: C128}


def _desc(sites, dtype_code=None):
    # the dtype code always describes the tensors; the library checks it
    # against the requested compute path
    m = thc_mps()
    m.L = len(sites)
    m.d = 4
    m.dtype = _CODE_OF.get(sites[0].dtype, -1)
    m.bond[0] = sites[0].shape[0]
    for i, s in enumerate(sites):
        if not (s.is_cuda and s.is_contiguous() and s.dim() == 3 and s.shape[1] == 4):
            raise ValueError("site tensors must be contiguous CUDA tensors [chi_l, 4, chi_r]")
        m.bond[i + 1] = s.shape[2]
        m.site[i] = s.data_ptr()
    m.owner = None
    return m


class _View:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


def _take(m):
    """Copy a library-owned output MPS into torch tensors and release the block."""
    typestr = _TYPESTR[m.dtype]
    out = []
    for i in range(m.L):
        shape = (m.bond[i], 4, m.bond[i + 1])
        out.append(torch.as_tensor(_View(m.site[i], shape, typestr), device="cuda").clone())
    LIB.thc_mps_free(C.byref(m), C.byref(TORCH_ALLOCATOR), _stream())
    return out


def _ham(t, chi, zeta):
    for x in (t, chi, zeta):
        if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
            raise ValueError("t, chi, zeta must be contiguous float64 CUDA tensors")
    h = thc_hamiltonian()
    h.L, h.N = chi.shape
    h.t, h.chi, h.zeta = t.data_ptr(), chi.data_ptr(), zeta.data_ptr()
    return h


def _opts(D_max, tol, path, term_begin=-1, term_end=-1, batch=0, chunk=0, merge_spin=False):
    return thc_opts(int(D_max), float(tol), _PATHS[path], int(term_begin), int(term_end), int(batch),
                    int(chunk), int(bool(merge_spin)))


def _code(path):
    return _DT[_PATHS[path]][0]


# --------------------------------------------------------------------- entry points
def thc_apply_H(t, chi, zeta, psi, D_max, tol=0.0, path="fp64", term_begin=-1, term_end=-1, batch=0,
                chunk=0, allocator=None, merge_spin=False):
    h = _ham(t, chi, zeta)
    d = _desc(psi, _code(path))
    o = _opts(D_max, tol, path, term_begin, term_end, batch, chunk, merge_spin)
    out = thc_mps()
    al = allocator if allocator is not None else TORCH_ALLOCATOR
    try:
        _check(LIB.thc_apply_H(C.byref(h), C.byref(d), C.byref(o), C.byref(out), C.byref(al), _stream()))
    except ThcError as e:
        e.out_owner = out.owner  # what the failed call left in the output descriptor
        raise
    return _take(out)


def thc_apply_H_batched(hams, psis, D_max, tol=0.0, path="fp64", batch=0):
    """H_i|psi_i> for independent instances (hams: list of (t, chi, zeta)),
    run concurrently on their own streams; returns the list of outputs."""
    n = len(psis)
    hs = [_ham(*h) for h in hams]
    ds = [_desc(p) for p in psis]
    harr = (C.POINTER(thc_hamiltonian) * n)(*[C.pointer(h) for h in hs])
    parr = (C.POINTER(thc_mps) * n)(*[C.pointer(d) for d in ds])
    outs = (thc_mps * n)()
    o = _opts(D_max, tol, path, batch=batch)
    _check(LIB.thc_apply_H_batched(n, harr, parr, C.byref(o), outs, C.byref(TORCH_ALLOCATOR), _stream()))
    return [_take(outs[i]) for i in range(n)]


def thc_layer_apply(psi, coef, sigma, dagger, D_max, tol=0.0, path="fp64"):
    if not (coef.is_cuda and coef.dtype == torch.float64):
        raise ValueError("coef must be a float64 CUDA tensor")
    d = _desc(psi, _code(path))
    o = _opts(D_max, tol, path)
    out = thc_mps()
    _check(LIB.thc_layer_apply(C.byref(d), coef.data_ptr(), int(sigma), int(dagger), C.byref(o),
                               C.byref(out), C.byref(TORCH_ALLOCATOR), _stream()))
    return _take(out)


def thc_compress(psi, D_max, tol=0.0, path="fp64"):
    d = _desc(psi, _code(path))
    o = _opts(D_max, tol, path)
    out = thc_mps()
    _check(LIB.thc_compress(C.byref(d), C.byref(o), C.byref(out), C.byref(TORCH_ALLOCATOR), _stream()))
    return _take(out)


def mps_inner(phi, psi):
    """<phi|psi> (conjugating phi); a float for real MPS, a complex for complex MPS."""
    a, b = _desc(phi), _desc(psi)
    re, im = C.c_double(), C.c_double()
    _check(LIB.mps_inner(C.byref(a), C.byref(b), C.byref(re), C.byref(im), _stream()))
    return complex(re.value, im.value) if phi[0].is_complex() else re.value


def mps_inner_noalloc(phi, psi):
    """<phi|psi> through the entry point that allocates nothing (its scratch is a
    fixed 16 MiB device array shared by all calls; see include/thc.h)."""
    code = F64 if phi[0].dtype == torch.float64 else F32
    a, b = _desc(phi, code), _desc(psi, code)
    re = C.c_double()
    _check(LIB.mps_inner_noalloc(C.byref(a), C.byref(b), C.byref(re), _stream()))
    return re.value


def mps_add_compress(coeffs, xs, D_max, tol=0.0, path="fp64"):
    n = len(xs)
    descs = [_desc(x, _code(path)) for x in xs]
    arr = (C.POINTER(thc_mps) * n)(*[C.pointer(d) for d in descs])
    cre = (C.c_double * n)(*[complex(c).real for c in coeffs])
    cim = (C.c_double * n)(*[complex(c).imag for c in coeffs])
    o = _opts(D_max, tol, path)
    out = thc_mps()
    _check(LIB.mps_add_compress(n, cre, cim, arr, C.byref(o), C.byref(out), C.byref(TORCH_ALLOCATOR),
                                _stream()))
    return _take(out)


def krylov_lanczos_ground(t, chi, zeta, psi0, K, D_max, tol=0.0, path="fp64", want_ground=False, batch=0,
                          merge_spin=False):
    h = _ham(t, chi, zeta)
    d = _desc(psi0, _code(path))
    o = _opts(D_max, tol, path, batch=batch, merge_spin=merge_spin)
    e = C.c_double()
    ritz = (C.c_double * K)()
    g = thc_mps()
    _check(LIB.krylov_lanczos_ground(C.byref(h), C.byref(d), int(K), C.byref(o), C.byref(e), ritz,
                                     C.byref(g) if want_ground else None, C.byref(TORCH_ALLOCATOR),
                                     _stream()))
    ground = _take(g) if want_ground else None
    return e.value, [ritz[i] for i in range(K)], ground


def krylov_lanczos_restarted(t, chi, zeta, psi0, K, cycles, D_max, lower=(), tol=0.0, path="fp64",
                             want_state=False):
    """Restarted Lanczos (optionally orthogonal to `lower` states); returns
    (lowest Ritz value of every cycle, last Ritz vector or None)."""
    h = _ham(t, chi, zeta)
    d = _desc(psi0, _code(path))
    lows = [_desc(x, _code(path)) for x in lower]
    arr = (C.POINTER(thc_mps) * max(len(lows), 1))(*[C.pointer(x) for x in lows])
    o = _opts(D_max, tol, path)
    en = (C.c_double * cycles)()
    g = thc_mps()
    _check(LIB.krylov_lanczos_restarted(C.byref(h), C.byref(d), int(K), int(cycles), len(lows), arr, C.byref(o),
                                        en, C.byref(g) if want_state else None, C.byref(TORCH_ALLOCATOR),
                                        _stream()))
    return [en[i] for i in range(cycles)], (_take(g) if want_state else None)


def krylov_expm_apply(t, chi, zeta, psi, dt, K, D_max, tol=0.0, path="fp64"):
    """One Krylov time step; psi real or complex, the result complex
    (complex128 on path "fp64", complex64 on "fp32"); returns (psi(dt), lost_norm)."""
    h = _ham(t, chi, zeta)
    d = _desc(psi, _code(path))
    o = _opts(D_max, tol, path)
    out = thc_mps()
    lost = C.c_double()
    _check(LIB.krylov_expm_apply(C.byref(h), C.byref(d), float(dt), int(K), C.byref(o), C.byref(out),
                                 C.byref(lost), C.byref(TORCH_ALLOCATOR), _stream()))
    return _take(out), lost.value


def thc_expect_grad(t, chi, zeta, phi, psi, path="fp64", batch=0, grads=True, term_begin=-1, term_end=-1):
    """<phi|H|psi> (exact) and, with grads, (dE/dt, dE/dchi, dE/dzeta, dE/dpsi sites);
    with a term range, of the sum of those terms only."""
    h = _ham(t, chi, zeta)
    a, b = _desc(phi), _desc(psi)
    o = _opts(1, 0.0, path, term_begin, term_end, batch=batch)
    v = C.c_double()
    L, N = chi.shape
    if grads:
        dt = torch.empty(L, L, dtype=torch.float64, device=t.device)
        dchi = torch.empty(L, N, dtype=torch.float64, device=t.device)
        dz = torch.empty(N, N, dtype=torch.float64, device=t.device)
        g = thc_mps()
        _check(LIB.thc_expect_grad(C.byref(h), C.byref(a), C.byref(b), C.byref(o), C.byref(v), dt.data_ptr(),
                                   dchi.data_ptr(), dz.data_ptr(), C.byref(g), C.byref(TORCH_ALLOCATOR), _stream()))
        return v.value, dt, dchi, dz, _take(g)
    _check(LIB.thc_expect_grad(C.byref(h), C.byref(a), C.byref(b), C.byref(o), C.byref(v), None, None, None, None,
                               C.byref(TORCH_ALLOCATOR), _stream()))
    return v.value


class ThcExpectation(torch.autograd.Function):
    """E = <phi|H(t, chi, zeta)|psi> as a differentiable function of t, chi,
    zeta and the sites of psi (phi is held fixed).  The library computes E and
    all of its derivatives in one pass of environment sweeps (thc_expect_grad);
    backward scales them by the incoming gradient."""

    @staticmethod
    def forward(ctx, t, chi, zeta, n_phi, *sites):
        phi, psi = list(sites[:n_phi]), list(sites[n_phi:])
        path = "fp64" if psi[0].dtype == torch.float64 else "fp32"
        v, dt, dchi, dz, dpsi = thc_expect_grad(t.detach(), chi.detach(), zeta.detach(),
                                                [x.detach() for x in phi], [x.detach() for x in psi], path=path)
        ctx.n_phi = n_phi
        ctx.save_for_backward(dt, dchi, dz, *dpsi)
        return torch.tensor(v, dtype=torch.float64, device=t.device)

    @staticmethod
    def backward(ctx, g):
        dt, dchi, dz, *dpsi = ctx.saved_tensors
        return (g * dt, g * dchi, g * dz, None, *([None] * ctx.n_phi), *[g.to(x.dtype) * x for x in dpsi])


def expectation(t, chi, zeta, phi, psi):
    """Differentiable <phi|H|psi> (see ThcExpectation)."""
    return ThcExpectation.apply(t, chi, zeta, len(phi), *phi, *psi)


def thc_kinetic_factors(t):
    L = t.shape[0]
    lam = torch.empty(L, dtype=torch.float64, device=t.device)
    u = torch.empty(L, L, dtype=torch.float64, device=t.device)
    _check(LIB.thc_kinetic_factors(L, t.data_ptr(), lam.data_ptr(), u.data_ptr(), _stream()))
    return lam, u


def build_info():
    return LIB.thc_build_info().decode()


def kernel_launches():
    return int(LIB.thc_kernel_launches())


def profile_enable(on=True):
    LIB.thc_profile_enable(1 if on else 0)


def profile_read():
    import json
    buf = C.create_string_buffer(1 << 20)
    n = LIB.thc_profile_read(buf, len(buf))
    if n > len(buf):
        raise RuntimeError("profile text truncated")
    return json.loads(buf.value.decode())
