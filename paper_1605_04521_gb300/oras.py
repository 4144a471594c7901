"""ctypes binding of the C ABI declared in include/oras.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Arrays are numpy arrays
(host) or torch CUDA tensors (device, `mem=ORAS_MEM_DEVICE`); complex arrays are complex128.
The library must be built (paper_1605_04521_gb300.build.build()); there is no fallback: if
the shared object is missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboras_gb300.so")

ORAS_OK = 0
ORAS_NOT_CONVERGED = 1
ORAS_PENDING = 2
ORAS_ERR_INVALID_ARG = -1
ORAS_ERR_BAD_MESH = -2
ORAS_ERR_OUT_OF_MEMORY = -3
ORAS_ERR_SINGULAR_LOCAL = -4
ORAS_ERR_DEVICE_TIMEOUT = -5
ORAS_ERR_CUDA = -6
ORAS_ERR_REJECTED = -7
ORAS_ERR_UNSUPPORTED = -8
ORAS_ERR_STATE = -9
ORAS_MEM_HOST = 0
ORAS_MEM_DEVICE = 1
ORAS_WEIGHTS_POU = 0
ORAS_WEIGHTS_NONE = 1
ORAS_OVERLAP_VERTEX = 0
ORAS_OVERLAP_FACE = 1
ORAS_LU_AUTO = 0
ORAS_LU_CUDA_CORES = 1
ORAS_APPLY_AUTO = 0
ORAS_APPLY_CUDA_CORES = 1
ORAS_TRANSMISSION_IMPEDANCE = 0
ORAS_TRANSMISSION_DIRICHLET = 1
ORAS_FACE_IMPEDANCE = 0
ORAS_FACE_METALLIC = 1


class oras_complex(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class oras_problem(C.Structure):
    _fields_ = [("nv", C.c_int64), ("xyz", C.c_void_p), ("nt", C.c_int64), ("tets", C.c_void_p),
                ("eps_r", C.c_void_p), ("mu_r", C.c_void_p), ("k0", C.c_double), ("r", C.c_int32),
                ("nsub", C.c_int32), ("overlap", C.c_int32), ("part", C.c_void_p), ("beta_face", C.c_void_p),
                ("face_kind", C.c_void_p)]


class oras_port(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("u", C.c_double * 3), ("v", C.c_double * 3), ("beta", C.c_double)]


class oras_options(C.Structure):
    _fields_ = [("restart", C.c_int32), ("max_iter", C.c_int32), ("factor_bits", C.c_int32),
                ("weights", C.c_int32), ("overlap_kind", C.c_int32), ("lu_engine", C.c_int32),
                ("lu_panel", C.c_int32), ("lu_group", C.c_int32), ("transmission", C.c_int32),
                ("graphs", C.c_int32), ("wait_ms", C.c_int32), ("apply_engine", C.c_int32),
                ("block", C.c_int32), ("recycle", C.c_int32), ("reserved", C.c_int32 * 2)]


class oras_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("pad", C.c_int32), ("relres", C.c_double)]


class oras_server_config(C.Structure):
    _fields_ = [("hbm_budget", C.c_int64), ("device", C.c_int32), ("max_active", C.c_int32),
                ("planners", C.c_int32), ("reserved", C.c_int32 * 5)]


class oras_ticket(C.Structure):
    _fields_ = [("submit_s", C.c_double), ("planned_s", C.c_double), ("admitted_s", C.c_double),
                ("done_s", C.c_double), ("footprint", C.c_int64), ("ndof", C.c_int64), ("k", C.c_int32),
                ("status", C.c_int32)]


class oras_server_counters(C.Structure):
    _fields_ = [("hbm_budget", C.c_int64), ("hbm_in_use", C.c_int64), ("hbm_peak", C.c_int64),
                ("queued", C.c_int32), ("active", C.c_int32), ("peak_active", C.c_int32),
                ("completed", C.c_int32), ("rejected", C.c_int32), ("pad", C.c_int32)]


EXPORTS = {
    "oras_last_error": (C.c_char_p, [C.c_void_p]),
    "oras_abi_version": (C.c_int32, []),
    "oras_create": (C.c_int, [C.POINTER(oras_problem), C.POINTER(oras_options), C.POINTER(C.c_void_p)]),
    "oras_factor": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int32]),
    "oras_setup": (C.c_int, [C.POINTER(oras_problem), C.POINTER(oras_options), C.POINTER(C.c_void_p)]),
    "oras_destroy": (None, [C.c_void_p]),
    "oras_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "oras_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p,
                             C.POINTER(oras_info), C.c_int32]),
    "oras_rhs_plane_wave": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "oras_rhs_dipole": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "oras_port_vector": (C.c_int, [C.c_void_p, C.POINTER(oras_port), C.c_void_p, C.POINTER(C.c_double), C.c_int32]),
    "oras_rhs_port": (C.c_int, [C.c_void_p, C.POINTER(oras_port), C.c_void_p, C.c_int32]),
    "oras_s_matrix": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]),
    "oras_s_error": (C.c_double, [C.c_void_p, C.c_void_p, C.c_int64]),
    "oras_constrained_dofs": (C.c_int, [C.c_void_p, C.c_void_p]),
    "oras_dense_eig": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "oras_recycle_reset": (C.c_int, [C.c_void_p]),
    "oras_ndof": (C.c_int64, [C.c_void_p]),
    "oras_nlocal": (C.c_int32, [C.c_void_p]),
    "oras_nsub": (C.c_int32, [C.c_void_p]),
    "oras_dofmap": (C.c_int, [C.c_void_p, C.c_void_p]),
    "oras_partition": (C.c_int, [C.c_void_p, C.c_void_p]),
    "oras_subdomain_size": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64)]),
    "oras_subdomain": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "oras_nnz": (C.c_int64, [C.c_void_p]),
    "oras_arena_bytes": (C.c_int64, [C.c_void_p]),
    "oras_element_matrices": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "oras_global_csr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "oras_matvec": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]),
    "oras_precond": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]),
    "oras_matvec_c64": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]),
    "oras_timings": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "oras_set_timing": (C.c_int, [C.c_void_p, C.c_int32]),
    "oras_reset_timings": (C.c_int, [C.c_void_p]),
    "oras_launch_count": (C.c_int64, []),
    "oras_precond_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "oras_wait_selftest": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "oras_footprint": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]),
    "oras_release_memory": (C.c_int, [C.c_int32]),
    "oras_autotune": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_void_p, C.c_int32]),
    "oras_lu_group": (C.c_int32, [C.c_void_p]),
    "oras_server_create": (C.c_int, [C.POINTER(oras_server_config), C.POINTER(C.c_void_p)]),
    "oras_submit": (C.c_int64, [C.c_void_p, C.POINTER(oras_problem), C.POINTER(oras_options), C.c_void_p,
                                C.c_int64, C.c_void_p, C.c_int32, C.c_double]),
    "oras_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.POINTER(oras_info), C.c_int32]),
    "oras_ticket_info": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(oras_ticket)]),
    "oras_ticket_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32]),
    "oras_server_error": (C.c_char_p, [C.c_void_p, C.c_int64]),
    "oras_server_stats": (C.c_int, [C.c_void_p, C.POINTER(oras_server_counters)]),
    "oras_server_destroy": (None, [C.c_void_p]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1605_04521_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class OrasError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"oras error {code}: {msg}")
        self.code = code


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _check(h, rc, allow=(ORAS_OK,)):
    if rc in allow:
        return rc
    msg = lib.oras_last_error(h)
    raise OrasError(rc, msg.decode() if msg else "")


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _problem(xyz, tets, eps_r, mu_r, k0, r, nsub, overlap, part, beta_face=None, face_kind=None):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    keep = [xyz, tets]
    p = oras_problem()
    p.nv, p.xyz, p.nt, p.tets = xyz.shape[0], xyz.ctypes.data, tets.shape[0], tets.ctypes.data
    if eps_r is not None:
        e = _c128(eps_r)
        keep.append(e)
        p.eps_r = e.ctypes.data
    if mu_r is not None:
        m = _c128(mu_r)
        keep.append(m)
        p.mu_r = m.ctypes.data
    p.k0, p.r, p.nsub, p.overlap = float(k0), int(r), int(nsub), int(overlap)
    if part is not None:
        pa = np.ascontiguousarray(part, dtype=np.int32)
        keep.append(pa)
        p.part = pa.ctypes.data
    if beta_face is not None:
        bf = np.ascontiguousarray(beta_face, dtype=np.float64).reshape(-1, 4)
        keep.append(bf)
        p.beta_face = bf.ctypes.data
    if face_kind is not None:
        fk = np.ascontiguousarray(face_kind, dtype=np.uint8).reshape(-1, 4)
        keep.append(fk)
        p.face_kind = fk.ctypes.data
    return p, keep


def _options(restart=0, max_iter=0, factor_bits=0, weights=0, overlap_kind=0, lu_engine=0, lu_panel=0, lu_group=0,
             transmission=0, graphs=0, wait_ms=0, apply_engine=0, block=0, recycle=0):
    o = oras_options()
    o.restart, o.max_iter, o.factor_bits, o.weights, o.overlap_kind = restart, max_iter, factor_bits, weights, overlap_kind
    o.lu_engine = lu_engine
    o.lu_panel = lu_panel
    o.lu_group = lu_group
    o.transmission = transmission
    o.graphs = graphs
    o.wait_ms = wait_ms
    o.apply_engine = apply_engine
    o.block = block
    o.recycle = recycle
    return o


def oras_create(xyz, tets, r, nsub, overlap, part=None, beta_face=None, face_kind=None, **opts):
    """Host integer set-up; returns the handle (c_void_p).  beta_face: (nt, 4) impedance
    coefficients of the outer faces (face q of tet t is opposite tets[t, q]) or None; face_kind:
    (nt, 4) ORAS_FACE_IMPEDANCE / ORAS_FACE_METALLIC on the same faces, or None."""
    p, keep = _problem(xyz, tets, None, None, 1.0, r, nsub, overlap, part, beta_face, face_kind)
    o = _options(**opts)
    h = C.c_void_p()
    _check(None, lib.oras_create(C.byref(p), C.byref(o), C.byref(h)))
    del keep
    return h


def oras_setup(xyz, tets, eps_r, mu_r, k0, r, nsub, overlap, part=None, beta_face=None, face_kind=None,
               **opts):
    """oras_create + oras_factor: host mesh xyz (nv, 3), tets (nt, 4), per-tet complex eps_r and
    mu_r (None: 1), wave number k0, degree r, nsub subdomains (RCB unless part is given),
    overlap layers, beta_face (nt, 4) or None, face_kind (nt, 4) or None; opts are oras_options
    fields.  Returns the handle."""
    p, keep = _problem(xyz, tets, eps_r, mu_r, k0, r, nsub, overlap, part, beta_face, face_kind)
    o = _options(**opts)
    h = C.c_void_p()
    _check(None, lib.oras_setup(C.byref(p), C.byref(o), C.byref(h)))
    del keep
    return h


def oras_factor(h, eps_r, mu_r, k0, mem=ORAS_MEM_HOST):
    """(Re)assembles A and the local matrices for new materials on the handle's mesh and factors
    them (batched LU)."""
    if mem == ORAS_MEM_HOST:
        eps_r = _c128(eps_r)
        mu_r = None if mu_r is None else _c128(mu_r)
    return _check(h, lib.oras_factor(h, _ptr(eps_r), _ptr(mu_r), float(k0), mem))


def oras_destroy(h):
    """Frees the handle; its device memory returns to the device's memory pool."""
    lib.oras_destroy(h)


def oras_set_stream(h, stream_ptr):
    """Runs the handle's work on a caller's CUDA stream (e.g. torch.cuda.Stream().cuda_stream)."""
    return _check(h, lib.oras_set_stream(h, C.c_void_p(stream_ptr)))


def oras_set_timing(h, on):
    return _check(h, lib.oras_set_timing(h, int(on)))


KERNEL_CLASSES = ["element", "global_rows", "local_rows", "lu_tournament", "lu_swap", "lu_trsm",
                  "lu_update", "apply", "spmv", "orth", "other", "spmv64", "lu_panel"]


def oras_timings(h):
    """{class: (milliseconds, launches)} accumulated since the last reset."""
    n = 2 * len(KERNEL_CLASSES)
    t = np.zeros(n)
    _check(h, lib.oras_timings(h, _ptr(t), n))
    return {c: (t[2 * i], int(t[2 * i + 1])) for i, c in enumerate(KERNEL_CLASSES)}


def oras_reset_timings(h):
    return _check(h, lib.oras_reset_timings(h))


def oras_launch_count():
    return int(lib.oras_launch_count())


def oras_ndof(h):
    return int(lib.oras_ndof(h))


def oras_nlocal(h):
    return int(lib.oras_nlocal(h))


def oras_nsub(h):
    return int(lib.oras_nsub(h))


def oras_nnz(h):
    return int(lib.oras_nnz(h))


def oras_arena_bytes(h):
    return int(lib.oras_arena_bytes(h))


def oras_dofmap(h, nt):
    out = np.empty((nt, oras_nlocal(h)), dtype=np.int32)
    _check(h, lib.oras_dofmap(h, _ptr(out)))
    return out


def oras_partition(h, nt):
    out = np.empty(nt, dtype=np.int32)
    _check(h, lib.oras_partition(h, _ptr(out)))
    return out


def oras_subdomain_size(h, s):
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(h, lib.oras_subdomain_size(h, s, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def oras_subdomain(h, s):
    n, nt, _ = oras_subdomain_size(h, s)
    dofs = np.empty(n, dtype=np.int32)
    pou = np.empty(n, dtype=np.uint8)
    tets = np.empty(nt, dtype=np.int32)
    _check(h, lib.oras_subdomain(h, s, _ptr(dofs), _ptr(pou), _ptr(tets)))
    return dofs, pou, tets


def oras_element_matrices(h, tets):
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    nl = oras_nlocal(h)
    out = np.empty((len(tets), nl, nl), dtype=np.complex128)
    _check(h, lib.oras_element_matrices(h, _ptr(tets), len(tets), _ptr(out)))
    return out


def oras_global_csr(h):
    n = oras_ndof(h)
    nnz = oras_nnz(h)
    rowptr = np.empty(n + 1, dtype=np.int64)
    cols = np.empty(nnz, dtype=np.int32)
    vals = np.empty(nnz, dtype=np.complex128)
    _check(h, lib.oras_global_csr(h, _ptr(rowptr), _ptr(cols), _ptr(vals)))
    return rowptr, cols, vals


def _vec_call(fn, h, x, k, mem, out=None):
    n = oras_ndof(h)
    if mem == ORAS_MEM_HOST:
        x = np.asfortranarray(np.asarray(x, dtype=np.complex128).reshape(n, k) if k > 1 else
                              np.asarray(x, dtype=np.complex128).reshape(n, 1))
        y = np.empty((n, k), dtype=np.complex128, order="F")
        _check(h, fn(h, _ptr(x), _ptr(y), k, mem))
        return y if k > 1 else y[:, 0]
    _check(h, fn(h, _ptr(x), _ptr(out), k, mem))
    return out


def oras_matvec(h, x, k=1, mem=ORAS_MEM_HOST, out=None):
    """y = A x (host: (N,) or (N, k) complex128; device: torch tensors, N x k column-major)."""
    return _vec_call(lib.oras_matvec, h, x, k, mem, out)


def oras_matvec_c64(h, x, k=1, mem=ORAS_MEM_HOST, out=None):
    """y = A x for complex64 x (host: (N,) or (N, k); device: torch complex64, N x k column-major);
    y complex128."""
    n = oras_ndof(h)
    if mem == ORAS_MEM_HOST:
        xx = np.asfortranarray(np.asarray(x, dtype=np.complex64).reshape(n, k))
        y = np.empty((n, k), dtype=np.complex128, order="F")
        _check(h, lib.oras_matvec_c64(h, _ptr(xx), _ptr(y), k, mem))
        return y if k > 1 else y[:, 0]
    _check(h, lib.oras_matvec_c64(h, _ptr(x), _ptr(out), k, mem))
    return out


def oras_precond(h, v, k=1, mem=ORAS_MEM_HOST, out=None):
    """z = M^-1 v, the ORAS preconditioner (OAS with weights=ORAS_WEIGHTS_NONE); layouts as in
    oras_matvec."""
    return _vec_call(lib.oras_precond, h, v, k, mem, out)


def oras_solve(h, rhs, tol, k=1, mem=ORAS_MEM_HOST, out=None):
    """Returns (x, infos, rc); host: rhs (N,) or (N, k) complex; device: torch tensors,
    column-major N x k (i.e. shape (k, N) contiguous)."""
    n = oras_ndof(h)
    info = (oras_info * k)()
    if mem == ORAS_MEM_HOST:
        b = np.asfortranarray(np.asarray(rhs, dtype=np.complex128).reshape(n, k))
        x = np.empty((n, k), dtype=np.complex128, order="F")
        rc = _check(h, lib.oras_solve(h, _ptr(b), k, float(tol), _ptr(x), info, mem),
                    allow=(ORAS_OK, ORAS_NOT_CONVERGED))
        x = x if k > 1 else x[:, 0]
    else:
        rc = _check(h, lib.oras_solve(h, _ptr(rhs), k, float(tol), _ptr(out), info, mem),
                    allow=(ORAS_OK, ORAS_NOT_CONVERGED))
        x = out
    infos = [dict(iterations=i.iterations, restarts=i.restarts, converged=bool(i.converged),
                  relres=i.relres) for i in info]
    return x, infos, rc


def oras_rhs_dipole(h, x0, direction, mem=ORAS_MEM_HOST, out=None):
    """Point-dipole load b_a = w_a(x0) . direction (complex128, length N)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    d = np.ascontiguousarray(direction, dtype=np.float64)
    if mem == ORAS_MEM_HOST:
        out = np.empty(oras_ndof(h), dtype=np.complex128)
    _check(h, lib.oras_rhs_dipole(h, _ptr(x0), _ptr(d), _ptr(out), mem))
    return out


def port(origin, u, v, beta):
    """oras_port of the rectangle {origin + s u + t v}, TE10 mode sin(pi s) v/|v|."""
    P = oras_port()
    for i in range(3):
        P.origin[i], P.u[i], P.v[i] = float(origin[i]), float(u[i]), float(v[i])
    P.beta = float(beta)
    return P


def oras_port_vector(h, P):
    """(p, norm): p_a = int_port w_a . E0 (complex128 [N], real values) and int_port |E0|^2."""
    out = np.empty(oras_ndof(h), dtype=np.complex128)
    nrm = C.c_double()
    _check(h, lib.oras_port_vector(h, C.byref(P), _ptr(out), C.byref(nrm), ORAS_MEM_HOST))
    return out, nrm.value


def oras_rhs_port(h, P):
    """Load of the port transmitting its incoming TE10 mode (complex128 [N])."""
    out = np.empty(oras_ndof(h), dtype=np.complex128)
    _check(h, lib.oras_rhs_port(h, C.byref(P), _ptr(out), ORAS_MEM_HOST))
    return out


def oras_s_matrix(h, ports, X):
    """S [nports, k] of the fields X ((N,) or (N, k) complex, host)."""
    n = oras_ndof(h)
    X = np.asfortranarray(np.asarray(X, dtype=np.complex128).reshape(n, -1))
    k = X.shape[1]
    arr = (oras_port * len(ports))(*ports)
    S = np.empty((len(ports), k), dtype=np.complex128)
    _check(h, lib.oras_s_matrix(h, len(ports), C.cast(arr, C.c_void_p), _ptr(X), k, _ptr(S), ORAS_MEM_HOST))
    return S


def oras_s_error(S, S_ref):
    """Relative error of Sec. 5.2 between two scattering matrices (the library's host formula)."""
    S = _c128(S).ravel()
    R = _c128(S_ref).ravel()
    return float(lib.oras_s_error(_ptr(S), _ptr(R), S.size))


def oras_dense_eig(A):
    """(eigenvalues, unit eigenvectors as columns) of a small dense complex matrix, by the
    library's host QR algorithm."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    n = A.shape[0]
    w = np.empty(n, dtype=np.complex128)
    V = np.empty((n, n), dtype=np.complex128)
    rc = lib.oras_dense_eig(n, _ptr(A), _ptr(w), _ptr(V))
    if rc != ORAS_OK:
        raise OrasError(rc, "oras_dense_eig failed")
    return w, V


def oras_recycle_reset(h):
    _check(h, lib.oras_recycle_reset(h))


def oras_constrained_dofs(h):
    out = np.empty(oras_ndof(h), dtype=np.uint8)
    _check(h, lib.oras_constrained_dofs(h, _ptr(out)))
    return out


def oras_rhs_plane_wave(h, d, p, mem=ORAS_MEM_HOST, out=None):
    """Impedance data of the plane wave p exp(-i gamma d.x) on the outer boundary, as a load."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    p = _c128(p)
    if mem == ORAS_MEM_HOST:
        out = np.empty(oras_ndof(h), dtype=np.complex128)
    _check(h, lib.oras_rhs_plane_wave(h, _ptr(d), _ptr(p), _ptr(out), mem))
    return out


def oras_precond_noalloc(h, v, z, k=1):
    """z = M^{-1} v without any device allocation; v, z: torch CUDA complex128 tensors holding
    N x k column-major data (shape (k, N) contiguous, or (N,) for k = 1)."""
    return _check(h, lib.oras_precond_noalloc(h, _ptr(v), _ptr(z), int(k)))


def oras_wait_selftest(h):
    """Runs every bounded-wait primitive on a condition nothing satisfies, with the handle's
    wait_ms; returns (rc, detail): ORAS_ERR_DEVICE_TIMEOUT and the mask 7 when each gave up."""
    detail = C.c_int32()
    rc = lib.oras_wait_selftest(h, C.byref(detail))
    _check(h, rc, allow=(ORAS_OK, ORAS_ERR_DEVICE_TIMEOUT))
    return rc, detail.value


AUTOTUNE_WIDTHS = (4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192)


def oras_autotune(h):
    """Returns (panel width chosen, {(width, group): factorisation ms} (empty when cached)).
    The chosen raster group is oras_lu_group(h)."""
    panel = C.c_int32()
    ms = np.full(len(AUTOTUNE_WIDTHS) + 3, -1.0)
    _check(h, lib.oras_autotune(h, C.byref(panel), _ptr(ms), len(ms)))
    cands = [(w, 8) for w in AUTOTUNE_WIDTHS]
    best_w = max(((w, t) for (w, _), t in zip(cands, ms[:len(AUTOTUNE_WIDTHS)]) if t >= 0), key=lambda x: -x[1],
                 default=(panel.value, 0))[0]
    cands += [(best_w, g) for g in (16, 32, 64)]
    times = {c: t for c, t in zip(cands, ms) if t >= 0}
    return panel.value, times


def oras_lu_group(h):
    return lib.oras_lu_group(h)


def oras_release_memory(device=0):
    """Returns the unused memory of the device's memory pool to the driver."""
    rc = lib.oras_release_memory(int(device))
    if rc != ORAS_OK:
        raise OrasError(rc, f"oras_release_memory({device}) failed")


def oras_footprint(h, k=1):
    """Device bytes oras_factor + an oras_solve of k right-hand sides allocate."""
    b = C.c_int64()
    _check(h, lib.oras_footprint(h, int(k), C.byref(b)))
    return b.value


# ------------------------------------------------------------------ serving
class ServerError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"oras server error {code}: {msg}")
        self.code = code


def _scheck(srv, rc, ticket=0, allow=(ORAS_OK,)):
    if rc in allow:
        return rc
    msg = lib.oras_server_error(srv, ticket)
    raise ServerError(rc, msg.decode() if msg else "")


def oras_server_create(hbm_budget=0, device=0, max_active=4, planners=2):
    """Serving runtime: `max_active` worker slots (one CUDA stream each), `planners` host set-up
    threads, admission by device footprint within hbm_budget bytes (0: 0.9 of free memory)."""
    cfg = oras_server_config()
    cfg.hbm_budget, cfg.device, cfg.max_active, cfg.planners = int(hbm_budget), int(device), int(max_active), int(planners)
    srv = C.c_void_p()
    _scheck(None, lib.oras_server_create(C.byref(cfg), C.byref(srv)))
    return srv


def oras_submit(srv, xyz, tets, eps_r, mu_r, k0, r, nsub, overlap, part=None, rhs=None, dipoles=None,
                tol=1e-8, **opts):
    """Queues one solve; rhs: host (N,) or (N, k) complex, or dipoles: (k, 6) positions and
    directions.  Returns the ticket."""
    p, keep = _problem(xyz, tets, eps_r, mu_r, k0, r, nsub, overlap, part)
    o = _options(**opts)
    if rhs is not None:
        b = np.asfortranarray(np.asarray(rhs, dtype=np.complex128))
        if b.ndim == 1:
            b = b.reshape(-1, 1, order="F")
        n, k = b.shape
        t = lib.oras_submit(srv, C.byref(p), C.byref(o), _ptr(b), n, None, k, float(tol))
    else:
        d = np.ascontiguousarray(dipoles, dtype=np.float64).reshape(-1, 6)
        t = lib.oras_submit(srv, C.byref(p), C.byref(o), None, 0, _ptr(d), d.shape[0], float(tol))
    del keep
    if t < 0:
        _scheck(srv, int(t))
    return int(t)


def oras_ticket_info(srv, ticket):
    rec = oras_ticket()
    _scheck(srv, lib.oras_ticket_info(srv, int(ticket), C.byref(rec)))
    return {f: getattr(rec, f) for f, _ in oras_ticket._fields_}


def oras_ticket_wait(srv, ticket, timeout_ms=-1):
    return _scheck(srv, lib.oras_ticket_wait(srv, int(ticket), int(timeout_ms)), allow=(ORAS_OK, ORAS_PENDING))


def oras_wait(srv, ticket, timeout_ms=-1):
    """Returns (x, infos, rc): x (N, k) complex (or (N,) for k = 1), None when the request
    failed; rc is the request's status, ORAS_PENDING (x None) if it is still running.  Raises
    ServerError for an unknown or already collected ticket."""
    if oras_ticket_wait(srv, ticket, timeout_ms) == ORAS_PENDING:
        return None, None, ORAS_PENDING
    rec = oras_ticket_info(srv, ticket)
    n, k = rec["ndof"], rec["k"]
    x = np.empty((max(n, 1), k), dtype=np.complex128, order="F")
    info = (oras_info * k)()
    live = rec["status"] != ORAS_PENDING
    rc = lib.oras_wait(srv, int(ticket), _ptr(x), n, info, 0)
    if rc == ORAS_ERR_STATE or (rc == ORAS_ERR_INVALID_ARG and not live):
        _scheck(srv, rc)
    if rc not in (ORAS_OK, ORAS_NOT_CONVERGED):
        return None, None, rc
    infos = [dict(iterations=i.iterations, restarts=i.restarts, converged=bool(i.converged),
                  relres=i.relres) for i in info]
    return (x if k > 1 else x[:, 0]), infos, rc


def oras_server_error(srv, ticket=0):
    msg = lib.oras_server_error(srv, int(ticket))
    return msg.decode() if msg else ""


def oras_server_stats(srv):
    c = oras_server_counters()
    _scheck(srv, lib.oras_server_stats(srv, C.byref(c)))
    return {f: getattr(c, f) for f, _ in oras_server_counters._fields_ if f != "pad"}


def oras_server_destroy(srv):
    lib.oras_server_destroy(srv)
