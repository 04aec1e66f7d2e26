"""Thin ctypes binding of libopf.so (include/opf.h), same names as the C ABI.

Argument marshalling only: every step of the time step runs in the library's
CUDA kernels.  If the library has not been built this module raises -- there
is no fallback path.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libopf.so")

OPF_OK, OPF_EINVAL, OPF_ECUDA, OPF_ENAN, OPF_ETIMEOUT, OPF_ENOMEM = 0, -1, -2, -3, -4, -5

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


_pdp = ctypes.POINTER(ctypes.POINTER(ctypes.c_double))
NK_RESIDUAL = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                               _pdp, _pdp, ctypes.c_int)
NK_JV = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                         _pdp, _pdp, _pdp)


class NkOpts(ctypes.Structure):
    _fields_ = [("max_newton", ctypes.c_int), ("max_krylov", ctypes.c_int), ("max_hook", ctypes.c_int),
                ("tol", ctypes.c_double), ("gmres_tol", ctypes.c_double), ("delta0", ctypes.c_double),
                ("dt", ctypes.c_double), ("eps", ctypes.c_double), ("fix_T", ctypes.c_int),
                ("fix_s", ctypes.c_int), ("precision", ctypes.c_int),
                ("forcing", ctypes.c_void_p), ("rot", ctypes.c_double * 3)]


def nk_opts(**kw):
    """Newton-Krylov options; forcing= a state-layout complex array (kept alive
    on the returned object) or None, rot= (Omega_x, Omega_y, Omega_z)."""
    o = NkOpts(max_newton=30, max_krylov=60, max_hook=12, tol=1e-10, gmres_tol=1e-3, delta0=0.0,
               dt=0.01, eps=1e-7, fix_T=0, fix_s=0, precision=0, forcing=None)
    for k, v in kw.items():
        if k == "forcing":
            if v is not None:
                arr = np.ascontiguousarray(v, dtype=np.complex128)
                o._forcing_keep = arr
                o.forcing = arr.ctypes.data
            continue
        if k == "rot":
            o.rot = (ctypes.c_double * 3)(*[float(x) for x in v])
            continue
        setattr(o, k, v)
    return o


class OpfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"opf error {code}: {msg}")
        self.code = code


def lib():
    """Load libopf.so once (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libopf.so is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, cp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_char_p
        L.opf_create.restype = vp
        L.opf_create.argtypes = [i, i, i, i, d, d, d]
        L.opf_destroy.restype = None
        L.opf_destroy.argtypes = [vp]
        L.opf_last_error.restype = cp
        L.opf_last_error.argtypes = []
        for name in ("opf_set_state", "opf_get_state", "opf_set_state_device", "opf_get_state_device"):
            getattr(L, name).restype = i
            getattr(L, name).argtypes = [vp, vp]
        L.opf_step.restype = i
        L.opf_step.argtypes = [vp, i]
        L.opf_energy.restype = i
        L.opf_energy.argtypes = [vp, _dp]
        L.opf_wall_residual.restype = i
        L.opf_wall_residual.argtypes = [vp, _dp]
        L.opf_nonlinear.restype = i
        L.opf_nonlinear.argtypes = [vp, vp, vp]
        L.opf_set_option.restype = i
        L.opf_set_option.argtypes = [vp, cp, d]
        L.opf_get_option.restype = i
        L.opf_get_option.argtypes = [vp, cp, _dp]
        for name in ("opf_get_dt", "opf_get_time", "opf_get_beta"):
            getattr(L, name).restype = i
            getattr(L, name).argtypes = [vp, _dp]
        L.opf_set_stream.restype = i
        L.opf_set_stream.argtypes = [vp, vp]
        L.opf_kernel_times.restype = i
        L.opf_kernel_times.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(cp), _dp,
                                       ctypes.POINTER(i), i]
        L.opf_ens_create.restype = vp
        ip = ctypes.POINTER(ctypes.c_int)
        L.opf_ens_create.argtypes = [i, ip, ip, ip, ip, _dp, _dp, _dp]
        L.opf_ens_destroy.restype = None
        L.opf_ens_destroy.argtypes = [vp]
        L.opf_ens_count.restype = i
        L.opf_ens_count.argtypes = [vp, ip]
        for name in ("opf_ens_set_state", "opf_ens_get_state", "opf_ens_set_state_device",
                     "opf_ens_get_state_device"):
            getattr(L, name).restype = i
            getattr(L, name).argtypes = [vp, i, vp]
        L.opf_ens_step.restype = i
        L.opf_ens_step.argtypes = [vp, i]
        L.opf_ens_energy.restype = i
        L.opf_ens_energy.argtypes = [vp, i, _dp]
        L.opf_ens_get_time.restype = i
        L.opf_ens_get_time.argtypes = [vp, i, _dp]
        L.opf_ens_set_option.restype = i
        L.opf_ens_set_option.argtypes = [vp, cp, d]
        L.opf_ens_set_stream.restype = i
        L.opf_ens_set_stream.argtypes = [vp, vp]
        L.opf_ens_kernel_times.restype = i
        L.opf_ens_kernel_times.argtypes = [vp, i, ip, ctypes.POINTER(cp), _dp, ip, i]
        L.opf_fma_rate.restype = i
        L.opf_fma_rate.argtypes = [i, _dp]
        L.opf_nk_core.restype = i
        L.opf_nk_core.argtypes = [i, i, _dp, _dp, NK_RESIDUAL, NK_JV, vp, ctypes.POINTER(NkOpts),
                                  _dp, ctypes.POINTER(i)]
        L.opf_nk_solve.restype = i
        L.opf_nk_solve.argtypes = [i, i, i, i, d, d, i, vp, _dp, _dp, ctypes.POINTER(NkOpts), _dp,
                                   ctypes.POINTER(i)]
        L.opf_nk_solve_ms.restype = i
        L.opf_nk_solve_ms.argtypes = [i, i, i, i, d, d, i, i, vp, _dp, _dp, ctypes.POINTER(NkOpts), _dp,
                                      ctypes.POINTER(i)]
        L.opf_arnoldi_core.restype = i
        L.opf_arnoldi_core.argtypes = [i, i, _dp, i, i, LINEAR_MAP, vp, _dp, _dp, _dp, ctypes.POINTER(i)]
        L.opf_floquet.restype = i
        L.opf_floquet.argtypes = [i, i, i, i, d, d, i, vp, _dp, _dp, i, i, d, d, i, ctypes.c_ulonglong, vp,
                                  _dp, _dp, _dp]
        L.opf_net_create.restype = vp
        L.opf_net_create.argtypes = [i, i, i, i, ctypes.c_ulonglong]
        L.opf_net_destroy.restype = None
        L.opf_net_destroy.argtypes = [vp]
        L.opf_net_param_count.restype = i
        L.opf_net_param_count.argtypes = [vp, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long)]
        L.opf_net_get_params.restype = i
        L.opf_net_get_params.argtypes = [vp, vp, i]
        L.opf_net_set_params.restype = i
        L.opf_net_set_params.argtypes = [vp, vp]
        L.opf_net_forward.restype = i
        L.opf_net_forward.argtypes = [vp, vp, i, vp, vp]
        L.opf_net_gradients.restype = i
        L.opf_net_gradients.argtypes = [vp, vp, vp, vp, i, ctypes.c_float, _dp]
        L.opf_net_train_step.restype = i
        L.opf_net_train_step.argtypes = [vp, vp, vp, vp, i, ctypes.c_float, ctypes.c_float, _dp]
        L.opf_net_gather_augment.restype = i
        L.opf_net_gather_augment.argtypes = [vp, i, i, i, i, i, i, vp, vp, vp, ctypes.c_long, vp, vp, vp, vp, vp]
        L.opf_nonlinear_noalloc.restype = i
        L.opf_nonlinear_noalloc.argtypes = [i, i, i, i, d, d, vp, vp, vp]
        L.opf_set_forcing.restype = i
        L.opf_set_forcing.argtypes = [vp, vp]
        L.opf_change_resolution.restype = i
        L.opf_change_resolution.argtypes = [i, i, i, vp, i, i, i, i, vp]
        L.opf_create_mesh.restype = vp
        L.opf_create_mesh.argtypes = [i, i, i, i, d, d, d, _dp]
        L.opf_setup_query_mesh.restype = i
        L.opf_setup_query_mesh.argtypes = [i, i, i, i, d, d, d, _dp, cp, _dp, ctypes.c_long,
                                           ctypes.POINTER(ctypes.c_long)]
        L.opf_setup_query.restype = i
        L.opf_setup_query.argtypes = [i, i, i, i, d, d, d, cp, _dp, ctypes.c_long,
                                      ctypes.POINTER(ctypes.c_long)]
        _lib = L
    return _lib


def _check(rc):
    if rc != OPF_OK:
        raise OpfError(rc, lib().opf_last_error().decode())


class Handle:
    """Owns an opf_t*; shape information for marshalling."""

    def __init__(self, ptr, N, K, M):
        self.ptr, self.N, self.K, self.M = ptr, N, K, M
        self.shape = (3, M, 2 * K - 1, N)

    def __del__(self):
        try:
            opf_destroy(self)
        except Exception:
            pass


def _state_buffer(h, arr):
    a = np.ascontiguousarray(arr, dtype=np.complex128)
    if a.shape != h.shape:
        raise ValueError(f"state must have shape {h.shape}, got {a.shape}")
    return a


def opf_create(N, K, M, m_p, alpha, Re, dt):
    ptr = lib().opf_create(N, K, M, m_p, alpha, Re, dt)
    if not ptr:
        raise OpfError(OPF_EINVAL, lib().opf_last_error().decode())
    return Handle(ptr, N, K, M)


def opf_create_mesh(N, K, M, m_p, alpha, Re, dt, r):
    """opf_create on a user radial mesh r (N increasing points, r[-1] = 1)."""
    ra = np.ascontiguousarray(r, dtype=np.float64)
    if ra.shape != (N,):
        raise OpfError(OPF_EINVAL, "opf_create_mesh: r must hold N points")
    ptr = lib().opf_create_mesh(N, K, M, m_p, alpha, Re, dt, ra.ctypes.data_as(_dp))
    if not ptr:
        raise OpfError(OPF_EINVAL, lib().opf_last_error().decode())
    return Handle(ptr, N, K, M)


def opf_destroy(h):
    if h.ptr:
        lib().opf_destroy(h.ptr)
        h.ptr = None


def opf_set_state(h, state):
    a = _state_buffer(h, state)
    _check(lib().opf_set_state(h.ptr, a.ctypes.data))


def opf_get_state(h, out=None):
    out = np.empty(h.shape, dtype=np.complex128) if out is None else out
    if out.shape != h.shape or out.dtype != np.complex128 or not out.flags.c_contiguous:
        raise ValueError("output must be a C-contiguous complex128 array of the state shape")
    _check(lib().opf_get_state(h.ptr, out.ctypes.data))
    return out


def opf_set_state_device(h, dev_ptr):
    """dev_ptr: integer device address of a complex128 state (e.g. tensor.data_ptr())."""
    _check(lib().opf_set_state_device(h.ptr, ctypes.c_void_p(dev_ptr)))


def opf_get_state_device(h, dev_ptr):
    _check(lib().opf_get_state_device(h.ptr, ctypes.c_void_p(dev_ptr)))


def opf_step(h, n=1):
    _check(lib().opf_step(h.ptr, int(n)))


def opf_energy(h):
    out = (ctypes.c_double * 3)()
    _check(lib().opf_energy(h.ptr, out))
    return np.array(out[:])


def opf_wall_residual(h):
    out = (ctypes.c_double * 2)()
    _check(lib().opf_wall_residual(h.ptr, out))
    return np.array(out[:])


def opf_nonlinear(h, state):
    a = _state_buffer(h, state)
    out = np.empty(h.shape, dtype=np.complex128)
    _check(lib().opf_nonlinear(h.ptr, a.ctypes.data, out.ctypes.data))
    return out


def opf_nonlinear_noalloc(N, K, M, m_p, alpha, Re, d_state, d_out, stream=0):
    """Allocation-free nonlinear term; d_state / d_out are integer device
    addresses of complex128 buffers in the state layout (e.g. data_ptr())."""
    _check(lib().opf_nonlinear_noalloc(int(N), int(K), int(M), int(m_p), float(alpha), float(Re),
                                       ctypes.c_void_p(d_state), ctypes.c_void_p(d_out),
                                       ctypes.c_void_p(stream)))


def opf_fma_rate(precision):
    """Measured FMA throughput of the current device in TFLOP/s (0 FP64, 1 FP32)."""
    out = ctypes.c_double(0.0)
    _check(lib().opf_fma_rate(int(precision), ctypes.byref(out)))
    return out.value


def opf_set_option(h, key, value):
    _check(lib().opf_set_option(h.ptr, key.encode(), float(value)))


def opf_get_option(h, key):
    v = ctypes.c_double()
    _check(lib().opf_get_option(h.ptr, key.encode(), ctypes.byref(v)))
    return v.value


def _get_scalar(fn, h):
    v = ctypes.c_double()
    _check(fn(h.ptr, ctypes.byref(v)))
    return v.value


def opf_get_dt(h):
    return _get_scalar(lib().opf_get_dt, h)


def opf_get_time(h):
    return _get_scalar(lib().opf_get_time, h)


def opf_get_beta(h):
    return _get_scalar(lib().opf_get_beta, h)


def opf_set_stream(h, stream_handle):
    """stream_handle: integer cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream)."""
    _check(lib().opf_set_stream(h.ptr, ctypes.c_void_p(stream_handle)))


def opf_kernel_times(h, reset=False):
    cap = 16
    count = ctypes.c_int()
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_double * cap)()
    n = (ctypes.c_int * cap)()
    _check(lib().opf_kernel_times(h.ptr, cap, ctypes.byref(count), names, ms, n, int(reset)))
    return {names[i].decode(): (ms[i], n[i]) for i in range(count.value)}


class EnsHandle:
    """Owns an opf_ens_t*; per-trajectory state shapes for marshalling."""

    def __init__(self, ptr, shapes):
        self.ptr, self.shapes = ptr, shapes

    def __del__(self):
        try:
            opf_ens_destroy(self)
        except Exception:
            pass


def opf_ens_create(N, K, M, m_p, alpha, Re, dt):
    """Sequences of equal length (one entry per trajectory)."""
    n = len(N)
    ci = lambda v: (ctypes.c_int * n)(*[int(x) for x in v])
    cd = lambda v: (ctypes.c_double * n)(*[float(x) for x in v])
    ptr = lib().opf_ens_create(n, ci(N), ci(K), ci(M), ci(m_p), cd(alpha), cd(Re), cd(dt))
    if not ptr:
        raise OpfError(OPF_EINVAL, lib().opf_last_error().decode())
    return EnsHandle(ptr, [(3, M[j], 2 * K[j] - 1, N[j]) for j in range(n)])


def opf_ens_destroy(e):
    if e.ptr:
        lib().opf_ens_destroy(e.ptr)
        e.ptr = None


def opf_ens_set_state(e, i, state):
    a = np.ascontiguousarray(state, dtype=np.complex128)
    if a.shape != e.shapes[i]:
        raise ValueError(f"state {i} must have shape {e.shapes[i]}")
    _check(lib().opf_ens_set_state(e.ptr, int(i), a.ctypes.data))


def opf_ens_get_state(e, i):
    out = np.empty(e.shapes[i], dtype=np.complex128)
    _check(lib().opf_ens_get_state(e.ptr, int(i), out.ctypes.data))
    return out


def opf_ens_step(e, n=1):
    _check(lib().opf_ens_step(e.ptr, int(n)))


def opf_ens_energy(e, i):
    out = (ctypes.c_double * 3)()
    _check(lib().opf_ens_energy(e.ptr, int(i), out))
    return np.array(out[:])


def opf_ens_get_time(e, i):
    v = ctypes.c_double()
    _check(lib().opf_ens_get_time(e.ptr, int(i), ctypes.byref(v)))
    return v.value


def opf_ens_set_option(e, key, value):
    _check(lib().opf_ens_set_option(e.ptr, key.encode(), float(value)))


def opf_ens_set_stream(e, stream_handle):
    _check(lib().opf_ens_set_stream(e.ptr, ctypes.c_void_p(stream_handle)))


def opf_ens_kernel_times(e, reset=False):
    cap = 16
    count = ctypes.c_int()
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_double * cap)()
    n = (ctypes.c_int * cap)()
    _check(lib().opf_ens_kernel_times(e.ptr, cap, ctypes.byref(count), names, ms, n, int(reset)))
    return {names[i].decode(): (ms[i], n[i]) for i in range(count.value)}


def opf_nk_core(x0, F, JV, scale=None, **opts):
    """Newton-Krylov-hookstep on count problems: x0 (count, n) float64;
    F(idx, xs) -> list of residual arrays; JV(idx, xs, vs) -> list of arrays
    (idx: problem indices of this batch).  Returns (x, residual, iters)."""
    x = np.ascontiguousarray(x0, dtype=np.float64).copy()
    count, n = x.shape
    sc = np.ones(count) if scale is None else np.ascontiguousarray(scale, dtype=np.float64)

    def view(ptrs, cnt):
        return [np.ctypeslib.as_array(ptrs[j], shape=(n,)) for j in range(cnt)]

    def f_cb(ctx, cnt, idx, xp, fp, commit):
        try:
            ids = [idx[j] for j in range(cnt)]
            out = F(ids, [a.copy() for a in view(xp, cnt)])
            for dst, src in zip(view(fp, cnt), out):
                dst[:] = src
            return 0
        except Exception:
            return -1

    def jv_cb(ctx, cnt, idx, xp, vp, jp):
        try:
            ids = [idx[j] for j in range(cnt)]
            out = JV(ids, [a.copy() for a in view(xp, cnt)], [a.copy() for a in view(vp, cnt)])
            for dst, src in zip(view(jp, cnt), out):
                dst[:] = src
            return 0
        except Exception:
            return -1

    fcb, jcb = NK_RESIDUAL(f_cb), NK_JV(jv_cb)
    res = np.zeros(count)
    it = (ctypes.c_int * count)()
    o = nk_opts(**opts)
    _check(lib().opf_nk_core(n, count, x.ctypes.data_as(_dp), sc.ctypes.data_as(_dp), fcb, jcb, None,
                             ctypes.byref(o), res.ctypes.data_as(_dp), it))
    return x, res, np.array(it[:])


def opf_nk_solve(N, K, M, m_p, alpha, Re, states, T, s, **opts):
    """Periodic-orbit / travelling-wave search for a list of guesses; returns
    (states, T, s, relative residuals, Newton iterations)."""
    count = len(states)
    st = np.ascontiguousarray(np.stack(states), dtype=np.complex128)
    Ta = np.ascontiguousarray(T, dtype=np.float64).copy()
    sa = np.ascontiguousarray(s, dtype=np.float64).copy()
    res = np.zeros(count)
    it = (ctypes.c_int * count)()
    o = nk_opts(**opts)
    _check(lib().opf_nk_solve(N, K, M, m_p, alpha, Re, count, st.ctypes.data, Ta.ctypes.data_as(_dp),
                              sa.ctypes.data_as(_dp), ctypes.byref(o), res.ctypes.data_as(_dp), it))
    return list(st), Ta, sa, res, np.array(it[:])


LINEAR_MAP = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _pdp, _pdp)


def opf_arnoldi_core(v0, A, kdim, nev):
    """Leading eigenvalues of count linear maps (host Arnoldi): v0 (count, n);
    A(idx, vs) -> list of A v arrays.  Returns (eigenvalues (count, nev)
    complex, residual estimates (count, nev), Krylov dimensions (count,))."""
    v = np.ascontiguousarray(v0, dtype=np.float64)
    count, n = v.shape

    def cb(ctx, cnt, idx, vp, ap):
        try:
            ids = [idx[j] for j in range(cnt)]
            vs = [np.ctypeslib.as_array(vp[j], shape=(n,)).copy() for j in range(cnt)]
            out = A(ids, vs)
            for j in range(cnt):
                np.ctypeslib.as_array(ap[j], shape=(n,))[:] = out[j]
            return 0
        except Exception:
            return -1

    fn = LINEAR_MAP(cb)
    er = np.zeros((count, nev))
    ei = np.zeros((count, nev))
    rs = np.zeros((count, nev))
    ku = (ctypes.c_int * count)()
    _check(lib().opf_arnoldi_core(n, count, v.ctypes.data_as(_dp), int(kdim), int(nev), fn, None,
                                  er.ctypes.data_as(_dp), ei.ctypes.data_as(_dp), rs.ctypes.data_as(_dp), ku))
    return er + 1j * ei, rs, np.array(ku[:])


def opf_floquet(N, K, M, m_p, alpha, Re, states, T, s, kdim, nev, dt, eps=1e-7, precision=0, seed=1,
                start=None):
    """Floquet multipliers of count states (time-T maps with axial shift s):
    returns (multipliers (count, nev) complex, residual estimates)."""
    count = len(states)
    st = np.ascontiguousarray(np.stack(states), dtype=np.complex128)
    Ta = np.ascontiguousarray(T, dtype=np.float64)
    sa = np.ascontiguousarray(s, dtype=np.float64)
    sv = None if start is None else np.ascontiguousarray(np.stack(start), dtype=np.complex128)
    er = np.zeros((count, nev))
    ei = np.zeros((count, nev))
    rs = np.zeros((count, nev))
    _check(lib().opf_floquet(N, K, M, m_p, float(alpha), float(Re), count, st.ctypes.data, Ta.ctypes.data_as(_dp),
                             sa.ctypes.data_as(_dp), int(kdim), int(nev), float(dt), float(eps), int(precision),
                             ctypes.c_ulonglong(seed), None if sv is None else sv.ctypes.data,
                             er.ctypes.data_as(_dp), ei.ctypes.data_as(_dp), rs.ctypes.data_as(_dp)))
    return er + 1j * ei, rs


def opf_set_forcing(h, forcing):
    """Constant body force (state layout, components r, theta, z); None removes it."""
    if forcing is None:
        _check(lib().opf_set_forcing(h.ptr, None))
        return
    a = np.ascontiguousarray(forcing, dtype=np.complex128)
    _check(lib().opf_set_forcing(h.ptr, a.ctypes.data))


def opf_change_resolution(state, N2, K2, M2, m_p):
    """state (3, M1, 2K1-1, N1) -> the same flow at (N2, K2, M2)."""
    a = np.ascontiguousarray(state, dtype=np.complex128)
    _, M1, nk1, N1 = a.shape
    out = np.empty((3, M2, 2 * K2 - 1, N2), dtype=np.complex128)
    _check(lib().opf_change_resolution(N1, (nk1 + 1) // 2, M1, a.ctypes.data, N2, K2, M2, m_p, out.ctypes.data))
    return out


def opf_nk_solve_ms(N, K, M, m_p, alpha, Re, sections, T, s, **opts):
    """Multiple shooting: sections[i] is the list of S section starts of
    guess i.  Returns (sections, T, s, relative residuals, Newton iterations)."""
    count, S = len(sections), len(sections[0])
    st = np.ascontiguousarray(np.stack([np.stack(x) for x in sections]), dtype=np.complex128)
    Ta = np.ascontiguousarray(T, dtype=np.float64).copy()
    sa = np.ascontiguousarray(s, dtype=np.float64).copy()
    res = np.zeros(count)
    it = (ctypes.c_int * count)()
    o = nk_opts(**opts)
    _check(lib().opf_nk_solve_ms(N, K, M, m_p, alpha, Re, count, S, st.ctypes.data, Ta.ctypes.data_as(_dp),
                                 sa.ctypes.data_as(_dp), ctypes.byref(o), res.ctypes.data_as(_dp), it))
    return [list(x) for x in st], Ta, sa, res, np.array(it[:])


class NetHandle:
    def __init__(self, ptr, cin, hidden, L, nout):
        self.ptr, self.cin, self.hidden, self.L, self.nout = ptr, cin, hidden, L, nout

    def __del__(self):
        try:
            opf_net_destroy(self)
        except Exception:
            pass


def opf_net_create(cin, hidden, L, nout, seed=1):
    ptr = lib().opf_net_create(cin, hidden, L, nout, seed)
    if not ptr:
        raise OpfError(OPF_EINVAL, lib().opf_last_error().decode())
    return NetHandle(ptr, cin, hidden, L, nout)


def opf_net_destroy(n):
    if n.ptr:
        lib().opf_net_destroy(n.ptr)
        n.ptr = None


def opf_net_param_count(n):
    tot = ctypes.c_long()
    sizes = (ctypes.c_long * 8)()
    _check(lib().opf_net_param_count(n.ptr, ctypes.byref(tot), sizes))
    return tot.value, list(sizes)


def opf_net_get_params(n, grads=False):
    tot, _ = opf_net_param_count(n)
    out = np.empty(tot, dtype=np.float32)
    _check(lib().opf_net_get_params(n.ptr, out.ctypes.data, int(grads)))
    return out


def opf_net_set_params(n, flat):
    a = np.ascontiguousarray(flat, dtype=np.float32)
    _check(lib().opf_net_set_params(n.ptr, a.ctypes.data))


def opf_net_forward(n, d_x, B, d_y, d_z):
    """device pointers (float32): x [B][L][cin] -> y [B][L][cin], z [B][nout]"""
    _check(lib().opf_net_forward(n.ptr, ctypes.c_void_p(d_x), int(B), ctypes.c_void_p(d_y),
                                 ctypes.c_void_p(d_z)))


def opf_net_gradients(n, d_x, d_ty, d_tz, B, lam):
    loss = ctypes.c_double()
    _check(lib().opf_net_gradients(n.ptr, ctypes.c_void_p(d_x), ctypes.c_void_p(d_ty), ctypes.c_void_p(d_tz),
                                   int(B), float(lam), ctypes.byref(loss)))
    return loss.value


def opf_net_train_step(n, d_x, d_ty, d_tz, B, lam, lr):
    loss = ctypes.c_double()
    _check(lib().opf_net_train_step(n.ptr, ctypes.c_void_p(d_x), ctypes.c_void_p(d_ty), ctypes.c_void_p(d_tz),
                                    int(B), float(lam), float(lr), ctypes.byref(loss)))
    return loss.value


def opf_net_gather_augment(net, d_x, d_y, d_z, rows, idx, ang, L, ncomp, nkf, mf, nz, d_bx, d_by, d_bz):
    """Device minibatch: rows idx of the device sets, each turned by the
    phases ang[b] = (alpha a, m_p phi); d_* are device addresses."""
    ia = np.ascontiguousarray(idx, dtype=np.int32)
    aa = np.ascontiguousarray(ang, dtype=np.float32).reshape(-1)
    B = ia.shape[0]
    if aa.shape[0] != 2 * B:
        raise OpfError(OPF_EINVAL, "opf_net_gather_augment: ang needs two phases per sample")
    _check(lib().opf_net_gather_augment(net.ptr, B, L, ncomp, nkf, mf, nz, d_x, d_y, d_z, int(rows),
                                        ia.ctypes.data, aa.ctypes.data, d_bx, d_by, d_bz))


def opf_setup_query(N, K, M, m_p, alpha, Re, dt, what, r=None):
    """One array of the host setup (see opf.h); r: a user radial mesh or None."""
    L = lib()
    n = ctypes.c_long()
    ra = None if r is None else np.ascontiguousarray(r, dtype=np.float64)
    rp = None if ra is None else ra.ctypes.data_as(_dp)
    _check(L.opf_setup_query_mesh(N, K, M, m_p, alpha, Re, dt, rp, what.encode(), None, 0, ctypes.byref(n)))
    out = np.empty(n.value, dtype=np.float64)
    _check(L.opf_setup_query_mesh(N, K, M, m_p, alpha, Re, dt, rp, what.encode(),
                                  out.ctypes.data_as(_dp), n.value, ctypes.byref(n)))
    return out
