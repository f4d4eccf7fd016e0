"""Thin Python binding of the C ABI in include/dgfs.h (argument marshalling only).

Functions keep the C names (dgfs_plan_create, dgfs_collide, ...).  Tensors are
passed as raw device/host pointers; every step of the computation runs in the
CUDA library ``_lib/libdgfs.so``.  There is no CPU fallback: if the library
cannot be loaded, every call raises.
"""
import ctypes
import math
import os

import torch

from . import _build

FP64, FP32_TC, TF32, BF16X3 = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp32_tc": FP32_TC, "tf32": TF32, "bf16x3": BF16X3}
STATUS = {0: "DGFS_OK", 1: "DGFS_EINVAL", 2: "DGFS_ENOMEM", 3: "DGFS_ECUDA", 4: "DGFS_ETIMEOUT",
          5: "DGFS_EUNSUPPORTED"}


class DgfsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


class dgfs_pair(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("alpha", ctypes.c_double), ("d", ctypes.c_double),
                ("beta_override", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p


def library_path():
    return _build.LIB


def lib():
    """Load (building first if needed) the CUDA library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i, d, ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        sig = {
            "dgfs_plan_create": (i, [ctypes.POINTER(_P), i, d, i, i, i, _P, _P, i, i, i]),
            "dgfs_plan_destroy": (i, [_P]),
            "dgfs_collide": (i, [_P, i, _P, _P, _P]),
            "dgfs_collide_host": (i, [_P, i, _P, _P, _P]),
            "dgfs_collide_noalloc": (i, [_P, i, _P, _P, _P]),
            "dgfs_collide_backward": (i, [_P, i, _P, _P, _P, _P, i, _P]),
            "dgfs_moments": (i, [_P, i, _P, _P, _P]),
            "dgfs_plan_info": (i, [_P, _P]),
            "dgfs_plan_pair_tables": (i, [_P, i, i, _P, _P, _P, _P, _P, _P, _P]),
            "dgfs_plan_launch_count": (i, [_P, ctypes.POINTER(ll)]),
            "dgfs_plan_profile": (i, [_P, i]),
            "dgfs_plan_check": (i, [_P]),
            "dgfs_plan_selftest_wait": (i, [_P, i, _P]),
            "dgfs_relax_step": (i, [_P, i, _P, _P, d, _P]),
            "dgfs_graph_capture": (i, [i, _P, _P, _P, _P, d, i, ctypes.POINTER(_P)]),
            "dgfs_graph_launch": (i, [_P, _P]),
            "dgfs_graph_kernel_count": (i, [_P, ctypes.POINTER(ll)]),
            "dgfs_graph_destroy": (i, [_P]),
            "dgfs_batch_create": (i, [i, _P, _P, _P, _P, d, ctypes.POINTER(_P)]),
            "dgfs_batch_launch": (i, [_P, _P]),
            "dgfs_batch_destroy": (i, [_P]),
            "dgfs_plan_autotune": (i, [_P, i, _P, _P, _P, ctypes.POINTER(d)]),
            "dgfs_plan_profile_read": (i, [_P, i, _P, _P, _P, ctypes.POINTER(i)]),
            "dgfs_plan_set_collapse": (i, [_P, i]),
            "dgfs_plan_set_kernel_variant": (i, [_P, i]),
            "dgfs_plan_set_schedule": (i, [_P, i]),
            "dgfs_plan_get_schedule": (i, [_P, ctypes.POINTER(i)]),
            "dgfs_batch_set_schedule": (i, [_P, i]),
            "dgfs_debug_worklist_trace": (i, [_P, ctypes.c_size_t]),
            "dgfs_debug_worklist_chunk": (i, [i]),
            "dgfs_plan_set_hermitian": (i, [_P, i]),
            "dgfs_dealias_work_bytes": (i, [_P, i, i, ctypes.POINTER(ctypes.c_size_t)]),
            "dgfs_collide_dealiased": (i, [_P, i, i, _P, _P, _P, ctypes.c_size_t, _P]),
            "dgfs_dg_create": (i, [ctypes.POINTER(_P), _P, i, i, d, d, _P]),
            "dgfs_dg_destroy": (i, [_P]),
            "dgfs_dg_nodes": (i, [_P, _P]),
            "dgfs_dg_rhs": (i, [_P, _P, _P, _P, _P]),
            "dgfs_dg_step": (i, [_P, _P, d, i, _P]),
            "dgfs_dg_traces": (i, [_P, _P, _P, _P, _P]),
            "dgfs_dg_rhs_halo": (i, [_P, _P, _P, _P, _P, _P, _P]),
            "dgfs_dg_stage": (i, [_P, _P, _P, _P, d, d, d, i, _P, _P, _P]),
            "dgfs_status_string": (ctypes.c_char_p, [i]),
            "dgfs_last_error": (ctypes.c_char_p, []),
            "dgfs_version": (ctypes.c_char_p, []),
            "dgfs_probe_mma_rate": (i, [i, i, i, ctypes.POINTER(d)]),
            "dgfs_debug_fail_alloc": (None, [i]),
            "dgfs_debug_live_allocations": (ll, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    """Names of the dgfs_* functions the loaded library exports (checked by tests
    against include/dgfs.h without calling any of them)."""
    L = lib()
    import re
    hdr = open(os.path.join(_build.ROOT, "include", "dgfs.h")).read()
    names = re.findall(r"\b(dgfs_[a-z0-9_]+)\s*\(", hdr)
    return {n: hasattr(L, n) for n in names}


def _check(st, what):
    if st != 0:
        msg = lib().dgfs_last_error().decode(errors="replace")
        raise DgfsError(st, "%s failed: %s: %s" % (what, STATUS.get(st, st), msg))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------ C-named wrappers
def dgfs_probe_mma_rate(device=0, kind="tf32", iters=4096):
    """Measured tcgen05 issue rate (TFLOP/s) of kind 'tf32' or 'bf16' MMAs, M = 128, N = 256, all SMs."""
    v = ctypes.c_double(0.0)
    k = {"tf32": 0, "bf16": 1}[kind] if isinstance(kind, str) else int(kind)
    _check(lib().dgfs_probe_mma_rate(int(device), k, int(iters), ctypes.byref(v)), "dgfs_probe_mma_rate")
    return float(v.value)


def dgfs_debug_fail_alloc(n):
    """Host-side fault injection: the n-th allocation of the library from now fails (0: off)."""
    lib().dgfs_debug_fail_alloc(int(n))


def dgfs_debug_live_allocations():
    return int(lib().dgfs_debug_live_allocations())


def dgfs_version():
    return lib().dgfs_version().decode()


def dgfs_status_string(s):
    return lib().dgfs_status_string(int(s)).decode()


def dgfs_last_error():
    return lib().dgfs_last_error().decode(errors="replace")


def dgfs_plan_create(N, L, M, N_rho, masses, pairs, precision=FP64, max_points=1, device=0):
    S = len(masses)
    m = (ctypes.c_double * S)(*[float(x) for x in masses])
    pr = (dgfs_pair * (S * S))()
    for k, p in enumerate(pairs):
        pr[k].omega = float(p["omega"])
        pr[k].alpha = float(p["alpha"])
        pr[k].d = float(p.get("d", 1.0))
        pr[k].beta_override = float(p.get("beta_override", math.nan))
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    h = _P()
    _check(lib().dgfs_plan_create(ctypes.byref(h), int(N), float(L), int(M), int(N_rho), S,
                                  ctypes.cast(m, _P), ctypes.cast(pr, _P), int(precision),
                                  int(max_points), int(device)), "dgfs_plan_create")
    return h


def dgfs_plan_destroy(h):
    _check(lib().dgfs_plan_destroy(h), "dgfs_plan_destroy")


def dgfs_collide(h, P, f, Q, stream=None):
    _check(lib().dgfs_collide(h, int(P), _ptr(f), _ptr(Q), _stream(stream)), "dgfs_collide")


def dgfs_collide_noalloc(h, P, f, Q, stream=None):
    _check(lib().dgfs_collide_noalloc(h, int(P), _ptr(f), _ptr(Q), _stream(stream)), "dgfs_collide_noalloc")


def dgfs_collide_host(h, P, f_host, Q_host, stream=None):
    _check(lib().dgfs_collide_host(h, int(P), _ptr(f_host), _ptr(Q_host), _stream(stream)),
           "dgfs_collide_host")


def dgfs_collide_backward(h, P, f, dQ, df, domega=None, domega_on_host=False, stream=None):
    _check(lib().dgfs_collide_backward(h, int(P), _ptr(f), _ptr(dQ), _ptr(df),
                                       _ptr(domega) if domega is not None else None,
                                       1 if domega_on_host else 0, _stream(stream)), "dgfs_collide_backward")


def dgfs_moments(h, P, Q, out, stream=None):
    _check(lib().dgfs_moments(h, int(P), _ptr(Q), _ptr(out), _stream(stream)), "dgfs_moments")


def dgfs_plan_info(h):
    out = (ctypes.c_double * 16)()
    _check(lib().dgfs_plan_info(h, ctypes.cast(out, _P)), "dgfs_plan_info")
    keys = ("N", "L", "M", "N_rho", "S", "precision", "max_points", "workspace_bytes", "table_bytes", "chunk",
            "rs_blocks", "nterms", "groups_a", "groups_b", "tuned", "collapse")
    return {k: out[i] for i, k in enumerate(keys)}


def dgfs_plan_pair_tables(h, p, q, N, M, N_rho, with_b=True):
    import numpy as np
    n = N ** 3
    sc = np.empty(8)
    rho, wr = np.empty(N_rho), np.empty(N_rho)
    sig, ws = np.empty((M, 3)), np.empty(M)
    b = np.empty((N_rho, M, N, N, N), dtype=np.complex128) if with_b else None
    c = np.empty((N, N, N), dtype=np.complex128)
    cp = lambda a: a.ctypes.data_as(_P) if a is not None else None
    _check(lib().dgfs_plan_pair_tables(h, int(p), int(q), cp(sc), cp(rho), cp(wr), cp(sig), cp(ws), cp(b),
                                       cp(c)), "dgfs_plan_pair_tables")
    keys = ("R", "beta", "gamma", "eta", "dlogbeta", "cq", "cp", "overridden")
    return dict(scalars=dict(zip(keys, sc.tolist())), rho=rho, w_rho=wr, sigma=sig, w_sigma=ws, b=b, c=c)


def dgfs_plan_set_collapse(h, enable):
    _check(lib().dgfs_plan_set_collapse(h, int(bool(enable))), "dgfs_plan_set_collapse")


def dgfs_plan_set_hermitian(h, enable):
    _check(lib().dgfs_plan_set_hermitian(h, int(bool(enable))), "dgfs_plan_set_hermitian")


def dgfs_plan_set_kernel_variant(h, variant):
    _check(lib().dgfs_plan_set_kernel_variant(h, int(variant)), "dgfs_plan_set_kernel_variant")


def dgfs_plan_set_schedule(h, mode):
    _check(lib().dgfs_plan_set_schedule(h, int(mode)), "dgfs_plan_set_schedule")


def dgfs_plan_get_schedule(h):
    v = ctypes.c_int(0)
    _check(lib().dgfs_plan_get_schedule(h, ctypes.byref(v)), "dgfs_plan_get_schedule")
    return int(v.value)


def dgfs_debug_worklist_trace(buf):
    """buf: a CUDA int64 tensor of 4 words per task to record, or None (off)."""
    if buf is None:
        _check(lib().dgfs_debug_worklist_trace(None, 0), "dgfs_debug_worklist_trace")
    else:
        _check(lib().dgfs_debug_worklist_trace(_ptr(buf), buf.numel() * 8), "dgfs_debug_worklist_trace")


def dgfs_debug_worklist_chunk(rs_per_wave):
    _check(lib().dgfs_debug_worklist_chunk(int(rs_per_wave)), "dgfs_debug_worklist_chunk")


def dgfs_batch_set_schedule(h, mode):
    _check(lib().dgfs_batch_set_schedule(h, int(mode)), "dgfs_batch_set_schedule")


def dgfs_dealias_work_bytes(h, P, N):
    v = ctypes.c_size_t(0)
    _check(lib().dgfs_dealias_work_bytes(h, int(P), int(N), ctypes.byref(v)), "dgfs_dealias_work_bytes")
    return int(v.value)


def dgfs_collide_dealiased(h, P, N, f, Q, work, stream=None):
    _check(lib().dgfs_collide_dealiased(h, int(P), int(N), _ptr(f), _ptr(Q), _ptr(work),
                                        ctypes.c_size_t(work.numel() * work.element_size()), _stream(stream)),
           "dgfs_collide_dealiased")


def dgfs_plan_launch_count(h):
    v = ctypes.c_longlong(0)
    _check(lib().dgfs_plan_launch_count(h, ctypes.byref(v)), "dgfs_plan_launch_count")
    return int(v.value)


def dgfs_relax_step(h, P, f, Q, dt, stream=None):
    _check(lib().dgfs_relax_step(h, int(P), _ptr(f), _ptr(Q), float(dt), _stream(stream)), "dgfs_relax_step")


def dgfs_graph_capture(plans, Ps, fs, Qs, dt=0.0, steps=1):
    """plans: list of plan handles; fs, Qs: lists of device tensors (bound at capture)."""
    k = len(plans)
    ph = (_P * k)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    pp = (ctypes.c_int * k)(*[int(x) for x in Ps])
    fp = (_P * k)(*[t.data_ptr() for t in fs])
    qp = (_P * k)(*[t.data_ptr() for t in Qs])
    g = _P()
    _check(lib().dgfs_graph_capture(k, ctypes.cast(ph, _P), ctypes.cast(pp, _P), ctypes.cast(fp, _P),
                                    ctypes.cast(qp, _P), float(dt), int(steps), ctypes.byref(g)),
           "dgfs_graph_capture")
    return g


def dgfs_graph_launch(g, stream=None):
    _check(lib().dgfs_graph_launch(g, _stream(stream)), "dgfs_graph_launch")


def dgfs_graph_kernel_count(g):
    v = ctypes.c_longlong(0)
    _check(lib().dgfs_graph_kernel_count(g, ctypes.byref(v)), "dgfs_graph_kernel_count")
    return int(v.value)


def dgfs_graph_destroy(g):
    _check(lib().dgfs_graph_destroy(g), "dgfs_graph_destroy")


def dgfs_batch_create(plans, Ps, fs, Qs, dt=0.0):
    """plans: list of distinct plan handles; fs, Qs: lists of device tensors
    (their addresses are fixed in the batch)."""
    k = len(plans)
    ph = (_P * k)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    pp = (ctypes.c_int * k)(*[int(x) for x in Ps])
    fp = (_P * k)(*[t.data_ptr() for t in fs])
    qp = (_P * k)(*[t.data_ptr() for t in Qs])
    b = _P()
    _check(lib().dgfs_batch_create(k, ctypes.cast(ph, _P), ctypes.cast(pp, _P), ctypes.cast(fp, _P),
                                   ctypes.cast(qp, _P), float(dt), ctypes.byref(b)), "dgfs_batch_create")
    return b


def dgfs_batch_launch(b, stream=None):
    _check(lib().dgfs_batch_launch(b, _stream(stream)), "dgfs_batch_launch")


def dgfs_batch_destroy(b):
    _check(lib().dgfs_batch_destroy(b), "dgfs_batch_destroy")


def dgfs_plan_autotune(h, P, f, Q, stream=None):
    best = ctypes.c_double(0.0)
    _check(lib().dgfs_plan_autotune(h, int(P), _ptr(f), _ptr(Q), _stream(stream), ctypes.byref(best)),
           "dgfs_plan_autotune")
    return float(best.value)


def dgfs_plan_selftest_wait(h, expire, stream=None):
    _check(lib().dgfs_plan_selftest_wait(h, 1 if expire else 0, _stream(stream)), "dgfs_plan_selftest_wait")


def dgfs_plan_check(h):
    _check(lib().dgfs_plan_check(h), "dgfs_plan_check")


def dgfs_plan_profile(h, enable):
    _check(lib().dgfs_plan_profile(h, 1 if enable else 0), "dgfs_plan_profile")


def dgfs_plan_profile_read(h, max_classes=64):
    names = ctypes.create_string_buffer(64 * max_classes)
    counts = (ctypes.c_longlong * max_classes)()
    ms = (ctypes.c_double * max_classes)()
    nc = ctypes.c_int(0)
    _check(lib().dgfs_plan_profile_read(h, max_classes, ctypes.cast(names, _P), ctypes.cast(counts, _P),
                                        ctypes.cast(ms, _P), ctypes.byref(nc)), "dgfs_plan_profile_read")
    out = {}
    for c in range(nc.value):
        nm = names.raw[64 * c:64 * c + 64].split(b"\0", 1)[0].decode()
        out[nm] = (int(counts[c]), float(ms[c]))
    return out


# --------------------------------------------------------------- convenience
class Plan:
    """Owns a dgfs_plan; tensors in, tensors out (all computation in the library)."""

    def __init__(self, N, L, M, N_rho, masses, pairs, precision="fp64", max_points=1, device=0):
        self.N, self.L, self.M, self.N_rho = int(N), float(L), int(M), int(N_rho)
        self.S = len(masses)
        self.masses = list(masses)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.max_points = int(max_points)
        self.device = torch.device("cuda", device)
        self.dtype = torch.float64 if self.precision == FP64 else torch.float32
        self._h = dgfs_plan_create(N, L, M, N_rho, masses, pairs, self.precision, max_points, device)

    def close(self):
        if getattr(self, "_h", None):
            dgfs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self):
        return self.N ** 3

    def _check_f(self, f):
        if not (f.is_cuda and f.dtype == self.dtype and f.is_contiguous()):
            raise ValueError("f must be a contiguous %s CUDA tensor" % self.dtype)
        P = f.shape[0]
        if f.numel() != P * self.S * self.n:
            raise ValueError("f must have shape [P][S][N][N][N]")
        return P

    def collide(self, f, Q=None, stream=None):
        P = self._check_f(f)
        if Q is None:
            Q = torch.empty((P, self.S, self.S, self.N, self.N, self.N), dtype=self.dtype, device=f.device)
        dgfs_collide(self._h, P, f, Q, stream)
        return Q

    def collide_host(self, f_host, Q_host, stream=None):
        P = f_host.shape[0]
        dgfs_collide_host(self._h, P, f_host, Q_host, stream)
        return Q_host

    def backward(self, f, dQ, stream=None):
        P = self._check_f(f)
        df = torch.empty_like(f)
        dom = torch.zeros(self.S * self.S, dtype=torch.float64, device=f.device)
        dgfs_collide_backward(self._h, P, f, dQ.contiguous(), df, dom, False, stream)
        return df, dom

    def moments(self, Q, stream=None):
        P = Q.shape[0]
        out = torch.empty((P, self.S, self.S, 5), dtype=torch.float64, device=Q.device)
        dgfs_moments(self._h, P, Q, out, stream)
        return out

    def info(self):
        return dgfs_plan_info(self._h)

    def pair_tables(self, p, q, with_b=True):
        return dgfs_plan_pair_tables(self._h, p, q, self.N, self.M, self.N_rho, with_b)

    def launch_count(self):
        return dgfs_plan_launch_count(self._h)

    def set_collapse(self, enable):
        dgfs_plan_set_collapse(self._h, enable)

    def set_hermitian(self, enable):
        """Switch the declared Hermitian form (Nyquist planes removed) on or off."""
        dgfs_plan_set_hermitian(self._h, enable)

    def set_kernel_variant(self, variant):
        dgfs_plan_set_kernel_variant(self._h, variant)

    def set_schedule(self, mode):
        """0: one launch per stage and job; 1: one persistent work-list launch."""
        dgfs_plan_set_schedule(self._h, mode)

    def schedule(self):
        return dgfs_plan_get_schedule(self._h)

    def collide_dealiased(self, f, N, Q=None, work=None):
        """Linear-convolution operator on the N grid (this plan is built at 3N/2)."""
        if not (f.is_cuda and f.dtype == self.dtype and f.is_contiguous() and f.shape[2:] == (N, N, N)):
            raise ValueError("f must be a contiguous %s CUDA tensor [P][S][N][N][N]" % self.dtype)
        P = f.shape[0]
        if Q is None:
            Q = torch.empty((P, self.S, self.S, N, N, N), dtype=self.dtype, device=f.device)
        if work is None:
            work = torch.empty(dgfs_dealias_work_bytes(self._h, P, N), dtype=torch.uint8, device=f.device)
        dgfs_collide_dealiased(self._h, P, N, f, Q, work)
        return Q

    def check(self):
        dgfs_plan_check(self._h)

    def relax_step(self, f, Q, dt, stream=None):
        dgfs_relax_step(self._h, f.shape[0], f, Q, dt, stream)

    def autotune(self, f, Q=None, stream=None):
        if Q is None:
            Q = torch.empty((f.shape[0], self.S, self.S, self.N, self.N, self.N), dtype=self.dtype,
                            device=f.device)
        return dgfs_plan_autotune(self._h, f.shape[0], f, Q, stream)

    def profile(self, enable=True):
        dgfs_plan_profile(self._h, enable)

    def profile_read(self):
        return dgfs_plan_profile_read(self._h)


# ------------------------------------------------------------ 1-D DG transport
class Batch:
    """A batched work list over distinct plans (dgfs_batch_create): `plans`
    are Plan objects, fs and Qs device tensors whose addresses stay fixed."""

    def __init__(self, plans, fs, Qs, dt=0.0):
        self.plans, self.fs, self.Qs = list(plans), list(fs), list(Qs)
        if not (len(self.plans) == len(self.fs) == len(self.Qs)):
            raise ValueError("plans, fs and Qs must have the same length")
        for pl, f, Q in zip(self.plans, self.fs, self.Qs):
            P = pl._check_f(f)
            if not (Q.is_cuda and Q.dtype == pl.dtype and Q.is_contiguous() and Q.numel() == P * pl.S * pl.S * pl.n):
                raise ValueError("Q must be a contiguous %s CUDA tensor of shape [P][S][S][N][N][N]" % pl.dtype)
        self._h = dgfs_batch_create([pl._h for pl in self.plans], [f.shape[0] for f in self.fs], self.fs,
                                    self.Qs, dt)

    def launch(self, stream=None):
        dgfs_batch_launch(self._h, stream)

    def set_schedule(self, mode):
        """0: per-stage launches per round; 1: persistent work lists (default)."""
        dgfs_batch_set_schedule(self._h, mode)

    def close(self):
        if getattr(self, "_h", None):
            dgfs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dgfs_dg_create(plan_h, Ne, K, x0, x1, walls):
    """walls: ((T_left, (ux, uy, uz)), (T_right, (ux, uy, uz)))."""
    import numpy as np
    w = np.array([walls[0][0], *walls[0][1], walls[1][0], *walls[1][1]], dtype=np.float64)
    h = _P()
    _check(lib().dgfs_dg_create(ctypes.byref(h), plan_h, int(Ne), int(K), float(x0), float(x1),
                                w.ctypes.data_as(_P)), "dgfs_dg_create")
    return h


def dgfs_dg_destroy(h):
    _check(lib().dgfs_dg_destroy(h), "dgfs_dg_destroy")


def dgfs_dg_nodes(h, P):
    import numpy as np
    x = np.empty(P)
    _check(lib().dgfs_dg_nodes(h, x.ctypes.data_as(_P)), "dgfs_dg_nodes")
    return x


def dgfs_dg_rhs(h, f, Q, rhs, stream=None):
    _check(lib().dgfs_dg_rhs(h, _ptr(f), _ptr(Q) if Q is not None else None, _ptr(rhs), _stream(stream)),
           "dgfs_dg_rhs")


def dgfs_dg_step(h, f, dt, with_collisions=True, stream=None):
    _check(lib().dgfs_dg_step(h, _ptr(f), float(dt), int(bool(with_collisions)), _stream(stream)), "dgfs_dg_step")


def _opt(t):
    return _ptr(t) if t is not None else None


def dgfs_dg_traces(h, f, left, right, stream=None):
    _check(lib().dgfs_dg_traces(h, _ptr(f), _opt(left), _opt(right), _stream(stream)), "dgfs_dg_traces")


def dgfs_dg_rhs_halo(h, f, Q, rhs, halo_left, halo_right, stream=None):
    _check(lib().dgfs_dg_rhs_halo(h, _ptr(f), _opt(Q), _ptr(rhs), _opt(halo_left), _opt(halo_right),
                                  _stream(stream)), "dgfs_dg_rhs_halo")


def dgfs_dg_stage(h, f_in, f0, out, a0, a1, dt, with_collisions, halo_left, halo_right, stream=None):
    _check(lib().dgfs_dg_stage(h, _ptr(f_in), _opt(f0), _ptr(out), float(a0), float(a1), float(dt),
                               int(bool(with_collisions)), _opt(halo_left), _opt(halo_right), _stream(stream)),
           "dgfs_dg_stage")


class Slab:
    """Owns a DG discretisation of [x0, x1] (Ne elements x K Gauss nodes) built on a Plan."""

    def __init__(self, plan, Ne, K, x0, x1, walls):
        self.plan, self.Ne, self.K = plan, int(Ne), int(K)
        self.P = self.Ne * self.K
        self._h = dgfs_dg_create(plan._h, Ne, K, x0, x1, walls)
        self.x = dgfs_dg_nodes(self._h, self.P)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            try:
                dgfs_dg_destroy(h)
            except Exception:
                pass
            self._h = None

    def _check_f(self, f):
        p = self.plan
        shape = (self.P, p.S, p.N, p.N, p.N)
        if tuple(f.shape) != shape or f.dtype != p.dtype or not f.is_cuda or not f.is_contiguous():
            raise ValueError("f must be a contiguous %s CUDA tensor of shape %s" % (p.dtype, shape))

    def rhs(self, f, Q=None, out=None):
        self._check_f(f)
        if out is None:
            out = torch.empty_like(f)
        dgfs_dg_rhs(self._h, f, Q, out)
        return out

    def step(self, f, dt, with_collisions=True):
        self._check_f(f)
        dgfs_dg_step(self._h, f, dt, with_collisions)
        return f

    def traces(self, f):
        """(left, right) boundary traces, FP64 [S][N^3] device tensors."""
        self._check_f(f)
        p = self.plan
        left = torch.empty((p.S, p.N ** 3), dtype=torch.float64, device=f.device)
        right = torch.empty_like(left)
        dgfs_dg_traces(self._h, f, left, right)
        return left, right

    def rhs_halo(self, f, Q=None, halo_left=None, halo_right=None, out=None):
        self._check_f(f)
        if out is None:
            out = torch.empty_like(f)
        dgfs_dg_rhs_halo(self._h, f, Q, out, halo_left, halo_right)
        return out

    def stage(self, f_in, f0, out, a0, a1, dt, with_collisions=True, halo_left=None, halo_right=None):
        self._check_f(f_in)
        self._check_f(out)
        dgfs_dg_stage(self._h, f_in, f0, out, a0, a1, dt, with_collisions, halo_left, halo_right)
        return out
