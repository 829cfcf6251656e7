"""Python binding of the C ABI in ``include/mqs.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA library
``_lib/libmqs.so``.  The module-level functions carry the C names
(``mqs_create``, ``mqs_upload_mesh``, ...); ``Context`` wraps them with
handles and numpy / torch arrays.  Arrays may be numpy arrays (host) or CUDA
torch tensors (device); device tensors are passed as raw device pointers.

The library must be built first (``__graft_entry__.build()`` or
``python -m paper_2507_19246_gb300.build``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

# The banded Parareal driver keeps up to 16 fine chunks in flight on streams
# of their own.  CUDA multiplexes streams onto CUDA_DEVICE_MAX_CONNECTIONS
# hardware queues (8 unless set), and streams that share a queue serialise
# behind each other's event waits.  The setting is read when CUDA initialises
# in the process, so it only takes effect if nothing has initialised CUDA yet;
# an explicit setting by the caller is kept.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np

from . import build as _build

MQS_OK, MQS_EINVAL, MQS_ENOMEM, MQS_ECUDA, MQS_ENOTCONV = 0, -1, -2, -3, -4
MQS_FP64, MQS_MIXED = 0, 1
MQS_QOI_ENERGY, MQS_QOI_JOULE = 0, 1
MQS_ST_NOTCONV, MQS_ST_NONFINITE, MQS_ST_NOTSPD, MQS_ST_TIMEOUT = 1, 2, 4, 8
MQS_SOLVER_PCG, MQS_SOLVER_BANDED = 0, 1
MQS_TEST_HOOK_STALL = 1
MQS_REQ_LEVEL, MQS_REQ_SLICE = 0, 1

_lib = None
_P = C.c_void_p
_i32, _i64, _f64 = C.c_int32, C.c_int64, C.c_double

_SIGS = {
    "mqs_last_error": (C.c_char_p, []),
    "mqs_create": (C.c_int, [C.POINTER(_P), C.c_int, _P]),
    "mqs_set_stream": (C.c_int, [_P, _P]),
    "mqs_destroy": (C.c_int, [_P]),
    "mqs_upload_mesh": (C.c_int, [_P, _i32, _P, _i32, _P, _P, _i32, _P, _P, _P, _i32,
                                  C.POINTER(_i32)]),
    "mqs_mesh_info": (C.c_int, [_P, _i32, C.POINTER(_i32), C.POINTER(_i64)]),
    "mqs_mesh_bandwidth": (C.c_int, [_P, _i32, C.POINTER(_i32)]),
    "mqs_set_solver": (C.c_int, [_P, _i32, _i32]),
    "mqs_set_samples": (C.c_int, [_P, _i32, _i32, _i32, _P, C.POINTER(_i32)]),
    "mqs_set_time": (C.c_int, [_P, _i32, _f64, _f64, _f64, _i32]),
    "mqs_propagate": (C.c_int, [_P, _i32, _i32, _f64, _f64, _i32, _i32, _i32, _f64, _i32, _f64,
                                _i32, C.POINTER(_i32)]),
    "mqs_read_qoi": (C.c_int, [_P, _i32, _P, _P]),
    "mqs_read_state": (C.c_int, [_P, _i32, _i32, _P]),
    "mqs_read_stats": (C.c_int, [_P, _i32, _P]),
    "mqs_apply": (C.c_int, [_P, _i32, _i32, _f64, _P, _P]),
    "mqs_mlmc_reset": (C.c_int, [_P, _i32]),
    "mqs_mlmc_accumulate": (C.c_int, [_P, _i32, _i32]),
    "mqs_mlmc_readout": (C.c_int, [_P, _P, C.POINTER(_f64), C.POINTER(_f64)]),
    "mqs_profile": (C.c_int, [_P, _i32]),
    "mqs_profile_read": (C.c_int, [_P, _P]),
    "mqs_profile_trace": (C.c_int, [_P, _i32, _P, _i32, C.POINTER(_i32)]),
    "mqs_measure_peak": (C.c_int, [_i32, _P, _i32, C.POINTER(_f64)]),
    "mqs_propagate_noalloc": (C.c_int, [_i32, _P, _i32, _P, _P, _i64, _i32, _P, _P, _P, _P, _i32,
                                        _P, _P, _P, _f64, _f64, _i32, _f64, _i32, _f64, _i32, _P,
                                        _P, _P]),
    "mqs_set_test_hook": (C.c_int, [_P, _i32]),
    "mqs_lane_slots": (C.c_int, [_P, _i32, C.POINTER(_i32)]),
    "mqs_server_create": (C.c_int, [_P, _i64, _i32, _i32, _f64, C.POINTER(_P)]),
    "mqs_server_destroy": (C.c_int, [_P]),
    "mqs_server_submit": (C.c_int, [_P, _i32, _i32, _P, _i32, _i32, _f64, _f64, _i32, _f64, _i32,
                                    _i64, _P, _P, C.POINTER(_i64)]),
    "mqs_server_progress": (C.c_int, [_P, C.POINTER(_i32), C.POINTER(_i32)]),
    "mqs_server_footprint": (C.c_int, [_P, _i32, _i32, _i32, C.POINTER(_i64)]),
    "mqs_server_poll": (C.c_int, [_P, _i32, _P, _P, _P, _P, C.POINTER(_i32)]),
    "mqs_free_batch": (C.c_int, [_P, _i32]),
    "mqs_free_mesh": (C.c_int, [_P, _i32]),
}


class MQSError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} returned {code}: {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libmqs.so (built in-tree); raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _check(fn, code):
    if code != MQS_OK:
        raise MQSError(fn, code, load().mqs_last_error().decode(errors="replace"))


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor (host or CUDA)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


# ----------------------------------------------------------------- C names
def mqs_last_error() -> str:
    return load().mqs_last_error().decode(errors="replace")


def mqs_create(device: int = 0, stream: int = None) -> int:
    h = _P()
    _check("mqs_create", load().mqs_create(C.byref(h), device, stream))
    return h.value


def mqs_set_stream(ctx, stream):
    _check("mqs_set_stream", load().mqs_set_stream(ctx, stream))


def mqs_destroy(ctx):
    _check("mqs_destroy", load().mqs_destroy(ctx))


def mqs_upload_mesh(ctx, mesh) -> int:
    xy = _host(mesh.xy, np.float64)
    tri = _host(mesh.tri, np.int32)
    reg = _host(mesh.region, np.int32)
    dr = _host(mesh.dirichlet, np.uint8)
    ph = _host(mesh.src_phase, np.int32)
    cf = _host(mesh.src_coef, np.float64)
    out = _i32()
    _check("mqs_upload_mesh", load().mqs_upload_mesh(
        ctx, xy.shape[0], _ptr(xy), tri.shape[0], _ptr(tri), _ptr(reg), mesh.n_regions, _ptr(dr),
        _ptr(ph), _ptr(cf), mesh.n_phases, C.byref(out)))
    return out.value


def mqs_mesh_info(ctx, mesh_id):
    n, z = _i32(), _i64()
    _check("mqs_mesh_info", load().mqs_mesh_info(ctx, mesh_id, C.byref(n), C.byref(z)))
    return n.value, z.value


def mqs_mesh_bandwidth(ctx, mesh_id) -> int:
    bw = _i32()
    _check("mqs_mesh_bandwidth", load().mqs_mesh_bandwidth(ctx, mesh_id, C.byref(bw)))
    return bw.value


def mqs_set_solver(ctx, batch, solver):
    _check("mqs_set_solver", load().mqs_set_solver(ctx, batch, solver))


def mqs_set_samples(ctx, mesh_id, params) -> int:
    if isinstance(params, np.ndarray) or not hasattr(params, "data_ptr"):
        params = _host(params, np.float64)
    ns, npar = params.shape
    out = _i32()
    _check("mqs_set_samples", load().mqs_set_samples(ctx, mesh_id, ns, npar, _ptr(params),
                                                     C.byref(out)))
    return out.value


def mqs_set_time(ctx, batch, t0, t_end, freq_hz, qoi_kind):
    _check("mqs_set_time", load().mqs_set_time(ctx, batch, t0, t_end, freq_hz, qoi_kind))


def mqs_propagate(ctx, batch, level, dt_level, dt_prev=0.0, n_slices=1, coarse_factor=1,
                  max_par_iters=1, par_tol=0.0, precision=MQS_FP64, cg_tol=1e-12,
                  cg_max_iters=5000) -> int:
    it = _i32()
    _check("mqs_propagate", load().mqs_propagate(
        ctx, batch, level, dt_level, dt_prev, n_slices, coarse_factor, max_par_iters, par_tol,
        precision, cg_tol, cg_max_iters, C.byref(it)))
    return it.value


def mqs_read_qoi(ctx, batch, qoi, status=None):
    _check("mqs_read_qoi", load().mqs_read_qoi(ctx, batch, _ptr(qoi), _ptr(status)))


def mqs_read_state(ctx, batch, which, a):
    _check("mqs_read_state", load().mqs_read_state(ctx, batch, which, _ptr(a)))


MQS_N_STATS = 8


def mqs_read_stats(ctx, batch):
    s = np.zeros(MQS_N_STATS)
    _check("mqs_read_stats", load().mqs_read_stats(ctx, batch, _ptr(s)))
    return s


def mqs_apply(ctx, batch, which, dt, x, y):
    _check("mqs_apply", load().mqs_apply(ctx, batch, which, dt, _ptr(x), _ptr(y)))


def mqs_mlmc_reset(ctx, n_levels):
    _check("mqs_mlmc_reset", load().mqs_mlmc_reset(ctx, n_levels))


def mqs_mlmc_accumulate(ctx, batch, level):
    _check("mqs_mlmc_accumulate", load().mqs_mlmc_accumulate(ctx, batch, level))


def mqs_mlmc_readout(ctx, n_levels):
    lv = np.zeros((n_levels, 3))
    est, rmse = _f64(), _f64()
    _check("mqs_mlmc_readout", load().mqs_mlmc_readout(ctx, _ptr(lv), C.byref(est), C.byref(rmse)))
    return lv, est.value, rmse.value


def mqs_profile(ctx, enable):
    _check("mqs_profile", load().mqs_profile(ctx, int(bool(enable))))


def mqs_profile_read(ctx):
    out = np.zeros(7)
    _check("mqs_profile_read", load().mqs_profile_read(ctx, _ptr(out)))
    return out


def mqs_profile_trace(ctx, kind, max_launches=100000):
    out = np.zeros(2 * max_launches)
    cnt = _i32()
    _check("mqs_profile_trace", load().mqs_profile_trace(ctx, kind, _ptr(out), max_launches,
                                                         C.byref(cnt)))
    return out[:2 * min(cnt.value, max_launches)].reshape(-1, 2)


def mqs_measure_peak(device, stream, precision):
    out = _f64()
    _check("mqs_measure_peak", load().mqs_measure_peak(device, stream, precision, C.byref(out)))
    return out.value


def mqs_propagate_noalloc(device, stream, n, rowptr, colidx, nnz, n_lanes, A, M, K, Dinv,
                          n_phases, F, src_amp, src_phase, t0, dt, n_steps, freq_hz, qoi_kind,
                          cg_tol, cg_max_iters, a_out, qoi_out, status_out=None):
    """Sequential stepping that allocates no memory (see include/mqs.h);
    array arguments are device tensors except src_amp/src_phase (host or device)."""
    _check("mqs_propagate_noalloc", load().mqs_propagate_noalloc(
        device, stream, n, _ptr(rowptr), _ptr(colidx), nnz, n_lanes, _ptr(A), _ptr(M), _ptr(K),
        _ptr(Dinv), n_phases, _ptr(F), _ptr(src_amp), _ptr(src_phase), t0, dt, n_steps, freq_hz,
        qoi_kind, cg_tol, cg_max_iters, _ptr(a_out), _ptr(qoi_out), _ptr(status_out)))


def mqs_lane_slots(ctx, precision=MQS_FP64) -> int:
    out = _i32()
    _check("mqs_lane_slots", load().mqs_lane_slots(ctx, precision, C.byref(out)))
    return out.value


def mqs_set_test_hook(ctx, hook):
    _check("mqs_set_test_hook", load().mqs_set_test_hook(ctx, int(hook)))


def mqs_server_create(ctx, hbm_budget=0, n_streams=8, max_batch_lanes=608, freq_hz=50.0):
    out = _P()
    _check("mqs_server_create", load().mqs_server_create(ctx, int(hbm_budget), n_streams,
                                                         max_batch_lanes, freq_hz, C.byref(out)))
    return out.value


def mqs_server_destroy(srv):
    _check("mqs_server_destroy", load().mqs_server_destroy(srv))


def mqs_server_submit(srv, mesh_id, params, kind, qoi_kind, t0, dt, n_steps, dt_prev=0.0,
                      n_steps_prev=0, k0=0, a_init=None, a_out=None) -> int:
    p = _host(params, np.float64)
    ai = None if a_init is None else _host(a_init, np.float64)
    rid = _i64()
    _check("mqs_server_submit", load().mqs_server_submit(
        srv, mesh_id, p.size, _ptr(p), kind, qoi_kind, t0, dt, n_steps, dt_prev, n_steps_prev, k0,
        _ptr(ai) if ai is not None else None, _ptr(a_out) if a_out is not None else None,
        C.byref(rid)))
    return rid.value


def mqs_server_footprint(srv, mesh_id, qoi_kind, lanes) -> int:
    out = _i64()
    _check("mqs_server_footprint", load().mqs_server_footprint(srv, mesh_id, qoi_kind, lanes,
                                                               C.byref(out)))
    return out.value


def mqs_server_progress(srv):
    inf, q = _i32(), _i32()
    _check("mqs_server_progress", load().mqs_server_progress(srv, C.byref(inf), C.byref(q)))
    return inf.value, q.value


def mqs_server_poll(srv, max_n=4096):
    ids = np.zeros(max_n, dtype=np.int64)
    qoi = np.zeros((max_n, 2))
    st = np.zeros(max_n, dtype=np.int32)
    tm = np.zeros((max_n, 3))
    cnt = _i32()
    _check("mqs_server_poll", load().mqs_server_poll(srv, max_n, _ptr(ids), _ptr(qoi), _ptr(st),
                                                     _ptr(tm), C.byref(cnt)))
    c = cnt.value
    return ids[:c], qoi[:c], st[:c], tm[:c]


class Server:
    """Request server on a context (mqs_server_*): submit level samples and
    Parareal slices, call progress() often, collect results with poll()."""

    def __init__(self, ctx, hbm_budget=0, n_streams=8, max_batch_lanes=608, freq_hz=50.0):
        self.h = mqs_server_create(ctx.h, hbm_budget, n_streams, max_batch_lanes, freq_hz)

    def close(self):
        if self.h:
            mqs_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, mesh_id, params, kind, qoi_kind, t0, dt, n_steps, **kw):
        return mqs_server_submit(self.h, mesh_id, params, kind, qoi_kind, t0, dt, n_steps, **kw)

    def progress(self):
        return mqs_server_progress(self.h)

    def footprint(self, mesh_id, qoi_kind, lanes):
        return mqs_server_footprint(self.h, mesh_id, qoi_kind, lanes)

    def poll(self, max_n=4096):
        return mqs_server_poll(self.h, max_n)

    def drain(self, sleep_s=0.0005, timeout_s=600.0):
        """progress() until nothing is queued or in flight; all results."""
        import time
        out = {}
        t0 = time.time()
        while True:
            inf, q = self.progress()
            for i, qq, st, tm in zip(*self.poll()):
                out[int(i)] = (qq.copy(), int(st), tm.copy())
            if inf == 0 and q == 0:
                for i, qq, st, tm in zip(*self.poll()):
                    out[int(i)] = (qq.copy(), int(st), tm.copy())
                return out
            if time.time() - t0 > timeout_s:
                raise TimeoutError("server did not drain")
            time.sleep(sleep_s)


def mqs_free_batch(ctx, batch):
    _check("mqs_free_batch", load().mqs_free_batch(ctx, batch))


def mqs_free_mesh(ctx, mesh_id):
    _check("mqs_free_mesh", load().mqs_free_mesh(ctx, mesh_id))


# ----------------------------------------------------------------- convenience
class Context:
    """A library context on one GPU; methods mirror the C entry points."""

    def __init__(self, device: int = 0, stream=None):
        self.device = device
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = None
        self.h = mqs_create(device, stream)
        self._n = {}

    def close(self):
        if self.h:
            mqs_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        mqs_set_stream(self.h, stream)

    def upload_mesh(self, mesh) -> int:
        return mqs_upload_mesh(self.h, mesh)

    def mesh_info(self, mesh_id):
        return mqs_mesh_info(self.h, mesh_id)

    def mesh_bandwidth(self, mesh_id):
        return mqs_mesh_bandwidth(self.h, mesh_id)

    def set_solver(self, batch, solver):
        mqs_set_solver(self.h, batch, solver)

    def set_samples(self, mesh_id, params) -> int:
        b = mqs_set_samples(self.h, mesh_id, params)
        self._n[b] = (mesh_id, int(params.shape[0]))
        return b

    def set_time(self, batch, t0, t_end, freq_hz=50.0, qoi_kind=MQS_QOI_JOULE):
        mqs_set_time(self.h, batch, t0, t_end, freq_hz, qoi_kind)

    def propagate(self, batch, level, dt_level, **kw) -> int:
        return mqs_propagate(self.h, batch, level, dt_level, **kw)

    def read_qoi(self, batch):
        ns = self._n[batch][1]
        q = np.zeros((ns, 2))
        st = np.zeros(ns, dtype=np.int32)
        mqs_read_qoi(self.h, batch, q, st)
        return q, st

    def read_state(self, batch, which=0):
        mesh_id, ns = self._n[batch]
        n, _ = self.mesh_info(mesh_id)
        a = np.zeros((ns, n))
        mqs_read_state(self.h, batch, which, a)
        return a

    def read_stats(self, batch):
        return mqs_read_stats(self.h, batch)

    def apply(self, batch, which, dt, x):
        x = _host(x, np.float64)
        y = np.zeros_like(x)
        mqs_apply(self.h, batch, which, dt, x, y)
        return y

    def mlmc_reset(self, n_levels):
        self._levels = n_levels
        mqs_mlmc_reset(self.h, n_levels)

    def mlmc_accumulate(self, batch, level):
        mqs_mlmc_accumulate(self.h, batch, level)

    def mlmc_readout(self):
        return mqs_mlmc_readout(self.h, self._levels)

    def profile(self, enable=True):
        mqs_profile(self.h, enable)

    def profile_read(self):
        """[launches, step-kernel launches, ms, sweep-kernel launches, ms,
        step-kernel covered ms, sweep-kernel covered ms]"""
        return mqs_profile_read(self.h)

    def lane_slots(self, precision=MQS_FP64):
        return mqs_lane_slots(self.h, precision)

    def set_test_hook(self, hook):
        mqs_set_test_hook(self.h, hook)

    def profile_trace(self, kind):
        """[launches][2]: start and end (ms) of each recorded launch of a kind."""
        return mqs_profile_trace(self.h, kind)

    def free_batch(self, batch):
        mqs_free_batch(self.h, batch)
        self._n.pop(batch, None)

    def free_mesh(self, mesh_id):
        mqs_free_mesh(self.h, mesh_id)
