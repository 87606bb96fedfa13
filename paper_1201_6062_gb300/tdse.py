"""ctypes binding of the C ABI in include/tdse.h (argument marshalling only).

Every computation runs in the CUDA kernels of lib/libtdse.so; PyTorch only
provides device memory and streams.  Importing this module loads the library
and raises ImportError if it has not been built (there is no CPU fallback).
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libtdse.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libtdse.so is not built (run __graft_entry__.build() or python paper_1201_6062_gb300/build.py)")

_lib = ctypes.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTSUP = range(6)
RK4, TAYLOR, LANCZOS = 0, 1, 2
HOLD_LEFT, HOLD_MID = 0, 1
FP64, FP32, DF32, BF16X3 = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp32": FP32, "df32": DF32, "bf16x3": BF16X3}
SCHEMES = {"rk4": RK4, "taylor": TAYLOR, "lanczos": LANCZOS}
LENGTH, VELOCITY = 0, 1
GAUGES = {"length": LENGTH, "velocity": VELOCITY}

_vp = ctypes.c_void_p
_i = ctypes.c_int
_l = ctypes.c_long
_d = ctypes.c_double

_SIGS = {
    "tdse_version": ([], _i),
    "tdse_last_error": ([], ctypes.c_char_p),
    "tdse_create": ([_vp, _vp, _i, _i, _i, ctypes.POINTER(_vp)], _i),
    "tdse_destroy": ([_vp], None),
    "tdse_size": ([_vp], _l),
    "tdse_hmatvec": ([_vp, _d, _vp, _vp, _i, _vp], _i),
    "tdse_propagate": ([_vp, _vp, _vp, _i, _d, _l, _i, _i, _i, _vp], _i),
    "tdse_propagate_host": ([_vp, _vp, _vp, _i, _d, _l, _i, _i, _i, _vp], _i),
    "tdse_norm": ([_vp, _vp, _i, _vp, _vp], _i),
    "tdse_sync": ([_vp, _vp], _i),
    "tdse_populations": ([_vp, _vp, _i, _vp, _vp, _vp, _vp, _vp], _i),
    "tdse_propagate_batch": ([_vp, _vp, _vp, _i, _i, _d, _l, _i, _i, _i, _vp], _i),
    "tdse_adjoint": ([_vp, _vp, _vp, _i, _d, _l, _i, _i, _i, _vp, _i, _vp, _vp, _vp, _vp], _i),
    "tdse_profile_enable": ([_vp, _i], _i),
    "tdse_profile_read": ([_vp, ctypes.POINTER(_d), ctypes.POINTER(_l), ctypes.POINTER(_l)], _i),
    "tdse_set_gauge": ([_vp, _i], _i),
    "tdse_vector_potential_sin2": ([_d, _d, _d, _d, _d, _l, _vp, _vp], _i),
    "tdse_group_create": ([_vp, _i, ctypes.POINTER(_vp)], _i),
    "tdse_group_destroy": ([_vp], None),
    "tdse_group_propagate": ([_vp, _vp, _vp, _i, _d, _l, _vp], _i),
    "tdse_plan_info": ([_vp] + [ctypes.POINTER(_i)] * 5, _i),
    "tdse_set_device_memory_limit": ([ctypes.c_longlong], _i),
    "tdse_device_memory_in_use": ([], ctypes.c_longlong),
    "tdse_inject_wait_timeout": ([_vp, _l, _vp], _i),
    "tdse_group_plan_info": ([_vp, _i] + [ctypes.POINTER(_i)] * 7, _i),
    "tdse_group_set_persistent": ([_vp, _i, _i, _i], _i),
    "tdse_set_batch_persistent": ([_vp, _i], _i),
    "tdse_group_persistent_info": ([_vp] + [ctypes.POINTER(_i)] * 5, _i),
}
class _FieldFn(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("E0", ctypes.c_double), ("omega", ctypes.c_double),
                ("cycles", ctypes.c_double), ("a0", ctypes.c_double)]


class _RkfStats(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_long), ("rejected", ctypes.c_long), ("forced", ctypes.c_long),
                ("t", ctypes.c_double), ("dt", ctypes.c_double), ("err", ctypes.c_double), ("a", ctypes.c_double)]


FIELD_KINDS = {"sin2": 0, "const": 1}
_SIGS["tdse_propagate_rkf45"] = ([_vp, _vp, ctypes.POINTER(_FieldFn), _d, _d, _d, _d, _d, _d, _l,
                                  ctypes.POINTER(_RkfStats), _vp], _i)
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class TDSEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("tdse status %d: %s" % (status, msg))
        self.status = status


def _check(st):
    if st != OK:
        raise TDSEError(st, _lib.tdse_last_error().decode())


def version():
    return _lib.tdse_version()


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_c(t, N, B=None, name="c"):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.complex128:
        raise TypeError("%s must be a CUDA complex128 tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    want = N if B is None else B * N
    if t.numel() != want:
        raise ValueError("%s has %d amplitudes, expected %d" % (name, t.numel(), want))
    return t


def _dev_f64(t, n, name):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float64:
        raise TypeError("%s must be a CUDA float64 tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if n is not None and t.numel() != n:
        raise ValueError("%s has %d samples, expected %d" % (name, t.numel(), n))
    return t


def set_device_memory_limit(nbytes):
    """Cap the device memory all contexts and groups hold together (0: no cap);
    allocations beyond it fail with ENOMEM."""
    _check(_lib.tdse_set_device_memory_limit(int(nbytes)))


def device_memory_in_use():
    return int(_lib.tdse_device_memory_in_use())


def vector_potential_sin2(E0, omega, cycles, t0, h, nsamples, out=None, stream=None):
    """A(t0 + k h) = -int_0^t E for the sin^2 pulse, k < nsamples (Sec. 5,
    five-point Gauss-Legendre per interval); a CUDA float64 tensor."""
    if out is None:
        out = torch.empty(int(nsamples), dtype=torch.float64, device="cuda")
    _dev_f64(out, int(nsamples), "out")
    _check(_lib.tdse_vector_potential_sin2(float(E0), float(omega), float(cycles), float(t0), float(h),
                                           int(nsamples), _ptr(out), _stream(stream)))
    return out


class Hamiltonian:
    """One field-free Hamiltonian (energies E, upper dipole blocks U_l)
    resident on the GPU in the storage format of `precision`."""

    def __init__(self, energies, dipoles, lmax, n, precision="fp64"):
        E = np.ascontiguousarray(energies, dtype=np.float64).reshape(-1)
        if E.size != (lmax + 1) * n:
            raise ValueError("energies must have (lmax+1)*n entries")
        if lmax > 0:
            U = np.ascontiguousarray(dipoles, dtype=np.float64).reshape(lmax, n, n)
            up = U.ctypes.data_as(_vp)
        else:
            U, up = None, None
        self.lmax, self.n, self.N = int(lmax), int(n), (lmax + 1) * n
        self.precision = precision
        h = _vp()
        _check(_lib.tdse_create(E.ctypes.data_as(_vp), up, int(lmax), int(n), PRECISIONS[precision], ctypes.byref(h)))
        self._h = h
        self.energies = E
        self.gauge = "length"

    def close(self):
        if getattr(self, "_h", None):
            _lib.tdse_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def propagate_rkf45(self, c, t0, t1, dt0, tol, field="sin2", E0=0.0, omega=1.0, cycles=10, a0=0.0,
                        dt_min=0.0, dt_max=float("inf"), max_attempts=10 ** 7, stream=None):
        """Adaptive Runge-Kutta-Fehlberg 4(5) from t0 to t1 (synchronises the
        stream).  Returns dict(accepted, rejected, forced, t, dt, err, A)."""
        c = _dev_c(c, self.N)
        fn = _FieldFn(FIELD_KINDS[field], float(E0), float(omega), float(cycles), float(a0))
        st = _RkfStats()
        _check(_lib.tdse_propagate_rkf45(self._h, _ptr(c), ctypes.byref(fn), float(t0), float(t1), float(dt0),
                                         float(tol), float(dt_min), float(min(dt_max, 1e300)), int(max_attempts),
                                         ctypes.byref(st), _stream(stream)))
        return dict(accepted=st.accepted, rejected=st.rejected, forced=st.forced, t=st.t, dt=st.dt, err=st.err,
                    A=st.a)

    def set_gauge(self, gauge):
        """"length" (f = E(t), D real symmetric) or "velocity" (f = A(t), D = i K)."""
        _check(_lib.tdse_set_gauge(self._h, GAUGES[gauge]))
        self.gauge = gauge

    def nfield(self, nsteps, samples_per_step=1):
        return samples_per_step * nsteps + 1

    def hmatvec(self, x, f, minus_i=False, y=None, stream=None):
        x = _dev_c(x, self.N, name="x")
        if y is None:
            y = torch.empty_like(x)
        _check(_lib.tdse_hmatvec(self._h, float(f), _ptr(x), _ptr(y), int(bool(minus_i)), _stream(stream)))
        return y

    def propagate(self, c, field, dt, nsteps, scheme="rk4", order=4, hold=HOLD_LEFT, samples_per_step=1,
                  stream=None):
        """Advance c (in place) over nsteps steps; returns c.  Asynchronous on
        the stream: device-side failures (a bounded wait that gave up, a
        Lanczos step too long for its Krylov exponential) surface at sync()."""
        c = _dev_c(c, self.N)
        field = _dev_f64(field, self.nfield(nsteps, samples_per_step), "field")
        _check(_lib.tdse_propagate(self._h, _ptr(c), _ptr(field), int(samples_per_step), float(dt), int(nsteps),
                                   SCHEMES[scheme], int(order), int(hold), _stream(stream)))
        return c

    def propagate_host(self, c, field, dt, nsteps, scheme="rk4", order=4, hold=HOLD_LEFT, samples_per_step=1,
                       stream=None):
        """Same as propagate on host (CPU) tensors: copies in, propagates, copies back, synchronises."""
        if c.device.type != "cpu" or c.dtype != torch.complex128 or not c.is_contiguous() or c.numel() != self.N:
            raise TypeError("c must be a contiguous CPU complex128 tensor of N amplitudes")
        if field.device.type != "cpu" or field.dtype != torch.float64 or not field.is_contiguous():
            raise TypeError("field must be a contiguous CPU float64 tensor")
        if field.numel() != self.nfield(nsteps, samples_per_step):
            raise ValueError("field has the wrong number of samples")
        _check(_lib.tdse_propagate_host(self._h, _ptr(c), _ptr(field), int(samples_per_step), float(dt), int(nsteps),
                                        SCHEMES[scheme], int(order), int(hold), _stream(stream)))
        return c

    def sync(self, stream=None):
        """Wait for this context's work and raise TDSEError on a device-side timeout."""
        _check(_lib.tdse_sync(self._h, _stream(stream)))

    def norm(self, c, B=1, stream=None):
        c = _dev_c(c, self.N, B)
        out = torch.empty(B, dtype=torch.float64, device=c.device)
        _check(_lib.tdse_norm(self._h, _ptr(c), int(B), _ptr(out), _stream(stream)))
        return out

    def populations(self, c, B=1, per_state=True, per_l=True, stream=None):
        c = _dev_c(c, self.N, B)
        dev = c.device
        ps = torch.empty(B, self.N, dtype=torch.float64, device=dev) if per_state else None
        pl = torch.empty(B, self.lmax + 1, dtype=torch.float64, device=dev) if per_l else None
        bound = torch.empty(B, dtype=torch.float64, device=dev)
        ion = torch.empty(B, dtype=torch.float64, device=dev)
        _check(_lib.tdse_populations(self._h, _ptr(c), int(B), _ptr(ps), _ptr(pl), _ptr(bound), _ptr(ion),
                                     _stream(stream)))
        return dict(per_state=ps, per_l=pl, bound=bound, ionised=ion)

    def profile(self, on=True):
        """Enable or disable tracing of the block-product launches."""
        _check(_lib.tdse_profile_enable(self._h, int(bool(on))))

    def profile_read(self):
        """(device ms of traced block products, their launches, all kernel launches) since the last read."""
        ms, nmv, nk = _d(), _l(), _l()
        _check(_lib.tdse_profile_read(self._h, ctypes.byref(ms), ctypes.byref(nmv), ctypes.byref(nk)))
        return ms.value, nmv.value, nk.value

    def inject_wait_timeout(self, timeout_ns, stream=None):
        """Test hook: one bounded device wait runs out after timeout_ns; the next sync() raises ETIMEOUT."""
        _check(_lib.tdse_inject_wait_timeout(self._h, int(timeout_ns), _stream(stream)))

    def set_batch_persistent(self, on=True):
        """bf16x3: run every stage of a batch in one persistent launch (default) or one launch per stage."""
        _check(_lib.tdse_set_batch_persistent(self._h, 1 if on else 0))

    def plan_info(self):
        """Launch shape of the block product: dict(ctas, ctas_per_sm, threads, ring, persistent)."""
        v = [_i() for _ in range(5)]
        _check(_lib.tdse_plan_info(self._h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("ctas", "ctas_per_sm", "threads", "ring", "persistent"), [x.value for x in v]))

    def adjoint(self, c0, field, dt, nsteps, weights, scheme="rk4", order=4, hold=HOLD_LEFT, samples_per_step=1,
                checkpoint_every=64, stream=None):
        """Loss L = sum_a w_a |c_a(T)|^2 and dL/dfield by the discrete adjoint.

        Returns (grad_field, c_final, loss) as CUDA tensors."""
        c0 = _dev_c(c0, self.N, name="c0")
        nF = self.nfield(nsteps, samples_per_step)
        field = _dev_f64(field, nF, "field")
        weights = _dev_f64(weights, self.N, "weights")
        grad = torch.empty(nF, dtype=torch.float64, device=c0.device)
        cT = torch.empty_like(c0)
        loss = torch.empty(1, dtype=torch.float64, device=c0.device)
        _check(_lib.tdse_adjoint(self._h, _ptr(c0), _ptr(field), int(samples_per_step), float(dt), int(nsteps),
                                 SCHEMES[scheme], int(order), int(hold), _ptr(weights), int(checkpoint_every),
                                 _ptr(grad), _ptr(cT), _ptr(loss), _stream(stream)))
        return grad, cT, loss


class FieldLoss(torch.autograd.Function):
    """L(field) = sum_a w_a |c_a(T)|^2 for c(T) propagated from c0 under `field`,
    differentiable with respect to the field samples.

    The forward pass runs tdse_adjoint, which propagates with checkpoints and
    returns the gradient together with the loss; backward scales that
    gradient by the incoming grad.  Usage:
        loss = FieldLoss.apply(field, H, c0, weights, dt, nsteps, opts)
    with opts a dict of adjoint() keyword arguments."""

    @staticmethod
    def forward(ctx, field, H, c0, weights, dt, nsteps, opts=None):
        grad, cT, loss = H.adjoint(c0, field.detach().contiguous(), dt, nsteps, weights, **(opts or {}))
        ctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        return gout * grad, None, None, None, None, None, None


def _batch_propagate(self, c, field, B, dt, nsteps, scheme="rk4", order=4, hold=HOLD_LEFT, samples_per_step=1,
                     stream=None):
    """Advance B states c [B, N] (in place) under their own fields field [B, S];
    one Hamiltonian for all of them."""
    c = _dev_c(c, self.N, B)
    field = _dev_f64(field, B * self.nfield(nsteps, samples_per_step), "field")
    _check(_lib.tdse_propagate_batch(self._h, _ptr(c), _ptr(field), int(B), int(samples_per_step), float(dt),
                                     int(nsteps), SCHEMES[scheme], int(order), int(hold), _stream(stream)))
    return c


Hamiltonian.propagate_batch = _batch_propagate


_lib.tdse_group_sync.argtypes = [_vp, _vp]
_lib.tdse_group_sync.restype = _i
_lib.tdse_group_tune.argtypes = [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_d), _vp]
_lib.tdse_group_tune.restype = _i
_lib.tdse_group_tuning_save.argtypes = [_vp, ctypes.c_char_p]
_lib.tdse_group_tuning_save.restype = _i
_lib.tdse_group_tuning_load.argtypes = [_vp, ctypes.c_char_p, ctypes.POINTER(_i)]
_lib.tdse_group_tuning_load.restype = _i


class Group:
    """Several Hamiltonians of different (lmax, n) advanced together (uneven
    batch): per stage one product launch per thread-layout bucket and its
    members' update, one RK4 step replayed as a CUDA graph; or (tune() or
    set_persistent()) every stage of every system in one persistent launch.
    The member Hamiltonians must outlive the group and must not be propagated
    on their own while the group runs (their scratch vectors are shared)."""

    def __init__(self, hams):
        self.hams = list(hams)
        arr = (_vp * len(self.hams))(*[h.handle for h in self.hams])
        g = _vp()
        _check(_lib.tdse_group_create(arr, len(self.hams), ctypes.byref(g)))
        self._g = g

    def close(self):
        if getattr(self, "_g", None):
            _lib.tdse_group_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def propagate(self, cs, fields, dt, nsteps, samples_per_step=1, stream=None):
        if len(cs) != len(self.hams) or len(fields) != len(self.hams):
            raise ValueError("need one state and one field per system")
        for h, c, f in zip(self.hams, cs, fields):
            _dev_c(c, h.N)
            _dev_f64(f, h.nfield(nsteps, samples_per_step), "field")
        ca = (_vp * len(cs))(*[c.data_ptr() for c in cs])
        fa = (_vp * len(fields))(*[f.data_ptr() for f in fields])
        _check(_lib.tdse_group_propagate(self._g, ca, fa, int(samples_per_step), float(dt), int(nsteps),
                                         _stream(stream)))
        return cs

    def sync(self, stream=None):
        _check(_lib.tdse_group_sync(self._g, _stream(stream)))

    def plan_info(self):
        """Per bucket: dict(members, ctas, ctas_per_sm, threads, ring, rows_per_stage)."""
        nb = _i()
        _check(_lib.tdse_group_plan_info(self._g, -1, ctypes.byref(nb), None, None, None, None, None, None))
        out = []
        for b in range(nb.value):
            v = [_i() for _ in range(6)]
            _check(_lib.tdse_group_plan_info(self._g, b, None, *[ctypes.byref(x) for x in v]))
            out.append(dict(zip(("members", "ctas", "ctas_per_sm", "threads", "ring", "rows_per_stage"),
                                [x.value for x in v])))
        return out

    def set_persistent(self, on=True, layout=-1, rows_per_stage=0):
        """Run later propagations as one persistent launch for all systems
        (on=True; layout -1: the largest n's own, rows_per_stage 0: the
        plan's), or bucketed (on=False)."""
        _check(_lib.tdse_group_set_persistent(self._g, 1 if on else 0, int(layout), int(rows_per_stage)))

    def persistent_info(self):
        """dict(on, ctas, ctas_per_sm, threads, rows_per_stage) of the single launch (zeros when bucketed)."""
        v = [_i() for _ in range(5)]
        _check(_lib.tdse_group_persistent_info(self._g, *[ctypes.byref(x) for x in v]))
        return dict(zip(("on", "ctas", "ctas_per_sm", "threads", "rows_per_stage"), [x.value for x in v]))

    def save_tuning(self, path):
        """Write the buckets' tile shapes (thread layout, rows per stage) to a text file."""
        _check(_lib.tdse_group_tuning_save(self._g, os.fsencode(path)))

    def load_tuning(self, path):
        """Apply the matching lines of a tuning file; returns how many buckets were re-planned."""
        n = _i()
        _check(_lib.tdse_group_tuning_load(self._g, os.fsencode(path), ctypes.byref(n)))
        return n.value

    def tune(self, reps=3, stream=None):
        """Autotune every bucket's tile shape (thread layout and rows per ring
        stage), then keep the buckets or one persistent launch, whichever runs
        whole RK4 steps faster; returns (rows per stage of the bucket with the
        most bytes, summed ms of one product)."""
        rs, ms = _i(), _d()
        _check(_lib.tdse_group_tune(self._g, int(reps), ctypes.byref(rs), ctypes.byref(ms), _stream(stream)))
        return rs.value, ms.value
