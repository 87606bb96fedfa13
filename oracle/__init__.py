"""Plain FP64 CPU oracle for the eigenstate-basis TDSE propagator.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users of this package; the GPU
library never imports, links or calls it, and it shares no code with the GPU
library.  The arithmetic lives in ``tdse_oracle.c`` (plain loops, FP64); this
module only compiles it with gcc and marshals numpy arrays through ctypes.

Functions follow the paper (Ó Broin & Nikolopoulos, arXiv:1201.6062):
  dmatvec / hmatvec   Sec. 4, block form of the Hamiltonian-vector product
  rk4                 App. B, Eqs. "RKFinal"/"RKDeriv", classic tableau
  taylor              App. B, Eq. "taylor" (recursion read as T_m = dt/m M T_{m-1})
  populations         Sec. 5 (continuum population = ionisation), Sec. 5.1 (unitarity)
  lanczos             short-iterative Lanczos (the method Sec. 5.2 proposes next)
  adjoint             discrete adjoint of rk4 / taylor (the paper has no adjoint;
                      pinned by finite differences and a forward-mode tangent)
"""
import contextlib
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdse_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force=False):
    """Compile tdse_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _open(path):
    lib = ctypes.CDLL(path)
    _declare(lib)
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _open(_LIB)
    return _lib


@contextlib.contextmanager
def variant(source_text, tag):
    """Mutation testing: compile `source_text` (a modified tdse_oracle.c) in a
    temporary directory and route every wrapper of this module through it
    inside the `with` block."""
    global _lib
    d = tempfile.mkdtemp(prefix="oracle_%s_" % tag)
    src, so = os.path.join(d, "v.c"), os.path.join(d, "libv.so")
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", so, src, "-lm"])
    saved = _lib
    _lib = _open(so)
    try:
        yield
    finally:
        _lib = saved
        shutil.rmtree(d, ignore_errors=True)


def source():
    """The oracle's C source text (for mutation tests)."""
    with open(_SRC) as f:
        return f.read()


def _declare(lib):
    L, I, D = ctypes.c_long, ctypes.c_int, ctypes.c_double
    lib.orc_threads.restype = I
    lib.orc_set_threads.argtypes = [I]
    lib.orc_dmatvec.argtypes = [I, I, _dp, _dp, _dp]
    lib.orc_hmatvec.argtypes = [I, I, _dp, _dp, D, _dp, _dp]
    lib.orc_field_at.argtypes = [_dp, I, L, I]
    lib.orc_field_at.restype = D
    lib.orc_rk4.argtypes = [I, I, _dp, _dp, _dp, _dp, I, D, L]
    lib.orc_rk4.restype = L
    lib.orc_taylor.argtypes = [I, I, _dp, _dp, _dp, _dp, I, D, L, I, I]
    lib.orc_taylor.restype = L
    lib.orc_lanczos.argtypes = [I, I, _dp, _dp, _dp, _dp, I, D, L, I, I]
    lib.orc_lanczos.restype = L
    lib.orc_tridiag_eig.argtypes = [I, _dp, _dp, _dp]
    lib.orc_tridiag_eig.restype = I
    lib.orc_populations.argtypes = [I, I, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    lib.orc_set_gauge.argtypes = [I]
    lib.orc_vector_potential_sin2.argtypes = [D, D, D, D, D, L, _dp]
    lib.orc_rkf45_tableau.argtypes = [_dp, _dp, _dp, _dp]
    lib.orc_rkf45.argtypes = [I, I, _dp, _dp, _dp, I, D, D, D, D, D, D, D, D, D, D, L,
                              ctypes.POINTER(L), _dp]
    lib.orc_rkf45.restype = L
    lib.orc_adjoint.argtypes = [I, I, _dp, _dp, _dp, _dp, I, D, L, I, I, I, _dp, _dp, _dp]


def _p(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _cvec(c):
    """complex128 vector -> contiguous interleaved float64 view (copy)."""
    c = np.ascontiguousarray(c, dtype=np.complex128).copy()
    return c, c.view(np.float64)


def _dims(E, U, lmax, n):
    E = _f64(E).reshape(-1)
    if lmax > 0:
        U = _f64(U).reshape(lmax, n, n)
    else:
        U = np.zeros((1,), np.float64)
    assert E.size == (lmax + 1) * n
    return E, U


def threads():
    return _load().orc_threads()


def set_threads(t):
    _load().orc_set_threads(int(t))


def dmatvec(lmax, n, U, x):
    """y = D x (dipole part only)."""
    _, U = _dims(np.zeros((lmax + 1) * n), U, lmax, n)
    x, xv = _cvec(x)
    y = np.zeros_like(x)
    _load().orc_dmatvec(lmax, n, _p(U), _p(xv), _p(y.view(np.float64)))
    return y


def hmatvec(lmax, n, E, U, f, x):
    """y = H(f) x = E o x + f D x."""
    E, U = _dims(E, U, lmax, n)
    x, xv = _cvec(x)
    y = np.zeros_like(x)
    _load().orc_hmatvec(lmax, n, _p(E), _p(U), float(f), _p(xv), _p(y.view(np.float64)))
    return y


def field_at(F, samples_per_step, k, h):
    F = _f64(F)
    return _load().orc_field_at(_p(F), samples_per_step, k, h)


def _check_field(F, sps, nsteps):
    F = _f64(F).reshape(-1)
    need = (2 * nsteps + 1) if sps == 2 else (nsteps + 1)
    if sps not in (1, 2) or F.size < need:
        raise ValueError("field needs %d samples for samples_per_step=%d" % (need, sps))
    return F


def rk4(lmax, n, E, U, c0, F, dt, nsteps, samples_per_step=1):
    """Propagate c0 over nsteps classic RK4 steps; returns (c, matvec_count)."""
    E, U = _dims(E, U, lmax, n)
    F = _check_field(F, samples_per_step, nsteps)
    c, cv = _cvec(c0)
    nmv = _load().orc_rk4(lmax, n, _p(E), _p(U), _p(cv), _p(F), samples_per_step, float(dt), int(nsteps))
    return c, nmv


def taylor(lmax, n, E, U, c0, F, dt, nsteps, order, samples_per_step=1, hold=0):
    """Propagate c0 over nsteps truncated-Taylor steps of the given order."""
    E, U = _dims(E, U, lmax, n)
    F = _check_field(F, samples_per_step, nsteps)
    c, cv = _cvec(c0)
    nmv = _load().orc_taylor(lmax, n, _p(E), _p(U), _p(cv), _p(F), samples_per_step, float(dt),
                             int(nsteps), int(order), int(hold))
    return c, nmv


def lanczos(lmax, n, E, U, c0, F, dt, nsteps, m, samples_per_step=1, hold=1):
    """Short-iterative Lanczos propagation with m products per step; returns (c, matvecs)."""
    E, U = _dims(E, U, lmax, n)
    F = _check_field(F, samples_per_step, nsteps)
    c, cv = _cvec(c0)
    r = _load().orc_lanczos(lmax, n, _p(E), _p(U), _p(cv), _p(F), samples_per_step, float(dt), int(nsteps),
                            int(m), int(hold))
    if r < 0:
        raise RuntimeError("tridiagonal eigensolver did not converge in %d steps" % (-r))
    return c, r


def rkf45_tableau():
    """Fehlberg 4(5) coefficients as the oracle holds them: (c[6], a[6x6], b5[6], b4[6])."""
    c, a, b5, b4 = np.zeros(6), np.zeros(36), np.zeros(6), np.zeros(6)
    _load().orc_rkf45_tableau(_p(c), _p(a), _p(b5), _p(b4))
    return c, a.reshape(6, 6), b5, b4


def rkf45(lmax, n, E, U, c0, t0, t1, dt0, tol, field="sin2", E0=0.0, omega=1.0, cycles=10, a0=0.0,
          dt_min=0.0, dt_max=np.inf, max_attempts=10 ** 7):
    """Adaptive Runge-Kutta-Fehlberg 4(5) from t0 to t1.

    field: "sin2" (the Sec. 5 pulse: E(t) in the length gauge, A(t) from a0 by
    Gauss-Legendre in the velocity gauge) or "const" (f = E0).
    Returns (c, info) with info = dict(accepted, rejected, forced, t, dt, err, A, products)."""
    E, U = _dims(E, U, lmax, n)
    c, cv = _cvec(c0)
    st = (ctypes.c_long * 4)()
    tout = np.zeros(4)
    kind = {"sin2": 0, "const": 1}[field]
    prods = _load().orc_rkf45(lmax, n, _p(E), _p(U), _p(cv), kind, float(E0), float(omega), float(cycles),
                              float(a0), float(t0), float(t1), float(dt0), float(tol), float(dt_min),
                              float(min(dt_max, 1e300)), int(max_attempts), st, _p(tout))
    info = dict(accepted=st[0], rejected=st[1], forced=st[2], stalled=bool(st[3]), t=tout[0], dt=tout[1],
                err=tout[2], A=tout[3], products=prods)
    return c, info


def tridiag_eig(d, e):
    """Eigenvalues and eigenvectors (columns) of the symmetric tridiagonal (d, e)."""
    d = _f64(d).copy()
    m = d.size
    ee = np.zeros(m)
    ee[: m - 1] = _f64(e)[: m - 1]
    z = np.zeros((m, m))
    if _load().orc_tridiag_eig(m, _p(d), _p(ee), _p(z)) != 0:
        raise RuntimeError("no convergence")
    return d, z


def set_gauge(gauge):
    """'length' (D real symmetric) or 'velocity' (D = i K, K real antisymmetric)."""
    _load().orc_set_gauge(1 if gauge == "velocity" else 0)


class gauge:
    """Context manager selecting the coupling gauge of every oracle call inside it."""

    def __init__(self, name):
        self.name = name

    def __enter__(self):
        set_gauge(self.name)

    def __exit__(self, *a):
        set_gauge("length")


def vector_potential_sin2(E0, omega, cycles, t0, h, nsamples):
    """A(t0 + k h) = -int_0^t E of the sin^2 pulse, 5-point Gauss-Legendre per interval."""
    out = np.zeros(int(nsamples))
    _load().orc_vector_potential_sin2(float(E0), float(omega), float(cycles), float(t0), float(h), int(nsamples),
                                      _p(out))
    return out


def populations(lmax, n, E, c):
    """Returns dict(per_state, per_l, bound, ionised, norm)."""
    E = _f64(E).reshape(-1)
    c, cv = _cvec(c)
    N = (lmax + 1) * n
    ps = np.zeros(N)
    pl = np.zeros(lmax + 1)
    b = ctypes.c_double()
    io = ctypes.c_double()
    nr = ctypes.c_double()
    _load().orc_populations(lmax, n, _p(E), _p(cv), _p(ps), _p(pl), ctypes.byref(b), ctypes.byref(io),
                            ctypes.byref(nr))
    return dict(per_state=ps, per_l=pl, bound=b.value, ionised=io.value, norm=nr.value)


def adjoint(lmax, n, E, U, c0, F, dt, nsteps, weights, scheme="rk4", order=4, samples_per_step=1, hold=0):
    """Loss L = sum w |c(T)|^2 and its gradient with respect to every field sample.

    Returns (grad[F.shape], c_final, loss)."""
    E, U = _dims(E, U, lmax, n)
    F = _check_field(F, samples_per_step, nsteps)
    w = _f64(weights).reshape(-1)
    assert w.size == (lmax + 1) * n
    c, cv = _cvec(c0)
    grad = np.zeros_like(F)
    loss = ctypes.c_double()
    sch = 0 if scheme == "rk4" else 1
    _load().orc_adjoint(lmax, n, _p(E), _p(U), _p(cv), _p(F), samples_per_step, float(dt), int(nsteps),
                        sch, int(order), int(hold), _p(w), _p(grad), ctypes.byref(loss))
    return grad, c, loss.value
