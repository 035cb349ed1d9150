"""FP64 CPU oracle for the Q1 phase-field method -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
may import this package.  The library path of the product never does, and
this package never imports the product.

The arithmetic lives in ``pf_oracle.c`` (plain element loops in FP64, built by
``oracle.build``); this module only marshals numpy arrays.  Each wrapper names
the equation of the paper (JAX-PF, Hu et al.) that it computes.

Parity pins (tests/test_oracle_*.py check them without a GPU):
  lumped_mass          closed form h^d {1, 1/2, 1/4, 1/8}; sum = domain volume
  residual             = gradient of energy (central FD); independent dense
                         NumPy assembler on 4x4 / 5x7 meshes; the Q1 stiffness
                         stencil closed form (8/3, -1/3); K 1 = 0; uniform
                         fixed points 0, 1/2, 1
  ac_explicit          cosine-mode growth factor (exact eigenvector of the
                         Neumann Q1 operators); 1-D tanh equilibrium profile,
                         width and interfacial energy; monotone energy decrease
  ch_explicit          cosine-mode growth factor; exact mass conservation;
                         monotone energy decrease
  hessian / jvp        central FD of the residual; symmetry u.Jv = v.Ju
  implicit_adjoint     central FD of the objective in L and kappa
  chsplit (implicit CH) JVP = central FD of the residual; exact conservation of
                       c; first-order agreement with the explicit step as dt -> 0;
                       energy decrease
  newton / gmres       FP64 re-evaluation of the root's residual; GMRES on a
                         problem with known solution
  ch_adjoint           central FD of the loss (scalars, a smooth direction of
                         the mobility field, single nodes); per-step
                         dot-product test against the linearised forward map
  Elastic (Eq. 3-4, III.1, 21-22)
                       element stiffness against an independent 3-point Gauss
                         assembly; symmetry, the six rigid-body modes; uniform-
                         strain energy and the patch test; uniform eigenstrain
                         solved exactly (u = m x); the volume identity
                         V = V0 + int tr eps0 of a traction-free body; Eshelby's
                         radial solution of a spherical inclusion; adjoint
                         sensitivities against central FD and E-invariance
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

OR_DOUBLE_WELL = 0
OR_FAN_CHEN = 1
OR_COUPLED = 2


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int64 * 3), ("h", C.c_double * 3)]


class Params(C.Structure):
    _fields_ = [("energy", C.c_int), ("nf", C.c_int), ("W", C.c_double),
                ("kappa", C.c_double), ("mob", C.c_double), ("alpha", C.c_double),
                ("beta", C.c_double), ("gamma", C.c_double),
                ("mob_field", C.POINTER(C.c_double)), ("mob2", C.c_double)]


def lib():
    global _LIB
    if _LIB is None:
        from . import build as _b
        path = _b.build()
        L = C.CDLL(path)
        P = C.POINTER(C.c_double)
        M = C.POINTER(Mesh)
        Pp = C.POINTER(Params)
        L.or_nnodes.restype = C.c_int64
        L.or_nnodes.argtypes = [M]
        L.or_lumped_mass.argtypes = [M, P]
        L.or_energy.restype = C.c_double
        L.or_energy.argtypes = [M, Pp, P]
        L.or_residual.argtypes = [M, Pp, P, P]
        L.or_hessian_apply.argtypes = [M, Pp, P, P, P]
        L.or_mobility_stiffness_apply.argtypes = [M, Pp, P, P]
        L.or_ac_explicit.argtypes = [M, Pp, C.c_double, C.c_int64, P]
        L.or_ch_chemical_potential.argtypes = [M, Pp, P, P]
        L.or_ch_explicit.argtypes = [M, Pp, C.c_double, C.c_int64, P]
        L.or_coupled_explicit.argtypes = [M, Pp, C.c_double, C.c_int64, P]
        L.or_implicit_adjoint.restype = C.c_double
        L.or_implicit_adjoint.argtypes = [M, Pp, C.c_double, C.c_int64, P, C.c_double, P]
        L.or_chsplit_residual.argtypes = [M, Pp, C.c_double, P, P, P]
        L.or_chsplit_jvp.argtypes = [M, Pp, C.c_double, P, P, P]
        L.or_chsplit_newton.restype = C.c_int
        L.or_chsplit_newton.argtypes = [M, Pp, C.c_double, P, P, C.c_double, C.c_int, C.c_int,
                                        C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_double)]
        L.or_mass_integral.restype = C.c_double
        L.or_mass_integral.argtypes = [M, P]
        L.or_implicit_residual.argtypes = [M, Pp, C.c_double, P, P, P]
        L.or_implicit_jvp.argtypes = [M, Pp, C.c_double, P, P, P]
        L.or_gmres.restype = C.c_int
        L.or_gmres.argtypes = [M, Pp, C.c_double, P, P, P, C.c_int, C.c_int, C.c_double,
                               C.POINTER(C.c_int)]
        L.or_newton.restype = C.c_int
        L.or_newton.argtypes = [M, Pp, C.c_double, P, P, C.c_double, C.c_int, C.c_int,
                                C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_double)]
        I = C.c_int
        L.or_conv3d_fwd.argtypes = [P, I, I, I, I, P, P, I, P]
        L.or_conv3d_bwd_data.argtypes = [P, I, I, I, I, P, I, P]
        L.or_conv3d_bwd_weight.argtypes = [P, I, I, I, I, P, I, P, P]
        L.or_ch_adjoint.restype = C.c_double
        L.or_ch_adjoint.argtypes = [M, Pp, C.c_double, C.c_int64, P, P, C.c_int, P, P, P]
        L.or_set_threads.argtypes = [C.c_int]
        D = C.c_double
        L.or_elastic_lame.argtypes = [D, D, P, P]
        L.or_elastic_apply.argtypes = [M, D, D, P, P]
        L.or_elastic_rhs.argtypes = [M, D, D, D, D, D, P]
        L.or_elastic_volume_functional.restype = D
        L.or_elastic_volume_functional.argtypes = [M, P]
        L.or_elastic_cg.restype = C.c_int
        L.or_elastic_cg.argtypes = [M, D, D, P, P, D, C.c_int, C.POINTER(C.c_int)]
        L.or_elastic_sensitivity.restype = D
        L.or_elastic_sensitivity.argtypes = [M, D, D, D, D, D, P, D, C.c_int, P, P]
        _LIB = L
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def mesh(shape, h=1.0):
    """Mesh for a node array of `shape` = (ny, nx) or (nz, ny, nx)."""
    dim = len(shape)
    hs = (h,) * dim if np.isscalar(h) else tuple(h)
    n = list(reversed(shape)) + [1] * (3 - dim)
    hh = list(hs) + [1.0] * (3 - dim)
    return Mesh(dim, (C.c_int64 * 3)(*n), (C.c_double * 3)(*hh))


class Problem:
    """A mesh plus the material parameters of one phase-field model.

    energy: 'double_well' (f = W c^2 (1-c)^2, Eq. 5-6 with the Supp. 3
    polynomial), 'fan_chen' (grain growth) or 'coupled' (Eq. 7 with the Supp. 3
    polynomials; fields [c, eta], no c gradient term; mob = M_c, mob2 = M_eta,
    kappa = kappa_eta); nf fields; mob = L (AC) or M (CH); mob_field =
    per-node mobility multiplier (CH only).
    """

    def __init__(self, shape, h=1.0, energy="double_well", nf=1, W=1.0, kappa=1.0, mob=1.0,
                 alpha=1.0, beta=1.0, gamma=1.5, mob_field=None, mob2=0.0):
        self.shape = tuple(shape)
        self.nf = 2 if energy == "coupled" else nf
        self.m = mesh(self.shape, h)
        self._mf = None if mob_field is None else _f64(mob_field).ravel()
        kind = {"double_well": OR_DOUBLE_WELL, "fan_chen": OR_FAN_CHEN, "coupled": OR_COUPLED}
        self.p = Params(kind[energy], self.nf, W, kappa, mob, alpha, beta, gamma,
                        None if self._mf is None else _ptr(self._mf), mob2)
        self.nnodes = int(np.prod(self.shape))

    def _fshape(self):
        return self.shape if self.nf == 1 else (self.nf,) + self.shape

    def _out(self, nf=None):
        nf = self.nf if nf is None else nf
        return np.zeros((nf,) + self.shape if nf > 1 else self.shape, dtype=np.float64)

    # -- operators --
    def lumped_mass(self):
        out = np.zeros(self.shape)
        lib().or_lumped_mass(C.byref(self.m), _ptr(out))
        return out

    def energy(self, U):
        U = _f64(U)
        return lib().or_energy(C.byref(self.m), C.byref(self.p), _ptr(U))

    def residual(self, U):
        """r = dE_h/dU (Eq. 11's r without the mobility factor)."""
        U = _f64(U)
        out = self._out()
        lib().or_residual(C.byref(self.m), C.byref(self.p), _ptr(U), _ptr(out))
        return out

    def hessian_apply(self, U, v):
        U, v = _f64(U), _f64(v)
        out = self._out()
        lib().or_hessian_apply(C.byref(self.m), C.byref(self.p), _ptr(U), _ptr(v), _ptr(out))
        return out

    def mobility_stiffness_apply(self, mu):
        mu = _f64(mu)
        out = self._out(1)
        lib().or_mobility_stiffness_apply(C.byref(self.m), C.byref(self.p), _ptr(mu), _ptr(out))
        return out

    def chemical_potential(self, c):
        c = _f64(c)
        out = self._out(1)
        lib().or_ch_chemical_potential(C.byref(self.m), C.byref(self.p), _ptr(c), _ptr(out))
        return out

    def mass_integral(self, c):
        c = _f64(c)
        return lib().or_mass_integral(C.byref(self.m), _ptr(c))

    # -- time stepping --
    def ac_explicit(self, U, dt, nsteps):
        U = _f64(U).copy()
        lib().or_ac_explicit(C.byref(self.m), C.byref(self.p), dt, nsteps, _ptr(U))
        return U

    def ch_explicit(self, c, dt, nsteps):
        c = _f64(c).copy()
        lib().or_ch_explicit(C.byref(self.m), C.byref(self.p), dt, nsteps, _ptr(c))
        return c

    def coupled_explicit(self, U, dt, nsteps):
        """Coupled AC-CH explicit steps (Eq. 7, 9-12): U = [c, eta] planes."""
        U = _f64(U).copy()
        lib().or_coupled_explicit(C.byref(self.m), C.byref(self.p), dt, nsteps, _ptr(U))
        return U

    def implicit_residual(self, dt, Un, U):
        Un, U = _f64(Un), _f64(U)
        out = self._out()
        lib().or_implicit_residual(C.byref(self.m), C.byref(self.p), dt, _ptr(Un), _ptr(U),
                                   _ptr(out))
        return out

    def implicit_jvp(self, dt, U, v):
        U, v = _f64(U), _f64(v)
        out = self._out()
        lib().or_implicit_jvp(C.byref(self.m), C.byref(self.p), dt, _ptr(U), _ptr(v), _ptr(out))
        return out

    def gmres(self, dt, U, b, restart=30, maxit=1000, rtol=1e-10):
        U, b = _f64(U), _f64(b)
        x = np.zeros_like(b)
        it = C.c_int(0)
        ok = lib().or_gmres(C.byref(self.m), C.byref(self.p), dt, _ptr(U), _ptr(b), _ptr(x),
                            restart, maxit, rtol, C.byref(it))
        return x, bool(ok), it.value

    def newton(self, dt, Un, U0=None, abs_tol=1e-10, max_newton=30, restart=30, gmres_rtol=1e-10):
        Un = _f64(Un)
        U = Un.copy() if U0 is None else _f64(U0).copy()
        ni, gi, fn = C.c_int(0), C.c_int(0), C.c_double(0)
        ok = lib().or_newton(C.byref(self.m), C.byref(self.p), dt, _ptr(Un), _ptr(U), abs_tol,
                             max_newton, restart, gmres_rtol, C.byref(ni), C.byref(gi),
                             C.byref(fn))
        return U, dict(ok=bool(ok), newton_iters=ni.value, gmres_iters=gi.value,
                       final_norm=fn.value)

    def implicit_adjoint(self, U0, dt, nsteps, abs_tol=1e-12):
        """Objective O = domain average of U^N after nsteps implicit steps (Eq. 19)
        and its sensitivities [dO/dL, dO/dkappa] by the adjoint of Supp. 2."""
        U0 = _f64(U0)
        g = np.zeros(2)
        O = lib().or_implicit_adjoint(C.byref(self.m), C.byref(self.p), dt, nsteps, _ptr(U0),
                                      abs_tol, _ptr(g))
        return O, g

    # -- implicit split Cahn-Hilliard (Eq. 9-10, 13): U = [c, mu] --
    def chsplit_residual(self, dt, cn, U):
        cn, U = _f64(cn), _f64(U)
        out = np.zeros((2,) + self.shape)
        lib().or_chsplit_residual(C.byref(self.m), C.byref(self.p), dt, _ptr(cn), _ptr(U),
                                  _ptr(out))
        return out

    def chsplit_jvp(self, dt, U, v):
        U, v = _f64(U), _f64(v)
        out = np.zeros((2,) + self.shape)
        lib().or_chsplit_jvp(C.byref(self.m), C.byref(self.p), dt, _ptr(U), _ptr(v), _ptr(out))
        return out

    def chsplit_newton(self, dt, cn, U0=None, abs_tol=1e-10, max_newton=30, restart=30,
                       gmres_rtol=1e-10):
        """One backward-Euler step of the split CH system from composition cn;
        U0 = [c, mu] initial guess (default [cn, M^-1 r(cn)])."""
        cn = _f64(cn)
        U = (np.stack([cn, self.chemical_potential(cn)]) if U0 is None else _f64(U0)).copy()
        ni, gi, fn = C.c_int(0), C.c_int(0), C.c_double(0)
        ok = lib().or_chsplit_newton(C.byref(self.m), C.byref(self.p), dt, _ptr(cn), _ptr(U),
                                     abs_tol, max_newton, restart, gmres_rtol, C.byref(ni),
                                     C.byref(gi), C.byref(fn))
        return U, dict(ok=bool(ok), newton_iters=ni.value, gmres_iters=gi.value,
                       final_norm=fn.value)

    def ch_adjoint(self, c0, target, dt, nsteps, nodal_loss=False, want_field=True):
        c0, target = _f64(c0), _f64(target)
        gs = np.zeros(3)
        gmf = np.zeros(self.shape) if want_field else None
        lam0 = np.zeros(self.shape)
        loss = lib().or_ch_adjoint(C.byref(self.m), C.byref(self.p), dt, nsteps, _ptr(c0),
                                   _ptr(target), int(nodal_loss), _ptr(gs),
                                   _ptr(gmf) if want_field else None, _ptr(lam0))
        return loss, dict(kappa=gs[0], W=gs[1], M=gs[2], mob_field=gmf, c0=lam0)


# ---- 3x3x3 convolution of the learned surrogate (one sample, [C][D][H][W]) ----

def conv3d(x, w, b=None):
    """y = conv(x, w) + b: 3x3x3 stencil, stride 1, zero padding 1.  w[co][ci][3][3][3]."""
    x, w = _f64(x), _f64(w)
    ci, d, h, ww = x.shape
    co = w.shape[0]
    y = np.zeros((co, d, h, ww))
    bb = None if b is None else _f64(b)
    lib().or_conv3d_fwd(_ptr(x), ci, d, h, ww, _ptr(w), None if bb is None else _ptr(bb), co,
                        _ptr(y))
    return y


def conv3d_bwd_data(dy, w):
    dy, w = _f64(dy), _f64(w)
    co, d, h, ww = dy.shape
    ci = w.shape[1]
    dx = np.zeros((ci, d, h, ww))
    lib().or_conv3d_bwd_data(_ptr(dy), co, d, h, ww, _ptr(w), ci, _ptr(dx))
    return dx


def conv3d_bwd_weight(x, dy):
    x, dy = _f64(x), _f64(dy)
    ci, d, h, ww = x.shape
    co = dy.shape[0]
    dw = np.zeros((co, ci, 3, 3, 3))
    db = np.zeros(co)
    lib().or_conv3d_bwd_weight(_ptr(x), ci, d, h, ww, _ptr(dy), co, _ptr(dw), _ptr(db))
    return dw, db


# ---- Eshelby inclusion: linear elasticity with a misfit eigenstrain ----

class Elastic:
    """Q1 small-strain elasticity on a (nz, ny, nx) node grid with spacing h
    (Eq. 3-4); displacements [3][nz][ny][nx] (x, y, z components).  The
    eigenstrain is m phi(r) I, phi = (1 - tanh(l (r - a))) / 2, r = |x| from
    node (0, 0, 0) (Eq. III.1, inclusion reading); x = 0, y = 0, z = 0 are
    symmetry planes, the other faces traction-free."""

    def __init__(self, shape, h=1.0):
        assert len(shape) == 3
        self.shape = tuple(shape)
        self.m = mesh(self.shape, h)

    def _out(self):
        return np.zeros((3,) + self.shape)

    @staticmethod
    def lame(E, nu):
        lam, mu = np.zeros(1), np.zeros(1)
        lib().or_elastic_lame(E, nu, _ptr(lam), _ptr(mu))
        return float(lam[0]), float(mu[0])

    def apply(self, u, lam, mu):
        """K u, assembled over all elements, no constraints."""
        u = _f64(u)
        out = self._out()
        lib().or_elastic_apply(C.byref(self.m), lam, mu, _ptr(u), _ptr(out))
        return out

    def rhs(self, lam, mu, m, l, a):
        """Eigenstrain load f = int B^T C eps0."""
        f = self._out()
        lib().or_elastic_rhs(C.byref(self.m), lam, mu, m, l, a, _ptr(f))
        return f

    def volume_functional(self):
        """(V0, g) with V = V0 + g . u the small-strain volume."""
        g = self._out()
        V0 = lib().or_elastic_volume_functional(C.byref(self.m), _ptr(g))
        return V0, g

    def cg(self, b, lam, mu, rtol=1e-12, maxit=20000):
        """K u = b on the unconstrained degrees of freedom (CG from zero)."""
        b = _f64(b)
        u = self._out()
        it = C.c_int(0)
        ok = lib().or_elastic_cg(C.byref(self.m), lam, mu, _ptr(b), _ptr(u), rtol, maxit,
                                 C.byref(it))
        return u, bool(ok), it.value

    def solve(self, E, nu, m, l, a, rtol=1e-12, maxit=20000):
        lam, mu = self.lame(E, nu)
        return self.cg(self.rhs(lam, mu, m, l, a), lam, mu, rtol, maxit)

    def sensitivity(self, E, nu, m, l, a, g=None, rtol=1e-12, maxit=20000):
        """(O, [dO/dE, dO/dnu], u) for O = g . u (g = the volume functional if
        None, and then O = V includes V0), Eq. 21-22."""
        V0 = 0.0
        if g is None:
            V0, g = self.volume_functional()
        g = _f64(g)
        u = self._out()
        grads = np.zeros(2)
        O = lib().or_elastic_sensitivity(C.byref(self.m), E, nu, m, l, a, _ptr(g), rtol, maxit,
                                         _ptr(u), _ptr(grads))
        return O + V0, grads, u


def set_threads(n):
    """Threads of the oracle's OpenMP loops (n <= 0: one per processor)."""
    lib().or_set_threads(int(n))
