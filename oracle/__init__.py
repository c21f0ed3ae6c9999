"""FP64 CPU oracle for the resonant-line Monte Carlo path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never does, and it shares no code with the C source here
(``rascas_oracle.c``), which restates the method of Michel-Dansac et al.
(2020) step by step in double precision.

The wrapper marshals a ``synth.Workload`` into the oracle's own C struct and
runs packet ranges, optionally on several host threads (ctypes releases the
GIL for the duration of each C call; each thread has its own tallies, summed
afterwards in a fixed order, so the result does not depend on the thread
count up to floating-point summation order of whole-chunk tallies).

Parity status of each function (pins live in tests/test_oracle_*.py):
  ora_philox4x32_10 .... pinned (published known-answer vectors)
  ora_voigt ............ pinned (quadrature of the H(a,x) integral, limits)
  ora_faddeeva ......... pinned (scipy wofz, quadrature of H's integral, limits,
                         normalisation, derivatives against differences)
  ora_u0/u_par sampler . pinned (chi-square against the normalised density)
  ora_mu_sample ........ pinned (CDF inversion identities, chi-square, <mu>=g)
  ora_onb .............. pinned (orthonormality)
  walk / ray_tau ....... pinned (brute-force leaf lookup, closed-form tau)
  ora_run / ora_event .. pinned (MFP, conservation, symmetry, pure absorber,
                         error budget, Neufeld / Dijkstra spectra, Harrington)
  peeling .............. pinned (4 pi * peeled flux = escape fraction, symmetry,
                         empty medium); no cut-off (rays walked until exp(-tau)
                         underflows in FP64, which changes no tally)
  line_props ........... pinned (a at T = 10, 1e2, 1e4 K as printed in Sect. 3.4.2;
                         sigma integrated over frequency = pi e^2 f / (m_e c))
  core-skipping u_perp . pinned (radius law of the truncated 2-D Gaussian,
                         x_crit = 0 identical to the plain draw, slab spectra)
  ray_columns .......... pinned (closed-form chords of a uniform sphere, same
                         leaves as ray_tau)
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rascas_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "librascas_oracle.so")
_lock = threading.Lock()
_lib = None

C_CGS = 2.99792458e10  # oracle-side copy, used only to build frequencies from wavelengths

MAXLINE, MAXCHAN, MAXDIR = 4, 4, 8
ACTIVE, ESCAPED, ABSORBED, CAPPED, ERROR = 0, 1, 2, 3, 4


def build(force=False):
    """Compile the oracle with gcc (no FP contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class Cfg(C.Structure):
    _fields_ = [
        ("son", C.c_void_p), ("n_HI", C.c_void_p), ("vx", C.c_void_p), ("vy", C.c_void_p),
        ("vz", C.c_void_p), ("T", C.c_void_p), ("n_dust", C.c_void_p), ("n_metal", C.c_void_p),
        ("noct", C.c_int64), ("nleaf", C.c_int64), ("box_cm", C.c_double),
        ("dom_kind", C.c_int64), ("dom_c", C.c_double * 3), ("dom_size", C.c_double), ("dom_inner", C.c_double),
        ("nline", C.c_int64),
        ("line_nu", C.c_double * MAXLINE), ("line_A", C.c_double * MAXLINE),
        ("line_f", C.c_double * MAXLINE), ("line_m", C.c_double * MAXLINE),
        ("line_abund", C.c_double * MAXLINE),
        ("line_dens", C.c_int64 * MAXLINE), ("line_phase", C.c_int64 * MAXLINE),
        ("line_nchan", C.c_int64 * MAXLINE),
        ("chan_A", (C.c_double * MAXCHAN) * MAXLINE), ("chan_nu", (C.c_double * MAXCHAN) * MAXLINE),
        ("dust_sigma", C.c_double), ("dust_albedo", C.c_double), ("dust_g", C.c_double),
        ("recoil", C.c_int64), ("isotropic", C.c_int64), ("keep_dir", C.c_int64),
        ("max_scatt", C.c_int64), ("max_steps", C.c_int64),
        ("x_gauss", C.c_double), ("seed", C.c_uint64),
        ("nu_lo", C.c_double), ("nu_hi", C.c_double),
        ("nbin", C.c_int64), ("ndir", C.c_int64), ("npix", C.c_int64), ("cube", C.c_int64),
        ("dirs", (C.c_double * 3) * MAXDIR), ("fov", C.c_double), ("img_c", C.c_double * 3),
        ("voigt", C.c_int64),
        ("core_skip", C.c_double), ("core_skip_f", C.c_double),
    ]


class State(C.Structure):
    _fields_ = [
        ("p", C.c_double * 3), ("k", C.c_double * 3), ("nu", C.c_double),
        ("leaf", C.c_int64), ("level", C.c_int64), ("ijk", C.c_int64 * 3),
        ("pid", C.c_uint64), ("ndraw", C.c_uint64),
        ("nscatt", C.c_int64), ("nsteps", C.c_int64), ("status", C.c_int64),
        ("path", C.c_double),
    ]


class Tally(C.Structure):
    _fields_ = [
        ("spec", C.c_void_p), ("pspec", C.c_void_p), ("pimg", C.c_void_p), ("pcube", C.c_void_p),
        ("ncross", C.c_int64), ("nscatt_line", C.c_int64), ("nscatt_dust", C.c_int64),
        ("npeel", C.c_int64), ("events", C.c_void_p), ("nev", C.c_int64), ("cap", C.c_int64),
    ]


EVENT_DTYPE = np.dtype([("p", "<f8", 3), ("leaf", "<i8"), ("level", "<i8"), ("ijk", "<i8", 3), ("dir", "<i8"),
                        ("w", "<f8"), ("nu", "<f8")])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, i64, u64 = C.POINTER(C.c_double), C.c_int64, C.c_uint64
            L.ora_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.ora_word.restype = C.c_uint32
            L.ora_word.argtypes = [u64, u64, u64]
            L.ora_voigt.restype = C.c_double
            L.ora_voigt.argtypes = [C.c_double, C.c_double]
            L.ora_faddeeva.restype = None
            L.ora_faddeeva.argtypes = [C.c_double, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.ora_faddeeva_derivs.restype = None
            L.ora_faddeeva_derivs.argtypes = [C.c_double, C.c_double] + [C.POINTER(C.c_double)] * 3
            L.ora_u0.restype = C.c_double
            L.ora_u0.argtypes = [C.c_double, C.c_double]
            L.ora_mu_sample.restype = C.c_double
            L.ora_mu_sample.argtypes = [C.c_int, C.c_double, C.c_double]
            L.ora_phase.restype = C.c_double
            L.ora_phase.argtypes = [C.c_int, C.c_double, C.c_double]
            L.ora_onb.argtypes = [dp, dp, dp]
            L.ora_sample_upar_n.argtypes = [C.POINTER(Cfg), u64, C.c_double, C.c_double, i64, dp]
            L.ora_locate.restype = i64
            L.ora_locate.argtypes = [C.POINTER(Cfg), dp, dp, C.POINTER(i64), C.POINTER(i64)]
            L.ora_opacity.restype = C.c_double
            L.ora_opacity.argtypes = [C.POINTER(Cfg), i64, C.c_double, dp]
            L.ora_ray_tau.restype = C.c_double
            L.ora_ray_tau.argtypes = [C.POINTER(Cfg), dp, dp, C.c_double, C.c_double,
                                      C.POINTER(i64), dp, i64, C.POINTER(i64)]
            L.ora_init_state.restype = C.c_int
            L.ora_init_state.argtypes = [C.POINTER(Cfg), C.POINTER(State), dp, dp, C.c_double, u64]
            L.ora_event.restype = C.c_int
            L.ora_event.argtypes = [C.POINTER(Cfg), C.POINTER(State), C.POINTER(Tally)]
            L.ora_run.restype = C.c_int
            L.ora_run.argtypes = [C.POINTER(Cfg), i64, dp, dp, dp, C.POINTER(u64),
                                  C.POINTER(C.c_int32), C.POINTER(i64), dp, dp, dp, dp, C.POINTER(Tally)]
            L.ora_peel_from_events.argtypes = [C.POINTER(Cfg), C.c_void_p, i64, C.POINTER(Tally)]
            L.ora_adjoint_events.argtypes = [C.POINTER(Cfg), C.c_void_p, i64, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p]
            L.ora_voigt_derivs.argtypes = [C.c_double, C.c_double, dp, dp, dp]
            L.ora_emission.argtypes = [C.POINTER(Cfg), C.POINTER(State), C.POINTER(Tally)]
            L.ora_line_props.argtypes = [C.POINTER(Cfg), i64, i64, C.c_double, dp]
            L.ora_sample_uperp_n.argtypes = [C.POINTER(Cfg), u64, C.c_double, C.c_double, i64, dp]
            L.ora_core_skip_xcrit.restype = C.c_double
            L.ora_core_skip_xcrit.argtypes = [C.POINTER(Cfg), i64, i64, i64]
            L.ora_ray_columns.restype = i64
            L.ora_ray_columns.argtypes = [C.POINTER(Cfg), dp, dp, dp]
            for f in ("ora_sizeof_cfg", "ora_sizeof_state", "ora_sizeof_tally", "ora_sizeof_event"):
                getattr(L, f).restype = i64
            assert L.ora_sizeof_cfg() == C.sizeof(Cfg)
            assert L.ora_sizeof_state() == C.sizeof(State)
            assert L.ora_sizeof_tally() == C.sizeof(Tally)
            assert L.ora_sizeof_event() == EVENT_DTYPE.itemsize
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class Oracle:
    """A workload marshalled into the oracle's configuration."""

    def __init__(self, wl):
        self.wl = wl
        m = wl.medium
        self._keep = {
            "son": np.ascontiguousarray(m.tree.son, dtype=np.int32),
            "n_HI": _f32(m.n_HI), "vx": _f32(m.vx), "vy": _f32(m.vy), "vz": _f32(m.vz),
            "T": _f32(m.T), "n_dust": _f32(m.n_dust), "n_metal": _f32(m.n_metal),
        }
        cf = Cfg()
        for k, v in self._keep.items():
            setattr(cf, k, v.ctypes.data)
        cf.noct, cf.nleaf, cf.box_cm = m.tree.noct, m.tree.nleaf, m.box_cm
        d = wl.domain
        cf.dom_kind = d.kind
        cf.dom_c[:] = list(d.centre)
        cf.dom_size = d.size
        cf.dom_inner = getattr(d, "inner", 0.0)
        assert len(wl.lines) <= MAXLINE
        cf.nline = len(wl.lines)
        for i, ln in enumerate(wl.lines):
            cf.line_nu[i] = C_CGS / (ln.lambda_A * 1e-8)
            cf.line_A[i], cf.line_f[i], cf.line_m[i] = ln.A_ul, ln.f_lu, ln.mass_g
            cf.line_abund[i] = ln.abundance
            cf.line_dens[i] = 1 if ln.density == 1 else 0
            cf.line_phase[i] = ln.phase
            chans = ln.all_channels()
            assert len(chans) <= MAXCHAN
            cf.line_nchan[i] = len(chans)
            for c, (A, lam) in enumerate(chans):
                cf.chan_A[i][c] = A
                cf.chan_nu[i][c] = C_CGS / (lam * 1e-8)
        cf.dust_sigma, cf.dust_albedo, cf.dust_g = wl.dust.sigma, wl.dust.albedo, wl.dust.g
        ph = wl.physics
        cf.recoil, cf.isotropic, cf.keep_dir = ph.recoil, ph.isotropic, ph.keep_direction
        cf.max_scatt, cf.max_steps = ph.max_scatt, ph.max_steps
        cf.x_gauss, cf.seed = ph.x_gauss, ph.seed
        cf.voigt = getattr(ph, "voigt", 0)
        cf.core_skip = getattr(ph, "core_skip", 0.0)
        cf.core_skip_f = getattr(ph, "core_skip_f", 0.0)
        det = wl.detector
        cf.nu_lo, cf.nu_hi, cf.nbin = det.nu_lo, det.nu_hi, det.nbin
        dirs = np.asarray(det.dirs, dtype=np.float64).reshape(-1, 3)
        assert dirs.shape[0] <= MAXDIR
        cf.ndir = dirs.shape[0]
        for i in range(dirs.shape[0]):
            v = dirs[i] / np.linalg.norm(dirs[i])
            cf.dirs[i][:] = list(v)
        cf.npix, cf.fov, cf.cube = det.npix, det.fov, det.cube
        cf.img_c[:] = list(det.centre)
        self.cfg = cf

    # -------------------------------------------------------------- runs
    def _alloc_tally(self):
        c = self.cfg
        t = {"spec": np.zeros(c.nbin)}
        t["pspec"] = np.zeros(max(1, c.ndir * c.nbin))
        t["pimg"] = np.zeros(max(1, c.ndir * c.npix * c.npix))
        t["pcube"] = np.zeros(max(1, c.ndir * c.npix * c.npix * c.nbin)) if c.cube else None
        ty = Tally()
        ty.spec, ty.pspec, ty.pimg = t["spec"].ctypes.data, t["pspec"].ctypes.data, t["pimg"].ctypes.data
        ty.pcube = t["pcube"].ctypes.data if t["pcube"] is not None else None
        return ty, t

    def _run_range(self, pk, lo, hi, record=0):
        n = hi - lo
        pos = np.ascontiguousarray(pk.pos[lo:hi], dtype=np.float64)
        dr = np.ascontiguousarray(pk.dir[lo:hi], dtype=np.float64)
        nu = np.ascontiguousarray(pk.nu[lo:hi], dtype=np.float64)
        ids = np.ascontiguousarray(pk.ids[lo:hi], dtype=np.uint64)
        out = {"status": np.zeros(n, np.int32), "nscatt": np.zeros(n, np.int64),
               "nu": np.zeros(n), "pos": np.zeros((n, 3)), "dir": np.zeros((n, 3)), "path": np.zeros(n)}
        ty, t = self._alloc_tally()
        if record:
            ev = np.zeros(record, dtype=EVENT_DTYPE)
            ty.events, ty.cap = ev.ctypes.data, record
        lib().ora_run(C.byref(self.cfg), n, _dp(pos), _dp(dr), _dp(nu),
                      ids.ctypes.data_as(C.POINTER(C.c_uint64)),
                      out["status"].ctypes.data_as(C.POINTER(C.c_int32)),
                      out["nscatt"].ctypes.data_as(C.POINTER(C.c_int64)),
                      _dp(out["nu"]), _dp(out["pos"]), _dp(out["dir"]), _dp(out["path"]), C.byref(ty))
        t["ncross"], t["nscatt_line"], t["nscatt_dust"], t["npeel"] = (
            ty.ncross, ty.nscatt_line, ty.nscatt_dust, ty.npeel)
        if record:
            if ty.nev > record:
                raise RuntimeError("event record overflow: %d > %d" % (ty.nev, record))
            t["events"] = ev[: ty.nev]
        return out, t

    def run(self, packets=None, lo=0, hi=None, threads=1, chunk=None, record_events=0):
        """Propagate packets [lo, hi) of the workload (or of ``packets``);
        record_events > 0 keeps up to that many peeling events per chunk."""
        pk = packets if packets is not None else self.wl.packets
        hi = pk.n if hi is None else hi
        if threads <= 1:
            parts = [self._run_range(pk, lo, hi, record_events)]
        else:
            chunk = chunk or max(1, (hi - lo + threads * 4 - 1) // (threads * 4))
            bounds = [(a, min(hi, a + chunk)) for a in range(lo, hi, chunk)]
            with ThreadPoolExecutor(threads) as ex:
                parts = list(ex.map(lambda b: self._run_range(pk, *b, record_events), bounds))
        out = {k: np.concatenate([p[0][k] for p in parts]) for k in parts[0][0]}
        tal = {}
        for k in parts[0][1]:
            if parts[0][1][k] is None:
                tal[k] = None
            elif k == "events":
                tal[k] = np.concatenate([p[1][k] for p in parts])
            else:
                tal[k] = sum(p[1][k] for p in parts)
        c = self.cfg
        if c.ndir:
            tal["pspec"] = tal["pspec"].reshape(c.ndir, c.nbin)
            tal["pimg"] = tal["pimg"].reshape(c.ndir, c.npix, c.npix) if c.npix else None
            if tal["pcube"] is not None:
                tal["pcube"] = tal["pcube"].reshape(c.ndir, c.npix, c.npix, c.nbin)
        return out, tal

    def _shape(self, tal):
        c = self.cfg
        if c.ndir:
            tal["pspec"] = tal["pspec"].reshape(c.ndir, c.nbin)
            tal["pimg"] = tal["pimg"].reshape(c.ndir, c.npix, c.npix) if c.npix else None
            if tal["pcube"] is not None:
                tal["pcube"] = tal["pcube"].reshape(c.ndir, c.npix, c.npix, c.nbin)
        return tal

    def peel_from_events(self, events):
        """Peeled spectra / images / cubes of a fixed event record with the
        current leaf fields (the forward map the adjoint differentiates)."""
        ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
        ty, t = self._alloc_tally()
        lib().ora_peel_from_events(C.byref(self.cfg), ev.ctypes.data, ev.size, C.byref(ty))
        return self._shape(t)

    def adjoint(self, events, g_cube=None, g_img=None, g_spec=None):
        """dL/d(n_HI, vx, vy, vz, T, n_dust) per leaf, [6, nleaf], for
        L = sum(g_cube*cube) + sum(g_img*img) + sum(g_spec*spec) over a fixed
        event record (optical depths of the peeling rays differentiated)."""
        ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
        arr = [None if g is None else np.ascontiguousarray(g, dtype=np.float64) for g in (g_cube, g_img, g_spec)]
        grad = np.zeros((6, self.cfg.nleaf))
        lib().ora_adjoint_events(C.byref(self.cfg), ev.ctypes.data, ev.size,
                                 *[None if a is None else a.ctypes.data for a in arr], grad.ctypes.data)
        return grad

    def set_field(self, name, values):
        """Replace one leaf field (float32 copy kept alive by the wrapper)."""
        v = np.ascontiguousarray(values, dtype=np.float32)
        self._keep[name] = v
        setattr(self.cfg, name, v.ctypes.data)

    # -------------------------------------------------------------- pieces
    def locate(self, p, k=(1.0, 1.0, 1.0)):
        """Leaf entered at p moving along k (the cell containing p + eps k)."""
        p = np.ascontiguousarray(p, dtype=np.float64)
        k = np.ascontiguousarray(k, dtype=np.float64)
        lv = C.c_int64()
        ijk = (C.c_int64 * 3)()
        leaf = lib().ora_locate(C.byref(self.cfg), _dp(p), _dp(k), C.byref(lv), ijk)
        return leaf, lv.value, tuple(ijk)

    def opacity(self, leaf, nu_ext, k):
        k = np.ascontiguousarray(k, dtype=np.float64)
        return lib().ora_opacity(C.byref(self.cfg), int(leaf), float(nu_ext), _dp(k))

    def ray_tau(self, p, k, nu_ext, tau_stop=math.inf, cap=0):
        p = np.ascontiguousarray(p, dtype=np.float64)
        k = np.ascontiguousarray(k, dtype=np.float64)
        cells = np.zeros(max(cap, 1), np.int64)
        lens = np.zeros(max(cap, 1))
        nc = C.c_int64()
        tau = lib().ora_ray_tau(C.byref(self.cfg), _dp(p), _dp(k), float(nu_ext), float(tau_stop),
                                cells.ctypes.data_as(C.POINTER(C.c_int64)) if cap else None,
                                _dp(lens) if cap else None, cap, C.byref(nc))
        n = min(nc.value, cap)
        return tau, cells[:n], lens[:n], nc.value

    def line_props(self, il, leaf, nu_gas):
        """(v_th, Delta nu_D, a, x, sigma) of line il in a leaf at gas-frame
        frequency nu_gas (Sect. 3.1.1)."""
        out = np.zeros(5)
        lib().ora_line_props(C.byref(self.cfg), int(il), int(leaf), float(nu_gas), _dp(out))
        return tuple(float(v) for v in out)

    def uperp_samples(self, x_in, x_crit, n, pid=0):
        """n perpendicular-velocity pairs [n, 2] drawn at x_in with the
        core-skipping threshold x_crit (0 = the plain draw)."""
        out = np.zeros(2 * n)
        lib().ora_sample_uperp_n(C.byref(self.cfg), int(pid), float(x_in), float(x_crit), n, _dp(out))
        return out.reshape(n, 2)

    def core_skip_xcrit(self, il, leaf, level):
        return lib().ora_core_skip_xcrit(C.byref(self.cfg), int(il), int(leaf), int(level))

    def ray_columns(self, p, k):
        """(N_HI, N_dust, N_metal) from p along k to the domain border and the
        number of leaves crossed."""
        p = np.ascontiguousarray(p, dtype=np.float64)
        k = np.ascontiguousarray(k, dtype=np.float64)
        cols = np.zeros(3)
        n = lib().ora_ray_columns(C.byref(self.cfg), _dp(p), _dp(k), _dp(cols))
        return cols, n

    def upar_samples(self, x, a, n, pid=0):
        out = np.zeros(n)
        lib().ora_sample_upar_n(C.byref(self.cfg), pid, float(x), float(a), n, _dp(out))
        return out

    def new_state(self, p, k, nu, pid):
        s = State()
        p = np.ascontiguousarray(p, dtype=np.float64)
        k = np.ascontiguousarray(k, dtype=np.float64)
        lib().ora_init_state(C.byref(self.cfg), C.byref(s), _dp(p), _dp(k), float(nu), int(pid))
        return s

    def event(self, s, record_events=0):
        """Advance state s by one event; optionally return its peeling events."""
        ty, t = self._alloc_tally()
        if record_events:
            ev = np.zeros(record_events, dtype=EVENT_DTYPE)
            ty.events, ty.cap = ev.ctypes.data, record_events
        r = lib().ora_event(C.byref(self.cfg), C.byref(s), C.byref(ty))
        if record_events:
            t["events"] = ev[: min(ty.nev, record_events)]
        return r, t

    def emission_events(self, s, cap=64):
        """Peeling events of the emission of a packet in state s."""
        ty, t = self._alloc_tally()
        ev = np.zeros(cap, dtype=EVENT_DTYPE)
        ty.events, ty.cap = ev.ctypes.data, cap
        lib().ora_emission(C.byref(self.cfg), C.byref(s), C.byref(ty))
        return ev[: min(ty.nev, cap)]


# ---------------------------------------------------------------- helpers
def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().ora_philox4x32_10(c, k, o)
    return [o[i] for i in range(4)]


def word(seed, pid, n):
    return lib().ora_word(seed, pid, n)


def voigt(a, x, method=0):
    """H(a, x): method 0 the Tasitsiomi (2006) form, 1 the Faddeeva function."""
    if method == 1:
        return faddeeva(a, x).real
    return lib().ora_voigt(float(a), float(x))


def faddeeva(a, x):
    """w(x + ia) by the trapezoidal rule with its pole residue (Re w = H)."""
    re, im = C.c_double(), C.c_double()
    lib().ora_faddeeva(float(a), float(x), C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def faddeeva_derivs(a, x):
    """(H, dH/da, dH/dx) of the Faddeeva H."""
    v = [C.c_double() for _ in range(3)]
    lib().ora_faddeeva_derivs(float(a), float(x), *[C.byref(t) for t in v])
    return tuple(t.value for t in v)


def u0(x, a):
    return lib().ora_u0(float(x), float(a))


def mu_sample(kind, r, g=0.0):
    return lib().ora_mu_sample(int(kind), float(r), float(g))


def phase(kind, mu, g=0.0):
    return lib().ora_phase(int(kind), float(mu), float(g))


def onb(n):
    n = np.ascontiguousarray(n, dtype=np.float64)
    b1, b2 = np.zeros(3), np.zeros(3)
    lib().ora_onb(_dp(n), _dp(b1), _dp(b2))
    return b1, b2


PH_ISO, PH_CORE, PH_WING, PH_HG = 0, 1, 2, 3
