"""ctypes binding of librascas_gb300.so (C ABI: include/rascas_gb300.h).

Names follow the C calls (``rascas_<name>`` -> ``Context.<name>``).  Arrays:
numpy arrays are host buffers (RASCAS_HOST); torch CUDA tensors are device
buffers (RASCAS_DEVICE) used on torch's current stream.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

HOST, DEVICE = 0, 1
PK_ACTIVE, PK_ESCAPED, PK_ABSORBED, PK_CAPPED, PK_ERROR = 0, 1, 2, 3, 4
DOMAIN_SPHERE, DOMAIN_SLAB, DOMAIN_CUBE, DOMAIN_SHELL = 0, 1, 2, 3
VOIGT_TASITSIOMI, VOIGT_FADDEEVA = 0, 1
TALLY_SPECTRUM, TALLY_PEEL_SPECTRA, TALLY_PEEL_IMAGES, TALLY_PEEL_CUBES = 0, 1, 2, 3
MAX_LINES, MAX_CHAN, MAX_DIRS = 4, 4, 8
C_CGS = 2.99792458e10

_STATUS = {0: "OK", -1: "E_ARG", -2: "E_OOM", -3: "E_CUDA", -4: "E_STATE", -5: "E_TIMEOUT", -6: "E_CAPPED"}


class Octree(C.Structure):
    _fields_ = [("noct", C.c_int32), ("nleaf", C.c_int32), ("son", C.c_void_p),
                ("n_HI", C.c_void_p), ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p),
                ("T", C.c_void_p), ("n_dust", C.c_void_p), ("n_metal", C.c_void_p), ("box_cm", C.c_double)]


class Domain(C.Structure):
    _fields_ = [("kind", C.c_int32), ("centre", C.c_double * 3), ("size", C.c_double), ("inner", C.c_double)]


class Line(C.Structure):
    _fields_ = [("nu0", C.c_double), ("A_ul", C.c_double), ("f_lu", C.c_double), ("mass_g", C.c_double),
                ("abundance", C.c_double), ("density", C.c_int32), ("phase", C.c_int32), ("nchan", C.c_int32),
                ("chan_A", C.c_double * MAX_CHAN), ("chan_nu", C.c_double * MAX_CHAN)]


class Dust(C.Structure):
    _fields_ = [("sigma", C.c_double), ("albedo", C.c_double), ("g", C.c_double)]


class Physics(C.Structure):
    _fields_ = [("recoil", C.c_int32), ("isotropic", C.c_int32), ("keep_dir", C.c_int32),
                ("fail_on_cap", C.c_int32), ("x_gauss", C.c_double), ("max_scatt", C.c_int64),
                ("max_steps", C.c_int64), ("tau_stop", C.c_double), ("seed", C.c_uint64),
                ("core_skip", C.c_double), ("core_skip_f", C.c_double)]


class Detector(C.Structure):
    _fields_ = [("nu_lo", C.c_double), ("nu_hi", C.c_double), ("nbin", C.c_int32), ("ndir", C.c_int32),
                ("npix", C.c_int32), ("cube", C.c_int32), ("dirs", (C.c_double * 3) * MAX_DIRS),
                ("fov", C.c_double), ("centre", C.c_double * 3)]


class PacketsIn(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("dir", C.c_void_p), ("nu", C.c_void_p), ("id", C.c_void_p)]


class PacketsOut(C.Structure):
    _fields_ = [("status", C.c_void_p), ("nscatt", C.c_void_p), ("nu", C.c_void_p), ("pos", C.c_void_p),
                ("dir", C.c_void_p), ("path", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "packets", "escaped", "absorbed", "capped", "errors", "nscatt_line", "nscatt_dust", "ncross",
        "npeel_rays", "npeel_cells", "upar_trials", "leaf_loads", "son_loads", "nbor_loads")] + [
        ("kernel_ms", C.c_double)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class Event(C.Structure):
    _fields_ = [("p", C.c_double * 3), ("k", C.c_double * 3), ("nu", C.c_double),
                ("leaf", C.c_int32), ("level", C.c_int32), ("ijk", C.c_int32 * 3), ("status", C.c_int32),
                ("ndraw", C.c_int64), ("nscatt", C.c_int64), ("nsteps", C.c_int64)]


class Model(C.Structure):
    _fields_ = [("tree", Octree), ("domain", Domain), ("nu_lo", C.c_double), ("nu_hi", C.c_double),
                ("packets", PacketsIn), ("npackets", C.c_int64)]


class Tune(C.Structure):
    _fields_ = [("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("refill", C.c_int32), ("ms", C.c_double)]


BATCH_PERSISTENT, BATCH_PER_MODEL = 0, 1

EVENT_DTYPE = np.dtype([("p", "<f8", 3), ("k", "<f8", 3), ("nu", "<f8"), ("leaf", "<i4"), ("level", "<i4"),
                        ("ijk", "<i4", 3), ("status", "<i4"), ("ndraw", "<i8"), ("nscatt", "<i8"),
                        ("nsteps", "<i8")])
assert EVENT_DTYPE.itemsize == C.sizeof(Event)

_lib = None


def library_path():
    return _build.LIB


def lib():
    """Load the CUDA library (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "rascas_create": [C.POINTER(vp), C.c_int],
            "rascas_destroy": [vp],
            "rascas_set_stream": [vp, vp],
            "rascas_load_octree": [vp, C.POINTER(Octree), C.c_int],
            "rascas_set_domain": [vp, C.POINTER(Domain)],
            "rascas_set_lines": [vp, C.POINTER(Line), i32, C.POINTER(Dust)],
            "rascas_set_physics": [vp, C.POINTER(Physics)],
            "rascas_set_limits": [vp, i64, C.c_double],
            "rascas_ray_columns": [vp, i64, vp, vp, C.c_double, C.c_double, vp, vp, vp, C.c_int],
            "rascas_propagate_batch_packets": [vp, i32, C.POINTER(PacketsOut), C.c_int, C.POINTER(Stats)],
            "rascas_set_detector": [vp, C.POINTER(Detector)],
            "rascas_zero_tallies": [vp],
            "rascas_set_peel_capacity": [vp, i64],
            "rascas_propagate": [vp, C.POINTER(PacketsIn), i64, C.POINTER(PacketsOut), C.c_int, C.POINTER(Stats)],
            "rascas_get_tally": [vp, C.c_int, vp, C.c_size_t, C.c_int],
            "rascas_ray_tau": [vp, i64, vp, vp, vp, vp, vp, vp, i32, vp, C.c_int],
            "rascas_trace": [vp, C.POINTER(PacketsIn), i64, i32, vp, vp, C.c_int],
            "rascas_eval_voigt": [vp, i64, vp, vp, vp, C.c_int],
            "rascas_set_voigt": [vp, C.c_int],
            "rascas_sample_upar": [vp, i64, vp, vp, vp, vp, vp, C.c_int],
            "rascas_update_fields": [vp, vp, vp, vp, vp, vp, vp, vp, C.c_int],
            "rascas_peel_adjoint": [vp, C.POINTER(PacketsIn), i64, vp, vp, vp, vp, C.c_int],
            "rascas_load_batch": [vp, C.POINTER(Model), i32, i32, C.c_int],
            "rascas_propagate_batch": [vp, i32, C.POINTER(Stats)],
            "rascas_get_batch_spectra": [vp, vp, C.c_size_t, C.c_int],
            "rascas_autotune_batch": [vp, i64, C.POINTER(Tune), C.POINTER(Tune), i32, C.POINTER(i32)],
            "rascas_set_batch_launch": [vp, C.POINTER(Tune)],
            "rascas_probe_issue_rates": [vp, C.POINTER(C.c_double)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.rascas_last_error.argtypes = [vp]
        L.rascas_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr()
    return a.ctypes.data


def _mem(*arrays):
    kinds = {(_is_torch(a) and a.is_cuda) for a in arrays if a is not None}
    if len(kinds) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return DEVICE if kinds == {True} else HOST


def _c(a, dtype):
    """Contiguous array of the given numpy dtype (host) or torch dtype (device)."""
    if a is None:
        return None
    if _is_torch(a):
        import torch
        td = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32,
              np.int64: torch.int64, np.uint64: torch.int64}[dtype]
        return a.to(td).contiguous()
    return np.ascontiguousarray(a, dtype=dtype)


class RascasError(RuntimeError):
    pass


class Context:
    """One library context on one CUDA device (rascas_create)."""

    def __init__(self, device=0):
        self._L = lib()
        self._h = C.c_void_p()
        r = self._L.rascas_create(C.byref(self._h), int(device))
        if r != 0:
            raise RascasError("rascas_create failed: %s" % _STATUS.get(r, r))
        self._keep = {}
        self.det = None
        self.nline = 0

    def close(self):
        if self._h:
            self._L.rascas_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, r, what):
        if r != 0:
            msg = self._L.rascas_last_error(self._h).decode()
            raise RascasError("%s: %s (%s)" % (what, _STATUS.get(r, r), msg))

    # ------------------------------------------------------------ set-up
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        h = getattr(stream, "cuda_stream", stream)
        self._ck(self._L.rascas_set_stream(self._h, C.c_void_p(h) if h else None), "set_stream")

    def load_octree(self, son, n_HI, vx, vy, vz, T, n_dust, n_metal=None, box_cm=1.0):
        arrs = [_c(son, np.int32)] + [_c(a, np.float32) for a in (n_HI, vx, vy, vz, T, n_dust, n_metal)]
        mem = _mem(*arrs)
        t = Octree()
        t.noct = int(arrs[0].shape[0]) // 8
        t.nleaf = int(arrs[1].shape[0])
        self.nleaf = t.nleaf
        t.son, t.n_HI, t.vx, t.vy, t.vz, t.T, t.n_dust, t.n_metal = [_ptr(a) for a in arrs]
        t.box_cm = float(box_cm)
        self._ck(self._L.rascas_load_octree(self._h, C.byref(t), mem), "load_octree")

    def set_domain(self, kind, centre, size, inner=0.0):
        d = Domain()
        d.kind = int(kind)
        d.centre[:] = [float(v) for v in centre]
        d.size = float(size)
        d.inner = float(inner)
        self._ck(self._L.rascas_set_domain(self._h, C.byref(d)), "set_domain")

    def set_lines(self, lines, dust=None):
        """lines: objects with lambda_A, A_ul, f_lu, mass_g, density, abundance,
        phase and all_channels() -> [(A, lambda_A)] (Table 1 rows)."""
        arr = (Line * len(lines))()
        for i, ln in enumerate(lines):
            L = arr[i]
            L.nu0 = C_CGS / (ln.lambda_A * 1e-8)
            L.A_ul, L.f_lu, L.mass_g = ln.A_ul, ln.f_lu, ln.mass_g
            L.abundance = ln.abundance
            L.density = 1 if ln.density == 1 else 0
            L.phase = ln.phase
            ch = ln.all_channels()
            L.nchan = len(ch)
            for c, (A, lam) in enumerate(ch):
                L.chan_A[c] = A
                L.chan_nu[c] = C_CGS / (lam * 1e-8)
        d = Dust()
        if dust is not None:
            d.sigma, d.albedo, d.g = dust.sigma, dust.albedo, dust.g
        self.nline = len(lines)
        self._ck(self._L.rascas_set_lines(self._h, arr, len(lines), C.byref(d)), "set_lines")

    def set_voigt(self, method):
        """H(a,x) method of every later call: VOIGT_TASITSIOMI or VOIGT_FADDEEVA."""
        self._ck(self._L.rascas_set_voigt(self._h, int(method)), "set_voigt")

    def set_physics(self, recoil=1, isotropic=0, keep_dir=0, x_gauss=8.0, max_scatt=0, max_steps=0,
                    tau_stop=50.0, seed=0, fail_on_cap=0, core_skip=0.0, core_skip_f=0.0):
        p = Physics()
        p.recoil, p.isotropic, p.keep_dir, p.fail_on_cap = int(recoil), int(isotropic), int(keep_dir), int(fail_on_cap)
        p.x_gauss = float(x_gauss)
        p.max_scatt, p.max_steps = int(max_scatt), int(max_steps)
        p.tau_stop = float(tau_stop) if math.isfinite(tau_stop) else 1e300
        p.seed = int(seed)
        p.core_skip, p.core_skip_f = float(core_skip), float(core_skip_f)
        self._ck(self._L.rascas_set_physics(self._h, C.byref(p)), "set_physics")

    def set_limits(self, max_iterations=0, time_limit_s=0.0):
        """Bounded device work (rascas_set_limits): 0 = no limit."""
        self._ck(self._L.rascas_set_limits(self._h, int(max_iterations), float(time_limit_s)), "set_limits")

    def set_detector(self, nu_lo, nu_hi, nbin, dirs=(), npix=0, fov=1.0, centre=(0.5, 0.5, 0.5), cube=0):
        d = Detector()
        d.nu_lo, d.nu_hi, d.nbin = float(nu_lo), float(nu_hi), int(nbin)
        dirs = np.asarray(dirs, dtype=np.float64).reshape(-1, 3)
        d.ndir = dirs.shape[0]
        for i in range(d.ndir):
            d.dirs[i][:] = list(dirs[i])
        d.npix, d.fov, d.cube = int(npix), float(fov), int(cube)
        d.centre[:] = [float(v) for v in centre]
        self._ck(self._L.rascas_set_detector(self._h, C.byref(d)), "set_detector")
        self.det = (int(nbin), d.ndir, int(npix), int(cube))

    def zero_tallies(self):
        self._ck(self._L.rascas_zero_tallies(self._h), "zero_tallies")

    def set_peel_capacity(self, records):
        self._ck(self._L.rascas_set_peel_capacity(self._h, int(records)), "set_peel_capacity")

    def setup(self, wl):
        """Load a workload description (medium, domain, lines, dust, physics,
        detector) -- any object with the attributes of synth.Workload."""
        m = wl.medium
        self.load_octree(m.tree.son, m.n_HI, m.vx, m.vy, m.vz, m.T, m.n_dust,
                         m.n_metal if any(l.density == 1 for l in wl.lines) else None, m.box_cm)
        self.set_domain(wl.domain.kind, wl.domain.centre, wl.domain.size, getattr(wl.domain, "inner", 0.0))
        self.set_lines(wl.lines, wl.dust)
        ph = wl.physics
        self.set_physics(ph.recoil, ph.isotropic, ph.keep_direction, ph.x_gauss, ph.max_scatt, ph.max_steps,
                         ph.tau_stop, ph.seed, 0, getattr(ph, "core_skip", 0.0), getattr(ph, "core_skip_f", 0.0))
        self.set_voigt(getattr(ph, "voigt", VOIGT_TASITSIOMI))
        d = wl.detector
        self.set_detector(d.nu_lo, d.nu_hi, d.nbin, d.dirs, d.npix, d.fov, d.centre, d.cube)

    # ------------------------------------------------------------ hot path
    def propagate(self, pos, dir, nu, ids, out=None, stats=True):
        """Propagate packets.  out: None, or a dict with any of status, nscatt,
        nu, pos, dir, path arrays (same kind as the inputs).  Returns a dict of
        run statistics (or None with stats=False)."""
        pos, dir, nu = _c(pos, np.float64), _c(dir, np.float64), _c(nu, np.float64)
        ids = _c(ids, np.uint64)
        mem = _mem(pos, dir, nu, ids)
        n = int(nu.shape[0])
        pin = PacketsIn(_ptr(pos), _ptr(dir), _ptr(nu), _ptr(ids))
        pout = None
        if out is not None:
            pout = PacketsOut(*[_ptr(out.get(k)) for k in ("status", "nscatt", "nu", "pos", "dir", "path")])
        st = Stats() if stats else None
        self._stream_sync_torch(mem)
        r = self._L.rascas_propagate(self._h, C.byref(pin), n, C.byref(pout) if pout else None, mem,
                                     C.byref(st) if st else None)
        self._ck(r, "propagate")
        return st.as_dict() if st else None

    def get_tally(self, kind, device=None):
        nbin, ndir, npix, cube = self.det
        shape = {TALLY_SPECTRUM: (nbin,), TALLY_PEEL_SPECTRA: (ndir, nbin),
                 TALLY_PEEL_IMAGES: (ndir, npix, npix), TALLY_PEEL_CUBES: (ndir, npix, npix, nbin)}[kind]
        count = int(np.prod(shape))
        if device is not None:
            import torch
            dst = torch.empty(shape, dtype=torch.float32, device=device)
            self._ck(self._L.rascas_get_tally(self._h, kind, C.c_void_p(dst.data_ptr()), count, DEVICE), "get_tally")
            return dst
        dst = np.zeros(shape, dtype=np.float32)
        self._ck(self._L.rascas_get_tally(self._h, kind, C.c_void_p(dst.ctypes.data), count, HOST), "get_tally")
        return dst

    def ray_tau(self, pos, dir, nu, cap=0):
        pos, dir, nu = _c(pos, np.float64), _c(dir, np.float64), _c(nu, np.float64)
        mem = _mem(pos, dir, nu)
        n = int(nu.shape[0])
        if mem == DEVICE:
            import torch
            dev = nu.device
            tau = torch.empty(n, dtype=torch.float64, device=dev)
            ncell = torch.empty(n, dtype=torch.int32, device=dev)
            cells = torch.empty((n, cap), dtype=torch.int32, device=dev) if cap else None
            lens = torch.empty((n, cap), dtype=torch.float64, device=dev) if cap else None
        else:
            tau = np.zeros(n)
            ncell = np.zeros(n, np.int32)
            cells = np.zeros((n, cap), np.int32) if cap else None
            lens = np.zeros((n, cap)) if cap else None
        self._stream_sync_torch(mem)
        r = self._L.rascas_ray_tau(self._h, n, _ptr(pos), _ptr(dir), _ptr(nu), _ptr(tau), _ptr(cells), _ptr(lens),
                                   int(cap), _ptr(ncell), mem)
        self._ck(r, "ray_tau")
        return tau, cells, lens, ncell

    def ray_columns(self, pos, dir, sigma_HI=0.0, sigma_dust=0.0):
        """Column densities [n, 3] (N_HI, N_dust, N_metal) from pos along dir
        to the domain border, the continuum optical depth sigma_HI N_HI +
        sigma_dust N_dust [n] and the leaves crossed [n]."""
        pos, dir = _c(pos, np.float64), _c(dir, np.float64)
        mem = _mem(pos, dir)
        n = int(pos.shape[0])
        if mem == DEVICE:
            import torch
            dev = pos.device
            cols = torch.empty((n, 3), dtype=torch.float64, device=dev)
            tau = torch.empty(n, dtype=torch.float64, device=dev)
            ncell = torch.empty(n, dtype=torch.int32, device=dev)
        else:
            cols, tau, ncell = np.zeros((n, 3)), np.zeros(n), np.zeros(n, np.int32)
        self._stream_sync_torch(mem)
        r = self._L.rascas_ray_columns(self._h, n, _ptr(pos), _ptr(dir), float(sigma_HI), float(sigma_dust),
                                       _ptr(cols), _ptr(tau), _ptr(ncell), mem)
        self._ck(r, "ray_columns")
        return cols, tau, ncell

    def trace(self, pos, dir, nu, ids, max_events):
        """Events of each packet (host arrays only): structured array
        [n, max_events] (fields of rascas_event) and the counts [n]."""
        pos, dir, nu = _c(pos, np.float64), _c(dir, np.float64), _c(nu, np.float64)
        ids = _c(ids, np.uint64)
        n = int(nu.shape[0])
        ev = np.zeros((n, max_events), dtype=EVENT_DTYPE)
        cnt = np.zeros(n, np.int32)
        pin = PacketsIn(_ptr(pos), _ptr(dir), _ptr(nu), _ptr(ids))
        r = self._L.rascas_trace(self._h, C.byref(pin), n, int(max_events), ev.ctypes.data, cnt.ctypes.data, HOST)
        self._ck(r, "trace")
        return ev, cnt

    def eval_voigt(self, a, x):
        a, x = _c(a, np.float32), _c(x, np.float64)
        mem = _mem(a, x)
        n = int(x.shape[0])
        if mem == DEVICE:
            import torch
            H = torch.empty(n, dtype=torch.float32, device=x.device)
        else:
            H = np.zeros(n, np.float32)
        self._stream_sync_torch(mem)
        self._ck(self._L.rascas_eval_voigt(self._h, n, _ptr(a), _ptr(x), _ptr(H), mem), "eval_voigt")
        return H

    def sample_upar(self, x, a, ids):
        x, a, ids = _c(x, np.float64), _c(a, np.float32), _c(ids, np.uint64)
        mem = _mem(x, a, ids)
        n = int(x.shape[0])
        if mem == DEVICE:
            import torch
            u = torch.empty(n, dtype=torch.float32, device=x.device)
            nd = torch.empty(n, dtype=torch.int32, device=x.device)
        else:
            u, nd = np.zeros(n, np.float32), np.zeros(n, np.int32)
        self._stream_sync_torch(mem)
        self._ck(self._L.rascas_sample_upar(self._h, n, _ptr(x), _ptr(a), _ptr(ids), _ptr(u), _ptr(nd), mem),
                 "sample_upar")
        return u, nd

    def probe_issue_rates(self):
        """Measured issue rates (warp-instructions/s, whole device) of the FP32
        FMA, FP64 FMA, MUFU and IMAD pipes."""
        r = (C.c_double * 4)()
        self._ck(self._L.rascas_probe_issue_rates(self._h, r), "probe_issue_rates")
        return {"ffma": r[0], "dfma": r[1], "mufu": r[2], "imad": r[3]}

    # ------------------------------------------------------------ adjoint
    def update_fields(self, n_HI, vx, vy, vz, T, n_dust, n_metal=None):
        arrs = [_c(a, np.float32) for a in (n_HI, vx, vy, vz, T, n_dust, n_metal)]
        mem = _mem(*arrs)
        self._stream_sync_torch(mem)
        self._ck(self._L.rascas_update_fields(self._h, *[_ptr(a) for a in arrs], mem), "update_fields")

    def peel_adjoint(self, pos, dir, nu, ids, g_cube=None, g_img=None, g_spec=None, nleaf=None):
        """[6, nleaf] gradient (n_HI, vx, vy, vz, T, n_dust) of
        sum(g_cube*cube) + sum(g_img*img) + sum(g_spec*spec) with the
        scattering record of these packets held fixed."""
        pos, dir, nu = _c(pos, np.float64), _c(dir, np.float64), _c(nu, np.float64)
        ids = _c(ids, np.uint64)
        gs = [_c(g, np.float32) for g in (g_cube, g_img, g_spec)]
        mem = _mem(pos, dir, nu, ids, *gs)
        n = int(nu.shape[0])
        if nleaf is None:
            nleaf = self.nleaf
        if mem == DEVICE:
            import torch
            grad = torch.zeros((6, nleaf), dtype=torch.float32, device=nu.device)
        else:
            grad = np.zeros((6, nleaf), np.float32)
        pin = PacketsIn(_ptr(pos), _ptr(dir), _ptr(nu), _ptr(ids))
        self._stream_sync_torch(mem)
        self._ck(self._L.rascas_peel_adjoint(self._h, C.byref(pin), n, *[_ptr(g) for g in gs], _ptr(grad), mem),
                 "peel_adjoint")
        return grad

    # ------------------------------------------------------------ batches
    def load_batch(self, workloads, nbin):
        """Load independent models (objects with medium, domain, detector
        (nu_lo, nu_hi) and packets, like synth.Workload) as one batch.  Lines,
        dust and physics must already be set on the context."""
        arr = (Model * len(workloads))()
        keep = []
        for i, wl in enumerate(workloads):
            m = wl.medium
            a = [np.ascontiguousarray(m.tree.son, dtype=np.int32)] + [
                np.ascontiguousarray(x, dtype=np.float32) for x in (m.n_HI, m.vx, m.vy, m.vz, m.T, m.n_dust)]
            pk = wl.packets
            b = [np.ascontiguousarray(pk.pos, dtype=np.float64), np.ascontiguousarray(pk.dir, dtype=np.float64),
                 np.ascontiguousarray(pk.nu, dtype=np.float64), np.ascontiguousarray(pk.ids, dtype=np.uint64)]
            keep += a + b
            M = arr[i]
            M.tree.noct, M.tree.nleaf = a[0].size // 8, a[1].size
            M.tree.son, M.tree.n_HI, M.tree.vx, M.tree.vy, M.tree.vz, M.tree.T, M.tree.n_dust = [x.ctypes.data for x in a]
            M.tree.n_metal = None
            M.tree.box_cm = float(m.box_cm)
            M.domain.kind = wl.domain.kind
            M.domain.centre[:] = [float(v) for v in wl.domain.centre]
            M.domain.size = float(wl.domain.size)
            M.domain.inner = float(getattr(wl.domain, "inner", 0.0))
            M.nu_lo, M.nu_hi = float(wl.detector.nu_lo), float(wl.detector.nu_hi)
            M.packets = PacketsIn(*[x.ctypes.data for x in b])
            M.npackets = int(pk.n)
        self.batch_shape = (len(workloads), int(nbin))
        self._batch_counts = [int(wl.packets.n) for wl in workloads]
        self._ck(self._L.rascas_load_batch(self._h, arr, len(workloads), int(nbin), HOST), "load_batch")

    def propagate_batch(self, mode=BATCH_PERSISTENT):
        st = Stats()
        self._ck(self._L.rascas_propagate_batch(self._h, int(mode), C.byref(st)), "propagate_batch")
        return st.as_dict()

    def propagate_batch_packets(self, mode=BATCH_PERSISTENT):
        """propagate_batch with per-packet results (host arrays, models in
        load order): (dict of status, nscatt, nu, pos, dir, path; stats)."""
        n = sum(self._batch_counts)
        out = {"status": np.zeros(n, np.int32), "nscatt": np.zeros(n, np.int64), "nu": np.zeros(n),
               "pos": np.zeros((n, 3)), "dir": np.zeros((n, 3)), "path": np.zeros(n)}
        pout = PacketsOut(*[_ptr(out[k]) for k in ("status", "nscatt", "nu", "pos", "dir", "path")])
        st = Stats()
        self._ck(self._L.rascas_propagate_batch_packets(self._h, int(mode), C.byref(pout), HOST, C.byref(st)),
                 "propagate_batch_packets")
        return out, st.as_dict()

    def get_batch_spectra(self):
        dst = np.zeros(self.batch_shape, dtype=np.float32)
        self._ck(self._L.rascas_get_batch_spectra(self._h, C.c_void_p(dst.ctypes.data), dst.size, HOST),
                 "get_batch_spectra")
        return dst

    def set_batch_launch(self, block=128, blocks_per_sm=0, refill=1):
        t = Tune()
        t.block, t.blocks_per_sm, t.refill = int(block), int(blocks_per_sm), int(refill)
        self._ck(self._L.rascas_set_batch_launch(self._h, C.byref(t)), "set_batch_launch")

    def autotune_batch(self, max_scatt=1000):
        best = Tune()
        tried = (Tune * 64)()
        nt = C.c_int32()
        self._ck(self._L.rascas_autotune_batch(self._h, int(max_scatt), C.byref(best), tried, 64, C.byref(nt)),
                 "autotune_batch")
        return {"best": (best.block, best.blocks_per_sm, best.ms), "refill": best.refill,
                "tried": [(tried[i].block, tried[i].blocks_per_sm, tried[i].ms, tried[i].refill)
                          for i in range(nt.value)]}

    def _stream_sync_torch(self, mem):
        """Device calls run on torch's current stream."""
        if mem == DEVICE:
            import torch
            self.set_stream(torch.cuda.current_stream())
