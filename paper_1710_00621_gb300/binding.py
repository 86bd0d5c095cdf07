"""ctypes binding of libcmbws (argument marshalling only; every step runs in the library).

Tensors passed as vectors or maps must be CUDA, float64 and contiguous; the library
reads and writes them in place on the given stream (default: torch's current stream).
"""
import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "libcmbws.so")
HEADER = os.path.join(ROOT, "include", "cmbws.h")

CMBWS_GRID_GL = 0
CMBWS_GRID_HEALPIX = 1
CMBWS_FP64 = 0
CMBWS_FP32 = 1
CMBWS_FP32X2 = 2
CMBWS_TF32 = 3
CMBWS_3XTF32 = 4
CMBWS_BF16 = 5
CMBWS_BF16X3 = 6

_ERRORS = {-1: "CMBWS_ERR_ARG", -2: "CMBWS_ERR_CUDA", -3: "CMBWS_ERR_NOMEM",
           -4: "CMBWS_ERR_SINGULAR", -5: "CMBWS_ERR_BREAKDOWN", -6: "CMBWS_ERR_NOT_CONVERGED",
           -7: "CMBWS_ERR_TIMEOUT", -8: "CMBWS_ERR_COMM"}

_lib = None


class CmbwsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class ModelDesc(ctypes.Structure):
    _fields_ = [("ncomp", ctypes.c_int), ("nobs", ctypes.c_int),
                ("lmax_comp", ctypes.POINTER(ctypes.c_int)),
                ("band_grid", ctypes.POINTER(ctypes.c_void_p)),
                ("beam", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))),
                ("cl", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))),
                ("ninv", ctypes.POINTER(ctypes.c_void_p)),
                ("mix_scalar", ctypes.POINTER(ctypes.c_double)),
                ("mix_grid", ctypes.POINTER(ctypes.c_void_p)),
                ("mix_map", ctypes.POINTER(ctypes.c_void_p))]


class CgOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("precond", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("timeout_s", ctypes.c_double), ("cert_prec", ctypes.c_int)]


class CgReport(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("n_sht", ctypes.c_int), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def library_path():
    return LIB_PATH


def load_library(path=None):
    """Load libcmbws.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libcmbws.so not found at {p}; run __graft_entry__.build() first")
    lib = ctypes.CDLL(p)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.cmbws_last_error.restype = ctypes.c_char_p
    lib.cmbws_version.restype = ctypes.c_char_p
    lib.cmbws_plan_grid.argtypes = [i, i, i, ctypes.POINTER(vp)]
    lib.cmbws_grid_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(i),
                                    ctypes.POINTER(ctypes.POINTER(d)), ctypes.POINTER(ctypes.POINTER(d))]
    lib.cmbws_grid_rings.argtypes = [vp, ctypes.POINTER(ctypes.POINTER(d)),
                                     ctypes.POINTER(ctypes.POINTER(i)),
                                     ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)), ctypes.POINTER(i)]
    lib.cmbws_grid_destroy.argtypes = [vp]
    lib.cmbws_sht_synth.argtypes = [vp, i, vp, vp, i, vp]
    lib.cmbws_sht_analysis.argtypes = [vp, i, vp, vp, i, i, vp]
    lib.cmbws_sht_analysis_noalloc.argtypes = [vp, i, vp, vp, i, i, vp]
    lib.cmbws_model_create.argtypes = [ctypes.POINTER(ModelDesc), i, vp, ctypes.POINTER(vp)]
    lib.cmbws_model_destroy.argtypes = [vp]
    lib.cmbws_model_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(i),
                                     ctypes.POINTER(i)]
    lib.cmbws_apply_A.argtypes = [vp, vp, vp, vp]
    lib.cmbws_apply_precond.argtypes = [vp, vp, vp, vp]
    lib.cmbws_rhs.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, vp]
    lib.cmbws_project.argtypes = [vp, vp, ctypes.POINTER(vp), vp]
    lib.cmbws_grad_terms.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, vp]
    lib.cmbws_grad_mix_maps.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                        ctypes.POINTER(vp), vp]
    lib.cmbws_model_add_mask_precond.argtypes = [vp, i, i, vp, i, vp]
    lib.cmbws_apply_M_add.argtypes = [vp, vp, vp, vp]
    lib.cmbws_apply_M_diag.argtypes = [vp, vp, vp, vp]
    lib.cmbws_model_merge_precond.argtypes = [vp, ctypes.POINTER(i), vp]
    lib.cmbws_model_set_vcycle.argtypes = [vp, i]
    lib.cmbws_model_set_graphs.argtypes = [vp, i]
    lib.cmbws_set_autotune.argtypes = [i]
    lib.cmbws_grid_tuning.argtypes = [vp, i, i, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(i)]
    u64 = ctypes.c_uint64
    lib.cmbws_draw.argtypes = [u64, u64, u64, ctypes.c_int64, ctypes.c_int64, i, vp, vp]
    lib.cmbws_cr_rhs.argtypes = [vp, ctypes.POINTER(vp), u64, u64, vp, vp]
    lib.cmbws_cr_sample.argtypes = [vp, ctypes.POINTER(vp), u64, u64, vp, ctypes.POINTER(CgOpts),
                                    ctypes.POINTER(CgReport), vp]
    lib.cmbws_powerlaw_mixing.argtypes = [d, vp, vp, ctypes.c_int64, vp, vp]
    lib.cmbws_profile_enable.argtypes = [i]
    lib.cmbws_device_status.argtypes = [vp]
    lib.cmbws_cg_history.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(d), i,
                                     ctypes.POINTER(i)]
    lib.cmbws_cg_track_error.argtypes = [vp, vp, vp]
    lib.cmbws_cg_checkpointing.argtypes = [vp, i]
    lib.cmbws_model_set_precond_prec.argtypes = [vp, i]
    lib.cmbws_model_set_shard.argtypes = [vp, ctypes.POINTER(i), i]
    lib.cmbws_cg_solve_sharded.argtypes = [vp, vp, vp, ctypes.POINTER(CgOpts), vp, vp,
                                           ctypes.POINTER(CgReport), vp]
    lib.cmbws_cg_state_export.argtypes = [vp, vp, vp, vp, ctypes.POINTER(d), vp]
    lib.cmbws_cg_resume.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.POINTER(d),
                                    ctypes.POINTER(CgOpts), ctypes.POINTER(CgReport), vp]
    lib.cmbws_testing_stall_waits.argtypes = [ctypes.c_longlong]
    lib.cmbws_profile_read.argtypes = [ctypes.POINTER(d), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d),
                                       ctypes.POINTER(d), i]
    lib.cmbws_cg_solve.argtypes = [vp, vp, vp, ctypes.POINTER(CgOpts), ctypes.POINTER(CgReport), vp]
    lib.cmbws_cg_solve_batched.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                           ctypes.POINTER(CgOpts), ctypes.POINTER(CgReport), i, vp]
    _lib = lib
    return lib


def exported_symbols():
    """Names of the functions declared in include/cmbws.h."""
    src = open(HEADER).read()
    return sorted(set(re.findall(r"\b(cmbws_[A-Za-z_0-9]+)\s*\(", src)))


def _check(code):
    if code != 0:
        raise CmbwsError(code, load_library().cmbws_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dptr(t, n=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA float64 tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n}")
    return ctypes.c_void_p(t.data_ptr())


class Grid:
    """A planned ring grid (owns the library handle)."""

    def __init__(self, handle, kind, n, lmax):
        self.handle = handle
        self.kind, self.n, self.lmax = kind, n, lmax
        npix = ctypes.c_int64()
        nring = ctypes.c_int()
        th = ctypes.POINTER(ctypes.c_double)()
        w = ctypes.POINTER(ctypes.c_double)()
        _check(load_library().cmbws_grid_info(handle, ctypes.byref(npix), ctypes.byref(nring),
                                              ctypes.byref(th), ctypes.byref(w)))
        self.npix, self.nring = npix.value, nring.value
        self.theta = np.ctypeslib.as_array(th, (self.nring,)).copy()
        self.weight = np.ctypeslib.as_array(w, (self.nring,)).copy()
        ph = ctypes.POINTER(ctypes.c_double)()
        nphi = ctypes.POINTER(ctypes.c_int)()
        off = ctypes.POINTER(ctypes.c_int64)()
        L = ctypes.c_int()
        _check(load_library().cmbws_grid_rings(handle, ctypes.byref(ph), ctypes.byref(nphi),
                                               ctypes.byref(off), ctypes.byref(L)))
        self.phi0 = np.ctypeslib.as_array(ph, (self.nring,)).copy()
        self.nphi = np.ctypeslib.as_array(nphi, (self.nring,)).copy()
        self.offset = np.ctypeslib.as_array(off, (self.nring + 1,)).copy()

    def pixel_coords(self):
        """(cos theta, phi) of every pixel, ring order."""
        z = np.repeat(np.cos(self.theta), self.nphi)
        ph = np.concatenate([self.phi0[r] + 2 * np.pi * np.arange(self.nphi[r]) / self.nphi[r]
                             for r in range(self.nring)])
        return z, ph

    def pixel_weights(self):
        return np.repeat(self.weight, self.nphi)

    def close(self):
        if self.handle:
            load_library().cmbws_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cmbws_plan_grid(kind, n, lmax):
    h = ctypes.c_void_p()
    _check(load_library().cmbws_plan_grid(int(kind), int(n), int(lmax), ctypes.byref(h)))
    return Grid(h, kind, n, lmax)


def cmbws_grid_info(grid):
    return grid.npix, grid.nring, grid.theta, grid.weight


def cmbws_grid_rings(grid):
    return grid.phi0, grid.nphi, grid.offset, grid.lmax


def cmbws_grid_destroy(grid):
    grid.close()


def cmbws_sht_synth(grid, prec, alm, map_out, nmaps=1, stream=None):
    nalm = (grid.lmax + 1) ** 2
    _check(load_library().cmbws_sht_synth(grid.handle, int(prec), _dptr(alm, nmaps * nalm, "alm"),
                                          _dptr(map_out, nmaps * grid.npix, "map"), int(nmaps),
                                          _stream(stream)))


def cmbws_sht_analysis(grid, prec, map_in, alm, nmaps=1, weighted=1, stream=None):
    nalm = (grid.lmax + 1) ** 2
    _check(load_library().cmbws_sht_analysis(grid.handle, int(prec),
                                             _dptr(map_in, nmaps * grid.npix, "map"),
                                             _dptr(alm, nmaps * nalm, "alm"), int(nmaps),
                                             int(weighted), _stream(stream)))


def cmbws_sht_analysis_noalloc(grid, prec, map_in, alm, nmaps=1, weighted=1, stream=None):
    """cmbws_sht_analysis without device allocation (32 MiB static workspace per GPU)."""
    nalm = (grid.lmax + 1) ** 2
    _check(load_library().cmbws_sht_analysis_noalloc(grid.handle, int(prec),
                                                     _dptr(map_in, nmaps * grid.npix, "map"),
                                                     _dptr(alm, nmaps * nalm, "alm"), int(nmaps),
                                                     int(weighted), _stream(stream)))


class Model:
    """A model handle (owns it); keeps its grids alive."""

    def __init__(self, handle, grids, lmax_comp, nobs=None):
        self.handle = handle
        self.nobs = len(grids) if nobs is None else nobs
        self.all_grids = grids
        self.grids = grids[:self.nobs]
        self.lmax_comp = list(lmax_comp)
        nvec = ctypes.c_int64()
        na = ctypes.c_int()
        nm = ctypes.c_int()
        _check(load_library().cmbws_model_info(handle, ctypes.byref(nvec), ctypes.byref(na),
                                               ctypes.byref(nm)))
        self.nvec, self.nsht_A, self.nsht_M = nvec.value, na.value, nm.value

    def close(self):
        if self.handle:
            load_library().cmbws_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _handle(g):
    return g.handle.value if isinstance(g.handle, ctypes.c_void_p) else g.handle


def cmbws_model_create(lmax_comp, band_grids, beams, cls, ninv, mix_scalar, prec=CMBWS_FP64,
                       stream=None, mix_grids=None, mix_maps=None):
    """lmax_comp: [ncomp] ints; band_grids: [nobs] Grid; beams: [nobs] arrays b_l (l <= L_nu);
    cls: [ncomp] arrays C_l or None; ninv: [nobs] CUDA float64 maps; mix_scalar: [nobs, ncomp];
    mix_grids / mix_maps: optional [nobs][ncomp] Grid / CUDA float64 map (None = scalar pair)."""
    ncomp, nobs = len(lmax_comp), len(band_grids)
    q = np.ascontiguousarray(np.asarray(mix_scalar, dtype=np.float64).reshape(nobs, ncomp))
    lk = (ctypes.c_int * ncomp)(*[int(v) for v in lmax_comp])
    gh = (ctypes.c_void_p * nobs)(*[_handle(g) for g in band_grids])
    keep = []
    bp = (ctypes.POINTER(ctypes.c_double) * nobs)()
    for nu in range(nobs):
        b = np.ascontiguousarray(np.asarray(beams[nu], dtype=np.float64))
        if b.size < band_grids[nu].lmax + 1:
            raise ValueError(f"beam {nu} needs {band_grids[nu].lmax + 1} entries")
        keep.append(b)
        bp[nu] = b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cp = (ctypes.POINTER(ctypes.c_double) * ncomp)()
    for k in range(ncomp):
        if cls[k] is None:
            cp[k] = ctypes.POINTER(ctypes.c_double)()
        else:
            c = np.ascontiguousarray(np.asarray(cls[k], dtype=np.float64))
            if c.size < lmax_comp[k] + 1:
                raise ValueError(f"C_l of component {k} needs {lmax_comp[k] + 1} entries")
            keep.append(c)
            cp[k] = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    nv = (ctypes.c_void_p * nobs)(*[_dptr(ninv[nu], band_grids[nu].npix, f"ninv[{nu}]").value
                                    for nu in range(nobs)])
    mg = ctypes.POINTER(ctypes.c_void_p)()
    mm = ctypes.POINTER(ctypes.c_void_p)()
    extra_grids = []
    if mix_maps is not None:
        mg = (ctypes.c_void_p * (nobs * ncomp))()
        mm = (ctypes.c_void_p * (nobs * ncomp))()
        for nu in range(nobs):
            for k in range(ncomp):
                t = mix_maps[nu][k]
                if t is None:
                    continue
                g = mix_grids[nu][k]
                extra_grids.append(g)
                mg[nu * ncomp + k] = _handle(g)
                mm[nu * ncomp + k] = _dptr(t, g.npix, f"mix_map[{nu}][{k}]").value
    desc = ModelDesc(ncomp, nobs, lk, gh, bp, cp, nv, q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     mg, mm)
    h = ctypes.c_void_p()
    _check(load_library().cmbws_model_create(ctypes.byref(desc), int(prec), _stream(stream),
                                             ctypes.byref(h)))
    mdl = Model(h, list(band_grids) + extra_grids, lmax_comp, nobs=nobs)
    mdl.mix_grids = ([[None if mix_maps[nu][k] is None else mix_grids[nu][k] for k in range(ncomp)]
                      for nu in range(nobs)] if mix_maps is not None else None)
    return mdl


def cmbws_model_destroy(model):
    model.close()


def cmbws_model_info(model):
    return model.nvec, model.nsht_A, model.nsht_M


def cmbws_apply_A(model, x, y, stream=None):
    _check(load_library().cmbws_apply_A(model.handle, _dptr(x, model.nvec, "x"),
                                        _dptr(y, model.nvec, "y"), _stream(stream)))


def cmbws_apply_precond(model, r, z, stream=None):
    _check(load_library().cmbws_apply_precond(model.handle, _dptr(r, model.nvec, "r"),
                                               _dptr(z, model.nvec, "z"), _stream(stream)))


def cmbws_rhs(model, d, b, omega1=None, omega2=None, stream=None):
    nobs = len(model.grids)
    dp = (ctypes.c_void_p * nobs)(*[_dptr(d[nu], model.grids[nu].npix, f"d[{nu}]").value
                                    for nu in range(nobs)])
    if omega1 is not None:
        w1 = (ctypes.c_void_p * nobs)(*[_dptr(omega1[nu], model.grids[nu].npix, f"omega1[{nu}]").value
                                        for nu in range(nobs)])
    else:
        w1 = ctypes.POINTER(ctypes.c_void_p)()
    w2 = _dptr(omega2, model.nvec, "omega2") if omega2 is not None else ctypes.c_void_p()
    _check(load_library().cmbws_rhs(model.handle, dp, w1, w2, _dptr(b, model.nvec, "b"),
                                    _stream(stream)))


CMBWS_TUNE_DEFAULT = 0
CMBWS_TUNE_HEURISTIC = 1
CMBWS_TUNE_MEASURED = 2
SYNTH_TILES = [(2, 128), (1, 128), (1, 64), (4, 64)]   # (ring pairs per thread, threads per CTA)


def cmbws_set_autotune(mode):
    """Tile choice of the Legendre synthesis: CMBWS_TUNE_DEFAULT, _HEURISTIC or _MEASURED."""
    _check(load_library().cmbws_set_autotune(int(mode)))


def cmbws_grid_tuning(grid, prec, nmaps):
    """The measured tile decision for synthesis on a grid: {"variant", "tile", "ms"} or None."""
    v = ctypes.c_int()
    n = ctypes.c_int()
    ms = (ctypes.c_float * 8)()
    _check(load_library().cmbws_grid_tuning(grid.handle, int(prec), int(nmaps), ctypes.byref(v),
                                            ms, ctypes.byref(n)))
    if v.value < 0:
        return None
    return {"variant": v.value, "tile": SYNTH_TILES[v.value], "ms": [ms[i] for i in range(n.value)]}


def cmbws_model_set_graphs(model, on):
    """Replay the solvers' operator applies from CUDA graphs (True) or launch them eagerly."""
    _check(load_library().cmbws_model_set_graphs(model.handle, 1 if on else 0))


CMBWS_VCYCLE_BASIC = 0
CMBWS_VCYCLE_OPTIMIZED = 1


def cmbws_model_set_vcycle(model, kind):
    """V-cycle of the mask preconditioners: CMBWS_VCYCLE_BASIC or CMBWS_VCYCLE_OPTIMIZED."""
    _check(load_library().cmbws_model_set_vcycle(model.handle, int(kind)))


def cmbws_model_merge_precond(model, group, stream=None):
    """Merge bands in the preconditioner (App. A.3): group[nu] = merged row of band nu
    (ids 0..G-1, bands of a row on one grid), or None for one row per band."""
    lib = load_library()
    if group is None:
        gp = ctypes.POINTER(ctypes.c_int)()
    else:
        if len(group) != model.nobs:
            raise ValueError(f"group needs {model.nobs} entries")
        gp = (ctypes.c_int * model.nobs)(*[int(g) for g in group])
    _check(lib.cmbws_model_merge_precond(model.handle, gp, _stream(stream)))
    nvec = ctypes.c_int64()
    na = ctypes.c_int()
    nm = ctypes.c_int()
    _check(lib.cmbws_model_info(model.handle, ctypes.byref(nvec), ctypes.byref(na), ctypes.byref(nm)))
    model.nsht_M = nm.value


CMBWS_DRAW_NORMAL = 0
CMBWS_DRAW_UNIFORM = 1


def cmbws_draw(seed, sample, stream_id, offset, out, kind=CMBWS_DRAW_NORMAL, stream=None):
    """out[t] = variate offset + t of the counter-based stream (seed, sample, stream_id);
    out: CUDA float64 tensor (its length is n)."""
    n = int(out.numel())
    _check(load_library().cmbws_draw(int(seed), int(sample), int(stream_id), int(offset), n,
                                     int(kind), _dptr(out, n, "out") if n else ctypes.c_void_p(),
                                     _stream(stream)))


def _band_ptrs(model, d, name):
    nobs = len(model.grids)
    return (ctypes.c_void_p * nobs)(*[_dptr(d[nu], model.grids[nu].npix, f"{name}[{nu}]").value
                                      for nu in range(nobs)])


def cmbws_cr_rhs(model, d, seed, sample, b, stream=None):
    """b of constrained realization `sample` with omega_1, omega_2 drawn on the device."""
    _check(load_library().cmbws_cr_rhs(model.handle, _band_ptrs(model, d, "d"), int(seed),
                                       int(sample), _dptr(b, model.nvec, "b"), _stream(stream)))


def cmbws_cr_sample(model, d, seed, sample, x, tol=1e-6, maxiter=1000, precond=1, inner_tol=1e-3,
                    max_outer=20, timeout_s=0.0, cert_prec=CMBWS_FP64, stream=None, check=True):
    """Draw constrained realization `sample` into x (x holds the initial guess)."""
    opts = CgOpts(float(tol), int(maxiter), int(precond), float(inner_tol), int(max_outer),
                  float(timeout_s), int(cert_prec))
    rep = CgReport()
    code = load_library().cmbws_cr_sample(model.handle, _band_ptrs(model, d, "d"), int(seed),
                                          int(sample), _dptr(x, model.nvec, "x"),
                                          ctypes.byref(opts), ctypes.byref(rep), _stream(stream))
    if check:
        _check(code)
    out = rep.as_dict()
    out["code"] = code
    return out


def cmbws_powerlaw_mixing(nu_ratio, beta, q, mask=None, stream=None):
    """q = mask (nu / nu_0)^beta on the device (beta, mask, q: CUDA float64 of equal length)."""
    n = int(q.numel())
    mp = _dptr(mask, n, "mask") if mask is not None else ctypes.c_void_p()
    _check(load_library().cmbws_powerlaw_mixing(float(nu_ratio), _dptr(beta, n, "beta"), mp, n,
                                                _dptr(q, n, "q"), _stream(stream)))


def cmbws_grad_terms(model, x, lam, d, out, omega1=None, omega2=None, stream=None):
    """out[nu * ncomp + k] = dL/dq_{nu,k}, out[nobs * ncomp + k] = dL/dt_k given the solution x
    and the adjoint solution lam (A lam = dL/dx); out: CUDA float64 of nobs * ncomp + ncomp."""
    nobs, ncomp = model.nobs, len(model.lmax_comp)
    dp = (ctypes.c_void_p * nobs)(*[_dptr(d[nu], model.grids[nu].npix, f"d[{nu}]").value
                                    for nu in range(nobs)])
    if omega1 is not None:
        w1 = (ctypes.c_void_p * nobs)(*[_dptr(omega1[nu], model.grids[nu].npix, f"omega1[{nu}]").value
                                        for nu in range(nobs)])
    else:
        w1 = ctypes.POINTER(ctypes.c_void_p)()
    w2 = _dptr(omega2, model.nvec, "omega2") if omega2 is not None else ctypes.c_void_p()
    _check(load_library().cmbws_grad_terms(model.handle, _dptr(x, model.nvec, "x"),
                                           _dptr(lam, model.nvec, "lam"), dp, w1, w2,
                                           _dptr(out, nobs * ncomp + ncomp, "out"), _stream(stream)))


def cmbws_grad_mix_maps(model, x, lam, d, out, omega1=None, stream=None):
    """out[nu][k] (CUDA float64 of the mixing grid's npix, or None) <- dL/dq_{nu,k}(p) of every
    variable pair, given the solution x and the adjoint solution lam (A lam = dL/dx)."""
    nobs, ncomp = model.nobs, len(model.lmax_comp)
    mg = getattr(model, "mix_grids", None)
    dp = (ctypes.c_void_p * nobs)(*[_dptr(d[nu], model.grids[nu].npix, f"d[{nu}]").value
                                    for nu in range(nobs)])
    if omega1 is not None:
        w1 = (ctypes.c_void_p * nobs)(*[_dptr(omega1[nu], model.grids[nu].npix, f"omega1[{nu}]").value
                                        for nu in range(nobs)])
    else:
        w1 = ctypes.POINTER(ctypes.c_void_p)()
    op = (ctypes.c_void_p * (nobs * ncomp))()
    for nu in range(nobs):
        for k in range(ncomp):
            t = out[nu][k]
            if t is None:
                continue
            if mg is None or mg[nu][k] is None:
                raise ValueError(f"out[{nu}][{k}]: pair ({nu}, {k}) has scalar mixing")
            op[nu * ncomp + k] = _dptr(t, mg[nu][k].npix, f"out[{nu}][{k}]").value
    _check(load_library().cmbws_grad_mix_maps(model.handle, _dptr(x, model.nvec, "x"),
                                              _dptr(lam, model.nvec, "lam"), dp, w1, op,
                                              _stream(stream)))


def cmbws_model_add_mask_precond(model, comp, nside, mask, max_bottom=400, stream=None):
    """Attach the mask-restricted multigrid preconditioner of component `comp` (HEALPix mask map
    of 12 nside^2 CUDA float64, nonzero inside the mask); solves with precond=2 use M_PI + M_mask."""
    _check(load_library().cmbws_model_add_mask_precond(
        model.handle, int(comp), int(nside), _dptr(mask, 12 * nside * nside, "mask"),
        int(max_bottom), _stream(stream)))


def cmbws_apply_M_add(model, r, z, stream=None):
    """z = M_PI r + the mask preconditioners' M_mask r."""
    _check(load_library().cmbws_apply_M_add(model.handle, _dptr(r, model.nvec, "r"),
                                            _dptr(z, model.nvec, "z"), _stream(stream)))


def cmbws_apply_M_diag(model, r, z, stream=None):
    """z = M_diag r (block-diagonal comparison preconditioner)."""
    _check(load_library().cmbws_apply_M_diag(model.handle, _dptr(r, model.nvec, "r"),
                                             _dptr(z, model.nvec, "z"), _stream(stream)))


def cmbws_project(model, x, d, stream=None):
    """d[nu] = P_nu x for every band (d: list of CUDA float64 maps, written)."""
    nobs = len(model.grids)
    dp = (ctypes.c_void_p * nobs)(*[_dptr(d[nu], model.grids[nu].npix, f"d[{nu}]").value
                                    for nu in range(nobs)])
    _check(load_library().cmbws_project(model.handle, _dptr(x, model.nvec, "x"), dp, _stream(stream)))


PROFILE_STAGES = ("legendre_synth", "legendre_adjoint", "adjoint_reduce", "ring_fft", "harmonic",
                  "cg_vector")


def cmbws_device_status(stream=None):
    """Synchronise the stream and raise CmbwsError (CMBWS_ERR_TIMEOUT) if a bounded
    device-side wait of a library kernel ran out since the last check."""
    _check(load_library().cmbws_device_status(_stream(stream)))


def cmbws_testing_stall_waits(wait_cycles):
    """Test support: make the tensor-core synthesis CTAs wait up to wait_cycles SM clocks on an
    mbarrier phase that never completes (0 switches it off)."""
    _check(load_library().cmbws_testing_stall_waits(int(wait_cycles)))


def cmbws_profile_enable(on=True):
    _check(load_library().cmbws_profile_enable(1 if on else 0))


PROFILE_ARITH = ("fp32", "fp64", "fp32x2", "tf32", "3xtf32", "bf16", "bf16x3")


def cmbws_profile_read(reset=True):
    """{(stage, arith): (milliseconds, launches, algorithmic flops, elements, elements x maps,
    algorithmic bytes)} since the last reset; arith in PROFILE_ARITH."""
    ns, na = len(PROFILE_STAGES), len(PROFILE_ARITH)
    arrs = [(ctypes.c_double * (na * ns))() for _ in range(5)]
    n = (ctypes.c_int64 * (na * ns))()
    ms, fl, el, me, by = arrs
    _check(load_library().cmbws_profile_read(ms, n, fl, el, me, by, 1 if reset else 0))
    out = {}
    for i in range(na * ns):
        out[(PROFILE_STAGES[i % ns], PROFILE_ARITH[i // ns])] = (ms[i], n[i], fl[i], el[i], me[i],
                                                                 by[i])
    return out


def cmbws_cg_solve(model, b, x, tol=1e-6, maxiter=1000, precond=1, inner_tol=1e-3, max_outer=20,
                   timeout_s=0.0, cert_prec=CMBWS_FP64, stream=None, check=True):
    """Solve A x = b in place (x holds the initial guess). Returns the report as a dict."""
    opts = CgOpts(float(tol), int(maxiter), int(precond), float(inner_tol), int(max_outer),
                  float(timeout_s), int(cert_prec))
    rep = CgReport()
    code = load_library().cmbws_cg_solve(model.handle, _dptr(b, model.nvec, "b"),
                                         _dptr(x, model.nvec, "x"), ctypes.byref(opts),
                                         ctypes.byref(rep), _stream(stream))
    if check:
        _check(code)
    out = rep.as_dict()
    out["code"] = code
    return out


def cmbws_model_set_precond_prec(model, prec=-1):
    """Arithmetic of M_PI's transforms inside the solvers (-1: the model's own)."""
    _check(load_library().cmbws_model_set_precond_prec(model.handle, int(prec)))


def cmbws_cg_history(model):
    """(rel_res, rel_err) per CG iteration of the model's last solve (rel_err -1 when no
    reference solution is tracked)."""
    n = ctypes.c_int()
    _check(load_library().cmbws_cg_history(model.handle, None, None, 0, ctypes.byref(n)))
    res = (ctypes.c_double * max(n.value, 1))()
    err = (ctypes.c_double * max(n.value, 1))()
    _check(load_library().cmbws_cg_history(model.handle, res, err, n.value, ctypes.byref(n)))
    return np.array(res[:n.value]), np.array(err[:n.value])


def cmbws_cg_track_error(model, x_true=None, stream=None):
    ptr = None if x_true is None else _dptr(x_true, model.nvec, "x_true")
    _check(load_library().cmbws_cg_track_error(model.handle, ptr, _stream(stream)))


def cmbws_cg_checkpointing(model, on=True):
    _check(load_library().cmbws_cg_checkpointing(model.handle, 1 if on else 0))


def cmbws_cg_state_export(model, d, r, p, stream=None):
    """Copy the checkpointed PCG state into d, r, p (device vectors); returns the scalars
    [iterations, r.z, r.r]."""
    sc = (ctypes.c_double * 3)()
    _check(load_library().cmbws_cg_state_export(model.handle, _dptr(d, model.nvec, "d"),
                                                _dptr(r, model.nvec, "r"),
                                                _dptr(p, model.nvec, "p"), sc, _stream(stream)))
    return [sc[0], sc[1], sc[2]]


def cmbws_cg_resume(model, b, x, d, r, p, scalars, tol=1e-6, maxiter=1000, precond=1,
                    inner_tol=1e-3, max_outer=20, timeout_s=0.0, cert_prec=CMBWS_FP64, stream=None,
                    check=True):
    """Continue an exported PCG state (x: the interrupted solve's initial guess; overwritten with
    the solution).  Returns the report as a dict."""
    opts = CgOpts(float(tol), int(maxiter), int(precond), float(inner_tol), int(max_outer),
                  float(timeout_s), int(cert_prec))
    rep = CgReport()
    sc = (ctypes.c_double * 3)(*[float(v) for v in scalars])
    code = load_library().cmbws_cg_resume(model.handle, _dptr(b, model.nvec, "b"),
                                          _dptr(x, model.nvec, "x"), _dptr(d, model.nvec, "d"),
                                          _dptr(r, model.nvec, "r"), _dptr(p, model.nvec, "p"), sc,
                                          ctypes.byref(opts), ctypes.byref(rep), _stream(stream))
    if check:
        _check(code)
    out = rep.as_dict()
    out["code"] = code
    return out


def cmbws_model_set_shard(model, owned, prior=1):
    """owned: [nobs] 0 / 1 flags (None drops the shard); prior: 1 if this shard adds the prior."""
    if owned is None:
        _check(load_library().cmbws_model_set_shard(model.handle, None, int(prior)))
        return
    arr = (ctypes.c_int * model.nobs)(*[int(v) for v in owned])
    _check(load_library().cmbws_model_set_shard(model.handle, arr, int(prior)))


def cmbws_cg_solve_sharded(model, b, x, allreduce, tol=1e-6, maxiter=1000, precond=1,
                           inner_tol=1e-3, max_outer=20, timeout_s=0.0, cert_prec=CMBWS_FP64,
                           stream=None, check=True):
    """PCG over a band-sharded operator; allreduce: a ctypes callback (sharding.make_allreduce)."""
    opts = CgOpts(float(tol), int(maxiter), int(precond), float(inner_tol), int(max_outer),
                  float(timeout_s), int(cert_prec))
    rep = CgReport()
    fn = ctypes.cast(allreduce, ctypes.c_void_p)
    code = load_library().cmbws_cg_solve_sharded(model.handle, _dptr(b, model.nvec, "b"),
                                                 _dptr(x, model.nvec, "x"), ctypes.byref(opts), fn,
                                                 None, ctypes.byref(rep), _stream(stream))
    if check:
        _check(code)
    out = rep.as_dict()
    out["code"] = code
    return out


def cmbws_cg_solve_batched(models, b, x, tol=1e-6, maxiter=1000, precond=1, inner_tol=1e-3,
                           max_outer=20, timeout_s=0.0, cert_prec=CMBWS_FP64, nworkers=8,
                           stream=None, check=True):
    """Solve the independent systems models[i] x[i] = b[i] concurrently; returns the reports."""
    n = len(models)
    opts = CgOpts(float(tol), int(maxiter), int(precond), float(inner_tol), int(max_outer),
                  float(timeout_s), int(cert_prec))
    reps = (CgReport * n)()
    mh = (ctypes.c_void_p * n)(*[_handle(m) for m in models])
    bp = (ctypes.c_void_p * n)(*[_dptr(b[i], models[i].nvec, f"b[{i}]").value for i in range(n)])
    xp = (ctypes.c_void_p * n)(*[_dptr(x[i], models[i].nvec, f"x[{i}]").value for i in range(n)])
    code = load_library().cmbws_cg_solve_batched(mh, n, bp, xp, ctypes.byref(opts), reps,
                                                 int(nworkers), _stream(stream))
    if check:
        _check(code)
    out = [r.as_dict() for r in reps]
    for r in out:
        r["code"] = r["status"]
    return out
