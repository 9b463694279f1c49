"""Python binding of the C ABI in ``include/blast.h`` (ctypes, marshalling only).

Every function named ``blast_*`` here forwards to the C entry point of the same
name; every step of the computation runs in the library's CUDA kernels.  The
library is built in-tree (``paper_2410_03632_gb300/_lib/libblast.so``); if it
cannot be loaded, importing this module's functions raises instead of falling
back to anything else.

``Plan`` is a thin convenience wrapper that owns a ``blast_plan*`` and turns
numpy arrays or torch tensors into ``blast_request`` structs.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

BLAST_OK, BLAST_EINVAL, BLAST_ENOMEM, BLAST_ENOTREADY = 0, -1, -2, -3
BLAST_ETIMEOUT, BLAST_EDEVICE, BLAST_ENOBASIS, BLAST_EBUSY = -4, -5, -6, -7
BLAST_FP64, BLAST_FP32, BLAST_BF16S = 0, 1, 2
BLAST_BASIS_FP64, BLAST_BASIS_FP32, BLAST_BASIS_BF16S = 1, 2, 4
BASIS_ALL = BLAST_BASIS_FP64 | BLAST_BASIS_FP32 | BLAST_BASIS_BF16S

_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class blast_plan_desc(ctypes.Structure):
    _fields_ = [("n_ell", ctypes.c_int), ("ell", ctypes.POINTER(ctypes.c_int32)),
                ("n_chi", ctypes.c_int), ("chi_min", ctypes.c_double), ("chi_max", ctypes.c_double),
                ("n_R", ctypes.c_int), ("R_min", ctypes.c_double), ("R_max", ctypes.c_double),
                ("n_cheb", ctypes.c_int), ("k_min", ctypes.c_double), ("k_max", ctypes.c_double),
                ("k_map", ctypes.c_int), ("n_kquad", ctypes.c_int),
                ("max_clust", ctypes.c_int), ("max_lens", ctypes.c_int), ("device", ctypes.c_int),
                ("r_form", ctypes.c_int), ("ell_real", ctypes.POINTER(ctypes.c_double))]


class blast_request(ctypes.Structure):
    _fields_ = [("n_clust", ctypes.c_int), ("n_lens", ctypes.c_int),
                ("kern_chi", _vp), ("kern_Rchi", _vp), ("growth_chi", _vp), ("growth_Rchi", _vp),
                ("n_ptab", ctypes.c_int), ("k_tab", _vp), ("p_tab", _vp),
                ("ell_mask_lo", ctypes.c_uint64), ("ell_mask_hi", ctypes.c_uint64),
                ("mem_space", ctypes.c_int)]


class BlastError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: {lib().blast_status_str(status).decode()} ({status})")
        self.status = status


_LIB = None
_LOCK = threading.Lock()


def lib():
    """Load (building first if stale) the in-tree CUDA library."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.SO
            if not os.path.exists(path) or not _build.up_to_date():
                path = _build.build()
            L = ctypes.CDLL(path)
            i, d, sz = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
            P = _vp
            L.blast_plan_create.argtypes = [ctypes.POINTER(blast_plan_desc), ctypes.POINTER(P)]
            L.blast_plan_destroy.argtypes = [P]
            L.blast_plan_nodes.argtypes = [P, _dp, _dp, _dp]
            L.blast_npairs.argtypes = [i, i]
            L.blast_precompute_basis.argtypes = [P, ctypes.c_uint, P]
            L.blast_basis_get.argtypes = [P, P, i, P]
            L.blast_basis_set.argtypes = [P, P, i, ctypes.c_uint, P]
            L.blast_basis_save.argtypes = [P, ctypes.c_char_p]
            L.blast_basis_load.argtypes = [P, ctypes.c_char_p, ctypes.c_uint]
            L.blast_cl.argtypes = [P, ctypes.POINTER(blast_request), i, P, i, P]
            L.blast_cl_batch.argtypes = [P, i, ctypes.POINTER(blast_request), i, ctypes.POINTER(P), i, P]
            L.blast_request_footprint.argtypes = [P, ctypes.POINTER(blast_request)]
            L.blast_request_footprint.restype = sz
            L.blast_status_str.argtypes = [i]
            L.blast_status_str.restype = ctypes.c_char_p
            L.blast_cl_noalloc.argtypes = [P, ctypes.POINTER(blast_request), P, P]
            L.blast_set_coef_envelope.argtypes = [P, P]
            L.blast_limber_k.argtypes = [P, _dp]
            L.blast_autotune.argtypes = [P, i, ctypes.POINTER(blast_request), ctypes.c_char_p, P]
            L.blast_tuned_params.argtypes = [P, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
            L.blast_cl_nonsep.argtypes = [P, ctypes.POINTER(blast_request), P, P, i, P]
            L.blast_test_trip_wait.argtypes = [P, i]
            L.blast_cl_limber.argtypes = [P, ctypes.POINTER(blast_request), P, i, P, i, P]
            L.blast_cl_nonlinear.argtypes = [P, ctypes.POINTER(blast_request), i, P, P, i, P]
            L.blast_profile_enable.argtypes = [P, i]
            L.blast_profile_read.argtypes = [P, i, _dp, ctypes.POINTER(ctypes.c_longlong)]
            L.blast_profile_reset.argtypes = [P]
            L.blast_server_create.argtypes = [ctypes.POINTER(P), i, sz, i, ctypes.POINTER(P)]
            L.blast_submit.argtypes = [P, i, ctypes.POINTER(blast_request), i, ctypes.POINTER(ctypes.c_uint64)]
            L.blast_poll.argtypes = [P, ctypes.c_uint64, P, ctypes.POINTER(i), ctypes.c_int64]
            L.blast_server_destroy.argtypes = [P]
            L.blast_server_reserved.argtypes = [P]
            L.blast_server_reserved.restype = sz
            L.blast_graph_create.argtypes = [P, i, ctypes.POINTER(blast_request), i, ctypes.POINTER(P),
                                             ctypes.POINTER(P)]
            L.blast_graph_launch.argtypes = [P, P]
            L.blast_graph_reserved.argtypes = [P]
            L.blast_graph_reserved.restype = sz
            L.blast_graph_destroy.argtypes = [P]
            _LIB = L
    return _LIB


def _check(rc, what):
    if rc != BLAST_OK:
        raise BlastError(rc, what)


# ---------------------------------------------------------------------------- C names
def blast_plan_create(desc: blast_plan_desc):
    h = _vp()
    _check(lib().blast_plan_create(ctypes.byref(desc), ctypes.byref(h)), "blast_plan_create")
    return h


def blast_plan_destroy(h):
    return lib().blast_plan_destroy(h)


def blast_npairs(ng, ns):
    return lib().blast_npairs(ng, ns)


def blast_precompute_basis(h, mask, stream=None):
    _check(lib().blast_precompute_basis(h, mask, stream), "blast_precompute_basis")


def blast_basis_save(h, path):
    _check(lib().blast_basis_save(h, path.encode()), "blast_basis_save")


def blast_basis_load(h, path, mask):
    _check(lib().blast_basis_load(h, path.encode(), mask), "blast_basis_load")


def blast_cl(h, req, precision, out_ptr, out_mem_space, stream=None):
    return lib().blast_cl(h, ctypes.byref(req), precision, out_ptr, out_mem_space, stream)


def blast_cl_batch(h, reqs, precision, out_ptrs, out_mem_space, stream=None):
    n = len(reqs)
    arr = (blast_request * n)(*reqs)
    outs = (_vp * n)(*out_ptrs)
    return lib().blast_cl_batch(h, n, arr, precision, outs, out_mem_space, stream)


def blast_cl_noalloc(h, req, out_ptr, stream=None):
    """FP64 C_l of one cosmology without any device allocation (device inputs
    and output); scratch comes from a fixed array inside the library."""
    return lib().blast_cl_noalloc(h, ctypes.byref(req), out_ptr, stream)


def blast_test_trip_wait(h, tile):
    return lib().blast_test_trip_wait(h, tile)


def blast_cl_nonsep(h, req, p_nodes_ptr, out_ptr, out_mem_space, stream=None):
    return lib().blast_cl_nonsep(h, ctypes.byref(req), p_nodes_ptr, out_ptr, out_mem_space, stream)


def blast_autotune(h, reqs, cache_path=None, stream=None):
    arr = (blast_request * len(reqs))(*reqs)
    path = None if cache_path is None else str(cache_path).encode()
    return lib().blast_autotune(h, len(reqs), arr, path, stream)


def blast_tuned_params(h):
    g, w, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().blast_tuned_params(h, ctypes.byref(g), ctypes.byref(w), ctypes.byref(n)), "blast_tuned_params")
    return g.value, w.value, n.value


def blast_limber_k(h, L, X):
    k = np.empty((L, X))
    _check(lib().blast_limber_k(h, k.ctypes.data_as(_dp)), "blast_limber_k")
    return k


def blast_cl_limber(h, req, p_nl_ptr, extended, out_ptr, out_mem_space, stream=None):
    return lib().blast_cl_limber(h, ctypes.byref(req), p_nl_ptr, extended, out_ptr, out_mem_space, stream)


def blast_cl_nonlinear(h, req, precision, p_nl_ptr, out_ptr, out_mem_space, stream=None):
    return lib().blast_cl_nonlinear(h, ctypes.byref(req), precision, p_nl_ptr, out_ptr, out_mem_space, stream)


def blast_set_coef_envelope(h, env=None):
    """env: numpy float64 array of n_cheb positive values, or None for the default."""
    if env is None:
        return lib().blast_set_coef_envelope(h, None)
    env = np.ascontiguousarray(env, dtype=np.float64)
    return lib().blast_set_coef_envelope(h, env.ctypes.data)


def blast_request_footprint(h, req):
    return lib().blast_request_footprint(h, ctypes.byref(req))


def blast_status_str(rc):
    return lib().blast_status_str(rc).decode()


BLAST_K_FIT, BLAST_K_WEIGHTS, BLAST_K_CONTRACT, BLAST_K_CONTRACT_TC, BLAST_K_REDUCE = 0, 1, 2, 3, 4
KERNEL_CLASS_NAMES = ["fit", "weights", "contract", "contract_tc", "reduce"]


def blast_server_create(plan_handles, hbm_budget, max_slots):
    arr = (_vp * len(plan_handles))(*plan_handles)
    h = _vp()
    _check(lib().blast_server_create(arr, len(plan_handles), hbm_budget, max_slots, ctypes.byref(h)),
           "blast_server_create")
    return h


def blast_submit(h, plan_idx, req, precision):
    """(status, ticket)."""
    t = ctypes.c_uint64()
    rc = lib().blast_submit(h, plan_idx, ctypes.byref(req), precision, ctypes.byref(t))
    return rc, t.value


def blast_poll(h, ticket, out_ptr, timeout_us=-1):
    """(status, done)."""
    d = ctypes.c_int()
    rc = lib().blast_poll(h, ticket, out_ptr, ctypes.byref(d), timeout_us)
    return rc, d.value


def blast_server_destroy(h):
    return lib().blast_server_destroy(h)


def blast_graph_create(h, reqs, precision, out_ptrs):
    """Handle of a captured batch (device inputs and outputs)."""
    n = len(reqs)
    arr = (blast_request * n)(*reqs)
    outs = (_vp * n)(*out_ptrs)
    g = _vp()
    _check(lib().blast_graph_create(h, n, arr, precision, outs, ctypes.byref(g)), "blast_graph_create")
    return g


def blast_graph_launch(g, stream=None):
    return lib().blast_graph_launch(g, stream)


def blast_graph_reserved(g):
    return lib().blast_graph_reserved(g)


def blast_graph_destroy(g):
    return lib().blast_graph_destroy(g)


def blast_server_reserved(h):
    """Device bytes the server reserved at creation."""
    return lib().blast_server_reserved(h)


def blast_profile_enable(h, enable):
    _check(lib().blast_profile_enable(h, int(enable)), "blast_profile_enable")


def blast_profile_read(h, cls):
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(lib().blast_profile_read(h, cls, ctypes.byref(ms), ctypes.byref(n)), "blast_profile_read")
    return ms.value, n.value


def blast_profile_reset(h):
    _check(lib().blast_profile_reset(h), "blast_profile_reset")


# ---------------------------------------------------------------------------- helpers
def _ptr(a):
    """Address of a contiguous float64 numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    assert a.flags["C_CONTIGUOUS"] and a.dtype == np.float64
    return a.ctypes.data


def ell_mask(sel, L):
    """(lo, hi) bitmask words for plan ell indices ``sel`` (None = all)."""
    if sel is None:
        return 0, 0
    lo = hi = 0
    for e in sel:
        assert 0 <= e < L
        if e < 64:
            lo |= 1 << int(e)
        else:
            hi |= 1 << int(e - 64)
    return lo, hi


class Plan:
    """Owns one ``blast_plan``.  ``spec`` is any object with the fields of
    ``blast_plan_desc`` (e.g. ``synth.PlanSpec``)."""

    def __init__(self, spec, device: int = 0):
        self.spec = spec
        self.device = device
        ells = np.asarray(spec.ells)
        self._ellr = np.ascontiguousarray(ells, dtype=np.float64)
        self._ell = np.ascontiguousarray(np.floor(self._ellr), dtype=np.int32)
        d = blast_plan_desc()
        d.n_ell = self._ell.size
        d.ell = self._ell.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        if np.any(self._ellr != np.floor(self._ellr)):  # non-integer multipoles
            d.ell_real = self._ellr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.n_chi, d.chi_min, d.chi_max = spec.n_chi, spec.chi_min, spec.chi_max
        d.n_R, d.R_min, d.R_max = spec.n_R, spec.R_min, spec.R_max
        d.n_cheb, d.k_min, d.k_max, d.k_map = spec.n_cheb, spec.k_min, spec.k_max, spec.k_map
        d.n_kquad, d.max_clust, d.max_lens, d.device = spec.n_kquad, spec.max_clust, spec.max_lens, device
        d.r_form = int(getattr(spec, "r_form", 0))
        self.h = blast_plan_create(d)
        self.L, self.X, self.Rn, self.N = d.n_ell, d.n_chi, d.n_R, d.n_cheb
        self.Q = self.X * self.Rn

    def close(self):
        if self.h:
            blast_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nodes(self):
        chi, R, kc = np.empty(self.X), np.empty(self.Rn), np.empty(self.N)
        _check(lib().blast_plan_nodes(self.h, chi.ctypes.data_as(_dp), R.ctypes.data_as(_dp),
                                      kc.ctypes.data_as(_dp)), "blast_plan_nodes")
        return chi, R, kc

    def precompute(self, mask=BASIS_ALL, stream=None):
        blast_precompute_basis(self.h, mask, stream)

    def basis(self):
        out = np.empty((3, self.L, self.N, self.Q))
        _check(lib().blast_basis_get(self.h, out.ctypes.data, 0, None), "blast_basis_get")
        return out

    def set_basis(self, T, mask=BASIS_ALL):
        T = np.ascontiguousarray(T, dtype=np.float64)
        assert T.shape == (3, self.L, self.N, self.Q)
        _check(lib().blast_basis_set(self.h, T.ctypes.data, 0, mask, None), "blast_basis_set")

    def request(self, rq, ell_sel=None, device_arrays=None):
        """blast_request for a synth.Request; ``device_arrays`` (a dict of
        device tensors with the same field names) switches to mem_space 1."""
        src = device_arrays if device_arrays is not None else rq.__dict__
        r = blast_request()
        r.n_clust, r.n_lens = rq.n_clust, rq.n_lens
        r.kern_chi, r.kern_Rchi = _ptr(src["kern_chi"]), _ptr(src["kern_Rchi"])
        r.growth_chi, r.growth_Rchi = _ptr(src["growth_chi"]), _ptr(src["growth_Rchi"])
        r.n_ptab = int(rq.k_tab.size)
        r.k_tab, r.p_tab = _ptr(src["k_tab"]), _ptr(src["p_tab"])
        r.ell_mask_lo, r.ell_mask_hi = ell_mask(ell_sel, self.L)
        r.mem_space = 1 if device_arrays is not None else 0
        r._keep = src  # keep arrays alive with the struct
        return r

    def n_sel(self, ell_sel):
        return self.L if ell_sel is None else len(ell_sel)

    def cl(self, rq, precision=BLAST_FP64, ell_sel=None):
        """C[pair][ell] on the host for one synth.Request (host inputs)."""
        r = self.request(rq, ell_sel)
        out = np.empty((blast_npairs(rq.n_clust, rq.n_lens), self.n_sel(ell_sel)))
        _check(blast_cl(self.h, r, precision, out.ctypes.data, 0), "blast_cl")
        return out

    def limber(self, rq, p_nl=None, extended=False, ell_sel=None):
        """C^Limber (host arrays): the request's linear P, or p_nl[n_ell][n_chi]."""
        r = self.request(rq, ell_sel)
        out = np.empty((blast_npairs(rq.n_clust, rq.n_lens), self.n_sel(ell_sel)))
        pn = None if p_nl is None else np.ascontiguousarray(p_nl, dtype=np.float64)
        _check(blast_cl_limber(self.h, r, None if pn is None else pn.ctypes.data, int(bool(extended)),
                               out.ctypes.data, 0), "blast_cl_limber")
        return out

    def nonsep(self, rq, p_nodes, ell_sel=None):
        """Beyond-Limber C_l of a non-separable P sampled at the Chebyshev k-nodes of
        every chi-R node, p_nodes[n_chi * n_R][n_cheb] (host arrays)."""
        r = self.request(rq, ell_sel)
        out = np.empty((blast_npairs(rq.n_clust, rq.n_lens), self.n_sel(ell_sel)))
        pn = np.ascontiguousarray(p_nodes, dtype=np.float64)
        assert pn.shape == (self.Q, self.N)
        _check(blast_cl_nonsep(self.h, r, pn.ctypes.data, out.ctypes.data, 0), "blast_cl_nonsep")
        return out

    def nonlinear(self, rq, p_nl, precision=BLAST_FP64, ell_sel=None):
        """C_tot = C_lin + C^Limber(P_delta) - C^Limber(P_lin) (host arrays)."""
        r = self.request(rq, ell_sel)
        out = np.empty((blast_npairs(rq.n_clust, rq.n_lens), self.n_sel(ell_sel)))
        pn = np.ascontiguousarray(p_nl, dtype=np.float64)
        _check(blast_cl_nonlinear(self.h, r, precision, pn.ctypes.data, out.ctypes.data, 0), "blast_cl_nonlinear")
        return out

    def cl_batch(self, rqs, precision=BLAST_FP64, ell_sels=None):
        ell_sels = ell_sels or [None] * len(rqs)
        reqs = [self.request(rq, s) for rq, s in zip(rqs, ell_sels)]
        outs = [np.empty((blast_npairs(rq.n_clust, rq.n_lens), self.n_sel(s))) for rq, s in zip(rqs, ell_sels)]
        _check(blast_cl_batch(self.h, reqs, precision, [o.ctypes.data for o in outs], 0), "blast_cl_batch")
        return outs


class Server:
    """Owns one ``blast_server`` over ``plans`` (``Plan`` objects that must
    outlive it and are not used elsewhere meanwhile)."""

    def __init__(self, plans, hbm_budget=8 << 30, max_slots=256):
        self.plans = list(plans)
        self.h = blast_server_create([p.h for p in self.plans], hbm_budget, max_slots)

    def submit(self, plan_idx, rq, precision=BLAST_FP64, ell_sel=None):
        """(status, ticket) for a synth.Request; inputs are copied before it returns."""
        r = self.plans[plan_idx].request(rq, ell_sel)
        return blast_submit(self.h, plan_idx, r, precision)

    def reserved(self):
        return blast_server_reserved(self.h)

    def poll(self, ticket, shape, timeout_us=-1):
        """(status, C or None)."""
        out = np.empty(shape)
        rc, done = blast_poll(self.h, ticket, out.ctypes.data, timeout_us)
        return rc, (out if done and rc == BLAST_OK else None)

    def close(self):
        if self.h:
            blast_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
