"""Python binding of the C ABI declared in include/gw.h (ctypes).

Argument marshalling only: every step of the GW path runs in the CUDA
library. Device arrays are torch tensors (complex128, contiguous, on the
context's device); their data pointers are passed straight through. The
library must have been built (``python -m paper_2406_18479_gb300.build``);
loading raises if it is missing, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libgw_gb300.so")

GW_OK, GW_EINVAL, GW_ENOMEM, GW_ECUDA, GW_ETIMEOUT, GW_EDEVTIMEOUT = 0, 1, 2, 3, 4, 5
GW_ENOTFINITE, GW_ENOTCONV, GW_EAGAIN, GW_ENOTIMPL = 6, 7, 8, 9
GW_FP64, GW_MIXED_BF16X4 = 0, 1
GW_MIXED_BF16X3 = GW_MIXED_BF16X4          # former name (the scheme has four slices)
GW_V_AUTO, GW_V_ALL_PAIRS, GW_V_PER_Q = 0, 1, 2
PRECISIONS = {"fp64": GW_FP64, "bf16x4": GW_MIXED_BF16X4, "bf16x3": GW_MIXED_BF16X4}

# Every symbol declared in include/gw.h.
ABI_SYMBOLS = [
    "gw_version", "gw_last_error", "gw_sample_count", "gw_grid_build", "gw_create", "gw_destroy",
    "gw_workspace_bytes", "gw_set_grids", "gw_set_coulomb", "gw_polarization", "gw_to_matsubara", "gw_to_tau",
    "gw_aux_dyson", "gw_screened_interaction", "gw_self_energy", "gw_sigma_eval", "gw_sigma_eval_q", "gw_dyson_G",
    "gw_mix", "gw_synchronize", "gw_profile_enable", "gw_launch_count", "gw_profile_slots",
    "gw_profile_read", "gw_polarization_noalloc", "gw_job_bytes", "gw_server_create",
    "gw_server_destroy", "gw_submit", "gw_poll", "gw_batch_create", "gw_batch_destroy",
    "gw_batch_set_coulomb", "gw_batch_sigma_eval", "gw_batch_autotune", "gw_batch_tuned", "gw_batch_synchronize",
    "gw_density", "gw_sigma_inf", "gw_set_mu", "gw_particle_number", "gw_find_mu", "gw_diis_create",
    "gw_diis_destroy", "gw_diis_push", "gw_diis_extrapolate", "gw_scgw_bytes", "gw_scgw", "gw_diis_push_residual",
    "gw_commutator_residual", "gw_gf2_self_energy", "gw_gf2_exchange", "gw_k_interpolate", "gw_ir_grids", "gw_set_overlap", "gw_checkpoint_write", "gw_checkpoint_read", "gw_selftest_bounded_wait", "gw_check_guards", "gw_debug_mark_guard",
]
GW_BATCH_SERIAL, GW_BATCH_STREAMS, GW_BATCH_GRAPH, GW_BATCH_GROUPED, GW_BATCH_GROUPED_GRAPH = 0, 1, 2, 3, 4
BATCH_MODES = {"serial": GW_BATCH_SERIAL, "streams": GW_BATCH_STREAMS, "graph": GW_BATCH_GRAPH,
               "grouped": GW_BATCH_GROUPED, "grouped_graph": GW_BATCH_GROUPED_GRAPH}


class GWError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gw error {code}: {msg}")
        self.code = code


class gw_config(ctypes.Structure):
    _fields_ = [
        ("nk", ctypes.c_int * 3), ("nao", ctypes.c_int), ("naux", ctypes.c_int), ("ntau", ctypes.c_int),
        ("beta", ctypes.c_double), ("mu", ctypes.c_double), ("spin_factor", ctypes.c_double),
        ("precision", ctypes.c_int), ("tau_chunk", ctypes.c_int), ("v_slices", ctypes.c_int),
        ("v_packed", ctypes.c_int), ("slice_pass", ctypes.c_int), ("tile_n", ctypes.c_int),
    ]


class gw_job(ctypes.Structure):
    _fields_ = [
        ("cfg", gw_config), ("H_host", ctypes.c_void_p), ("V_host", ctypes.c_void_p),
        ("G0_host", ctypes.c_void_p), ("Sigma_out_host", ctypes.c_void_p), ("G_out_host", ctypes.c_void_p),
        ("alpha", ctypes.c_double), ("tol", ctypes.c_double), ("itermax", ctypes.c_int),
        ("static_part", ctypes.c_int), ("diis_size", ctypes.c_int), ("diis_start", ctypes.c_int),
        ("n_electrons", ctypes.c_double), ("mu_lo", ctypes.c_double), ("mu_hi", ctypes.c_double),
        ("mu_tol", ctypes.c_double), ("diis_kind", ctypes.c_int), ("method", ctypes.c_int),
        ("S_host", ctypes.c_void_p),
    ]


class gw_scgw_options(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double), ("tol", ctypes.c_double), ("itermax", ctypes.c_int),
        ("static_part", ctypes.c_int), ("diis_size", ctypes.c_int), ("diis_start", ctypes.c_int),
        ("n_electrons", ctypes.c_double), ("mu_lo", ctypes.c_double), ("mu_hi", ctypes.c_double),
        ("mu_tol", ctypes.c_double), ("diis_kind", ctypes.c_int), ("method", ctypes.c_int),
        ("resume", ctypes.c_int),
    ]


class gw_scgw_result(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("max_abs_dsigma", ctypes.c_double), ("mu", ctypes.c_double),
        ("n_electrons", ctypes.c_double),
    ]


class gw_job_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("iterations", ctypes.c_int), ("max_abs_dsigma", ctypes.c_double),
        ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_end", ctypes.c_double),
        ("mu", ctypes.c_double),
    ]


_lib = None


def lib():
    """The loaded library (loaded once). Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run python -m paper_2406_18479_gb300.build)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, ll, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
    L.gw_version.restype = ctypes.c_char_p
    L.gw_last_error.restype = ctypes.c_char_p
    L.gw_sample_count.argtypes = [i, i]
    L.gw_grid_build.argtypes = [i, d, i, vp, vp, vp, vp]
    L.gw_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(gw_config), vp]
    L.gw_destroy.argtypes = [vp]
    L.gw_workspace_bytes.argtypes = [vp]
    L.gw_workspace_bytes.restype = ctypes.c_size_t
    L.gw_set_coulomb.argtypes = [vp, vp]
    L.gw_set_grids.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.gw_polarization.argtypes = [vp, vp, vp]
    L.gw_to_matsubara.argtypes = [vp, i, vp, vp, i, ll]
    L.gw_to_tau.argtypes = [vp, i, vp, vp, i, ll]
    L.gw_aux_dyson.argtypes = [vp, vp, vp]
    L.gw_screened_interaction.argtypes = [vp, vp, vp]
    L.gw_self_energy.argtypes = [vp, vp, vp, vp]
    L.gw_sigma_eval.argtypes = [vp, vp, vp]
    L.gw_sigma_eval_q.argtypes = [vp, vp, vp, i, i, vp, vp]
    L.gw_dyson_G.argtypes = [vp, vp, vp, vp]
    L.gw_mix.argtypes = [vp, vp, vp, d, ctypes.POINTER(d)]
    L.gw_synchronize.argtypes = [vp]
    L.gw_polarization_noalloc.argtypes = [ctypes.POINTER(ctypes.c_int), i, i, i, d, vp, vp, vp, vp]
    L.gw_profile_enable.argtypes = [vp, i]
    L.gw_launch_count.argtypes = [vp]
    L.gw_launch_count.restype = ctypes.c_longlong
    L.gw_profile_read.argtypes = [vp, i, ctypes.c_char_p, i, ctypes.POINTER(ll), ctypes.POINTER(d),
                                  ctypes.POINTER(d), ctypes.POINTER(d)]
    L.gw_job_bytes.argtypes = [ctypes.POINTER(gw_config)]
    L.gw_job_bytes.restype = ctypes.c_size_t
    L.gw_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t, i]
    L.gw_server_destroy.argtypes = [vp]
    L.gw_submit.argtypes = [vp, ctypes.POINTER(gw_job), ctypes.POINTER(ctypes.c_uint64)]
    L.gw_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(gw_job_result), i]
    L.gw_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(gw_config), i, i, ctypes.c_size_t, vp]
    L.gw_batch_destroy.argtypes = [vp]
    L.gw_batch_set_coulomb.argtypes = [vp, ctypes.POINTER(vp)]
    L.gw_batch_sigma_eval.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i]
    L.gw_batch_autotune.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i)]
    L.gw_batch_tuned.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i)]
    L.gw_batch_synchronize.argtypes = [vp]
    L.gw_density.argtypes = [vp, vp, vp]
    L.gw_sigma_inf.argtypes = [vp, vp, vp]
    L.gw_set_mu.argtypes = [vp, d]
    L.gw_particle_number.argtypes = [vp, vp, ctypes.POINTER(d)]
    L.gw_find_mu.argtypes = [vp, vp, vp, d, d, d, d, vp, ctypes.POINTER(d)]
    L.gw_diis_create.argtypes = [ctypes.POINTER(vp), ctypes.c_longlong, ctypes.c_longlong, i, vp]
    L.gw_diis_push_residual.argtypes = [vp, vp, vp]
    L.gw_commutator_residual.argtypes = [vp, vp, vp, vp, vp, vp]
    L.gw_gf2_self_energy.argtypes = [vp, vp, vp]
    L.gw_gf2_exchange.argtypes = [vp, vp, vp]
    L.gw_set_overlap.argtypes = [vp, vp]
    L.gw_selftest_bounded_wait.argtypes = [d, ctypes.POINTER(i), vp]
    L.gw_check_guards.argtypes = [vp]
    L.gw_debug_mark_guard.argtypes = [vp, i]
    L.gw_checkpoint_write.argtypes = [ctypes.c_char_p, ctypes.POINTER(gw_config), d, i, i, vp, vp, vp]
    L.gw_checkpoint_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(gw_config), ctypes.POINTER(d),
                                     ctypes.POINTER(i), i, vp, vp, vp]
    L.gw_ir_grids.argtypes = [d, d, d, i, ctypes.POINTER(i), vp, vp, vp, vp, vp, vp, vp]
    L.gw_k_interpolate.argtypes = [ctypes.POINTER(i), vp, ctypes.c_longlong, i, ctypes.POINTER(d), vp, vp]
    L.gw_diis_destroy.argtypes = [vp]
    L.gw_diis_push.argtypes = [vp, vp, vp]
    L.gw_diis_extrapolate.argtypes = [vp, vp, ctypes.POINTER(d), ctypes.POINTER(i)]
    L.gw_scgw_bytes.argtypes = [ctypes.POINTER(gw_config), ctypes.POINTER(gw_scgw_options)]
    L.gw_scgw_bytes.restype = ctypes.c_size_t
    L.gw_scgw.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(gw_scgw_options), ctypes.POINTER(gw_scgw_result)]
    _lib = L
    return L


def _check(rc):
    if rc != GW_OK:
        raise GWError(rc, lib().gw_last_error().decode())


def gw_version() -> str:
    return lib().gw_version().decode()


def gw_sample_count(ntau: int, stat: int) -> int:
    return lib().gw_sample_count(ntau, stat)


def gw_grid_build(ntau: int, beta: float, stat: int):
    """(tau [ntau], idx [nw], F [nw][ntau], B [ntau][nw]) as numpy arrays (host)."""
    nw = gw_sample_count(ntau, stat)
    if nw < 0:
        raise GWError(GW_EINVAL, "bad grid size")
    tau = np.zeros(ntau)
    idx = np.zeros(nw, np.int64)
    F = np.zeros((nw, ntau), np.complex128)
    B = np.zeros((ntau, nw), np.complex128)
    _check(lib().gw_grid_build(ntau, float(beta), stat, tau.ctypes.data, idx.ctypes.data,
                               F.ctypes.data, B.ctypes.data))
    return tau, idx, F, B


def _ptr(t, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_cuda:
        raise GWError(GW_EINVAL, "expected a complex128 CUDA tensor")
    if not t.is_contiguous():
        raise GWError(GW_EINVAL, "expected a contiguous tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise GWError(GW_EINVAL, f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class gw_ctx:
    """Owner of one gw_ctx* (gw_create ... gw_destroy)."""

    def __init__(self, nk3, nao, naux, ntau, beta, mu=0.0, spin_factor=2.0, precision="fp64",
                 tau_chunk=0, v_slices=0, stream=None, v_packed=False, slice_pass=False, tile_n=0):
        import torch
        self.nk3 = tuple(int(x) for x in nk3)
        self.nk = int(np.prod(self.nk3))
        self.nao, self.naux, self.ntau = int(nao), int(naux), int(ntau)
        self.beta, self.mu = float(beta), float(mu)
        self.nwb = gw_sample_count(ntau, 0)
        self.nwf = gw_sample_count(ntau, 1)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.v_packed = int(v_packed)
        cfg = gw_config((ctypes.c_int * 3)(*self.nk3), self.nao, self.naux, self.ntau, self.beta,
                        self.mu, float(spin_factor), prec, int(tau_chunk), int(v_slices), self.v_packed,
                        int(bool(slice_pass)), int(tile_n))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib().gw_create(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream)))
        self._h = h
        self._keep = None

    @property
    def handle(self):
        if self._h is None:
            raise GWError(GW_EINVAL, "context destroyed")
        return self._h

    def shapes(self):
        nk, nao, naux, ntau = self.nk, self.nao, self.naux, self.ntau
        v = (nk * (nk + 1) // 2, naux, nao, nao) if self.v_packed else (nk, nk, naux, nao, nao)
        return {"V": v, "G": (nk, ntau, nao, nao), "H": (nk, nao, nao),
                "Pt": (nk, ntau, naux, naux), "Pw": (nk, self.nwb, naux, naux),
                "Sig": (nk, ntau, nao, nao)}

    def workspace_bytes(self) -> int:
        return int(lib().gw_workspace_bytes(self.handle))

    def destroy(self):
        if self._h is not None:
            lib().gw_destroy(self._h)
            self._h = None
            self._keep = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def gw_create(nk3, nao, naux, ntau, beta, **kw) -> gw_ctx:
    return gw_ctx(nk3, nao, naux, ntau, beta, **kw)


def gw_destroy(ctx: gw_ctx):
    ctx.destroy()


def _host_arr(a, shape, dtype, name):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=dtype)
    if tuple(a.shape) != tuple(shape):
        raise GWError(GW_EINVAL, f"{name}: expected shape {tuple(shape)}, got {a.shape}")
    return a


def gw_set_grids(ctx: gw_ctx, tau, Fb, Bb, Ff, Bf, omega_f, omega_b=None):
    """Replaces the context's grids (host arrays, copied); see include/gw.h for the symmetry rules."""
    T, nb, nf = ctx.ntau, ctx.nwb, ctx.nwf
    arrs = [_host_arr(tau, (T,), np.float64, "tau"), _host_arr(Fb, (nb, T), np.complex128, "Fb"),
            _host_arr(Bb, (T, nb), np.complex128, "Bb"), _host_arr(Ff, (nf, T), np.complex128, "Ff"),
            _host_arr(Bf, (T, nf), np.complex128, "Bf"), _host_arr(omega_b, (nb,), np.float64, "omega_b"),
            _host_arr(omega_f, (nf,), np.float64, "omega_f")]
    ptr = [None if a is None else ctypes.c_void_p(a.ctypes.data) for a in arrs]
    _check(lib().gw_set_grids(ctx.handle, *ptr))


def gw_set_coulomb(ctx: gw_ctx, V):
    _check(lib().gw_set_coulomb(ctx.handle, _ptr(V, ctx.shapes()["V"])))
    ctx._keep = V          # the library borrows V


def gw_polarization(ctx: gw_ctx, G, P0t):
    s = ctx.shapes()
    _check(lib().gw_polarization(ctx.handle, _ptr(G, s["G"]), _ptr(P0t, s["Pt"])))


def gw_to_matsubara(ctx: gw_ctx, stat: int, x, out):
    nb, nelem = x.shape[0], int(np.prod(x.shape[2:]))
    _check(lib().gw_to_matsubara(ctx.handle, stat, _ptr(x), _ptr(out), nb, nelem))


def gw_to_tau(ctx: gw_ctx, stat: int, x, out):
    nb, nelem = x.shape[0], int(np.prod(x.shape[2:]))
    _check(lib().gw_to_tau(ctx.handle, stat, _ptr(x), _ptr(out), nb, nelem))


def gw_aux_dyson(ctx: gw_ctx, P0w, Pw):
    s = ctx.shapes()
    _check(lib().gw_aux_dyson(ctx.handle, _ptr(P0w, s["Pw"]), _ptr(Pw, s["Pw"])))


def gw_screened_interaction(ctx: gw_ctx, P0t, Pt):
    s = ctx.shapes()
    _check(lib().gw_screened_interaction(ctx.handle, _ptr(P0t, s["Pt"]), _ptr(Pt, s["Pt"])))


def gw_self_energy(ctx: gw_ctx, G, Pt, Sig):
    s = ctx.shapes()
    _check(lib().gw_self_energy(ctx.handle, _ptr(G, s["G"]), _ptr(Pt, s["Pt"]), _ptr(Sig, s["Sig"])))


def gw_sigma_eval(ctx: gw_ctx, G, Sig):
    s = ctx.shapes()
    _check(lib().gw_sigma_eval(ctx.handle, _ptr(G, s["G"]), _ptr(Sig, s["Sig"])))


def gw_sigma_eval_q(ctx: gw_ctx, G, Sig, q_begin: int, q_end: int, P0t=None, Pt=None):
    """Sig <- the part of one evaluation from the momentum transfers q in [q_begin, q_end);
    P0t, Pt (optional, [q_end - q_begin][ntau][naux][naux]) receive the range's P0 and P~."""
    s = ctx.shapes()
    nq = int(q_end) - int(q_begin)
    blk = (max(nq, 0),) + tuple(s["Pt"][1:])
    _check(lib().gw_sigma_eval_q(ctx.handle, _ptr(G, s["G"]), _ptr(Sig, s["Sig"]), int(q_begin), int(q_end),
                                 _ptr(P0t, blk) if P0t is not None else None,
                                 _ptr(Pt, blk) if Pt is not None else None))


def gw_dyson_G(ctx: gw_ctx, H, Sig, G):
    s = ctx.shapes()
    _check(lib().gw_dyson_G(ctx.handle, _ptr(H, s["H"]), _ptr(Sig, s["Sig"]), _ptr(G, s["G"])))


def gw_mix(ctx: gw_ctx, Sig_new, Sig_inout, alpha: float) -> float:
    s = ctx.shapes()
    d = ctypes.c_double(0.0)
    _check(lib().gw_mix(ctx.handle, _ptr(Sig_new, s["Sig"]), _ptr(Sig_inout, s["Sig"]), float(alpha),
                        ctypes.byref(d)))
    return d.value


def gw_synchronize(ctx: gw_ctx):
    _check(lib().gw_synchronize(ctx.handle))


def gw_profile_enable(ctx: gw_ctx, on: bool = True):
    _check(lib().gw_profile_enable(ctx.handle, 1 if on else 0))


def gw_launch_count(ctx: gw_ctx) -> int:
    return int(lib().gw_launch_count(ctx.handle))


def gw_profile_read(ctx: gw_ctx) -> dict:
    """{kernel name: {"launches", "ms", "flops", "bytes"}} for every slot with launches."""
    out = {}
    for slot in range(lib().gw_profile_slots()):
        name = ctypes.create_string_buffer(64)
        n = ctypes.c_longlong(0)
        ms, fl, by = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        _check(lib().gw_profile_read(ctx.handle, slot, name, 64, ctypes.byref(n), ctypes.byref(ms),
                                     ctypes.byref(fl), ctypes.byref(by)))
        if n.value:
            out[name.value.decode()] = {"launches": n.value, "ms": ms.value, "flops": fl.value,
                                        "bytes": by.value}
    return out


def gw_polarization_noalloc(nk3, nao, naux, ntau, spin_factor, V, G, P0t, stream=None):
    """P0(tau) without a context or any device allocation (see include/gw.h), for callers whose
    device memory is already committed to their own pools or who may not allocate after start-up.

    V, G and P0t must live on the current CUDA device (and the stream too). The first call on a
    device must come before any stream capture; calls that overlap on the GPU share the
    library's one scratch array and race.
    """
    import torch
    nk = int(np.prod(nk3))
    s = stream if stream is not None else torch.cuda.current_stream()
    cur = torch.cuda.current_device()
    for name, t in (("V", V), ("G", G), ("P0t", P0t)):
        if isinstance(t, torch.Tensor) and t.is_cuda and t.device.index != cur:
            raise GWError(GW_EINVAL, f"{name} is on cuda:{t.device.index}, the current device is cuda:{cur}")
    if s.device.index != cur:
        raise GWError(GW_EINVAL, f"the stream belongs to cuda:{s.device.index}, the current device is cuda:{cur}")
    arr = (ctypes.c_int * 3)(*[int(x) for x in nk3])
    _check(lib().gw_polarization_noalloc(arr, int(nao), int(naux), int(ntau), float(spin_factor),
                                         _ptr(V, (nk, nk, naux, nao, nao)), _ptr(G, (nk, ntau, nao, nao)),
                                         _ptr(P0t, (nk, ntau, naux, naux)), ctypes.c_void_p(s.cuda_stream)))


# ---- request loop -------------------------------------------------------------------------


def make_config(nk3, nao, naux, ntau, beta, mu=0.0, spin_factor=2.0, precision="fp64", tau_chunk=0,
                v_slices=0, v_packed=False, slice_pass=False, tile_n=0):
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return gw_config((ctypes.c_int * 3)(*[int(x) for x in nk3]), int(nao), int(naux), int(ntau), float(beta),
                     float(mu), float(spin_factor), prec, int(tau_chunk), int(v_slices), int(bool(v_packed)),
                     int(bool(slice_pass)), int(tile_n))


def gw_job_bytes(cfg: gw_config) -> int:
    """Device bytes one job with this configuration holds while it runs (0: invalid)."""
    return int(lib().gw_job_bytes(ctypes.byref(cfg)))


def _host(a, shape, name, writable=False):
    """Address of a C-contiguous complex128 host array (numpy, or a CPU torch tensor)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.complex128 or not a.is_contiguous() or tuple(a.shape) != tuple(shape):
                raise GWError(GW_EINVAL, f"{name}: expected a contiguous complex128 CPU tensor of shape {shape}")
            return ctypes.c_void_p(a.data_ptr())
    except ImportError:
        pass
    if not isinstance(a, np.ndarray) or a.dtype != np.complex128 or not a.flags.c_contiguous \
            or tuple(a.shape) != tuple(shape) or (writable and not a.flags.writeable):
        raise GWError(GW_EINVAL, f"{name}: expected a C-contiguous complex128 array of shape {shape}")
    return ctypes.c_void_p(a.ctypes.data)


class gw_server:
    """Owner of one gw_server* (gw_server_create ... gw_server_destroy).

    submit() returns a job id; the host arrays of a job are kept alive here until
    poll() has returned its finished result.
    """

    def __init__(self, hbm_budget: int, max_slots: int = 4):
        h = ctypes.c_void_p()
        _check(lib().gw_server_create(ctypes.byref(h), ctypes.c_size_t(int(hbm_budget)), int(max_slots)))
        self._h = h
        self._keep = {}

    def submit(self, cfg: gw_config, H, V, G0, Sigma_out=None, G_out=None, alpha=0.7, tol=1e-8,
               itermax=20, static_part=False, diis_size=0, diis_start=2, n_electrons=0.0, mu_lo=-5.0,
               mu_hi=5.0, mu_tol=1e-10, diis_kind="diis", method="gw", S=None) -> int:
        nk = cfg.nk[0] * cfg.nk[1] * cfg.nk[2]
        nao, naux, ntau = cfg.nao, cfg.naux, cfg.ntau
        vshape = (nk * (nk + 1) // 2, naux, nao, nao) if cfg.v_packed else (nk, nk, naux, nao, nao)
        job = gw_job(cfg, _host(H, (nk, nao, nao), "H"), _host(V, vshape, "V"),
                     _host(G0, (nk, ntau, nao, nao), "G0"),
                     None if Sigma_out is None else _host(Sigma_out, (nk, ntau, nao, nao), "Sigma_out", True),
                     None if G_out is None else _host(G_out, (nk, ntau, nao, nao), "G_out", True),
                     float(alpha), float(tol), int(itermax), int(bool(static_part)), int(diis_size),
                     int(diis_start), float(n_electrons), float(mu_lo), float(mu_hi), float(mu_tol),
                     _code(DIIS_KINDS, diis_kind), _code(METHODS, method),
                     None if S is None else _host(S, (nk, nao, nao), "S"))
        jid = ctypes.c_uint64()
        _check(lib().gw_submit(self._h, ctypes.byref(job), ctypes.byref(jid)))
        self._keep[jid.value] = (H, V, G0, Sigma_out, G_out, S)
        return jid.value

    def poll(self, job_id: int, timeout_us: int = -1):
        """(rc, result dict): rc is GW_OK once the job finished, else GW_EAGAIN / GW_ETIMEOUT."""
        r = gw_job_result()
        rc = lib().gw_poll(self._h, ctypes.c_uint64(job_id), ctypes.byref(r), int(timeout_us))
        if rc not in (GW_OK, GW_EAGAIN, GW_ETIMEOUT):
            _check(rc)
        if rc == GW_OK:
            self._keep.pop(job_id, None)
        return rc, {"status": r.status, "iterations": r.iterations, "max_abs_dsigma": r.max_abs_dsigma,
                    "t_submit": r.t_submit, "t_start": r.t_start, "t_end": r.t_end, "mu": r.mu}

    def destroy(self):
        if self._h is not None:
            lib().gw_server_destroy(self._h)
            self._h = None
            self._keep = {}

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ---- batched evaluation of independent systems ------------------------------------------------


class gw_batch:
    """Owner of one gw_batch* (gw_batch_create ... gw_batch_destroy); cfgs are gw_config
    structures (see make_config). The torch tensors handed in are kept alive here."""

    def __init__(self, cfgs, max_streams=8, hbm_budget=0, stream=None):
        import torch
        self.n = len(cfgs)
        self.cfgs = (gw_config * self.n)(*cfgs)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib().gw_batch_create(ctypes.byref(h), self.cfgs, self.n, int(max_streams),
                                     ctypes.c_size_t(int(hbm_budget)), ctypes.c_void_p(self.stream.cuda_stream)))
        self._h = h
        self._keep = {}

    def _shape(self, i, what):
        c = self.cfgs[i]
        nk = c.nk[0] * c.nk[1] * c.nk[2]
        if what == "V":
            return (nk, nk, c.naux, c.nao, c.nao)
        return (nk, c.ntau, c.nao, c.nao)

    def _ptrs(self, tensors, what):
        if len(tensors) != self.n:
            raise GWError(GW_EINVAL, f"expected {self.n} {what} tensors")
        return (ctypes.c_void_p * self.n)(*[_ptr(t, self._shape(i, what)) for i, t in enumerate(tensors)])

    def set_coulomb(self, V):
        _check(lib().gw_batch_set_coulomb(self._h, self._ptrs(V, "V")))
        self._keep["V"] = list(V)

    def sigma_eval(self, G, Sig, mode="graph"):
        m = BATCH_MODES[mode] if isinstance(mode, str) else int(mode)
        _check(lib().gw_batch_sigma_eval(self._h, self._ptrs(G, "G"), self._ptrs(Sig, "Sig"), m))
        self._keep["G"], self._keep["Sig"] = list(G), list(Sig)

    def autotune(self, G, Sig):
        chosen = (ctypes.c_int * self.n)()
        _check(lib().gw_batch_autotune(self._h, self._ptrs(G, "G"), self._ptrs(Sig, "Sig"), chosen))
        return list(chosen)

    def tuned(self):
        """[(tau batch, tile width)] of every system (gw_batch_tuned)."""
        out = []
        for i in range(self.n):
            t, w = ctypes.c_int(0), ctypes.c_int(0)
            _check(lib().gw_batch_tuned(self._h, i, ctypes.byref(t), ctypes.byref(w)))
            out.append((t.value, w.value))
        return out

    def synchronize(self):
        _check(lib().gw_batch_synchronize(self._h))

    def destroy(self):
        if self._h is not None:
            lib().gw_batch_destroy(self._h)
            self._h = None
            self._keep = {}

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ---- static part, chemical potential, DIIS (Eq. sigma_inf, Sec. 2.4, Sec. 5.3) -------------


def gw_density(ctx: gw_ctx, G, gamma):
    nk, nao = ctx.nk, ctx.nao
    _check(lib().gw_density(ctx.handle, _ptr(G, (nk, ctx.ntau, nao, nao)), _ptr(gamma, (nk, nao, nao))))


def gw_sigma_inf(ctx: gw_ctx, G, SigInf):
    nk, nao = ctx.nk, ctx.nao
    _check(lib().gw_sigma_inf(ctx.handle, _ptr(G, (nk, ctx.ntau, nao, nao)), _ptr(SigInf, (nk, nao, nao))))


def gw_set_mu(ctx: gw_ctx, mu: float):
    _check(lib().gw_set_mu(ctx.handle, float(mu)))
    ctx.mu = float(mu)


def gw_particle_number(ctx: gw_ctx, G) -> float:
    n = ctypes.c_double()
    _check(lib().gw_particle_number(ctx.handle, _ptr(G, (ctx.nk, ctx.ntau, ctx.nao, ctx.nao)), ctypes.byref(n)))
    return n.value


def gw_find_mu(ctx: gw_ctx, Heff, Sig, n_target, mu_lo, mu_hi, tol, G) -> float:
    nk, nao = ctx.nk, ctx.nao
    mu = ctypes.c_double()
    _check(lib().gw_find_mu(ctx.handle, _ptr(Heff, (nk, nao, nao)), _ptr(Sig, (nk, ctx.ntau, nao, nao)),
                            float(n_target), float(mu_lo), float(mu_hi), float(tol),
                            _ptr(G, (nk, ctx.ntau, nao, nao)), ctypes.byref(mu)))
    ctx.mu = mu.value
    return mu.value


class gw_diis:
    """Owner of one gw_diis* (Pulay extrapolation of the self-energy)."""

    def __init__(self, n_elem, max_vectors=5, stream=None, n_residual=0):
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.max_vectors = int(max_vectors)
        h = ctypes.c_void_p()
        _check(lib().gw_diis_create(ctypes.byref(h), ctypes.c_longlong(int(n_elem)),
                                    ctypes.c_longlong(int(n_residual)), self.max_vectors,
                                    ctypes.c_void_p(self.stream.cuda_stream)))
        self._h = h
        self.n = int(n_elem)

    def push(self, sigma_in, sigma_out):
        _check(lib().gw_diis_push(self._h, _ptr(sigma_in), _ptr(sigma_out)))

    def push_residual(self, sigma_out, residual):
        _check(lib().gw_diis_push_residual(self._h, _ptr(sigma_out), _ptr(residual)))

    def extrapolate(self, out):
        c = (ctypes.c_double * self.max_vectors)()
        m = ctypes.c_int()
        _check(lib().gw_diis_extrapolate(self._h, _ptr(out), c, ctypes.byref(m)))
        return list(c)[:m.value]

    def destroy(self):
        if self._h is not None:
            lib().gw_diis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


DIIS_KINDS = {"diis": 0, "cdiis": 1}
METHODS = {"gw": 0, "gf2": 1, "hf": 2}


def _code(table, x):
    return table[x] if isinstance(x, str) else int(x)


def scgw_options(alpha=0.5, tol=1e-8, itermax=20, static_part=True, diis_size=0, diis_start=2, n_electrons=0.0,
                 mu_lo=-5.0, mu_hi=5.0, mu_tol=1e-10, diis_kind="diis", method="gw", resume=False) -> gw_scgw_options:
    return gw_scgw_options(float(alpha), float(tol), int(itermax), int(bool(static_part)), int(diis_size),
                           int(diis_start), float(n_electrons), float(mu_lo), float(mu_hi), float(mu_tol),
                           _code(DIIS_KINDS, diis_kind), _code(METHODS, method), int(bool(resume)))


def gw_gf2_self_energy(ctx: gw_ctx, G, Sig):
    s = ctx.shapes()
    _check(lib().gw_gf2_self_energy(ctx.handle, _ptr(G, s["G"]), _ptr(Sig, s["Sig"])))


def gw_gf2_exchange(ctx: gw_ctx, G, SigX):
    s = ctx.shapes()
    _check(lib().gw_gf2_exchange(ctx.handle, _ptr(G, s["G"]), _ptr(SigX, s["Sig"])))


def gw_commutator_residual(ctx: gw_ctx, H, SigInf, Sig, G, e):
    s = ctx.shapes()
    nk, nao = ctx.nk, ctx.nao
    _check(lib().gw_commutator_residual(ctx.handle, _ptr(H, s["H"]),
                                        None if SigInf is None else _ptr(SigInf, (nk, nao, nao)),
                                        _ptr(Sig, s["Sig"]), _ptr(G, s["G"]), _ptr(e, (nk, ctx.nwf, nao, nao))))


def gw_scgw_bytes(cfg: gw_config, opt: gw_scgw_options) -> int:
    return int(lib().gw_scgw_bytes(ctypes.byref(cfg), ctypes.byref(opt)))


def gw_scgw(ctx: gw_ctx, H, G, Sigma=None, SigInf=None, opt: gw_scgw_options = None):
    """Runs the loop (G in: G0, out: the last G). Returns (status, result dict); status is GW_OK or
    GW_ENOTCONV, any other failure raises."""
    s = ctx.shapes()
    opt = opt if opt is not None else scgw_options()
    r = gw_scgw_result()
    rc = lib().gw_scgw(ctx.handle, _ptr(H, s["H"]), _ptr(G, s["G"]),
                       None if Sigma is None else _ptr(Sigma, s["Sig"]),
                       None if SigInf is None else _ptr(SigInf, (ctx.nk, ctx.nao, ctx.nao)),
                       ctypes.byref(opt), ctypes.byref(r))
    if rc != GW_ENOTCONV:
        _check(rc)
    if opt.n_electrons > 0:
        ctx.mu = r.mu
    return rc, {"iterations": r.iterations, "max_abs_dsigma": r.max_abs_dsigma, "mu": r.mu,
                "n_electrons": r.n_electrons}


def gw_k_interpolate(nk3, X, f, Xf, stream=None):
    """X [nk][...] on the nk3 mesh -> Xf [len(f)][...] at the fractional k coordinates f [nkf][3]."""
    import torch
    nk = int(np.prod(nk3))
    if X.shape[0] != nk or Xf.shape[0] != len(f) or tuple(X.shape[1:]) != tuple(Xf.shape[1:]):
        raise GWError(GW_EINVAL, "gw_k_interpolate: shapes do not match")
    fa = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1, 3))
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().gw_k_interpolate((ctypes.c_int * 3)(*[int(x) for x in nk3]), _ptr(X),
                                  ctypes.c_longlong(X[0].numel() if nk else 0), int(len(fa)),
                                  fa.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(Xf),
                                  ctypes.c_void_p(st.cuda_stream)))


def gw_ir_grids(beta, lam=1e4, eps=1e-10):
    """IR grids (see include/gw.h): (tau, Fb, Bb, Ff, Bf, omega_f, omega_b) in the argument order of
    gw_set_grids(ctx, tau, Fb, Bb, Ff, Bf, omega_f, omega_b); len(tau) is the ntau of the context."""
    n = ctypes.c_int(0)
    _check(lib().gw_ir_grids(float(beta), float(lam), float(eps), 0, ctypes.byref(n), None, None, None, None, None,
                             None, None))
    T = n.value
    nb, nf = gw_sample_count(T, 0), gw_sample_count(T, 1)
    tau = np.zeros(T)
    Fb, Bb = np.zeros((nb, T), complex), np.zeros((T, nb), complex)
    Ff, Bf = np.zeros((nf, T), complex), np.zeros((T, nf), complex)
    wb, wf = np.zeros(nb), np.zeros(nf)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    _check(lib().gw_ir_grids(float(beta), float(lam), float(eps), T, ctypes.byref(n), p(tau), p(Fb), p(Bb), p(Ff),
                             p(Bf), p(wb), p(wf)))
    return tau, Fb, Bb, Ff, Bf, wf, wb


def gw_set_overlap(ctx: gw_ctx, S=None):
    """Overlap S [nk][nao][nao] of Eq. dyson (borrowed), or None for S = I."""
    _check(lib().gw_set_overlap(ctx.handle, None if S is None else _ptr(S, (ctx.nk, ctx.nao, ctx.nao))))
    ctx._keep_s = S


def gw_checkpoint_write(path, cfg: gw_config, mu, iteration, arrays: dict):
    """arrays: name -> complex128 numpy array (host); see include/gw.h for the format."""
    items = [(k, np.ascontiguousarray(v, dtype=np.complex128)) for k, v in arrays.items()]
    n = len(items)
    names = (ctypes.c_char_p * max(n, 1))(*[k.encode() for k, _ in items])
    data = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for _, a in items])
    counts = (ctypes.c_longlong * max(n, 1))(*[a.size for _, a in items])
    _check(lib().gw_checkpoint_write(str(path).encode(), ctypes.byref(cfg), float(mu), int(iteration), n,
                                     ctypes.cast(names, ctypes.c_void_p), ctypes.cast(data, ctypes.c_void_p),
                                     ctypes.cast(counts, ctypes.c_void_p)))


def gw_checkpoint_read(path, shapes: dict, cfg: gw_config = None):
    """shapes: name -> shape of the arrays to read. Returns (cfg, mu, iteration, {name: array})."""
    cfg = cfg if cfg is not None else make_config((1, 1, 1), 1, 1, 1, 1.0)
    out = {k: np.zeros(tuple(v), complex) for k, v in shapes.items()}
    n = len(out)
    names = (ctypes.c_char_p * max(n, 1))(*[k.encode() for k in out])
    data = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for a in out.values()])
    counts = (ctypes.c_longlong * max(n, 1))(*[a.size for a in out.values()])
    mu, it = ctypes.c_double(), ctypes.c_int()
    _check(lib().gw_checkpoint_read(str(path).encode(), ctypes.byref(cfg), ctypes.byref(mu), ctypes.byref(it), n,
                                    ctypes.cast(names, ctypes.c_void_p), ctypes.cast(data, ctypes.c_void_p),
                                    ctypes.cast(counts, ctypes.c_void_p)))
    return cfg, mu.value, it.value, out


def gw_selftest_bounded_wait(limit_s=0.2, stream=None):
    """(status, code) of the bounded-wait self-test: GW_EDEVTIMEOUT and 99 when the wait gave up."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    code = ctypes.c_int(0)
    rc = lib().gw_selftest_bounded_wait(float(limit_s), ctypes.byref(code), ctypes.c_void_p(st.cuda_stream))
    return rc, code.value


def gw_check_guards(ctx: gw_ctx):
    """Raises GWError if a kernel wrote past the end of one of the context's workspaces."""
    _check(lib().gw_check_guards(ctx.handle))


def gw_debug_mark_guard(ctx: gw_ctx, index: int = 0):
    """Test hook: change one byte of a guard zone so that gw_check_guards must report it."""
    _check(lib().gw_debug_mark_guard(ctx.handle, int(index)))
