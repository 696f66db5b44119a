"""MUFFIN multispectral deconvolution with ADA-PT tuning on GB300 (sm_103a).

Python binding of the C ABI in ``include/muffin.h``: argument marshalling
only, every step of the iteration runs in ``libmuffin.so``.  Arrays may be
CUDA torch tensors (used in place, on the current torch stream) or host
arrays (numpy or CPU tensors, copied by the library inside the call); all
cubes are float32 ``[L, n, n]``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import native
from .native import MUFFIN_WARM, MuffinError, SureRecord

__all__ = ["Plan", "Server", "MuffinError", "filter_taps", "dct_table", "library",
           "estimate_bytes"]


def library():
    return native.load()


def _dictionary(name) -> int:
    """Spatial dictionary code: "daubechies" (union of Daubechies bases) or
    "iuwt" (starlet)."""
    codes = {"daubechies": 0, "iuwt": 1}
    if name not in codes:
        raise ValueError(f"dictionary must be one of {sorted(codes)}, got {name!r}")
    return codes[name]


def _ptr(a, keep: list, dtype=np.float32):
    """Raw pointer of a contiguous float32 array (torch tensor or numpy)."""
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float32 or not a.is_contiguous():
                raise TypeError("tensors must be contiguous float32")
            keep.append(a)
            return ctypes.c_void_p(a.data_ptr())
    except ImportError:
        pass
    arr = np.asarray(a)
    if arr.dtype != dtype or not arr.flags.c_contiguous:
        raise TypeError(f"arrays must be C-contiguous {np.dtype(dtype).name}")
    keep.append(arr)
    return ctypes.c_void_p(arr.ctypes.data)


def _stream_handle():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def filter_taps(p: int) -> np.ndarray:
    """db<p> scaling filter as built by the library (host FP64)."""
    h = (ctypes.c_double * (2 * p))()
    native.check(library().muffin_filter_taps(p, h))
    return np.array(h[:], dtype=np.float64)


def dct_table(L: int) -> np.ndarray:
    C = (ctypes.c_double * (L * L))()
    native.check(library().muffin_dct_table(L, C))
    return np.array(C[:], dtype=np.float64).reshape(L, L)


class Plan:
    """A MUFFIN plan for L bands of n x n pixels (see ``muffin_plan_create``)."""

    def __init__(self, n: int, nbands: int, psf, *, n_wavelets: int = 8,
                 levels: int = 3, sigma: float = 10.0, step_rule: int = 0,
                 tau_safety: float = 0.99, positivity: bool = True,
                 sure: bool = False, alpha=None, beta=None, stream=None,
                 batch: int = 1, dictionary: str = "daubechies", precision: str = "tf32",
                 tau: float = 0.0):
        lib = library()
        self._lib = lib
        self.n, self.L, self.B = n, nbands, batch
        self.dictionary = dictionary
        # coefficient planes per band: K bases, or J + 1 starlet planes
        self.K = levels + 1 if dictionary == "iuwt" else n_wavelets
        p = native.Params()
        lib.muffin_params_default(ctypes.byref(p), n, nbands)
        p.n_wavelets, p.levels, p.sigma = n_wavelets, levels, sigma
        p.step_rule, p.tau_safety = step_rule, tau_safety
        p.positivity, p.sure, p.batch = int(positivity), int(sure), int(batch)
        p.dictionary = _dictionary(dictionary)
        if precision not in ("tf32", "fp32"):
            raise ValueError(f"precision must be 'tf32' or 'fp32', got {precision!r}")
        p.precision = 1 if precision == "fp32" else 0
        p.tau = float(tau)
        keep = []
        handle = ctypes.c_void_p()
        st = stream if stream is not None else _stream_handle()
        native.check(lib.muffin_plan_create(
            ctypes.byref(p), _ptr(psf, keep), _ptr(alpha, keep), _ptr(beta, keep),
            st, ctypes.byref(handle)))
        self._h = handle

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.muffin_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- queries
    @property
    def device_bytes(self) -> int:
        return int(self._lib.muffin_plan_device_bytes(self._h))

    @property
    def lipschitz(self):
        """beta = max ||H_l||^2 (a list of B values when the plan is batched)."""
        b = (ctypes.c_double * self.B)()
        native.check(self._lib.muffin_plan_lipschitz(self._h, b))
        return b[0] if self.B == 1 else list(b)

    def load_psf(self, psf, b0: int = 0, b1: int = None) -> None:
        """Replace the PSFs of cubes [b0, b1) (state kept)."""
        keep = []
        b1 = self.B if b1 is None else b1
        native.check(self._lib.muffin_plan_load_psf(self._h, int(b0), int(b1), _ptr(psf, keep)))

    def graphs(self, on: bool = True) -> None:
        native.check(self._lib.muffin_plan_graphs(self._h, int(on)))

    def autotune(self, cache: str | None = None) -> native.TuneInfo:
        """Pick the fastest launch variants for this shape (results do not
        change); the next solve must start cold."""
        info = native.TuneInfo()
        path = None if cache is None else os.fsencode(cache)
        native.check(self._lib.muffin_plan_autotune(self._h, path, ctypes.byref(info)))
        return info

    def set_spectral_kernel(self, tcgen05: bool) -> None:
        """Spectral step on the tcgen05 tensor cores (64-band plans) or on
        the mma.sync kernel."""
        native.check(self._lib.muffin_plan_set_spectral_kernel(self._h, int(bool(tcgen05))))

    def inject_timeout(self, on: bool) -> None:
        """Test hook: make the tensor-core waits of the next calls run out."""
        native.check(self._lib.muffin_plan_inject_timeout(self._h, int(bool(on))))

    def schedule(self) -> dict:
        """The launch choices of the per-iteration schedule (muffin_schedule)."""
        sc = native.Schedule()
        native.check(self._lib.muffin_plan_get_schedule(self._h, ctypes.byref(sc)))
        return {f: getattr(sc, f) for f, _ in native.Schedule._fields_}

    def set_schedule(self, **kw) -> None:
        """Change some launch choices (keys of ``schedule()``); the next solve
        starts cold."""
        cur = self.schedule()
        unknown = set(kw) - set(cur)
        if unknown:
            raise ValueError(f"unknown schedule keys {sorted(unknown)}")
        cur.update(kw)
        sc = native.Schedule(**{k: int(v) for k, v in cur.items()})
        native.check(self._lib.muffin_plan_set_schedule(self._h, ctypes.byref(sc)))

    def set_tuning(self, syn_packed: int = 0, dct_ctas_per_sm: int = 0) -> None:
        native.check(self._lib.muffin_plan_set_tuning(self._h, int(syn_packed),
                                                      int(dct_ctas_per_sm)))

    # -- solvers
    def solve(self, dirty, x, iters: int, mu, gamma, warm: bool = False) -> native.Info:
        """mu, gamma: scalars (all cubes) or sequences of B values."""
        keep, info = [], native.Info()
        flags = MUFFIN_WARM if warm else 0
        if np.ndim(mu) == 0 and np.ndim(gamma) == 0:
            native.check(self._lib.muffin_solve(
                self._h, _ptr(dirty, keep), _ptr(x, keep), int(iters), float(mu),
                float(gamma), flags, ctypes.byref(info)))
        else:
            m = (ctypes.c_double * self.B)(*np.broadcast_to(np.asarray(mu, float), self.B))
            g = (ctypes.c_double * self.B)(*np.broadcast_to(np.asarray(gamma, float), self.B))
            native.check(self._lib.muffin_solve_batch(
                self._h, _ptr(dirty, keep), _ptr(x, keep), int(iters), m, g, flags,
                ctypes.byref(info)))
        return info

    def sure_tune(self, dirty, delta, noise_var, x, theta, iters: int, *,
                  window: int = 10, eta=(1e-3, 1e-3), theta_min: float = 1e-8,
                  reset: bool = True, eps: float, warm: bool = False):
        """Returns (theta, trace, info); trace is a list of dicts per window.

        For a batched plan theta is a [B][2] array-like and the returned
        theta and trace are lists over the B cubes."""
        keep = []
        sp = native.SureParams()
        self._lib.muffin_sure_params_default(ctypes.byref(sp))
        sp.iters, sp.window = int(iters), int(window)
        sp.eta_mu, sp.eta_gamma = float(eta[0]), float(eta[1])
        sp.theta_min, sp.reset_each_window, sp.eps = theta_min, int(reset), float(eps)
        B = self.B
        th_in = np.broadcast_to(np.asarray(theta, dtype=np.float64).reshape(-1, 2), (B, 2))
        th = (ctypes.c_double * (2 * B))(*th_in.ravel())
        cap = int(iters) // int(window) + 1
        rec = (SureRecord * (cap * B))()
        nv = None
        if noise_var is not None:
            nv_arr = np.ascontiguousarray(noise_var, dtype=np.float64)
            keep.append(nv_arr)
            nv = ctypes.c_void_p(nv_arr.ctypes.data)
        info = native.Info()
        native.check(self._lib.muffin_sure_tune(
            self._h, _ptr(dirty, keep), _ptr(delta, keep), nv, ctypes.byref(sp),
            _ptr(x, keep), th, rec, MUFFIN_WARM if warm else 0, ctypes.byref(info)))
        def cube_trace(c):
            return [dict(k=r.k, mu=r.mu, gamma=r.gamma, sugar_mu=r.sugar_mu,
                         sugar_gamma=r.sugar_gamma, psure=r.psure, tau=r.tau)
                    for r in rec[c * cap: c * cap + info.records]]
        if B == 1:
            return (th[0], th[1]), cube_trace(0), info
        return ([(th[2 * c], th[2 * c + 1]) for c in range(B)],
                [cube_trace(c) for c in range(B)], info)

    def sure_global(self, dirty, delta, noise_var, x, theta, n_c: int, outer: int, *,
                    eta=(1e-3, 1e-3), theta_min: float = 1e-8, eps: float):
        """Global SUGAR descent (Eq. globalgrad): `outer` steps, each after n_c
        iterations from the same initial cube x.  Returns (theta, trace, info)
        with one trace record per step (lists over cubes when B > 1)."""
        keep = []
        sp = native.SureParams()
        self._lib.muffin_sure_params_default(ctypes.byref(sp))
        sp.iters, sp.window = int(n_c), int(n_c)
        sp.eta_mu, sp.eta_gamma = float(eta[0]), float(eta[1])
        sp.theta_min, sp.reset_each_window, sp.eps = theta_min, 1, float(eps)
        B = self.B
        th_in = np.broadcast_to(np.asarray(theta, dtype=np.float64).reshape(-1, 2), (B, 2))
        th = (ctypes.c_double * (2 * B))(*th_in.ravel())
        cap = max(1, int(outer))
        rec = (SureRecord * (cap * B))()
        nv_arr = np.ascontiguousarray(noise_var, dtype=np.float64)
        keep.append(nv_arr)
        info = native.Info()
        native.check(self._lib.muffin_sure_global(
            self._h, _ptr(dirty, keep), _ptr(delta, keep), ctypes.c_void_p(nv_arr.ctypes.data),
            ctypes.byref(sp), int(outer), _ptr(x, keep), th, rec, ctypes.byref(info)))
        def cube_trace(c):
            return [dict(k=r.k, mu=r.mu, gamma=r.gamma, sugar_mu=r.sugar_mu,
                         sugar_gamma=r.sugar_gamma, psure=r.psure, tau=r.tau)
                    for r in rec[c * cap: c * cap + info.records]]
        if B == 1:
            return (th[0], th[1]), cube_trace(0), info
        return ([(th[2 * c], th[2 * c + 1]) for c in range(B)],
                [cube_trace(c) for c in range(B)], info)

    def sure_global_auto(self, dirty, delta, noise_var, x, theta, n_cap: int, outer: int, *,
                         check: int, tol: float, eta=(1e-3, 1e-3), theta_min: float = 1e-8,
                         eps: float):
        """Global SUGAR descent with n_c chosen by watching ||SUGAR_{0:k}||
        every `check` iterations (``muffin_sure_global_auto``); the trace
        records' k is the n_c of each step."""
        keep = []
        sp = native.SureParams()
        self._lib.muffin_sure_params_default(ctypes.byref(sp))
        sp.iters, sp.window = int(n_cap), int(check)
        sp.eta_mu, sp.eta_gamma = float(eta[0]), float(eta[1])
        sp.theta_min, sp.eps = theta_min, float(eps)
        B = self.B
        th_in = np.broadcast_to(np.asarray(theta, dtype=np.float64).reshape(-1, 2), (B, 2))
        th = (ctypes.c_double * (2 * B))(*th_in.ravel())
        cap = max(1, int(outer))
        rec = (SureRecord * (cap * B))()
        nv_arr = np.ascontiguousarray(noise_var, dtype=np.float64)
        keep.append(nv_arr)
        info = native.Info()
        native.check(self._lib.muffin_sure_global_auto(
            self._h, _ptr(dirty, keep), _ptr(delta, keep), ctypes.c_void_p(nv_arr.ctypes.data),
            ctypes.byref(sp), int(outer), int(check), float(tol), _ptr(x, keep), th, rec,
            ctypes.byref(info)))
        def cube_trace(c):
            return [dict(k=r.k, mu=r.mu, gamma=r.gamma, sugar_mu=r.sugar_mu,
                         sugar_gamma=r.sugar_gamma, psure=r.psure, tau=r.tau)
                    for r in rec[c * cap: c * cap + info.records]]
        if B == 1:
            return (th[0], th[1]), cube_trace(0), info
        return ([(th[2 * c], th[2 * c + 1]) for c in range(B)],
                [cube_trace(c) for c in range(B)], info)

    def noise_mad(self, dirty) -> np.ndarray:
        """Per-band noise variances sigma_l^2 of a dirty cube by the wavelet
        MAD (``muffin_noise_mad``): [L] (or [B][L] for a batched plan)."""
        keep = []
        out = (ctypes.c_double * (self.B * self.L))()
        native.check(self._lib.muffin_noise_mad(self._h, _ptr(dirty, keep), out))
        v = np.array(out[:], dtype=np.float64)
        return v if self.B == 1 else v.reshape(self.B, self.L)

    # -- convergence monitor
    def set_monitor(self, every: int = 0, objective: bool = False, rel_tol: float = 0.0,
                    off: bool = False) -> None:
        """Check the iterates every `every` iterations (``muffin_plan_set_monitor``)."""
        if off:
            native.check(self._lib.muffin_plan_set_monitor(self._h, None))
            return
        mp = native.MonitorParams(int(every), int(bool(objective)), float(rel_tol))
        native.check(self._lib.muffin_plan_set_monitor(self._h, ctypes.byref(mp)))

    def monitor_records(self) -> list:
        cnt = ctypes.c_int32()
        native.check(self._lib.muffin_plan_monitor_read(self._h, None, 0, ctypes.byref(cnt)))
        arr = (native.MonitorRecord * max(1, cnt.value))()
        native.check(self._lib.muffin_plan_monitor_read(self._h, arr, cnt.value,
                                                        ctypes.byref(cnt)))
        return [dict(k=r.k, cube=r.cube, rel_change=r.rel_change, objective=r.objective,
                     nonfinite=int(r.nonfinite)) for r in arr[: cnt.value]]

    def objective(self, dirty, x, mu, gamma):
        """Eqs. probopt/RegAll per cube (a float when the plan holds one cube)."""
        keep = []
        B = self.B
        m = (ctypes.c_double * B)(*np.broadcast_to(np.asarray(mu, float), B))
        g = (ctypes.c_double * B)(*np.broadcast_to(np.asarray(gamma, float), B))
        f = (ctypes.c_double * B)()
        native.check(self._lib.muffin_objective(self._h, _ptr(dirty, keep), _ptr(x, keep),
                                                m, g, f))
        return f[0] if B == 1 else list(f)

    # -- weights (Eq. 2regpar)
    def set_weights(self, alpha=None, beta=None) -> None:
        """alpha [B][n*n] pixel weights, beta [B][L] band weights (None keeps)."""
        keep = []
        a = None if alpha is None else _ptr(np.ascontiguousarray(alpha, np.float32)
                                             if isinstance(alpha, np.ndarray) else alpha, keep)
        b = None if beta is None else _ptr(np.ascontiguousarray(beta, np.float32)
                                           if isinstance(beta, np.ndarray) else beta, keep)
        native.check(self._lib.muffin_plan_set_weights(self._h, a, b))

    def weights_from_x0(self, x0, eps_alpha: float, eps_beta: float):
        """Install alpha_n = 1/(||W_lambda x0^n|| + eps_alpha) and beta_l =
        1/(||W_s x0_l|| + eps_beta); returns them as (alpha [B][n][n],
        beta [B][L]) numpy arrays (the cube axis dropped when B == 1)."""
        keep = []
        B, L, n = self.B, self.L, self.n
        a = np.empty((B, n, n), np.float32)
        b = np.empty((B, L), np.float32)
        native.check(self._lib.muffin_plan_weights_from_x0(
            self._h, _ptr(x0, keep), float(eps_alpha), float(eps_beta),
            ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(b.ctypes.data)))
        return (a[0], b[0]) if B == 1 else (a, b)

    # -- profile
    def profile(self, on: bool = True) -> None:
        native.check(self._lib.muffin_profile_enable(self._h, int(on)))

    def profile_stats(self) -> list:
        cnt = ctypes.c_int32()
        native.check(self._lib.muffin_profile_read(self._h, None, 0, ctypes.byref(cnt)))
        arr = (native.KernelStat * max(1, cnt.value))()
        native.check(self._lib.muffin_profile_read(self._h, arr, cnt.value, ctypes.byref(cnt)))
        return [dict(name=a.name.decode(), launches=int(a.launches), total_ms=a.total_ms,
                     bytes_per_launch=a.bytes_per_launch, flops_per_launch=a.flops_per_launch)
                for a in arr[: cnt.value]]

    # -- checkpoints
    def state_export(self) -> bytes:
        sz = ctypes.c_size_t()
        native.check(self._lib.muffin_state_size(self._h, ctypes.byref(sz)))
        buf = ctypes.create_string_buffer(sz.value)
        native.check(self._lib.muffin_state_export(self._h, buf, sz.value))
        return buf.raw

    def state_arrays(self) -> dict:
        """The iterates of ``state_export`` as numpy arrays (layout of the
        blob documented in muffin.h): x, v, t [G][C][B*L][n][n] and u
        [G][C][B*L][K][n][n] for the G chain groups (G = 2 with ADA-PT: on y
        and on y + eps delta) of C chains each (primal, d/dmu, d/dgamma),
        b, and with ADA-PT b_bar and H^T delta [B*L][n][n]; mu, gamma [B]."""
        blob = self.state_export()
        hdr = np.frombuffer(blob, dtype=np.int32, count=14)
        n, L, K, sure, B = (int(v) for v in (hdr[2], hdr[3], hdr[4], hdr[6], hdr[7]))
        off = 56
        cub = np.frombuffer(blob, dtype=np.float64, count=3 * B, offset=off).reshape(B, 3)
        off += 24 * B
        NL, G = B * L * n * n, 2 if sure else 1
        C = 3 if sure else 1
        out = {"mu": cub[:, 1].copy(), "gamma": cub[:, 2].copy()}

        def take(count, shape):
            nonlocal off
            a = np.frombuffer(blob, dtype=np.float32, count=count, offset=off).reshape(shape)
            off += 4 * count
            return a.copy()
        cube = (B * L, n, n)
        parts = {k: [] for k in ("x", "u", "v", "t")}
        for _ in range(G):
            parts["x"].append(take(C * NL, (C,) + cube))
            parts["u"].append(take(C * NL * K, (C, B * L, K, n, n)))
            parts["v"].append(take(C * NL, (C,) + cube))
            parts["t"].append(take(C * NL, (C,) + cube))
        out.update({k: np.stack(v) for k, v in parts.items()})
        out["b"] = take(NL, cube)
        if sure:
            out["bbar"] = take(NL, cube)
            out["htd"] = take(NL, cube)
        return out

    def state_import(self, blob: bytes) -> None:
        buf = ctypes.create_string_buffer(blob, len(blob))
        native.check(self._lib.muffin_state_import(self._h, buf, len(blob)))

    # -- single operators
    def op_gradient(self, x, g, dirty=None):
        keep = []
        native.check(self._lib.muffin_op_gradient(
            self._h, _ptr(x, keep), _ptr(dirty, keep), _ptr(g, keep)))

    def op_analysis(self, x, u):
        keep = []
        native.check(self._lib.muffin_op_analysis(self._h, _ptr(x, keep), _ptr(u, keep)))

    def op_synthesis(self, u, x):
        keep = []
        native.check(self._lib.muffin_op_synthesis(self._h, _ptr(u, keep), _ptr(x, keep)))

    def load_visibilities(self, vis, weights):
        """Visibility-domain data term (see ``muffin_plan_load_visibilities``):
        vis [B][L][n][n] complex per-cell sums (numpy complex or a torch
        complex64 tensor, or float32 [..., 2] re/im pairs), weights
        [B][L][n][n] float32 natural weights.  A following ``solve`` with
        dirty = None runs on this data term."""
        keep = []
        if isinstance(vis, np.ndarray) and np.iscomplexobj(vis):
            vis = np.ascontiguousarray(vis.astype(np.complex64)).view(np.float32)
        elif hasattr(vis, "is_complex") and vis.is_complex():
            import torch
            vis = torch.view_as_real(vis.to(torch.complex64)).contiguous()
        if isinstance(weights, np.ndarray):
            weights = np.ascontiguousarray(weights, np.float32)
        native.check(self._lib.muffin_plan_load_visibilities(
            self._h, _ptr(vis, keep), _ptr(weights, keep)))

    def op_dct(self, x, v, inverse: bool = False):
        keep = []
        native.check(self._lib.muffin_op_dct(self._h, _ptr(x, keep), _ptr(v, keep),
                                             int(inverse)))


def estimate_bytes(n: int, nbands: int, *, n_wavelets: int = 8, levels: int = 3,
                   sure: bool = False, batch: int = 1, dictionary: str = "daubechies",
                   precision: str = "tf32") -> int:
    """Device bytes a plan of this shape allocates."""
    lib = library()
    p = native.Params()
    lib.muffin_params_default(ctypes.byref(p), n, nbands)
    p.n_wavelets, p.levels, p.sure, p.batch = n_wavelets, levels, int(sure), batch
    p.dictionary = _dictionary(dictionary)
    p.precision = 1 if precision == "fp32" else 0
    out = ctypes.c_size_t()
    native.check(lib.muffin_plan_estimate_bytes(ctypes.byref(p), ctypes.byref(out)))
    return int(out.value)


class Server:
    """Continuous-batching request server (see ``muffin_server_create``)."""

    def __init__(self, *, hbm_budget_bytes: int = 0, max_batch: int = 8,
                 n_wavelets: int = 8, levels: int = 3, sigma: float = 10.0,
                 chunk: int = 10, max_active_voxels: int = 0, stream=None):
        lib = library()
        self._lib = lib
        p = native.ServerParams()
        lib.muffin_server_params_default(ctypes.byref(p))
        p.hbm_budget_bytes, p.max_batch, p.chunk = int(hbm_budget_bytes), int(max_batch), int(chunk)
        p.n_wavelets, p.levels, p.sigma = n_wavelets, levels, sigma
        if max_active_voxels:
            p.max_active_voxels = int(max_active_voxels)
        h = ctypes.c_void_p()
        st = stream if stream is not None else _stream_handle()
        native.check(lib.muffin_server_create(ctypes.byref(p), st, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.muffin_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, psf, dirty, mu: float, gamma: float, iters: int) -> int:
        keep = []
        L, n = int(np.shape(dirty)[-3]), int(np.shape(dirty)[-1])
        t = ctypes.c_uint64()
        native.check(self._lib.muffin_serve_submit(
            self._h, n, L, _ptr(psf, keep), _ptr(dirty, keep), float(mu), float(gamma),
            int(iters), ctypes.byref(t)))
        return int(t.value)

    def step(self):
        a, q = ctypes.c_int32(), ctypes.c_int32()
        native.check(self._lib.muffin_serve_step(self._h, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def poll(self, ticket: int, out=None) -> bool:
        keep, d = [], ctypes.c_int32()
        native.check(self._lib.muffin_serve_poll(self._h, ctypes.c_uint64(ticket),
                                                 ctypes.byref(d), _ptr(out, keep)))
        return bool(d.value)

    def stats(self):
        b, p = ctypes.c_size_t(), ctypes.c_int32()
        native.check(self._lib.muffin_server_stats(self._h, ctypes.byref(b), ctypes.byref(p)))
        return int(b.value), int(p.value)
