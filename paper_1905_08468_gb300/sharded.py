"""Band-sharded MUFFIN over several GPUs (one process per GPU).

Sec. 2.3 distributes an iteration of Algorithm 2 over nodes: the per-band
work (gradient, spatial synthesis, primal prox, spatial analysis and the
dual update of U: eqs. grad2 .. stpu) on slaves that own bands, and the
per-pixel spectral work (eqs. vt, v, upt) on a master that gathers every
band of every pixel.  Here every rank is both: rank r owns a contiguous
block of bands for the spatial half and a contiguous block of pixels for the
spectral half, and the gather/scatter of the paper becomes two all-to-all
exchanges per iteration:

    z = 2 x~ - x    [bands of r][all pixels]  ->  [all bands][pixels of r]
    t               [all bands][pixels of r]  ->  [bands of r][all pixels]

The primal step tau comes from the whole cube's step condition (Sec. 2.2):
beta = max_l ||H_l||^2 is an all-reduce (max) over the ranks' bands.

This module is the data plane (partitions, exchanges, the iteration loop).
The compute is a backend object with the calls ``lipschitz()``,
``spatial(t_band, mu, gamma, tau) -> z_band``, ``spectral(z_pix, p0, gamma)
-> t_pix`` and ``x()``; :class:`GpuBackend` binds them to the library's
``muffin_shard_spatial`` / ``muffin_shard_spectral``.  Weights alpha_n,
beta_l are all ones (the workloads' setting).  The exchanges run on
torch.distributed: NCCL with CUDA tensors, or gloo with host tensors.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import native


def band_ranges(L: int, P: int):
    """Contiguous, balanced band blocks [l0, l1) of the P ranks."""
    edges = [(L * r) // P for r in range(P + 1)]
    return [(edges[r], edges[r + 1]) for r in range(P)]


def pixel_ranges(N: int, P: int):
    """Contiguous pixel blocks [p0, p1) whose sizes are multiples of 4 (the
    spectral kernels read 16-byte groups); the last block takes the rest."""
    if N % 4:
        raise ValueError("the pixel count must be a multiple of 4")
    q = N // 4
    edges = [4 * ((q * r) // P) for r in range(P + 1)]
    return [(edges[r], edges[r + 1]) for r in range(P)]


def step_tau(beta: float, L: int, N: int, mu: float, gamma: float, K: int,
             sigma: float = 10.0, safety: float = 0.99) -> float:
    """tau of the step condition (Sec. 2.2, the paper's sum form) with unit
    weights: safety / (beta/2 + sigma (K L mu^2 + N gamma^2))."""
    return safety / (0.5 * beta + sigma * (K * mu * mu * L + gamma * gamma * N))


class BandShardedSolver:
    """Plain MUFFIN (Algorithm 2, fixed mu, gamma) sharded by bands.

    ``dist`` is ``torch.distributed`` with an initialised process group;
    ``backend`` computes this rank's halves; ``host_exchange`` moves the
    exchanged arrays through host memory (gloo)."""

    def __init__(self, dist, backend, n: int, L: int, K: int, sigma: float = 10.0,
                 safety: float = 0.99, host_exchange: bool = False):
        import torch
        self.torch, self.dist, self.be = torch, dist, backend
        self.n, self.L, self.N, self.K = n, L, n * n, K
        self.P, self.r = dist.get_world_size(), dist.get_rank()
        self.bands = band_ranges(L, self.P)
        self.pix = pixel_ranges(self.N, self.P)
        self.l0, self.l1 = self.bands[self.r]
        self.p0, self.p1 = self.pix[self.r]
        self.sigma, self.safety, self.host = sigma, safety, host_exchange
        b = torch.tensor([float(backend.lipschitz())], dtype=torch.float64)
        dist.all_reduce(b, op=dist.ReduceOp.MAX)
        self.beta = float(b.item())

    def tau(self, mu: float, gamma: float) -> float:
        return step_tau(self.beta, self.L, self.N, mu, gamma, self.K, self.sigma, self.safety)

    def _a2a(self, send, out, send_sizes, recv_sizes):
        t = self.torch
        if self.host:
            s, o = send.cpu(), t.empty(out.shape, dtype=out.dtype)
            self.dist.all_to_all_single(o, s, recv_sizes, send_sizes)
            out.copy_(o)
        else:
            self.dist.all_to_all_single(out, send, recv_sizes, send_sizes)
        return out

    def bands_to_pixels(self, z_band):
        """[Lr][N] on this rank -> [L][Np] (every band of this rank's pixels)."""
        t = self.torch
        Lr = self.l1 - self.l0
        z = z_band.reshape(Lr, self.N)
        send = t.cat([z[:, p0:p1].reshape(-1) for p0, p1 in self.pix])
        np_ = self.p1 - self.p0
        out = t.empty(self.L * np_, dtype=z.dtype, device=z.device)
        self._a2a(send, out, [Lr * (p1 - p0) for p0, p1 in self.pix],
                  [(l1 - l0) * np_ for l0, l1 in self.bands])
        return out.reshape(self.L, np_)

    def pixels_to_bands(self, t_pix):
        """[L][Np] on this rank -> [Lr][N] (this rank's bands, every pixel)."""
        t = self.torch
        Lr = self.l1 - self.l0
        np_ = self.p1 - self.p0
        send = t.cat([t_pix[l0:l1].reshape(-1) for l0, l1 in self.bands])
        out = t.empty(Lr * self.N, dtype=t_pix.dtype, device=t_pix.device)
        self._a2a(send, out, [(l1 - l0) * np_ for l0, l1 in self.bands],
                  [Lr * (p1 - p0) for p0, p1 in self.pix])
        parts = []
        off = 0
        for p0, p1 in self.pix:
            sz = Lr * (p1 - p0)
            parts.append(out[off: off + sz].reshape(Lr, p1 - p0))
            off += sz
        return t.cat(parts, dim=1).reshape(Lr, self.n, self.n)

    def solve(self, iters: int, mu: float, gamma: float):
        """`iters` iterations from the backend's started state; returns this
        rank's bands of X."""
        tau = self.tau(mu, gamma)
        t_band = self.be.zeros_band()
        for _ in range(iters):
            z_band = self.be.spatial(t_band, mu, gamma, tau)
            z_pix = self.bands_to_pixels(z_band)
            t_pix = self.be.spectral(z_pix, self.p0, gamma)
            t_band = self.pixels_to_bands(t_pix)
        return self.be.x()


class GpuBackend:
    """This rank's halves on the GPU: a plan of its bands for the spatial
    half (started by a zero-iteration solve) and a plan of every band for
    the spectral half of its pixel block."""

    def __init__(self, pkg, torch, n: int, L: int, l0: int, l1: int, p0: int, p1: int,
                 psf_bands, dirty_bands, x0_bands=None, n_wavelets: int = 8,
                 levels: int = 3, sigma: float = 10.0):
        self.torch, self.pkg = torch, pkg
        self.n, self.L, self.Lr = n, L, l1 - l0
        dev = torch.device("cuda")
        self.spat = pkg.Plan(n, self.Lr, psf_bands, n_wavelets=n_wavelets, levels=levels,
                             sigma=sigma)
        ident = np.zeros((L, n, n), np.float32)
        ident[:, 0, 0] = 1.0
        self.spec = pkg.Plan(n, L, ident, n_wavelets=1, levels=0, sigma=sigma)
        self.x_dev = torch.zeros((self.Lr, n, n), device=dev) if x0_bands is None else \
            torch.as_tensor(np.ascontiguousarray(x0_bands, np.float32)).to(dev)
        self.dirty = torch.as_tensor(np.ascontiguousarray(dirty_bands, np.float32)).to(dev)
        self.spat.solve(self.dirty, self.x_dev, 0, 0.0, 0.0)       # start the state
        np_ = p1 - p0
        self.v = torch.zeros((L, np_), device=dev)
        self.t = torch.empty((L, np_), device=dev)
        self.z = torch.empty((self.Lr, n, n), device=dev)
        self._lib = pkg.library()

    def lipschitz(self) -> float:
        return float(self.spat.lipschitz)

    def zeros_band(self):
        return self.torch.zeros((self.Lr, self.n, self.n), device="cuda")

    def spatial(self, t_band, mu, gamma, tau):
        t_band = t_band.contiguous()
        native.check(self._lib.muffin_shard_spatial(
            self.spat._h, ctypes.c_void_p(t_band.data_ptr()), ctypes.c_void_p(self.z.data_ptr()),
            float(mu), float(gamma), float(tau)))
        return self.z

    def spectral(self, z_pix, p0, gamma):
        z_pix = z_pix.contiguous()
        native.check(self._lib.muffin_shard_spectral(
            self.spec._h, ctypes.c_void_p(z_pix.data_ptr()), ctypes.c_void_p(self.v.data_ptr()),
            ctypes.c_void_p(self.t.data_ptr()), int(p0), int(z_pix.shape[1]), float(gamma)))
        return self.t

    def x(self):
        """This rank's bands of X (a host copy of the spatial plan's state)."""
        out = np.empty((self.Lr, self.n, self.n), np.float32)
        st = self.spat.state_arrays()
        out[...] = st["x"][0, 0]
        return out
