"""Seeded synthetic inputs for MUFFIN multispectral deconvolution.

This package is the one module shared by the FP64 CPU oracle and the CUDA
path.  It draws skies, PSFs, dirty cubes, noise variances and the FDMC probe
vector from one seed; it holds none of the deconvolution method's arithmetic
(no gradient, wavelet, DCT, proximal, derivative or risk-estimate step).
"""
from .generator import (Cube, VisCube, WORKLOADS, make_cube, make_visibilities,
                        make_workload, fdmc_eps, serve_stream)

__all__ = ["Cube", "VisCube", "WORKLOADS", "make_cube", "make_visibilities",
           "make_workload", "fdmc_eps", "serve_stream"]
