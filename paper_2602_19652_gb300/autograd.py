"""torch.autograd.Function over st_simulate / st_backward.

SpectraFn.apply(ctx, scene, params, k_band, mics, emitter[, beta_band]) returns the complex64
spectra [3][M][F] and differentiates them with respect to the reflection band values k_band
[n_mat][n_bands], the microphone positions mics [M][3], the emitter position [3] (through the
diffraction and direct paths, and through the specular hit points: ray directions and triangle chains
frozen, each hit point moving on its triangle's plane) and, when given, the lobe widths beta_band
[n_mat][n_bands] (radians), with the path set of the forward call frozen.  PyTorch passes
dL/dRe S + j dL/dIm S as the incoming gradient, which is the convention st_backward expects."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib


class SpectraFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, sim, scene, params, k_band, mics, emitter, beta_band=None):
        k_np = k_band.detach().cpu().numpy().astype(np.float32)
        b_np = scene.beta_band if beta_band is None else beta_band.detach().cpu().numpy().astype(np.float32)
        scene.set_materials(scene.band_hz, k_np, b_np, scene.diff_band)
        sim.set_receivers(mics.detach())
        e = emitter.detach().cpu().numpy().astype(np.float32)
        sim.set_emitter(e, sim.quat, sim.dirs, None, sim.fov_half)
        out = sim.simulate(scene, params)
        fctx.sim, fctx.scene = sim, scene
        fctx.shapes = (tuple(k_band.shape), tuple(mics.shape))
        fctx.devices = (k_band.device, mics.device, emitter.device,
                        None if beta_band is None else beta_band.device)
        return out

    @staticmethod
    def backward(fctx, grad_out):
        sim, scene = fctx.sim, fctx.scene
        dev = grad_out.device
        g = grad_out.contiguous().to(torch.complex64)
        need_k, need_m, need_e = fctx.needs_input_grad[3:6]
        gk = torch.zeros(fctx.shapes[0], dtype=torch.float32, device=dev) if need_k else None
        gm = torch.zeros(fctx.shapes[1], dtype=torch.float32, device=dev) if need_m else None
        ge = torch.zeros(3, dtype=torch.float32, device=dev) if need_e else None
        vp = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        if gk is not None or gm is not None or ge is not None:
            sim._check(sim.L.st_backward(sim.h, scene.h, vp(g), vp(gk), vp(gm), vp(ge)))
        gb = None
        if len(fctx.needs_input_grad) > 6 and fctx.needs_input_grad[6]:
            gb = torch.zeros(fctx.shapes[0], dtype=torch.float32, device=dev)
            sim._check(sim.L.st_backward_beta(sim.h, scene.h, vp(g), vp(gb)))
        out = [None, None, None, gk, gm, ge, gb]
        for i, d in zip((3, 4, 5, 6), fctx.devices):
            if out[i] is not None:
                out[i] = out[i].to(d)
        return tuple(out)
