"""torch.autograd wrapper of the peeled spectral cube.

``PeeledCube.apply(ctx, packets, n_HI, vx, vy, vz, T, n_dust)`` loads the leaf
fields (CUDA tensors) into the library context, propagates the packets and
returns the peeled cube [ndir, npix, npix, nbin] as a CUDA tensor.  Its
backward calls ``rascas_peel_adjoint``: the gradient of the loss with respect
to each leaf's n_HI, velocity, temperature and dust density with the
scattering record of the forward pass held fixed (the same packets are
replayed with the same random streams and fields, and only the optical depths
of the peeling rays are differentiated).  The context's fields must not change
between forward and backward.
"""
from __future__ import annotations

import torch

from . import _native as N


class PeeledCube(torch.autograd.Function):
    @staticmethod
    def forward(fctx, rctx, packets, n_HI, vx, vy, vz, T, n_dust):
        pos, dr, nu, ids = packets
        rctx.update_fields(n_HI, vx, vy, vz, T, n_dust)
        rctx.zero_tallies()
        rctx.propagate(pos, dr, nu, ids, out=None, stats=False)
        cube = rctx.get_tally(N.TALLY_PEEL_CUBES, device=nu.device)
        fctx.rctx = rctx
        fctx.packets = packets
        fctx.nleaf = int(n_HI.shape[0])
        return cube

    @staticmethod
    def backward(fctx, g_cube):
        pos, dr, nu, ids = fctx.packets
        grad = fctx.rctx.peel_adjoint(pos, dr, nu, ids, g_cube=g_cube.contiguous(), nleaf=fctx.nleaf)
        return (None, None) + tuple(grad[j] for j in range(6))
