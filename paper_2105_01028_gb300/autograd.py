"""Detector curves as a differentiable function of the optical maps (PyTorch autograd).

``detector_curves(mua, mus, prob, nsteps)`` runs the forward model with checkpoints and
returns the FP64 detector curves [n_det, nbins]; its backward pass calls the library's
adjoint (include/trinity.h, ``trinity_adjoint``), so ``loss.backward()`` yields dL/dmu_a
and dL/dmu_s per voxel.  The gradient is the exact derivative of the discrete scheme
(Eqs. 9, 10, 12-14); the paper itself has no adjoint (Section 4 names inverse problems
as future work).  Everything runs in the library on the current CUDA device; this module
only moves tensors.
"""
import numpy as np
import torch

from . import Forward


class _DetectorCurves(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mua, mus, prob, nsteps, every):
        shape = (prob["nz"], prob["ny"], prob["nx"])
        if tuple(mua.shape) != shape or tuple(mus.shape) != shape:
            raise ValueError("mua and mus must have shape (nz, ny, nx)")
        p = dict(prob)
        p["mua"] = mua.detach().to(torch.float32).contiguous()
        p["mus"] = mus.detach().to(torch.float32).contiguous()
        nid = prob["nidx"]
        if p["mua"].is_cuda:
            p["nidx"] = torch.as_tensor(np.asarray(nid, dtype=np.float32)).to(p["mua"].device)
        else:
            p["mua"], p["mus"] = p["mua"].numpy(), p["mus"].numpy()
        fw = Forward(p)
        fw.run_checkpointed(int(nsteps), int(every))
        ctx.fw = fw
        ctx.shape = shape
        ctx.meta = (mua.dtype, mua.device, mus.dtype, mus.device)
        return torch.as_tensor(fw.detectors(), dtype=torch.float64, device=mua.device)

    @staticmethod
    def backward(ctx, gE):
        fw = ctx.fw
        ga, gs = fw.adjoint(gE.detach().to(torch.float64).cpu().numpy())
        fw.close()
        da, dva, ds, dvs = ctx.meta
        ga = torch.as_tensor(ga.reshape(ctx.shape), device=dva).to(da)
        gs = torch.as_tensor(gs.reshape(ctx.shape), device=dvs).to(ds)
        return ga, gs, None, None, None


def detector_curves(mua, mus, prob, nsteps, every=50):
    """FP64 detector curves [n_det, nbins] after ``nsteps`` steps of ``prob`` with the
    absorption and scattering maps ``mua``, ``mus`` (tensors of shape (nz, ny, nx))."""
    return _DetectorCurves.apply(mua, mus, prob, nsteps, every)
