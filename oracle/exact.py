"""Exact per-voxel source function for piecewise-uniform optics.

Test infrastructure (like the rest of ``oracle``): only tests and the benchmark's CPU
legs use it.

The source iteration (Eq. 12, §2.4 steps 5-6) converges to the fixed point of
S = a P (Q + b1 o S).  Every voxel's system is independent within a step, and it
depends on the voxel only through its optics (mu_t fixes b1 per direction, mu_s / mu_t
fixes a).  Voxels that share (mu_t, a) share the operator
    M = (I - a P B1)^-1 a P,       B1 = diag(b1(mu_t ds_d)),
so S = M Q in one product.  This is the limit the paper's iteration approaches, reached
directly; it applies where the optics take few distinct values (a homogeneous slab: one
class; a phantom of uniform inclusions: a handful).
"""
import numpy as np

from . import RING_DEPTH
from .fresnel import apply_interfaces
from .solver import Solver, _retarded, ray_weights


def optics_classes(model):
    """(class index per voxel, list of (mu_t, albedo)) for the distinct optics pairs."""
    key = np.stack([model.mut, model.albedo], axis=1)
    uniq, inv = np.unique(key, axis=0, return_inverse=True)
    return inv.ravel(), [tuple(u) for u in uniq]


def exact_operator(P, albedo, b1):
    """M = (I - a P diag(b1))^-1 a P by a library linear solve (FP64)."""
    na = P.shape[0]
    A = np.eye(na) - albedo * P * b1[None, :]
    return np.linalg.solve(A, albedo * P)


class ExactSolver(Solver):
    """The forward model with S = M_class Q in place of the source iteration."""

    def __init__(self, prob):
        super().__init__(prob)
        m = self.m
        self.cls, pairs = optics_classes(m)
        self.M = []
        for mut, a in pairs:
            _, _, b1 = ray_weights(mut * m.lat.ds)
            self.M.append(exact_operator(m.P, a, b1))

    def step(self):
        m, seg, n = self.m, self.seg, self.n
        I_up = _retarded(self._hist, seg, n, "I", m)
        S_up = _retarded(self._hist, seg, n, "S", m)
        Q = I_up * seg["T"] + S_up * seg["b0"]
        if m.interfaces:
            apply_interfaces(m.interfaces, Q)
        S = np.zeros_like(Q)
        for c, M in enumerate(self.M):
            sel = self.cls == c
            S[:, sel] = M @ Q[:, sel]
        I = Q + seg["b1"] * S
        self.I[n % RING_DEPTH] = I
        self.S[n % RING_DEPTH] = S
        self.iters_max.append(1)
        self.iters_mean.append(1.0)
        self._tally(I, n)
        self.n += 1
