"""Two-level angular grid: transport on fine directions, source function on coarse ones.

Test infrastructure (like the rest of ``oracle``): only tests and the benchmark's CPU
legs use it.

§2.1 (text after Eq. 12): the paper's fiducial runs carry the radiative transfer on 3072
HEALPix directions (N_side 16) and evaluate the source function on 192 (N_side 4), each
coarse bin using the mean intensity of its 16 finer bins.  Per step, with ch(c) the
children of coarse direction c and par(f) the parent of fine direction f:

    Q_f  = I_up,f T_f + S_up,par(f) b0_f           (Eq. 10; S lives on the coarse grid)
    S_c  = a sum_c' P_cc' mean_{f in ch(c')} I_f,   I_f = Q_f + b1_f S_par(f)
so the coarse system is S_c = a P (Qbar + b1bar o S)_c with Qbar_c and b1bar_c the means
of Q_f and b1_f over ch(c): the one-level source iteration on coarse arrays.  Then
I_f = Q_f + b1_f S_par(f).  Energy and detectors use the fine I (weights 4 pi / N_fine).
"""
import numpy as np

from . import RING_DEPTH
from .fresnel import apply_interfaces
from .healpix import parent_map
from .solver import Solver, _retarded, source_iteration


class TwoLevelSolver(Solver):
    """``prob["nside"]`` is the transport grid, ``prob["nside_scatter"]`` the coarse one."""

    def __init__(self, prob):
        super().__init__(prob)
        m = self.m
        self.parent = parent_map(int(prob["nside"]), m.nside_s)
        self.nc = 12 * m.nside_s ** 2
        self.S = np.zeros((RING_DEPTH, self.nc, m.nv))
        counts = np.bincount(self.parent, minlength=self.nc)
        if np.any(counts != counts[0]):
            raise ValueError("every coarse direction needs the same number of children")
        self.nchild = int(counts[0])

    def _hist(self, which, lev, d, u):
        if which == "I":
            return self.I[lev % RING_DEPTH, d, u] * (lev >= self.hist_from)
        return self.S[lev % RING_DEPTH, self.parent[d], u] * (lev >= self.hist_from)

    def coarse_mean(self, X):
        """Mean over each coarse direction's children: [N_fine, n] -> [N_coarse, n]."""
        out = np.zeros((self.nc, X.shape[1]))
        np.add.at(out, self.parent, X)
        return out / self.nchild

    def step(self):
        m, seg, n = self.m, self.seg, self.n
        I_up = _retarded(self._hist, seg, n, "I", m)
        S_up = _retarded(self._hist, seg, n, "S", m)
        Q = I_up * seg["T"] + S_up * seg["b0"]
        if m.interfaces:
            apply_interfaces(m.interfaces, Q)
        Qc = self.coarse_mean(Q)
        b1c = self.coarse_mean(seg["b1"])
        S_prev = self.S[(n - 1) % RING_DEPTH] if n > 0 else np.zeros((self.nc, m.nv))
        Sc, iters = source_iteration(m, Qc, b1c, S_prev, m.albedo, np.max(np.abs(S_prev)))
        I = Q + seg["b1"] * Sc[self.parent]
        self.I[n % RING_DEPTH] = I
        self.S[n % RING_DEPTH] = Sc
        self.iters_max.append(int(iters.max()))
        self.iters_mean.append(float(iters.mean()))
        self._tally(I, n)
        self.n += 1
