"""Discrete adjoint of the forward model: gradient of a detector misfit w.r.t. mu_a, mu_s.

The paper names inverse problems only as future work (§4); it has no adjoint.  This is
the exact reverse-mode derivative of the discrete scheme in ``solver`` (Eqs. 9, 10, 12
with the readings listed there), FP64, with every level stored (small grids only).

Forward step n, per voxel v and direction d (x = mu_t ds_d; T, b0, b1 of Eq. 9):
    Q_n = T I_up + b0 S_up         (I_up, S_up: upwind values at the retarded time)
    S_n = a P (Q_n + b1 o S_n)     (fixed point of the source iteration, a = mu_s/mu_t)
    I_n = Q_n + b1 o S_n
    E[k, bin(n)] += sum_{v,d} W_k(v, d) I_n(v, d)
Backward step n (adjoints Ibar_n, Sbar_n collect every later use of level n):
    Ibar_n += sum_k G[k, bin(n)] W_k          (G = dL/dE)
    Sbar_tot = Sbar_n + b1 o Ibar_n
    y = a P (Sbar_tot + b1 o y)               (transposed scattering: P is symmetric, so
    z = Sbar_tot + b1 o y                      it has the forward iteration's form)
    Qbar = Ibar_n + y
    dL/da   += z . (P I_n)      dL/db1 += S_n o Qbar
    dL/dT   += Qbar o I_up      dL/db0 += Qbar o S_up
    Ibar, Sbar of the upwind samples at levels n-m, n-m-1 += (1-f, f) x (T, b0) Qbar
and dT/dx = -T, db0/dx = (T (1 + x + x^2) - 1) / x^2, db1/dx = b0 / x,
dx/dmu_t = ds_d, mu_t = mu_a + mu_s, a = mu_s / mu_t.  The warm start of the iteration
does not change the fixed point and has no adjoint.  With index interfaces, Q is
multiplied by the (fixed) split F, so Qbar picks up F^T before the upwind push.
"""
import numpy as np

from . import RING_DEPTH
from .solver import Solver, _retarded, source_iteration, step_bin


def ray_weight_derivatives(x):
    """dT/dx, db0/dx, db1/dx (series for small x, where the closed forms cancel)."""
    x = np.asarray(x, dtype=np.float64)
    T = np.exp(-x)
    small = x < 1e-2
    xs = np.where(small, 1.0, x)
    dT = -T
    db0 = np.where(small, 0.5 - 2 * x / 3 + 3 * x**2 / 8 - 2 * x**3 / 15 + 5 * x**4 / 144,
                   (T * (1.0 + xs + xs * xs) - 1.0) / (xs * xs))
    db1 = np.where(small, 0.5 - x / 3 + x**2 / 8 - x**3 / 30 + x**4 / 144,
                   (1.0 - (1.0 + xs) * T) / (xs * xs))
    return dT, db0, db1


class StoringSolver(Solver):
    """Forward solver that keeps every level (I, S, I_up, S_up) for the adjoint."""

    def __init__(self, prob):
        super().__init__(prob)
        self.all_I, self.all_S, self.all_Iup, self.all_Sup = [], [], [], []

    def _hist(self, which, lev, d, u):
        arr = self.all_I if which == "I" else self.all_S
        out = np.zeros(np.shape(lev))
        for L in np.unique(lev):
            if L < 0:
                continue
            mk = lev == L
            out[mk] = arr[L][d[mk], u[mk]]
        return out

    def step(self):
        m, seg, n = self.m, self.seg, self.n
        I_up = _retarded(self._hist, seg, n, "I", m)
        S_up = _retarded(self._hist, seg, n, "S", m)
        Q = I_up * seg["T"] + S_up * seg["b0"]
        if m.interfaces:
            from .fresnel import apply_interfaces
            apply_interfaces(m.interfaces, Q)
        S_prev = self.all_S[n - 1] if n > 0 else np.zeros((m.na, m.nv))
        S, iters = source_iteration(m, Q, seg["b1"], S_prev, m.albedo, np.max(np.abs(S_prev)))
        I = Q + seg["b1"] * S
        self.all_I.append(I)
        self.all_S.append(S)
        self.all_Iup.append(I_up)
        self.all_Sup.append(S_up)
        self.I[n % RING_DEPTH] = I
        self.S[n % RING_DEPTH] = S
        self.iters_max.append(int(iters.max()))
        self.iters_mean.append(float(iters.mean()))
        self._tally(I, n)
        self.n += 1


def transpose_interfaces(ops, Qbar):
    """F^T Qbar at every interface voxel (F is the split that ``apply_interfaces`` applies:
    a crossing direction j gives its value to the (d, w) entries and keeps nothing)."""
    out = Qbar.copy()
    for v, cols in ops.items():
        q = Qbar[:, v]
        for j, outs in cols.items():
            out[j, v] = sum(wgt * q[d] for d, wgt in outs)
    return out


def misfit(det, det_obs):
    """Least-squares detector misfit 1/2 sum (E - E_obs)^2 and its gradient dL/dE."""
    r = det - det_obs
    return 0.5 * float(np.sum(r * r)), r


def gradient(prob, nsteps, det_obs):
    """(L, dL/dmu_a, dL/dmu_s) for the misfit against ``det_obs`` after ``nsteps`` steps.

    Gradients are per voxel, flat [N_v]; the problem's own tolerance ends both the forward
    and the transposed iterations, so a tight ``tol`` gives the exact gradient.  Voxels
    with mu_t = 0 have no albedo and get the transport term only."""
    fwd = StoringSolver(prob)
    fwd.run(nsteps)
    m, seg = fwd.m, fwd.seg
    L, G = misfit(fwd.det, det_obs)
    na, nv = m.na, m.nv
    up, mlev, f = seg["up"], seg["m"], seg["f"]
    T, b0, b1 = seg["T"], seg["b0"], seg["b1"]
    x = m.mut[None, :] * m.lat.ds[:, None]
    dT, db0, db1 = ray_weight_derivatives(x)
    Ibar = [np.zeros((na, nv)) for _ in range(nsteps)]
    Sbar = [np.zeros((na, nv)) for _ in range(nsteps)]
    g_x = np.zeros((na, nv))   # dL/dx summed over steps
    g_a = np.zeros(nv)         # dL/da
    h2dt = m.h * m.h * m.dt
    dd = np.arange(na)[:, None] * np.ones_like(up)
    inside = up >= 0
    for n in range(nsteps - 1, -1, -1):
        b = step_bin(n, m.dt, m.bin_width)
        if b < m.nbins:
            for k, det in enumerate(m.dets):
                cols = np.broadcast_to(det["voxels"][None, :], (na, det["voxels"].size))
                rows = np.broadcast_to(np.arange(na)[:, None], cols.shape)
                np.add.at(Ibar[n], (rows, cols),
                          G[k, b] * h2dt * np.broadcast_to(det["weight"][:, None], cols.shape))
        S_tot = Sbar[n] + b1 * Ibar[n]
        y, _ = source_iteration(m, S_tot, b1, np.zeros((na, nv)), m.albedo, 0.0)
        z = S_tot + b1 * y
        Qbar = Ibar[n] + y
        I_n, S_n = fwd.all_I[n], fwd.all_S[n]
        PI = m.P @ I_n
        g_a += np.sum(z * PI, axis=0)
        Qpre = transpose_interfaces(m.interfaces, Qbar) if m.interfaces else Qbar
        g_x += Qpre * (dT * fwd.all_Iup[n] + db0 * fwd.all_Sup[n]) + S_n * Qbar * db1
        for ell, wgt in ((0, 1.0 - f), (1, f)):
            lev = n - mlev - ell
            ok = inside & (lev >= 0)
            for L_ in np.unique(lev[ok]):
                mk = ok & (lev == L_)
                np.add.at(Ibar[L_], (dd[mk], up[mk]), (wgt * T * Qpre)[mk])
                np.add.at(Sbar[L_], (dd[mk], up[mk]), (wgt * b0 * Qpre)[mk])
    g_mut = np.sum(g_x * m.lat.ds[:, None], axis=0)
    mua, mus, mut = m.mua, m.mut - m.mua, m.mut
    safe = mut > 0
    da_dmua = np.where(safe, -mus / np.where(safe, mut * mut, 1.0), 0.0)
    da_dmus = np.where(safe, mua / np.where(safe, mut * mut, 1.0), 0.0)
    return L, g_mut + g_a * da_dmua, g_mut + g_a * da_dmus, fwd.det
