"""FP8 scatter variant, tried on the CPU and rejected: its error against the FP64 oracle.

The BF16-scatter kernel carries the iterate X = Q + b1 S as two BF16 terms (hi, lo) and
multiplies them by bf16(P) with FP32 accumulation.  The FP8 variant replaces the X terms
by E4M3 terms (3 mantissa bits), each with its own per-voxel scale (the largest |value|
of the voxel's term maps to 448, the largest finite E4M3), and keeps P in BF16 (an FP8 P
would perturb the discrete phase function itself).  Everything else is the kernel's
arithmetic: the diagonal row-sum correction r X, S = (1 - eps) Y, the isotropic
rebalance, the stop rule with its stall exit.

This module emulates both on the CPU (numpy; rounding to BF16 / E4M3 written out below)
on a 10^3 box with the small workload's optics and 48 directions, and states their
detector-curve error against the FP64 oracle in relative L2 norm (the BF16-scatter bar is
1e-3).  Measured here: BF16 x 2 terms 1.2e-4; E4M3 x 2 terms 4.2e-3; E4M3 x 3 terms
1.5e-4.  Two FP8 terms leave ~1e-3 relative noise in every product (the 3-bit mantissa of
the second term), which the slow contraction (1 / (1 - a b1) ~ 14) amplifies past the
bar; three terms match BF16.  Three FP8 MMAs at twice the BF16 rate take 3/4 of the
tensor time of two BF16 MMAs, but the BF16 kernel is bound by its epilogue, not by the
tensor pipe, and splitting X into three scaled E4M3 terms adds epilogue work, so the
variant is not built.
"""
import numpy as np
import pytest

import workloads as W
from oracle.solver import Solver, _retarded


def round_bf16(x):
    """Round to the nearest BF16 value (8-bit mantissa, ties to even), as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def round_e4m3(x):
    """Round to the nearest OCP FP8 E4M3 value (3-bit mantissa, exponent bias 7, smallest
    normal 2^-6, subnormal spacing 2^-9, saturating at 448), ties to even, as float64."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, ex = np.frexp(np.where(a > 0, a, 1.0))
    e = np.maximum(ex - 1, -6)            # binade of the leading bit (normals), or the subnormal one
    step = np.ldexp(1.0, e - 3)           # spacing of 3 mantissa bits in that binade
    q = np.minimum(np.round(a / step) * step, 448.0)  # np.round ties to even
    return np.where(a > 0, np.sign(x) * q, 0.0)


def split_terms(X, kind, nterms):
    """X ([N_a, voxels]) as a sum of ``nterms`` low-precision terms.  BF16: hi = bf16(X),
    lo = bf16(X - hi).  E4M3: each term carries its own per-voxel scale (max |residual| of
    the voxel mapped to 448)."""
    terms = []
    R = X.copy()
    for _ in range(nterms):
        if kind == "bf16":
            t = round_bf16(R)
        else:
            m = np.max(np.abs(R), axis=0)
            s = np.where(m > 0, m / 448.0, 1.0)
            t = round_e4m3(R / s[None, :]) * s[None, :]
        terms.append(t)
        R = R - t
    return terms


class LowPrecisionScatter(Solver):
    """The oracle's time loop with the tensor-core kernel's source iteration, its operands
    rounded as the hardware would (products and sums in float64: FP32 accumulation of
    exactly representable products is not what limits the error here)."""

    def __init__(self, prob, kind, nterms):
        super().__init__(prob)
        self.kind, self.nterms = kind, nterms
        Pb = round_bf16(self.m.P)
        self.Pb = Pb
        self.r = 1.0 - Pb.sum(axis=1)

    def step(self):
        m, seg, n = self.m, self.seg, self.n
        I_up = _retarded(self._hist, seg, n, "I", m)
        S_up = _retarded(self._hist, seg, n, "S", m)
        Q = I_up * seg["T"] + S_up * seg["b0"]
        b1 = seg["b1"]
        a = m.albedo
        S = self.S[(n - 1) % 5].copy() if n > 0 else np.zeros((m.na, m.nv))
        sglob = np.abs(S).max()
        rho = a * b1.max(axis=0)
        den = m.na - a * b1.sum(axis=0)
        act = np.arange(m.nv)
        best = np.full(m.nv, np.inf)
        stall = np.zeros(m.nv, dtype=np.int64)
        for _ in range(m.max_iters):
            if act.size == 0:
                break
            Sa = S[:, act]
            X = Q[:, act] + b1[:, act] * Sa
            Y = sum(self.Pb @ t for t in split_terms(X, self.kind, self.nterms)) + self.r[:, None] * X
            Sh = a[None, act] * Y
            dl = Sh - Sa
            D = np.abs(dl).max(axis=0)
            Sm = np.abs(Sh).max(axis=0)
            imp = D < best[act]
            best[act] = np.where(imp, D, best[act])
            stall[act] = np.where(imp, 0, stall[act] + 1)
            r = rho[act]
            done = (r / (1 - r)) * D <= m.tol * np.maximum(Sm, 1e-6 * sglob)
            done |= stall[act] >= 3
            c = np.where(done, 0.0, a[act] * np.sum(b1[:, act] * dl, axis=0) / den[act])
            S[:, act] = Sh + c[None, :]
            act = act[~done]
        I = Q + b1 * S
        self.I[n % 5] = I
        self.S[n % 5] = S
        self._tally(I, n)
        self.n += 1


@pytest.fixture(scope="module")
def emulated():
    prob = W.homogeneous(10, 10, 10, 2, 0.01, 10.0, steps=40, tol=1e-6)
    prob["source"] = dict(face=4, u_mm=5.0, v_mm=5.0, half_angle_deg=15.0, pulse_steps=1, energy=1.0)
    prob["detectors"] = [dict(face=4, u_mm=5.5 + s, v_mm=5.5, radius_mm=0.5, half_angle_deg=15.0)
                         for s in (2.0, 3.0)]
    prob["nbins"] = 12
    ref = Solver(dict(prob, tol=1e-10))
    ref.run(40)
    out = {}
    for kind, nt in (("bf16", 2), ("e4m3", 2), ("e4m3", 3)):
        s = LowPrecisionScatter(prob, kind, nt)
        s.run(40)
        out[(kind, nt)] = float(np.linalg.norm(s.det - ref.det) / np.linalg.norm(ref.det))
    return out


def test_rounding_helpers():
    assert round_e4m3(np.array([448.0, 500.0, 1.0, 1.0625, 1.0626, 2.0 ** -9, 0.0])).tolist() == \
        [448.0, 448.0, 1.0, 1.0, 1.125, 2.0 ** -9, 0.0]
    assert round_e4m3(np.array([-3.3]))[0] == -3.25
    assert round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert round_bf16(np.array([1.0 + 3 * 2.0 ** -9]))[0] == 1.0 + 2.0 ** -7


def test_fp8_scatter_misses_the_bf16_bar(emulated):
    bf16, fp8x2, fp8x3 = emulated[("bf16", 2)], emulated[("e4m3", 2)], emulated[("e4m3", 3)]
    print("detector rel L2 vs FP64 oracle: bf16x2 %.2e  e4m3x2 %.2e  e4m3x3 %.2e" % (bf16, fp8x2, fp8x3))
    assert bf16 <= 1e-3            # the built BF16-scatter form meets its bar
    assert fp8x2 > 1e-3            # two FP8 terms do not
    assert fp8x3 < fp8x2           # a third term helps but costs a third MMA
