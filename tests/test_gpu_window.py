"""The benched kernels against the oracle at full size, inside the developed solve.

The bench times the 96x96x64 slab around step 620 and the 128x128x96 phantom after its
spin-up.  At these sizes the FP64 oracle cannot run the whole solve, but every value of
level n of a voxel depends only on the stored levels n-4 .. n-1 and on that voxel's own
source iteration: the oracle recomputes level n at sampled voxels from the GPU's own
stored history (one step of Eq. 10, the interface split, the source iteration converged
to 1e-10) and the two are compared element by element.  Voxels are drawn at random over
the glow (every voxel whose brightest direction exceeds 1e-4 of the field's peak), plus
the source voxel and, on the phantom, voxels on the air cylinder's wall and inside the
absorbing spheres.

Bars, per element against the field's peak: FP32 1e-5 (the FP32 bar); BF16-scatter 1e-3
(the BF16 mode's bar; one step of the two-term BF16 product is far inside it).  The
phantom runs through the general per-voxel kernel forms (mu_t and n vary), the slab
through the uniform-medium instances.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
BAR = {"fp32": 1e-5, "bf16": 1e-3}


def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2105_01028_gb300 as P
    return P


def _run_and_check(prob, steps, extra_vox, seed, n_sample=256):
    P = _lib()
    from oracle.solver import Model, one_step_at
    fw = P.Forward(prob)
    fw.run(steps)
    fw.sync()
    n = steps - 1
    hist = {}
    for back in range(1, 5):
        hist[n - back] = (fw.field(P.FIELD_I, back), fw.field(P.FIELD_S, back))
    I_n, S_n = fw.field(P.FIELD_I, 0), fw.field(P.FIELD_S, 0)
    fw.close()

    glow = np.nonzero(np.abs(I_n).max(axis=0) > 1e-4 * np.abs(I_n).max())[0]
    rng = np.random.default_rng(seed)
    vox = set(int(v) for v in rng.choice(glow, min(n_sample, glow.size), replace=False))
    vox |= set(int(v) for v in extra_vox)
    vox = np.array(sorted(vox))

    def h(which, lev, d, u):
        out = np.zeros(np.shape(lev))
        for L, (Ia, Sa) in hist.items():
            m = lev == L
            if np.any(m):
                out[m] = (Ia if which == "I" else Sa)[d[m], u[m]]
        return out

    s_glob = float(np.abs(hist[n - 1][1]).max())
    p = dict(prob, tol=1e-10, max_iters=20000)
    I_ref, S_ref, _ = one_step_at(Model(p), n, h, vox, s_glob)
    bar = BAR[prob["precision"]]
    eI = np.abs(I_n[:, vox] - I_ref).max() / np.abs(I_n).max()
    eS = np.abs(S_n[:, vox] - S_ref).max() / np.abs(S_n).max()
    assert eI <= bar, eI
    assert eS <= bar, eS
    return glow.size, eI, eS


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_slab_at_the_benched_window(precision):
    """The bench's slab at step 620 (its timed window is steps 603..632)."""
    prob = W.config_slab(steps=620, precision=precision)
    nx, ny = prob["nx"], prob["ny"]
    src = (0 * ny + ny // 2) * nx + nx // 2
    nglow, eI, eS = _run_and_check(prob, 620, [src], seed=11)
    assert nglow > 100000  # the light fills much of the slab by then


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_phantom_after_spin_up(precision):
    """The 128x128x96 phantom (air cylinder with refraction and reflection at its wall,
    three absorbing spheres) after 200 steps, when light has reached the cylinder."""
    prob = W.config_hetero(steps=200, precision=precision)
    nz, ny, nx = prob["nz"], prob["ny"], prob["nx"]
    extra = [(nz // 2 * ny + ny // 2) * nx + 0]
    cyl = prob["cylinder"]
    rng = np.random.default_rng(6)
    for k in range(24):  # just outside and inside the cylinder wall, at the source's height
        rr = cyl["radius"] + (0.6 if k % 2 else -0.6)
        x = int(cyl["center"][0] + rr * np.cos(0.5 * k))
        y = int(cyl["center"][1] + rr * np.sin(0.5 * k))
        z = int(nz // 2 + rng.integers(-8, 9))
        extra.append((z * ny + y) * nx + x)
    for c, r, _ in prob["spheres"]:
        extra.append((int(c[2]) * ny + int(c[1])) * nx + int(c[0]))
    _run_and_check(prob, 200, extra, seed=12)
