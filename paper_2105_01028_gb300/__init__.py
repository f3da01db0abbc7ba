"""GB300-native forward model of time-dependent radiative transfer (TRINITY, arXiv:2105.01028).

The compute runs in ``libtrinity.so`` (hand-written sm_103a CUDA behind a C ABI, see
include/trinity.h).  This package is the thin Python side: ``Forward`` marshals a
problem description into the C calls and reads results back.  PyTorch is optional and
only used to pass device buffers and the current CUDA stream.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import GridDesc, TrinityError, OK, W_NOT_CONVERGED

FP32, BF16 = 0, 1
FIELD_I, FIELD_S, FIELD_U = 0, 1, 2
_PREC = {"fp32": FP32, "bf16": BF16}
_BOUND = {"vacuum": 0, "periodic": 1, "mirror": 2}

__all__ = ["Forward", "Server", "TrinityError", "grid_desc", "footprint_bytes",
           "adjoint_footprint_bytes", "healpix_dirs",
           "phase_matrix", "lattice_tables", "cone_weights", "lib"]


def lib():
    return _lib.load()


def grid_desc(prob):
    """trinity_grid_desc of a problem dict (sizes, angles, time step, precision, tolerance)."""
    return GridDesc(int(prob["nx"]), int(prob["ny"]), int(prob["nz"]), float(prob["h"]),
                    int(prob["nside"]), float(prob["courant"]), float(prob["n_ref"]),
                    _BOUND[prob.get("boundary", "vacuum")], _PREC[prob.get("precision", "fp32")],
                    float(prob.get("tol", 1e-6)), int(prob.get("max_iters", 2000)),
                    int(prob.get("nside_scatter") or 0))


def footprint_bytes(prob):
    d = grid_desc(prob)
    return int(lib().trinity_footprint_bytes(ctypes.byref(d)))


def adjoint_footprint_bytes(prob, nsteps, every=50):
    """Extra device bytes of a checkpointed run plus its adjoint."""
    d = grid_desc(prob)
    return int(lib().trinity_adjoint_footprint_bytes(ctypes.byref(d), int(nsteps), int(every),
                                                     len(prob.get("detectors", [])),
                                                     int(prob.get("nbins", 1))))


def _ptr(a):
    """(pointer, ptr_kind, keep-alive) of a numpy array (host) or a torch CUDA tensor."""
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        if not a.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), 1, a
    arr = np.ascontiguousarray(a, dtype=np.float32)
    return arr.ctypes.data_as(ctypes.c_void_p), 0, arr


class Forward:
    """One forward-model context on the current CUDA device.

    ``prob`` is a problem dict (see the ``workloads`` module for the keys).  ``stream`` is
    a raw cudaStream_t handle (int) or None for the default stream.
    """

    def __init__(self, prob, stream=None):
        self.L = lib()
        self.prob = prob
        desc = grid_desc(prob)
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream else None
        rc = self.L.trinity_create_grid(ctypes.byref(desc), st, ctypes.byref(h))
        if rc != OK:
            raise TrinityError(rc, "trinity_create_grid failed")
        self.h = h
        self.nv = desc.nx * desc.ny * desc.nz
        self.na = 12 * desc.nside * desc.nside
        ns = desc.nside_scatter or desc.nside
        self.na_s = 12 * ns * ns  # directions of S (coarser on a two-level angular grid)
        self._check(self.set_optics(prob["mua"], prob["mus"], prob["nidx"], prob["g"]))
        if prob.get("fresnel", False):
            self._check(self.L.trinity_set_fresnel(self.h, 1))
        if not prob.get("sweep_tma", True):  # the plain-load sweep (bit-identical results)
            self._check(self.L.trinity_set_sweep_tma(self.h, 0))
        warm = prob.get("warm_start", "extrapolated")  # or "previous": S(n-1) as the paper states
        if warm not in ("extrapolated", "previous"):
            raise ValueError("warm_start must be 'extrapolated' or 'previous'")
        self._check(self.L.trinity_set_warm_start(self.h, 1 if warm == "extrapolated" else 0))
        ex = prob.get("exact", False)
        if ex:  # True / "tc": tensor cores where the grid allows; "simt": FP32 SIMT form
            self._check(self.L.trinity_set_exact_solve(self.h, 2 if ex == "simt" else 1))
        src = prob.get("source")
        if src is not None:
            self._check(self.L.trinity_set_source(self.h, int(src["face"]), float(src["u_mm"]),
                                                  float(src["v_mm"]), float(src["half_angle_deg"]),
                                                  int(src["pulse_steps"]), float(src["energy"])))
        self.n_det = 0
        for det in prob.get("detectors", []):
            did = ctypes.c_int()
            self._check(self.L.trinity_add_detector(self.h, int(det["face"]), float(det["u_mm"]),
                                                    float(det["v_mm"]), float(det["radius_mm"]),
                                                    float(det["half_angle_deg"]), ctypes.byref(did)))
            self.n_det += 1
        self.nbins = int(prob.get("nbins", 1))
        self._check(self.L.trinity_set_bins(self.h, float(prob.get("bin_ps", 10.0)), self.nbins))

    # -- plumbing
    def _check(self, rc):
        if rc not in (OK, W_NOT_CONVERGED):
            raise TrinityError(rc, self.L.trinity_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.L.trinity_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- inputs
    def set_optics(self, mua, mus, nidx, g):
        pa, ka, keep_a = _ptr(mua)
        ps, ks, keep_s = _ptr(mus)
        pn, kn, keep_n = _ptr(nidx)
        if not (ka == ks == kn):
            raise ValueError("optics maps must all be host arrays or all device tensors")
        return self.L.trinity_set_optics(self.h, pa, ps, pn, float(g), ka)

    def exact_classes(self):
        """Optics classes of the exact solve (0 when it is off)."""
        n = ctypes.c_int()
        self._check(self.L.trinity_exact_classes(self.h, ctypes.byref(n)))
        return n.value

    def exact_form(self):
        """Form of the exact solve that runs: "tc" (tensor cores), "simt" (FP32 SIMT) or None."""
        f = ctypes.c_int()
        self._check(self.L.trinity_exact_form(self.h, ctypes.byref(f)))
        return {0: None, 1: "tc", 2: "simt"}[f.value]

    def interface_count(self):
        n = ctypes.c_int()
        self._check(self.L.trinity_interface_count(self.h, ctypes.byref(n)))
        return n.value

    def set_initial_state(self, I0, S0):
        pi, ki, keep_i = _ptr(I0)
        ps, ks, keep_s = _ptr(S0)
        return self._check(self.L.trinity_set_initial_state(self.h, pi, ps, ki))

    # -- stepping
    def step(self, nsteps=1):
        """Advance and return the per-step max iteration counts (synchronous)."""
        out = (ctypes.c_int * max(nsteps, 1))()
        rc = self._check(self.L.trinity_step(self.h, int(nsteps), out))
        self.last_status = rc
        return np.array(out[:nsteps], dtype=np.int64)

    def run(self, nsteps):
        """Queue ``nsteps`` steps (CUDA-graph replay); returns without waiting."""
        return self._check(self.L.trinity_run(self.h, int(nsteps)))

    def profile(self, nsteps):
        """Advance ``nsteps`` steps timing each kernel with CUDA events; returns the summed
        device ms of (sweep, source iteration, tallies)."""
        ms = np.zeros(3)
        self._check(self.L.trinity_profile_steps(self.h, int(nsteps), ms.ctypes.data_as(_lib.P_double)))
        return ms

    def sync(self):
        self.last_status = self._check(self.L.trinity_sync(self.h))
        return self.last_status

    # -- adjoint
    def run_checkpointed(self, nsteps, every=50):
        """``nsteps`` steps from step 0, saving checkpoints every ``every`` steps for
        ``adjoint`` (synchronous)."""
        self.last_status = self._check(self.L.trinity_run_checkpointed(self.h, int(nsteps), int(every)))
        return self.last_status

    def adjoint(self, dL_dE, out=None):
        """dL/dmu_a, dL/dmu_s per voxel (FP64, flat [N_v]) for the misfit whose gradient
        with respect to the detector curves is ``dL_dE`` [n_det, nbins].  With ``out`` =
        (ga, gs), two contiguous float64 CUDA tensors of N_v elements, the gradients are
        written there and dL_dE may be a CUDA tensor too."""
        if out is not None:
            ga, gs = out
            if not (getattr(ga, "is_cuda", False) and getattr(gs, "is_cuda", False)
                    and getattr(dL_dE, "is_cuda", False)):
                raise ValueError("device outputs need a device dL_dE")
            for t in (dL_dE, ga, gs):
                if not t.is_contiguous() or str(t.dtype) != "torch.float64":
                    raise ValueError("device adjoint buffers must be contiguous float64")
            self.last_status = self._check(self.L.trinity_adjoint(
                self.h, ctypes.c_void_p(dL_dE.data_ptr()), dL_dE.numel(),
                ctypes.c_void_p(ga.data_ptr()), ctypes.c_void_p(gs.data_ptr()), 1))
            return ga, gs
        G = self._grad_input(dL_dE)
        ga = np.zeros(self.nv)
        gs = np.zeros(self.nv)
        self.last_status = self._check(self.L.trinity_adjoint(
            self.h, G.ctypes.data_as(ctypes.c_void_p), G.size, ga.ctypes.data_as(ctypes.c_void_p),
            gs.ctypes.data_as(ctypes.c_void_p), 0))
        return ga, gs

    def adjoint_profile(self, dL_dE):
        """``adjoint`` with per-phase device times: returns (ga, gs, stats), stats as in
        trinity_adjoint_profile (ms of restores, recomputed steps, store copies, transposed
        solves, pushes, final kernel; mean transposed-solve iterations)."""
        G = self._grad_input(dL_dE)
        ga = np.zeros(self.nv)
        gs = np.zeros(self.nv)
        st = np.zeros(7)
        self.last_status = self._check(self.L.trinity_adjoint_profile(
            self.h, G.ctypes.data_as(ctypes.c_void_p), G.size, ga.ctypes.data_as(ctypes.c_void_p),
            gs.ctypes.data_as(ctypes.c_void_p), 0, st.ctypes.data_as(_lib.P_double)))
        return ga, gs, st

    def _grad_input(self, dL_dE):
        G = np.ascontiguousarray(dL_dE, dtype=np.float64)
        if G.size != self.n_det * self.nbins:
            raise ValueError("dL_dE must have n_det * nbins entries")
        return G

    def reset(self):
        return self._check(self.L.trinity_reset(self.h))

    # -- outputs
    def kernels_per_step(self):
        """Kernel launches of one time step with the current inputs."""
        n = ctypes.c_int()
        self._check(self.L.trinity_kernels_per_step(self.h, ctypes.byref(n)))
        return n.value

    def sweep_form(self):
        """Form of the ray sweep: "plain", "tma" (TMA-staged upwind planes) or "two-level"."""
        f = ctypes.c_int()
        self._check(self.L.trinity_sweep_form(self.h, ctypes.byref(f)))
        return ("plain", "tma", "two-level")[f.value]

    def steps_done(self):
        n = ctypes.c_int()
        self._check(self.L.trinity_steps_done(self.h, ctypes.byref(n)))
        return n.value

    def detectors(self):
        out = np.zeros((self.n_det, self.nbins))
        self._check(self.L.trinity_read_detectors(
            self.h, out.ctypes.data_as(_lib.P_double), out.size))
        return out

    def energy(self, nsteps=None):
        """(N(t), escaped) per step of the last ``nsteps`` steps."""
        b = self.balance(nsteps)
        return b["energy"], b["escaped"]

    def balance(self, nsteps=None):
        """Photon accounting per step (FP64, from the device): energy in the box, escaped,
        absorbed, and the balance residual (see trinity_read_energy)."""
        nsteps = self.steps_done() if nsteps is None else nsteps
        out = {k: np.zeros(nsteps) for k in ("energy", "escaped", "absorbed", "residual")}
        self._check(self.L.trinity_read_energy(self.h, *(out[k].ctypes.data_as(_lib.P_double)
                                                         for k in ("energy", "escaped", "absorbed",
                                                                   "residual")), nsteps))
        return out

    def iterations(self, nsteps=None):
        nsteps = self.steps_done() if nsteps is None else nsteps
        mx = np.zeros(nsteps, dtype=np.int32)
        mean = np.zeros(nsteps)
        self._check(self.L.trinity_read_iterations(self.h, mx.ctypes.data_as(_lib.P_int),
                                                   mean.ctypes.data_as(_lib.P_double), nsteps))
        return mx, mean

    def executed_iterations(self, nsteps=None):
        """Per step, the iterations the tensor-core kernel executed per voxel (its tiles run
        until their slowest voxel stops); zeros in the other modes."""
        nsteps = self.steps_done() if nsteps is None else nsteps
        out = np.zeros(nsteps)
        self._check(self.L.trinity_read_executed_iterations(self.h, out.ctypes.data_as(_lib.P_double), nsteps))
        return out

    def field(self, what=FIELD_I, back=0, out=None):
        """Field at level steps_done-1-back as a host array [N_a, N_v] (or into a CUDA tensor);
        S has the source function's N_a (coarser on a two-level angular grid); FIELD_U is the
        energy density per voxel, [N_v]."""
        if out is not None and getattr(out, "is_cuda", False):
            self._check(self.L.trinity_read_field(self.h, what, back, ctypes.c_void_p(out.data_ptr()),
                                                  out.numel() * 4, 1))
            return out
        if what == FIELD_U:
            arr = np.empty(self.nv, dtype=np.float32)
        else:
            arr = np.empty((self.na_s if what == FIELD_S else self.na, self.nv), dtype=np.float32)
        self._check(self.L.trinity_read_field(self.h, what, back, arr.ctypes.data_as(ctypes.c_void_p),
                                              arr.nbytes, 0))
        return arr


REQ_QUEUED, REQ_ACTIVE, REQ_DONE, REQ_FAILED, REQ_CANCELLED = range(5)


class Server:
    """Many forward solves at once: requests are admitted by device-memory footprint into
    slots and advanced round-robin on their own streams (see trinity_serve_* in
    include/trinity.h)."""

    def __init__(self, hbm_budget_bytes, max_slots=8, steps_per_slice=32):
        self.L = lib()
        h = ctypes.c_void_p()
        rc = self.L.trinity_serve_create(int(hbm_budget_bytes), int(max_slots), int(steps_per_slice),
                                         ctypes.byref(h))
        if rc != OK:
            raise TrinityError(rc, "trinity_serve_create failed")
        self.h = h
        self._shape = {}

    def submit(self, prob):
        """Queue a solve of ``prob`` (a problem dict, ``steps`` time steps); returns its id.
        Raises TrinityError for malformed or over-budget requests."""
        mua = np.ascontiguousarray(prob["mua"], dtype=np.float32)
        mus = np.ascontiguousarray(prob["mus"], dtype=np.float32)
        nid = np.ascontiguousarray(prob["nidx"], dtype=np.float32)
        dets = prob.get("detectors", [])
        darr = (_lib.DetectorDesc * max(len(dets), 1))()
        for k, d in enumerate(dets):
            darr[k] = _lib.DetectorDesc(int(d["face"]), float(d["u_mm"]), float(d["v_mm"]),
                                        float(d["radius_mm"]), float(d["half_angle_deg"]))
        src = prob.get("source")
        sd = _lib.SourceDesc(0, 0.0, 0.0, 15.0, 0, 0.0) if src is None else _lib.SourceDesc(
            int(src["face"]), float(src["u_mm"]), float(src["v_mm"]), float(src["half_angle_deg"]),
            int(src["pulse_steps"]), float(src["energy"]))
        req = _lib.Request(grid_desc(prob), mua.ctypes.data, mus.ctypes.data, nid.ctypes.data,
                           float(prob["g"]), sd, len(dets), darr, float(prob.get("bin_ps", 10.0)),
                           int(prob.get("nbins", 1)), int(prob["steps"]), int(bool(prob.get("fresnel", False))))
        rid = ctypes.c_uint64()
        rc = self.L.trinity_serve_submit(self.h, ctypes.byref(req), ctypes.byref(rid))
        if rc != OK:
            raise TrinityError(rc, "trinity_serve_submit rejected the request")
        self._shape[rid.value] = (len(dets), int(prob.get("nbins", 1)))
        return rid.value

    def poll(self, rid):
        """(state, status, detectors or None, latency_ms or None) without blocking."""
        nd, nb = self._shape[rid]
        det = np.zeros((nd, nb))
        st = ctypes.c_int()
        lat = ctypes.c_double(-1.0)
        rc = self.L.trinity_serve_poll(self.h, rid, ctypes.byref(st), det.ctypes.data_as(_lib.P_double),
                                       det.size, ctypes.byref(lat))
        if st.value < REQ_DONE:
            return st.value, rc, None, None
        return st.value, rc, (det if st.value == REQ_DONE else None), lat.value

    def wait(self, rid, timeout_s=600.0):
        rc = self.L.trinity_serve_wait(self.h, rid, float(timeout_s))
        if rc != OK:
            raise TrinityError(rc, "request %d did not finish in time" % rid)
        return self.poll(rid)

    def cancel(self, rid):
        return self.L.trinity_serve_cancel(self.h, rid)

    def stats(self):
        c, f = ctypes.c_uint64(), ctypes.c_uint64()
        mc = ctypes.c_int()
        used = ctypes.c_size_t()
        self.L.trinity_serve_stats(self.h, ctypes.byref(c), ctypes.byref(f), ctypes.byref(mc), ctypes.byref(used))
        return dict(completed=c.value, failed=f.value, max_concurrent=mc.value, bytes_in_use=used.value)

    def close(self):
        if getattr(self, "h", None):
            self.L.trinity_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- host tables (no GPU needed)

def healpix_dirs(nside):
    n = 12 * nside * nside
    out = np.zeros((n, 3))
    rc = lib().trinity_healpix_dirs(nside, out.ctypes.data_as(_lib.P_double), out.size)
    if rc != OK:
        raise TrinityError(rc, "healpix_dirs")
    return out


def phase_matrix(nside, g):
    n = 12 * nside * nside
    out = np.zeros((n, n))
    geff = ctypes.c_double()
    rc = lib().trinity_phase_matrix(nside, float(g), out.ctypes.data_as(_lib.P_double), out.size,
                                    ctypes.byref(geff))
    if rc != OK:
        raise TrinityError(rc, "phase_matrix")
    return out, geff.value


def lattice_tables(nside, nx, ny, nz, h=1.0, periodic=False):
    n = 12 * nside * nside
    nmax = max(nx, ny, nz)
    dom_sgn = np.zeros((n, 2), dtype=np.int32)
    ds = np.zeros(n)
    offs = np.zeros((n, 2, nmax), dtype=np.int8)
    rc = lib().trinity_lattice_tables(nside, nx, ny, nz, float(h), int(periodic),
                                      dom_sgn.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      ds.ctypes.data_as(_lib.P_double),
                                      offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), offs.size)
    if rc != OK:
        raise TrinityError(rc, "lattice_tables")
    return dom_sgn, ds, offs


def interface_entries(nside, nidx, h=1.0, periodic=False):
    """(voxel, j, d, weight) arrays of the interface split for an n map [nz, ny, nx]."""
    nm = np.ascontiguousarray(nidx, dtype=np.float32)
    nz, ny, nx = nm.shape
    cnt = ctypes.c_size_t()
    L = lib()
    args = (nside, nx, ny, nz, float(h), int(periodic), nm.ctypes.data_as(ctypes.c_void_p))
    rc = L.trinity_interface_entries(*args, None, None, None, None, 0, ctypes.byref(cnt))
    if rc != OK:
        raise TrinityError(rc, "interface_entries")
    n = cnt.value
    vox, j, d = (np.zeros(n, dtype=np.int32) for _ in range(3))
    w = np.zeros(n)
    rc = L.trinity_interface_entries(*args, vox.ctypes.data_as(ctypes.c_void_p), j.ctypes.data_as(ctypes.c_void_p),
                                     d.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p), n,
                                     ctypes.byref(cnt))
    if rc != OK:
        raise TrinityError(rc, "interface_entries")
    return vox, j, d, w


def parent_map(nside_fine, nside_coarse):
    """Coarse RING pixel containing each fine pixel's centre (int array [12 nside_fine^2])."""
    out = np.zeros(12 * nside_fine * nside_fine, dtype=np.int32)
    rc = lib().trinity_parent_map(int(nside_fine), int(nside_coarse), out.ctypes.data_as(_lib.P_int), out.size)
    if rc != OK:
        raise TrinityError(rc, "trinity_parent_map failed")
    return out


def cone_weights(nside, face, half_angle_deg, inward):
    n = 12 * nside * nside
    out = np.zeros(n)
    rc = lib().trinity_cone_weights(nside, face, float(half_angle_deg), int(inward),
                                    out.ctypes.data_as(_lib.P_double), n)
    if rc != OK:
        raise TrinityError(rc, "cone_weights")
    return out
