"""The time loop of the forward model, FP64, plain and unblocked.

Problem description: a dict (see ``workloads``) with the grid, optics maps, source,
detectors and iteration controls.  Everything below follows the paper's calculation
steps (§2.4): per time step, solve the transfer equation on every ray (Step 3), build
the source function (Step 5), repeat until the two agree (Step 6), go to the next
step (Step 7).  Domain decomposition and halo exchange (Steps 2 and 4) do not apply
to one address space.

Per voxel v and direction d, at time level n (time step dt):

* Eq. 10: I(n) = I_up * exp(-x) + S_up * b0(x) + S(n) * b1(x), with x = mu_t(v) ds_d the
  optical depth of the segment from the upwind ray sample to v, and
  b0 = [1 - (1 + x) e^-x] / x, b1 = [x - 1 + e^-x] / x the weights of Eq. 9 (linear source
  between the two samples, Eq. 8).  mu_t, a = mu_s/mu_t and n are those of v (the nearest
  grid point of the ray point, text under Eq. 10).
* The upwind values are taken at the retarded time t - ds_d / c(v) (Eq. 10), that is
  delta = ds_d n(v) / (c0 dt) steps back, linearly interpolated between time levels
  n - m and n - m - 1 (m = floor(delta)).  Levels before 0 are zero.
* Q(v, d) := I_up exp(-x) + S_up b0(x) holds everything that is known before the source
  iteration, so Eq. 10 reads I(n) = Q + b1 * S(n).
* Eq. 12 with Eq. 2: S_i = a(v) * sum_j P_ij I_j(n).  Substituting Eq. 10 gives a linear
  fixed point per voxel, S = a P (Q + b1 o S), which is iterated from the previous
  step's S(n-1) (§2.1, last paragraph before Eq. 13).  The paper stops "when consistent"
  and names no tolerance.  Reading: voxel v stops at the first iteration k with
      rho/(1-rho) ||S^k - S^(k-1)||_inf <= tol * max(||S^k||_inf, FLOOR * S_glob),
  where rho = a(v) max_d b1(v, d) bounds ||a P B1||_inf (P has unit row sums), so the
  stopped iterate is within tol of the fixed point relative to the voxel's own source,
  and S_glob = max |S(n-1)| over the whole grid.  The floor matters where the fixed point
  is zero (the pulse has passed, Q = 0): there a purely relative test never holds.
* Index interfaces (§3.3, Eqs. 13-14; reading in ``fresnel``): with ``fresnel`` set, Q of
  the directions whose segment crosses an index step is split into the specular and
  Snell directions before the source iteration.
* Boundaries: absorbing ("vacuum", §3.1: photons reaching the box boundary are lost,
  nothing re-enters), periodic, or mirror (test configurations).  The pulse enters
  through the face voxel of the source spot, for the directions of the source cone,
  during the first ``pulse_steps`` levels; the ghost sample outside the face has S = 0.
  Mirror (specular reflection at every face, read as the method of images): a ghost
  upwind sample, at most one voxel outside on each axis, takes I and S of its image -
  the voxel reached by reflecting it back across each face it lies beyond, which is the
  nearest voxel inside - in the direction reflected in those faces (its components along
  them negated), at the same retarded levels.
* Detectors (§3.1): the outgoing flux through the face voxels of a disk, weighted per
  direction by the acceptance cone: E[k, bin(n)] += sum_v sum_d alpha_d Omega_cap
  (Omega_d . n_out) I(v, d) h^2 dt, with bin(n) = floor((n + 1/2) dt / bin_width).
* Photon accounting, per step n (FP64): N(n) = h^3 / c0 sum_v n_v sum_d w I (the photon
  energy of the samples: energy density I / c per unit solid angle, c = c0 / n, §2.1 under
  Eq. 1); escaped(n) = sum over face voxels and outgoing d of w (Omega_d . n_out) I h^2 dt;
  absorbed(n) = h^3 dt sum_v mu_a(v) sum_d w I (the absorption rate mu_a c times the
  energy N, Eq. 1's mu_a term); injected(n) = the source's inflow through its face voxel
  in step n; residual(n) = N(-1) + sum_{k<=n} [injected - escaped - absorbed](k) - N(n),
  N(-1) the energy of the state before step 0.  The residual is the scheme's own photon
  balance error, not a rounding check: it is zero once the light has left a box without
  absorption, while a short pulse is in flight it oscillates because a sample sees the
  pulse once per delay (a fraction of the steps), and in a closed box it follows the
  discrete decay rate's departure from exp(-mu_a c t).
"""
import numpy as np

from . import C0_MM_PER_NS, RING_DEPTH
from .healpix import ring_directions, pixel_weight
from .phase import phase_matrix
from .geometry import RayLattice, face_axes, floor_snapped
from .cones import cone_fractions, cap_solid_angle
from .fresnel import interface_operators, apply_interfaces

SERIES_X = 1e-3  # below this optical depth the Eq. 9 weights use their Taylor series
FLOOR = 1e-6     # absolute stop floor, relative to the grid-wide max |S| of the previous level


def reflection_table(dirs):
    """refl[d, mask]: the direction whose vector is Omega_d with the components of the axes
    in ``mask`` (bit 0 = x, 1 = y, 2 = z) negated.  The HEALPix pixel set is symmetric under
    each such reflection; a missing partner raises."""
    na = dirs.shape[0]
    out = np.empty((na, 8), dtype=np.int64)
    for mask in range(8):
        s = np.array([-1.0 if (mask >> a) & 1 else 1.0 for a in range(3)])
        dots = (dirs * s[None, :]) @ dirs.T
        best = np.argmax(dots, axis=1)
        if np.any(dots[np.arange(na), best] < 1.0 - 1e-12):
            raise ValueError("direction set is not symmetric under a face reflection")
        out[:, mask] = best
    return out


def time_step(courant, h, n_ref):
    """dt such that a photon at c0/n_ref crosses ``courant`` voxels per step (§3.1)."""
    return courant * h * n_ref / C0_MM_PER_NS


def ray_weights(x):
    """exp(-x), b0(x), b1(x) of Eq. 9 / Eq. 10 (b0 weights S_up, b1 weights S(n)).

    For x < 1e-3 the removable 0/0 is avoided with the Taylor series
    b0 = x/2 - x^2/3 + x^3/8 - x^4/30,  b1 = x/2 - x^2/6 + x^3/24 - x^4/120.
    """
    x = np.asarray(x, dtype=np.float64)
    T = np.exp(-x)
    small = x < SERIES_X
    xs = np.where(small, 1.0, x)
    b0 = np.where(small, x / 2 - x**2 / 3 + x**3 / 8 - x**4 / 30, (1.0 - (1.0 + xs) * T) / xs)
    b1 = np.where(small, x / 2 - x**2 / 6 + x**3 / 24 - x**4 / 120, (xs - 1.0 + T) / xs)
    return T, b0, b1


def face_spot(shape_zyx, h, face, u_mm, v_mm):
    """Face voxel (iu, iv) that contains the point (u_mm, v_mm) of a face."""
    nz, ny, nx = shape_zyx
    n = (nx, ny, nz)
    _, _, (ua, va) = face_axes(face)
    iu, iv = int(np.floor(u_mm / h)), int(np.floor(v_mm / h))
    if not (0 <= iu < n[ua] and 0 <= iv < n[va]):
        raise ValueError("point outside the face")
    return iu, iv


def face_voxel_flat(shape_zyx, face, iu, iv):
    """Flat voxel index of face voxel (iu, iv) of ``face``."""
    nz, ny, nx = shape_zyx
    n = (nx, ny, nz)
    ax, sign, (ua, va) = face_axes(face)
    p = [0, 0, 0]
    p[ax] = 0 if sign < 0 else n[ax] - 1
    p[ua], p[va] = iu, iv
    return (p[2] * ny + p[1]) * nx + p[0]


def disk_voxels(shape_zyx, h, face, u_mm, v_mm, radius_mm):
    """Flat indices of the face voxels whose centre lies within ``radius_mm`` of (u, v)."""
    nz, ny, nx = shape_zyx
    n = (nx, ny, nz)
    _, _, (ua, va) = face_axes(face)
    out = []
    for iu in range(n[ua]):
        for iv in range(n[va]):
            du = (iu + 0.5) * h - u_mm
            dv = (iv + 0.5) * h - v_mm
            if du * du + dv * dv <= radius_mm * radius_mm * (1.0 + 1e-12):
                out.append(face_voxel_flat(shape_zyx, face, iu, iv))
    return np.array(sorted(out), dtype=np.int64)


def source_amplitudes(dirs, w, face, half_angle_deg, h, dt, pulse_steps, energy):
    """Inflow intensity per direction that injects ``energy`` through one face voxel.

    The power entering through a face voxel along d is I w |Omega_d . n| h^2, so
    I_d = E alpha_d / (w |Omega_d . n| h^2 pulse_steps dt) carries E alpha_d in total.
    """
    alpha = cone_fractions(dirs, face, half_angle_deg, inward=True)
    ax, sign, _ = face_axes(face)
    cos_in = -sign * dirs[:, ax]
    if np.any((alpha > 0) & (cos_in <= 0)):
        raise ValueError("source cone reaches an outgoing direction")
    amp = np.zeros(dirs.shape[0])
    on = alpha > 0
    amp[on] = energy * alpha[on] / (w * cos_in[on] * h * h * pulse_steps * dt)
    return amp


def detector_weights(dirs, face, half_angle_deg):
    """Per-direction flux weight alpha_d Omega_cap (Omega_d . n_out) of a detector cone."""
    alpha = cone_fractions(dirs, face, half_angle_deg, inward=False)
    ax, sign, _ = face_axes(face)
    cos_out = sign * dirs[:, ax]
    if np.any((alpha > 0) & (cos_out <= 0)):
        raise ValueError("detector cone reaches an incoming direction")
    return alpha * cap_solid_angle(half_angle_deg) * np.where(alpha > 0, cos_out, 0.0)


def step_bin(n, dt, bin_width):
    """Detector time bin of step n: floor((n + 1/2) dt / bin_width)."""
    return int(floor_snapped((n + 0.5) * dt / bin_width))


class Model:
    """Precomputed, step-independent data of one problem (all FP64)."""

    def __init__(self, prob):
        self.prob = prob
        nz, ny, nx = prob["nz"], prob["ny"], prob["nx"]
        self.shape = (nz, ny, nx)
        self.nv = nx * ny * nz
        self.h = float(prob["h"])
        self.dirs = ring_directions(prob["nside"])
        self.na = self.dirs.shape[0]
        self.w = pixel_weight(prob["nside"])
        # the source function's angular grid (§2.1: 192 bins fed by 3072 transport bins
        # in the paper's fiducial runs); the transport grid unless a coarser one is named
        self.nside_s = int(prob.get("nside_scatter") or prob["nside"])
        self.P = phase_matrix(self.nside_s, float(prob["g"]))
        self.boundary = prob.get("boundary", "vacuum")
        if self.boundary not in ("vacuum", "periodic", "mirror"):
            raise ValueError("unknown boundary %r" % self.boundary)
        self.periodic = self.boundary == "periodic"
        self.mirror = self.boundary == "mirror"
        self.lat = RayLattice(self.dirs, self.shape, self.h, self.periodic)
        self.reflect = reflection_table(self.dirs) if self.mirror else None
        self.dt = time_step(prob["courant"], self.h, prob["n_ref"])
        mua = np.asarray(prob["mua"], dtype=np.float64).ravel()
        mus = np.asarray(prob["mus"], dtype=np.float64).ravel()
        self.nidx = np.asarray(prob["nidx"], dtype=np.float64).ravel()
        self.mut = mua + mus
        self.mua = mua
        self.albedo = np.where(self.mut > 0, mus / np.where(self.mut > 0, self.mut, 1.0), 0.0)
        self.tol = float(prob.get("tol", 1e-6))
        self.max_iters = int(prob.get("max_iters", 2000))

        # source inflow
        self.src = None
        src = prob.get("source")
        if src is not None and self.boundary == "vacuum":
            face = int(src["face"])
            iu, iv = face_spot(self.shape, self.h, face, src["u_mm"], src["v_mm"])
            amp = src.get("amp")
            if amp is None:
                amp = source_amplitudes(self.dirs, self.w, face, src["half_angle_deg"], self.h,
                                        self.dt, int(src["pulse_steps"]), float(src["energy"]))
            amp = np.asarray(amp, dtype=np.float64)
            for d in np.nonzero(amp)[0]:
                if self.lat.entry_face(d) != face:
                    raise ValueError("source direction does not enter through the source face")
            self.src = dict(face=face, voxel=face_voxel_flat(self.shape, face, iu, iv),
                            amp=amp, pulse_steps=int(src["pulse_steps"]))

        # detectors
        self.dets = []
        for det in prob.get("detectors", []):
            face = int(det["face"])
            vox = disk_voxels(self.shape, self.h, face, det["u_mm"], det["v_mm"], det["radius_mm"])
            wgt = detector_weights(self.dirs, face, det["half_angle_deg"])
            self.dets.append(dict(face=face, voxels=vox, weight=wgt))
        self.bin_width = float(prob.get("bin_ps", 10.0)) * 1e-3
        self.nbins = int(prob.get("nbins", 1))

        # index interfaces (Eqs. 13-14)
        self.interfaces = interface_operators(self) if prob.get("fresnel", False) else {}

        # face outflow for the escaped-energy tally
        self.faces = []
        if self.boundary == "vacuum":
            for face in range(6):
                ax, sign, (ua, va) = face_axes(face)
                n = (nx, ny, nz)
                vox = np.array([face_voxel_flat(self.shape, face, iu, iv)
                                for iu in range(n[ua]) for iv in range(n[va])], dtype=np.int64)
                cos_out = sign * self.dirs[:, ax]
                self.faces.append((vox, np.where(cos_out > 0, cos_out, 0.0)))

    def segment_data(self, voxels=None):
        """Per (d, v) upwind index, delay split (m, f) and Eq. 9 weights for a voxel set."""
        vox = np.arange(self.nv) if voxels is None else np.asarray(voxels, dtype=np.int64)
        up = np.stack([self.lat.upwind_index(d, vox) for d in range(self.na)])
        delta = self.lat.ds[:, None] * self.nidx[None, vox] / (C0_MM_PER_NS * self.dt)
        if np.any(delta < 1.0) or np.any(delta >= RING_DEPTH - 1):
            raise ValueError("retarded delay outside [1, %d) steps" % (RING_DEPTH - 1))
        m = np.floor(delta).astype(np.int64)
        f = delta - m
        x = self.mut[None, vox] * self.lat.ds[:, None]
        T, b0, b1 = ray_weights(x)
        seg = dict(vox=vox, up=up, m=m, f=f, T=T, b0=b0, b1=b1)
        if self.mirror:
            # image of each ghost upwind sample and the reflected direction it is read in
            nx, ny, nz = self.shape[2], self.shape[1], self.shape[0]
            n = (nx, ny, nz)
            img = np.full(up.shape, -1, dtype=np.int64)
            dstar = np.tile(np.arange(self.na)[:, None], (1, vox.size))
            for d in range(self.na):
                ghost = up[d] < 0
                if not np.any(ghost):
                    continue
                q = self.lat.upwind_coords(d, vox[ghost])
                mask = np.zeros(q[0].shape, dtype=np.int64)
                for a in range(3):
                    out = (q[a] < 0) | (q[a] >= n[a])
                    mask |= out.astype(np.int64) << a
                    q[a] = np.clip(q[a], 0, n[a] - 1)
                img[d, ghost] = (q[2] * ny + q[1]) * nx + q[0]
                dstar[d, ghost] = self.reflect[d, mask]
            seg["img"], seg["dstar"] = img, dstar
        return seg

    def inflow(self, seg, level):
        """Inflow intensity at time ``level`` for the (d, v) pairs with up == -1."""
        out = np.zeros(seg["up"].shape)
        if self.src is None:
            return out
        if not isinstance(level, np.ndarray):
            level = np.full(seg["up"].shape, level)
        on = (level >= 0) & (level < self.src["pulse_steps"])
        at_spot = (seg["vox"][None, :] == self.src["voxel"]) & (seg["up"] == -1)
        amp = self.src["amp"][:, None] * np.ones_like(out)
        return np.where(on & at_spot, amp, 0.0)


def _retarded(hist, seg, n, which, model):
    """Upwind value of field ``which`` at time n - delta (linear in time, Eq. 10)."""
    up = seg["up"]
    m, f = seg["m"], seg["f"]
    dd = np.arange(up.shape[0])[:, None] * np.ones_like(up)
    vals = []
    for lev in (n - m, n - m - 1):
        v = np.zeros(up.shape)
        ok = (up >= 0) & (lev >= -(RING_DEPTH - 1))
        v[ok] = hist(which, lev[ok], dd[ok], up[ok])
        if "img" in seg:  # mirror faces: the image sample in the reflected direction
            im = (up < 0) & (lev >= -(RING_DEPTH - 1))
            v[im] = hist(which, lev[im], seg["dstar"][im], seg["img"][im])
        if which == "I":
            v = v + model.inflow(seg, lev)
        vals.append(v)
    return (1.0 - f) * vals[0] + f * vals[1]


def source_iteration(model, Q, b1, S0, albedo, s_glob):
    """Per-voxel fixed point S = a P (Q + b1 o S) by plain iteration (Eq. 12, §2.4 Steps 5-6).

    Q, b1, S0: [N_a, n]; albedo: [n]; s_glob: max |S(n-1)| over the grid.
    Returns (S, iterations per voxel).
    """
    P = model.P
    rho = albedo * np.max(b1, axis=0)
    S = S0.copy()
    iters = np.zeros(Q.shape[1], dtype=np.int64)
    act = np.arange(Q.shape[1])
    for k in range(1, model.max_iters + 1):
        if act.size == 0:
            break
        X = Q[:, act] + b1[:, act] * S[:, act]
        Snew = albedo[None, act] * (P @ X)
        dS = np.max(np.abs(Snew - S[:, act]), axis=0)
        smax = np.max(np.abs(Snew), axis=0)
        S[:, act] = Snew
        iters[act] = k
        r = rho[act]
        done = r / (1.0 - r) * dS <= model.tol * np.maximum(smax, FLOOR * s_glob)
        act = act[~done]
    return S, iters


class Solver:
    """Full-grid time stepping with a D-level history ring."""

    def __init__(self, prob, init=None):
        """``init`` = (I0, S0), arrays broadcastable to [N_a, N_v]: the field at every
        level before 0 (a state that has existed for ever).  Default: zero history."""
        self.m = Model(prob)
        m = self.m
        self.seg = m.segment_data()
        self.I = np.zeros((RING_DEPTH, m.na, m.nv))
        self.S = np.zeros((RING_DEPTH, m.na, m.nv))
        self.hist_from = 0
        if init is not None:
            for lev in range(-(RING_DEPTH - 1), 0):
                self.I[lev % RING_DEPTH] = init[0]
                self.S[lev % RING_DEPTH] = init[1]
            self.hist_from = -(RING_DEPTH - 1)
        self.n = 0
        self.det = np.zeros((len(m.dets), m.nbins))
        self.energy = []
        self.escaped = []
        self.absorbed = []
        self.injected = []
        self.residual = []
        # energy of the state before step 0 (the held initial level, else nothing)
        self.energy_init = 0.0
        if init is not None:
            I0 = np.broadcast_to(np.asarray(init[0], dtype=np.float64), (m.na, m.nv))
            self.energy_init = m.h**3 / C0_MM_PER_NS * np.sum(m.nidx[None, :] * m.w * I0)
        self._balance = self.energy_init
        self.iters_max = []
        self.iters_mean = []

    def _hist(self, which, lev, d, u):
        arr = self.I if which == "I" else self.S
        return arr[lev % RING_DEPTH, d, u] * (lev >= self.hist_from)

    def step(self):
        m, seg, n = self.m, self.seg, self.n
        I_up = _retarded(self._hist, seg, n, "I", m)
        S_up = _retarded(self._hist, seg, n, "S", m)
        Q = I_up * seg["T"] + S_up * seg["b0"]
        if m.interfaces:
            apply_interfaces(m.interfaces, Q)
        if n > 0 or self.hist_from < 0:
            S_prev = self.S[(n - 1) % RING_DEPTH]
        else:
            S_prev = np.zeros((m.na, m.nv))
        S, iters = source_iteration(m, Q, seg["b1"], S_prev, m.albedo, np.max(np.abs(S_prev)))
        I = Q + seg["b1"] * S
        self.I[n % RING_DEPTH] = I
        self.S[n % RING_DEPTH] = S
        self.iters_max.append(int(iters.max()))
        self.iters_mean.append(float(iters.mean()))
        self._tally(I, n)
        self.n += 1

    def _tally(self, I, n):
        m = self.m
        h2dt = m.h * m.h * m.dt
        b = step_bin(n, m.dt, m.bin_width)
        for k, det in enumerate(m.dets):
            if b < m.nbins:
                self.det[k, b] += h2dt * np.sum(det["weight"][:, None] * I[:, det["voxels"]])
        N = m.h**3 / C0_MM_PER_NS * np.sum(m.nidx[None, :] * m.w * I)
        self.energy.append(N)
        esc = 0.0
        for vox, cos_out in m.faces:
            esc += m.w * h2dt * np.sum(cos_out[:, None] * I[:, vox])
        self.escaped.append(esc)
        ab = m.h**3 * m.dt * m.w * np.sum(m.mua[None, :] * I)
        self.absorbed.append(ab)
        inj = injected_energy(m, n)
        self.injected.append(inj)
        self._balance += inj - esc - ab
        self.residual.append(self._balance - N)

    def run(self, nsteps):
        for _ in range(nsteps):
            self.step()
        return self.result()

    def result(self):
        return dict(detectors=self.det.copy(), energy=np.array(self.energy),
                    escaped=np.array(self.escaped), absorbed=np.array(self.absorbed),
                    injected=np.array(self.injected), residual=np.array(self.residual),
                    iters_max=np.array(self.iters_max),
                    iters_mean=np.array(self.iters_mean), steps=self.n)

    def level(self, which, back=0):
        """Field at time level n-1-back (the most recent completed level for back=0)."""
        arr = self.I if which == "I" else self.S
        lev = self.n - 1 - back
        if lev < 0:
            return np.zeros(arr.shape[1:])
        return arr[lev % RING_DEPTH].copy()


def injected_energy(model, n):
    """Energy the source's inflow carries into the box during step n: the ghost sample's
    intensity at level n times w |Omega_d . n| h^2 dt, summed over the source directions."""
    src = model.src
    if src is None or not (0 <= n < src["pulse_steps"]):
        return 0.0
    ax, _, _ = face_axes(src["face"])
    return float(np.sum(src["amp"] * model.w * np.abs(model.dirs[:, ax])) * model.h**2 * model.dt)


def energy_density(model, I):
    """Photon energy density per voxel, u = (n / c0) sum_d w I_d (§3.1 plots its maps; the
    energy density of radiance I per unit solid angle is I / c, c = c0 / n)."""
    return model.nidx / C0_MM_PER_NS * model.w * np.sum(I, axis=0)


def one_step_at(model, n, hist, voxels, s_glob):
    """I(n), S(n) at the given voxels from supplied history (a local, one-step check).

    ``model`` is a ``Model`` of the problem.  ``hist(which, levels, dirs, voxels)`` returns
    stored field values (levels >= 0 are stored ones; negative levels must return zero
    unless the problem has an initial state).  Everything at level n of a voxel depends
    only on levels < n and on S(n) of the same voxel, so a large run can be checked, or
    the oracle's per-voxel work timed, sample by sample.  ``s_glob`` is max |S(n-1)| over
    the whole grid.
    """
    seg = model.segment_data(voxels)
    I_up = _retarded(hist, seg, n, "I", model)
    S_up = _retarded(hist, seg, n, "S", model)
    Q = I_up * seg["T"] + S_up * seg["b0"]
    vox = seg["vox"]
    if model.interfaces:
        pos = {int(v): k for k, v in enumerate(vox)}
        sub = {pos[v]: ops for v, ops in model.interfaces.items() if v in pos}
        apply_interfaces(sub, Q)
    lev = np.full(vox.shape, n - 1)
    S_prev = np.stack([hist("S", lev, np.full(vox.shape, d), vox) for d in range(model.na)])
    S, iters = source_iteration(model, Q, seg["b1"], S_prev, model.albedo[vox], s_glob)
    return Q + seg["b1"] * S, S, iters
