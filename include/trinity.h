/*
 * trinity.h -- C ABI of the GB300 time-dependent radiative-transfer forward model.
 *
 * The library solves the time-dependent radiative transfer equation (Eq. 1 of
 * Yajima et al., "TRINITY: a three-dimensional time-dependent radiative transfer code
 * for in-vivo near-infrared imaging", arXiv:2105.01028) on a uniform voxel grid with
 * HEALPix directions, with the paper's retarded long-characteristic update (Eqs. 9-10)
 * and per-step source iteration (Eq. 12, Section 2.4 steps 3, 5, 6, 7), and bins the
 * escaping light into time-resolved detector curves (Section 3.1).
 *
 * Conventions for every entry point:
 *   - Units: mm, 1/mm, ns.  Voxel arrays are [nz][ny][nx] (x fastest), float32.
 *   - Directions are HEALPix RING order, N_a = 12 * nside^2.  Device fields are laid out
 *     [direction][voxel].
 *   - Faces are 0..5 = -x, +x, -y, +y, -z, +z.  A point on a face is (u, v) in mm along
 *     the face's two other axes in increasing order (x face: (y, z); y face: (x, z);
 *     z face: (x, y)).
 *   - Inputs are copied; the caller keeps ownership of every pointer it passes.  Output
 *     buffers are allocated by the caller.  ``ptr_kind`` 0 = host pointer, 1 = device
 *     pointer (device memory of the context's GPU).
 *   - Every call returns a trinity_status; on error the context keeps a message readable
 *     with trinity_last_error().  Nothing aborts the process and no exception crosses
 *     the ABI.  Calls on one context are not thread-safe; separate contexts are
 *     independent.
 *   - All device work of a context is issued on the stream given at creation (0 = the
 *     legacy default stream); calls that return data to the host synchronise that stream.
 *   - Device-side waits inside kernels are bounded; a wait that runs out sets an error
 *     word that the next call reports as TRINITY_E_TIMEOUT.
 */
#ifndef TRINITY_H
#define TRINITY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct trinity_ctx trinity_ctx;

typedef enum {
  TRINITY_OK = 0,
  TRINITY_W_NOT_CONVERGED = 1, /* completed, but some voxel hit max_iters in a step */
  TRINITY_E_INVALID = -1,      /* bad argument or unsupported combination */
  TRINITY_E_OOM = -2,          /* device allocation failed */
  TRINITY_E_CUDA = -3,         /* a CUDA call failed (message has the CUDA error) */
  TRINITY_E_STATE = -4,        /* call not allowed in the context's current state */
  TRINITY_E_TIMEOUT = -5,      /* a bounded device-side wait ran out */
  TRINITY_E_UNSUPPORTED = -6   /* the device cannot run this (e.g. not sm_103) */
} trinity_status;

enum { TRINITY_BOUNDARY_VACUUM = 0, TRINITY_BOUNDARY_PERIODIC = 1, TRINITY_BOUNDARY_MIRROR = 2 };
enum { TRINITY_FP32 = 0, TRINITY_BF16 = 1 };
enum { TRINITY_FIELD_I = 0, TRINITY_FIELD_S = 1, TRINITY_FIELD_U = 2 };

/*
 * Grid and solver description.
 *   nx, ny, nz   voxels per axis (>= 2 each); h_mm voxel size.
 *   nside        HEALPix resolution of the transport: 1, 2 or 4 (12, 48, 192 directions);
 *                up to 16 (3072) with a coarser nside_scatter.
 *   courant      c0 * dt / (n_ref * h): the time step dt = courant * h * n_ref / c0
 *                (the paper's rule "dt = fraction x light-crossing time of a grid",
 *                Sections 2.2 and 3.1).
 *   n_ref        refractive index used to define dt.
 *   boundary     TRINITY_BOUNDARY_VACUUM (absorbing faces, Section 3.1), _PERIODIC, or
 *                _MIRROR (test configuration: every face reflects specularly, by the
 *                method of images: a ray sample whose upwind sample lies outside the box
 *                takes I and S of that sample's image - the nearest voxel inside - in the
 *                direction reflected in the faces it lay beyond, at its own retarded
 *                levels).  Periodic and mirror boxes take no source and count no escape;
 *                mirror is not available on a two-level grid or for the adjoint
 *                (TRINITY_E_UNSUPPORTED).
 *   precision    TRINITY_FP32 (all arithmetic FP32) or TRINITY_BF16 (the angular
 *                scattering sum of Eq. 12 in BF16 with FP32 accumulation on the tensor
 *                cores; transport FP32; detector and energy sums FP64 in both modes).
 *   tol          source-iteration tolerance (relative, see trinity_step).
 *   max_iters    source-iteration cap per step (>= 1).
 *   nside_scatter  0 (or nside): one angular grid.  Otherwise the source function lives
 *                on the coarser HEALPix grid nside_scatter (1, 2 or 4) while the transport
 *                runs on nside (2, 4, 8 or 16, a multiple): each coarse bin takes the mean
 *                intensity of its (nside / nside_scatter)^2 finer bins, as the paper's
 *                fiducial runs do with 3072 transport and 192 source-function bins
 *                (Section 2.1, text after Eq. 12).  Per step the sweep forms Q on the fine
 *                directions and its mean over each coarse bin's children, the source
 *                iteration runs on the coarse bins with b1 the children's mean b1, and
 *                I = Q + b1 S(parent) is formed on the fine directions.  Fields: I has
 *                12 nside^2 directions, S 12 nside_scatter^2.  No adjoint on two levels.
 */
typedef struct {
  int nx, ny, nz;
  double h_mm;
  int nside;
  double courant;
  double n_ref;
  int boundary;
  int precision;
  double tol;
  int max_iters;
  int nside_scatter;
} trinity_grid_desc;

/* Bytes of device memory a context with this description allocates (for admission
 * control).  Returns 0 for an invalid description. */
size_t trinity_footprint_bytes(const trinity_grid_desc* desc);

/* Create a context: checks the device (sm_103), builds the direction table, the ray
 * lattice (Section 2.1, rays independent of the grid; Section 2.4 step 1) and allocates
 * the time-level history of I and S (the paper keeps several time bins of I and S,
 * Section 2.2).  ``cuda_stream`` is a cudaStream_t or NULL.  *out is NULL on error. */
int trinity_create_grid(const trinity_grid_desc* desc, void* cuda_stream, trinity_ctx** out);

/* Optical maps (Eq. 1): mu_a, mu_s (1/mm, >= 0) and refractive index n (>= 1) per voxel,
 * [nz][ny][nx] float32, host (ptr_kind 0) or device (1) pointers; g is the global
 * Henyey-Greenstein anisotropy (Eq. 11), -1 < g < 1.  Every voxel's retarded delay
 * ds * n / (c0 dt) must lie in [1, 4) steps, else TRINITY_E_INVALID.  Must be called
 * before the first step; calling it again resets the run. */
int trinity_set_optics(trinity_ctx* ctx, const float* mua, const float* mus, const float* n,
                       double g, int ptr_kind);
int trinity_set_optics_uniform(trinity_ctx* ctx, double mua, double mus, double g, double n);

/* Refraction and reflection at refractive-index steps (Eqs. 13-14; Section 3.3 applies
 * them at the grid points next to a region of different index).  With ``on`` set, at
 * every voxel whose upwind ray sample lies in a voxel of different n, the light arriving
 * along that direction is split, after the sweep and before the source iteration, into
 * the specular direction (Fresnel reflectance R, Eq. 14) and the Snell direction (1 - R,
 * Eq. 13), each snapped to the nearest pixel; the interface normal is the
 * central-difference gradient of the n map.  The split conserves photons.  The table is
 * rebuilt from the n map of each trinity_set_optics call.  Before the first step. */
int trinity_set_fresnel(trinity_ctx* ctx, int on);

/* Exact per-voxel source function instead of the source iteration, for piecewise-uniform
 * optics.  The iteration of Eq. 12 (Section 2.4 steps 5-6) converges to the fixed point
 * of S = a P (Q + b1 S); voxels with the same (mu_t, mu_a/mu_t) share the operator
 * M = (I - a P B1)^-1 a P (B1 = diag b1(mu_t ds_d)), so with ``on`` set each step takes
 * S = M Q in one product per voxel.  The operators are built on the host in FP64 (from
 * the FP32 phase matrix with its diagonal correction, the matrix the iteration applies)
 * at this call and at every trinity_set_optics, and applied in either precision mode in
 * one of two forms:
 *   on = 1: on the tensor cores where the grid allows it (192 directions and a voxel count
 *           that is a multiple of 4): three TF32 products, M_hi Q_hi + M_hi Q_lo +
 *           M_lo Q_hi with x_hi = tf32(x), x_lo = tf32(x - x_hi), accumulated in FP32
 *           (each operand carries ~22 significant bits; M and Q are non-negative, so the
 *           result is within a few 2^-22 of the FP32 product); otherwise as on = 2;
 *   on = 2: FP32 products on the SIMT cores;
 *   on = 0: off (the source iteration).
 * TRINITY_E_UNSUPPORTED if the optics have more than 8 distinct pairs (the mode is then
 * off) or on a two-level angular grid; TRINITY_E_INVALID for another ``on``.  Before the
 * first step. */
int trinity_set_exact_solve(trinity_ctx* ctx, int on);

/* Initial guess of each step's source iteration (Eq. 12, Section 2.4 steps 5-6):
 *   mode = 1 (default): the linear extrapolation in time 2 S(n-1) - S(n-2) (S(n-1) at the
 *            first stored level); the adjoint's transposed solve likewise starts from
 *            2 y(n+1) - y(n+2) of the two reverse steps before it;
 *   mode = 0: the previous level S(n-1), as Section 2.4 states it (and y(n+1)).
 * The iteration converges to the same fixed point and stops by the same rule either way;
 * the extrapolated guess starts closer to it, so fewer iterations are needed.
 * TRINITY_E_INVALID for another mode; TRINITY_E_STATE after the first step. */
int trinity_set_warm_start(trinity_ctx* ctx, int mode);

/* Number of optics classes the exact solve uses (0 when it is off). */
int trinity_exact_classes(const trinity_ctx* ctx, int* n);

/* Form of the exact solve that runs: 1 tensor cores, 2 FP32 SIMT, 0 off (or no optics
 * set yet). */
int trinity_exact_form(const trinity_ctx* ctx, int* form);

/* Number of interface voxels in the context's current table. */
int trinity_interface_count(const trinity_ctx* ctx, int* n);

/* Collimated pulse (Section 3.1): enters through the face voxel containing (u_mm, v_mm)
 * of ``face``, within a cone of ``half_angle_deg`` around the inward normal, during the
 * first ``pulse_steps`` time levels, carrying ``energy`` in total.  The cone's solid
 * angle is shared among directions by nearest pixel centre.  Only vacuum boundaries. */
int trinity_set_source(trinity_ctx* ctx, int face, double u_mm, double v_mm,
                       double half_angle_deg, int pulse_steps, double energy);

/* A surface detector (Section 3.1): the face voxels whose centres lie within radius_mm
 * of (u_mm, v_mm) collect the outgoing flux inside a cone of half_angle_deg around the
 * outward normal.  *det_id receives its index (0, 1, ...).  Before the first step. */
int trinity_add_detector(trinity_ctx* ctx, int face, double u_mm, double v_mm,
                         double radius_mm, double half_angle_deg, int* det_id);

/* Detector time bins: step n (covering [n dt, (n+1) dt)) goes to bin
 * floor((n + 1/2) dt / bin_ps); steps past nbins are not binned.  Before the first step. */
int trinity_set_bins(trinity_ctx* ctx, double bin_ps, int nbins);

/* The field at every time level before 0 (default: zero).  I0, S0 are [N_a][nz*ny*nx]
 * float32.  Before the first step. */
int trinity_set_initial_state(trinity_ctx* ctx, const float* I0, const float* S0, int ptr_kind);

/* Advance ``nsteps`` time steps.  Each step: the ray sweep (Eq. 10 with retarded upwind
 * I and S, linear in time between stored levels), the per-voxel source iteration
 * S = a P (Q + b1 S) of Eq. 12 with an isotropic rebalance after each update, started
 * from 2 S(n-1) - S(n-2) (trinity_set_warm_start) and stopped when
 *   rho/(1-rho) |S^k - S^(k-1)|_inf <= tol * scale,  scale = max(|S^k|_inf, 1e-6 max|S(n-1)|)
 * (rho = a * max_d b1, a bound on the contraction) or when the iterate sits at the noise
 * floor of the mode's arithmetic: FP32 mode, the change has not reached a new minimum for
 * three iterations; BF16 mode, |S^k - S^(k-1)|_inf <= 2^-17 scale (the resolution of X
 * carried as two BF16 terms) or no new minimum for two iterations.  Then the detector and
 * energy tallies.  iters_out (may be
 * NULL) receives the largest iteration count of each step.  Returns
 * TRINITY_W_NOT_CONVERGED if any voxel hit max_iters. */
int trinity_step(trinity_ctx* ctx, int nsteps, int* iters_out);

/* Same as trinity_step without per-step read-back: the steps are replayed from a
 * captured CUDA graph and the call returns once they are queued (no host sync). */
int trinity_run(trinity_ctx* ctx, int nsteps);

/* Advance ``nsteps`` steps with CUDA events around each kernel (on the context's stream)
 * and return the summed device time in ms of the sweep, the source iteration and the
 * tallies (tally + step counter): kernel_ms[3].  Synchronous; for measurement. */
int trinity_profile_steps(trinity_ctx* ctx, int nsteps, double* kernel_ms);

/* Block until queued work is done; reports errors of earlier asynchronous calls. */
int trinity_sync(trinity_ctx* ctx);

/* Detector curves, FP64 [n_det][nbins] (n must equal n_det * nbins). */
int trinity_read_detectors(trinity_ctx* ctx, double* out, size_t n);

/* Per-step photon accounting of the last ``nsteps`` completed steps, each [nsteps] FP64,
 * accumulated in FP64 on the device (Section 3.1 absorbing boundary; Eq. 1's mu_a term):
 *   N_t       photon energy in the box after the step, N = sum_v h^3 n_v / c0 sum_d w I
 *             (radiance I carries energy density I / c per unit solid angle, c = c0 / n);
 *   escaped   energy leaving through the faces in the step, sum of w (Omega . n_out) I h^2 dt
 *             over face voxels and outgoing directions;
 *   absorbed  energy absorbed in the step, h^3 dt sum_v mu_a sum_d w I (rate mu_a c times N);
 *   residual  the photon balance after the step: (energy before step 0) + (energy injected
 *             by the source so far) - (escaped and absorbed so far) - N_t.  It measures the
 *             discrete scheme's departure from photon conservation, not rounding: zero
 *             (to FP32 rounding of the fields) once the light has left a box without
 *             absorption; while a short pulse is in flight it oscillates, since N counts
 *             ray samples and a sample sees the pulse once per retarded delay.
 * Any pointer may be NULL. */
int trinity_read_energy(trinity_ctx* ctx, double* N_t, double* escaped, double* absorbed, double* residual,
                        size_t nsteps);

/* Per-step iteration statistics of the last ``nsteps`` steps: max and mean per voxel. */
int trinity_read_iterations(trinity_ctx* ctx, int* iters_max, double* iters_mean, size_t nsteps);

/* Iterations the BF16 tensor-core kernel executed per voxel in each of the last
 * ``nsteps`` steps: a 128-voxel tile iterates until its slowest voxel stops, so this mean
 * is at least the per-voxel mean of trinity_read_iterations; their ratio is the tile's
 * idle work.  Zero in the other modes (they do not count it). */
int trinity_read_executed_iterations(trinity_ctx* ctx, double* executed_mean, size_t nsteps);

/* Copy a field at time level (steps_done - 1 - back), 0 <= back <= 4, into ``out``
 * (``bytes`` = its size): TRINITY_FIELD_I or _S, [N_a][nz*ny*nx] float32 (S on the
 * source function's directions); or TRINITY_FIELD_U, the photon energy density per voxel
 * u = (n / c0) sum_d w I (the quantity whose maps Section 3.1 shows), [nz*ny*nx] float32,
 * summed in FP64 on the device.  Reading U uses the context's scratch for Q: call it
 * between steps, not while steps are queued on another thread. */
int trinity_read_field(trinity_ctx* ctx, int what, int back, void* out, size_t bytes, int ptr_kind);

/* Steps completed so far. */
int trinity_steps_done(const trinity_ctx* ctx, int* n);

/* Kernel launches one time step issues with the context's current inputs (sweep or
 * sweeps, interface split, source iteration, tallies, step counter). */
int trinity_kernels_per_step(const trinity_ctx* ctx, int* n);

/* Form of the ray sweep a step runs: 0 plain loads (one kernel), 1 upwind planes staged
 * through TMA tile loads (one kernel per dominant-axis class, run concurrently: vacuum
 * faces, a uniform refractive index, nx a multiple of 4), 2 the fused two-level sweep. */
int trinity_sweep_form(const trinity_ctx* ctx, int* form);

/* on = 0: the plain-load sweep even where the TMA-staged one applies (both perform the
 * same FP32 operations on the same values, so results are bit-identical); on = 1
 * (default): the TMA-staged sweep where it applies.  Before the first step. */
int trinity_set_sweep_tma(trinity_ctx* ctx, int on);

/* Zero the fields, tallies and step counter; keep grid, optics, source and detectors. */
int trinity_reset(trinity_ctx* ctx);

const char* trinity_last_error(const trinity_ctx* ctx);
void trinity_destroy(trinity_ctx* ctx);

/* Self-test of the tensor-core tile used by TRINITY_BF16: D = A B^T for one 128 x na tile
 * (na = 48 or 192) with A [128][K] and B [na][K] bf16 (row-major, K = na rounded up to a
 * multiple of 64, padding zero) and D [128][na] float32; host pointers.  Same operand
 * layouts, descriptors and TMEM read-out as the iteration kernel.  For testing. */
int trinity_tc_selftest(int na, const uint16_t* A, const uint16_t* B, float* D);

/* ---- Adjoint: gradient of a detector misfit with respect to mu_a and mu_s. ----
 *
 * The paper has no adjoint (Section 4 names inverse problems as future work).  These
 * calls give the exact reverse-mode derivative of the discrete forward model above
 * (Eqs. 9, 10, 12 and the index interfaces of Eqs. 13-14) for a scalar misfit L whose
 * derivative with respect to the detector curves, dL/dE [n_det][nbins], the caller
 * supplies.  The reverse sweep gathers nothing: each voxel pushes its ray adjoint to its
 * upwind sample at the two retarded levels it was interpolated from, and the transposed
 * scattering solve y = a P (q + b1 y) is the forward iteration again (P is symmetric).
 * Forward levels are recomputed from checkpoints segment by segment.  All reverse-sweep
 * arithmetic is FP32 with FP64 gradient sums; in TRINITY_BF16 mode the recomputed
 * forward steps run in BF16 (as the original ones did) and the reverse sweep in FP32. */

/* Device bytes that trinity_run_checkpointed plus trinity_adjoint add to a context:
 * ceil(nsteps / every) + 1 checkpoints of 4 levels of I and S, a store of every + 4
 * levels of I and S for one segment, the adjoint levels and the gradient sums.  0 for
 * invalid arguments. */
size_t trinity_adjoint_footprint_bytes(const trinity_grid_desc* desc, int nsteps, int every, int n_det,
                                       int nbins);

/* Run ``nsteps`` forward steps from step 0 (the context must be fresh or reset), saving
 * the state before steps 0, every, 2 every, ... and after the last step (levels n-4..n-1
 * of I and S and max |S(n-1)|: everything a step reads).  Same results as trinity_step.
 * TRINITY_E_OOM if the checkpoints do not fit; TRINITY_E_STATE if steps were taken. */
int trinity_run_checkpointed(trinity_ctx* ctx, int nsteps, int every);

/* Reverse sweep over the steps of the last trinity_run_checkpointed (no steps may follow
 * it).  dL_dE: FP64 [n_det][nbins], n = n_det * nbins.  grad_mua, grad_mus: FP64
 * [nz*ny*nx], receive dL/dmu_a and dL/dmu_s per voxel (where mu_a = mu_s = 0 only the
 * transport term, the albedo there being undefined).  ptr_kind applies to all three
 * pointers.  The forward state after the last step is restored, so stepping may continue
 * (after which the checkpoints no longer apply).  May be called again with another dL_dE.
 * Returns TRINITY_W_NOT_CONVERGED if a transposed solve hit max_iters somewhere. */
int trinity_adjoint(trinity_ctx* ctx, const double* dL_dE, size_t n, double* grad_mua, double* grad_mus,
                    int ptr_kind);

/* trinity_adjoint with CUDA events around each phase (on the context's stream).  stats
 * (host, 7 doubles) receives the summed device ms of [0] checkpoint restores, [1] the
 * recomputed forward steps, [2] the copies into the segment store, [3] detector injection
 * and transposed scattering solves, [4] transposed interface splits and upwind pushes,
 * [5] the final gradient kernel, and [6] the mean iterations of the transposed solves
 * per voxel and step.  For measurement. */
int trinity_adjoint_profile(trinity_ctx* ctx, const double* dL_dE, size_t n, double* grad_mua,
                            double* grad_mus, int ptr_kind, double* stats);

/* ---- Serving: many forward solves at once on one GPU. ----
 *
 * Reconstruction needs many forward models.  A server queues solve requests and admits
 * them, in arrival order, into slots while their device footprint
 * (trinity_footprint_bytes) fits the budget and a slot is free.  Each admitted request
 * runs in its own context on its own CUDA stream; a worker thread advances all active
 * requests round-robin in slices of graph-replayed steps, so their kernels overlap on the
 * device, and returns the detector curves and the latency (submission to completion).
 * Results do not depend on what else is running.  All CUDA work happens on the worker
 * thread of the server (on the device current when the first request is submitted). */
typedef struct trinity_server trinity_server;

typedef struct {
  int face;              /* 0..5; pulse_steps = 0 means no source */
  double u_mm, v_mm;
  double half_angle_deg;
  int pulse_steps;
  double energy;
} trinity_source_desc;

typedef struct {
  int face;
  double u_mm, v_mm, radius_mm, half_angle_deg;
} trinity_detector_desc;

typedef struct {
  trinity_grid_desc grid;
  const float *mua, *mus, *n; /* host, [nz][ny][nx]; copied at submission */
  double g;
  trinity_source_desc source;
  int n_detectors;
  const trinity_detector_desc* detectors; /* copied at submission */
  double bin_ps;
  int nbins;
  int nsteps;
  int fresnel; /* 1: refraction / reflection at index steps (trinity_set_fresnel) */
} trinity_request;

/* States reported by trinity_serve_poll. */
enum { TRINITY_REQ_QUEUED = 0, TRINITY_REQ_ACTIVE = 1, TRINITY_REQ_DONE = 2, TRINITY_REQ_FAILED = 3,
       TRINITY_REQ_CANCELLED = 4 };

/* A server with a device-memory budget (bytes), at most ``max_slots`` concurrent solves,
 * advancing each by ``steps_per_slice`` steps per turn. */
int trinity_serve_create(size_t hbm_budget_bytes, int max_slots, int steps_per_slice,
                         trinity_server** out);

/* Queue a request (inputs are copied); *req_id receives its id.  TRINITY_E_OOM if its
 * footprint exceeds the whole budget, TRINITY_E_INVALID for a malformed request.
 * Other failures (device errors, invalid optics) surface through trinity_serve_poll. */
int trinity_serve_submit(trinity_server* srv, const trinity_request* req, uint64_t* req_id);

/* Non-blocking: *state receives TRINITY_REQ_*; once done, the detector curves
 * ([n_detectors][nbins], n must match; may be NULL) and the latency in ms are written.
 * Returns the request's final status once it has one. */
int trinity_serve_poll(trinity_server* srv, uint64_t req_id, int* state, double* detectors,
                       size_t n, double* latency_ms);

/* Block until the request is done, failed or cancelled, or ``timeout_s`` passes
 * (TRINITY_E_TIMEOUT). */
int trinity_serve_wait(trinity_server* srv, uint64_t req_id, double timeout_s);

/* Cancel a queued or running request (a running one stops at its next slice). */
int trinity_serve_cancel(trinity_server* srv, uint64_t req_id);

/* Completed and failed counts, the largest number of concurrent solves seen, and the
 * device bytes currently held by admitted requests. */
int trinity_serve_stats(trinity_server* srv, uint64_t* completed, uint64_t* failed,
                        int* max_concurrent, size_t* bytes_in_use);

/* Cancel everything still queued or running, join the worker and free the server. */
void trinity_serve_destroy(trinity_server* srv);

/* ---- Source iteration that allocates nothing ----
 *
 * The paper has no counterpart of this call; it exists for callers that cannot call
 * cudaMalloc where they need a solve (their framework's memory pool owns the device, or
 * the code runs where allocation is forbidden).  It runs the per-voxel source iteration
 * S = (1 - eps) P (Q + b1 o S) of the FP32 mode (same arithmetic and stop rule as
 * trinity_step) on caller-owned device buffers and allocates no device memory: its
 * scratch (per-voxel contraction bounds, a max-reduction cell, iteration counters) is a
 * static device array of 4 MiB + 16 B that every GPU loading the library holds until the
 * process exits.
 *   na       12, 48 or 192 directions; nvox voxels, 1 <= nvox <= 1048576 (the scratch
 *            limit: larger sizes return TRINITY_E_INVALID without running).
 *   P        [na][na] FP32, symmetric with unit row sums up to rounding (e.g. the matrix of
 *            trinity_phase_matrix in FP32); the row-sum defect is corrected inside.
 *   Q, b1    [na][nvox] FP32: the known part of Eq. 10 and the weight of S(n) in it.
 *   eps      [nvox] FP32: mu_a / mu_t (1 where mu_t = 0).
 *   S_prev   [na][nvox] FP32: the start of the iteration (the previous step's S).
 *   S_out, I_out [na][nvox] FP32 outputs: S and I = Q + b1 o S.
 *   tol, max_iters as in trinity_grid_desc; *iters_max (may be NULL) gets the largest
 *   iteration count.  All pointers except iters_max are device pointers of the current
 *   device; the work runs on ``stream`` (a cudaStream_t or NULL) and the call returns
 *   after it finishes.  TRINITY_W_NOT_CONVERGED if a voxel reached max_iters.
 * The first call on a device looks up the scratch array's device address (a host-side
 * step, once per device); make that first call before any stream capture.  Every call
 * shares the one array and clears the parts that must start at zero, so calls whose GPU
 * work overlaps (concurrent streams, threads or processes sharing the library on one
 * device) race on it and must be serialised by the caller. */
int trinity_source_iteration_noalloc(int na, int nvox, const float* P, const float* Q,
                                     const float* b1, const float* eps, const float* S_prev,
                                     float* S_out, float* I_out, double tol, int max_iters,
                                     int* iters_max, void* stream);

/* ---- Host-side tables (no GPU needed): the same FP64 tables the context builds. ---- */

/* HEALPix RING pixel centres as unit vectors, out[N_a][3] (Section 2.1). */
int trinity_healpix_dirs(int nside, double* out, size_t n);

/* The normalised discrete phase matrix of Eq. 12, out[N_a][N_a] (row i = outgoing
 * direction): P = D K D with K_ij = w * HG(Omega_i . Omega_j; g_eff) (Eq. 11), unit row
 * and column sums, and mean cosine g.  *g_eff (may be NULL) receives g_eff. */
int trinity_phase_matrix(int nside, double g, double* out, size_t n, double* g_eff);

/* Ray-lattice tables of one grid: per direction dom axis and sign (int32 [N_a][2]),
 * sample spacing ds (double [N_a]) and per-slab transverse offsets
 * (int8 [N_a][2][max(nx,ny,nz)]). */
int trinity_lattice_tables(int nside, int nx, int ny, int nz, double h_mm, int periodic,
                           int32_t* dom_sgn, double* ds, int8_t* offsets, size_t n_offsets);

/* The interface split of trinity_set_fresnel for an n map ([nz][ny][nx] float32), as
 * entries (voxel, arriving direction j, receiving direction d, weight), sorted by voxel
 * then j; *count receives the number of entries.  Pass NULL outputs (or cap too small)
 * to query the count only. */
int trinity_interface_entries(int nside, int nx, int ny, int nz, double h_mm, int periodic,
                              const float* nmap, int* vox, int* j, int* d, double* w, size_t cap,
                              size_t* count);

/* Parent of every fine direction in the HEALPix hierarchy, out[12 nside_fine^2] (RING
 * index of the coarse pixel that contains the fine pixel's centre; Section 2.1 evaluates
 * the source function on coarse bins from the mean of their finer bins).  nside_fine
 * must be a multiple of nside_coarse. */
int trinity_parent_map(int nside_fine, int nside_coarse, int* out, size_t n);

/* Cone weights alpha_d (double [N_a]) of a face: the fraction of a cap of half_angle_deg
 * around the inward (inward = 1) or outward normal nearest to each direction. */
int trinity_cone_weights(int nside, int face, double half_angle_deg, int inward, double* out,
                         size_t n);

#ifdef __cplusplus
}
#endif

#endif /* TRINITY_H */
