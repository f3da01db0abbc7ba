// C ABI of the forward model (declared in include/trinity.h): context lifetime, inputs,
// the per-step launch sequence, CUDA-graph replay and read-backs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <string>
#include <vector>

#include "device.cuh"
#include "host_tables.h"
#include "trinity.h"

using namespace trinity;

struct trinity_ctx {
  trinity_grid_desc desc{};
  cudaStream_t stream = nullptr;
  int device = 0;
  GridParams g{};
  double dt = 0.0;
  double w = 0.0;
  double g_aniso = 0.0;
  std::vector<double> dirs;  // [na][3]
  Lattice lat;
  std::vector<DirInfo> hdirs;
  bool optics_set = false;
  bool locked = false;  // inputs are frozen once the first step has been queued
  bool has_init = false;
  std::string err;

  // detectors
  struct Det {
    int face;
    std::vector<int> vox;
    std::vector<double> weight;  // per direction, alpha * Omega_cap * cos_out
  };
  std::vector<Det> dets;
  double bin_ps = 10.0;
  int nbins = 0;

  // device buffers
  float *I = nullptr, *S = nullptr, *Q = nullptr;
  float *mut = nullptr, *eps = nullptr, *nidx = nullptr;
  float* d_rcorr32 = nullptr;
  float* P32 = nullptr;
  uint16_t* Pbf = nullptr;
  DirInfo* d_dirs = nullptr;
  int8_t* d_offs = nullptr;
  int *d_det_vox = nullptr, *d_det_dir = nullptr, *d_det_id = nullptr;
  float* d_det_w = nullptr;
  int n_det_entries = 0;
  double* d_det = nullptr;
  // run state
  int* d_step = nullptr;
  unsigned* d_smax = nullptr;
  int* d_nonconv = nullptr;
  int* d_error = nullptr;
  int* d_tile_ctr = nullptr;
  float* d_rcorr = nullptr;
  uint8_t* d_cls = nullptr;
  float* d_cls_ds = nullptr;
  int ncls = 0;
  int* d_iters_max = nullptr;
  unsigned long long* d_iters_sum = nullptr;
  unsigned long long* d_tile_iters = nullptr;
  double* d_energy = nullptr;
  double* d_escaped = nullptr;
  double* d_absorbed = nullptr;
  double* d_residual = nullptr;
  double* d_balance = nullptr;   // [1] running photon balance (see advance_kernel)
  double energy_init = 0.0;      // energy of the state before step 0
  int* d_refl = nullptr;         // [na][8] reflected directions (mirror faces)
  int* d_bins = nullptr;
  int capacity = 0;
  int steps_done = 0;  // steps queued so far
  int nonconv_seen = 0;

  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  // TMA-staged sweep (uniform n, vacuum faces, nx % 4 == 0): tensor maps of the rings and
  // the directions of each dominant-axis class
  bool tma = false;
  // BF16 iteration: TMA descriptors of the I and S rings for the tiles' write-out
  alignas(64) unsigned char out_maps[256] = {};
  bool tma_out = false;
  cudaStream_t side[2] = {nullptr, nullptr};  // the TMA sweep's classes run concurrently
  bool tma_off = false;                       // trinity_set_sweep_tma(ctx, 0)
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  SweepMaps maps{};
  int* d_dlist[3] = {nullptr, nullptr, nullptr};
  int ndir[3] = {0, 0, 0};
  int8_t* d_hsh = nullptr;  // per direction: bit 0 / 1 set when its y / z lattice offsets are positive
  GridParams graph_g{}, graph_gs{};  // the parameters the captured kernels were given

  // two-level angular grid: S on na_s coarse directions, each the mean of nch children
  int na_s = 0;              // directions of S (= g.na on one grid)
  int nch = 1;               // children per coarse direction (1 on one grid)
  bool two_level = false;
  GridParams g_s{};          // the scatter's view: na = na_s, energy weight of a coarse bin
  int* d_children = nullptr; // [na_s][nch] fine directions of each coarse one (ascending)
  float* d_b1ds = nullptr;   // [na_s][nch] ray spacings whose b1 the scatter averages
  float* Qc = nullptr;       // [na_s][N_v] mean Q over each coarse bin's children
  float* Ic = nullptr;       // [5][na_s][N_v] coarse mean intensity (written by the scatter)

  // exact per-voxel source function for piecewise-uniform optics
  bool exact = false;
  int exact_mode = 0;          // 1: tensor-core form where it applies, 2: FP32 SIMT form
  bool exact_tc = false;       // the tensor-core form runs
  int n_xcls = 0;
  float* d_Mimg = nullptr;     // [classes][6 chunks][hi, lo][192][32] operator images (tensor-core form)
  uint8_t* d_tmask = nullptr;  // [128-voxel tiles] classes present in each tile
  alignas(64) unsigned char qmap[128] = {};  // TMA descriptor of Q (tensor-core form)
  float* d_Mt = nullptr;       // [classes][na][na] operators M = (I - a P B1)^-1 a P, transposed
  float* d_b1tab = nullptr;    // [classes][na] b1 of each class and direction
  float* d_xmua = nullptr;     // [classes] mu_a of each class (absorbed-energy tally)
  uint8_t* d_xcls = nullptr;   // [nv] optics class of each voxel
  std::vector<float> h_P32, h_rc32, h_mut, h_eps;  // host copies the operators are built from

  // index interfaces (Eqs. 13-14)
  bool fresnel = false;
  std::vector<float> nmap;  // host copy of the refractive-index map
  int n_iface = 0;
  int *d_if_vox = nullptr, *d_if_rowptr = nullptr, *d_if_src = nullptr;
  float* d_if_w = nullptr;
  uint8_t* d_if_keep = nullptr;
  // the transposed split F^T in the same gather form (rows indexed by the crossing direction)
  int *d_ift_rowptr = nullptr, *d_ift_src = nullptr;
  float* d_ift_w = nullptr;

  // adjoint: checkpoints of a checkpointed run and the reverse-sweep buffers
  int ck_every = 0, ck_steps = 0, n_ckpt = 0;  // checkpoints at 0, every, ..., and at ck_steps
  bool ck_valid = false;
  float* d_ckpt = nullptr;          // [n_ckpt][I levels c-4..c-1, S levels c-4..c-1][na][nv]
  unsigned* d_ckpt_smax = nullptr;  // [n_ckpt] max |S(c-1)|
  float *d_stI = nullptr, *d_stS = nullptr;  // segment store [every + 4][na][nv]
  float *d_aI = nullptr, *d_aS = nullptr;    // adjoint levels Ibar, Sbar [5][na][nv]
  float *d_Qb = nullptr, *d_Y = nullptr;     // Qbar; [2] y of the last two reverse steps (warm start)
  double *d_gA = nullptr, *d_gmut = nullptr, *d_gmua = nullptr, *d_gmus = nullptr, *d_G = nullptr;
  unsigned* d_ymax = nullptr;       // [2] max |y| of the last two reverse steps
  int* d_adj_nonconv = nullptr;
  unsigned long long* d_adj_iters = nullptr;  // iterations of the transposed solves, summed
  // tallies of the recomputed forward steps go here, not into the run's own
  int* d_re_iters_max = nullptr;
  unsigned long long* d_re_iters_sum = nullptr;
  double *d_re_energy = nullptr, *d_re_escaped = nullptr, *d_re_det = nullptr;
  double *d_re_absorbed = nullptr, *d_re_residual = nullptr, *d_re_balance = nullptr;
  int* d_re_nonconv = nullptr;
  int re_capacity = 0;
};

namespace {

int fail(trinity_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? TRINITY_E_OOM : TRINITY_E_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

bool desc_valid(const trinity_grid_desc* d, std::string* why) {
  if (!d) {
    *why = "null description";
    return false;
  }
  if (d->nx < 2 || d->ny < 2 || d->nz < 2) {
    *why = "every grid axis needs at least 2 voxels";
    return false;
  }
  if (static_cast<long long>(d->nx) * d->ny * d->nz > (1LL << 30)) {
    *why = "grid too large";
    return false;
  }
  if (d->nx > 127 * 1024 || d->ny > 127 * 1024 || d->nz > 127 * 1024) {
    *why = "grid axis too long";
    return false;
  }
  if (!(d->h_mm > 0.0) || !(d->courant > 0.0) || !(d->n_ref >= 1.0)) {
    *why = "h_mm, courant must be > 0 and n_ref >= 1";
    return false;
  }
  const int ns = d->nside_scatter == 0 ? d->nside : d->nside_scatter;
  if (ns == d->nside) {
    if (d->nside != 1 && d->nside != 2 && d->nside != 4) {
      *why = "nside must be 1, 2 or 4";
      return false;
    }
  } else if ((ns != 1 && ns != 2 && ns != 4) ||
             (d->nside != 2 && d->nside != 4 && d->nside != 8 && d->nside != 16) ||
             d->nside % ns != 0 || d->nside < ns || (d->nside / ns) * (d->nside / ns) > 64) {
    *why = "two-level grid: nside_scatter 1, 2 or 4 and nside 2..16 a multiple of it";
    return false;
  }
  if (d->boundary != TRINITY_BOUNDARY_VACUUM && d->boundary != TRINITY_BOUNDARY_PERIODIC &&
      d->boundary != TRINITY_BOUNDARY_MIRROR) {
    *why = "unknown boundary";
    return false;
  }
  if (d->precision != TRINITY_FP32 && d->precision != TRINITY_BF16) {
    *why = "unknown precision";
    return false;
  }
  if (!(d->tol > 0.0) || d->max_iters < 1) {
    *why = "tol must be > 0 and max_iters >= 1";
    return false;
  }
  return true;
}

size_t footprint(const trinity_grid_desc* d) {
  const size_t nv = static_cast<size_t>(d->nx) * d->ny * d->nz;
  const size_t na = 12u * d->nside * d->nside;
  const int nsc = d->nside_scatter == 0 ? d->nside : d->nside_scatter;
  const size_t na_s = 12u * nsc * nsc;
  size_t b = 0;
  b += kRing * na * nv * sizeof(float);        // I history
  b += kRing * na_s * nv * sizeof(float);      // S history
  b += na * nv * sizeof(float);                // Q
  if (na_s != na) b += (kRing + 1) * na_s * nv * sizeof(float);  // coarse I history, Qbar
  b += 3 * nv * sizeof(float);                 // optics
  b += na_s * na_s * (sizeof(float) + sizeof(uint16_t));
  return b;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

RunState run_state(trinity_ctx* c) {
  RunState rs;
  rs.step = c->d_step;
  rs.smax = c->d_smax;
  rs.iters_max = c->d_iters_max;
  rs.iters_sum = c->d_iters_sum;
  rs.tile_iters = c->d_tile_iters;
  rs.energy = c->d_energy;
  rs.escaped = c->d_escaped;
  rs.absorbed = c->d_absorbed;
  rs.residual = c->d_residual;
  rs.balance = c->d_balance;
  rs.nonconv = c->d_nonconv;
  rs.bins = c->d_bins;
  rs.error = c->d_error;
  rs.tile_ctr = c->d_tile_ctr;
  return rs;
}

// Per-step arrays sized for ``need`` steps (regrown by doubling; drops the graph).
int ensure_capacity(trinity_ctx* ctx, int need) {
  if (need <= ctx->capacity) return TRINITY_OK;
  int cap = std::max(256, ctx->capacity);
  while (cap < need) cap *= 2;
  int* im = nullptr;
  unsigned long long *is = nullptr, *ti = nullptr;
  double *en = nullptr, *es = nullptr, *ab = nullptr, *re = nullptr;
  int* bins = nullptr;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(dalloc(&im, cap));
  CK(dalloc(&is, cap));
  CK(dalloc(&ti, cap));
  CK(dalloc(&en, cap));
  CK(dalloc(&es, cap));
  CK(dalloc(&ab, cap));
  CK(dalloc(&re, cap));
  CK(dalloc(&bins, cap));
  // clears and copies on the context's stream: ordered with the kernels that follow
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(ti, 0, cap * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(im, 0, cap * sizeof(int), st));
  CK(cudaMemsetAsync(is, 0, cap * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(en, 0, cap * sizeof(double), st));
  CK(cudaMemsetAsync(es, 0, cap * sizeof(double), st));
  CK(cudaMemsetAsync(ab, 0, cap * sizeof(double), st));
  CK(cudaMemsetAsync(re, 0, cap * sizeof(double), st));
  if (ctx->capacity > 0) {
    const size_t c0 = static_cast<size_t>(ctx->capacity);
    CK(cudaMemcpyAsync(im, ctx->d_iters_max, c0 * sizeof(int), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(is, ctx->d_iters_sum, c0 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ti, ctx->d_tile_iters, c0 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(en, ctx->d_energy, c0 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(es, ctx->d_escaped, c0 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ab, ctx->d_absorbed, c0 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(re, ctx->d_residual, c0 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    cudaFree(ctx->d_iters_max);
    cudaFree(ctx->d_iters_sum);
    cudaFree(ctx->d_tile_iters);
    cudaFree(ctx->d_energy);
    cudaFree(ctx->d_escaped);
    cudaFree(ctx->d_absorbed);
    cudaFree(ctx->d_residual);
    cudaFree(ctx->d_bins);
  }
  // detector bin of every step: floor((n + 1/2) dt / bin), integers snapped (FP64)
  std::vector<int> hb(cap);
  const double bw = ctx->bin_ps * 1e-3;
  for (int n = 0; n < cap; ++n) {
    const long b = floor_snap((n + 0.5) * ctx->dt / bw);
    hb[n] = (b >= 0 && b < ctx->nbins) ? static_cast<int>(b) : -1;
  }
  CK(cudaMemcpyAsync(bins, hb.data(), cap * sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  ctx->d_iters_max = im;
  ctx->d_iters_sum = is;
  ctx->d_tile_iters = ti;
  ctx->d_energy = en;
  ctx->d_escaped = es;
  ctx->d_absorbed = ab;
  ctx->d_residual = re;
  ctx->d_bins = bins;
  ctx->capacity = cap;
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  return TRINITY_OK;
}

// Freeze the inputs: upload detector entries and bins before the first step.
int lock_inputs(trinity_ctx* ctx) {
  if (ctx->locked) return TRINITY_OK;
  if (!ctx->optics_set) return fail(ctx, TRINITY_E_STATE, "set_optics must come before stepping");
  std::vector<int> vox, dir, id;
  std::vector<float> wt;
  const double h2dt = ctx->desc.h_mm * ctx->desc.h_mm * ctx->dt;
  for (size_t k = 0; k < ctx->dets.size(); ++k)
    for (int v : ctx->dets[k].vox)
      for (int d = 0; d < ctx->g.na; ++d)
        if (ctx->dets[k].weight[d] != 0.0) {
          vox.push_back(v);
          dir.push_back(d);
          id.push_back(static_cast<int>(k));
          wt.push_back(static_cast<float>(ctx->dets[k].weight[d] * h2dt));
        }
  ctx->n_det_entries = static_cast<int>(vox.size());
  CK(dalloc(&ctx->d_det_vox, vox.size()));
  CK(dalloc(&ctx->d_det_dir, dir.size()));
  CK(dalloc(&ctx->d_det_id, id.size()));
  CK(dalloc(&ctx->d_det_w, wt.size()));
  if (!vox.empty()) {
    CK(cudaMemcpy(ctx->d_det_vox, vox.data(), vox.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_det_dir, dir.data(), dir.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_det_id, id.data(), id.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_det_w, wt.data(), wt.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  const size_t ndet = ctx->dets.size() * static_cast<size_t>(std::max(ctx->nbins, 1));
  CK(dalloc(&ctx->d_det, ndet));
  CK(cudaMemset(ctx->d_det, 0, ndet * sizeof(double)));
  CK(cudaMemcpy(ctx->d_dirs, ctx->hdirs.data(), ctx->hdirs.size() * sizeof(DirInfo),
                cudaMemcpyHostToDevice));
  // the photon balance starts from the energy of the state held before step 0
  ctx->energy_init = 0.0;
  if (ctx->has_init) {
    const size_t nv = ctx->g.nv, na = ctx->g.na;
    std::vector<float> I0(na * nv);
    CK(cudaMemcpy(I0.data(), ctx->I + static_cast<size_t>(ring_slot(-1)) * na * nv, na * nv * 4,
                  cudaMemcpyDeviceToHost));
    double e = 0.0;
    for (size_t v = 0; v < nv; ++v) {
      double sv = 0.0;
      for (size_t d = 0; d < na; ++d) sv += I0[d * nv + v];
      e += sv * ctx->nmap[v];
    }
    ctx->energy_init = e * static_cast<double>(ctx->g.e_scale);  // the factor the kernels use
  }
  CK(cudaMemcpy(ctx->d_balance, &ctx->energy_init, sizeof(double), cudaMemcpyHostToDevice));
  ctx->locked = true;
  return TRINITY_OK;
}

BfTables bf_tables(trinity_ctx* c) {
  BfTables t;
  t.rcorr = c->d_rcorr;
  t.cls = c->d_cls;
  t.cls_ds = c->d_cls_ds;
  t.ncls = c->ncls;
  t.nch = c->nch;
  t.out_maps = c->tma_out ? c->out_maps : nullptr;
  return t;
}

void free_interfaces(trinity_ctx* c) {
  cudaFree(c->d_if_vox);
  cudaFree(c->d_if_rowptr);
  cudaFree(c->d_if_src);
  cudaFree(c->d_if_w);
  cudaFree(c->d_if_keep);
  cudaFree(c->d_ift_rowptr);
  cudaFree(c->d_ift_src);
  cudaFree(c->d_ift_w);
  c->d_if_vox = c->d_if_rowptr = c->d_if_src = nullptr;
  c->d_ift_rowptr = c->d_ift_src = nullptr;
  c->d_if_w = nullptr;
  c->d_ift_w = nullptr;
  c->d_if_keep = nullptr;
  c->n_iface = 0;
}

// Build and upload the interface table from the current n map (host FP64 decisions).
int build_interface_table(trinity_ctx* ctx) {
  free_interfaces(ctx);
  if (!ctx->fresnel || ctx->nmap.empty()) return TRINITY_OK;
  InterfaceTable T;
  try {
    T = build_interfaces(ctx->dirs, ctx->lat, ctx->g.nx, ctx->g.ny, ctx->g.nz, ctx->desc.h_mm,
                         ctx->g.periodic != 0, ctx->nmap);
  } catch (const std::exception& e) {
    return fail(ctx, TRINITY_E_INVALID, e.what());
  }
  ctx->n_iface = static_cast<int>(T.vox.size());
  if (ctx->n_iface == 0) return TRINITY_OK;
  CK(dalloc(&ctx->d_if_vox, T.vox.size()));
  CK(dalloc(&ctx->d_if_rowptr, T.rowptr.size()));
  CK(dalloc(&ctx->d_if_src, T.src.size()));
  CK(dalloc(&ctx->d_if_w, T.w.size()));
  CK(dalloc(&ctx->d_if_keep, T.keep.size()));
  CK(cudaMemcpy(ctx->d_if_vox, T.vox.data(), T.vox.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_if_rowptr, T.rowptr.data(), T.rowptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!T.src.empty()) {
    CK(cudaMemcpy(ctx->d_if_src, T.src.data(), T.src.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_if_w, T.w.data(), T.w.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(ctx->d_if_keep, T.keep.data(), T.keep.size(), cudaMemcpyHostToDevice));
  // F^T: out[j] = keep[j] q[j] + sum over the entries (j -> d, w) of w q[d]
  const int na = ctx->g.na;
  std::vector<int> trp, tsrc;
  std::vector<float> tw;
  for (size_t i = 0; i < T.vox.size(); ++i) {
    std::vector<std::vector<std::pair<int, float>>> rows(na);
    for (int d = 0; d < na; ++d)
      for (int e = T.rowptr[i * (na + 1) + d]; e < T.rowptr[i * (na + 1) + d + 1]; ++e)
        rows[T.src[e]].push_back({d, T.w[e]});
    for (int j = 0; j < na; ++j) {
      trp.push_back(static_cast<int>(tsrc.size()));
      for (const auto& e : rows[j]) {
        tsrc.push_back(e.first);
        tw.push_back(e.second);
      }
    }
    trp.push_back(static_cast<int>(tsrc.size()));
  }
  CK(dalloc(&ctx->d_ift_rowptr, trp.size()));
  CK(dalloc(&ctx->d_ift_src, tsrc.size()));
  CK(dalloc(&ctx->d_ift_w, tw.size()));
  CK(cudaMemcpy(ctx->d_ift_rowptr, trp.data(), trp.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!tsrc.empty()) {
    CK(cudaMemcpy(ctx->d_ift_src, tsrc.data(), tsrc.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_ift_w, tw.data(), tw.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  return TRINITY_OK;
}

void free_adjoint(trinity_ctx* c) {
  void* bufs[] = {c->d_ckpt,      c->d_ckpt_smax,   c->d_stI,         c->d_stS,
                  c->d_aI,        c->d_aS,          c->d_Qb,          c->d_Y,
                  c->d_gA,        c->d_gmut,        c->d_gmua,        c->d_gmus,
                  c->d_G,         c->d_ymax,        c->d_adj_nonconv, c->d_re_iters_max,
                  c->d_re_iters_sum, c->d_re_energy, c->d_re_escaped, c->d_re_det,
                  c->d_re_nonconv, c->d_adj_iters, c->d_re_absorbed, c->d_re_residual,
                  c->d_re_balance};
  for (void* p : bufs)
    if (p) cudaFree(p);
  c->d_ckpt = c->d_stI = c->d_stS = c->d_aI = c->d_aS = c->d_Qb = c->d_Y = nullptr;
  c->d_ckpt_smax = c->d_ymax = nullptr;
  c->d_gA = c->d_gmut = c->d_gmua = c->d_gmus = c->d_G = nullptr;
  c->d_re_energy = c->d_re_escaped = c->d_re_det = nullptr;
  c->d_re_absorbed = c->d_re_residual = c->d_re_balance = nullptr;
  c->d_adj_nonconv = c->d_re_iters_max = c->d_re_nonconv = nullptr;
  c->d_re_iters_sum = c->d_adj_iters = nullptr;
  c->re_capacity = 0;
  c->ck_valid = false;
  c->n_ckpt = c->ck_every = c->ck_steps = 0;
}

size_t adjoint_bytes(size_t na, size_t nv, int nsteps, int every, int ndet_bins) {
  const size_t lvl = na * nv * sizeof(float);
  const size_t nck = static_cast<size_t>((nsteps + every - 1) / every) + 1;
  size_t b = nck * 8 * lvl + nck * sizeof(unsigned);  // checkpoints
  b += static_cast<size_t>(every + 4) * 2 * lvl;      // segment store
  b += 13 * lvl;                                      // adjoint levels, Qbar, two warm-start levels
  b += 4 * nv * sizeof(double);                       // gradient sums and outputs
  b += static_cast<size_t>(ndet_bins) * 2 * sizeof(double) +
       static_cast<size_t>(nsteps) * (2 * sizeof(double) + sizeof(int) + sizeof(unsigned long long));
  return b;
}

// Copy levels c-4..c-1 of I and S (ring slots) into checkpoint k, with max |S(c-1)|.
int save_checkpoint(trinity_ctx* ctx, int k, int c) {
  const size_t lvl = static_cast<size_t>(ctx->g.na) * ctx->g.nv;
  float* base = ctx->d_ckpt + static_cast<size_t>(k) * 8 * lvl;
  for (int j = 0; j < 4; ++j) {
    const size_t slot = static_cast<size_t>(ring_slot(c - 4 + j));
    CK(cudaMemcpyAsync(base + j * lvl, ctx->I + slot * lvl, lvl * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(base + (4 + j) * lvl, ctx->S + slot * lvl, lvl * 4, cudaMemcpyDeviceToDevice,
                       ctx->stream));
  }
  CK(cudaMemcpyAsync(ctx->d_ckpt_smax + k, ctx->d_smax + ((c - 1) & 1), sizeof(unsigned),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  return TRINITY_OK;
}

// Put checkpoint k (taken before step c) back into the ring, the step counter and smax;
// with ``store`` also into the first four levels of the segment store.
int restore_checkpoint(trinity_ctx* ctx, int k, int c, bool store) {
  const size_t lvl = static_cast<size_t>(ctx->g.na) * ctx->g.nv;
  const float* base = ctx->d_ckpt + static_cast<size_t>(k) * 8 * lvl;
  for (int j = 0; j < 4; ++j) {
    const size_t slot = static_cast<size_t>(ring_slot(c - 4 + j));
    CK(cudaMemcpyAsync(ctx->I + slot * lvl, base + j * lvl, lvl * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->S + slot * lvl, base + (4 + j) * lvl, lvl * 4, cudaMemcpyDeviceToDevice,
                       ctx->stream));
    if (store) {
      CK(cudaMemcpyAsync(ctx->d_stI + j * lvl, base + j * lvl, lvl * 4, cudaMemcpyDeviceToDevice,
                         ctx->stream));
      CK(cudaMemcpyAsync(ctx->d_stS + j * lvl, base + (4 + j) * lvl, lvl * 4, cudaMemcpyDeviceToDevice,
                         ctx->stream));
    }
  }
  CK(launch_adj_restore(ctx->d_step, c, ctx->d_smax, ctx->d_ckpt_smax + k, ctx->stream));
  return TRINITY_OK;
}

// Sweep (Eq. 10's known part Q) and the interface split; on a two-level grid also the
// mean of Q over each coarse direction's children.
// The step's sweep stages its upwind planes through the TMA: supported box, uniform
// refractive index (one retarded delay per direction), not switched off.
bool sweep_uses_tma(const trinity_ctx* ctx) {
  return !ctx->two_level && ctx->tma && !ctx->tma_off && ctx->g.n_u >= 1.0f;
}

int enqueue_transport(trinity_ctx* ctx, const RunState& rs) {
  const GridParams& g = ctx->g;
  if (ctx->two_level) {
    CK(launch_sweep2(g, ctx->d_dirs, ctx->d_offs, ctx->d_children, ctx->nch, ctx->na_s, ctx->I, ctx->S,
                     ctx->mut, ctx->nidx, ctx->Q, ctx->Qc, rs, ctx->stream));
  } else if (sweep_uses_tma(ctx)) {
    const int* dl[3] = {ctx->d_dlist[0], ctx->d_dlist[1], ctx->d_dlist[2]};
    // the three dominant-axis classes on the context's stream and two side streams (forked
    // and joined by events, so a captured step holds them as parallel graph nodes)
    const cudaStream_t st3[3] = {ctx->stream, ctx->side[0], ctx->side[1]};
    CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
    for (int k = 0; k < 2; ++k) CK(cudaStreamWaitEvent(ctx->side[k], ctx->ev_fork, 0));
    CK(launch_sweep_tma(g, ctx->d_dirs, dl, ctx->ndir, ctx->d_offs, ctx->d_hsh, ctx->maps, ctx->mut, ctx->Q, rs,
                        st3));
    for (int k = 0; k < 2; ++k) {
      CK(cudaEventRecord(ctx->ev_join[k], ctx->side[k]));
      CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join[k], 0));
    }
  } else {
    CK(launch_sweep(g, ctx->d_dirs, ctx->d_offs, ctx->I, ctx->S, ctx->mut, ctx->nidx, ctx->d_refl, ctx->Q, rs,
                    ctx->stream));
  }
  CK(launch_interface(ctx->n_iface, g.na, ctx->d_if_vox, ctx->d_if_rowptr, ctx->d_if_src, ctx->d_if_w,
                      ctx->d_if_keep, ctx->Q, g.nv, ctx->stream));
  if (ctx->two_level)
    CK(launch_recoarsen(ctx->n_iface, ctx->d_if_vox, ctx->d_children, ctx->nch, ctx->na_s, ctx->Q, ctx->Qc,
                        g.nv, ctx->stream));
  return TRINITY_OK;
}

// The per-voxel source iteration (Eq. 12) on the source function's directions.
int enqueue_scatter(trinity_ctx* ctx, const RunState& rs) {
  const GridParams& gs = ctx->g_s;
  if (ctx->exact && ctx->exact_tc) {
    CK(launch_exact_tc(gs, ctx->qmap, ctx->d_Mimg, ctx->d_tmask, ctx->d_b1tab, ctx->n_xcls, ctx->d_xcls,
                       ctx->d_xmua, ctx->Qc, ctx->nidx, ctx->Ic, ctx->S, rs, ctx->stream));
  } else if (ctx->exact) {
    CK(launch_exact_fp32(gs, ctx->d_b1ds, ctx->nch, ctx->d_Mt, ctx->d_b1tab, ctx->d_xcls, ctx->d_xmua, ctx->Qc,
                         ctx->mut, ctx->nidx, ctx->Ic, ctx->S, rs, ctx->stream));
  } else if (ctx->desc.precision == TRINITY_BF16) {
    CK(launch_scatter_bf16(gs, bf_tables(ctx), ctx->Pbf, ctx->Qc, ctx->mut, ctx->eps, ctx->nidx, ctx->Ic,
                           ctx->S, static_cast<float>(ctx->desc.tol), ctx->desc.max_iters, rs,
                           ctx->stream));
  } else {
    CK(launch_scatter_fp32(gs, ctx->d_b1ds, ctx->nch, ctx->P32, ctx->d_rcorr32, ctx->Qc, ctx->mut, ctx->eps,
                           ctx->nidx, ctx->Ic, ctx->S, static_cast<float>(ctx->desc.tol), ctx->desc.max_iters,
                           rs, ctx->stream));
  }
  return TRINITY_OK;
}

// I on the transport directions (two-level grid), the tallies and the step counter.
int enqueue_finish(trinity_ctx* ctx, const RunState& rs, double* det) {
  const GridParams& g = ctx->g;
  if (ctx->two_level)
    CK(launch_refine(g, ctx->d_dirs, ctx->d_children, ctx->nch, ctx->na_s, ctx->mut, ctx->Q, ctx->S, ctx->I,
                     rs, ctx->stream));
  CK(launch_tally(g, ctx->d_dirs, ctx->I, ctx->d_det_vox, ctx->d_det_dir, ctx->d_det_w,
                  ctx->d_det_id, ctx->n_det_entries, det, ctx->nbins, rs, ctx->stream));
  CK(launch_advance(ctx->g, rs, ctx->stream));
  return TRINITY_OK;
}

// The launches of one time step (all on ctx->stream; the step index lives on the device).
// ``rs`` and ``det`` take the step's tallies.
int enqueue_step_with(trinity_ctx* ctx, const RunState& rs, double* det) {
  int rc = enqueue_transport(ctx, rs);
  if (rc == TRINITY_OK) rc = enqueue_scatter(ctx, rs);
  if (rc == TRINITY_OK) rc = enqueue_finish(ctx, rs, det);
  return rc;
}

int enqueue_step(trinity_ctx* ctx) { return enqueue_step_with(ctx, run_state(ctx), ctx->d_det); }

int check_device_error(trinity_ctx* ctx) {
  int e = 0;
  CK(cudaMemcpy(&e, ctx->d_error, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) return fail(ctx, TRINITY_E_TIMEOUT, "a bounded device wait ran out (code " + std::to_string(e) + ")");
  return TRINITY_OK;
}

uint16_t to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;  // round to nearest even (inputs are finite)
  return static_cast<uint16_t>(u >> 16);
}

constexpr int kMaxExactClasses = 8;

// Optics classes and their exact operators M = (I - a P~ B1)^-1 a P~ (FP64 solve; P~ is
// the FP32 phase matrix plus its diagonal correction, the matrix the iteration applies).
int build_exact(trinity_ctx* ctx) {
  if (!ctx->exact || !ctx->optics_set) return TRINITY_OK;
  if (ctx->two_level)
    return fail(ctx, TRINITY_E_UNSUPPORTED, "the exact solve covers one angular grid (nside_scatter = nside)");
  const int na = ctx->g.na;
  const size_t nv = ctx->g.nv;
  std::vector<std::pair<uint64_t, int>> keys;
  std::vector<uint8_t> cls(nv);
  std::vector<std::pair<float, float>> pairs;
  for (size_t v = 0; v < nv; ++v) {
    uint32_t a, b;
    std::memcpy(&a, &ctx->h_mut[v], 4);
    std::memcpy(&b, &ctx->h_eps[v], 4);
    const uint64_t key = (static_cast<uint64_t>(a) << 32) | b;
    size_t k = 0;
    while (k < keys.size() && keys[k].first != key) ++k;
    if (k == keys.size()) {
      if (keys.size() == kMaxExactClasses)
        return fail(ctx, TRINITY_E_UNSUPPORTED,
                    "the exact solve needs piecewise-uniform optics: more than 8 distinct (mu_t, mu_a/mu_t) pairs");
      keys.push_back({key, static_cast<int>(k)});
      pairs.push_back({ctx->h_mut[v], ctx->h_eps[v]});
    }
    cls[v] = static_cast<uint8_t>(k);
  }
  std::vector<double> Pt(static_cast<size_t>(na) * na);
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < na; ++j)
      Pt[static_cast<size_t>(i) * na + j] =
          static_cast<double>(ctx->h_P32[static_cast<size_t>(i) * na + j]) + (i == j ? double(ctx->h_rc32[i]) : 0.0);
  std::vector<float> Mt(pairs.size() * static_cast<size_t>(na) * na);
  std::vector<double> Mall(pairs.size() * static_cast<size_t>(na) * na);
  std::vector<float> b1tab(pairs.size() * static_cast<size_t>(na));
  for (size_t c = 0; c < pairs.size(); ++c) {
    const double mt = pairs[c].first, a = 1.0 - static_cast<double>(pairs[c].second);
    std::vector<double> A(static_cast<size_t>(na) * na), B(static_cast<size_t>(na) * na);
    std::vector<double> b1(na);
    for (int d = 0; d < na; ++d) {
      b1[d] = ray_b1_fp64(mt * static_cast<double>(static_cast<float>(ctx->lat.ds[d])));
      b1tab[c * na + d] = static_cast<float>(b1[d]);
    }
    for (int i = 0; i < na; ++i)
      for (int j = 0; j < na; ++j) {
        const double p = Pt[static_cast<size_t>(i) * na + j];
        A[static_cast<size_t>(i) * na + j] = (i == j ? 1.0 : 0.0) - a * p * b1[j];
        B[static_cast<size_t>(i) * na + j] = a * p;
      }
    std::vector<double> M;
    try {
      M = solve_dense(A, B, na);
    } catch (const std::exception& e) {
      return fail(ctx, TRINITY_E_INVALID, e.what());
    }
    for (int i = 0; i < na; ++i)
      for (int j = 0; j < na; ++j) {
        Mt[(c * na + j) * static_cast<size_t>(na) + i] = static_cast<float>(M[static_cast<size_t>(i) * na + j]);
        Mall[(c * na + i) * static_cast<size_t>(na) + j] = M[static_cast<size_t>(i) * na + j];
      }
  }
  // mu_a of each class, formed as the iteration kernels form it (eps * mu_t in FP32)
  std::vector<float> xmua(pairs.size());
  for (size_t c = 0; c < pairs.size(); ++c) xmua[c] = pairs[c].second * pairs[c].first;
  cudaFree(ctx->d_Mt);
  cudaFree(ctx->d_xcls);
  cudaFree(ctx->d_b1tab);
  cudaFree(ctx->d_xmua);
  ctx->d_Mt = nullptr;
  ctx->d_xcls = nullptr;
  ctx->d_b1tab = nullptr;
  ctx->d_xmua = nullptr;
  CK(dalloc(&ctx->d_Mt, Mt.size()));
  CK(dalloc(&ctx->d_xcls, nv));
  CK(dalloc(&ctx->d_b1tab, b1tab.size()));
  CK(dalloc(&ctx->d_xmua, xmua.size()));
  CK(cudaMemcpy(ctx->d_xmua, xmua.data(), xmua.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_Mt, Mt.data(), Mt.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_b1tab, b1tab.data(), b1tab.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_xcls, cls.data(), nv, cudaMemcpyHostToDevice));
  ctx->n_xcls = static_cast<int>(pairs.size());
  // the tensor-core form: operator images, per-tile class masks and Q's TMA descriptor
  cudaFree(ctx->d_Mimg);
  cudaFree(ctx->d_tmask);
  ctx->d_Mimg = nullptr;
  ctx->d_tmask = nullptr;
  ctx->exact_tc = false;
  if (ctx->exact_mode != 2 && exact_tc_supported(ctx->g_s, ctx->n_xcls) &&
      make_exact_qmap(ctx->g_s, ctx->Qc, ctx->qmap) == cudaSuccess) {
    std::vector<float> img;
    std::vector<uint8_t> mask;
    exact_tc_images(Mall.data(), ctx->n_xcls, &img);
    exact_tc_tile_masks(cls.data(), static_cast<int>(nv), &mask);
    CK(dalloc(&ctx->d_Mimg, img.size()));
    CK(dalloc(&ctx->d_tmask, mask.size()));
    CK(cudaMemcpy(ctx->d_Mimg, img.data(), img.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_tmask, mask.data(), mask.size(), cudaMemcpyHostToDevice));
    ctx->exact_tc = true;
  }
  return TRINITY_OK;
}

}  // namespace

extern "C" {

size_t trinity_footprint_bytes(const trinity_grid_desc* desc) {
  std::string why;
  if (!desc_valid(desc, &why)) return 0;
  return footprint(desc);
}

int trinity_create_grid(const trinity_grid_desc* desc, void* cuda_stream, trinity_ctx** out) {
  if (!out) return TRINITY_E_INVALID;
  *out = nullptr;
  std::string why;
  if (!desc_valid(desc, &why)) return TRINITY_E_INVALID;
  trinity_ctx* ctx = nullptr;
  try {
    ctx = new trinity_ctx();
  } catch (...) {
    return TRINITY_E_OOM;
  }
  auto bail = [&](int code) {
    trinity_destroy(ctx);
    return code;
  };
  ctx->desc = *desc;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(TRINITY_E_CUDA);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess) return bail(TRINITY_E_CUDA);
  if (!(prop.major == 10 && prop.minor == 3)) return bail(TRINITY_E_UNSUPPORTED);
  const int nside_s = desc->nside_scatter == 0 ? desc->nside : desc->nside_scatter;
  if (desc->precision == TRINITY_BF16 && !scatter_bf16_supported(12 * nside_s * nside_s))
    return bail(TRINITY_E_UNSUPPORTED);

  GridParams& g = ctx->g;
  g.nx = desc->nx;
  g.ny = desc->ny;
  g.nz = desc->nz;
  g.nv = desc->nx * desc->ny * desc->nz;
  g.na = 12 * desc->nside * desc->nside;
  g.periodic = desc->boundary == TRINITY_BOUNDARY_PERIODIC;
  g.mirror = desc->boundary == TRINITY_BOUNDARY_MIRROR;
  g.hist_from = 0;
  g.src_voxel = -1;
  g.pulse_steps = 0;
  g.h = static_cast<float>(desc->h_mm);
  ctx->dt = desc->courant * desc->h_mm * desc->n_ref / kC0;
  ctx->w = 4.0 * 3.14159265358979323846 / g.na;
  g.e_scale = static_cast<float>(desc->h_mm * desc->h_mm * desc->h_mm / kC0 * ctx->w);
  g.a_scale = desc->h_mm * desc->h_mm * desc->h_mm * ctx->dt * ctx->w;
  g.inj_step = 0.0;
  g.mut_u = -1.0f;
  g.n_u = 0.0f;
  try {
    ctx->dirs = healpix_dirs(desc->nside);
    ctx->lat = build_lattice(ctx->dirs, g.nx, g.ny, g.nz, desc->h_mm, g.periodic != 0);
  } catch (const std::exception& e) {
    return bail(TRINITY_E_INVALID);
  }
  g.nmax = ctx->lat.nmax;
  double dsmax = 0.0;
  ctx->hdirs.resize(g.na);
  const double h2dt = desc->h_mm * desc->h_mm * ctx->dt;
  for (int d = 0; d < g.na; ++d) {
    DirInfo& di = ctx->hdirs[d];
    std::memset(&di, 0, sizeof(di));
    di.dom = ctx->lat.dom[d];
    di.sgn = ctx->lat.sgn[d];
    int j = 0, ax[2];
    for (int a = 0; a < 3; ++a)
      if (a != di.dom) ax[j++] = a;
    di.a0 = ax[0];
    di.a1 = ax[1];
    di.ds = static_cast<float>(ctx->lat.ds[d]);
    const double dc = ctx->lat.ds[d] / (kC0 * ctx->dt);
    di.dcoef = static_cast<float>(dc);
    di.dcoef_lo = static_cast<float>(dc - static_cast<double>(di.dcoef));
    dsmax = std::max(dsmax, ctx->lat.ds[d]);
    for (int f = 0; f < 6; ++f) {
      const double c = ((f % 2) ? 1.0 : -1.0) * ctx->dirs[3 * d + f / 2];
      di.wcos_out[f] = c > 0 ? static_cast<float>(ctx->w * c * h2dt) : 0.0f;
    }
  }
  g.ds_max = static_cast<float>(dsmax);

  // angular grids: S and the source iteration on na_s directions; on a two-level grid
  // each coarse direction c owns the nch fine directions whose centres it contains
  ctx->na_s = 12 * nside_s * nside_s;
  ctx->two_level = ctx->na_s != g.na;
  std::vector<int> children;   // [na_s][nch]
  std::vector<float> b1ds;     // [na_s][nch]
  if (ctx->two_level) {
    std::vector<int> par;
    try {
      par = parent_map(desc->nside, nside_s);
    } catch (const std::exception&) {
      return bail(TRINITY_E_INVALID);
    }
    ctx->nch = g.na / ctx->na_s;
    std::vector<int> fill(ctx->na_s, 0);
    children.assign(static_cast<size_t>(ctx->na_s) * ctx->nch, -1);
    for (int f = 0; f < g.na; ++f) {  // ascending fine index within each coarse bin
      const int c = par[f];
      if (fill[c] >= ctx->nch) return bail(TRINITY_E_INVALID);
      children[static_cast<size_t>(c) * ctx->nch + fill[c]++] = f;
    }
  } else {
    ctx->nch = 1;
    children.resize(g.na);
    for (int d = 0; d < g.na; ++d) children[d] = d;
  }
  b1ds.resize(children.size());
  for (size_t k = 0; k < children.size(); ++k) b1ds[k] = static_cast<float>(ctx->lat.ds[children[k]]);
  g.warm = 1;  // the iteration starts from 2 S(n-1) - S(n-2) (trinity_set_warm_start)
  ctx->g_s = g;
  ctx->g_s.na = ctx->na_s;
  ctx->g_s.e_scale = static_cast<float>(desc->h_mm * desc->h_mm * desc->h_mm / kC0 *
                                        (4.0 * 3.14159265358979323846 / ctx->na_s));
  ctx->g_s.a_scale = desc->h_mm * desc->h_mm * desc->h_mm * ctx->dt * (4.0 * 3.14159265358979323846 / ctx->na_s);
  if (g.mirror && ctx->two_level) return bail(TRINITY_E_UNSUPPORTED);  // the two-level sweep has no images

  const size_t nv = g.nv, na = g.na, na_s = ctx->na_s;
  if (dalloc(&ctx->I, kRing * na * nv) != cudaSuccess || dalloc(&ctx->S, kRing * na_s * nv) != cudaSuccess ||
      dalloc(&ctx->Q, na * nv) != cudaSuccess || dalloc(&ctx->mut, nv) != cudaSuccess ||
      dalloc(&ctx->eps, nv) != cudaSuccess || dalloc(&ctx->nidx, nv) != cudaSuccess ||
      dalloc(&ctx->P32, na_s * na_s) != cudaSuccess || dalloc(&ctx->Pbf, na_s * na_s) != cudaSuccess ||
      dalloc(&ctx->d_dirs, na) != cudaSuccess ||
      dalloc(&ctx->d_offs, ctx->lat.off.size()) != cudaSuccess || dalloc(&ctx->d_step, 1) != cudaSuccess ||
      dalloc(&ctx->d_smax, 2) != cudaSuccess || dalloc(&ctx->d_nonconv, 1) != cudaSuccess ||
      dalloc(&ctx->d_error, 1) != cudaSuccess || dalloc(&ctx->d_tile_ctr, 2) != cudaSuccess ||
      dalloc(&ctx->d_balance, 1) != cudaSuccess || (g.mirror && dalloc(&ctx->d_refl, 8 * na) != cudaSuccess) ||
      dalloc(&ctx->d_rcorr, na_s) != cudaSuccess || dalloc(&ctx->d_rcorr32, na_s) != cudaSuccess ||
      dalloc(&ctx->d_cls, na_s) != cudaSuccess || dalloc(&ctx->d_cls_ds, 16 * ctx->nch) != cudaSuccess ||
      dalloc(&ctx->d_children, children.size()) != cudaSuccess ||
      dalloc(&ctx->d_b1ds, b1ds.size()) != cudaSuccess ||
      (ctx->two_level && (dalloc(&ctx->Qc, na_s * nv) != cudaSuccess ||
                          dalloc(&ctx->Ic, kRing * na_s * nv) != cudaSuccess))) {
    cudaGetLastError();
    return bail(TRINITY_E_OOM);
  }
  if (!ctx->two_level) {
    ctx->Qc = ctx->Q;  // one grid: the scatter reads Q and writes I directly
    ctx->Ic = ctx->I;
  }
  if (desc->precision == TRINITY_BF16) {
    ctx->tma_out = make_scatter_out_maps(ctx->g_s, ctx->Ic, ctx->S, ctx->out_maps) == cudaSuccess;
    if (!ctx->tma_out) cudaGetLastError();  // plain stores
  }
  if (g.mirror) {
    // refl[d][mask]: the direction of Omega_d with the components of the axes in mask
    // negated (the HEALPix pixel set is symmetric under every face reflection)
    std::vector<int> refl(8 * na);
    for (size_t d = 0; d < na; ++d)
      for (int mask = 0; mask < 8; ++mask) {
        double t[3];
        for (int a = 0; a < 3; ++a) t[a] = ctx->dirs[3 * d + a] * (((mask >> a) & 1) ? -1.0 : 1.0);
        int best = -1;
        double bd = -2.0;
        for (size_t e = 0; e < na; ++e) {
          const double dot = t[0] * ctx->dirs[3 * e] + t[1] * ctx->dirs[3 * e + 1] + t[2] * ctx->dirs[3 * e + 2];
          if (dot > bd) {
            bd = dot;
            best = static_cast<int>(e);
          }
        }
        if (bd < 1.0 - 1e-12) return bail(TRINITY_E_INVALID);
        refl[d * 8 + mask] = best;
      }
    if (cudaMemcpy(ctx->d_refl, refl.data(), refl.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(TRINITY_E_CUDA);
  }
  if (cudaMemcpy(ctx->d_offs, ctx->lat.off.data(), ctx->lat.off.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(ctx->d_children, children.data(), children.size() * sizeof(int), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(ctx->d_b1ds, b1ds.data(), b1ds.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(TRINITY_E_CUDA);
  {
    // classes of equal ray-sample spacing (the tensor-core kernel tabulates b1 per class);
    // on a two-level grid a class is the list of a coarse direction's children spacings
    const int nch = ctx->nch;
    std::vector<uint8_t> cls(na_s);
    std::vector<std::vector<float>> cds;
    for (size_t c = 0; c < na_s; ++c) {
      std::vector<float> key(b1ds.begin() + c * nch, b1ds.begin() + (c + 1) * nch);
      std::sort(key.begin(), key.end());
      size_t k = 0;
      while (k < cds.size() && cds[k] != key) ++k;
      if (k == cds.size()) cds.push_back(key);
      cls[c] = static_cast<uint8_t>(k < 255 ? k : 255);
    }
    ctx->ncls = static_cast<int>(cds.size());
    if (desc->precision == TRINITY_BF16 && ctx->ncls > 16) return bail(TRINITY_E_UNSUPPORTED);
    std::vector<float> flat(16 * static_cast<size_t>(nch), 0.0f);
    for (size_t k = 0; k < cds.size() && k < 16; ++k)
      std::copy(cds[k].begin(), cds[k].end(), flat.begin() + k * nch);
    if (cudaMemcpy(ctx->d_cls, cls.data(), na_s, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->d_cls_ds, flat.data(), flat.size() * sizeof(float), cudaMemcpyHostToDevice) !=
            cudaSuccess)
      return bail(TRINITY_E_CUDA);
  }
  if (!ctx->two_level && sweep_tma_supported(g)) {
    // directions of each dominant-axis class, for the TMA-staged sweep
    std::vector<int> cl[3];
    for (int d = 0; d < g.na; ++d) cl[ctx->lat.dom[d]].push_back(d);
    bool ok = make_sweep_maps(g, ctx->I, ctx->S, &ctx->maps) == cudaSuccess;
    for (int c = 0; c < 3 && ok; ++c) {
      ctx->ndir[c] = static_cast<int>(cl[c].size());
      ok = dalloc(&ctx->d_dlist[c], cl[c].size()) == cudaSuccess &&
           (cl[c].empty() || cudaMemcpy(ctx->d_dlist[c], cl[c].data(), cl[c].size() * sizeof(int),
                                        cudaMemcpyHostToDevice) == cudaSuccess);
    }
    // the sign of each transverse lattice offset (all offsets of a direction and axis share it)
    std::vector<int8_t> hsh(g.na, 0);
    for (int d = 0; d < g.na; ++d)
      for (int j = 0; j < 2; ++j)
        for (int k = 0; k < g.nmax; ++k)
          if (ctx->lat.off[(static_cast<size_t>(d) * 2 + j) * g.nmax + k] > 0) hsh[d] |= static_cast<int8_t>(1 << j);
    ok = ok && dalloc(&ctx->d_hsh, hsh.size()) == cudaSuccess &&
         cudaMemcpy(ctx->d_hsh, hsh.data(), hsh.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k)
      ok = cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&ctx->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    ctx->tma = ok;
    if (!ok) cudaGetLastError();  // fall back to the plain-load sweep
  }
  if (trinity_reset(ctx) != TRINITY_OK) return bail(TRINITY_E_CUDA);
  *out = ctx;
  return TRINITY_OK;
}

int trinity_set_optics(trinity_ctx* ctx, const float* mua, const float* mus, const float* n, double g,
                       int ptr_kind) {
  if (!ctx) return TRINITY_E_INVALID;
  if (!mua || !mus || !n || (ptr_kind != 0 && ptr_kind != 1))
    return fail(ctx, TRINITY_E_INVALID, "null optics pointer or bad ptr_kind");
  if (!(g > -1.0 && g < 1.0)) return fail(ctx, TRINITY_E_INVALID, "g must lie in (-1, 1)");
  const size_t nv = ctx->g.nv;
  std::vector<float> a(nv), s(nv), r(nv);
  if (ptr_kind == 1) {
    CK(cudaMemcpy(a.data(), mua, nv * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(s.data(), mus, nv * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(r.data(), n, nv * 4, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(a.data(), mua, nv * 4);
    std::memcpy(s.data(), mus, nv * 4);
    std::memcpy(r.data(), n, nv * 4);
  }
  double nmin = 1e30, nmax = -1e30, dsmin = 1e30, dsmax = 0.0;
  for (double ds : ctx->lat.ds) {
    dsmin = std::min(dsmin, ds);
    dsmax = std::max(dsmax, ds);
  }
  std::vector<float> mt(nv), al(nv);  // al: eps = mu_a / mu_t (1 where mu_t = 0)
  for (size_t v = 0; v < nv; ++v) {
    if (!(a[v] >= 0.0f) || !(s[v] >= 0.0f) || !std::isfinite(a[v]) || !std::isfinite(s[v]) ||
        !(r[v] >= 1.0f) || !std::isfinite(r[v]))
      return fail(ctx, TRINITY_E_INVALID, "optics need mu_a, mu_s >= 0 and n >= 1, finite");
    nmin = std::min(nmin, double(r[v]));
    nmax = std::max(nmax, double(r[v]));
    mt[v] = a[v] + s[v];
    const double t64 = static_cast<double>(a[v]) + static_cast<double>(s[v]);
    al[v] = t64 > 0.0 ? static_cast<float>(static_cast<double>(a[v]) / t64) : 1.0f;
  }
  const double dlo = dsmin * nmin / (kC0 * ctx->dt), dhi = dsmax * nmax / (kC0 * ctx->dt);
  if (dlo < 1.0 || dhi >= kRing - 1)
    return fail(ctx, TRINITY_E_INVALID,
                "retarded delay outside [1, 4) steps: choose courant so that c dt < h |Omega_dom|");
  std::vector<double> P;
  try {
    P = phase_matrix(ctx->desc.nside_scatter == 0 ? ctx->desc.nside : ctx->desc.nside_scatter, g, nullptr);
  } catch (const std::exception& e) {
    return fail(ctx, TRINITY_E_INVALID, e.what());
  }
  std::vector<float> P32(P.size());
  std::vector<uint16_t> Pb(P.size());
  for (size_t k = 0; k < P.size(); ++k) {
    P32[k] = static_cast<float>(P[k]);
    Pb[k] = to_bf16(P32[k]);
  }
  // diagonal correction that gives bf16(P) + diag(r) unit row and column sums
  const int na = ctx->na_s;
  std::vector<float> rc(na);
  for (int i = 0; i < na; ++i) {
    double rs = 0.0;
    for (int j = 0; j < na; ++j) {
      const uint32_t u = static_cast<uint32_t>(Pb[static_cast<size_t>(i) * na + j]) << 16;
      float f;
      std::memcpy(&f, &u, 4);
      rs += f;
    }
    rc[i] = static_cast<float>(1.0 - rs);
  }
  CK(cudaMemcpy(ctx->d_rcorr, rc.data(), na * sizeof(float), cudaMemcpyHostToDevice));
  // the same correction for the FP32 matrix of the plain mode
  for (int i = 0; i < na; ++i) {
    double rs = 0.0;
    for (int j = 0; j < na; ++j) rs += P32[static_cast<size_t>(i) * na + j];
    rc[i] = static_cast<float>(1.0 - rs);
  }
  CK(cudaMemcpy(ctx->d_rcorr32, rc.data(), na * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->mut, mt.data(), nv * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->eps, al.data(), nv * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->nidx, r.data(), nv * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->P32, P32.data(), P32.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->Pbf, Pb.data(), Pb.size() * 2, cudaMemcpyHostToDevice));
  ctx->g_aniso = g;
  ctx->optics_set = true;
  // A uniform mu_t or n lets the sweeps take exp, b0, b1 and the retarded delay once per
  // direction instead of once per voxel (the same FP32 operations on the same values).
  const auto same_bits = [](const std::vector<float>& x) {
    return std::all_of(x.begin(), x.end(), [&](float y) { return std::memcmp(&y, &x[0], 4) == 0; });
  };
  ctx->g.mut_u = same_bits(mt) ? mt[0] : -1.0f;
  ctx->g.n_u = same_bits(r) ? r[0] : 0.0f;
  ctx->g_s.mut_u = ctx->g.mut_u;
  ctx->g_s.n_u = ctx->g.n_u;
  ctx->nmap = r;

  ctx->h_P32 = P32;
  ctx->h_rc32 = rc;
  ctx->h_mut = mt;
  ctx->h_eps = al;
  {
    const int rc3 = build_exact(ctx);
    if (rc3 != TRINITY_OK) return rc3;
  }
  {
    const int rc2 = build_interface_table(ctx);
    if (rc2 != TRINITY_OK) return rc2;
  }
  if (ctx->locked) return trinity_reset(ctx);
  return TRINITY_OK;
}

int trinity_set_optics_uniform(trinity_ctx* ctx, double mua, double mus, double g, double n) {
  if (!ctx) return TRINITY_E_INVALID;
  const size_t nv = ctx->g.nv;
  std::vector<float> a(nv, float(mua)), s(nv, float(mus)), r(nv, float(n));
  return trinity_set_optics(ctx, a.data(), s.data(), r.data(), g, 0);
}

int trinity_set_fresnel(trinity_ctx* ctx, int on) {
  if (!ctx) return TRINITY_E_INVALID;
  if (ctx->locked) return fail(ctx, TRINITY_E_STATE, "interfaces must be set before the first step");
  ctx->fresnel = on != 0;
  return build_interface_table(ctx);
}

int trinity_set_exact_solve(trinity_ctx* ctx, int on) {
  if (!ctx) return TRINITY_E_INVALID;
  if (ctx->locked) return fail(ctx, TRINITY_E_STATE, "the exact solve must be chosen before the first step");
  if (on < 0 || on > 2) return fail(ctx, TRINITY_E_INVALID, "exact solve: on must be 0, 1 or 2");
  ctx->exact = on != 0;
  ctx->exact_mode = on;
  const int rc = build_exact(ctx);
  if (rc != TRINITY_OK) {
    ctx->exact = false;
    ctx->exact_tc = false;
  }
  return rc;
}

int trinity_exact_classes(const trinity_ctx* ctx, int* n) {
  if (!ctx || !n) return TRINITY_E_INVALID;
  *n = ctx->exact ? ctx->n_xcls : 0;
  return TRINITY_OK;
}

int trinity_set_warm_start(trinity_ctx* ctx, int mode) {
  if (!ctx) return TRINITY_E_INVALID;
  if (mode != 0 && mode != 1) return fail(ctx, TRINITY_E_INVALID, "warm start: mode must be 0 or 1");
  if (ctx->locked) return fail(ctx, TRINITY_E_STATE, "the warm start must be chosen before the first step");
  ctx->g.warm = mode;
  ctx->g_s.warm = mode;
  return TRINITY_OK;
}

int trinity_exact_form(const trinity_ctx* ctx, int* form) {
  if (!ctx || !form) return TRINITY_E_INVALID;
  *form = !ctx->exact || !ctx->optics_set ? 0 : (ctx->exact_tc ? 1 : 2);
  return TRINITY_OK;
}

int trinity_interface_count(const trinity_ctx* ctx, int* n) {
  if (!ctx || !n) return TRINITY_E_INVALID;
  *n = ctx->n_iface;
  return TRINITY_OK;
}

int trinity_set_source(trinity_ctx* ctx, int face, double u_mm, double v_mm, double half_angle_deg,
                       int pulse_steps, double energy) {
  if (!ctx) return TRINITY_E_INVALID;
  if (ctx->locked) return fail(ctx, TRINITY_E_STATE, "source must be set before the first step");
  if (ctx->g.periodic || ctx->g.mirror) return fail(ctx, TRINITY_E_INVALID, "a source needs vacuum boundaries");
  if (face < 0 || face > 5 || pulse_steps < 1 || !(energy >= 0.0))
    return fail(ctx, TRINITY_E_INVALID, "bad face, pulse_steps or energy");
  const int nn[3] = {ctx->g.nx, ctx->g.ny, ctx->g.nz};
  const int ax = face / 2;
  const int ua = ax == 0 ? 1 : 0, va = ax == 2 ? 1 : 2;
  const long iu = static_cast<long>(std::floor(u_mm / ctx->desc.h_mm));
  const long iv = static_cast<long>(std::floor(v_mm / ctx->desc.h_mm));
  if (iu < 0 || iu >= nn[ua] || iv < 0 || iv >= nn[va])
    return fail(ctx, TRINITY_E_INVALID, "source point outside the face");
  std::vector<double> alpha;
  try {
    alpha = cone_weights(ctx->dirs, face, half_angle_deg, true);
  } catch (const std::exception& e) {
    return fail(ctx, TRINITY_E_INVALID, e.what());
  }
  const double h = ctx->desc.h_mm;
  const int entry_sgn = (face % 2 == 0) ? 1 : -1;
  double inj = 0.0;
  for (int d = 0; d < ctx->g.na; ++d) {
    ctx->hdirs[d].src_amp = 0.0f;
    if (alpha[d] == 0.0) continue;
    const double cos_in = -((face % 2) ? 1.0 : -1.0) * ctx->dirs[3 * d + ax];
    if (ctx->lat.dom[d] != ax || ctx->lat.sgn[d] != entry_sgn || !(cos_in > 0.0))
      return fail(ctx, TRINITY_E_INVALID, "source cone reaches a direction that does not enter through the face");
    const double amp = energy * alpha[d] / (ctx->w * cos_in * h * h * pulse_steps * ctx->dt);
    ctx->hdirs[d].src_amp = static_cast<float>(amp);
    // the energy the FP32 amplitude actually carries in per pulse step
    inj += static_cast<double>(ctx->hdirs[d].src_amp) * ctx->w * cos_in * h * h * ctx->dt;
  }
  ctx->g.inj_step = inj;
  int c[3];
  c[ax] = (face % 2) ? nn[ax] - 1 : 0;
  c[ua] = static_cast<int>(iu);
  c[va] = static_cast<int>(iv);
  ctx->g.src_voxel = (c[2] * nn[1] + c[1]) * nn[0] + c[0];
  ctx->g.pulse_steps = pulse_steps;
  return TRINITY_OK;
}

int trinity_add_detector(trinity_ctx* ctx, int face, double u_mm, double v_mm, double radius_mm,
                         double half_angle_deg, int* det_id) {
  if (!ctx) return TRINITY_E_INVALID;
  if (ctx->locked) return fail(ctx, TRINITY_E_STATE, "detectors must be added before the first step");
  if (face < 0 || face > 5 || !(radius_mm > 0.0)) return fail(ctx, TRINITY_E_INVALID, "bad face or radius");
  trinity_ctx::Det det;
  det.face = face;
  try {
    const std::vector<double> alpha = cone_weights(ctx->dirs, face, half_angle_deg, false);
    const double cap = 2.0 * 3.14159265358979323846 * (1.0 - std::cos(half_angle_deg * 3.14159265358979323846 / 180.0));
    const int ax = face / 2;
    const double sgn = (face % 2) ? 1.0 : -1.0;
    det.weight.assign(ctx->g.na, 0.0);
    for (int d = 0; d < ctx->g.na; ++d) {
      if (alpha[d] == 0.0) continue;
      const double c = sgn * ctx->dirs[3 * d + ax];
      if (!(c > 0.0)) return fail(ctx, TRINITY_E_INVALID, "detector cone reaches an incoming direction");
      det.weight[d] = alpha[d] * cap * c;
    }
  } catch (const std::exception& e) {
    return fail(ctx, TRINITY_E_INVALID, e.what());
  }
  const int nn[3] = {ctx->g.nx, ctx->g.ny, ctx->g.nz};
  const int ax = face / 2;
  const int ua = ax == 0 ? 1 : 0, va = ax == 2 ? 1 : 2;
  const double h = ctx->desc.h_mm;
  for (int iu = 0; iu < nn[ua]; ++iu)
    for (int iv = 0; iv < nn[va]; ++iv) {
      const double du = (iu + 0.5) * h - u_mm, dv = (iv + 0.5) * h - v_mm;
      if (du * du + dv * dv <= radius_mm * radius_mm * (1.0 + 1e-12)) {
        int c[3];
        c[ax] = (face % 2) ? nn[ax] - 1 : 0;
        c[ua] = iu;
        c[va] = iv;
        det.vox.push_back((c[2] * nn[1] + c[1]) * nn[0] + c[0]);
      }
    }
  std::sort(det.vox.begin(), det.vox.end());
  ctx->dets.push_back(det);
  if (det_id) *det_id = static_cast<int>(ctx->dets.size()) - 1;
  return TRINITY_OK;
}

int trinity_set_bins(trinity_ctx* ctx, double bin_ps, int nbins) {
  if (!ctx) return TRINITY_E_INVALID;
  if (ctx->locked) return fail(ctx, TRINITY_E_STATE, "bins must be set before the first step");
  if (!(bin_ps > 0.0) || nbins < 1) return fail(ctx, TRINITY_E_INVALID, "bad bin width or count");
  ctx->bin_ps = bin_ps;
  ctx->nbins = nbins;
  if (ctx->capacity > 0) {  // rebuild the bin table for the new width
    const int cap = ctx->capacity;
    ctx->capacity = 0;
    cudaFree(ctx->d_iters_max);
    cudaFree(ctx->d_iters_sum);
    cudaFree(ctx->d_tile_iters);
    cudaFree(ctx->d_energy);
    cudaFree(ctx->d_escaped);
    cudaFree(ctx->d_absorbed);
    cudaFree(ctx->d_residual);
    cudaFree(ctx->d_bins);
    ctx->d_iters_max = nullptr;
    ctx->d_iters_sum = nullptr;
    ctx->d_tile_iters = nullptr;
    ctx->d_energy = nullptr;
    ctx->d_escaped = nullptr;
    ctx->d_absorbed = nullptr;
    ctx->d_residual = nullptr;
    ctx->d_bins = nullptr;
    return ensure_capacity(ctx, cap);
  }
  return TRINITY_OK;
}

int trinity_set_initial_state(trinity_ctx* ctx, const float* I0, const float* S0, int ptr_kind) {
  if (!ctx) return TRINITY_E_INVALID;
  if (ctx->locked || ctx->steps_done > 0) return fail(ctx, TRINITY_E_STATE, "initial state must precede the first step");
  if (!I0 || !S0 || (ptr_kind != 0 && ptr_kind != 1)) return fail(ctx, TRINITY_E_INVALID, "bad initial state");
  const size_t cnt = static_cast<size_t>(ctx->g.na) * ctx->g.nv;
  const size_t cnt_s = static_cast<size_t>(ctx->na_s) * ctx->g.nv;
  const cudaMemcpyKind kind = ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int lev = -(kRing - 1); lev < 0; ++lev) {
    CK(cudaMemcpy(ctx->I + static_cast<size_t>(ring_slot(lev)) * cnt, I0, cnt * 4, kind));
    CK(cudaMemcpy(ctx->S + static_cast<size_t>(ring_slot(lev)) * cnt_s, S0, cnt_s * 4, kind));
  }
  std::vector<float> hs(cnt_s);
  CK(cudaMemcpy(hs.data(), S0, cnt_s * 4, ptr_kind ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
  float m = 0.0f;
  for (float x : hs) m = std::max(m, std::fabs(x));
  unsigned bits;
  std::memcpy(&bits, &m, 4);
  CK(cudaMemcpy(ctx->d_smax + 1, &bits, 4, cudaMemcpyHostToDevice));
  ctx->g.hist_from = -(kRing - 1);
  ctx->has_init = true;
  return TRINITY_OK;
}

int trinity_step(trinity_ctx* ctx, int nsteps, int* iters_out) {
  if (!ctx) return TRINITY_E_INVALID;
  if (nsteps < 0) return fail(ctx, TRINITY_E_INVALID, "nsteps < 0");
  int rc = lock_inputs(ctx);
  if (rc != TRINITY_OK) return rc;
  rc = ensure_capacity(ctx, ctx->steps_done + nsteps);
  if (rc != TRINITY_OK) return rc;
  for (int s = 0; s < nsteps; ++s) {
    rc = enqueue_step(ctx);
    if (rc != TRINITY_OK) return rc;
  }
  const int first = ctx->steps_done;
  ctx->steps_done += nsteps;
  CK(cudaStreamSynchronize(ctx->stream));
  rc = check_device_error(ctx);
  if (rc != TRINITY_OK) return rc;
  if (iters_out && nsteps > 0)
    CK(cudaMemcpy(iters_out, ctx->d_iters_max + first, nsteps * sizeof(int), cudaMemcpyDeviceToHost));
  int nc = 0;
  CK(cudaMemcpy(&nc, ctx->d_nonconv, sizeof(int), cudaMemcpyDeviceToHost));
  if (nc > ctx->nonconv_seen) {
    ctx->nonconv_seen = nc;
    ctx->err = "some voxels reached max_iters";
    return TRINITY_W_NOT_CONVERGED;
  }
  return TRINITY_OK;
}

int trinity_run(trinity_ctx* ctx, int nsteps) {
  if (!ctx) return TRINITY_E_INVALID;
  if (nsteps < 0) return fail(ctx, TRINITY_E_INVALID, "nsteps < 0");
  int rc = lock_inputs(ctx);
  if (rc != TRINITY_OK) return rc;
  rc = ensure_capacity(ctx, ctx->steps_done + nsteps);
  if (rc != TRINITY_OK) return rc;
  constexpr int kGraphSteps = 8;
  // kernels take the grid parameters by value: a change (e.g. an initial state after a
  // reset) needs a new capture
  if (ctx->graph && (std::memcmp(&ctx->graph_g, &ctx->g, sizeof(GridParams)) != 0 ||
                     std::memcmp(&ctx->graph_gs, &ctx->g_s, sizeof(GridParams)) != 0)) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  if (!ctx->graph) {
    cudaStream_t cap_stream;
    CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    cudaStream_t saved = ctx->stream;
    ctx->stream = cap_stream;
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
    int erc = TRINITY_OK;
    for (int s = 0; s < kGraphSteps && erc == TRINITY_OK; ++s) erc = enqueue_step(ctx);
    cudaError_t ce = cudaStreamEndCapture(cap_stream, &graph);
    ctx->stream = saved;
    cudaStreamDestroy(cap_stream);
    if (erc != TRINITY_OK) return erc;
    CK(ce);
    ce = cudaGraphInstantiate(&ctx->graph, graph, 0);
    cudaGraphDestroy(graph);
    CK(ce);
    ctx->graph_steps = kGraphSteps;
    ctx->graph_g = ctx->g;
    ctx->graph_gs = ctx->g_s;
  }
  int left = nsteps;
  while (left >= ctx->graph_steps) {
    CK(cudaGraphLaunch(ctx->graph, ctx->stream));
    left -= ctx->graph_steps;
  }
  for (int s = 0; s < left; ++s) {
    rc = enqueue_step(ctx);
    if (rc != TRINITY_OK) return rc;
  }
  ctx->steps_done += nsteps;
  return TRINITY_OK;
}

int trinity_profile_steps(trinity_ctx* ctx, int nsteps, double* kernel_ms) {
  if (!ctx || !kernel_ms) return TRINITY_E_INVALID;
  if (nsteps < 1) return fail(ctx, TRINITY_E_INVALID, "nsteps < 1");
  int rc = lock_inputs(ctx);
  if (rc != TRINITY_OK) return rc;
  rc = ensure_capacity(ctx, ctx->steps_done + nsteps);
  if (rc != TRINITY_OK) return rc;
  const RunState rs = run_state(ctx);
  std::vector<cudaEvent_t> ev(4 * static_cast<size_t>(nsteps));
  for (auto& e : ev) CK(cudaEventCreate(&e));
  for (int s = 0; s < nsteps; ++s) {
    cudaEvent_t* e = &ev[4 * static_cast<size_t>(s)];
    CK(cudaEventRecord(e[0], ctx->stream));
    rc = enqueue_transport(ctx, rs);
    if (rc != TRINITY_OK) return rc;
    CK(cudaEventRecord(e[1], ctx->stream));
    rc = enqueue_scatter(ctx, rs);
    if (rc != TRINITY_OK) return rc;
    CK(cudaEventRecord(e[2], ctx->stream));
    rc = enqueue_finish(ctx, rs, ctx->d_det);
    if (rc != TRINITY_OK) return rc;
    CK(cudaEventRecord(e[3], ctx->stream));
  }
  ctx->steps_done += nsteps;
  CK(cudaStreamSynchronize(ctx->stream));
  kernel_ms[0] = kernel_ms[1] = kernel_ms[2] = 0.0;
  for (int s = 0; s < nsteps; ++s) {
    for (int k = 0; k < 3; ++k) {
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, ev[4 * static_cast<size_t>(s) + k], ev[4 * static_cast<size_t>(s) + k + 1]));
      kernel_ms[k] += ms;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return check_device_error(ctx);
}

size_t trinity_adjoint_footprint_bytes(const trinity_grid_desc* desc, int nsteps, int every, int n_det,
                                       int nbins) {
  std::string why;
  if (!desc_valid(desc, &why) || nsteps < 1 || every < 1 || n_det < 0 || nbins < 1) return 0;
  const size_t nv = static_cast<size_t>(desc->nx) * desc->ny * desc->nz;
  const size_t na = 12u * desc->nside * desc->nside;
  return adjoint_bytes(na, nv, nsteps, std::min(every, nsteps), n_det * nbins);
}

int trinity_run_checkpointed(trinity_ctx* ctx, int nsteps, int every) {
  if (!ctx) return TRINITY_E_INVALID;
  if (nsteps < 1 || every < 1) return fail(ctx, TRINITY_E_INVALID, "nsteps and every must be >= 1");
  if (ctx->two_level)
    return fail(ctx, TRINITY_E_UNSUPPORTED, "the adjoint covers one angular grid (nside_scatter = nside)");
  if (ctx->g.mirror) return fail(ctx, TRINITY_E_UNSUPPORTED, "the adjoint covers vacuum and periodic boundaries");
  if (ctx->steps_done != 0)
    return fail(ctx, TRINITY_E_STATE, "a checkpointed run starts at step 0 (call trinity_reset)");
  int rc = lock_inputs(ctx);
  if (rc != TRINITY_OK) return rc;
  rc = ensure_capacity(ctx, nsteps);
  if (rc != TRINITY_OK) return rc;
  free_adjoint(ctx);
  every = std::min(every, nsteps);
  const size_t lvl = static_cast<size_t>(ctx->g.na) * ctx->g.nv;
  const int nseg = (nsteps + every - 1) / every;
  ctx->n_ckpt = nseg + 1;  // one before each segment and one after the last step
  if (dalloc(&ctx->d_ckpt, static_cast<size_t>(ctx->n_ckpt) * 8 * lvl) != cudaSuccess ||
      dalloc(&ctx->d_ckpt_smax, ctx->n_ckpt) != cudaSuccess) {
    cudaGetLastError();
    free_adjoint(ctx);
    return fail(ctx, TRINITY_E_OOM, "no device memory for the checkpoints");
  }
  for (int k = 0; k < nseg; ++k) {
    const int c = k * every;
    rc = save_checkpoint(ctx, k, c);
    if (rc != TRINITY_OK) return rc;
    const int K = std::min(every, nsteps - c);
    for (int s = 0; s < K; ++s) {
      rc = enqueue_step(ctx);
      if (rc != TRINITY_OK) return rc;
    }
  }
  rc = save_checkpoint(ctx, nseg, nsteps);
  if (rc != TRINITY_OK) return rc;
  ctx->steps_done = nsteps;
  ctx->ck_every = every;
  ctx->ck_steps = nsteps;
  ctx->ck_valid = true;
  return trinity_sync(ctx);
}

namespace {

// The reverse sweep.  With ``stats`` (7 doubles) each phase is bracketed by CUDA events
// on the context's stream and the summed device ms are returned: [0] checkpoint restores,
// [1] recomputed forward steps, [2] copies into the segment store, [3] detector injection
// and transposed solves, [4] transposed interface splits and upwind pushes, [5] the
// final gradient kernel; [6] = mean iterations of the transposed solves per voxel-step.
int adjoint_impl(trinity_ctx* ctx, const double* dL_dE, size_t n, double* grad_mua, double* grad_mus,
                 int ptr_kind, double* stats) {
  if (!ctx) return TRINITY_E_INVALID;
  if (!ctx->ck_valid || ctx->steps_done != ctx->ck_steps)
    return fail(ctx, TRINITY_E_STATE, "trinity_adjoint needs a completed trinity_run_checkpointed "
                                      "with no steps after it");
  const int ndb = static_cast<int>(ctx->dets.size()) * ctx->nbins;
  if (n != static_cast<size_t>(ndb) || (ndb > 0 && !dL_dE) || !grad_mua || !grad_mus ||
      (ptr_kind != 0 && ptr_kind != 1))
    return fail(ctx, TRINITY_E_INVALID, "bad adjoint arguments");
  const GridParams& g = ctx->g;
  const size_t nv = g.nv, lvl = static_cast<size_t>(g.na) * g.nv;
  const int N = ctx->ck_steps, every = ctx->ck_every;
  if (!ctx->d_stI) {
    bool ok = dalloc(&ctx->d_stI, static_cast<size_t>(every + 4) * lvl) == cudaSuccess &&
              dalloc(&ctx->d_stS, static_cast<size_t>(every + 4) * lvl) == cudaSuccess &&
              dalloc(&ctx->d_aI, kRing * lvl) == cudaSuccess && dalloc(&ctx->d_aS, kRing * lvl) == cudaSuccess &&
              dalloc(&ctx->d_Qb, lvl) == cudaSuccess && dalloc(&ctx->d_Y, 2 * lvl) == cudaSuccess &&
              dalloc(&ctx->d_gA, nv) == cudaSuccess && dalloc(&ctx->d_gmut, nv) == cudaSuccess &&
              dalloc(&ctx->d_gmua, nv) == cudaSuccess && dalloc(&ctx->d_gmus, nv) == cudaSuccess &&
              dalloc(&ctx->d_G, ndb) == cudaSuccess && dalloc(&ctx->d_ymax, 2) == cudaSuccess &&
              dalloc(&ctx->d_adj_nonconv, 1) == cudaSuccess && dalloc(&ctx->d_adj_iters, 1) == cudaSuccess &&
              dalloc(&ctx->d_re_iters_max, N) == cudaSuccess &&
              dalloc(&ctx->d_re_iters_sum, N) == cudaSuccess &&
              dalloc(&ctx->d_re_energy, N) == cudaSuccess && dalloc(&ctx->d_re_escaped, N) == cudaSuccess &&
              dalloc(&ctx->d_re_det, ndb) == cudaSuccess && dalloc(&ctx->d_re_nonconv, 1) == cudaSuccess &&
              dalloc(&ctx->d_re_absorbed, N) == cudaSuccess && dalloc(&ctx->d_re_residual, N) == cudaSuccess &&
              dalloc(&ctx->d_re_balance, 1) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return fail(ctx, TRINITY_E_OOM, "no device memory for the adjoint buffers");
    }
    ctx->re_capacity = N;
  }
  if (ndb > 0)
    CK(cudaMemcpyAsync(ctx->d_G, dL_dE, ndb * sizeof(double),
                       ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_aI, 0, kRing * lvl * 4, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_aS, 0, kRing * lvl * 4, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_Y, 0, 2 * lvl * 4, ctx->stream));  // y(n+1) and y(n+2) of the warm start
  CK(cudaMemsetAsync(ctx->d_gA, 0, nv * 8, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_gmut, 0, nv * 8, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_ymax, 0, 2 * sizeof(unsigned), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_adj_nonconv, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_adj_iters, 0, sizeof(unsigned long long), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_re_det, 0, std::max(ndb, 1) * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_re_iters_max, 0, N * sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_re_iters_sum, 0, N * sizeof(unsigned long long), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_re_energy, 0, N * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_re_escaped, 0, N * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_re_absorbed, 0, N * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_re_residual, 0, N * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_re_balance, 0, sizeof(double), ctx->stream));
  RunState rs = run_state(ctx);  // recomputed steps: same step counter, smax and bins
  rs.iters_max = ctx->d_re_iters_max;
  rs.iters_sum = ctx->d_re_iters_sum;
  rs.tile_iters = nullptr;
  rs.energy = ctx->d_re_energy;
  rs.escaped = ctx->d_re_escaped;
  rs.absorbed = ctx->d_re_absorbed;
  rs.residual = ctx->d_re_residual;
  rs.balance = ctx->d_re_balance;
  rs.nonconv = ctx->d_re_nonconv;
  const double bw = ctx->bin_ps * 1e-3;
  const float tol = static_cast<float>(ctx->desc.tol);
  const int nseg = ctx->n_ckpt - 1;
  // phase timing: one event before and one after each phase instance
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evs[6];
  auto mark = [&](int phase, bool start) -> cudaError_t {
    if (!stats) return cudaSuccess;
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    if (start)
      evs[phase].push_back({e, nullptr});
    else
      evs[phase].back().second = e;
    return cudaEventRecord(e, ctx->stream);
  };
  for (int k = nseg - 1; k >= 0; --k) {
    const int c = k * every;
    const int K = std::min(every, N - c);
    const int lev_base = c - 4;
    CK(mark(0, true));
    int rc = restore_checkpoint(ctx, k, c, true);
    if (rc != TRINITY_OK) return rc;
    CK(mark(0, false));
    for (int s = 0; s < K; ++s) {  // recompute the segment, keeping every level
      CK(mark(1, true));
      rc = enqueue_step_with(ctx, rs, ctx->d_re_det);
      if (rc != TRINITY_OK) return rc;
      CK(mark(1, false));
      const int lev = c + s;
      const size_t slot = static_cast<size_t>(ring_slot(lev));
      const size_t dst = static_cast<size_t>(lev - lev_base) * lvl;
      CK(mark(2, true));
      CK(cudaMemcpyAsync(ctx->d_stI + dst, ctx->I + slot * lvl, lvl * 4, cudaMemcpyDeviceToDevice, ctx->stream));
      CK(cudaMemcpyAsync(ctx->d_stS + dst, ctx->S + slot * lvl, lvl * 4, cudaMemcpyDeviceToDevice, ctx->stream));
      CK(mark(2, false));
    }
    for (int lev = c + K - 1; lev >= c; --lev) {
      const long b = floor_snap((lev + 0.5) * ctx->dt / bw);
      const int bin = (b >= 0 && b < ctx->nbins) ? static_cast<int>(b) : -1;
      float* aI_n = ctx->d_aI + static_cast<size_t>(ring_slot(lev)) * lvl;
      float* aS_n = ctx->d_aS + static_cast<size_t>(ring_slot(lev)) * lvl;
      const size_t here = static_cast<size_t>(lev - lev_base) * lvl;
      CK(mark(3, true));
      CK(launch_adj_inject(ctx->d_det_vox, ctx->d_det_dir, ctx->d_det_w, ctx->d_det_id, ctx->n_det_entries,
                           ctx->d_G, ctx->nbins, bin, aI_n, g.nv, ctx->d_ymax + (lev & 1), ctx->stream));
      CK(launch_adj_scatter_fp32(g, ctx->d_dirs, ctx->P32, ctx->d_rcorr32, ctx->mut, ctx->eps, aI_n, aS_n,
                                 ctx->d_stI + here, ctx->d_stS + here, ctx->d_Y,
                                 ctx->g.warm ? ctx->d_Y + lvl : nullptr, ctx->g.warm && lev <= N - 3 ? 1 : 0,
                                 ctx->d_Qb, ctx->d_gA,
                                 ctx->d_gmut, tol, ctx->desc.max_iters, ctx->d_ymax + ((lev + 1) & 1),
                                 ctx->d_ymax + (lev & 1), ctx->d_adj_nonconv, ctx->d_adj_iters,
                                 ctx->stream));
      CK(mark(3, false));
      CK(mark(4, true));
      CK(launch_interface(ctx->n_iface, g.na, ctx->d_if_vox, ctx->d_ift_rowptr, ctx->d_ift_src,
                          ctx->d_ift_w, ctx->d_if_keep, ctx->d_Qb, g.nv, ctx->stream));
      CK(launch_adj_push(g, ctx->d_dirs, ctx->d_offs, ctx->d_stI, ctx->d_stS, lev_base, lev, ctx->mut,
                         ctx->nidx, ctx->d_Qb, ctx->d_aI, ctx->d_aS, ctx->d_gmut, ctx->stream));
      CK(mark(4, false));
    }
  }
  // the forward state after the last step comes back, so stepping can continue
  CK(mark(0, true));
  {
    const int rc = restore_checkpoint(ctx, nseg, N, false);
    if (rc != TRINITY_OK) return rc;
  }
  CK(mark(0, false));
  CK(mark(5, true));
  CK(launch_adj_finish(g.nv, ctx->mut, ctx->eps, ctx->d_gA, ctx->d_gmut, ctx->d_gmua, ctx->d_gmus,
                       ctx->stream));
  CK(mark(5, false));
  CK(cudaStreamSynchronize(ctx->stream));
  if (stats) {
    for (int ph = 0; ph < 6; ++ph) {
      double tot = 0.0;
      for (auto& pr : evs[ph]) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, pr.first, pr.second));
        tot += ms;
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
      }
      stats[ph] = tot;
    }
    unsigned long long it = 0;
    CK(cudaMemcpy(&it, ctx->d_adj_iters, sizeof(it), cudaMemcpyDeviceToHost));
    stats[6] = static_cast<double>(it) / (static_cast<double>(N) * static_cast<double>(nv));
  }
  {
    const int rc = check_device_error(ctx);
    if (rc != TRINITY_OK) return rc;
  }
  const cudaMemcpyKind kind = ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpy(grad_mua, ctx->d_gmua, nv * sizeof(double), kind));
  CK(cudaMemcpy(grad_mus, ctx->d_gmus, nv * sizeof(double), kind));
  int nc = 0;
  CK(cudaMemcpy(&nc, ctx->d_adj_nonconv, sizeof(int), cudaMemcpyDeviceToHost));
  if (nc > 0) {
    ctx->err = "some voxels reached max_iters in the transposed solve";
    return TRINITY_W_NOT_CONVERGED;
  }
  return TRINITY_OK;
}

}  // namespace

int trinity_adjoint(trinity_ctx* ctx, const double* dL_dE, size_t n, double* grad_mua, double* grad_mus,
                    int ptr_kind) {
  return adjoint_impl(ctx, dL_dE, n, grad_mua, grad_mus, ptr_kind, nullptr);
}

int trinity_adjoint_profile(trinity_ctx* ctx, const double* dL_dE, size_t n, double* grad_mua,
                            double* grad_mus, int ptr_kind, double* stats) {
  if (!stats) return ctx ? fail(ctx, TRINITY_E_INVALID, "stats is null") : TRINITY_E_INVALID;
  return adjoint_impl(ctx, dL_dE, n, grad_mua, grad_mus, ptr_kind, stats);
}

int trinity_sync(trinity_ctx* ctx) {
  if (!ctx) return TRINITY_E_INVALID;
  CK(cudaStreamSynchronize(ctx->stream));
  int rc = check_device_error(ctx);
  if (rc != TRINITY_OK) return rc;
  int nc = 0;
  CK(cudaMemcpy(&nc, ctx->d_nonconv, sizeof(int), cudaMemcpyDeviceToHost));
  if (nc > ctx->nonconv_seen) {
    ctx->nonconv_seen = nc;
    ctx->err = "some voxels reached max_iters";
    return TRINITY_W_NOT_CONVERGED;
  }
  return TRINITY_OK;
}

int trinity_read_detectors(trinity_ctx* ctx, double* out, size_t n) {
  if (!ctx) return TRINITY_E_INVALID;
  const size_t want = ctx->dets.size() * static_cast<size_t>(ctx->nbins);
  if (n != want || (want > 0 && !out)) return fail(ctx, TRINITY_E_INVALID, "detector buffer size mismatch");
  if (want == 0) return TRINITY_OK;
  if (!ctx->locked) {
    std::fill(out, out + n, 0.0);
    return TRINITY_OK;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(out, ctx->d_det, want * sizeof(double), cudaMemcpyDeviceToHost));
  return TRINITY_OK;
}

int trinity_read_energy(trinity_ctx* ctx, double* N_t, double* escaped, double* absorbed, double* residual,
                        size_t nsteps) {
  if (!ctx) return TRINITY_E_INVALID;
  if (nsteps > static_cast<size_t>(ctx->steps_done)) return fail(ctx, TRINITY_E_INVALID, "more steps than done");
  if (nsteps == 0) return TRINITY_OK;
  const size_t first = ctx->steps_done - nsteps;
  CK(cudaStreamSynchronize(ctx->stream));
  const size_t b = nsteps * sizeof(double);
  if (N_t) CK(cudaMemcpy(N_t, ctx->d_energy + first, b, cudaMemcpyDeviceToHost));
  if (escaped) CK(cudaMemcpy(escaped, ctx->d_escaped + first, b, cudaMemcpyDeviceToHost));
  if (absorbed) CK(cudaMemcpy(absorbed, ctx->d_absorbed + first, b, cudaMemcpyDeviceToHost));
  if (residual) CK(cudaMemcpy(residual, ctx->d_residual + first, b, cudaMemcpyDeviceToHost));
  return TRINITY_OK;
}

int trinity_read_iterations(trinity_ctx* ctx, int* iters_max, double* iters_mean, size_t nsteps) {
  if (!ctx) return TRINITY_E_INVALID;
  if (nsteps > static_cast<size_t>(ctx->steps_done)) return fail(ctx, TRINITY_E_INVALID, "more steps than done");
  if (nsteps == 0) return TRINITY_OK;
  const size_t first = ctx->steps_done - nsteps;
  CK(cudaStreamSynchronize(ctx->stream));
  if (iters_max) CK(cudaMemcpy(iters_max, ctx->d_iters_max + first, nsteps * sizeof(int), cudaMemcpyDeviceToHost));
  if (iters_mean) {
    std::vector<unsigned long long> s(nsteps);
    CK(cudaMemcpy(s.data(), ctx->d_iters_sum + first, nsteps * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < nsteps; ++k) iters_mean[k] = double(s[k]) / double(ctx->g.nv);
  }
  return TRINITY_OK;
}

int trinity_read_executed_iterations(trinity_ctx* ctx, double* executed_mean, size_t nsteps) {
  if (!ctx || !executed_mean) return TRINITY_E_INVALID;
  if (nsteps > static_cast<size_t>(ctx->steps_done)) return fail(ctx, TRINITY_E_INVALID, "more steps than done");
  if (nsteps == 0) return TRINITY_OK;
  const size_t first = ctx->steps_done - nsteps;
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<unsigned long long> t(nsteps);
  CK(cudaMemcpy(t.data(), ctx->d_tile_iters + first, nsteps * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  for (size_t k2 = 0; k2 < nsteps; ++k2) executed_mean[k2] = double(t[k2]) / double(ctx->g.nv);
  return TRINITY_OK;
}

int trinity_read_field(trinity_ctx* ctx, int what, int back, void* out, size_t bytes, int ptr_kind) {
  if (!ctx) return TRINITY_E_INVALID;
  const size_t nv = ctx->g.nv;
  const size_t cnt = what == TRINITY_FIELD_U ? nv
                                             : static_cast<size_t>(what == TRINITY_FIELD_S ? ctx->na_s : ctx->g.na) * nv;
  if ((what != TRINITY_FIELD_I && what != TRINITY_FIELD_S && what != TRINITY_FIELD_U) || back < 0 ||
      back > kRing - 1 || bytes != cnt * 4 || !out || (ptr_kind != 0 && ptr_kind != 1))
    return fail(ctx, TRINITY_E_INVALID, "bad field request");
  const int lev = ctx->steps_done - 1 - back;
  CK(cudaStreamSynchronize(ctx->stream));
  const cudaMemcpyKind kind = ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (lev < ctx->g.hist_from) {
    if (ptr_kind)
      CK(cudaMemset(out, 0, bytes));
    else
      std::memset(out, 0, bytes);
    return TRINITY_OK;
  }
  if (what == TRINITY_FIELD_U) {
    // energy density of level lev, formed in the context's Q buffer (free between steps)
    const float* Ilev = ctx->I + static_cast<size_t>(ring_slot(lev)) * ctx->g.na * nv;
    const float scale = static_cast<float>(ctx->w / kC0);
    CK(launch_energy_density(ctx->g, Ilev, ctx->nidx, scale, ctx->Q, ctx->stream));
    CK(cudaMemcpyAsync(out, ctx->Q, bytes, kind, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return TRINITY_OK;
  }
  const float* base = (what == TRINITY_FIELD_I ? ctx->I : ctx->S) + static_cast<size_t>(ring_slot(lev)) * cnt;
  CK(cudaMemcpy(out, base, bytes, kind));
  return TRINITY_OK;
}

int trinity_kernels_per_step(const trinity_ctx* ctx, int* n) {
  if (!ctx || !n) return TRINITY_E_INVALID;
  int k = 0;
  if (ctx->two_level)
    k = 1 + 1 + 1 + 1;  // sweep2, scatter, refine, tally
  else if (sweep_uses_tma(ctx))
    k = (ctx->ndir[0] > 0) + (ctx->ndir[1] > 0) + (ctx->ndir[2] > 0) + 1 + 1;  // sweeps, scatter, tally
  else
    k = 1 + 1 + 1;  // sweep, scatter, tally
  if (ctx->n_iface > 0) k += ctx->two_level ? 2 : 1;  // interface split (and re-coarsening)
  *n = k + 1;  // the step counter
  return TRINITY_OK;
}

int trinity_sweep_form(const trinity_ctx* ctx, int* form) {
  if (!ctx || !form) return TRINITY_E_INVALID;
  *form = ctx->two_level ? 2 : (sweep_uses_tma(ctx) ? 1 : 0);
  return TRINITY_OK;
}

int trinity_set_sweep_tma(trinity_ctx* ctx, int on) {
  if (!ctx) return TRINITY_E_INVALID;
  if (ctx->locked) return fail(ctx, TRINITY_E_STATE, "the sweep form must be chosen before the first step");
  ctx->tma_off = on == 0;
  return TRINITY_OK;
}

int trinity_steps_done(const trinity_ctx* ctx, int* n) {
  if (!ctx || !n) return TRINITY_E_INVALID;
  *n = ctx->steps_done;
  return TRINITY_OK;
}

int trinity_reset(trinity_ctx* ctx) {
  if (!ctx) return TRINITY_E_INVALID;
  const size_t cnt = static_cast<size_t>(ctx->g.na) * ctx->g.nv;
  const size_t cnt_s = static_cast<size_t>(ctx->na_s) * ctx->g.nv;
  // every clear runs on the context's stream, so work queued on it afterwards sees it
  cudaStream_t st = ctx->stream;
  CK(cudaStreamSynchronize(st));
  CK(cudaMemsetAsync(ctx->I, 0, kRing * cnt * 4, st));
  CK(cudaMemsetAsync(ctx->S, 0, kRing * cnt_s * 4, st));
  CK(cudaMemsetAsync(ctx->Q, 0, cnt * 4, st));
  if (ctx->two_level) {
    CK(cudaMemsetAsync(ctx->Ic, 0, kRing * cnt_s * 4, st));
    CK(cudaMemsetAsync(ctx->Qc, 0, cnt_s * 4, st));
  }
  CK(cudaMemsetAsync(ctx->d_step, 0, sizeof(int), st));
  CK(cudaMemsetAsync(ctx->d_smax, 0, 2 * sizeof(unsigned), st));
  CK(cudaMemsetAsync(ctx->d_nonconv, 0, sizeof(int), st));
  CK(cudaMemsetAsync(ctx->d_error, 0, sizeof(int), st));
  CK(cudaMemsetAsync(ctx->d_tile_ctr, 0, 2 * sizeof(int), st));
  CK(cudaMemsetAsync(ctx->d_balance, 0, sizeof(double), st));
  if (ctx->capacity > 0) {
    const size_t c = static_cast<size_t>(ctx->capacity);
    CK(cudaMemsetAsync(ctx->d_iters_max, 0, c * sizeof(int), st));
    CK(cudaMemsetAsync(ctx->d_iters_sum, 0, c * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(ctx->d_tile_iters, 0, c * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(ctx->d_energy, 0, c * sizeof(double), st));
    CK(cudaMemsetAsync(ctx->d_escaped, 0, c * sizeof(double), st));
    CK(cudaMemsetAsync(ctx->d_absorbed, 0, c * sizeof(double), st));
    CK(cudaMemsetAsync(ctx->d_residual, 0, c * sizeof(double), st));
  }
  if (ctx->d_det)
    CK(cudaMemsetAsync(ctx->d_det, 0, ctx->dets.size() * std::max(ctx->nbins, 1) * sizeof(double), st));
  CK(cudaStreamSynchronize(st));
  ctx->g.hist_from = 0;
  ctx->has_init = false;
  ctx->steps_done = 0;
  ctx->nonconv_seen = 0;
  free_adjoint(ctx);
  // the captured graph stays valid: buffers are unchanged, and trinity_run recaptures if
  // the grid parameters changed
  return TRINITY_OK;
}

const char* trinity_last_error(const trinity_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

void trinity_destroy(trinity_ctx* ctx) {
  if (!ctx) return;
  free_interfaces(ctx);
  free_adjoint(ctx);
  if (ctx->two_level) {
    cudaFree(ctx->Qc);
    cudaFree(ctx->Ic);
  }
  cudaFree(ctx->d_children);
  cudaFree(ctx->d_b1ds);
  cudaFree(ctx->d_Mt);
  cudaFree(ctx->d_xcls);
  cudaFree(ctx->d_b1tab);
  cudaFree(ctx->d_xmua);
  cudaFree(ctx->d_Mimg);
  cudaFree(ctx->d_tmask);
  for (int c = 0; c < 3; ++c) cudaFree(ctx->d_dlist[c]);
  cudaFree(ctx->d_hsh);
  for (int k = 0; k < 2; ++k) {
    if (ctx->side[k]) cudaStreamDestroy(ctx->side[k]);
    if (ctx->ev_join[k]) cudaEventDestroy(ctx->ev_join[k]);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  void* bufs[] = {ctx->I,         ctx->S,          ctx->Q,           ctx->mut,       ctx->eps,
                  ctx->nidx,      ctx->P32,        ctx->Pbf,         ctx->d_dirs,    ctx->d_offs,
                  ctx->d_det_vox, ctx->d_det_dir,  ctx->d_det_id,    ctx->d_det_w,   ctx->d_det,
                  ctx->d_step,    ctx->d_smax,     ctx->d_nonconv,   ctx->d_error,   ctx->d_iters_max,
                  ctx->d_iters_sum, ctx->d_energy, ctx->d_escaped,   ctx->d_bins, ctx->d_tile_iters,
                  ctx->d_tile_ctr, ctx->d_rcorr,   ctx->d_cls,       ctx->d_cls_ds,
                  ctx->d_rcorr32, ctx->d_absorbed, ctx->d_residual,  ctx->d_balance, ctx->d_refl};
  for (void* p : bufs)
    if (p) cudaFree(p);
  delete ctx;
}

int trinity_tc_selftest(int na, const uint16_t* A, const uint16_t* B, float* D) {
  if (!A || !B || !D || (na != 48 && na != 192)) return TRINITY_E_INVALID;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return TRINITY_E_CUDA;
  if (!(prop.major == 10 && prop.minor == 3)) return TRINITY_E_UNSUPPORTED;
  const int kp = (na + 63) / 64 * 64;
  uint16_t *dA = nullptr, *dB = nullptr;
  float* dD = nullptr;
  int* dErr = nullptr;
  int rc = TRINITY_OK;
  if (cudaMalloc(&dA, 128 * kp * 2) != cudaSuccess || cudaMalloc(&dB, na * kp * 2) != cudaSuccess ||
      cudaMalloc(&dD, 128 * na * 4) != cudaSuccess || cudaMalloc(&dErr, 4) != cudaSuccess) {
    rc = TRINITY_E_OOM;
  } else if (cudaMemcpy(dA, A, 128 * kp * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(dB, B, na * kp * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemset(dErr, 0, 4) != cudaSuccess || tc_tile_selftest(na, dA, dB, dD, dErr, 0) != cudaSuccess ||
             cudaDeviceSynchronize() != cudaSuccess ||
             cudaMemcpy(D, dD, 128 * na * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
    rc = TRINITY_E_CUDA;
  } else {
    int e = 0;
    if (cudaMemcpy(&e, dErr, 4, cudaMemcpyDeviceToHost) != cudaSuccess) rc = TRINITY_E_CUDA;
    else if (e != 0) rc = TRINITY_E_TIMEOUT;
  }
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dD);
  cudaFree(dErr);
  return rc;
}

// ---- host-side tables ----

int trinity_healpix_dirs(int nside, double* out, size_t n) {
  if (nside < 1 || nside > 64 || !out) return TRINITY_E_INVALID;
  const std::vector<double> d = healpix_dirs(nside);
  if (n != d.size()) return TRINITY_E_INVALID;
  std::copy(d.begin(), d.end(), out);
  return TRINITY_OK;
}

int trinity_phase_matrix(int nside, double g, double* out, size_t n, double* g_eff) {
  if (nside < 1 || nside > 8 || !out) return TRINITY_E_INVALID;
  try {
    const std::vector<double> P = phase_matrix(nside, g, g_eff);
    if (n != P.size()) return TRINITY_E_INVALID;
    std::copy(P.begin(), P.end(), out);
  } catch (...) {
    return TRINITY_E_INVALID;
  }
  return TRINITY_OK;
}

int trinity_lattice_tables(int nside, int nx, int ny, int nz, double h_mm, int periodic,
                           int32_t* dom_sgn, double* ds, int8_t* offsets, size_t n_offsets) {
  if (nside < 1 || nside > 64 || nx < 1 || ny < 1 || nz < 1 || !(h_mm > 0.0)) return TRINITY_E_INVALID;
  try {
    const Lattice L = build_lattice(healpix_dirs(nside), nx, ny, nz, h_mm, periodic != 0);
    if (n_offsets != L.off.size()) return TRINITY_E_INVALID;
    for (int d = 0; d < L.na; ++d) {
      if (dom_sgn) {
        dom_sgn[2 * d] = L.dom[d];
        dom_sgn[2 * d + 1] = L.sgn[d];
      }
      if (ds) ds[d] = L.ds[d];
    }
    if (offsets) std::copy(L.off.begin(), L.off.end(), offsets);
  } catch (...) {
    return TRINITY_E_INVALID;
  }
  return TRINITY_OK;
}

int trinity_interface_entries(int nside, int nx, int ny, int nz, double h_mm, int periodic,
                              const float* nmap, int* vox, int* j, int* d, double* w, size_t cap,
                              size_t* count) {
  if (nside < 1 || nside > 64 || nx < 1 || ny < 1 || nz < 1 || !(h_mm > 0.0) || !nmap || !count)
    return TRINITY_E_INVALID;
  try {
    const std::vector<double> dirs = healpix_dirs(nside);
    const Lattice L = build_lattice(dirs, nx, ny, nz, h_mm, periodic != 0);
    const std::vector<float> nm(nmap, nmap + static_cast<size_t>(nx) * ny * nz);
    const InterfaceTable T = build_interfaces(dirs, L, nx, ny, nz, h_mm, periodic != 0, nm);
    *count = T.s_vox.size();
    if (cap < T.s_vox.size()) return vox ? TRINITY_E_INVALID : TRINITY_OK;
    for (size_t k = 0; k < T.s_vox.size(); ++k) {
      if (vox) vox[k] = T.s_vox[k];
      if (j) j[k] = T.s_j[k];
      if (d) d[k] = T.s_d[k];
      if (w) w[k] = T.s_w[k];
    }
  } catch (...) {
    return TRINITY_E_INVALID;
  }
  return TRINITY_OK;
}

int trinity_parent_map(int nside_fine, int nside_coarse, int* out, size_t n) {
  if (nside_fine < 1 || nside_fine > 64 || nside_coarse < 1 || !out) return TRINITY_E_INVALID;
  try {
    const std::vector<int> par = parent_map(nside_fine, nside_coarse);
    if (n != par.size()) return TRINITY_E_INVALID;
    std::copy(par.begin(), par.end(), out);
  } catch (...) {
    return TRINITY_E_INVALID;
  }
  return TRINITY_OK;
}

int trinity_cone_weights(int nside, int face, double half_angle_deg, int inward, double* out, size_t n) {
  if (nside < 1 || nside > 64 || !out) return TRINITY_E_INVALID;
  try {
    const std::vector<double> a = cone_weights(healpix_dirs(nside), face, half_angle_deg, inward != 0);
    if (n != a.size()) return TRINITY_E_INVALID;
    std::copy(a.begin(), a.end(), out);
  } catch (...) {
    return TRINITY_E_INVALID;
  }
  return TRINITY_OK;
}

}  // extern "C"
