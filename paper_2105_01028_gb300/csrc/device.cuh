// Device-side structures and small helpers shared by the kernels and the C-ABI layer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

namespace trinity {

// Per-direction constants of the ray lattice (built on the host in FP64, stored FP32).
struct DirInfo {
  int dom;        // dominant axis 0/1/2
  int sgn;        // travel sign along dom
  int a0, a1;     // transverse axes (increasing order)
  float ds;       // ray-sample spacing h / |Omega_dom| (mm)
  float dcoef;    // ds / (c0 dt): retarded delay in steps per unit refractive index (hi part)
  float dcoef_lo; // ds / (c0 dt) - dcoef (lo part: the delay's fraction is exact to FP32)
  float src_amp;  // inflow intensity while the pulse is on (0: not a source direction)
  float wcos_out[6];  // w * (Omega . n_out) * h^2 * dt for faces the ray leaves (else 0)
};

struct GridParams {
  int nx, ny, nz;
  int nv;           // nx * ny * nz
  int na;           // directions
  int nmax;         // stride of the offset table
  int periodic;
  int mirror;       // mirror faces: a ghost upwind sample reads its image (see sweep.cu)
  int hist_from;    // first valid time level: 0, or -4 with an initial state
  int warm;         // initial guess of the source iteration: 0 S(n-1), 1 2 S(n-1) - S(n-2)
  int src_voxel;    // flat voxel index of the source spot, -1 if none
  int pulse_steps;
  float h;
  float ds_max;     // max_d ds_d (for the contraction bound)
  float e_scale;    // h^3 / c0 * w  (energy per unit I * n)
  float mut_u;      // mu_t of every voxel when the medium's mu_t is uniform, else -1
  float n_u;        // n of every voxel when the refractive index is uniform, else 0
  double a_scale;   // h^3 dt w: absorbed energy per unit I * mu_a in one step
  double inj_step;  // energy the source's inflow carries in during each pulse step
};

// Per-run device counters and tallies (pointers into context-owned buffers).
struct RunState {
  int* step;                     // current time level n (advanced by the last kernel of a step)
  unsigned* smax;                // [2] max |S| of levels n-1 / n as float bits (ping-pong)
  int* iters_max;                // [capacity] per step
  unsigned long long* iters_sum; // [capacity] per step (sum over voxels)
  double* energy;                // [capacity] photon energy in the box after the step
  double* escaped;               // [capacity] energy leaving through the faces in the step
  double* absorbed;              // [capacity] energy absorbed (mu_a term of Eq. 1) in the step
  double* residual;              // [capacity] photon balance residual after the step
  double* balance;               // [1] energy before step 0 + injected - escaped - absorbed
  int* nonconv;                  // count of voxel-steps that hit max_iters
  int* bins;                     // [capacity] detector bin of each step (-1: none)
  int* error;                    // device error word (0 = ok)
  int* tile_ctr;                 // [2] work counters of the persistent kernels (ping-pong)
  unsigned long long* tile_iters; // [capacity] iterations executed x voxels per tile, summed
                                  // (tensor-core kernel; null: not counted)
};

// Tables of the tensor-core source iteration.
struct BfTables {
  const float* rcorr;    // [na] 1 - row sum of bf16(P): diagonal correction (FP32)
  const uint8_t* cls;    // [na] class of each direction's sample spacing ds
  const float* cls_ds;   // [ncls][nch] spacings of each class (b1 = mean of their b1)
  int ncls;              // <= 16
  int nch;               // 1, or the children per coarse direction on a two-level grid
  // TMA descriptors of the I and S rings (4-D: x, y, z, plane; boxes of one 8 x 4 x 4
  // brick and 8 directions) through which the tile's write-out is stored, or null: plain
  // stores.  Built by make_scatter_out_maps (nx a multiple of 4).
  const void* out_maps;  // 2 x 128 bytes
};
cudaError_t make_scatter_out_maps(const GridParams& gs, float* Iring, float* Sring, void* out);

__host__ __device__ inline int ring_slot(int level) { return ((level % 5) + 5) % 5; }

// Retarded delay delta = ds n / (c0 dt) split as m + f (m = floor(delta), 0 <= f < 1).
// dcoef is carried as hi + lo floats and the product with n is formed with its exact
// FMA error term, so f is accurate to FP32 rounding of f itself (a plain FP32 product
// would carry an absolute error of ~2e-7 into the time-interpolation weights).
__device__ __forceinline__ void retarded_delay(float dc_hi, float dc_lo, float n, int& m, float& f) {
  const float p = n * dc_hi;
  const float e = fmaf(n, dc_hi, -p);
  const float lo = fmaf(n, dc_lo, e);
  const float fl = floorf(p);
  float fr = (p - fl) + lo;
  m = static_cast<int>(fl);
  if (fr < 0.0f) {
    fr += 1.0f;
    m -= 1;
  } else if (fr >= 1.0f) {
    fr -= 1.0f;
    m += 1;
  }
  f = fr;
}

// exp(-x), b0(x), b1(x) of Eq. 9: b0 = [1 - (1+x) e^-x]/x, b1 = [x - 1 + e^-x]/x.
// For x < 1 the closed forms cancel catastrophically in FP32, so their Taylor series
// (from the series of exp) are summed to x^11, which is exact to FP32 rounding there.
__device__ __forceinline__ float ray_b0(float x, float T) {
  if (x < 1.0f) {
    float p = 1.0f / 43545600.0f;
    p = fmaf(p, x, -1.0f / 3991680.0f);
    p = fmaf(p, x, 1.0f / 403200.0f);
    p = fmaf(p, x, -1.0f / 45360.0f);
    p = fmaf(p, x, 1.0f / 5760.0f);
    p = fmaf(p, x, -1.0f / 840.0f);
    p = fmaf(p, x, 1.0f / 144.0f);
    p = fmaf(p, x, -1.0f / 30.0f);
    p = fmaf(p, x, 1.0f / 8.0f);
    p = fmaf(p, x, -1.0f / 3.0f);
    p = fmaf(p, x, 0.5f);
    return p * x;
  }
  return (1.0f - (1.0f + x) * T) / x;
}

__device__ __forceinline__ float ray_b1(float x, float T) {
  if (x < 1.0f) {
    float p = 1.0f / 479001600.0f;
    p = fmaf(p, x, -1.0f / 39916800.0f);
    p = fmaf(p, x, 1.0f / 3628800.0f);
    p = fmaf(p, x, -1.0f / 362880.0f);
    p = fmaf(p, x, 1.0f / 40320.0f);
    p = fmaf(p, x, -1.0f / 5040.0f);
    p = fmaf(p, x, 1.0f / 720.0f);
    p = fmaf(p, x, -1.0f / 120.0f);
    p = fmaf(p, x, 1.0f / 24.0f);
    p = fmaf(p, x, -1.0f / 6.0f);
    p = fmaf(p, x, 0.5f);
    return p * x;
  }
  return (x - 1.0f + T) / x;
}

// Kernel launchers (defined in kernels.cu / scatter_tc.cu).
cudaError_t launch_sweep(const GridParams& g, const DirInfo* dirs, const int8_t* offs,
                         const float* Iring, const float* Sring, const float* mut,
                         const float* nidx, const int* refl, float* Q, RunState rs, cudaStream_t st);
cudaError_t launch_scatter_fp32(const GridParams& g, const float* b1ds, int nch, const float* P,
                                const float* rcorr, const float* Q, const float* mut,
                                const float* eps,
                                const float* nidx, float* Iring, float* Sring, float tol,
                                int max_iters, RunState rs, cudaStream_t st);
cudaError_t launch_tally(const GridParams& g, const DirInfo* dirs, const float* Iring,
                         const int* det_vox, const int* det_dir, const float* det_w,
                         const int* det_id, int n_det_entries, double* det, int nbins,
                         RunState rs, cudaStream_t st);
cudaError_t launch_advance(const GridParams& g, RunState rs, cudaStream_t st);

// The TMA-staged one-level sweep (sweep_tma.cu): uniform refractive index, vacuum faces,
// nx a multiple of 4 and nx + 8 <= 256.  Tensor maps of the I and S rings, one per
// dominant-axis class (box shapes differ), 128 bytes each as the driver encodes them.
struct SweepMaps {
  alignas(64) unsigned char I[3][128];
  alignas(64) unsigned char S[3][128];
};
bool sweep_tma_supported(const GridParams& g);
cudaError_t make_sweep_maps(const GridParams& g, float* Iring, float* Sring, SweepMaps* out);
cudaError_t launch_sweep_tma(const GridParams& g, const DirInfo* dirs, const int* const dlist[3],
                             const int ndir[3], const int8_t* offs, const int8_t* hsh, const SweepMaps& maps,
                             const float* mut, float* Q, RunState rs, const cudaStream_t st[3]);
cudaError_t launch_energy_density(const GridParams& g, const float* I, const float* nidx, float scale, float* u,
                                  cudaStream_t st);
cudaError_t launch_interface(int nvox, int na, const int* vox, const int* rowptr, const int* src,
                             const float* w, const uint8_t* keep, float* Q, int nv, cudaStream_t st);
bool scatter_bf16_supported(int na);
cudaError_t launch_scatter_bf16(const GridParams& g, const BfTables& t, const uint16_t* Pbf,
                                const float* Q, const float* mut, const float* eps,
                                const float* nidx, float* Iring, float* Sring, float tol,
                                int max_iters, RunState rs, cudaStream_t st);
cudaError_t tc_tile_selftest(int na, const uint16_t* A, const uint16_t* B, float* D, int* err,
                             cudaStream_t st);

}  // namespace trinity

namespace trinity {

// Adjoint launchers (defined in adjoint.cu).
cudaError_t launch_adj_inject(const int* det_vox, const int* det_dir, const float* det_w,
                              const int* det_id, int n_entries, const double* G, int nbins, int b,
                              float* Ib_n, int nv, unsigned* ymax_cur, cudaStream_t st);
cudaError_t launch_adj_scatter_fp32(const GridParams& g, const DirInfo* dirs, const float* P,
                                    const float* rcorr, const float* mut, const float* eps,
                                    float* Ib_n, float* Sb_n, const float* I_n, const float* S_n,
                                    float* Y, float* Y2, int extrap, float* Qb, double* gA, double* gmut,
                                    float tol, int max_iters, const unsigned* yglob_prev, unsigned* ymax_cur,
                                    int* nonconv, unsigned long long* iters_sum, cudaStream_t st);
cudaError_t launch_adj_push(const GridParams& g, const DirInfo* dirs, const int8_t* offs,
                            const float* stI, const float* stS, int lev_base, int n,
                            const float* mut, const float* nidx, const float* Qb, float* IbR,
                            float* SbR, double* gmut, cudaStream_t st);
cudaError_t launch_adj_finish(int nv, const float* mut, const float* eps, const double* gA,
                              const double* gmut, double* gmua, double* gmus, cudaStream_t st);
cudaError_t launch_adj_restore(int* step, int c, unsigned* smax, const unsigned* saved,
                               cudaStream_t st);

}  // namespace trinity

namespace trinity {

// Two-level angular grid launchers (defined in twolevel.cu).
cudaError_t launch_sweep2(const GridParams& g, const DirInfo* dirs, const int8_t* offs, const int* children,
                          int nch, int na_s, const float* Iring, const float* Sring, const float* mut,
                          const float* nidx, float* Qf, float* Qc, RunState rs, cudaStream_t st);
cudaError_t launch_refine(const GridParams& g, const DirInfo* dirs, const int* children, int nch, int na_s,
                          const float* mut, const float* Qf, const float* Sring, float* Iring, RunState rs,
                          cudaStream_t st);
cudaError_t launch_recoarsen(int nvox, const int* vox, const int* children, int nch, int na_s, const float* Qf,
                             float* Qc, int nv, cudaStream_t st);

}  // namespace trinity

namespace trinity {

// Exact per-voxel source function for piecewise-uniform optics (defined in exact.cu).
// Mt: [classes][na][na] FP32, M transposed; cls: [nv] class of each voxel (< 32).
// b1tab: [classes][na] b1 of each class and direction (the 192-direction GEMM form uses it).
// mua_cls: [classes] mu_a of each class (absorbed-energy tally).
cudaError_t launch_exact_fp32(const GridParams& g, const float* b1ds, int nch, const float* Mt,
                              const float* b1tab, const uint8_t* cls, const float* mua_cls, const float* Q,
                              const float* mut, const float* nidx, float* Iring, float* Sring, RunState rs,
                              cudaStream_t st);

// The exact solve on the tensor cores (defined in exact_tc.cu): three TF32 products with
// FP32 accumulation in TMEM, for 192 directions, a voxel count that is a multiple of 4
// (the TMA's 16-byte row rule on Q) and at most 8 optics classes.
bool exact_tc_supported(const GridParams& g, int ncls);
int exact_tc_tiles(int nv);
// M: [classes][192][192] FP64 (row i = output direction); img receives the operators'
// shared-memory images (per class and 32-direction chunk: TF32 hi, then lo).
void exact_tc_images(const double* M, int ncls, std::vector<float>* img);
// Bit c of mask[t] is set when 128-voxel tile t holds a voxel of class c.
void exact_tc_tile_masks(const uint8_t* cls, int nv, std::vector<uint8_t>* mask);
// The TMA descriptor of Q ([192][nv] FP32) for 128-voxel x 32-direction boxes; out is 128 bytes.
cudaError_t make_exact_qmap(const GridParams& g, const float* Q, void* out);
cudaError_t launch_exact_tc(const GridParams& g, const void* qmap, const float* Mimg, const uint8_t* tmask,
                            const float* b1tab, int ncls, const uint8_t* cls, const float* mua_cls, const float* Q,
                            const float* nidx, float* Iring, float* Sring, RunState rs, cudaStream_t st);

}  // namespace trinity
