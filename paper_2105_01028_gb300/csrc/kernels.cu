// FP32 kernels of one time step: the per-voxel source iteration on CUDA cores (Eq. 12,
// Section 2.4 steps 5-6), the detector / escape tallies (Section 3.1), the interface
// split and the step counter.
#include <cfloat>
#include <cstdint>

#include "device.cuh"

namespace trinity {

namespace {

__device__ __forceinline__ int pick(int axis, int x, int y, int z) {
  return axis == 0 ? x : (axis == 1 ? y : z);
}

// ----------------------------------------------------------------------------------------
// Source iteration on CUDA cores (plain FP32 mode).
// A CTA owns a tile of kTile voxels; thread i < NA owns outgoing direction i of all of them.
// Isotropic rebalance (angular two-grid correction): after each plain update S_half of
// S_k, the voxel's isotropic error component is removed.  The error of S_half,
// f = S* - S_half, solves (1 - a P B1) f = a P B1 Delta with Delta = S_half - S_k; its
// projection on the constant vector (P has unit column sums) gives the scalar
//   c = a sum_j b1_j Delta_j / sum_j (1 - a b1_j),
// and S_{k+1} = S_half + c.  The isotropic mode is the slowest of the plain iteration
// (contraction a b1 ~ 0.93 at the workloads' optics); without it the iterate reaches the
// FP32 noise floor ~1/(1 - a b1) ~ 14 noise units short of the fixed point, always on the
// same side, and that bias accumulates over the steps.  The correction vanishes at the
// fixed point, so the fixed point is the plain iteration's.  The stop test is taken on
// the plain update (|S_half - S_k| bounds the error of S_half exactly as in the plain
// iteration), and a voxel that stops keeps S_half.
// Per iteration: Y[v][i] = sum_j P[i][j] X[v][j] + r_i X[v][i] (P symmetric, read as
// P[j][i] so a warp reads a contiguous row; r_i = 1 - sum_j P[i][j] restores the unit row
// and column sums that FP32 rounding of P breaks), S_new = (1 - eps) Y with
// eps = mu_a / mu_t (albedo a = 1 - eps: forming a itself in FP32 would misstate the
// small absorption 1 - a by up to 6e-5 relative), X = Q + b1 S.  The per-voxel stop test needs the
// max over directions of |S_new - S_old| and |S_new|: a warp "transpose" reduction leaves
// lane v holding the warp's maximum for voxel v, then the warps combine through smem.
// ----------------------------------------------------------------------------------------
constexpr int kTile = 16;  // voxels per CTA: small enough for two CTAs per SM
constexpr int kXStride = kTile + 4;  // padded row (floats) of the X tile in smem

template <int NA>
struct ScatterCfg {
  static constexpr int kThreads = ((NA + 31) / 32) * 32;
  static constexpr int kWarps = kThreads / 32;
};

struct OpMax {
  __device__ __forceinline__ float operator()(float a, float b) const { return fmaxf(a, b); }
};
struct OpSum {
  __device__ __forceinline__ float operator()(float a, float b) const { return a + b; }
};

// After the call lane l holds the reduction (max or sum) over the warp's lanes of
// vals[l mod V] (returned): lanes l and l ^ s for s >= V first combine all V values, then
// a butterfly halves the values each lane keeps while transposing them across lanes.
template <int V, typename Op>
__device__ __forceinline__ float warp_transpose_reduce(float (&vals)[V], int lane, Op op) {
#pragma unroll
  for (int s = 16; s >= V; s >>= 1) {
#pragma unroll
    for (int k = 0; k < V; ++k) vals[k] = op(vals[k], __shfl_xor_sync(0xffffffffu, vals[k], s));
  }
#pragma unroll
  for (int s = V / 2; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < s; ++k) {
      const float send = upper ? vals[k] : vals[k + s];
      const float keep = upper ? vals[k + s] : vals[k];
      const float recv = __shfl_xor_sync(0xffffffffu, send, s);
      vals[k] = op(keep, recv);
    }
  }
  return vals[0];
}

template <int NA>
__global__ void __launch_bounds__(ScatterCfg<NA>::kThreads, 2)
    scatter_fp32_kernel(GridParams g, const float* __restrict__ b1ds, int nch, const float* __restrict__ P,
                        const float* __restrict__ rcorr, const float* __restrict__ Q,
                        const float* __restrict__ mut, const float* __restrict__ eps,
                        const float* __restrict__ nidx,
                        float* __restrict__ Iring, float* __restrict__ Sring, float tol,
                        int max_iters, RunState rs) {
  constexpr int W = ScatterCfg<NA>::kWarps;
  __shared__ __align__(16) float Xs[2][NA][kXStride];
  __shared__ float red_d[W][32];  // per warp, lane v < kTile holds voxel v's reduction
  __shared__ float red_s[W][32];
  __shared__ float red_c[W][32];
  __shared__ float den_s[kTile], c_s[kTile];
  __shared__ float e_s[kTile], rho_s[kTile], best_s[kTile], mua_s[kTile];
  __shared__ int iters_s[kTile], stall_s[kTile];
  __shared__ unsigned act_s;

  const int n = *rs.step;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int i = tid;  // outgoing direction
  const bool live = i < NA;
  const int v0 = blockIdx.x * kTile;
  const size_t plane = static_cast<size_t>(g.nv);
  const float s_glob = __uint_as_float(rs.smax[(n - 1) & 1]);

  if (tid < kTile) {
    const int v = v0 + tid;
    float ev = 1.0f, rho = 0.0f, ma = 0.0f;
    if (v < g.nv) {
      ev = eps[v];
      const float mt = mut[v];
      const float xm = mt * g.ds_max;
      rho = (1.0f - ev) * ray_b1(xm, expf(-xm));  // b1 grows with x: max over d is at ds_max
      ma = ev * mt;                                // mu_a of the voxel
    }
    e_s[tid] = ev;
    rho_s[tid] = rho;
    mua_s[tid] = ma;
    iters_s[tid] = 0;
    best_s[tid] = 3.0e38f;
    stall_s[tid] = 0;
  }
  if (tid == 0)
    act_s = (g.nv - v0 >= kTile) ? (kTile == 32 ? 0xffffffffu : ((1u << kTile) - 1u)) : ((1u << (g.nv - v0)) - 1u);
  __syncthreads();

  float q[kTile], b1[kTile], so[kTile], acc[kTile];
  const float* dsl = b1ds + static_cast<size_t>(live ? i : 0) * nch;
  const float inv_nch = 1.0f / static_cast<float>(nch);
  const float ri = live ? rcorr[i] : 0.0f;
  const bool has_prev = (n - 1) >= g.hist_from;
  const bool has_prev2 = g.warm != 0 && (n - 2) >= g.hist_from;  // linear extrapolation in time
  const size_t prev_off = (static_cast<size_t>(ring_slot(n - 1)) * g.na + (live ? i : 0)) * plane;
  const size_t prev2_off = (static_cast<size_t>(ring_slot(n - 2)) * g.na + (live ? i : 0)) * plane;
#pragma unroll
  for (int v = 0; v < kTile; ++v) {
    const int vv = v0 + v;
    const bool ok = live && vv < g.nv;
    q[v] = ok ? __ldg(Q + static_cast<size_t>(i) * plane + vv) : 0.0f;
    // b1 of the direction, or the mean of its children's b1 on a two-level angular grid
    float bs = 0.0f;
    if (ok) {
      const float mu = mut[vv];
      for (int k = 0; k < nch; ++k) {
        const float xo = mu * dsl[k];
        bs += ray_b1(xo, expf(-xo));
      }
    }
    b1[v] = bs * inv_nch;
    so[v] = (ok && has_prev) ? Sring[prev_off + vv] : 0.0f;
    if (ok && has_prev2) so[v] = fmaf(2.0f, so[v], -Sring[prev2_off + vv]);
  }
  if (live) {
#pragma unroll
    for (int v = 0; v < kTile; v += 4) {
      float4 x4 = make_float4(q[v] + b1[v] * so[v], q[v + 1] + b1[v + 1] * so[v + 1],
                              q[v + 2] + b1[v + 2] * so[v + 2], q[v + 3] + b1[v + 3] * so[v + 3]);
      *reinterpret_cast<float4*>(&Xs[0][i][v]) = x4;
    }
  }
  {
    // rebalance denominators sum_j (1 - a b1_j) per voxel: a transpose-sum of b1 over the
    // directions (all threads; dead lanes add zero)
    float bsum[kTile];
#pragma unroll
    for (int v = 0; v < kTile; ++v) bsum[v] = b1[v];
    red_c[warp][lane] = warp_transpose_reduce(bsum, lane, OpSum());
  }
  __syncthreads();
  if (tid < kTile) {
    float sb = 0.0f;
#pragma unroll
    for (int w = 0; w < W; ++w) sb += red_c[w][tid];
    den_s[tid] = static_cast<float>(NA) - (1.0f - e_s[tid]) * sb;
    c_s[tid] = 0.0f;
  }
  unsigned act = act_s;
  int cur = 0;
  int k = 0;
  while (act != 0u && k < max_iters) {
    ++k;
    __syncthreads();
#pragma unroll
    for (int v = 0; v < kTile; ++v) acc[v] = 0.0f;
    if (live) {
      // Blocked accumulation: each block of kBlk terms is summed on its own and then added
      // to the total, which keeps the rounding noise of the ~200-term sum close to that of
      // a pairwise sum.  The iteration's attainable accuracy is set by that noise, divided
      // by (1 - rho) ~ 0.07 at the workloads' optics.
      constexpr int kBlk = (NA % 8 == 0) ? 8 : 4;
      const float* pcol = P + i;
#pragma unroll 1
      for (int j0 = 0; j0 < NA; j0 += kBlk) {
        float t[kTile];
#pragma unroll
        for (int v = 0; v < kTile; ++v) t[v] = 0.0f;
#pragma unroll
        for (int j = j0; j < j0 + kBlk; ++j) {
          const float p = __ldg(pcol + static_cast<size_t>(j) * NA);
          const float4* xr = reinterpret_cast<const float4*>(&Xs[cur][j][0]);
#pragma unroll
          for (int v4 = 0; v4 < kTile / 4; ++v4) {
            const float4 x4 = xr[v4];
            t[4 * v4 + 0] = fmaf(p, x4.x, t[4 * v4 + 0]);
            t[4 * v4 + 1] = fmaf(p, x4.y, t[4 * v4 + 1]);
            t[4 * v4 + 2] = fmaf(p, x4.z, t[4 * v4 + 2]);
            t[4 * v4 + 3] = fmaf(p, x4.w, t[4 * v4 + 3]);
          }
        }
#pragma unroll
        for (int v = 0; v < kTile; ++v) acc[v] += t[v];
      }
    }
    // epilogue: S_half = a * acc on active voxels, its change and b1-weighted change
    float dsv[kTile], smv[kTile], cvv[kTile];
#pragma unroll
    for (int v = 0; v < kTile; ++v) {
      const bool on = live && ((act >> v) & 1u);
      const float y = fmaf(ri, fmaf(b1[v], so[v], q[v]), acc[v]);  // + r_i X_i
      const float sn = fmaf(-e_s[v], y, y);                        // (1 - eps) y
      const float dl = sn - so[v];
      dsv[v] = on ? fabsf(dl) : 0.0f;
      smv[v] = on ? fabsf(sn) : 0.0f;
      cvv[v] = on ? b1[v] * dl : 0.0f;
      so[v] = on ? sn : so[v];
    }
    red_d[warp][lane] = warp_transpose_reduce(dsv, lane, OpMax());
    red_s[warp][lane] = warp_transpose_reduce(smv, lane, OpMax());
    red_c[warp][lane] = warp_transpose_reduce(cvv, lane, OpSum());
    __syncthreads();
    if (tid < 32) {  // one full warp: the ballot below is warp-collective
      const int v = tid;
      unsigned done = 0u;
      if (v < kTile && ((act >> v) & 1u)) {
        float D = 0.0f, Sm = 0.0f;
#pragma unroll
        for (int w = 0; w < W; ++w) {
          D = fmaxf(D, red_d[w][v]);
          Sm = fmaxf(Sm, red_s[w][v]);
        }
        const float r = rho_s[v];
        const float scale = fmaxf(Sm, 1e-6f * s_glob);
        if (D < best_s[v]) {
          best_s[v] = D;
          stall_s[v] = 0;
        } else {
          stall_s[v] += 1;
        }
        // stop: the error bound is within tol, or the change has stopped shrinking for
        // three iterations (the iterate has reached the noise floor of FP32 arithmetic and
        // fluctuates around the fixed point; a fixed floor on the change would instead stop
        // on one side of it every step and bias the result)
        const bool stop = (r / (1.0f - r)) * D <= tol * scale || stall_s[v] >= 3;
        if (stop) {
          done = 1u;
          iters_s[v] = k;
        }
        // isotropic correction of a voxel that goes on (a stopped voxel keeps S_half)
        float cs = 0.0f;
#pragma unroll
        for (int w = 0; w < W; ++w) cs += red_c[w][v];
        c_s[v] = stop ? 0.0f : (1.0f - e_s[v]) * cs / den_s[v];
      }
      const unsigned mask = __ballot_sync(0xffffffffu, done);
      if (tid == 0) act_s = act & ~mask;
    }
    __syncthreads();
    const unsigned was = act;
    act = act_s;
    // S_{k+1} = S_half + c; X = Q + b1 S for the next iteration
    const int nxt = cur ^ 1;
    if (live) {
#pragma unroll
      for (int v = 0; v < kTile; ++v)
        if ((was >> v) & 1u) so[v] += c_s[v];
#pragma unroll
      for (int v = 0; v < kTile; v += 4) {
        float4 x4 = make_float4(q[v] + b1[v] * so[v], q[v + 1] + b1[v + 1] * so[v + 1],
                                q[v + 2] + b1[v + 2] * so[v + 2], q[v + 3] + b1[v + 3] * so[v + 3]);
        *reinterpret_cast<float4*>(&Xs[nxt][i][v]) = x4;
      }
    }
    cur = nxt;
  }
  // voxels still active hit max_iters
  if (tid < kTile && ((act >> tid) & 1u)) {
    iters_s[tid] = k;
    atomicAdd(rs.nonconv, 1);
  }

  // write I(n) = Q + b1 S, S(n); tallies
  const size_t cur_off = (static_cast<size_t>(ring_slot(n)) * g.na + (live ? i : 0)) * plane;
  float esum = 0.0f, asum = 0.0f, smax = 0.0f;
  if (live) {
#pragma unroll
    for (int v = 0; v < kTile; ++v) {
      const int vv = v0 + v;
      if (vv < g.nv) {
        const float Iv = q[v] + b1[v] * so[v];
        Iring[cur_off + vv] = Iv;
        Sring[cur_off + vv] = so[v];
        esum = fmaf(Iv, nidx[vv], esum);
        asum = fmaf(Iv, mua_s[v], asum);
        smax = fmaxf(smax, fabsf(so[v]));
      }
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    esum += __shfl_xor_sync(0xffffffffu, esum, o);
    asum += __shfl_xor_sync(0xffffffffu, asum, o);
    smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  }
  __syncthreads();
  if (lane == 0) {
    red_d[warp][0] = esum;
    red_d[warp][1] = asum;
    red_s[warp][0] = smax;
  }
  __syncthreads();
  if (tid == 0) {
    double e = 0.0, ab = 0.0;
    float sm = 0.0f;
    for (int w = 0; w < W; ++w) {
      e += red_d[w][0];
      ab += red_d[w][1];
      sm = fmaxf(sm, red_s[w][0]);
    }
    atomicAdd(rs.energy + n, e * static_cast<double>(g.e_scale));
    atomicAdd(rs.absorbed + n, ab * g.a_scale);
    atomicMax(rs.smax + (n & 1), __float_as_uint(sm));
    int im = 0;
    unsigned long long is = 0;
    for (int v = 0; v < kTile && v0 + v < g.nv; ++v) {
      im = max(im, iters_s[v]);
      is += static_cast<unsigned long long>(iters_s[v]);
    }
    atomicMax(rs.iters_max + n, im);
    atomicAdd(rs.iters_sum + n, is);
  }
}

// ----------------------------------------------------------------------------------------
// Tallies of level n (Section 3.1): detector curves (FP64 bins) and the energy leaving
// through all faces.  Block 0 handles the detector entry list; the other blocks cover
// the face voxels (blockIdx.y = face).
// ----------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tally_kernel(GridParams g, const DirInfo* __restrict__ dirs,
                                                    const float* __restrict__ Iring,
                                                    const int* __restrict__ det_vox,
                                                    const int* __restrict__ det_dir,
                                                    const float* __restrict__ det_w,
                                                    const int* __restrict__ det_id, int n_entries,
                                                    double* __restrict__ det, int nbins, RunState rs) {
  __shared__ double red[8];
  const int n = *rs.step;
  const size_t plane = static_cast<size_t>(g.nv);
  const float* Icur = Iring + static_cast<size_t>(ring_slot(n)) * g.na * plane;
  const int face = blockIdx.y;
  if (face == 6) {
    // detector entries: weight already holds alpha * Omega_cap * cos * h^2 * dt
    const int b = rs.bins[n];
    if (b < 0 || b >= nbins) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_entries; e += gridDim.x * blockDim.x) {
      const double val = static_cast<double>(det_w[e]) *
                         static_cast<double>(Icur[static_cast<size_t>(det_dir[e]) * plane + det_vox[e]]);
      atomicAdd(det + static_cast<size_t>(det_id[e]) * nbins + b, val);
    }
    return;
  }
  if (g.periodic || g.mirror) return;  // closed box: nothing leaves
  const int ax = face >> 1;
  const int ua = ax == 0 ? 1 : 0;
  const int va = ax == 2 ? 1 : 2;
  const int nu = pick(ua, g.nx, g.ny, g.nz);
  const int nvv = pick(va, g.nx, g.ny, g.nz);
  const int pa = (face & 1) ? pick(ax, g.nx, g.ny, g.nz) - 1 : 0;
  double acc = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nu * nvv; t += gridDim.x * blockDim.x) {
    const int iu = t % nu, iv = t / nu;
    int c[3];
    c[ax] = pa;
    c[ua] = iu;
    c[va] = iv;
    const size_t v = (static_cast<size_t>(c[2]) * g.ny + c[1]) * g.nx + c[0];
    float s = 0.0f;
    for (int d = 0; d < g.na; ++d) {
      const float wc = dirs[d].wcos_out[face];
      if (wc != 0.0f) s = fmaf(wc, Icur[static_cast<size_t>(d) * plane + v], s);
    }
    acc += static_cast<double>(s);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(rs.escaped + n, s);
  }
}

// Photon energy density of one stored level (Section 3.1 plots its maps): u_v =
// (n_v / c0) sum_d w I_d, the energy density of radiance I per unit solid angle being
// I / c with c = c0 / n.  Thread per voxel; the directions are summed in FP64.
__global__ void __launch_bounds__(256) energy_density_kernel(GridParams g, const float* __restrict__ I,
                                                             const float* __restrict__ nidx, float scale,
                                                             float* __restrict__ u) {
  const size_t plane = static_cast<size_t>(g.nv);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.nv; v += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int d = 0; d < g.na; ++d) s += static_cast<double>(__ldg(I + static_cast<size_t>(d) * plane + v));
    u[v] = static_cast<float>(s * static_cast<double>(scale) * static_cast<double>(nidx[v]));
  }
}

// End of step n: the photon balance (energy before step 0 plus what came in minus what
// left or was absorbed), its residual against the energy in the box, and the step counter.
__global__ void advance_kernel(GridParams g, RunState rs) {
  const int n = *rs.step;
  double b = *rs.balance;
  if (n >= 0 && n < g.pulse_steps) b += g.inj_step;
  b -= rs.escaped[n] + rs.absorbed[n];
  *rs.balance = b;
  rs.residual[n] = b - rs.energy[n];
  *rs.step = n + 1;
}

// ----------------------------------------------------------------------------------------
// Index interfaces (Eqs. 13-14): at each interface voxel the light arriving through an
// index step is split into its specular and Snell directions.  Gather form, one warp per
// voxel: the warp stages the voxel's Q column in shared memory, then each lane forms its
// output directions as keep[d] Q[d] + sum_e w_e Q[src_e] in a fixed order.
// ----------------------------------------------------------------------------------------
constexpr int kIfaceWarps = 4;

__global__ void __launch_bounds__(32 * kIfaceWarps)
    interface_kernel(int nvox, int na, const int* __restrict__ vox, const int* __restrict__ rowptr,
                     const int* __restrict__ src, const float* __restrict__ w,
                     const uint8_t* __restrict__ keep, float* __restrict__ Q, size_t plane) {
  extern __shared__ float qs[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kIfaceWarps + warp;
  if (i >= nvox) return;  // whole warp
  float* q = qs + warp * na;
  const size_t v = static_cast<size_t>(vox[i]);
  for (int d = lane; d < na; d += 32) q[d] = Q[static_cast<size_t>(d) * plane + v];
  __syncwarp();
  const int* rp = rowptr + static_cast<size_t>(i) * (na + 1);
  const uint8_t* kp = keep + static_cast<size_t>(i) * na;
  for (int d = lane; d < na; d += 32) {
    float out = kp[d] ? q[d] : 0.0f;
    for (int e = rp[d]; e < rp[d + 1]; ++e) out = fmaf(w[e], q[src[e]], out);
    Q[static_cast<size_t>(d) * plane + v] = out;
  }
}

}  // namespace

cudaError_t launch_scatter_fp32(const GridParams& g, const float* b1ds, int nch, const float* P,
                                const float* rcorr, const float* Q, const float* mut,
                                const float* eps, const float* nidx, float* Iring, float* Sring,
                                float tol, int max_iters, RunState rs, cudaStream_t st) {
  const int tiles = (g.nv + kTile - 1) / kTile;
  switch (g.na) {
    case 12:
      scatter_fp32_kernel<12><<<tiles, ScatterCfg<12>::kThreads, 0, st>>>(
          g, b1ds, nch, P, rcorr, Q, mut, eps, nidx, Iring, Sring, tol, max_iters, rs);
      break;
    case 48:
      scatter_fp32_kernel<48><<<tiles, ScatterCfg<48>::kThreads, 0, st>>>(
          g, b1ds, nch, P, rcorr, Q, mut, eps, nidx, Iring, Sring, tol, max_iters, rs);
      break;
    case 192:
      scatter_fp32_kernel<192><<<tiles, ScatterCfg<192>::kThreads, 0, st>>>(
          g, b1ds, nch, P, rcorr, Q, mut, eps, nidx, Iring, Sring, tol, max_iters, rs);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_tally(const GridParams& g, const DirInfo* dirs, const float* Iring,
                         const int* det_vox, const int* det_dir, const float* det_w,
                         const int* det_id, int n_det_entries, double* det, int nbins,
                         RunState rs, cudaStream_t st) {
  const int maxface = g.nx * g.ny > g.ny * g.nz ? (g.nx * g.ny > g.nx * g.nz ? g.nx * g.ny : g.nx * g.nz)
                                                 : (g.ny * g.nz > g.nx * g.nz ? g.ny * g.nz : g.nx * g.nz);
  int bx = (maxface + 255) / 256;
  if (bx > 64) bx = 64;
  dim3 grid(bx, 7);
  tally_kernel<<<grid, 256, 0, st>>>(g, dirs, Iring, det_vox, det_dir, det_w, det_id,
                                     n_det_entries, det, nbins, rs);
  return cudaGetLastError();
}

cudaError_t launch_interface(int nvox, int na, const int* vox, const int* rowptr, const int* src,
                             const float* w, const uint8_t* keep, float* Q, int nv, cudaStream_t st) {
  if (nvox == 0) return cudaSuccess;
  const int blocks = (nvox + kIfaceWarps - 1) / kIfaceWarps;
  interface_kernel<<<blocks, 32 * kIfaceWarps, kIfaceWarps * na * sizeof(float), st>>>(
      nvox, na, vox, rowptr, src, w, keep, Q, static_cast<size_t>(nv));
  return cudaGetLastError();
}

cudaError_t launch_energy_density(const GridParams& g, const float* I, const float* nidx, float scale, float* u,
                                  cudaStream_t st) {
  int blocks = (g.nv + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  energy_density_kernel<<<blocks, 256, 0, st>>>(g, I, nidx, scale, u);
  return cudaGetLastError();
}

cudaError_t launch_advance(const GridParams& g, RunState rs, cudaStream_t st) {
  advance_kernel<<<1, 1, 0, st>>>(g, rs);
  return cudaGetLastError();
}

}  // namespace trinity
