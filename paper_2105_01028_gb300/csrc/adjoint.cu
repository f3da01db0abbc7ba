// Discrete adjoint of one time step: the gradient of a detector misfit L with respect to
// mu_a and mu_s per voxel.  The paper has no adjoint (Section 4 names inverse problems as
// future work); these kernels are the exact reverse-mode derivative of the forward
// kernels' scheme (Eqs. 9, 10, 12, 13-14), in FP32 with FP64 gradient sums.
//
// Forward step n, per voxel v and direction d (x = mu_t ds_d):
//   Q_n = F (T I_up + b0 S_up),  S_n = a P (Q_n + b1 S_n),  I_n = Q_n + b1 S_n,
//   E[k][bin(n)] += sum w_e I_n(e) over the detector entries e of detector k.
// Reverse step n, with Ibar_n, Sbar_n holding every later use of level n:
//   Ibar_n += G[k][bin(n)] w_e                                   (adj_inject)
//   y = a P (Sbar_n + b1 Ibar_n + b1 y),  Qbar = Ibar_n + y         (adj_scatter: the
//       transposed scattering solve; P is symmetric, so it has the forward form)
//   dL/da   += sum_d I_n (P z),  z = Sbar_n + b1 Ibar_n + b1 y
//   dL/dmu_t += sum_d ds_d S_n Qbar db1/dx
//   Qpre = F^T Qbar                                               (interface kernel)
//   dL/dmu_t += sum_d ds_d Qpre (dT/dx I_up + db0/dx S_up)          (adj_push)
//   Ibar, Sbar of the upwind sample at levels n-m, n-m-1 += (1-f, f) (T, b0) Qpre
#include <cfloat>
#include <cstdint>

#include "device.cuh"

namespace trinity {

namespace {

__device__ __forceinline__ int pick(int axis, int x, int y, int z) {
  return axis == 0 ? x : (axis == 1 ? y : z);
}

// db1/dx = b0(x) / x.  Below x = 1 the series of b0 divided by x (summed to x^10).
__device__ __forceinline__ float ray_b0_over_x(float x, float T) {
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
    return fmaf(p, x, 0.5f);
  }
  return (1.0f - (1.0f + x) * T) / (x * x);
}

// db0/dx = [T (1 + x + x^2) - 1] / x^2.  Below x = 1 its Taylor series
// sum_{j>=1} (-1)^(j+1) j^2 / (j+1)! x^(j-1), summed to j = 13.
__device__ __forceinline__ float ray_db0(float x, float T) {
  if (x < 1.0f) {
    float p = 169.0f / 87178291200.0f;
    p = fmaf(p, x, -144.0f / 6227020800.0f);
    p = fmaf(p, x, 121.0f / 479001600.0f);
    p = fmaf(p, x, -100.0f / 39916800.0f);
    p = fmaf(p, x, 81.0f / 3628800.0f);
    p = fmaf(p, x, -64.0f / 362880.0f);
    p = fmaf(p, x, 49.0f / 40320.0f);
    p = fmaf(p, x, -36.0f / 5040.0f);
    p = fmaf(p, x, 25.0f / 720.0f);
    p = fmaf(p, x, -16.0f / 120.0f);
    p = fmaf(p, x, 9.0f / 24.0f);
    p = fmaf(p, x, -4.0f / 6.0f);
    return fmaf(p, x, 0.5f);
  }
  return (T * (1.0f + x + x * x) - 1.0f) / (x * x);
}

// After the call lane l holds the warp's reduction of vals[l mod V] (returned): lanes l
// and l ^ s for s >= V first combine all V values, then a butterfly halves the values each
// lane keeps while transposing them across lanes.
template <bool kMax, int V>
__device__ __forceinline__ float warp_transpose(float (&vals)[V], int lane) {
#pragma unroll
  for (int s = 16; s >= V; s >>= 1) {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const float recv = __shfl_xor_sync(0xffffffffu, vals[k], s);
      vals[k] = kMax ? fmaxf(vals[k], recv) : vals[k] + recv;
    }
  }
#pragma unroll
  for (int s = V / 2; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < s; ++k) {
      const float send = upper ? vals[k] : vals[k + s];
      const float keep = upper ? vals[k + s] : vals[k];
      const float recv = __shfl_xor_sync(0xffffffffu, send, s);
      vals[k] = kMax ? fmaxf(keep, recv) : keep + recv;
    }
  }
  return vals[0];
}

// ----------------------------------------------------------------------------------------
// Detector injection: Ibar_n(d_e, v_e) += G[k_e][b] w_e.  Thread 0 also clears the running
// max |y| of this reverse step (read as the floor of the next step's stop rule).
// ----------------------------------------------------------------------------------------
__global__ void adj_inject_kernel(const int* __restrict__ det_vox, const int* __restrict__ det_dir,
                                  const float* __restrict__ det_w, const int* __restrict__ det_id,
                                  int n_entries, const double* __restrict__ G, int nbins, int b,
                                  float* __restrict__ Ib_n, size_t plane, unsigned* ymax_cur) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *ymax_cur = 0u;
  if (b < 0 || b >= nbins) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_entries; e += gridDim.x * blockDim.x) {
    const float val = static_cast<float>(G[static_cast<size_t>(det_id[e]) * nbins + b] *
                                         static_cast<double>(det_w[e]));
    atomicAdd(Ib_n + static_cast<size_t>(det_dir[e]) * plane + det_vox[e], val);
  }
}

// ----------------------------------------------------------------------------------------
// Transposed scattering solve, FP32 on CUDA cores.  Same tiling and iteration as the
// forward FP32 kernel (a CTA owns 16 voxels, thread i owns direction i, blocked sums of
// P X with the diagonal row-sum correction r_i, y = (1 - eps) (P X + r X), the same stop
// rule with a stall exit, the same isotropic rebalance after each plain update) with
// q = Sbar_n + b1 Ibar_n and a warm start from the previous reverse step's y, or (Y2
// given and ``extrap``) its linear extrapolation 2 y(n+1) - y(n+2).  The
// epilogue writes Qbar = Ibar_n + y, clears the consumed adjoint
// level, and adds the voxel's dL/da and the b1 part of dL/dmu_t to the FP64 sums.
// ----------------------------------------------------------------------------------------
constexpr int kTile = 16;  // voxels per CTA: small enough for two CTAs per SM
constexpr int kXStride = kTile + 4;

template <int NA>
struct AdjCfg {
  static constexpr int kThreads = ((NA + 31) / 32) * 32;
  static constexpr int kWarps = kThreads / 32;
};

template <int NA>
__global__ void __launch_bounds__(AdjCfg<NA>::kThreads, 2)
    adj_scatter_fp32_kernel(int nv, const DirInfo* __restrict__ dirs, float ds_max,
                            const float* __restrict__ P, const float* __restrict__ rcorr,
                            const float* __restrict__ mut, const float* __restrict__ eps,
                            float* __restrict__ Ib_n, float* __restrict__ Sb_n,
                            const float* __restrict__ I_n, const float* __restrict__ S_n,
                            float* __restrict__ Y, float* __restrict__ Y2, int extrap,
                            float* __restrict__ Qb, double* __restrict__ gA,
                            double* __restrict__ gmut, float tol, int max_iters,
                            const unsigned* __restrict__ yglob_prev, unsigned* ymax_cur,
                            int* nonconv, unsigned long long* iters_sum) {
  constexpr int W = AdjCfg<NA>::kWarps;
  __shared__ __align__(16) float Xs[2][NA][kXStride];
  __shared__ float red_d[W][32];  // per warp, lane v < kTile holds voxel v's reduction
  __shared__ float red_s[W][32];
  __shared__ float red_c[W][32];
  __shared__ float e_s[kTile], rho_s[kTile], best_s[kTile], den_s[kTile], c_s[kTile];
  __shared__ int stall_s[kTile], iters_s[kTile];
  __shared__ unsigned act_s;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int i = tid;
  const bool live = i < NA;
  const int v0 = blockIdx.x * kTile;
  const size_t plane = static_cast<size_t>(nv);
  const float y_glob = __uint_as_float(*yglob_prev);

  if (tid < kTile) {
    const int v = v0 + tid;
    float ev = 1.0f, rho = 0.0f;
    if (v < nv) {
      ev = eps[v];
      const float xm = mut[v] * ds_max;
      rho = (1.0f - ev) * ray_b1(xm, expf(-xm));
    }
    e_s[tid] = ev;
    rho_s[tid] = rho;
    best_s[tid] = 3.0e38f;
    stall_s[tid] = 0;
    iters_s[tid] = 0;
  }
  if (tid == 0)
    act_s = (nv - v0 >= kTile) ? (kTile == 32 ? 0xffffffffu : ((1u << kTile) - 1u)) : ((1u << (nv - v0)) - 1u);
  __syncthreads();

  float q[kTile], b1[kTile], so[kTile], acc[kTile];
  const float ds = live ? dirs[i].ds : 0.0f;
  const float ri = live ? rcorr[i] : 0.0f;
  const size_t row = static_cast<size_t>(live ? i : 0) * plane;
#pragma unroll
  for (int v = 0; v < kTile; ++v) {
    const int vv = v0 + v;
    const bool ok = live && vv < nv;
    const float xo = ok ? mut[vv] * ds : 0.0f;
    b1[v] = ok ? ray_b1(xo, expf(-xo)) : 0.0f;
    q[v] = ok ? fmaf(b1[v], Ib_n[row + vv], Sb_n[row + vv]) : 0.0f;
    so[v] = ok ? Y[row + vv] : 0.0f;
    if (ok && extrap) so[v] = fmaf(2.0f, so[v], -Y2[row + vv]);
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
    // rebalance denominators sum_j (1 - a b1_j) per voxel
    float bsum[kTile];
#pragma unroll
    for (int v = 0; v < kTile; ++v) bsum[v] = b1[v];
    red_c[warp][lane] = warp_transpose<false>(bsum, lane);
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
  bool first = true;
  // At least one pass, so that acc holds P z of the final iterate for every voxel.
  while ((act != 0u && k < max_iters) || first) {
    first = false;
    ++k;
    __syncthreads();
#pragma unroll
    for (int v = 0; v < kTile; ++v) acc[v] = 0.0f;
    if (live) {
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
    float dsv[kTile], smv[kTile], cvv[kTile];
#pragma unroll
    for (int v = 0; v < kTile; ++v) {
      const bool on = live && ((act >> v) & 1u);
      acc[v] = fmaf(ri, fmaf(b1[v], so[v], q[v]), acc[v]);  // (P + diag r) X
      const float yn = fmaf(-e_s[v], acc[v], acc[v]);
      const float dl = yn - so[v];
      dsv[v] = on ? fabsf(dl) : 0.0f;
      smv[v] = on ? fabsf(yn) : 0.0f;
      cvv[v] = on ? b1[v] * dl : 0.0f;
      so[v] = on ? yn : so[v];
    }
    red_d[warp][lane] = warp_transpose<true>(dsv, lane);
    red_s[warp][lane] = warp_transpose<true>(smv, lane);
    red_c[warp][lane] = warp_transpose<false>(cvv, lane);
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
        const float scale = fmaxf(Sm, 1e-6f * y_glob);
        if (D < best_s[v]) {
          best_s[v] = D;
          stall_s[v] = 0;
        } else {
          stall_s[v] += 1;
        }
        const bool stop = (r / (1.0f - r)) * D <= tol * scale || stall_s[v] >= 3;
        if (stop) {
          done = 1u;
          iters_s[v] = k;
        }
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
  if (tid < kTile && ((act >> tid) & 1u)) iters_s[tid] = k;
  if (tid == 0 && act != 0u) atomicAdd(nonconv, __popc(act));

  // epilogue: Qbar, warm start, cleared adjoint level, gradient sums
  float ga[kTile], gm[kTile];
  float ymx = 0.0f;
  const float db1c = live ? ds : 0.0f;
#pragma unroll
  for (int v = 0; v < kTile; ++v) {
    const int vv = v0 + v;
    ga[v] = 0.0f;
    gm[v] = 0.0f;
    if (live && vv < nv) {
      const size_t o = row + vv;
      const float qbar = Ib_n[o] + so[v];
      Qb[o] = qbar;
      if (Y2) Y2[o] = Y[o];  // this thread read Y[o] in the prologue; it still holds y(n+1)
      Y[o] = so[v];
      Ib_n[o] = 0.0f;
      Sb_n[o] = 0.0f;
      ymx = fmaxf(ymx, fabsf(so[v]));
      ga[v] = I_n[o] * acc[v];  // acc = (P + diag r) z with z = q + b1 y (converged)
      const float xo = mut[vv] * ds;
      gm[v] = db1c * S_n[o] * qbar * ray_b0_over_x(xo, expf(-xo));
    }
  }
  __syncthreads();
  red_d[warp][lane] = warp_transpose<false>(ga, lane);
  red_s[warp][lane] = warp_transpose<false>(gm, lane);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) ymx = fmaxf(ymx, __shfl_xor_sync(0xffffffffu, ymx, o));
  __syncthreads();
  if (tid < kTile && v0 + tid < nv) {
    double sa = 0.0, sm = 0.0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      sa += static_cast<double>(red_d[w][tid]);
      sm += static_cast<double>(red_s[w][tid]);
    }
    gA[v0 + tid] += sa;
    gmut[v0 + tid] += sm;
  }
  if (lane == 0) atomicMax(ymax_cur, __float_as_uint(ymx));
  if (tid == 0) {
    unsigned long long is = 0;
    for (int v = 0; v < kTile && v0 + v < nv; ++v) is += static_cast<unsigned long long>(iters_s[v]);
    atomicAdd(iters_sum, is);
  }
}

// ----------------------------------------------------------------------------------------
// Upwind push and the transport part of dL/dmu_t.  One thread per voxel v loops over the
// directions (so the per-voxel sum over d stays in a register); a warp covers 32
// consecutive x, so every access of a direction's plane is a contiguous run.  Within one
// direction the lattice maps voxels to upwind samples one to one (a translation per
// slab), so no two threads update the same adjoint entry: plain read-modify-writes.
// Forward levels come from the segment store, level L at index L - lev_base.
// ----------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) adj_push_kernel(GridParams g, const DirInfo* __restrict__ dirs,
                                                       const int8_t* __restrict__ offs,
                                                       const float* __restrict__ stI,
                                                       const float* __restrict__ stS, int lev_base,
                                                       int n, const float* __restrict__ mut,
                                                       const float* __restrict__ nidx,
                                                       const float* __restrict__ Qb,
                                                       float* __restrict__ IbR, float* __restrict__ SbR,
                                                       double* __restrict__ gmut) {
  extern __shared__ DirInfo dir_s[];
  for (int d = threadIdx.x; d < g.na; d += blockDim.x) dir_s[d] = dirs[d];
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.nv) return;
  const size_t plane = static_cast<size_t>(g.nv);
  const size_t lplane = plane * g.na;  // one time level of a field
  const int x = v % g.nx, y = (v / g.nx) % g.ny, z = v / (g.nx * g.ny);
  const float mu = __ldg(mut + v);
  const float nv_idx = __ldg(nidx + v);
  float acc = 0.0f;
#pragma unroll 1
  for (int d = 0; d < g.na; ++d) {
    const float qpre = __ldg(Qb + static_cast<size_t>(d) * plane + v);
    if (qpre == 0.0f) continue;
    const DirInfo& di = dir_s[d];
    const int dom = di.dom, sgn = di.sgn, a0 = di.a0, a1 = di.a1;
    const int nd = pick(dom, g.nx, g.ny, g.nz);
    const int n0 = pick(a0, g.nx, g.ny, g.nz);
    const int n1 = pick(a1, g.nx, g.ny, g.nz);
    const int pd = pick(dom, x, y, z), p0 = pick(a0, x, y, z), p1 = pick(a1, x, y, z);
    const int kp = sgn > 0 ? pd : nd - 1 - pd;
    int qd = pd - sgn;
    int q0 = p0 - offs[(static_cast<size_t>(d) * 2 + 0) * g.nmax + kp];
    int q1 = p1 - offs[(static_cast<size_t>(d) * 2 + 1) * g.nmax + kp];
    int kind = 0;
    if (g.periodic) {
      qd = (qd + nd) % nd;
      q0 = (q0 + n0) % n0;
      q1 = (q1 + n1) % n1;
    } else if (kp == 0) {
      kind = 1;
    } else if (q0 < 0 || q0 >= n0 || q1 < 0 || q1 >= n1) {
      kind = 2;
    }
    int m;
    float f;
    retarded_delay(di.dcoef, di.dcoef_lo, nv_idx, m, f);
    const int L0 = n - m, L1 = n - m - 1;
    const float xo = mu * di.ds;
    const float T = expf(-xo);
    const float b0 = ray_b0(xo, T);
    const float db0 = ray_db0(xo, T);
    float Iup = 0.0f, Sup = 0.0f;
    if (kind == 0) {
      const int sd = dom == 0 ? 1 : (dom == 1 ? g.nx : g.nx * g.ny);
      const int s0 = a0 == 0 ? 1 : (a0 == 1 ? g.nx : g.nx * g.ny);
      const int s1 = a1 == 0 ? 1 : (a1 == 1 ? g.nx : g.nx * g.ny);
      const size_t u = static_cast<size_t>(qd) * sd + static_cast<size_t>(q0) * s0 +
                       static_cast<size_t>(q1) * s1;
      const size_t du = static_cast<size_t>(d) * plane + u;
      float i0 = 0.0f, i1 = 0.0f, s0v = 0.0f, s1v = 0.0f;
      if (L0 >= g.hist_from) {
        const size_t o = static_cast<size_t>(L0 - lev_base) * lplane + du;
        i0 = __ldg(stI + o);
        s0v = __ldg(stS + o);
      }
      if (L1 >= g.hist_from) {
        const size_t o = static_cast<size_t>(L1 - lev_base) * lplane + du;
        i1 = __ldg(stI + o);
        s1v = __ldg(stS + o);
      }
      Iup = (1.0f - f) * i0 + f * i1;
      Sup = (1.0f - f) * s0v + f * s1v;
      // push to the upwind sample (levels before 0 are inputs, not parameters)
      const float tq = T * qpre, bq = b0 * qpre;
      if (L0 >= 0) {
        const size_t o = static_cast<size_t>(ring_slot(L0)) * lplane + du;
        IbR[o] = fmaf(1.0f - f, tq, IbR[o]);
        SbR[o] = fmaf(1.0f - f, bq, SbR[o]);
      }
      if (L1 >= 0) {
        const size_t o = static_cast<size_t>(ring_slot(L1)) * lplane + du;
        IbR[o] = fmaf(f, tq, IbR[o]);
        SbR[o] = fmaf(f, bq, SbR[o]);
      }
    } else if (kind == 1 && v == g.src_voxel && di.src_amp != 0.0f) {
      const float on0 = (L0 >= 0 && L0 < g.pulse_steps) ? 1.0f : 0.0f;
      const float on1 = (L1 >= 0 && L1 < g.pulse_steps) ? 1.0f : 0.0f;
      Iup = di.src_amp * ((1.0f - f) * on0 + f * on1);
    }
    acc = fmaf(di.ds * qpre, fmaf(-T, Iup, db0 * Sup), acc);
  }
  gmut[v] += static_cast<double>(acc);
}

__global__ void adj_finish_kernel(int nv, const float* __restrict__ mut, const float* __restrict__ eps,
                                  const double* __restrict__ gA, const double* __restrict__ gmut,
                                  double* __restrict__ gmua, double* __restrict__ gmus) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const double mt = mut[v], e = eps[v];
  // a = mu_s / mu_t: da/dmu_a = -(1 - eps) / mu_t, da/dmu_s = eps / mu_t (0 where mu_t = 0)
  const double ca = mt > 0.0 ? -(1.0 - e) / mt : 0.0;
  const double cs = mt > 0.0 ? e / mt : 0.0;
  gmua[v] = gmut[v] + gA[v] * ca;
  gmus[v] = gmut[v] + gA[v] * cs;
}

// Restore of a checkpoint's scalar state: the step counter and max |S| of level c - 1.
__global__ void adj_restore_kernel(int* step, int c, unsigned* smax, const unsigned* saved) {
  *step = c;
  smax[(c - 1) & 1] = *saved;
}

}  // namespace

cudaError_t launch_adj_inject(const int* det_vox, const int* det_dir, const float* det_w,
                              const int* det_id, int n_entries, const double* G, int nbins, int b,
                              float* Ib_n, int nv, unsigned* ymax_cur, cudaStream_t st) {
  int blocks = (n_entries + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 152) blocks = 152;
  adj_inject_kernel<<<blocks, 256, 0, st>>>(det_vox, det_dir, det_w, det_id, n_entries, G, nbins, b,
                                            Ib_n, static_cast<size_t>(nv), ymax_cur);
  return cudaGetLastError();
}

cudaError_t launch_adj_scatter_fp32(const GridParams& g, const DirInfo* dirs, const float* P,
                                    const float* rcorr, const float* mut, const float* eps,
                                    float* Ib_n, float* Sb_n, const float* I_n, const float* S_n,
                                    float* Y, float* Y2, int extrap, float* Qb, double* gA, double* gmut,
                                    float tol,
                                    int max_iters, const unsigned* yglob_prev, unsigned* ymax_cur,
                                    int* nonconv, unsigned long long* iters_sum, cudaStream_t st) {
  const int tiles = (g.nv + kTile - 1) / kTile;
#define TRINITY_ADJ_CASE(NA)                                                                   \
  case NA:                                                                                     \
    adj_scatter_fp32_kernel<NA><<<tiles, AdjCfg<NA>::kThreads, 0, st>>>(                       \
        g.nv, dirs, g.ds_max, P, rcorr, mut, eps, Ib_n, Sb_n, I_n, S_n, Y, Y2, extrap, Qb, gA,  \
        gmut, tol,                                                                             \
        max_iters, yglob_prev, ymax_cur, nonconv, iters_sum);                                  \
    break;
  switch (g.na) {
    TRINITY_ADJ_CASE(12)
    TRINITY_ADJ_CASE(48)
    TRINITY_ADJ_CASE(192)
    default:
      return cudaErrorInvalidValue;
  }
#undef TRINITY_ADJ_CASE
  return cudaGetLastError();
}

cudaError_t launch_adj_push(const GridParams& g, const DirInfo* dirs, const int8_t* offs,
                            const float* stI, const float* stS, int lev_base, int n,
                            const float* mut, const float* nidx, const float* Qb, float* IbR,
                            float* SbR, double* gmut, cudaStream_t st) {
  const int blocks = (g.nv + 255) / 256;
  adj_push_kernel<<<blocks, 256, g.na * sizeof(DirInfo), st>>>(g, dirs, offs, stI, stS, lev_base, n,
                                                               mut, nidx, Qb, IbR, SbR, gmut);
  return cudaGetLastError();
}

cudaError_t launch_adj_finish(int nv, const float* mut, const float* eps, const double* gA,
                              const double* gmut, double* gmua, double* gmus, cudaStream_t st) {
  adj_finish_kernel<<<(nv + 255) / 256, 256, 0, st>>>(nv, mut, eps, gA, gmut, gmua, gmus);
  return cudaGetLastError();
}

cudaError_t launch_adj_restore(int* step, int c, unsigned* smax, const unsigned* saved,
                               cudaStream_t st) {
  adj_restore_kernel<<<1, 1, 0, st>>>(step, c, smax, saved);
  return cudaGetLastError();
}

}  // namespace trinity
