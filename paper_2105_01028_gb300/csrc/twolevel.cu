// Two-level angular grid (Section 2.1, text after Eq. 12): the transport runs on fine
// HEALPix directions, the source function on coarse ones, each coarse bin taking the mean
// intensity of its children (the paper's fiducial runs: 3072 transport directions, 192
// source-function directions, 16 children each).  Per step:
//   sweep2:   Q_f = I_up,f T_f + S_up,par(f) b0_f for every child f of coarse direction c,
//             and Qbar_c = mean over the children (fused: one block row per coarse c)
//   (interface split on Q_f, then recoarsen at the interface voxels)
//   scatter:  the one-level source iteration on coarse arrays, S_c = a P (Qbar + b1bar S)
//             with b1bar_c the mean of the children's b1 (scatter kernels, nch > 1)
//   refine:   I_f = Q_f + b1_f S_par(f)
// The fine-direction order inside each coarse block is the children table's, ascending.
#include <cstdint>

#include "device.cuh"

namespace trinity {

namespace {

__device__ __forceinline__ int pick(int axis, int x, int y, int z) {
  return axis == 0 ? x : (axis == 1 ? y : z);
}

// One child direction's constants, staged in shared memory once per block.
struct Child {
  const float* ilev[5];  // plane d of I at level n - m (m = 0..4), null before the history
  const int8_t* off0;    // per-slab lattice offsets along a0 and a1
  const int8_t* off1;
  float* qf;             // plane d of Q_f
  int dom, sgn, a0, a1, nd, n0, n1, sd, s0, s1;
  float ds, dc_hi, dc_lo, src_amp;
  int m;                 // uniform refractive index: the delay's whole part ...
  float f, T, b0;        // ... and fraction; uniform mu_t: exp(-x) and b0(x)
};

// blockIdx.y = coarse direction c; a block covers whole x-rows as in the one-level sweep
// and strides over kRowSweeps2 groups of rows; each thread loops over the children of c
// for its voxel, so the coarse mean is a register sum in the children table's order.
// kUniN / kUniMu: uniform refractive index / mu_t, so each child's delay split (m, f) /
// exp(-x) and b0(x) are taken once per block (same FP32 operations on the same values).
constexpr int kRowSweeps2 = 4;
constexpr int kGroup = 4;  // children whose upwind loads are in flight together

template <bool kUniN, bool kUniMu>
__global__ void __launch_bounds__(256, 5) sweep2_kernel(GridParams g, const DirInfo* __restrict__ dirs,
                                                     const int8_t* __restrict__ offs,
                                                     const int* __restrict__ children, int nch, int na_s,
                                                     const float* __restrict__ Iring,
                                                     const float* __restrict__ Sring,
                                                     const float* __restrict__ mut,
                                                     const float* __restrict__ nidx,
                                                     float* __restrict__ Qf, float* __restrict__ Qc,
                                                     RunState rs) {
  extern __shared__ uint8_t sm2[];
  Child* cs = reinterpret_cast<Child*>(sm2);  // [nch]
  __shared__ int n_s;
  __shared__ const float* slev_s[5];  // plane c of coarse S at level n - m
  const int c = blockIdx.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const size_t plane = static_cast<size_t>(g.nv);
  if (tid == 0) {
    n_s = *rs.step;
    if (c == 0 && blockIdx.x == 0) {
      rs.smax[n_s & 1] = 0u;
      rs.tile_ctr[n_s & 1] = 0;
    }
  }
  __syncthreads();
  const int n = n_s;
  if (tid < 5) {
    const int L = n - tid;
    slev_s[tid] = L >= g.hist_from ? Sring + (static_cast<size_t>(ring_slot(L)) * na_s + c) * plane : nullptr;
  }
  for (int k = tid; k < nch; k += blockDim.x * blockDim.y) {
    const int d = children[c * nch + k];
    const DirInfo di = dirs[d];
    Child ch;
    for (int mm = 0; mm < 5; ++mm) {
      const int L = n - mm;
      ch.ilev[mm] = L >= g.hist_from ? Iring + (static_cast<size_t>(ring_slot(L)) * g.na + d) * plane : nullptr;
    }
    ch.off0 = offs + (static_cast<size_t>(d) * 2 + 0) * g.nmax;
    ch.off1 = offs + (static_cast<size_t>(d) * 2 + 1) * g.nmax;
    ch.qf = Qf + static_cast<size_t>(d) * plane;
    ch.dom = di.dom;
    ch.sgn = di.sgn;
    ch.a0 = di.a0;
    ch.a1 = di.a1;
    ch.nd = pick(di.dom, g.nx, g.ny, g.nz);
    ch.n0 = pick(di.a0, g.nx, g.ny, g.nz);
    ch.n1 = pick(di.a1, g.nx, g.ny, g.nz);
    ch.sd = di.dom == 0 ? 1 : (di.dom == 1 ? g.nx : g.nx * g.ny);
    ch.s0 = di.a0 == 0 ? 1 : (di.a0 == 1 ? g.nx : g.nx * g.ny);
    ch.s1 = di.a1 == 0 ? 1 : (di.a1 == 1 ? g.nx : g.nx * g.ny);
    ch.ds = di.ds;
    ch.dc_hi = di.dcoef;
    ch.dc_lo = di.dcoef_lo;
    ch.src_amp = di.src_amp;
    ch.m = 1;
    ch.f = ch.T = ch.b0 = 0.0f;
    if (kUniN) {
      int m;
      float f;
      retarded_delay(di.dcoef, di.dcoef_lo, g.n_u, m, f);
      ch.m = m < 1 ? 1 : (m > 3 ? 3 : m);
      ch.f = f;
    }
    if (kUniMu) {
      const float xo = g.mut_u * di.ds;
      const float T = expf(-xo);
      ch.T = T;
      ch.b0 = ray_b0(xo, T);
    }
    cs[k] = ch;
  }
  __syncthreads();
  const int nrows = g.ny * g.nz;
  const float inv = 1.0f / static_cast<float>(nch);
  float* qc = Qc + static_cast<size_t>(c) * plane;

  for (int row = blockIdx.x * blockDim.y + threadIdx.y; row < nrows; row += gridDim.x * blockDim.y) {
    const int y = row % g.ny, z = row / g.ny;
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      const int v = row * g.nx + x;
      const float mu = kUniMu ? 0.0f : __ldg(mut + v);
      const float nv_idx = kUniN ? 0.0f : __ldg(nidx + v);
      float acc = 0.0f;
      // children in groups of kGroup: the group's upwind loads are issued together, then
      // its Q_f are formed and stored in the children table's order
      for (int k0 = 0; k0 < nch; k0 += kGroup) {
        float i0[kGroup], i1[kGroup], s0v[kGroup], s1v[kGroup], fw[kGroup];
        int kind[kGroup], mg[kGroup];
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
          i0[j] = i1[j] = s0v[j] = s1v[j] = 0.0f;
          kind[j] = 3;
          mg[j] = 1;
          fw[j] = 0.0f;
          const int k = k0 + j;
          if (k >= nch) continue;
          const Child& ch = cs[k];
          const int dom = ch.dom, sgn = ch.sgn, nd = ch.nd, n0 = ch.n0, n1 = ch.n1;
          const int pd = pick(dom, x, y, z), p0 = pick(ch.a0, x, y, z), p1 = pick(ch.a1, x, y, z);
          const int kp = sgn > 0 ? pd : nd - 1 - pd;
          int qd = pd - sgn;
          int q0 = p0 - ch.off0[kp];
          int q1 = p1 - ch.off1[kp];
          int kd = 0;
          if (g.periodic) {
            qd = (qd + nd) % nd;
            q0 = (q0 + n0) % n0;
            q1 = (q1 + n1) % n1;
          } else if (kp == 0) {
            kd = 1;
          } else if (q0 < 0 || q0 >= n0 || q1 < 0 || q1 >= n1) {
            kd = 2;
          }
          int m;
          float f;
          if (kUniN) {
            m = ch.m;
            f = ch.f;
          } else {
            retarded_delay(ch.dc_hi, ch.dc_lo, nv_idx, m, f);
            m = m < 1 ? 1 : (m > 3 ? 3 : m);  // the optics check keeps every delay in [1, 4)
          }
          kind[j] = kd;
          mg[j] = m;
          fw[j] = f;
          if (kd == 0) {
            const int u = qd * ch.sd + q0 * ch.s0 + q1 * ch.s1;  // < nv <= 2^30
            const float* i0p = ch.ilev[m];
            const float* i1p = ch.ilev[m + 1];
            if (i0p) {
              i0[j] = __ldg(i0p + u);
              s0v[j] = __ldg(slev_s[m] + u);
            }
            if (i1p) {
              i1[j] = __ldg(i1p + u);
              s1v[j] = __ldg(slev_s[m + 1] + u);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
          if (kind[j] == 3) break;
          const Child& ch = cs[k0 + j];
          const float f = fw[j];
          float Iup = 0.0f, Sup = 0.0f;
          if (kind[j] == 0) {
            Iup = (1.0f - f) * i0[j] + f * i1[j];
            Sup = (1.0f - f) * s0v[j] + f * s1v[j];
          } else if (kind[j] == 1 && v == g.src_voxel && ch.src_amp != 0.0f) {
            const int L0 = n - mg[j], L1 = n - mg[j] - 1;
            const float on0 = (L0 >= 0 && L0 < g.pulse_steps) ? 1.0f : 0.0f;
            const float on1 = (L1 >= 0 && L1 < g.pulse_steps) ? 1.0f : 0.0f;
            Iup = ch.src_amp * ((1.0f - f) * on0 + f * on1);
          }
          float T, b0;
          if (kUniMu) {
            T = ch.T;
            b0 = ch.b0;
          } else {
            const float xo = mu * ch.ds;
            T = expf(-xo);
            b0 = ray_b0(xo, T);
          }
          const float q = Iup * T + Sup * b0;
          ch.qf[v] = q;
          acc += q;
        }
      }
      qc[v] = acc * inv;
    }
  }
}

// I_f(n) = Q_f + b1_f S_c(n) for every child f of coarse direction c = blockIdx.y.
// kUniMu: uniform mu_t, so each child's b1 is taken once per block.
template <bool kUniMu>
__global__ void __launch_bounds__(256) refine_kernel(GridParams g, const DirInfo* __restrict__ dirs,
                                                     const int* __restrict__ children, int nch, int na_s,
                                                     const float* __restrict__ mut,
                                                     const float* __restrict__ Qf,
                                                     const float* __restrict__ Sring,
                                                     float* __restrict__ Iring, RunState rs) {
  __shared__ int n_s;
  __shared__ int chd_s[64];
  __shared__ float ds_s[64];  // the child's ds, or its b1 when mu_t is uniform
  const int c = blockIdx.y;
  const int tid = threadIdx.x;
  for (int k = tid; k < nch; k += blockDim.x) {
    const int d = children[c * nch + k];
    chd_s[k] = d;
    if (kUniMu) {
      const float xo = g.mut_u * dirs[d].ds;
      ds_s[k] = ray_b1(xo, expf(-xo));
    } else {
      ds_s[k] = dirs[d].ds;
    }
  }
  if (tid == 0) n_s = *rs.step;
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + tid;
  if (v >= g.nv) return;
  const int n = n_s;
  const size_t plane = static_cast<size_t>(g.nv);
  const float s = Sring[(static_cast<size_t>(ring_slot(n)) * na_s + c) * plane + v];
  const float mu = kUniMu ? 0.0f : mut[v];
  float* Iout = Iring + static_cast<size_t>(ring_slot(n)) * g.na * plane;
  for (int k = 0; k < nch; ++k) {
    const size_t o = static_cast<size_t>(chd_s[k]) * plane + v;
    float b1;
    if (kUniMu) {
      b1 = ds_s[k];
    } else {
      const float xo = mu * ds_s[k];
      b1 = ray_b1(xo, expf(-xo));
    }
    Iout[o] = fmaf(b1, s, Qf[o]);
  }
}

// Qbar_c at the interface voxels after the split changed their Q_f (warp per voxel).
__global__ void recoarsen_kernel(int nvox, const int* __restrict__ vox, const int* __restrict__ children,
                                 int nch, int na_s, const float* __restrict__ Qf, float* __restrict__ Qc,
                                 size_t plane) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nvox) return;
  const size_t v = static_cast<size_t>(vox[warp]);
  const float inv = 1.0f / static_cast<float>(nch);
  for (int c = lane; c < na_s; c += 32) {
    float acc = 0.0f;
    for (int k = 0; k < nch; ++k) acc += Qf[static_cast<size_t>(children[c * nch + k]) * plane + v];
    Qc[static_cast<size_t>(c) * plane + v] = acc * inv;
  }
}

}  // namespace

cudaError_t launch_sweep2(const GridParams& g, const DirInfo* dirs, const int8_t* offs, const int* children,
                          int nch, int na_s, const float* Iring, const float* Sring, const float* mut,
                          const float* nidx, float* Qf, float* Qc, RunState rs, cudaStream_t st) {
  if (nch < 1 || nch > 64) return cudaErrorInvalidValue;
  int bx = ((g.nx + 31) / 32) * 32;
  if (bx > 256) bx = 256;
  const int by = 256 / bx;
  const int rows = g.ny * g.nz;
  dim3 block(bx, by);
  const int groups = (rows + by - 1) / by;
  dim3 grid((groups + kRowSweeps2 - 1) / kRowSweeps2, na_s);
  const size_t smem = nch * sizeof(Child);
  const bool un = g.n_u >= 1.0f, um = g.mut_u >= 0.0f;
  if (un && um)
    sweep2_kernel<true, true><<<grid, block, smem, st>>>(g, dirs, offs, children, nch, na_s, Iring, Sring, mut,
                                                         nidx, Qf, Qc, rs);
  else if (un)
    sweep2_kernel<true, false><<<grid, block, smem, st>>>(g, dirs, offs, children, nch, na_s, Iring, Sring, mut,
                                                          nidx, Qf, Qc, rs);
  else if (um)
    sweep2_kernel<false, true><<<grid, block, smem, st>>>(g, dirs, offs, children, nch, na_s, Iring, Sring, mut,
                                                          nidx, Qf, Qc, rs);
  else
    sweep2_kernel<false, false><<<grid, block, smem, st>>>(g, dirs, offs, children, nch, na_s, Iring, Sring,
                                                           mut, nidx, Qf, Qc, rs);
  return cudaGetLastError();
}

cudaError_t launch_refine(const GridParams& g, const DirInfo* dirs, const int* children, int nch, int na_s,
                          const float* mut, const float* Qf, const float* Sring, float* Iring, RunState rs,
                          cudaStream_t st) {
  if (nch < 1 || nch > 64) return cudaErrorInvalidValue;
  dim3 grid((g.nv + 255) / 256, na_s);
  if (g.mut_u >= 0.0f)
    refine_kernel<true><<<grid, 256, 0, st>>>(g, dirs, children, nch, na_s, mut, Qf, Sring, Iring, rs);
  else
    refine_kernel<false><<<grid, 256, 0, st>>>(g, dirs, children, nch, na_s, mut, Qf, Sring, Iring, rs);
  return cudaGetLastError();
}

cudaError_t launch_recoarsen(int nvox, const int* vox, const int* children, int nch, int na_s, const float* Qf,
                             float* Qc, int nv, cudaStream_t st) {
  if (nvox == 0) return cudaSuccess;
  const int threads = 128;
  const int blocks = (nvox * 32 + threads - 1) / threads;
  recoarsen_kernel<<<blocks, threads, 0, st>>>(nvox, vox, children, nch, na_s, Qf, Qc, static_cast<size_t>(nv));
  return cudaGetLastError();
}

}  // namespace trinity
