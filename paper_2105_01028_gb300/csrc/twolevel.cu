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

// blockIdx.y = coarse direction c; a block covers whole x-rows as in the one-level sweep.
// kUniN / kUniMu: uniform refractive index / mu_t, so each child's delay split (m, f) /
// exp(-x) and b0(x) are taken once per block (same FP32 operations on the same values).
template <bool kUniN, bool kUniMu>
__global__ void __launch_bounds__(256) sweep2_kernel(GridParams g, const DirInfo* __restrict__ dirs,
                                                     const int8_t* __restrict__ offs,
                                                     const int* __restrict__ children, int nch, int na_s,
                                                     const float* __restrict__ Iring,
                                                     const float* __restrict__ Sring,
                                                     const float* __restrict__ mut,
                                                     const float* __restrict__ nidx,
                                                     float* __restrict__ Qf, float* __restrict__ Qc,
                                                     RunState rs) {
  extern __shared__ DirInfo ch_s[];  // the nch children's constants
  __shared__ int n_s;
  __shared__ int chd_s[64];
  __shared__ int m_s[kUniN ? 64 : 1];
  __shared__ float f_s[kUniN ? 64 : 1];
  __shared__ float T_s[kUniMu ? 64 : 1];
  __shared__ float b0_s[kUniMu ? 64 : 1];
  const int c = blockIdx.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int k = tid; k < nch; k += blockDim.x * blockDim.y) {
    const int d = children[c * nch + k];
    const DirInfo di = dirs[d];
    chd_s[k] = d;
    ch_s[k] = di;
    if (kUniN) {
      int m;
      float f;
      retarded_delay(di.dcoef, di.dcoef_lo, g.n_u, m, f);
      m_s[k] = m;
      f_s[k] = f;
    }
    if (kUniMu) {
      const float xo = g.mut_u * di.ds;
      const float T = expf(-xo);
      T_s[k] = T;
      b0_s[k] = ray_b0(xo, T);
    }
  }
  if (tid == 0) {
    n_s = *rs.step;
    if (c == 0 && blockIdx.x == 0) {
      rs.smax[n_s & 1] = 0u;
      rs.tile_ctr[n_s & 1] = 0;
    }
  }
  __syncthreads();
  const int row = blockIdx.x * blockDim.y + threadIdx.y;
  if (row >= g.ny * g.nz) return;
  const int n = n_s;
  const int y = row % g.ny, z = row / g.ny;
  const size_t plane = static_cast<size_t>(g.nv);
  const size_t row_base = static_cast<size_t>(row) * g.nx;
  const float* Sc0 = Sring + static_cast<size_t>(c) * plane;  // plane c of a coarse level
  const size_t slevel = static_cast<size_t>(na_s) * plane;
  const size_t ilevel = static_cast<size_t>(g.na) * plane;
  const float inv = 1.0f / static_cast<float>(nch);

  for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
    const size_t v = row_base + x;
    const float mu = kUniMu ? 0.0f : __ldg(mut + v);
    const float nv_idx = kUniN ? 0.0f : __ldg(nidx + v);
    float acc = 0.0f;
    for (int k = 0; k < nch; ++k) {
      const DirInfo& di = ch_s[k];
      const int d = chd_s[k];
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
      if (kUniN) {
        m = m_s[k];
        f = f_s[k];
      } else {
        retarded_delay(di.dcoef, di.dcoef_lo, nv_idx, m, f);
      }
      const int L0 = n - m, L1 = n - m - 1;
      float Iup = 0.0f, Sup = 0.0f;
      if (kind == 0) {
        const int sd = dom == 0 ? 1 : (dom == 1 ? g.nx : g.nx * g.ny);
        const int s0 = a0 == 0 ? 1 : (a0 == 1 ? g.nx : g.nx * g.ny);
        const int s1 = a1 == 0 ? 1 : (a1 == 1 ? g.nx : g.nx * g.ny);
        const size_t u = static_cast<size_t>(qd) * sd + static_cast<size_t>(q0) * s0 +
                         static_cast<size_t>(q1) * s1;
        float i0 = 0.0f, i1 = 0.0f, s0v = 0.0f, s1v = 0.0f;
        if (L0 >= g.hist_from) {
          i0 = __ldg(Iring + static_cast<size_t>(ring_slot(L0)) * ilevel + static_cast<size_t>(d) * plane + u);
          s0v = __ldg(Sc0 + static_cast<size_t>(ring_slot(L0)) * slevel + u);
        }
        if (L1 >= g.hist_from) {
          i1 = __ldg(Iring + static_cast<size_t>(ring_slot(L1)) * ilevel + static_cast<size_t>(d) * plane + u);
          s1v = __ldg(Sc0 + static_cast<size_t>(ring_slot(L1)) * slevel + u);
        }
        Iup = (1.0f - f) * i0 + f * i1;
        Sup = (1.0f - f) * s0v + f * s1v;
      } else if (kind == 1 && static_cast<int>(v) == g.src_voxel && di.src_amp != 0.0f) {
        const float on0 = (L0 >= 0 && L0 < g.pulse_steps) ? 1.0f : 0.0f;
        const float on1 = (L1 >= 0 && L1 < g.pulse_steps) ? 1.0f : 0.0f;
        Iup = di.src_amp * ((1.0f - f) * on0 + f * on1);
      }
      float T, b0;
      if (kUniMu) {
        T = T_s[k];
        b0 = b0_s[k];
      } else {
        const float xo = mu * di.ds;
        T = expf(-xo);
        b0 = ray_b0(xo, T);
      }
      const float q = Iup * T + Sup * b0;
      Qf[static_cast<size_t>(d) * plane + v] = q;
      acc += q;
    }
    Qc[static_cast<size_t>(c) * plane + v] = acc * inv;
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
  dim3 grid((rows + by - 1) / by, na_s);
  const size_t smem = nch * sizeof(DirInfo);
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
