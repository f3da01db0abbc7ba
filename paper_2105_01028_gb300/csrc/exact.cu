// Exact per-voxel source function for piecewise-uniform optics.  The source iteration of
// Eq. 12 (Section 2.4 steps 5-6) converges to the fixed point of S = a P (Q + b1 S); a
// voxel's system depends on it only through (mu_t, a), so voxels of one optics class share
// M = (I - a P B1)^-1 a P (built on the host in FP64 from the FP32 phase matrix with its
// diagonal correction) and S = M Q is one product per voxel instead of an iteration.
//
// Mapping as in the FP32 iteration kernel: a CTA owns 32 voxels, thread i < NA owns output
// direction i; the tile's Q is staged in shared memory as X[j][v]; for every class present
// in the tile, acc[v] = sum_j M[i][j] X[j][v] in blocked sums of 8 terms (M stored
// transposed, so a warp reads a contiguous row of it).  Then I = Q + b1 S, the box energy
// and max |S| as in the iteration kernels.
#include <cstdint>

#include "device.cuh"

namespace trinity {

namespace {

constexpr int kTile = 32;
constexpr int kXStride = kTile + 4;

template <int NA>
struct ExCfg {
  static constexpr int kThreads = ((NA + 31) / 32) * 32;
  static constexpr int kWarps = kThreads / 32;
};

template <int NA>
__global__ void __launch_bounds__(ExCfg<NA>::kThreads)
    exact_fp32_kernel(GridParams g, const float* __restrict__ b1ds, int nch, const float* __restrict__ Mt,
                      const uint8_t* __restrict__ cls, const float* __restrict__ Q,
                      const float* __restrict__ mut, const float* __restrict__ nidx,
                      float* __restrict__ Iring, float* __restrict__ Sring, RunState rs) {
  constexpr int W = ExCfg<NA>::kWarps;
  __shared__ __align__(16) float Xs[NA][kXStride];
  __shared__ int cls_s[kTile];
  __shared__ unsigned present_s;
  __shared__ double esum_s[W];
  __shared__ float smax_s[W];

  const int n = *rs.step;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int i = tid;
  const bool live = i < NA;
  const int v0 = blockIdx.x * kTile;
  const size_t plane = static_cast<size_t>(g.nv);

  if (tid == 0) present_s = 0u;
  __syncthreads();
  if (tid < kTile) {
    const int v = v0 + tid;
    const int c = v < g.nv ? static_cast<int>(cls[v]) : -1;
    cls_s[tid] = c;
    if (c >= 0) atomicOr(&present_s, 1u << c);
  }
  if (live) {
#pragma unroll
    for (int v = 0; v < kTile; v += 4) {
      float4 x4;
      x4.x = v0 + v + 0 < g.nv ? __ldg(Q + static_cast<size_t>(i) * plane + v0 + v + 0) : 0.0f;
      x4.y = v0 + v + 1 < g.nv ? __ldg(Q + static_cast<size_t>(i) * plane + v0 + v + 1) : 0.0f;
      x4.z = v0 + v + 2 < g.nv ? __ldg(Q + static_cast<size_t>(i) * plane + v0 + v + 2) : 0.0f;
      x4.w = v0 + v + 3 < g.nv ? __ldg(Q + static_cast<size_t>(i) * plane + v0 + v + 3) : 0.0f;
      *reinterpret_cast<float4*>(&Xs[i][v]) = x4;
    }
  }
  __syncthreads();

  float s[kTile];
#pragma unroll
  for (int v = 0; v < kTile; ++v) s[v] = 0.0f;
  unsigned present = present_s;
  while (present != 0u) {
    const int c = __ffs(present) - 1;
    present &= present - 1u;
    float acc[kTile];
#pragma unroll
    for (int v = 0; v < kTile; ++v) acc[v] = 0.0f;
    if (live) {
      const float* mcol = Mt + static_cast<size_t>(c) * NA * NA + i;
#pragma unroll 1
      for (int j0 = 0; j0 < NA; j0 += 4) {
        float t[kTile];
#pragma unroll
        for (int v = 0; v < kTile; ++v) t[v] = 0.0f;
#pragma unroll
        for (int j = j0; j < j0 + 4; ++j) {
          const float m = __ldg(mcol + static_cast<size_t>(j) * NA);
          const float4* xr = reinterpret_cast<const float4*>(&Xs[j][0]);
#pragma unroll
          for (int v4 = 0; v4 < kTile / 4; ++v4) {
            const float4 x4 = xr[v4];
            t[4 * v4 + 0] = fmaf(m, x4.x, t[4 * v4 + 0]);
            t[4 * v4 + 1] = fmaf(m, x4.y, t[4 * v4 + 1]);
            t[4 * v4 + 2] = fmaf(m, x4.z, t[4 * v4 + 2]);
            t[4 * v4 + 3] = fmaf(m, x4.w, t[4 * v4 + 3]);
          }
        }
#pragma unroll
        for (int v = 0; v < kTile; ++v) acc[v] += t[v];
      }
    }
#pragma unroll
    for (int v = 0; v < kTile; ++v) s[v] = cls_s[v] == c ? acc[v] : s[v];
  }

  // I = Q + b1 S (b1 the mean over the direction's spacings), tallies
  const size_t cur_off = (static_cast<size_t>(ring_slot(n)) * g.na + (live ? i : 0)) * plane;
  const float* dsl = b1ds + static_cast<size_t>(live ? i : 0) * nch;
  const float inv_nch = 1.0f / static_cast<float>(nch);
  float esum = 0.0f, smax = 0.0f;
  if (live) {
#pragma unroll
    for (int v = 0; v < kTile; ++v) {
      const int vv = v0 + v;
      if (vv < g.nv) {
        const float mu = mut[vv];
        float bs = 0.0f;
        for (int k = 0; k < nch; ++k) {
          const float xo = mu * dsl[k];
          bs += ray_b1(xo, expf(-xo));
        }
        const float Iv = fmaf(bs * inv_nch, s[v], Xs[i][v]);
        Iring[cur_off + vv] = Iv;
        Sring[cur_off + vv] = s[v];
        esum = fmaf(Iv, nidx[vv], esum);
        smax = fmaxf(smax, fabsf(s[v]));
      }
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    esum += __shfl_xor_sync(0xffffffffu, esum, o);
    smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  }
  if (lane == 0) {
    esum_s[warp] = esum;
    smax_s[warp] = smax;
  }
  __syncthreads();
  if (tid == 0) {
    double e = 0.0;
    float sm = 0.0f;
    for (int w = 0; w < W; ++w) {
      e += esum_s[w];
      sm = fmaxf(sm, smax_s[w]);
    }
    int cnt = g.nv - v0 < kTile ? g.nv - v0 : kTile;
    atomicAdd(rs.energy + n, e * static_cast<double>(g.e_scale));
    atomicMax(rs.smax + (n & 1), __float_as_uint(sm));
    atomicMax(rs.iters_max + n, 1);
    atomicAdd(rs.iters_sum + n, static_cast<unsigned long long>(cnt));
  }
}

}  // namespace

cudaError_t launch_exact_fp32(const GridParams& g, const float* b1ds, int nch, const float* Mt,
                              const uint8_t* cls, const float* Q, const float* mut, const float* nidx,
                              float* Iring, float* Sring, RunState rs, cudaStream_t st) {
  const int tiles = (g.nv + kTile - 1) / kTile;
  switch (g.na) {
    case 12:
      exact_fp32_kernel<12><<<tiles, ExCfg<12>::kThreads, 0, st>>>(g, b1ds, nch, Mt, cls, Q, mut, nidx,
                                                                   Iring, Sring, rs);
      break;
    case 48:
      exact_fp32_kernel<48><<<tiles, ExCfg<48>::kThreads, 0, st>>>(g, b1ds, nch, Mt, cls, Q, mut, nidx,
                                                                   Iring, Sring, rs);
      break;
    case 192:
      exact_fp32_kernel<192><<<tiles, ExCfg<192>::kThreads, 0, st>>>(g, b1ds, nch, Mt, cls, Q, mut, nidx,
                                                                     Iring, Sring, rs);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace trinity
