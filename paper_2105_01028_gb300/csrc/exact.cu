// Exact per-voxel source function for piecewise-uniform optics.  The source iteration of
// Eq. 12 (Section 2.4 steps 5-6) converges to the fixed point of S = a P (Q + b1 S); a
// voxel's system depends on it only through (mu_t, a), so voxels of one optics class share
// M = (I - a P B1)^-1 a P (built on the host in FP64 from the FP32 phase matrix with its
// diagonal correction) and S = M Q is one product per voxel instead of an iteration.
//
// 12 and 48 directions, mapping as in the FP32 iteration kernel: a CTA owns 32 voxels,
// thread i < NA owns output direction i; the tile's Q is staged in shared memory as
// X[j][v]; for every class present in the tile, acc[v] = sum_j M[i][j] X[j][v] in blocked
// sums of 4 terms (M stored transposed, so a warp reads a contiguous row of it).  Then
// I = Q + b1 S, the box energy and max |S| as in the iteration kernels.  192 directions
// use the register-blocked form below.
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
                      const uint8_t* __restrict__ cls, const float* __restrict__ mua_cls,
                      const float* __restrict__ Q,
                      const float* __restrict__ mut, const float* __restrict__ nidx,
                      float* __restrict__ Iring, float* __restrict__ Sring, RunState rs) {
  constexpr int W = ExCfg<NA>::kWarps;
  __shared__ __align__(16) float Xs[NA][kXStride];
  __shared__ int cls_s[kTile];
  __shared__ unsigned present_s;
  __shared__ double esum_s[W], asum_s[W];
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
  float esum = 0.0f, asum = 0.0f, smax = 0.0f;
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
        asum = fmaf(Iv, mua_cls[cls_s[v]], asum);
        smax = fmaxf(smax, fabsf(s[v]));
      }
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    esum += __shfl_xor_sync(0xffffffffu, esum, o);
    asum += __shfl_xor_sync(0xffffffffu, asum, o);
    smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  }
  if (lane == 0) {
    esum_s[warp] = esum;
    asum_s[warp] = asum;
    smax_s[warp] = smax;
  }
  __syncthreads();
  if (tid == 0) {
    double e = 0.0, ab = 0.0;
    float sm = 0.0f;
    for (int w = 0; w < W; ++w) {
      e += esum_s[w];
      ab += asum_s[w];
      sm = fmaxf(sm, smax_s[w]);
    }
    int cnt = g.nv - v0 < kTile ? g.nv - v0 : kTile;
    atomicAdd(rs.energy + n, e * static_cast<double>(g.e_scale));
    atomicAdd(rs.absorbed + n, ab * g.a_scale);
    atomicMax(rs.smax + (n & 1), __float_as_uint(sm));
    atomicMax(rs.iters_max + n, 1);
    atomicAdd(rs.iters_sum + n, static_cast<unsigned long long>(cnt));
  }
}

// Register-blocked form for 192 directions.  A CTA of 256 threads owns 64 voxels: lane l
// takes voxels 2l, 2l+1 and warp w directions 24w..24w+23, so each thread keeps a 2 x 24
// block of S.  The tile's Q (all 192 directions x 64 voxels) sits in shared memory; M^T is
// staged through shared memory in chunks of 16 rows.  Per row j a thread loads its two
// values of Q (consecutive across the warp) and 24 of M (the same for the whole warp, a
// broadcast) and issues 48 FMAs; the outputs of a direction are two consecutive voxels per
// lane, so the warp's stores of I and S are contiguous runs.  The sums over j run in order
// (one FP32 product, no iteration to amplify their rounding).  b1 comes from a table per
// (class, direction): within an optics class mu_t is fixed.
constexpr int kGV = 64;     // voxels per CTA
constexpr int kGKc = 16;    // rows of M^T per staged chunk
constexpr int kGNa = 192;
constexpr int kGRi = 24;    // directions per warp

__global__ void __launch_bounds__(256, 2)
    exact_gemm192_kernel(GridParams g, const float* __restrict__ Mt, const float* __restrict__ b1tab,
                         const uint8_t* __restrict__ cls, const float* __restrict__ mua_cls,
                         const float* __restrict__ Q,
                         const float* __restrict__ nidx, float* __restrict__ Iring,
                         float* __restrict__ Sring, RunState rs) {
  extern __shared__ __align__(16) float gsm[];
  float* Xs = gsm;                    // [192][64]
  float* Ms = gsm + kGNa * kGV;       // [16][192]
  __shared__ int cls_s[kGV];
  __shared__ unsigned present_s;
  __shared__ double esum_s[8], asum_s[8];
  __shared__ float smax_s[8];

  const int n = *rs.step;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int vb = blockIdx.x * kGV;
  const size_t plane = static_cast<size_t>(g.nv);
  if (tid == 0) present_s = 0u;
  __syncthreads();
  if (tid < kGV) {
    const int v = vb + tid;
    const int c = v < g.nv ? static_cast<int>(cls[v]) : -1;
    cls_s[tid] = c;
    if (c >= 0) atomicOr(&present_s, 1u << c);
  }
  for (int e = tid; e < kGNa * kGV; e += 256) {
    const int j = e / kGV, v = e % kGV;
    Xs[e] = vb + v < g.nv ? __ldg(Q + static_cast<size_t>(j) * plane + vb + v) : 0.0f;
  }
  __syncthreads();

  const int vl0 = lane * 2, i0 = warp * kGRi;
  const size_t slot = static_cast<size_t>(ring_slot(n)) * g.na;
  float esum = 0.0f, asum = 0.0f, smax = 0.0f;
  unsigned present = present_s;
  while (present != 0u) {
    const int c = __ffs(present) - 1;
    present &= present - 1u;
    float acc[2][kGRi];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < kGRi; ++b) acc[a][b] = 0.0f;
    const float* Mc = Mt + static_cast<size_t>(c) * kGNa * kGNa;
#pragma unroll 1
    for (int j0 = 0; j0 < kGNa; j0 += kGKc) {
      __syncthreads();
      for (int e = tid; e < kGKc * kGNa; e += 256) Ms[e] = __ldg(Mc + static_cast<size_t>(j0) * kGNa + e);
      __syncthreads();
#pragma unroll 2
      for (int jj = 0; jj < kGKc; ++jj) {
        const float2 x = *reinterpret_cast<const float2*>(Xs + (j0 + jj) * kGV + vl0);
        const float4* mr = reinterpret_cast<const float4*>(Ms + jj * kGNa + i0);
#pragma unroll
        for (int q4 = 0; q4 < kGRi / 4; ++q4) {
          const float4 m = mr[q4];
          acc[0][4 * q4 + 0] = fmaf(m.x, x.x, acc[0][4 * q4 + 0]);
          acc[1][4 * q4 + 0] = fmaf(m.x, x.y, acc[1][4 * q4 + 0]);
          acc[0][4 * q4 + 1] = fmaf(m.y, x.x, acc[0][4 * q4 + 1]);
          acc[1][4 * q4 + 1] = fmaf(m.y, x.y, acc[1][4 * q4 + 1]);
          acc[0][4 * q4 + 2] = fmaf(m.z, x.x, acc[0][4 * q4 + 2]);
          acc[1][4 * q4 + 2] = fmaf(m.z, x.y, acc[1][4 * q4 + 2]);
          acc[0][4 * q4 + 3] = fmaf(m.w, x.x, acc[0][4 * q4 + 3]);
          acc[1][4 * q4 + 3] = fmaf(m.w, x.y, acc[1][4 * q4 + 3]);
        }
      }
    }
    // outputs of the voxels of class c
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int vl = vl0 + a, v = vb + vl;
      if (v >= g.nv || cls_s[vl] != c) continue;
      const float nv_idx = nidx[v];
      const float ma = mua_cls[c];
#pragma unroll
      for (int b = 0; b < kGRi; ++b) {
        const int i = i0 + b;
        const float sv = acc[a][b];
        const float Iv = fmaf(__ldg(b1tab + c * kGNa + i), sv, Xs[i * kGV + vl]);
        const size_t o = (slot + i) * plane + v;
        Iring[o] = Iv;
        Sring[o] = sv;
        esum = fmaf(Iv, nv_idx, esum);
        asum = fmaf(Iv, ma, asum);
        smax = fmaxf(smax, fabsf(sv));
      }
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    esum += __shfl_xor_sync(0xffffffffu, esum, o);
    asum += __shfl_xor_sync(0xffffffffu, asum, o);
    smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  }
  if (lane == 0) {
    esum_s[warp] = esum;
    asum_s[warp] = asum;
    smax_s[warp] = smax;
  }
  __syncthreads();
  if (tid == 0) {
    double e = 0.0, ab = 0.0;
    float sm = 0.0f;
    for (int w = 0; w < 8; ++w) {
      e += esum_s[w];
      ab += asum_s[w];
      sm = fmaxf(sm, smax_s[w]);
    }
    const int cnt = g.nv - vb < kGV ? g.nv - vb : kGV;
    atomicAdd(rs.energy + n, e * static_cast<double>(g.e_scale));
    atomicAdd(rs.absorbed + n, ab * g.a_scale);
    atomicMax(rs.smax + (n & 1), __float_as_uint(sm));
    atomicMax(rs.iters_max + n, 1);
    atomicAdd(rs.iters_sum + n, static_cast<unsigned long long>(cnt));
  }
}

}  // namespace

cudaError_t launch_exact_fp32(const GridParams& g, const float* b1ds, int nch, const float* Mt,
                              const float* b1tab, const uint8_t* cls, const float* mua_cls, const float* Q,
                              const float* mut, const float* nidx, float* Iring, float* Sring, RunState rs,
                              cudaStream_t st) {
  if (g.na == kGNa && b1tab) {
    constexpr size_t kDyn = (static_cast<size_t>(kGNa) * kGV + static_cast<size_t>(kGKc) * kGNa) * sizeof(float);
    static cudaError_t attr = [] {
      cudaError_t e = cudaFuncSetAttribute(exact_gemm192_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(kDyn));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(exact_gemm192_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
      return e;
    }();
    if (attr != cudaSuccess) return attr;
    const int blocks = (g.nv + kGV - 1) / kGV;
    exact_gemm192_kernel<<<blocks, 256, kDyn, st>>>(g, Mt, b1tab, cls, mua_cls, Q, nidx, Iring, Sring, rs);
    return cudaGetLastError();
  }
  const int tiles = (g.nv + kTile - 1) / kTile;
  switch (g.na) {
    case 12:
      exact_fp32_kernel<12><<<tiles, ExCfg<12>::kThreads, 0, st>>>(g, b1ds, nch, Mt, cls, mua_cls, Q, mut, nidx,
                                                                   Iring, Sring, rs);
      break;
    case 48:
      exact_fp32_kernel<48><<<tiles, ExCfg<48>::kThreads, 0, st>>>(g, b1ds, nch, Mt, cls, mua_cls, Q, mut, nidx,
                                                                   Iring, Sring, rs);
      break;
    case 192:
      exact_fp32_kernel<192><<<tiles, ExCfg<192>::kThreads, 0, st>>>(g, b1ds, nch, Mt, cls, mua_cls, Q, mut, nidx,
                                                                     Iring, Sring, rs);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace trinity
