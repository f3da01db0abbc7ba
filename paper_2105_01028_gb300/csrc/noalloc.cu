// Source iteration on caller-owned device buffers, with no device allocation at all.
//
// Some callers cannot call cudaMalloc at the point where they need a solve: code that
// runs inside a region where the device allocator must not be touched (for example a
// framework's own memory pool that owns every byte of the device, or a real-time loop
// that forbids allocation), or callers that hand out their own preallocated buffers and
// expect a library call to add nothing to the device footprint.  This file gives them
// one entry point that uses no allocator: the kernel's scratch memory (per-voxel
// contraction bounds, a max-reduction cell and iteration counters) lives in a
// file-scope static device array of fixed size, which every GPU that loads the library
// holds until the process exits.  Inputs and outputs are still the caller's.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "device.cuh"
#include "trinity.h"

namespace trinity {
namespace {

constexpr int kNoAllocMaxVoxels = 1 << 20;  // 1,048,576 voxels: 4 MiB of bounds
constexpr int kNaTile = 32;                   // voxels per CTA (as in the FP32 kernel)
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
  unsigned smax;       // max |S_prev| as float bits (the stop rule's floor scale)
  int iters_max;       // largest iteration count of the call
  int nonconv;         // voxels that reached max_iters
  int pad;
  float rho[kNoAllocMaxVoxels];  // per-voxel contraction bound (1 - eps) max_d b1
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array for the current device (looked up once per
// device; in host code the symbol's name is only a host-side stand-in).
int scratch_for_current_device(NoAllocScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TRINITY_E_CUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TRINITY_E_CUDA;
    g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_scratch_ptr[dev];
  return TRINITY_OK;
}

// Per voxel: rho = (1 - eps) max_d b1; and max |S_prev| over everything.
__global__ void noalloc_prepass(int na, int nvox, const float* __restrict__ b1, const float* __restrict__ eps,
                                const float* __restrict__ S_prev, NoAllocScratch* sc) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  float sm = 0.0f;
  if (v < nvox) {
    float bmax = 0.0f;
    for (int d = 0; d < na; ++d) {
      bmax = fmaxf(bmax, b1[static_cast<size_t>(d) * nvox + v]);
      sm = fmaxf(sm, fabsf(S_prev[static_cast<size_t>(d) * nvox + v]));
    }
    sc->rho[v] = (1.0f - eps[v]) * bmax;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) sm = fmaxf(sm, __shfl_xor_sync(0xffffffffu, sm, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&sc->smax, __float_as_uint(sm));
}

__device__ __forceinline__ float noalloc_transpose_max(float (&vals)[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < s; ++k) {
      const float send = upper ? vals[k] : vals[k + s];
      const float keep = upper ? vals[k + s] : vals[k];
      const float recv = __shfl_xor_sync(0xffffffffu, send, s);
      vals[k] = fmaxf(keep, recv);
    }
  }
  return vals[0];
}

// The FP32 source iteration (same arithmetic and stop rule as the context path), with b1
// given per (direction, voxel) instead of derived from the optics, and its scratch in the
// static array.
template <int NA>
__global__ void __launch_bounds__(((NA + 31) / 32) * 32)
    noalloc_iteration(int nvox, const float* __restrict__ P, const float* __restrict__ Q,
                      const float* __restrict__ b1g, const float* __restrict__ eps,
                      const float* __restrict__ S_prev, float* __restrict__ S_out, float* __restrict__ I_out,
                      float tol, int max_iters, NoAllocScratch* sc) {
  constexpr int W = ((NA + 31) / 32);
  constexpr int kBlk = (NA % 8 == 0) ? 8 : 4;
  __shared__ __align__(16) float Xs[2][NA][kNaTile + 4];
  __shared__ float red_d[W][kNaTile], red_s[W][kNaTile];
  __shared__ float e_s[kNaTile], rho_s[kNaTile], best_s[kNaTile];
  __shared__ int iters_s[kNaTile], stall_s[kNaTile];
  __shared__ unsigned act_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = tid;
  const bool live = i < NA;
  const int v0 = blockIdx.x * kNaTile;
  const size_t plane = static_cast<size_t>(nvox);
  const float s_glob = __uint_as_float(sc->smax);
  if (tid < kNaTile) {
    const int v = v0 + tid;
    e_s[tid] = v < nvox ? eps[v] : 1.0f;
    rho_s[tid] = v < nvox ? sc->rho[v] : 0.0f;
    best_s[tid] = 3.0e38f;
    stall_s[tid] = 0;
    iters_s[tid] = 0;
  }
  if (tid == 0) act_s = (nvox - v0 >= kNaTile) ? 0xffffffffu : ((1u << (nvox - v0)) - 1u);
  // row-sum correction of this P (FP64 sum): P + diag(r) has unit row sums
  float ri = 0.0f;
  if (live) {
    double rs = 0.0;
    for (int j = 0; j < NA; ++j) rs += static_cast<double>(P[static_cast<size_t>(i) * NA + j]);
    ri = static_cast<float>(1.0 - rs);
  }
  __syncthreads();
  float q[kNaTile], b1[kNaTile], so[kNaTile], acc[kNaTile];
#pragma unroll
  for (int v = 0; v < kNaTile; ++v) {
    const int vv = v0 + v;
    const bool ok = live && vv < nvox;
    q[v] = ok ? Q[static_cast<size_t>(i) * plane + vv] : 0.0f;
    b1[v] = ok ? b1g[static_cast<size_t>(i) * plane + vv] : 0.0f;
    so[v] = ok ? S_prev[static_cast<size_t>(i) * plane + vv] : 0.0f;
  }
  if (live) {
#pragma unroll
    for (int v = 0; v < kNaTile; v += 4)
      *reinterpret_cast<float4*>(&Xs[0][i][v]) =
          make_float4(q[v] + b1[v] * so[v], q[v + 1] + b1[v + 1] * so[v + 1], q[v + 2] + b1[v + 2] * so[v + 2],
                      q[v + 3] + b1[v + 3] * so[v + 3]);
  }
  unsigned act = act_s;
  int cur = 0, k = 0;
  while (act != 0u && k < max_iters) {
    ++k;
    __syncthreads();
#pragma unroll
    for (int v = 0; v < kNaTile; ++v) acc[v] = 0.0f;
    if (live) {
#pragma unroll 1
      for (int j0 = 0; j0 < NA; j0 += kBlk) {
        float t[kNaTile];
#pragma unroll
        for (int v = 0; v < kNaTile; ++v) t[v] = 0.0f;
#pragma unroll
        for (int j = j0; j < j0 + kBlk; ++j) {
          const float p = __ldg(P + static_cast<size_t>(j) * NA + i);  // P symmetric
          const float4* xr = reinterpret_cast<const float4*>(&Xs[cur][j][0]);
#pragma unroll
          for (int v4 = 0; v4 < kNaTile / 4; ++v4) {
            const float4 x4 = xr[v4];
            t[4 * v4 + 0] = fmaf(p, x4.x, t[4 * v4 + 0]);
            t[4 * v4 + 1] = fmaf(p, x4.y, t[4 * v4 + 1]);
            t[4 * v4 + 2] = fmaf(p, x4.z, t[4 * v4 + 2]);
            t[4 * v4 + 3] = fmaf(p, x4.w, t[4 * v4 + 3]);
          }
        }
#pragma unroll
        for (int v = 0; v < kNaTile; ++v) acc[v] += t[v];
      }
    }
    float dsv[kNaTile], smv[kNaTile];
#pragma unroll
    for (int v = 0; v < kNaTile; ++v) {
      const bool on = live && ((act >> v) & 1u);
      const float y = fmaf(ri, fmaf(b1[v], so[v], q[v]), acc[v]);
      const float sn = fmaf(-e_s[v], y, y);
      dsv[v] = on ? fabsf(sn - so[v]) : 0.0f;
      smv[v] = on ? fabsf(sn) : 0.0f;
      so[v] = on ? sn : so[v];
    }
    const int nxt = cur ^ 1;
    if (live) {
#pragma unroll
      for (int v = 0; v < kNaTile; v += 4)
        *reinterpret_cast<float4*>(&Xs[nxt][i][v]) =
            make_float4(q[v] + b1[v] * so[v], q[v + 1] + b1[v + 1] * so[v + 1], q[v + 2] + b1[v + 2] * so[v + 2],
                        q[v + 3] + b1[v + 3] * so[v + 3]);
    }
    red_d[warp][lane] = noalloc_transpose_max(dsv, lane);
    red_s[warp][lane] = noalloc_transpose_max(smv, lane);
    __syncthreads();
    if (tid < kNaTile) {
      const int v = tid;
      unsigned done = 0u;
      if ((act >> v) & 1u) {
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
        if ((r / (1.0f - r)) * D <= tol * scale || stall_s[v] >= 3) {
          done = 1u;
          iters_s[v] = k;
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, done);
      if (tid == 0) act_s = act & ~mask;
    }
    __syncthreads();
    act = act_s;
    cur = nxt;
  }
  if (tid < kNaTile && ((act >> tid) & 1u)) {
    iters_s[tid] = k;
    atomicAdd(&sc->nonconv, 1);
  }
  if (live) {
#pragma unroll
    for (int v = 0; v < kNaTile; ++v) {
      const int vv = v0 + v;
      if (vv < nvox) {
        S_out[static_cast<size_t>(i) * plane + vv] = so[v];
        I_out[static_cast<size_t>(i) * plane + vv] = fmaf(b1[v], so[v], q[v]);
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    int im = 0;
    for (int v = 0; v < kNaTile && v0 + v < nvox; ++v) im = max(im, iters_s[v]);
    atomicMax(&sc->iters_max, im);
  }
}

}  // namespace
}  // namespace trinity

using namespace trinity;

extern "C" int trinity_source_iteration_noalloc(int na, int nvox, const float* P, const float* Q, const float* b1,
                                                const float* eps, const float* S_prev, float* S_out, float* I_out,
                                                double tol, int max_iters, int* iters_max, void* stream) {
  if (na != 12 && na != 48 && na != 192) return TRINITY_E_INVALID;
  if (nvox < 1 || nvox > kNoAllocMaxVoxels) return TRINITY_E_INVALID;  // beyond the static scratch
  if (!P || !Q || !b1 || !eps || !S_prev || !S_out || !I_out || !(tol > 0.0) || max_iters < 1)
    return TRINITY_E_INVALID;
  NoAllocScratch* sc = nullptr;
  int rc = scratch_for_current_device(&sc);
  if (rc != TRINITY_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the counters and the max cell start at zero on every call; rho is overwritten below
  if (cudaMemsetAsync(sc, 0, offsetof(NoAllocScratch, rho), st) != cudaSuccess) return TRINITY_E_CUDA;
  noalloc_prepass<<<(nvox + 255) / 256, 256, 0, st>>>(na, nvox, b1, eps, S_prev, sc);
  const int tiles = (nvox + kNaTile - 1) / kNaTile;
  const float ftol = static_cast<float>(tol);
  if (na == 12)
    noalloc_iteration<12><<<tiles, 32, 0, st>>>(nvox, P, Q, b1, eps, S_prev, S_out, I_out, ftol, max_iters, sc);
  else if (na == 48)
    noalloc_iteration<48><<<tiles, 64, 0, st>>>(nvox, P, Q, b1, eps, S_prev, S_out, I_out, ftol, max_iters, sc);
  else
    noalloc_iteration<192><<<tiles, 192, 0, st>>>(nvox, P, Q, b1, eps, S_prev, S_out, I_out, ftol, max_iters, sc);
  if (cudaGetLastError() != cudaSuccess) return TRINITY_E_CUDA;
  int counters[2] = {0, 0};
  if (cudaMemcpyAsync(counters, &sc->iters_max, sizeof(counters), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return TRINITY_E_CUDA;
  if (iters_max) *iters_max = counters[0];
  return counters[1] > 0 ? TRINITY_W_NOT_CONVERGED : TRINITY_OK;
}
