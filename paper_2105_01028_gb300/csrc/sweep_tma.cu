// The one-level ray sweep with its upwind planes staged through the Tensor Memory
// Accelerator: Eq. 10 without its S(n) term, on the slab lattice of Section 2.1, for
// boxes with a uniform refractive index (the retarded delay is then the same for every
// voxel of a direction, so each output tile needs exactly two stored levels of I and S).
//
// Q(v, d) = T (I_up) + b0 (S_up), the upwind values interpolated in time between levels
// n - m and n - m - 1 (the same arithmetic as sweep.cu's kUniN forms).  Work items are
// (direction, tile) pairs of one dominant-axis class, handed out to persistent CTAs in a
// fixed order; per item one thread issues four TMA tile loads (I and S at the two levels)
// of the upwind region into shared memory, and the CTA computes the tile's Q from there
// while the next item's loads are in flight (two stages, one mbarrier each).
//   dom z: an item is R rows along y of one z slab; the upwind rows are those of slab
//          z - sgn shifted by the slab's lattice offsets (one contiguous (x, y) box);
//   dom y: R rows along z of one y slab, likewise;
//   dom x: a 4 x 4 block of (y, z) rows over a chunk of 32 voxels along x; the upwind
//          sample of voxel x lies in slab x - sgn shifted by that slab's offsets, so the
//          box covers the block plus one row of halo (5 x 5 rows) and each voxel picks its
//          row in shared memory.  A direction's offsets along a transverse axis all have
//          the sign of its slope there (they are differences of a monotone floor), so the
//          halo lies on one side only: hsh[d] bit 0 / 1 is set when the y / z offsets are
//          positive (the upwind rows are then y - 1 .. y + 3, else y .. y + 4).  Along x
//          the box spans the chunk plus four floats on the upwind side (x0 - 4 .. x0 + 31
//          for sgn > 0, x0 .. x0 + 35 for sgn < 0: the TMA's 16-byte rule on the innermost
//          coordinate), so its size does not grow with nx.
// dom y / z boxes span the rows' nx floats from x = 0; coordinates outside a box read
// zero, which is the vacuum boundary's "nothing enters through a side face".  The source
// face's inflow is added per voxel.
// The tensor maps view a whole ring (5 levels x N_a planes) as one 4-D tensor
// (x, y, z, plane), built on the host by the driver's encoder.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "device.cuh"

namespace trinity {

namespace {

constexpr int kRows = 16;       // rows per item (dom y, z)
constexpr int kBlk = 4;         // rows per item along each transverse axis (dom x)
constexpr int kXc = 32;         // voxels per item along x (dom x)
constexpr int kXw = kXc + 4;    // box width along x (dom x): the chunk and a 4-float upwind halo
constexpr int kPad = 0;         // box rows cover x in [0, nx) exactly (no out-of-range x)
constexpr int kStages = 2;      // items in flight per CTA
constexpr long long kTmaWait = 2000000000LL;  // ~1 s bound on every mbarrier wait

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void bar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!bar_try(bar, parity))
    if (clock64() - t0 > kTmaWait) return false;
  return true;
}

__device__ __forceinline__ void tma_load4(void* dst, const CUtensorMap* map, int x, int y, int z, int p,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(p), "r"(smem_addr(bar))
      : "memory");
}

// Box shape (rows along y, rows along z) of a dominant-axis class.
template <int DOM>
struct Box {
  static constexpr int RY = DOM == 2 ? kRows : (DOM == 1 ? 1 : kBlk + 1);
  static constexpr int RZ = DOM == 2 ? 1 : (DOM == 1 ? kRows : kBlk + 1);
};

// Per-direction constants of the current step (same for all of its items).
struct DirStep {
  int d, sgn, m;
  float f, T, b0, src_amp;
  int p0, p1;       // plane coordinates of levels n - m and n - m - 1 in the ring tensor
  bool h0, h1;      // the level lies in the stored history (else it reads as zero)
};

// Per-item constants, computed once by the issuing thread and read by the CTA.
struct ItemInfo {
  DirStep s;
  int oy, oz;   // box origin (y, z)
  int ra, rb;   // dom z: (z, y0); dom y: (y, z0); dom x: (y0, z0)
  int x0, ox;   // first voxel along x of the item; box origin along x
  int kp;       // slab index of the item's voxels (dom y, z)
  int dx;       // x shift of the upwind samples (dom y, z)
};

template <int DOM, bool kUniMu>
__global__ void __launch_bounds__(256) sweep_tma_kernel(GridParams g, const DirInfo* __restrict__ dirs,
                                                        const int* __restrict__ dlist, int ndir,
                                                        const int8_t* __restrict__ offs,
                                                        const int8_t* __restrict__ hsh,
                                                        const __grid_constant__ CUtensorMap tmI,
                                                        const __grid_constant__ CUtensorMap tmS,
                                                        const float* __restrict__ mut, float* __restrict__ Q,
                                                        RunState rs, int first) {
  using B = Box<DOM>;
  const int W = DOM == 0 ? kXw : g.nx + 2 * kPad;
  // floats per box slot: a TMA tile's shared-memory destination must be 128-byte aligned,
  // so each slot is rounded up to 32 floats
  const int box = (W * B::RY * B::RZ + 31) & ~31;
  extern __shared__ __align__(128) float sm_raw[];
  // [kStages][4 boxes: I0, I1, S0, S1][box], from a 128-byte aligned base
  float* sm = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(sm_raw) + 127) & ~uintptr_t(127));
  __shared__ __align__(8) uint64_t bar[kStages];
  __shared__ ItemInfo info_s[kStages];
  __shared__ int abort_s;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int n = *rs.step;
  if (first && blockIdx.x == 0 && tid == 0) {
    rs.smax[n & 1] = 0u;     // max |S(n)|, filled by this step's source iteration
    rs.tile_ctr[n & 1] = 0;  // work counter of this step's persistent kernel
  }
  // items of one direction
  const int ipd = DOM == 2 ? g.nz * ((g.ny + kRows - 1) / kRows)
                           : (DOM == 1 ? g.ny * ((g.nz + kRows - 1) / kRows)
                                       : ((g.ny + kBlk - 1) / kBlk) * ((g.nz + kBlk - 1) / kBlk) *
                                             ((g.nx + kXc - 1) / kXc));
  const int nitems = ndir * ipd;
  if (tid == 0) {
    for (int k = 0; k < kStages; ++k) bar_init(&bar[k]);
    abort_s = 0;
  }
  __syncthreads();

  // thread 0: the item's constants into info_s[stage], then its four TMA loads
  const auto issue = [&](int item, int stage) {
    ItemInfo it;
    DirStep& s = it.s;
    s.d = dlist[item / ipd];
    const DirInfo di = dirs[s.d];
    s.sgn = di.sgn;
    int m;
    float f;
    retarded_delay(di.dcoef, di.dcoef_lo, g.n_u, m, f);
    s.m = m < 1 ? 1 : (m > 3 ? 3 : m);
    s.f = f;
    s.src_amp = di.src_amp;
    if (kUniMu) {
      const float xo = g.mut_u * di.ds;
      s.T = expf(-xo);
      s.b0 = ray_b0(xo, s.T);
    } else {
      s.T = 0.0f;
      s.b0 = di.ds;  // the spacing, for the per-voxel weights
    }
    const int L0 = n - s.m, L1 = n - s.m - 1;
    s.h0 = L0 >= g.hist_from;
    s.h1 = L1 >= g.hist_from;
    s.p0 = ring_slot(L0) * g.na + s.d;
    s.p1 = ring_slot(L1) * g.na + s.d;
    const int t = item % ipd;
    const int8_t* off0 = offs + (static_cast<size_t>(s.d) * 2 + 0) * g.nmax;
    const int8_t* off1 = offs + (static_cast<size_t>(s.d) * 2 + 1) * g.nmax;
    if (DOM == 2) {
      const int nyb = (g.ny + kRows - 1) / kRows;
      const int z = t / nyb, y0 = (t % nyb) * kRows;
      it.kp = s.sgn > 0 ? z : g.nz - 1 - z;
      it.ra = z;
      it.rb = y0;
      it.oy = y0 - (it.kp > 0 ? off1[it.kp] : 0);
      it.oz = z - s.sgn;
      it.dx = it.kp > 0 ? off0[it.kp] : 0;
      it.x0 = 0;
      it.ox = -kPad;
    } else if (DOM == 1) {
      const int nzb = (g.nz + kRows - 1) / kRows;
      const int y = t / nzb, z0 = (t % nzb) * kRows;
      it.kp = s.sgn > 0 ? y : g.ny - 1 - y;
      it.ra = y;
      it.rb = z0;
      it.oy = y - s.sgn;
      it.oz = z0 - (it.kp > 0 ? off1[it.kp] : 0);
      it.dx = it.kp > 0 ? off0[it.kp] : 0;
      it.x0 = 0;
      it.ox = -kPad;
    } else {
      const int nyb = (g.ny + kBlk - 1) / kBlk, nxc = (g.nx + kXc - 1) / kXc;
      const int xc = t % nxc, t2 = t / nxc;
      const int zb = t2 / nyb, yb = t2 % nyb;
      it.x0 = xc * kXc;
      it.ox = s.sgn > 0 ? it.x0 - 4 : it.x0;
      it.ra = yb * kBlk;
      it.rb = zb * kBlk;
      const int h = hsh[s.d];
      it.oy = it.ra - (h & 1);
      it.oz = it.rb - ((h >> 1) & 1);
      it.kp = 0;
      it.dx = 0;
    }
    info_s[stage] = it;
    float* base = sm + static_cast<size_t>(stage) * 4 * box;
    if (smem_addr(base) & 127u) {  // never expected: the slots are 128-byte multiples
      atomicExch(rs.error, 4);
      bar_expect(&bar[stage], 0u);
      return;
    }
    const uint32_t bytes = static_cast<uint32_t>(W * B::RY * B::RZ) * 4u * ((s.h0 ? 2u : 0u) + (s.h1 ? 2u : 0u));
    bar_expect(&bar[stage], bytes);
    if (s.h0) {
      tma_load4(base + 0 * box, &tmI, it.ox, it.oy, it.oz, s.p0, &bar[stage]);
      tma_load4(base + 2 * box, &tmS, it.ox, it.oy, it.oz, s.p0, &bar[stage]);
    }
    if (s.h1) {
      tma_load4(base + 1 * box, &tmI, it.ox, it.oy, it.oz, s.p1, &bar[stage]);
      tma_load4(base + 3 * box, &tmS, it.ox, it.oy, it.oz, s.p1, &bar[stage]);
    }
  };

  const int i0 = blockIdx.x;
  if (tid == 0) {
    for (int k = 0; k < kStages; ++k)
      if (i0 + k * static_cast<int>(gridDim.x) < nitems) issue(i0 + k * gridDim.x, k);
  }
  uint32_t phase[kStages] = {};
  const size_t plane = static_cast<size_t>(g.nv);
  int it_no = 0;
  for (int item = i0; item < nitems; item += gridDim.x, ++it_no) {
    const int st = it_no % kStages;
    const bool ok = bar_wait(&bar[st], phase[st]);
    phase[st] ^= 1u;
    if (!ok) abort_s = 1;
    if (__syncthreads_or(!ok)) break;
    const ItemInfo it = info_s[st];
    const DirStep& s = it.s;
    const float* bI0 = sm + static_cast<size_t>(st) * 4 * box;
    const float* bI1 = bI0 + box;
    const float* bS0 = bI0 + 2 * box;
    const float* bS1 = bI0 + 3 * box;
    float* Qd = Q + static_cast<size_t>(s.d) * plane;
    const float w0 = 1.0f - s.f, w1 = s.f;
    const int L0 = n - s.m, L1 = n - s.m - 1;
    const float on0 = (L0 >= 0 && L0 < g.pulse_steps) ? 1.0f : 0.0f;
    const float on1 = (L1 >= 0 && L1 < g.pulse_steps) ? 1.0f : 0.0f;
    // Q of voxel v from shared-memory slot si (xs: the upwind sample's x, checked for a
    // side-face entry; ghost: the ray enters through the face normal to dom)
    const auto emit = [&](int v, int si, int xs, bool ghost) {
      float Iup, Sup;
      if (ghost) {
        Iup = (v == g.src_voxel && s.src_amp != 0.0f) ? s.src_amp * fmaf(w1, on1, w0 * on0) : 0.0f;
        Sup = 0.0f;
      } else if (xs < 0 || xs >= g.nx) {  // the ray entered through a side face: nothing enters
        Iup = 0.0f;
        Sup = 0.0f;
      } else {
        // a level before the stored history was not loaded (its buffer holds stale data)
        const float i0 = s.h0 ? bI0[si] : 0.0f, i1 = s.h1 ? bI1[si] : 0.0f;
        const float s0v = s.h0 ? bS0[si] : 0.0f, s1v = s.h1 ? bS1[si] : 0.0f;
        Iup = fmaf(w1, i1, w0 * i0);
        Sup = fmaf(w1, s1v, w0 * s0v);
      }
      float T, b0;
      if (kUniMu) {
        T = s.T;
        b0 = s.b0;
      } else {
        const float xo = __ldg(mut + v) * s.b0;
        T = expf(-xo);
        b0 = ray_b0(xo, T);
      }
      Qd[v] = fmaf(Sup, b0, Iup * T);
    };
    if (DOM == 2 || DOM == 1) {
      // warps over the item's rows, lanes along x
      const bool ghost = it.kp == 0;
      for (int r = warp; r < kRows; r += 8) {
        const int y = DOM == 2 ? it.rb + r : it.ra;
        const int z = DOM == 2 ? it.ra : it.rb + r;
        if (y >= g.ny || z >= g.nz) break;
        const int vrow = (z * g.ny + y) * g.nx;
        for (int x = lane; x < g.nx; x += 32) {
          const int xs = x - it.dx;
          emit(vrow + x, r * W + xs, xs, ghost);
        }
      }
    } else {
      // warps over the block's 16 rows, lanes along the item's voxels in x; each x has its
      // own slab offsets
      const int8_t* off0 = offs + (static_cast<size_t>(s.d) * 2 + 0) * g.nmax;
      const int8_t* off1 = offs + (static_cast<size_t>(s.d) * 2 + 1) * g.nmax;
#pragma unroll
      for (int xl = lane; xl < kXc; xl += 32) {
        const int x = it.x0 + xl;
        if (x >= g.nx) break;
        const int kp = s.sgn > 0 ? x : g.nx - 1 - x;
        const int dy = kp > 0 ? off0[kp] : 0, dz = kp > 0 ? off1[kp] : 0;
        const int xs = x - s.sgn;
        for (int r = warp; r < kBlk * kBlk; r += 8) {
          const int y = it.ra + (r % kBlk), z = it.rb + (r / kBlk);
          if (y >= g.ny || z >= g.nz) continue;
          emit((z * g.ny + y) * g.nx + x, ((z - it.oz - dz) * B::RY + (y - it.oy - dy)) * W + (xs - it.ox), xs,
               kp == 0);
        }
      }
    }
    __syncthreads();  // the stage's buffers and constants are free again
    if (tid == 0 && item + kStages * static_cast<int>(gridDim.x) < nitems) issue(item + kStages * gridDim.x, st);
  }
  if (abort_s) {
    // a wait ran out: record it, and let the copies still in flight land (bounded)
    if (tid == 0) {
      atomicExch(rs.error, 3);
      for (int k = 0; k < kStages; ++k) bar_wait(&bar[k], phase[k]);
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

}  // namespace

bool sweep_tma_supported(const GridParams& g) {
  if (g.periodic || g.mirror || g.nx % 4 != 0 || g.nx + 2 * kPad > 256) return false;
  // the largest item (dom y / z: 16 whole rows) must fit the shared memory of a CTA
  const size_t slot = (static_cast<size_t>(g.nx + 2 * kPad) * kRows + 31) & ~static_cast<size_t>(31);
  return kStages * 4 * slot * sizeof(float) + 128 <= 232448;
}

cudaError_t make_sweep_maps(const GridParams& g, float* Iring, float* Sring, SweepMaps* out) {
  if (!sweep_tma_supported(g)) return cudaErrorNotSupported;
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[4] = {static_cast<cuuint64_t>(g.nx), static_cast<cuuint64_t>(g.ny),
                              static_cast<cuuint64_t>(g.nz), static_cast<cuuint64_t>(5) * g.na};
  const cuuint64_t strides[3] = {static_cast<cuuint64_t>(g.nx) * 4, static_cast<cuuint64_t>(g.nx) * g.ny * 4,
                                 static_cast<cuuint64_t>(g.nv) * 4};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const cuuint32_t W = static_cast<cuuint32_t>(g.nx + 2 * kPad);
  const cuuint32_t boxes[3][4] = {{kXw, kBlk + 1, kBlk + 1, 1}, {W, 1, kRows, 1}, {W, kRows, 1, 1}};
  for (int c = 0; c < 3; ++c)
    for (int f = 0; f < 2; ++f) {
      CUtensorMap* m = reinterpret_cast<CUtensorMap*>(f == 0 ? out->I[c] : out->S[c]);
      const CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, f == 0 ? Iring : Sring, dims, strides,
                                  boxes[c], estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
  return cudaSuccess;
}

namespace {

template <int DOM>
cudaError_t launch_class(const GridParams& g, const DirInfo* dirs, const int* dlist, int ndir, const int8_t* offs,
                         const int8_t* hsh, const SweepMaps& maps, const float* mut, float* Q, RunState rs,
                         int first, int nsm, cudaStream_t st) {
  if (ndir == 0) return cudaSuccess;
  using Bx = Box<DOM>;
  const size_t w = DOM == 0 ? kXw : g.nx + 2 * kPad;
  const size_t slot = (w * Bx::RY * Bx::RZ + 31) & ~static_cast<size_t>(31);
  const size_t smem = kStages * 4 * slot * sizeof(float) + 128;  // + alignment slack
  CUtensorMap mI, mS;
  std::memcpy(&mI, maps.I[DOM], sizeof(CUtensorMap));
  std::memcpy(&mS, maps.S[DOM], sizeof(CUtensorMap));
  const bool um = g.mut_u >= 0.0f;
  auto kern = um ? sweep_tma_kernel<DOM, true> : sweep_tma_kernel<DOM, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  kern<<<nsm * per_sm, 256, smem, st>>>(g, dirs, dlist, ndir, offs, hsh, mI, mS, mut, Q, rs, first);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep_tma(const GridParams& g, const DirInfo* dirs, const int* const dlist[3],
                             const int ndir[3], const int8_t* offs, const int8_t* hsh, const SweepMaps& maps,
                             const float* mut, float* Q, RunState rs, const cudaStream_t st[3]) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cudaErrorUnknown;
  }
  // the first class launched (with directions) also clears this step's max |S| and work counter
  const int f2 = ndir[2] > 0, f1 = !f2 && ndir[1] > 0, f0 = !f2 && !f1;
  // the classes write disjoint planes of Q and only read the rings: st[k] may run them
  // concurrently (the caller joins the streams before the next kernel)
  cudaError_t e = launch_class<2>(g, dirs, dlist[2], ndir[2], offs, hsh, maps, mut, Q, rs, f2, nsm, st[0]);
  if (e == cudaSuccess) e = launch_class<1>(g, dirs, dlist[1], ndir[1], offs, hsh, maps, mut, Q, rs, f1, nsm, st[1]);
  if (e == cudaSuccess) e = launch_class<0>(g, dirs, dlist[0], ndir[0], offs, hsh, maps, mut, Q, rs, f0, nsm, st[2]);
  return e;
}

}  // namespace trinity
