// Exact per-voxel source function on the 5th-generation tensor cores (tcgen05), 192
// directions.  The source iteration of Eq. 12 (Section 2.4 steps 5-6) converges to the
// fixed point of S = a P (Q + b1 S); voxels of one optics class share the operator
// M = (I - a P B1)^-1 a P, so S = M Q is one (voxels x 192) x (192 x 192) product per step.
//
// Precision: three TF32 products with FP32 accumulation in tensor memory,
//   D = Q_hi M_hi^T + Q_lo M_hi^T + Q_hi M_lo^T,
// where x_hi = tf32(x) and x_lo = tf32(x - x_hi) (both rounded to nearest even), so every
// operand carries ~22 significant bits; the dropped Q_lo M_lo^T term is 2^-22 of the
// product.  Q and M are non-negative (M is a Neumann series of non-negative matrices), so
// no cancellation amplifies these relative errors.
//
// Work: a pass is one 128-voxel tile (consecutive flat voxel indices) against one optics
// class present in it (a tile that mixes classes is computed once per class and each
// voxel keeps the result of its own).  Persistent CTAs, one per SM, take tiles in a fixed
// stride.  K (the 192 source directions) is streamed in chunks of 32 through shared memory:
//   * warp 12 issues TMA loads of the tile's Q chunk ([32 directions] x [128 voxels] FP32,
//     voxel-contiguous as Q is stored) into a 3-deep raw ring;
//   * warps 0-3 (one voxel row per thread) read their row of the raw chunk, split it into
//     TF32 hi / lo and store both as K-major 128-byte-swizzled A operands (2 stages);
//   * warp 13 copies the class's pre-swizzled M_hi / M_lo chunk (built on the host) with
//     one bulk copy per stage;
//   * warp 14 issues the 12 MMAs of a chunk (M = 128, N = 192, K = 8 each) into one of two
//     TMEM accumulators (columns 0 and 256) and commits them to the stage's "empty" barrier,
//     and after a pass's last chunk to the accumulator's "full" barrier;
//   * warps 4-11 drain the other accumulator: warp w reads TMEM lanes 32 (w % 4) .. + 31
//     (one voxel per thread) and 96 of the 192 columns, forms I = Q + b1 S (Q read again,
//     from L2), writes I and S (coalesced along voxels) and the tallies.
// Every mbarrier wait is bounded (~1 s); a wait that runs out records error 5, the roles
// leave their loops, the copies and MMAs in flight are waited for (bounded) and TMEM is
// freed before the kernel returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "device.cuh"

namespace trinity {

namespace {

constexpr int kNa = 192;            // directions (N of the MMA and K of the product)
constexpr int kM = 128;             // voxels per tile (M of the MMA)
constexpr int kKc = 32;             // K per chunk: one 128-byte swizzle atom of FP32
constexpr int kNk = kNa / kKc;      // chunks per pass
constexpr int kRaw = 3;             // raw Q chunks in flight
constexpr int kOps = 2;             // operand stages
constexpr int kEpiWarps = 8;        // epilogue warps
constexpr int kThreads = (4 + kEpiWarps + 3) * 32;
constexpr int kWarpQ = 4 + kEpiWarps;   // TMA loader of Q
constexpr int kWarpB = kWarpQ + 1;      // bulk loader of M
constexpr int kWarpMma = kWarpQ + 2;    // MMA issuer, TMEM owner
constexpr int kEpiCols = kNa / (kEpiWarps / 4);  // columns per epilogue thread
constexpr int kEpiCh = 16;                       // TMEM load width
constexpr long long kWait = 2000000000LL;        // ~1 s bound on every mbarrier wait

constexpr int kABytes = kM * 128;                // one A term of a chunk
constexpr int kBBytes = kNa * 128;               // one B term of a chunk
constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;
constexpr int kRawBytes = kKc * kM * 4;
constexpr int kOffRaw = kOps * kStageBytes;
constexpr int kOffB1 = kOffRaw + kRaw * kRawBytes;          // [classes][192] b1
constexpr int kMaxCls = 8;
constexpr int kSmem = kOffB1 + kMaxCls * kNa * 4 + 1024;    // + alignment slack
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(kNa >> 3) << 17) |
                            (static_cast<uint32_t>(kM >> 4) << 24);  // F32 accumulate, TF32 A and B, K-major

__device__ __forceinline__ uint32_t sa(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(sa(b)), "r"(parity)
      : "memory");
  return ok != 0u;
}

// Bounded wait for the completion of the phase with the given parity; false if it ran out
// or another role has given up.
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  const long long t0 = clock64();
  while (!bar_try(b, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWait) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load2(void* dst, const CUtensorMap* map, int x, int y, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(sa(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(sa(b))
      : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   sa(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(sa(b))
               : "memory");
}

// 128-byte-swizzled K-major operand descriptor (8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(1) << 16) |
         (static_cast<uint64_t>(1024 >> 4) << 32) | (static_cast<uint64_t>(1) << 46) |
         (static_cast<uint64_t>(2) << 61);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(b))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Round an FP32 value to TF32 (10 stored mantissa bits), nearest even; finite inputs.
__device__ __forceinline__ float tf32_rne(float x) {
  uint32_t u = __float_as_uint(x);
  u += 0xFFFu + ((u >> 13) & 1u);
  return __uint_as_float(u & 0xFFFFE000u);
}

// Pass enumeration shared by every role: tiles blockIdx.x, + gridDim.x, ...; per tile the
// classes present in it, lowest first.
struct PassIter {
  int tile;
  unsigned rest;
  int cls;
  __device__ bool first(const uint8_t* tmask, int ntiles) {
    tile = static_cast<int>(blockIdx.x) - static_cast<int>(gridDim.x);
    rest = 0u;
    return next(tmask, ntiles);
  }
  __device__ bool next(const uint8_t* tmask, int ntiles) {
    while (rest == 0u) {
      tile += gridDim.x;
      if (tile >= ntiles) return false;
      rest = tmask[tile];
    }
    cls = __ffs(rest) - 1;
    rest &= rest - 1u;
    return true;
  }
};

__global__ void __launch_bounds__(kThreads, 1)
    exact_tc_kernel(GridParams g, const __grid_constant__ CUtensorMap qmap, const float* __restrict__ Mimg,
                    const uint8_t* __restrict__ tmask, int ntiles, const float* __restrict__ b1tab, int ncls,
                    const uint8_t* __restrict__ cls, const float* __restrict__ mua_cls, const float* __restrict__ Q,
                    const float* __restrict__ nidx, float* __restrict__ Iring, float* __restrict__ Sring,
                    RunState rs) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* b1s = reinterpret_cast<float*>(smem + kOffB1);

  __shared__ uint64_t raw_full[kRaw], raw_empty[kRaw];
  __shared__ uint64_t a_full[kOps], b_full[kOps], op_empty[kOps];
  __shared__ uint64_t d_full[2], d_empty[2];
  __shared__ uint32_t tmem_s;
  __shared__ int abort_s;
  __shared__ double esum_s[kEpiWarps], asum_s[kEpiWarps];
  __shared__ float smax_s[kEpiWarps];
  __shared__ unsigned cnt_s[kEpiWarps];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int* abort_v = &abort_s;
  const int n = *rs.step;

  if (tid == 0) {
    abort_s = 0;
    for (int i = 0; i < kRaw; ++i) {
      bar_init(&raw_full[i], 1);
      bar_init(&raw_empty[i], 128);
    }
    for (int i = 0; i < kOps; ++i) {
      bar_init(&a_full[i], 128);
      bar_init(&b_full[i], 1);
      bar_init(&op_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      bar_init(&d_full[i], 1);
      bar_init(&d_empty[i], kEpiWarps * 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // every operand and TMA destination must sit on its alignment (1024 B / 128 B)
    if ((sa(smem) & 1023u) != 0u || (sa(smem + kOffRaw) & 127u) != 0u) abort_s = 6;
  }
  for (int i = tid; i < ncls * kNa; i += blockDim.x) b1s[i] = b1tab[i];
  if (warp == kWarpMma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&tmem_s)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_s;
  const bool misaligned = abort_s == 6;
  if (misaligned && tid == 0) atomicExch(rs.error, 6);

  PassIter it;
  if (misaligned) {
    // nothing issued
  } else if (warp == kWarpQ) {
    // ---- Q chunks: TMA tile loads into the raw ring
    uint32_t ru = 0;
    if (lane == 0) {
      for (bool ok = it.first(tmask, ntiles); ok && !*abort_v; ok = it.next(tmask, ntiles)) {
        for (int k = 0; k < kNk; ++k, ++ru) {
          const int s = ru % kRaw;
          if (!bar_wait(&raw_empty[s], ((ru / kRaw) & 1u) ^ 1u, abort_v)) {
            atomicExch(const_cast<int*>(abort_v), 1);
            break;
          }
          bar_expect(&raw_full[s], kRawBytes);
          tma_load2(smem + kOffRaw + s * kRawBytes, &qmap, it.tile * kM, k * kKc, &raw_full[s]);
        }
      }
      // wait for the loads still in flight (after an abort)
      for (uint32_t u = ru > kRaw ? ru - kRaw : 0u; u < ru; ++u) {
        const long long t0 = clock64();
        while (!bar_try(&raw_full[u % kRaw], (u / kRaw) & 1u) && clock64() - t0 < kWait) {
        }
      }
    }
    __syncwarp();
  } else if (warp == kWarpB) {
    // ---- M chunks of the pass's class: one bulk copy of M_hi and M_lo per stage
    uint32_t bu = 0;
    if (lane == 0) {
      for (bool ok = it.first(tmask, ntiles); ok && !*abort_v; ok = it.next(tmask, ntiles)) {
        for (int k = 0; k < kNk; ++k, ++bu) {
          const int s = bu % kOps;
          if (!bar_wait(&op_empty[s], ((bu / kOps) & 1u) ^ 1u, abort_v)) {
            atomicExch(const_cast<int*>(abort_v), 1);
            break;
          }
          bar_expect(&b_full[s], 2 * kBBytes);
          bulk_load(smem + s * kStageBytes + 2 * kABytes,
                    Mimg + (static_cast<size_t>(it.cls) * kNk + k) * (2 * kBBytes / 4), 2 * kBBytes, &b_full[s]);
        }
      }
      for (uint32_t u = bu > kOps ? bu - kOps : 0u; u < bu; ++u) {
        const long long t0 = clock64();
        while (!bar_try(&b_full[u % kOps], (u / kOps) & 1u) && clock64() - t0 < kWait) {
        }
      }
    }
    __syncwarp();
  } else if (warp == kWarpMma) {
    // ---- MMA issue
    uint32_t au = 0, p = 0;
    bool issued = false;
    if (lane == 0) {
      for (bool ok = it.first(tmask, ntiles); ok && !*abort_v; ok = it.next(tmask, ntiles), ++p) {
        const uint32_t buf = p & 1u;
        if (!bar_wait(&d_empty[buf], ((p >> 1) & 1u) ^ 1u, abort_v)) {
          atomicExch(const_cast<int*>(abort_v), 1);
          break;
        }
        fence_after();
        const uint32_t d = tmem + buf * 256u;
        bool fail = false;
        for (int k = 0; k < kNk; ++k, ++au) {
          const int s = au % kOps;
          const uint32_t ph = (au / kOps) & 1u;
          if (!bar_wait(&a_full[s], ph, abort_v) || !bar_wait(&b_full[s], ph, abort_v)) {
            fail = true;
            break;
          }
          fence_after();
          const uint32_t aHi = sa(smem + s * kStageBytes), aLo = aHi + kABytes;
          const uint32_t bHi = aHi + 2 * kABytes, bLo = bHi + kBBytes;
#pragma unroll
          for (int kk = 0; kk < kKc / 8; ++kk) {
            const uint32_t ko = static_cast<uint32_t>(kk * 32);
            mma_tf32(d, desc_sw128(aLo + ko), desc_sw128(bHi + ko), (k | kk) != 0 ? 1u : 0u);
            mma_tf32(d, desc_sw128(aHi + ko), desc_sw128(bLo + ko), 1u);
            mma_tf32(d, desc_sw128(aHi + ko), desc_sw128(bHi + ko), 1u);
          }
          mma_commit(&op_empty[s]);
          issued = true;
        }
        if (fail) {
          atomicExch(const_cast<int*>(abort_v), 1);
          break;
        }
        mma_commit(&d_full[buf]);
      }
      // the MMAs in flight complete before TMEM is freed
      if (issued) {
        const uint32_t u = au - 1u;
        const long long t0 = clock64();
        while (!bar_try(&op_empty[u % kOps], (u / kOps) & 1u) && clock64() - t0 < kWait) {
        }
      }
    }
    __syncwarp();
  } else if (warp < 4) {
    // ---- converters: raw Q chunk -> TF32 hi / lo A operands, one voxel row per thread
    const int r = tid;
    uint32_t ru = 0, au = 0;
    bool stop = false;
    for (bool ok = it.first(tmask, ntiles); ok && !stop && !*abort_v; ok = it.next(tmask, ntiles)) {
      for (int k = 0; k < kNk; ++k, ++ru, ++au) {
        const int s = ru % kRaw;
        if (!bar_wait(&raw_full[s], (ru / kRaw) & 1u, abort_v)) {
          stop = true;
          break;
        }
        const float* raw = reinterpret_cast<const float*>(smem + kOffRaw + s * kRawBytes);
        float hi[kKc], lo[kKc];
#pragma unroll
        for (int j = 0; j < kKc; ++j) {
          const float q = raw[j * kM + r];
          hi[j] = tf32_rne(q);
          lo[j] = tf32_rne(q - hi[j]);
        }
        bar_arrive(&raw_empty[s]);
        const int so = au % kOps;
        if (!bar_wait(&op_empty[so], ((au / kOps) & 1u) ^ 1u, abort_v)) {
          stop = true;
          break;
        }
        uint8_t* aHi = smem + so * kStageBytes;
        uint8_t* aLo = aHi + kABytes;
#pragma unroll
        for (int c = 0; c < kKc / 4; ++c) {
          const uint32_t off = static_cast<uint32_t>(r * 128 + ((c ^ (r & 7)) << 4));
          *reinterpret_cast<float4*>(aHi + off) = make_float4(hi[4 * c], hi[4 * c + 1], hi[4 * c + 2], hi[4 * c + 3]);
          *reinterpret_cast<float4*>(aLo + off) = make_float4(lo[4 * c], lo[4 * c + 1], lo[4 * c + 2], lo[4 * c + 3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bar_arrive(&a_full[so]);
      }
    }
    if (stop) atomicExch(const_cast<int*>(abort_v), 1);
  } else {
    // ---- epilogue: S from TMEM, I = Q + b1 S, stores and tallies
    const int q4 = warp & 3, grp = (warp - 4) >> 2;
    const int row = q4 * 32 + lane;
    const int c0 = grp * kEpiCols;
    const size_t plane = static_cast<size_t>(g.nv);
    const size_t cur = static_cast<size_t>(ring_slot(n)) * kNa * plane;
    double esum = 0.0, asum = 0.0;
    float smax = 0.0f;
    unsigned cnt = 0u;
    uint32_t p = 0;
    for (bool ok = it.first(tmask, ntiles); ok && !*abort_v; ok = it.next(tmask, ntiles), ++p) {
      const uint32_t buf = p & 1u;
      if (!bar_wait(&d_full[buf], (p >> 1) & 1u, abort_v)) {
        atomicExch(const_cast<int*>(abort_v), 1);
        break;
      }
      fence_after();
      const int v = it.tile * kM + row;
      const bool mine = v < g.nv && static_cast<int>(cls[v]) == it.cls;
      const uint32_t t = tmem + (static_cast<uint32_t>(q4 * 32) << 16) + buf * 256u + static_cast<uint32_t>(c0);
      const float* b1c = b1s + it.cls * kNa + c0;
      float erow = 0.0f;
      // two 16-column chunks at a time: their 32 Q loads are issued before the TMEM loads
      static_assert((kEpiCols / kEpiCh) % 2 == 0, "chunks go in pairs");
#pragma unroll 1
      for (int ch = 0; ch < kEpiCols / kEpiCh; ch += 2) {
        float qv[2][kEpiCh];
        if (mine) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const float* qp = Q + static_cast<size_t>(c0 + (ch + u) * kEpiCh) * plane + v;
#pragma unroll
            for (int j = 0; j < kEpiCh; ++j) qv[u][j] = __ldcs(qp + static_cast<size_t>(j) * plane);
          }
        }
        float sv[2][kEpiCh];
        tmem_ld16(t + ch * kEpiCh, sv[0]);
        tmem_ld16(t + (ch + 1) * kEpiCh, sv[1]);
        if (mine) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int cc = (ch + u) * kEpiCh;
            float* ip = Iring + cur + static_cast<size_t>(c0 + cc) * plane + v;
            float* sp = Sring + cur + static_cast<size_t>(c0 + cc) * plane + v;
#pragma unroll
            for (int j = 0; j < kEpiCh; ++j) {
              const float Iv = fmaf(b1c[cc + j], sv[u][j], qv[u][j]);
              __stcs(ip + static_cast<size_t>(j) * plane, Iv);
              __stcs(sp + static_cast<size_t>(j) * plane, sv[u][j]);
              erow += Iv;
              smax = fmaxf(smax, fabsf(sv[u][j]));
            }
          }
        }
      }
      fence_before();
      bar_arrive(&d_empty[buf]);
      if (mine) {
        esum += static_cast<double>(erow) * static_cast<double>(nidx[v]);
        asum += static_cast<double>(erow) * static_cast<double>(mua_cls[it.cls]);
        cnt += grp == 0 ? 1u : 0u;
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      esum += __shfl_xor_sync(0xffffffffu, esum, o);
      asum += __shfl_xor_sync(0xffffffffu, asum, o);
      smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
      esum_s[warp - 4] = esum;
      asum_s[warp - 4] = asum;
      smax_s[warp - 4] = smax;
      cnt_s[warp - 4] = cnt;
    }
  }

  fence_before();
  __syncthreads();
  if (tid == 0) {
    if (abort_s == 1) atomicExch(rs.error, 5);
    if (!misaligned) {
      double e = 0.0, ab = 0.0;
      float sm = 0.0f;
      unsigned long long c = 0;
      for (int w = 0; w < kEpiWarps; ++w) {
        e += esum_s[w];
        ab += asum_s[w];
        sm = fmaxf(sm, smax_s[w]);
        c += cnt_s[w];
      }
      atomicAdd(rs.energy + n, e * static_cast<double>(g.e_scale));
      atomicAdd(rs.absorbed + n, ab * g.a_scale);
      atomicMax(rs.smax + (n & 1), __float_as_uint(sm));
      atomicMax(rs.iters_max + n, 1);
      atomicAdd(rs.iters_sum + n, c);
    }
  }
  if (warp == kWarpMma) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode_q = nullptr;

uint32_t f2u(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

float u2f(uint32_t u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

float host_tf32(float x) {
  uint32_t u = f2u(x);
  u += 0xFFFu + ((u >> 13) & 1u);
  return u2f(u & 0xFFFFE000u);
}

}  // namespace

bool exact_tc_supported(const GridParams& g, int ncls) {
  return g.na == kNa && g.nv % 4 == 0 && ncls >= 1 && ncls <= kMaxCls;
}

int exact_tc_tiles(int nv) { return (nv + kM - 1) / kM; }

// Host images of the operators, already in the kernel's shared-memory layout: for class c
// and chunk k, M_hi then M_lo, each 192 rows (output direction i) x 128 bytes (source
// directions 32 k .. 32 k + 31), the 16-byte group of directions 4 q .. 4 q + 3 stored at
// group position q ^ (i & 7).  M[i][j] = Mt[c][j][i]; hi = tf32(M), lo = tf32(M - hi).
void exact_tc_images(const double* M, int ncls, std::vector<float>* img) {
  img->assign(static_cast<size_t>(ncls) * kNk * 2 * kNa * kKc, 0.0f);
  for (int c = 0; c < ncls; ++c)
    for (int k = 0; k < kNk; ++k)
      for (int i = 0; i < kNa; ++i)
        for (int jj = 0; jj < kKc; ++jj) {
          const int j = k * kKc + jj;
          const double m = M[(static_cast<size_t>(c) * kNa + i) * kNa + j];
          const float hi = host_tf32(static_cast<float>(m));
          const float lo = host_tf32(static_cast<float>(m - static_cast<double>(hi)));
          const size_t base = (static_cast<size_t>(c) * kNk + k) * 2 * kNa * kKc;
          const size_t pos = static_cast<size_t>(i) * kKc + (((jj >> 2) ^ (i & 7)) << 2) + (jj & 3);
          (*img)[base + pos] = hi;
          (*img)[base + static_cast<size_t>(kNa) * kKc + pos] = lo;
        }
}

void exact_tc_tile_masks(const uint8_t* cls, int nv, std::vector<uint8_t>* mask) {
  mask->assign(exact_tc_tiles(nv), 0);
  for (int v = 0; v < nv; ++v) (*mask)[v / kM] |= static_cast<uint8_t>(1u << cls[v]);
}

cudaError_t make_exact_qmap(const GridParams& g, const float* Q, void* out) {
  if (!g_encode_q) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode_q = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  if ((reinterpret_cast<uintptr_t>(Q) & 15u) != 0u || g.nv % 4 != 0) return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(g.nv), static_cast<cuuint64_t>(kNa)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(g.nv) * 4};
  const cuuint32_t box[2] = {kM, kKc};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode_q(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                                const_cast<float*>(Q), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_exact_tc(const GridParams& g, const void* qmap, const float* Mimg, const uint8_t* tmask,
                            const float* b1tab, int ncls, const uint8_t* cls, const float* mua_cls, const float* Q,
                            const float* nidx, float* Iring, float* Sring, RunState rs, cudaStream_t st) {
  static int nsm = 0;
  static cudaError_t attr = cudaErrorUnknown;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cudaErrorUnknown;
    attr = cudaFuncSetAttribute(exact_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  }
  if (attr != cudaSuccess) return attr;
  if (!exact_tc_supported(g, ncls)) return cudaErrorInvalidValue;
  const int ntiles = exact_tc_tiles(g.nv);
  const int grid = ntiles < nsm ? ntiles : nsm;
  CUtensorMap m;
  std::memcpy(&m, qmap, sizeof(CUtensorMap));
  exact_tc_kernel<<<grid, kThreads, kSmem, st>>>(g, m, Mimg, tmask, ntiles, b1tab, ncls, cls, mua_cls, Q, nidx,
                                                 Iring, Sring, rs);
  return cudaGetLastError();
}

}  // namespace trinity
