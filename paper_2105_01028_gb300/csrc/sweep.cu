// The one-level ray sweep: Eq. 10 without its S(n) term, on the slab lattice of
// Section 2.1.
#include <cstdint>

#include "device.cuh"

namespace trinity {

namespace {

__device__ __forceinline__ int pick(int axis, int x, int y, int z) {
  return axis == 0 ? x : (axis == 1 ? y : z);
}

// Mirror faces: coordinate q of a ghost upwind sample on an axis of n voxels, brought back
// inside (the sample lies at most one voxel out, so its image across the face is the
// nearest voxel inside); ``mask`` collects the axes it lay beyond.
__device__ __forceinline__ int image_axis(int q, int n, unsigned bit, unsigned& mask) {
  if (q < 0) {
    mask |= bit;
    return 0;
  }
  if (q >= n) {
    mask |= bit;
    return n - 1;
  }
  return q;
}

// ----------------------------------------------------------------------------------------
// Q(v, d) = I_up exp(-x) + S_up b0(x), the known part of Eq. 10 at time level n.
// The upwind sample of v is the previous point of its long ray (slab lattice, Section
// 2.1): one slab back along dom(d), shifted by the per-slab offsets.  Its I and S are
// taken at the retarded time n - delta, delta = ds n(v) / (c0 dt), linearly
// interpolated between the stored levels n - m and n - m - 1 (m = floor(delta)).
//
// Mapping: blockIdx.y = direction; a block covers whole x-rows (threadIdx.x along x,
// threadIdx.y one row each) and strides over kRowSweeps groups of rows, so a warp reads
// contiguous, at most one-voxel-shifted runs of the upwind plane and the block's set-up
// is shared by several groups.  The direction's constants are staged in shared memory
// once per block, and the block resolves, once, where the five stored levels n - m
// (m = 0..4) of this direction's plane live, so a voxel indexes them by its delay's whole
// part m.
// kUniN / kUniMu: the refractive index / mu_t is the same in every voxel, so the delay's
// split (m, f) / exp(-x) and b0(x) are taken once per block, by the same FP32 operations
// on the same values as the per-voxel form, and the voxel loop reads neither map.
// Mirror faces (a test boundary: specular reflection by the method of images): a ghost
// upwind sample reads I and S of its image voxel in the direction reflected in the faces
// it lay beyond (refl[d][mask], mask bit a = axis a), at the voxel's own retarded levels.
// ----------------------------------------------------------------------------------------
constexpr int kRowSweeps = 8;  // row groups per block

template <bool kUniN, bool kUniMu>
__global__ void __launch_bounds__(256) sweep_kernel(GridParams g, const DirInfo* __restrict__ dirs,
                                                    const int8_t* __restrict__ offs,
                                                    const float* __restrict__ Iring,
                                                    const float* __restrict__ Sring,
                                                    const float* __restrict__ mut,
                                                    const float* __restrict__ nidx,
                                                    const int* __restrict__ refl,
                                                    float* __restrict__ Q, RunState rs) {
  __shared__ DirInfo di_s;
  __shared__ int n_s, m_s;
  __shared__ float f_s, T_s, b0_s;
  __shared__ const float* ilev_s[5];  // plane d of I at level n - m, null before the history
  __shared__ const float* slev_s[5];
  const int d = blockIdx.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid == 0) {
    const DirInfo di = dirs[d];
    di_s = di;
    n_s = *rs.step;
    if (d == 0 && blockIdx.x == 0) {
      rs.smax[n_s & 1] = 0u;     // max |S(n)|, filled by this step's source iteration
      rs.tile_ctr[n_s & 1] = 0;  // work counter of this step's persistent kernel
    }
    if (kUniN) {
      int m;
      float f;
      retarded_delay(di.dcoef, di.dcoef_lo, g.n_u, m, f);
      m_s = m < 1 ? 1 : (m > 3 ? 3 : m);
      f_s = f;
    }
    if (kUniMu) {
      const float xo = g.mut_u * di.ds;
      const float T = expf(-xo);
      T_s = T;
      b0_s = ray_b0(xo, T);
    }
  }
  __syncthreads();
  if (tid < 5) {
    const int L = n_s - tid;
    const size_t o = (static_cast<size_t>(ring_slot(L)) * g.na + d) * static_cast<size_t>(g.nv);
    ilev_s[tid] = L >= g.hist_from ? Iring + o : nullptr;
    slev_s[tid] = L >= g.hist_from ? Sring + o : nullptr;
  }
  __syncthreads();
  const int nrows = g.ny * g.nz;
  const int n = n_s;
  const int dom = di_s.dom, sgn = di_s.sgn, a0 = di_s.a0, a1 = di_s.a1;
  const float ds = di_s.ds, dc_hi = di_s.dcoef, dc_lo = di_s.dcoef_lo, src_amp = di_s.src_amp;
  const size_t plane = static_cast<size_t>(g.nv);
  const int8_t* off0 = offs + (static_cast<size_t>(d) * 2 + 0) * g.nmax;
  const int8_t* off1 = offs + (static_cast<size_t>(d) * 2 + 1) * g.nmax;
  const int nd = pick(dom, g.nx, g.ny, g.nz);
  const int n0 = pick(a0, g.nx, g.ny, g.nz);
  const int n1 = pick(a1, g.nx, g.ny, g.nz);
  const int sd = dom == 0 ? 1 : (dom == 1 ? g.nx : g.nx * g.ny);
  const int s0 = a0 == 0 ? 1 : (a0 == 1 ? g.nx : g.nx * g.ny);
  const int s1 = a1 == 0 ? 1 : (a1 == 1 ? g.nx : g.nx * g.ny);
  const size_t lev0 = static_cast<size_t>(d) * plane;
  const int m_u = kUniN ? m_s : 0;
  const float f_u = kUniN ? f_s : 0.0f;
  const float T_u = kUniMu ? T_s : 0.0f, b0_u = kUniMu ? b0_s : 0.0f;

  // Q of voxel v from its upwind sample u (kind 0), the inflow face (kind 1) or a side face
  // (kind 2: nothing enters, or with mirror faces the image); (qd, q0, q1) are the upwind
  // sample's unwrapped coordinates along dom, a0, a1.
  const auto update = [&](int v, int kind, int u, int qd, int q0, int q1) {
    int m;
    float f;
    if (kUniN) {
      m = m_u;
      f = f_u;
    } else {
      retarded_delay(dc_hi, dc_lo, __ldg(nidx + v), m, f);
      m = m < 1 ? 1 : (m > 3 ? 3 : m);  // the optics check keeps every delay in [1, 4)
    }
    const int L0 = n - m, L1 = n - m - 1;
    float Iup = 0.0f, Sup = 0.0f;
    if (kind == 0) {
      const float* i0p = ilev_s[m];
      const float* i1p = ilev_s[m + 1];
      float i0 = 0.0f, i1 = 0.0f, s0v = 0.0f, s1v = 0.0f;
      if (i0p) {
        i0 = __ldg(i0p + u);
        s0v = __ldg(slev_s[m] + u);
      }
      if (i1p) {
        i1 = __ldg(i1p + u);
        s1v = __ldg(slev_s[m + 1] + u);
      }
      Iup = fmaf(f, i1, (1.0f - f) * i0);
      Sup = fmaf(f, s1v, (1.0f - f) * s0v);
    } else if (g.mirror) {
      unsigned mask = 0u;
      const int cd = image_axis(qd, nd, 1u << dom, mask);
      const int c0 = image_axis(q0, n0, 1u << a0, mask);
      const int c1 = image_axis(q1, n1, 1u << a1, mask);
      const int img = cd * sd + c0 * s0 + c1 * s1;
      const ptrdiff_t doff = static_cast<ptrdiff_t>(refl[d * 8 + mask] - d) * static_cast<ptrdiff_t>(plane);
      float i0 = 0.0f, i1 = 0.0f, s0v = 0.0f, s1v = 0.0f;
      if (ilev_s[m]) {
        i0 = __ldg(ilev_s[m] + doff + img);
        s0v = __ldg(slev_s[m] + doff + img);
      }
      if (ilev_s[m + 1]) {
        i1 = __ldg(ilev_s[m + 1] + doff + img);
        s1v = __ldg(slev_s[m + 1] + doff + img);
      }
      Iup = fmaf(f, i1, (1.0f - f) * i0);
      Sup = fmaf(f, s1v, (1.0f - f) * s0v);
    } else if (kind == 1 && v == g.src_voxel && src_amp != 0.0f) {
      const float on0 = (L0 >= 0 && L0 < g.pulse_steps) ? 1.0f : 0.0f;
      const float on1 = (L1 >= 0 && L1 < g.pulse_steps) ? 1.0f : 0.0f;
      Iup = src_amp * fmaf(f, on1, (1.0f - f) * on0);
    }
    float T, b0;
    if (kUniMu) {
      T = T_u;
      b0 = b0_u;
    } else {
      const float xo = __ldg(mut + v) * ds;
      T = expf(-xo);
      b0 = ray_b0(xo, T);
    }
    Q[lev0 + v] = fmaf(Sup, b0, Iup * T);
  };

  for (int row = blockIdx.x * blockDim.y + threadIdx.y; row < nrows; row += gridDim.x * blockDim.y) {
    const int y = row % g.ny, z = row / g.ny;
    const int row_base = row * g.nx;
    if (a0 == 0) {
      // dom is y or z: the slab index, the offsets and the a1 coordinate are constant
      // along the row, and the upwind samples of the row are one contiguous run.
      const int pd = dom == 1 ? y : z;
      const int p1 = a1 == 1 ? y : z;
      const int kp = sgn > 0 ? pd : nd - 1 - pd;
      const int o0 = off0[kp];
      int qd = pd - sgn;
      int q1 = p1 - off1[kp];
      int row_kind = 0;
      if (g.periodic) {
        qd = (qd + nd) % nd;
        q1 = (q1 + n1) % n1;
      } else if (kp == 0) {
        row_kind = 1;
      } else if (q1 < 0 || q1 >= n1) {
        row_kind = 2;
      }
      const int urow = qd * sd + q1 * s1;
      for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
        int q0 = x - o0;
        int kind = row_kind;
        if (g.periodic) {
          q0 = (q0 + n0) % n0;
        } else if (kind == 0 && (q0 < 0 || q0 >= n0)) {
          kind = 2;
        }
        update(row_base + x, kind, urow + q0, qd, q0, q1);
      }
    } else {
      // dom is x: the slab index and the offsets change along the row
      for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
        const int kp = sgn > 0 ? x : nd - 1 - x;
        int qd = x - sgn;
        int q0 = y - off0[kp];
        int q1 = z - off1[kp];
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
        update(row_base + x, kind, qd * sd + q0 * s0 + q1 * s1, qd, q0, q1);
      }
    }
  }
}

}  // namespace

cudaError_t launch_sweep(const GridParams& g, const DirInfo* dirs, const int8_t* offs,
                         const float* Iring, const float* Sring, const float* mut,
                         const float* nidx, const int* refl, float* Q, RunState rs, cudaStream_t st) {
  if (g.mirror && !refl) return cudaErrorInvalidValue;
  int bx = ((g.nx + 31) / 32) * 32;
  if (bx > 256) bx = 256;
  const int by = 256 / bx;
  const int rows = g.ny * g.nz;
  dim3 block(bx, by);
  const int groups = (rows + by - 1) / by;
  dim3 grid((groups + kRowSweeps - 1) / kRowSweeps, g.na);
  const bool un = g.n_u >= 1.0f, um = g.mut_u >= 0.0f;
  if (un && um)
    sweep_kernel<true, true><<<grid, block, 0, st>>>(g, dirs, offs, Iring, Sring, mut, nidx, refl, Q, rs);
  else if (un)
    sweep_kernel<true, false><<<grid, block, 0, st>>>(g, dirs, offs, Iring, Sring, mut, nidx, refl, Q, rs);
  else if (um)
    sweep_kernel<false, true><<<grid, block, 0, st>>>(g, dirs, offs, Iring, Sring, mut, nidx, refl, Q, rs);
  else
    sweep_kernel<false, false><<<grid, block, 0, st>>>(g, dirs, offs, Iring, Sring, mut, nidx, refl, Q, rs);
  return cudaGetLastError();
}

}  // namespace trinity
