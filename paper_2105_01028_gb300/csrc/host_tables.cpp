// Host-side FP64 tables: HEALPix directions, normalised phase matrix, ray lattice,
// cone weights.  Plain C++ on the CPU, run once per context.
#include "host_tables.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace trinity {

namespace {
constexpr double kPi = 3.14159265358979323846;
constexpr double kSnap = 1e-9;     // integer snap margin for floor decisions
constexpr double kDomTie = 1e-12;  // dominant-axis tie margin
constexpr int kCapMu = 64;         // cap sampling: rings in cos(theta)
constexpr int kCapPhi = 256;       // cap sampling: points per ring
}  // namespace

long floor_snap(double y) {
  const double r = std::nearbyint(y);
  if (std::fabs(y - r) < kSnap) return static_cast<long>(r);
  return static_cast<long>(std::floor(y));
}

// HEALPix (Gorski et al. 2005) pixel centres, RING order (Section 2.1 of the paper:
// equal-area angular bins).  Ring i = 1 .. 4N-1 from the north pole.  Polar-cap rings
// hold 4i pixels at z = 1 - i^2/(3N^2), phi = (pi/2i)(j - 1/2); belt rings hold 4N
// pixels at z = 4/3 - 2i/(3N), phi = (pi/2N)(j - s/2) with s = (i - N + 1) mod 2; the
// southern cap mirrors the northern one.
// RING index of the pixel containing the direction (z, phi).  HEALPix pixel boundaries
// (Gorski et al. 2005): in the belt |z| <= 2/3 they are the lines of a square lattice
// in (t + w/2, t - w/2) with t = 2 N phi / pi and w = 3 N z / 2; in the caps they are the
// curves x = k and y = k with x = tp sigma, y = (1 - tp) sigma, sigma = N sqrt(3 (1 - |z|)),
// tp the fraction of phi inside its quarter.
long ring_pixel(int nside, double z, double phi) {
  const double N = nside;
  const long npix = 12L * nside * nside;
  phi = std::fmod(phi, 2.0 * kPi);
  if (phi < 0.0) phi += 2.0 * kPi;
  if (std::fabs(z) <= 2.0 / 3.0) {
    const double t = 2.0 * N * phi / kPi, w = 1.5 * N * z;
    const double half = 0.5 * (N - 1.0);
    // lattice cell of the point: centres at half + integers along both rotated axes
    const long ka = static_cast<long>(std::floor(t + 0.5 * w - half + 0.5));
    const long kb = static_cast<long>(std::floor(t - 0.5 * w - half + 0.5));
    const long ring = 2L * nside - (ka - kb);           // a0 - b0 = ka - kb
    const long s = ((ring - nside + 1) % 2 + 2) % 2;
    // j = (a0 + b0 + s) / 2 with a0 + b0 = ka + kb + 2 half = ka + kb + N - 1
    long j = (ka + kb + nside - 1 + s) / 2;
    j = ((j - 1) % (4L * nside) + 4L * nside) % (4L * nside) + 1;
    return 2L * nside * (nside - 1) + 4L * nside * (ring - nside) + (j - 1);
  }
  const double sigma = N * std::sqrt(3.0 * (1.0 - std::fabs(z)));
  double q = std::floor(phi / (0.5 * kPi));
  if (q > 3.0) q = 3.0;
  const double tp = phi / (0.5 * kPi) - q;
  const long kx = static_cast<long>(std::floor(tp * sigma));
  const long ky = static_cast<long>(std::floor((1.0 - tp) * sigma));
  const long ring = kx + ky + 1;  // counted from the nearer pole
  const long j = static_cast<long>(q) * ring + kx + 1;
  if (z > 0.0) return 2L * ring * (ring - 1) + (j - 1);
  return npix - 2L * ring * (ring + 1) + (j - 1);
}

std::vector<int> parent_map(int nside_fine, int nside_coarse) {
  if (nside_coarse < 1 || nside_fine % nside_coarse != 0)
    throw std::runtime_error("the transport nside must be a multiple of the source-function nside");
  const std::vector<double> d = healpix_dirs(nside_fine);
  const size_t n = d.size() / 3;
  std::vector<int> par(n);
  for (size_t f = 0; f < n; ++f)
    par[f] = static_cast<int>(ring_pixel(nside_coarse, d[3 * f + 2], std::atan2(d[3 * f + 1], d[3 * f])));
  return par;
}

std::vector<double> healpix_dirs(int nside) {
  if (nside < 1) throw std::runtime_error("nside must be >= 1");
  const int npix = 12 * nside * nside;
  std::vector<double> out;
  out.reserve(3 * static_cast<size_t>(npix));
  const double N = nside;
  for (int i = 1; i < 4 * nside; ++i) {
    double z;
    int count;
    double dphi, shift;
    if (i < nside) {
      z = 1.0 - double(i) * i / (3.0 * N * N);
      count = 4 * i;
      dphi = kPi / (2.0 * i);
      shift = 0.5;
    } else if (i <= 3 * nside) {
      z = 4.0 / 3.0 - 2.0 * i / (3.0 * N);
      count = 4 * nside;
      dphi = kPi / (2.0 * N);
      shift = 0.5 * ((i - nside + 1) % 2);
    } else {
      const int k = 4 * nside - i;
      z = -(1.0 - double(k) * k / (3.0 * N * N));
      count = 4 * k;
      dphi = kPi / (2.0 * k);
      shift = 0.5;
    }
    const double st = std::sqrt((1.0 - z) * (1.0 + z));
    for (int j = 1; j <= count; ++j) {
      const double phi = dphi * (j - shift);
      out.push_back(st * std::cos(phi));
      out.push_back(st * std::sin(phi));
      out.push_back(z);
    }
  }
  return out;
}

namespace {

// Eq. 11: Henyey-Greenstein phase function per steradian.
double hg(double mu, double g) {
  const double q = 1.0 + g * g - 2.0 * g * mu;
  return (1.0 - g * g) / (4.0 * kPi * q * std::sqrt(q));
}

// K_ij = w * HG(Omega_i . Omega_j; g), scaled to unit row (= column) sums by a symmetric
// diagonal D (damped Sinkhorn: d <- sqrt(d / (K d))), then returned as D K D.
std::vector<double> scaled_kernel(const std::vector<double>& dirs, double g) {
  const int n = static_cast<int>(dirs.size() / 3);
  const double w = 4.0 * kPi / n;
  std::vector<double> K(static_cast<size_t>(n) * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double mu = dirs[3 * i] * dirs[3 * j] + dirs[3 * i + 1] * dirs[3 * j + 1] +
                  dirs[3 * i + 2] * dirs[3 * j + 2];
      mu = std::min(1.0, std::max(-1.0, mu));
      K[static_cast<size_t>(i) * n + j] = w * hg(mu, g);
    }
  std::vector<double> d(n, 1.0), Kd(n);
  for (int it = 0; it < 200000; ++it) {
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += K[static_cast<size_t>(i) * n + j] * d[j];
      Kd[i] = s;
    }
    double err = 0.0;
    for (int i = 0; i < n; ++i) err = std::max(err, std::fabs(d[i] * Kd[i] - 1.0));
    if (err < 1e-14) break;
    if (it == 199999) throw std::runtime_error("phase-matrix scaling did not converge");
    for (int i = 0; i < n; ++i) d[i] = std::sqrt(d[i] / Kd[i]);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) K[static_cast<size_t>(i) * n + j] *= d[i] * d[j];
  return K;
}

double mean_cos(const std::vector<double>& P, const std::vector<double>& dirs) {
  const int n = static_cast<int>(dirs.size() / 3);
  double tot = 0.0;
  for (int i = 0; i < n; ++i) {
    double row = 0.0;
    for (int j = 0; j < n; ++j) {
      const double mu = dirs[3 * i] * dirs[3 * j] + dirs[3 * i + 1] * dirs[3 * j + 1] +
                        dirs[3 * i + 2] * dirs[3 * j + 2];
      row += P[static_cast<size_t>(i) * n + j] * mu;
    }
    tot += row;
  }
  return tot / n;
}

}  // namespace

// Eq. 12 with a normalised discrete kernel: P = D K(g_eff) D, unit row and column sums,
// g_eff chosen by bisection so that the mean scattering cosine of P equals g.
std::vector<double> phase_matrix(int nside, double g, double* g_eff) {
  if (!(g > -1.0 && g < 1.0)) throw std::runtime_error("g must lie in (-1, 1)");
  const std::vector<double> dirs = healpix_dirs(nside);
  const int n = static_cast<int>(dirs.size() / 3);
  if (g == 0.0) {
    if (g_eff) *g_eff = 0.0;
    return std::vector<double>(static_cast<size_t>(n) * n, 1.0 / n);
  }
  double lo = g > 0 ? 0.0 : -1.0 + 1e-12;
  double hi = g > 0 ? 1.0 - 1e-12 : 0.0;
  for (int it = 0; it < 200 && hi - lo >= 1e-15; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mean_cos(scaled_kernel(dirs, mid), dirs) < g)
      lo = mid;
    else
      hi = mid;
  }
  const double ge = 0.5 * (lo + hi);
  if (g_eff) *g_eff = ge;
  return scaled_kernel(dirs, ge);
}

// Slab-lattice long rays (Section 2.1: rays laid independently of the grid, each grid
// point takes the nearest ray; Section 2.4 step 1).  Dominant axis = largest |Omega|
// component (ties: z, then y, then x); slab k' counted along the travel direction;
// the ray through a slab-0 voxel centre sits in column c + floor(1/2 + k' t) at slab k',
// t = Omega_a / |Omega_dom|, so the upwind sample of a slab-k' voxel is shifted by
// Delta(k') = floor(1/2 + k' t) - floor(1/2 + (k'-1) t) in {-1, 0, 1}.
Lattice build_lattice(const std::vector<double>& dirs, int nx, int ny, int nz, double h,
                      bool periodic) {
  Lattice L;
  L.na = static_cast<int>(dirs.size() / 3);
  const int n[3] = {nx, ny, nz};
  L.nmax = std::max(nx, std::max(ny, nz));
  L.dom.resize(L.na);
  L.sgn.resize(L.na);
  L.ds.resize(L.na);
  L.off.assign(static_cast<size_t>(L.na) * 2 * L.nmax, 0);
  for (int d = 0; d < L.na; ++d) {
    const double om[3] = {dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2]};
    const double ax = std::fabs(om[0]), ay = std::fabs(om[1]), az = std::fabs(om[2]);
    int dom;
    if (az >= std::max(ax, ay) - kDomTie)
      dom = 2;
    else if (ay >= ax - kDomTie)
      dom = 1;
    else
      dom = 0;
    L.dom[d] = dom;
    L.sgn[d] = om[dom] > 0 ? 1 : -1;
    L.ds[d] = h / std::fabs(om[dom]);
    int j = 0;
    for (int a = 0; a < 3; ++a) {
      if (a == dom) continue;
      const double t = om[a] / std::fabs(om[dom]);
      for (int k = 0; k < n[dom]; ++k) {
        long delta = floor_snap(0.5 + k * t) - floor_snap(0.5 + (k - 1.0) * t);
        if (k == 0 && !periodic) delta = 0;
        if (delta < -1 || delta > 1) throw std::runtime_error("lattice offset out of range");
        L.off[(static_cast<size_t>(d) * 2 + j) * L.nmax + k] = static_cast<int8_t>(delta);
      }
      ++j;
    }
  }
  return L;
}

// 15-degree collimation of the pulse and the detectors (Section 3.1).  The cap around
// the face normal is sampled at kCapMu x kCapPhi equal-area points (cos theta uniform,
// phi uniform, both at cell midpoints) in the frame (e_u, e_v, normal); each point goes
// to the direction with the largest dot product; the weight of a direction is its share
// of the points.  Two best dot products closer than 1e-12 would make the assignment
// depend on rounding, so that raises.
std::vector<double> cone_weights(const std::vector<double>& dirs, int face,
                                 double half_angle_deg, bool inward) {
  if (face < 0 || face > 5) throw std::runtime_error("face must be 0..5");
  if (!(half_angle_deg > 0.0 && half_angle_deg < 90.0))
    throw std::runtime_error("cone half-angle must lie in (0, 90) degrees");
  const int na = static_cast<int>(dirs.size() / 3);
  const int ax = face / 2;
  const double out_sign = (face % 2 == 0) ? -1.0 : 1.0;
  double nrm[3] = {0, 0, 0}, eu[3] = {0, 0, 0}, ev[3] = {0, 0, 0};
  nrm[ax] = inward ? -out_sign : out_sign;
  int uv[2], j = 0;
  for (int a = 0; a < 3; ++a)
    if (a != ax) uv[j++] = a;
  eu[uv[0]] = 1.0;
  ev[uv[1]] = 1.0;
  const double ct = std::cos(half_angle_deg * kPi / 180.0);
  std::vector<long> count(na, 0);
  for (int k = 0; k < kCapMu; ++k) {
    const double mu = 1.0 - (k + 0.5) * (1.0 - ct) / kCapMu;
    const double st = std::sqrt((1.0 - mu) * (1.0 + mu));
    for (int l = 0; l < kCapPhi; ++l) {
      const double phi = 2.0 * kPi * (l + 0.5) / kCapPhi;
      const double cp = std::cos(phi), sp = std::sin(phi);
      double p[3];
      for (int a = 0; a < 3; ++a) p[a] = mu * nrm[a] + st * cp * eu[a] + st * sp * ev[a];
      double best = -2.0, second = -2.0;
      int arg = -1;
      for (int d = 0; d < na; ++d) {
        const double dot = p[0] * dirs[3 * d] + p[1] * dirs[3 * d + 1] + p[2] * dirs[3 * d + 2];
        if (dot > best) {
          second = best;
          best = dot;
          arg = d;
        } else if (dot > second) {
          second = dot;
        }
      }
      if (best - second < 1e-12) throw std::runtime_error("cone sample equidistant from two directions");
      ++count[arg];
    }
  }
  std::vector<double> alpha(na);
  for (int d = 0; d < na; ++d) alpha[d] = double(count[d]) / double(kCapMu * kCapPhi);
  return alpha;
}

}  // namespace trinity

namespace trinity {

namespace {

// Upwind voxel of (x, y, z) along direction d on the lattice; -1 if outside the box.
long upwind_voxel(const Lattice& L, int d, const int n[3], bool periodic, const int p[3]) {
  const int dom = L.dom[d];
  const int sgn = L.sgn[d];
  const int kp = sgn > 0 ? p[dom] : n[dom] - 1 - p[dom];
  int q[3] = {p[0], p[1], p[2]};
  q[dom] = p[dom] - sgn;
  int j = 0;
  for (int a = 0; a < 3; ++a) {
    if (a == dom) continue;
    q[a] = p[a] - L.off[(static_cast<size_t>(d) * 2 + j) * L.nmax + kp];
    ++j;
  }
  if (periodic) {
    for (int a = 0; a < 3; ++a) q[a] = ((q[a] % n[a]) + n[a]) % n[a];
  } else {
    if (kp == 0) return -1;
    for (int a = 0; a < 3; ++a)
      if (q[a] < 0 || q[a] >= n[a]) return -1;
  }
  return (static_cast<long>(q[2]) * n[1] + q[1]) * n[0] + q[0];
}

// Unpolarised Fresnel reflectance, cosine form 1/2 (r_s^2 + r_p^2) (= Eq. 14), with the
// cosine of the Snell angle (Eq. 13); R = 1 under total internal reflection.
double fresnel_reflectance(double n1, double n2, double cos1, double* cos2_out) {
  const double eta = n1 / n2;
  const double sin2t = eta * eta * (1.0 - cos1 * cos1);
  if (cos1 <= 0.0 || sin2t >= 1.0) {
    *cos2_out = 0.0;
    return 1.0;
  }
  const double cos2 = std::sqrt(1.0 - sin2t);
  const double rs = (n1 * cos1 - n2 * cos2) / (n1 * cos1 + n2 * cos2);
  const double rp = (n2 * cos1 - n1 * cos2) / (n2 * cos1 + n1 * cos2);
  *cos2_out = cos2;
  return 0.5 * (rs * rs + rp * rp);
}

int nearest_pixel(const std::vector<double>& dirs, const double v[3]) {
  const int na = static_cast<int>(dirs.size() / 3);
  double best = -3.0;
  std::vector<double> dots(na);
  for (int d = 0; d < na; ++d) {
    dots[d] = dirs[3 * d] * v[0] + dirs[3 * d + 1] * v[1] + dirs[3 * d + 2] * v[2];
    best = std::max(best, dots[d]);
  }
  for (int d = 0; d < na; ++d)
    if (dots[d] >= best - 1e-12) return d;
  return 0;
}

// d(n)/d(axis) at index i of a line of length len (central inside, one-sided at ends).
double grad1(const std::vector<float>& nm, long base, long stride, int i, int len, double h) {
  if (len < 2) return 0.0;
  if (i == 0) return (double(nm[base + stride]) - double(nm[base])) / h;
  if (i == len - 1) return (double(nm[base + i * stride]) - double(nm[base + (i - 1) * stride])) / h;
  return (double(nm[base + (i + 1) * stride]) - double(nm[base + (i - 1) * stride])) / (2.0 * h);
}

}  // namespace

InterfaceTable build_interfaces(const std::vector<double>& dirs, const Lattice& L, int nx, int ny,
                                int nz, double h, bool periodic, const std::vector<float>& nmap) {
  InterfaceTable T;
  const int na = static_cast<int>(dirs.size() / 3);
  T.na = na;
  const int n[3] = {nx, ny, nz};
  const long nv = static_cast<long>(nx) * ny * nz;
  // candidates: voxels with a different n anywhere in their 3x3x3 neighbourhood
  std::vector<long> cand;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long v = (static_cast<long>(z) * ny + y) * nx + x;
        bool diff = false;
        for (int dz = -1; dz <= 1 && !diff; ++dz)
          for (int dy = -1; dy <= 1 && !diff; ++dy)
            for (int dx = -1; dx <= 1 && !diff; ++dx) {
              int qx = x + dx, qy = y + dy, qz = z + dz;
              if (periodic) {
                qx = (qx + nx) % nx;
                qy = (qy + ny) % ny;
                qz = (qz + nz) % nz;
              } else if (qx < 0 || qy < 0 || qz < 0 || qx >= nx || qy >= ny || qz >= nz) {
                continue;
              }
              if (nmap[(static_cast<long>(qz) * ny + qy) * nx + qx] != nmap[v]) diff = true;
            }
        if (diff) cand.push_back(v);
      }
  (void)nv;
  for (long v : cand) {
    const int x = static_cast<int>(v % nx), y = static_cast<int>((v / nx) % ny), z = static_cast<int>(v / (static_cast<long>(nx) * ny));
    const int p[3] = {x, y, z};
    double g[3];
    g[0] = grad1(nmap, (static_cast<long>(z) * ny + y) * nx, 1, x, nx, h);
    g[1] = grad1(nmap, static_cast<long>(z) * ny * nx + x, nx, y, ny, h);
    g[2] = grad1(nmap, static_cast<long>(y) * nx + x, static_cast<long>(nx) * ny, z, nz, h);
    const double gn = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (gn == 0.0) continue;
    const double m[3] = {g[0] / gn, g[1] / gn, g[2] / gn};
    std::vector<std::vector<std::pair<int, double>>> rows(na);  // gather rows
    std::vector<uint8_t> keep(na, 1);
    bool any = false;
    for (int j = 0; j < na; ++j) {
      const long u = upwind_voxel(L, j, n, periodic, p);
      if (u < 0 || nmap[u] == nmap[v]) continue;
      const double n1 = nmap[u], n2 = nmap[v];
      const double om[3] = {dirs[3 * j], dirs[3 * j + 1], dirs[3 * j + 2]};
      const double dn = om[0] * m[0] + om[1] * m[1] + om[2] * m[2];
      const double cos1 = std::fabs(dn);
      double cos2 = 0.0;
      const double R = fresnel_reflectance(n1, n2, cos1, &cos2);
      const double omr[3] = {om[0] - 2.0 * dn * m[0], om[1] - 2.0 * dn * m[1], om[2] - 2.0 * dn * m[2]};
      const int dr = nearest_pixel(dirs, omr);
      std::vector<std::pair<int, double>> outs = {{dr, R}};
      if (R < 1.0) {
        const double eta = n1 / n2;
        const double s = dn >= 0 ? 1.0 : -1.0;
        const double omt[3] = {eta * om[0] + (cos2 - eta * cos1) * s * m[0],
                               eta * om[1] + (cos2 - eta * cos1) * s * m[1],
                               eta * om[2] + (cos2 - eta * cos1) * s * m[2]};
        outs.push_back({nearest_pixel(dirs, omt), 1.0 - R});
      }
      keep[j] = 0;
      any = true;
      for (const auto& o : outs) {
        rows[o.first].push_back({j, o.second});
        T.s_vox.push_back(static_cast<int>(v));
        T.s_j.push_back(j);
        T.s_d.push_back(o.first);
        T.s_w.push_back(o.second);
      }
    }
    if (!any) continue;
    T.vox.push_back(static_cast<int>(v));
    const int base = static_cast<int>(T.src.size());
    int cnt = 0;
    for (int d = 0; d < na; ++d) {
      T.rowptr.push_back(base + cnt);
      std::sort(rows[d].begin(), rows[d].end());
      for (const auto& e : rows[d]) {
        T.src.push_back(e.first);
        T.w64.push_back(e.second);
        T.w.push_back(static_cast<float>(e.second));
        ++cnt;
      }
    }
    T.rowptr.push_back(base + cnt);
    T.keep.insert(T.keep.end(), keep.begin(), keep.end());
  }
  return T;
}

}  // namespace trinity

namespace trinity {

std::vector<double> solve_dense(std::vector<double> A, std::vector<double> B, int n) {
  // Gaussian elimination with partial pivoting on [A | B], B with n columns
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = std::fabs(A[static_cast<size_t>(k) * n + k]);
    for (int r = k + 1; r < n; ++r) {
      const double a = std::fabs(A[static_cast<size_t>(r) * n + k]);
      if (a > best) {
        best = a;
        piv = r;
      }
    }
    if (!(best > 0.0)) throw std::runtime_error("singular system");
    if (piv != k)
      for (int c = 0; c < n; ++c) {
        std::swap(A[static_cast<size_t>(k) * n + c], A[static_cast<size_t>(piv) * n + c]);
        std::swap(B[static_cast<size_t>(k) * n + c], B[static_cast<size_t>(piv) * n + c]);
      }
    const double inv = 1.0 / A[static_cast<size_t>(k) * n + k];
    for (int r = k + 1; r < n; ++r) {
      const double f = A[static_cast<size_t>(r) * n + k] * inv;
      if (f == 0.0) continue;
      for (int c = k; c < n; ++c) A[static_cast<size_t>(r) * n + c] -= f * A[static_cast<size_t>(k) * n + c];
      for (int c = 0; c < n; ++c) B[static_cast<size_t>(r) * n + c] -= f * B[static_cast<size_t>(k) * n + c];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    const double inv = 1.0 / A[static_cast<size_t>(k) * n + k];
    for (int c = 0; c < n; ++c) {
      double acc = B[static_cast<size_t>(k) * n + c];
      for (int j = k + 1; j < n; ++j) acc -= A[static_cast<size_t>(k) * n + j] * B[static_cast<size_t>(j) * n + c];
      B[static_cast<size_t>(k) * n + c] = acc * inv;
    }
  }
  return B;
}

double ray_b1_fp64(double x) {
  if (x < 1e-3) return x / 2 - x * x / 6 + x * x * x / 24 - x * x * x * x / 120;
  return (x - 1.0 + std::exp(-x)) / x;
}

}  // namespace trinity
