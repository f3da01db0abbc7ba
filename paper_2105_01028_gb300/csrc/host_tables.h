// Host-side FP64 tables of the forward model: HEALPix directions, the normalised
// phase matrix, the long-ray lattice, cone weights.  Built once per context on the CPU.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace trinity {

constexpr double kC0 = 299.792458;  // mm/ns; c = c0 / n (Eq. 1)
constexpr int kRing = 5;            // stored time levels of I and S

// HEALPix RING pixel centres (x, y, z) per direction.
std::vector<double> healpix_dirs(int nside);

// RING index of the HEALPix pixel containing direction (z = cos theta, phi).
long ring_pixel(int nside, double z, double phi);

// Coarse pixel containing each fine pixel's centre (its parent in the nested hierarchy).
std::vector<int> parent_map(int nside_fine, int nside_coarse);

// X solving A X = B for dense n x n A and B (row-major, partial pivoting); throws if singular.
std::vector<double> solve_dense(std::vector<double> A, std::vector<double> B, int n);

// b1(x) of Eq. 9 in FP64 (Taylor series below x = 1e-3).
double ray_b1_fp64(double x);

// Normalised phase matrix of Eq. 12 (row-major N_a x N_a) and its g_eff.
std::vector<double> phase_matrix(int nside, double g, double* g_eff);

struct Lattice {
  int na = 0;
  int nmax = 0;                 // max(nx, ny, nz): stride of the offset table
  std::vector<int32_t> dom;     // dominant axis per direction
  std::vector<int32_t> sgn;     // +1 / -1 travel sign along dom
  std::vector<double> ds;       // h / |Omega_dom|
  std::vector<int8_t> off;      // [na][2][nmax] transverse offsets Delta_a(k')
};

// Throws std::runtime_error on an invalid grid.
Lattice build_lattice(const std::vector<double>& dirs, int nx, int ny, int nz, double h,
                      bool periodic);

// Fraction of a cap around the face's inward / outward normal nearest to each direction.
std::vector<double> cone_weights(const std::vector<double>& dirs, int face,
                                 double half_angle_deg, bool inward);

// floor(y), with y within 1e-9 of an integer taken as that integer.
long floor_snap(double y);

}  // namespace trinity

namespace trinity {

// Refraction / reflection at index steps (Eqs. 13-14), gather form per interface voxel:
// out[d] = keep[d] * Q[d] + sum over entries (src j, weight w) of row d of w * Q[j].
struct InterfaceTable {
  int na = 0;
  std::vector<int> vox;        // interface voxels (ascending)
  std::vector<int> rowptr;     // [vox.size()][na + 1] entry ranges per output direction
  std::vector<int> src;        // source direction j of each entry
  std::vector<float> w;        // weight of each entry (FP32 copy)
  std::vector<double> w64;     // weight of each entry (FP64)
  std::vector<uint8_t> keep;   // [vox.size()][na] 1 if direction d does not cross
  // scatter form (for inspection): (voxel, crossing j, target d, weight), sorted
  std::vector<int> s_vox, s_j, s_d;
  std::vector<double> s_w;
};

// Voxels whose upwind sample (ray lattice) lies in a voxel of different n: the arriving
// light along that direction is split into the specular and Snell directions (each
// snapped to the nearest pixel) with the Fresnel reflectance of Eq. 14.
InterfaceTable build_interfaces(const std::vector<double>& dirs, const Lattice& L, int nx, int ny,
                                int nz, double h, bool periodic, const std::vector<float>& nmap);

}  // namespace trinity
