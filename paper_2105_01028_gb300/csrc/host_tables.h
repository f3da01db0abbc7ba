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
