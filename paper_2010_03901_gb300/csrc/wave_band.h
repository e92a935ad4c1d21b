// Fourier Forwarding near-boundary solver U_B (Section 4.2): the band of grid points
// near the curve and its small-step operators, built on the host at plan time.
#pragma once
#include <cstdint>
#include <vector>

#include "plan_internal.h"

namespace fc2d {

// Column key of an operator entry: the kind in the top two bits, the index below.
//   unknown: index into the band's unknown list (the stepped values)
//   grid:    grid linear index j nx + i of an interface point (a value of U_FC)
//   bdry:    index of a plan boundary point (a Dirichlet datum)
constexpr uint32_t kKeyUnknown = 0u << 30;
constexpr uint32_t kKeyGrid = 1u << 30;
constexpr uint32_t kKeyBdry = 2u << 30;
constexpr uint32_t kKeyKind = 3u << 30;
constexpr uint32_t kKeyIndex = (1u << 30) - 1;

// Parameters of the closure (the reading of the paper's sketch; see wave_band.cpp).
constexpr int kUbHalfWidth = 4;    // order-8 central second difference away from the curve
constexpr int kUbPolyDeg = 3;      // degree of the boundary polynomial of a chord side
constexpr double kUbXiMin = 0.5;   // chord end points nearer than this (in h) are slaved
constexpr int kUbDissP = 4;        // the dissipation uses fourth differences
constexpr double kUbSigma = 0.3;   // dissipation coefficient
constexpr int kUbBandExtra = 2;    // the band reaches delta + 2h from the curve
constexpr double kUbCfl = 0.125;   // c dt / h
// Decision margin (in units of h) on the distance and crossing thresholds: points
// exactly on a threshold (symmetric grids produce them) are decided alike by any two
// evaluations that differ in the last bit.
constexpr double kUbTie = 1.0 / 1073741824.0;  // 2^-30

struct Csr {
  std::vector<int32_t> off;  // rows + 1
  std::vector<uint32_t> col; // keys
  std::vector<double> w;
};

struct WaveBand {
  int n_c = 0;
  double delta = 0.0;                  // n_c h: U_FC is the solution at distance >= delta
  double reach = 0.0;                  // delta + 2h: the band's outer distance
  std::vector<int32_t> unknown_lin;    // stepped grid points (ascending linear index)
  std::vector<int32_t> slaved_lin;     // grid points given by a boundary polynomial
  std::vector<double> unknown_dist, slaved_dist;
  std::vector<int32_t> iface_lin;      // interface points the operators reference
  Csr L;                               // second differences, one row per unknown
  Csr D;                               // dissipation B^T B / 2, one row per unknown
  Csr S;                               // slaved values, one row per slaved point
  std::vector<int32_t> near_lin;       // band points at distance < delta (ascending)
  std::vector<int32_t> near_src;       // >= 0: unknown index, < 0: -1 - slaved index
};

// Build U_B's band and operators for large-step width delta = n_c h, the band reaching
// reach_cells h from the curve (n_c + 2 with interface values from the full U_FC,
// ceil(sqrt(2) n_c) + 2 for the small-square procedure).
fc2d_status build_wave_band(const fc2d_plan_s* p, int n_c, int reach_cells, WaveBand& out);

// The small-square interface procedure (Section 4.2): squares of (2a+1)^2 grid points
// inside the domain, each with a P x P periodic expansion (P = 2a + 1 + C), serving the
// interface points within a - n_c of its centre (max norm, grid units).
constexpr int kSqP = 64;  // periodic length of a square's expansion
struct SquareSet {
  int a = 0, R = 0, P = kSqP, C = 0, d = 0;
  std::vector<int32_t> origin_j, origin_i;   // first grid row / column of each square
  std::vector<int32_t> served_off;           // [n_sq + 1]
  std::vector<int32_t> served_lin;           // grid linear index of each served point
  std::vector<int32_t> served_local;         // its row * P + column in the square's box
  std::vector<double> A, Q;                  // coarse continuation A [C][d], Gram Q [d][d]
};
fc2d_status build_wave_squares(const fc2d_plan_s* p, const WaveBand& band, int n_c,
                               SquareSet& out);

}  // namespace fc2d
