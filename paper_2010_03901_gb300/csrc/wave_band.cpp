// The band and small-step operators of the Fourier Forwarding near-boundary solver U_B
// (Section 4.2), built on the host.
//
// The paper sketches U_B only: explicit small steps on a set containing the grid
// points within c Delta T of the curve, second-order Taylor stepping at CFL 0.125
// (Section 4.2.1), Dirichlet data imposed by the embedded-boundary interpolation the
// paper cites (Appelo & Petersson 2012: values beyond the curve from a polynomial
// through the boundary datum and interior values along each grid line), and values at
// the band's inner edge from the interior propagator U_FC.  This file builds the
// operators of the reading the library follows:
//
// * band: grid points inside the curve at distance < delta + 2h (delta = n_c h); the
//   distance is |P - q(theta*)| with the nearest-point foot theta* by Newton's method;
// * every threshold decision (band, U_B's solution points at distance < delta, slaving
//   at xi < 1/2, the closest of several crossings) carries the margin kUbTie (in h), so
//   that points exactly on a threshold are decided alike by independent evaluations;
// * chords: the inside runs of a grid line between two consecutive crossings;
// * slaved points: a chord end point closer than h/2 to its crossing (along x or y) is
//   not stepped; its value is the boundary polynomial of that side at the point (the
//   closest crossing wins; ties: x before y, lower side first);
// * boundary polynomial of a chord side: the degree <= 3 Lagrange interpolant through
//   the crossing (its datum) and the 3 non-slaved chord points nearest it; a chord with
//   fewer takes all of them and the other crossing's datum;
// * second differences: along each axis the central difference of order 2 hw,
//   hw = min(4, k- + 1, k+ + 1) with k-/k+ the chord points before/after the point, so
//   at most one value beyond each crossing is used, the "ghost" value, which is the
//   boundary polynomial at the ghost's coordinate;
// * dissipation D = B^T B / 2, B the fourth differences (1, -4, 6, -4, 1)/16 over every
//   window of five consecutive non-slaved points of a chord holding an unknown.
// The stepping itself (ff.cu): u^{n+1} = 2u^n - u^{n-1} + (h/8)^2 L(u^n) - 0.3 D(u^n -
// u^{n-1}), with u^1 = u^0 + dt u_t^0 + (h/8)^2/2 L(u^0).
//
// The small-square procedure (build_wave_squares): squares of (2a+1)^2 grid points, all
// inside the domain, a = (P - C - 1)/2 (P = 64, C the continuation length), each serving
// the interface points q with |q - centre|_inf <= R = a - n_c (grid units), so that the
// disk of radius n_c h around q, its domain of dependence over a large step, lies in the
// square.  Placement: the interface points by increasing linear index; for the first one
// not yet served, among the centres within R of it whose square is inside, the one
// serving the most unserved points (ties: smaller row, then column) serves them all.
#include "wave_band.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <utility>

namespace fc2d {

namespace {

using Form = std::vector<std::pair<uint32_t, double>>;

void form_add(Form& f, uint32_t key, double w) {
  for (auto& e : f)
    if (e.first == key) {
      e.second += w;
      return;
    }
  f.push_back({key, w});
}

double factorial(int n) {
  double r = 1.0;
  for (int k = 2; k <= n; ++k) r *= double(k);
  return r;
}

// Order-2hw central second-difference weights on offsets -hw..hw (times 1/h^2), closed
// form: w_k = 2 (-1)^(k+1) (hw!)^2 / (k^2 (hw-k)! (hw+k)!), w_0 = -2 sum 1/k^2.
std::vector<double> central_weights(int hw) {
  std::vector<double> w(2 * hw + 1, 0.0);
  for (int k = 1; k <= hw; ++k) {
    const double num = 2.0 * ((k + 1) % 2 == 0 ? 1.0 : -1.0) * (factorial(hw) * factorial(hw));
    const double den = double(k * k) * factorial(hw - k) * factorial(hw + k);
    w[hw + k] = w[hw - k] = num / den;
  }
  double s = 0.0;
  for (int k = 1; k <= hw; ++k) s += 1.0 / double(k * k);
  w[hw] = -2.0 * s;
  return w;
}

std::vector<double> lagrange(const std::vector<double>& nodes, double x) {
  const size_t n = nodes.size();
  std::vector<double> w(n, 1.0);
  for (size_t j = 0; j < n; ++j)
    for (size_t k = 0; k < n; ++k)
      if (k != j) w[j] *= (x - nodes[k]) / (nodes[j] - nodes[k]);
  return w;
}

struct Builder {
  const fc2d_plan_s* p;
  int nx, ny;
  double h, a0, b0;
  std::vector<uint8_t> ins;     // inside mask [ny][nx]
  std::vector<double> dist;     // distance of band candidates (inf: far)
  std::vector<int8_t> slave;    // -1, or axis * 2 + (side > 0)
  std::vector<int32_t> uidx;    // unknown index or -1
  std::vector<int32_t> lin_u;
  std::map<int32_t, int> iface; // referenced interface points

  bool inside(int j, int i) const {
    return i >= 0 && j >= 0 && i < nx && j < ny && ins[(size_t)j * nx + i];
  }
  void step(int& j, int& i, int axis, int k) const {
    if (axis == 0)
      i += k;
    else
      j += k;
  }
  double coord(int j, int i, int axis) const { return axis == 0 ? a0 + h * double(i) : b0 + h * double(j); }
  bool is_slaved(int j, int i) const { return slave[(size_t)j * nx + i] >= 0; }
  bool is_unknown(int j, int i) const { return uidx[(size_t)j * nx + i] >= 0; }

  // Crossing bounding the chord of (j, i) on `side`: false if no chord of the line holds
  // the point (it lies on the curve where the line only touches it).
  bool crossing(int j, int i, int axis, int side, double& X, int64_t& b) const {
    const double c = coord(j, i, axis);
    int64_t o0, o1;
    if (axis == 0) {
      o0 = p->row_off[j];
      o1 = p->row_off[j + 1];
    } else {
      o0 = p->col_off[i];
      o1 = p->col_off[i + 1];
    }
    const int comp = axis == 0 ? 0 : 1;  // x of a row crossing, y of a column crossing
    auto val = [&](int64_t k) { return p->bdry_xy[2 * (size_t)k + comp]; };
    // last crossing <= c
    int64_t m = o0 - 1;
    for (int64_t k = o0; k < o1; ++k)
      if (val(k) <= c) m = k;
    const int64_t lo = m - ((m - o0) % 2 + 2) % 2;
    if (m < o0 || lo + 1 >= o1 || !(val(lo) <= c && c <= val(lo + 1))) return false;
    b = side > 0 ? lo + 1 : lo;
    X = val(b);
    return true;
  }

  int count(int j, int i, int axis, int side) const {
    int k = 0;
    for (;;) {
      int jj = j, ii = i;
      step(jj, ii, axis, (k + 1) * side);
      if (!inside(jj, ii)) return k;
      ++k;
    }
  }

  uint32_t key(int j, int i) {
    const int32_t lin = j * nx + i;
    if (uidx[lin] >= 0) return kKeyUnknown | (uint32_t)uidx[lin];
    iface.emplace(lin, (int)iface.size());
    return kKeyGrid | (uint32_t)lin;
  }

  fc2d_status poly(int j, int i, int axis, int side, double x, Form& out) {
    double X;
    int64_t b;
    if (!crossing(j, i, axis, side, X, b))
      return set_error(FC2D_ERR_GEOMETRY, "wave band: a grid point has no chord along a grid line");
    const int k = count(j, i, axis, side);
    int jj = j, ii = i;
    step(jj, ii, axis, k * side);
    std::vector<double> nodes{X};
    std::vector<uint32_t> keys{kKeyBdry | (uint32_t)b};
    while ((int)nodes.size() < kUbPolyDeg + 1) {
      if (!inside(jj, ii)) {
        double X2;
        int64_t b2;
        if (!crossing(j, i, axis, -side, X2, b2))
          return set_error(FC2D_ERR_GEOMETRY, "wave band: chord without a second crossing");
        nodes.push_back(X2);
        keys.push_back(kKeyBdry | (uint32_t)b2);
        break;
      }
      if (!is_slaved(jj, ii)) {
        nodes.push_back(coord(jj, ii, axis));
        keys.push_back(key(jj, ii));
      }
      step(jj, ii, axis, -side);
    }
    const std::vector<double> w = lagrange(nodes, x);
    out.clear();
    for (size_t n = 0; n < w.size(); ++n) form_add(out, keys[n], w[n]);
    return FC2D_OK;
  }

  fc2d_status value(int j, int i, Form& out) {
    const int8_t s = slave[(size_t)j * nx + i];
    if (s >= 0) {
      const int axis = s / 2, side = (s % 2) ? 1 : -1;
      return poly(j, i, axis, side, coord(j, i, axis), out);
    }
    out.clear();
    out.push_back({key(j, i), 1.0});
    return FC2D_OK;
  }

  fc2d_status laplacian_row(int j, int i, Form& form) {
    form.clear();
    const double h2 = h * h;
    Form f2;
    for (int axis = 0; axis < 2; ++axis) {
      const int km = count(j, i, axis, -1), kp = count(j, i, axis, +1);
      const int hw = std::min(kUbHalfWidth, std::min(km + 1, kp + 1));
      const std::vector<double> w = central_weights(hw);
      for (int k = -hw; k <= hw; ++k) {
        int jj = j, ii = i;
        step(jj, ii, axis, k);
        fc2d_status st;
        if (k < -km || k > kp)
          st = poly(j, i, axis, k > 0 ? 1 : -1, coord(jj, ii, axis), f2);
        else
          st = value(jj, ii, f2);
        if (st) return st;
        for (const auto& e : f2) form_add(form, e.first, w[k + hw] * e.second / h2);
      }
    }
    return FC2D_OK;
  }
};

// Distance to the curve of the inside points near it: each boundary node seeds the
// points within reach + 2 node spacings of it; the nearest node's parameter starts the
// foot search (best of 49 samples within +-1.5 k2, then Newton's method).
fc2d_status band_distances(Builder& bd, double reach) {
  const fc2d_plan_s* p = bd.p;
  const int B = p->prm.B;
  const double k2 = 2.0 * M_PI / B;
  std::vector<double> bx(B), by(B);
  double spacing = 0.0;
  for (int k = 0; k < B; ++k) p->curve.eval(k2 * k, bx[k], by[k]);
  for (int k = 0; k < B; ++k) {
    const int k1 = (k + 1) % B;
    spacing = std::max(spacing, std::hypot(bx[k1] - bx[k], by[k1] - by[k]));
  }
  const double R = reach + 2.0 * spacing;
  const size_t n = (size_t)bd.nx * bd.ny;
  std::vector<double> best(n, INFINITY), seed(n, 0.0);
  for (int k = 0; k < B; ++k) {
    const int i0 = std::max(0, (int)std::floor((bx[k] - R - bd.a0) / bd.h));
    const int i1 = std::min(bd.nx - 1, (int)std::ceil((bx[k] + R - bd.a0) / bd.h));
    const int j0 = std::max(0, (int)std::floor((by[k] - R - bd.b0) / bd.h));
    const int j1 = std::min(bd.ny - 1, (int)std::ceil((by[k] + R - bd.b0) / bd.h));
    for (int j = j0; j <= j1; ++j)
      for (int i = i0; i <= i1; ++i) {
        const size_t lin = (size_t)j * bd.nx + i;
        if (!bd.ins[lin]) continue;
        const double dx = bd.a0 + bd.h * i - bx[k], dy = bd.b0 + bd.h * j - by[k];
        const double d = std::hypot(dx, dy);
        if (d < R && d < best[lin]) {
          best[lin] = d;
          seed[lin] = k2 * k;
        }
      }
  }
  std::vector<int32_t> cand;
  std::vector<double> qx, qy, th;
  for (size_t lin = 0; lin < n; ++lin)
    if (best[lin] < INFINITY) {
      cand.push_back((int32_t)lin);
      qx.push_back(bd.a0 + bd.h * double(lin % bd.nx));
      qy.push_back(bd.b0 + bd.h * double(lin / bd.nx));
      th.push_back(seed[lin]);
    }
  std::vector<int> conv;
  fc2d_status st = foot_newton_gpu(p->curve, qx, qy, th, conv, 1.5 * k2);
  if (st) return st;
  bd.dist.assign(n, INFINITY);
  for (size_t m = 0; m < cand.size(); ++m) {
    double fx, fy;
    p->curve.eval(th[m], fx, fy);
    const double d = std::hypot(qx[m] - fx, qy[m] - fy);
    if (d < reach && !conv[m])
      return set_error(FC2D_ERR_NOT_CONVERGED, "wave band: foot search did not converge");
    bd.dist[cand[m]] = d;
  }
  return FC2D_OK;
}

void to_csr(const std::vector<Form>& rows, Csr& out) {
  out.off.assign(1, 0);
  out.col.clear();
  out.w.clear();
  for (const Form& f : rows) {
    for (const auto& e : f) {
      out.col.push_back(e.first);
      out.w.push_back(e.second);
    }
    out.off.push_back((int32_t)out.col.size());
  }
}

}  // namespace

fc2d_status build_wave_band(const fc2d_plan_s* p, int n_c, int reach_cells, WaveBand& out) {
  Builder bd;
  bd.p = p;
  bd.nx = p->grid.nx;
  bd.ny = p->grid.ny;
  bd.h = p->grid.h;
  bd.a0 = p->grid.a0;
  bd.b0 = p->grid.b0;
  const size_t n = (size_t)bd.nx * bd.ny;
  bd.ins.assign(n, 0);
  for (int j = 0; j < bd.ny; ++j)
    for (int k = p->row_iv_off[j]; k < p->row_iv_off[j + 1]; ++k)
      for (int i = p->row_iv[2 * k]; i <= p->row_iv[2 * k + 1]; ++i) bd.ins[(size_t)j * bd.nx + i] = 1;
  out = WaveBand();
  out.n_c = n_c;
  out.delta = n_c * bd.h;
  out.reach = double(reach_cells) * bd.h;
  fc2d_status st = band_distances(bd, out.reach);
  if (st) return st;
  // band and slaving
  std::vector<int32_t> band;
  for (size_t lin = 0; lin < n; ++lin)
    if (bd.ins[lin] && bd.dist[lin] < out.reach - kUbTie * bd.h) band.push_back((int32_t)lin);
  bd.slave.assign(n, -1);
  for (int32_t lin : band) {
    const int j = lin / bd.nx, i = lin % bd.nx;
    double best = INFINITY;
    for (int axis = 0; axis < 2; ++axis)
      for (int side = -1; side <= 1; side += 2) {
        int jj = j, ii = i;
        bd.step(jj, ii, axis, side);
        if (bd.inside(jj, ii)) continue;
        double X;
        int64_t b;
        if (!bd.crossing(j, i, axis, side, X, b)) continue;
        const double xi = std::fabs(X - bd.coord(j, i, axis)) / bd.h;
        if (xi < kUbXiMin - kUbTie && xi < best - kUbTie) {
          best = xi;
          bd.slave[lin] = (int8_t)(axis * 2 + (side > 0 ? 1 : 0));
        }
      }
  }
  bd.uidx.assign(n, -1);
  for (int32_t lin : band)
    if (bd.slave[lin] < 0) {
      bd.uidx[lin] = (int32_t)bd.lin_u.size();
      bd.lin_u.push_back(lin);
      out.unknown_lin.push_back(lin);
      out.unknown_dist.push_back(bd.dist[lin]);
    } else {
      out.slaved_lin.push_back(lin);
      out.slaved_dist.push_back(bd.dist[lin]);
    }
  // second differences
  std::vector<Form> rows(bd.lin_u.size());
  for (size_t r = 0; r < bd.lin_u.size(); ++r) {
    const int32_t lin = bd.lin_u[r];
    if ((st = bd.laplacian_row(lin / bd.nx, lin % bd.nx, rows[r]))) return st;
  }
  to_csr(rows, out.L);
  // dissipation: rows of B over windows of five non-slaved chord points, each window
  // once (at its first unknown); then D = B^T B / 2 restricted to the unknowns' rows
  {
    const double coef[kUbDissP + 1] = {1.0 / 16, -4.0 / 16, 6.0 / 16, -4.0 / 16, 1.0 / 16};
    std::vector<Form> D(bd.lin_u.size());
    for (int axis = 0; axis < 2; ++axis)
      for (int32_t lin : bd.lin_u) {
        const int j = lin / bd.nx, i = lin % bd.nx;
        for (int start = -kUbDissP; start <= 0; ++start) {
          int pj[kUbDissP + 1], pi[kUbDissP + 1];
          bool ok = true;
          int first = -1;
          for (int k = 0; k <= kUbDissP; ++k) {
            pj[k] = j;
            pi[k] = i;
            bd.step(pj[k], pi[k], axis, start + k);
            if (!bd.inside(pj[k], pi[k]) || bd.is_slaved(pj[k], pi[k])) ok = false;
            else if (first < 0 && bd.is_unknown(pj[k], pi[k])) first = k;
          }
          if (!ok || pj[first] != j || pi[first] != i) continue;
          Form win;
          for (int k = 0; k <= kUbDissP; ++k) form_add(win, bd.key(pj[k], pi[k]), coef[k]);
          for (const auto& a : win) {
            if ((a.first & kKeyKind) != kKeyUnknown) continue;
            Form& row = D[a.first & kKeyIndex];
            for (const auto& b : win) form_add(row, b.first, 0.5 * a.second * b.second);
          }
        }
      }
    to_csr(D, out.D);
  }
  // slaved values
  {
    std::vector<Form> S(out.slaved_lin.size());
    for (size_t r = 0; r < S.size(); ++r) {
      const int32_t lin = out.slaved_lin[r];
      if ((st = bd.value(lin / bd.nx, lin % bd.nx, S[r]))) return st;
    }
    to_csr(S, out.S);
  }
  for (const auto& e : bd.iface) out.iface_lin.push_back(e.first);
  // the points where U_B is the solution (eq. (4.9)): distance < delta
  {
    size_t a = 0, b = 0;
    while (a < out.unknown_lin.size() || b < out.slaved_lin.size()) {
      const bool take_u = b >= out.slaved_lin.size() ||
                          (a < out.unknown_lin.size() && out.unknown_lin[a] < out.slaved_lin[b]);
      if (take_u) {
        if (out.unknown_dist[a] < out.delta - kUbTie * bd.h) {
          out.near_lin.push_back(out.unknown_lin[a]);
          out.near_src.push_back((int32_t)a);
        }
        ++a;
      } else {
        if (out.slaved_dist[b] < out.delta - kUbTie * bd.h) {
          out.near_lin.push_back(out.slaved_lin[b]);
          out.near_src.push_back(-1 - (int32_t)b);
        }
        ++b;
      }
    }
  }
  return FC2D_OK;
}

fc2d_status build_wave_squares(const fc2d_plan_s* p, const WaveBand& band, int n_c,
                               SquareSet& out) {
  out = SquareSet();
  const int nx = p->grid.nx, ny = p->grid.ny, C = p->prm.C, d = p->prm.d, n_r = p->prm.n_r;
  out.P = kSqP;
  out.C = C;
  out.d = d;
  out.a = (kSqP - C - 1) / 2;
  out.R = out.a - n_c;
  if (out.R < 0 || 2 * out.a + 1 + C != kSqP)
    return set_error(FC2D_ERR_UNSUPPORTED, "small squares: n_c too large for a 64-point box");
  const int a = out.a, R = out.R;
  // summed-area table of the inside mask
  std::vector<int64_t> S((size_t)(nx + 1) * (ny + 1), 0);
  for (int j = 0; j < ny; ++j) {
    int64_t run = 0;
    std::vector<uint8_t> row(nx, 0);
    for (int k = p->row_iv_off[j]; k < p->row_iv_off[j + 1]; ++k)
      for (int i = p->row_iv[2 * k]; i <= p->row_iv[2 * k + 1]; ++i) row[i] = 1;
    for (int i = 0; i < nx; ++i) {
      run += row[i];
      S[(size_t)(j + 1) * (nx + 1) + i + 1] = S[(size_t)j * (nx + 1) + i + 1] + run;
    }
  }
  auto inside_square = [&](int cj, int ci) {
    const int j0 = cj - a, j1 = cj + a + 1, i0 = ci - a, i1 = ci + a + 1;
    if (j0 < 0 || i0 < 0 || j1 > ny || i1 > nx) return false;
    const int64_t v = S[(size_t)j1 * (nx + 1) + i1] - S[(size_t)j0 * (nx + 1) + i1] -
                      S[(size_t)j1 * (nx + 1) + i0] + S[(size_t)j0 * (nx + 1) + i0];
    return v == (int64_t)(2 * a + 1) * (2 * a + 1);
  };
  const std::vector<int32_t>& q = band.iface_lin;  // ascending
  const int n = (int)q.size();
  std::vector<int32_t> qj(n), qi(n), owner(n, -1);
  for (int t = 0; t < n; ++t) {
    qj[t] = q[t] / nx;
    qi[t] = q[t] % nx;
  }
  // interface points by row, for the neighbourhood queries
  std::vector<std::vector<int32_t>> by_row(ny);
  for (int t = 0; t < n; ++t) by_row[qj[t]].push_back(t);
  std::vector<std::vector<int32_t>> served;
  for (int t = 0; t < n; ++t) {
    if (owner[t] >= 0) continue;
    std::vector<int32_t> loc;
    for (int j = std::max(0, qj[t] - 2 * R); j <= std::min(ny - 1, qj[t] + 2 * R); ++j)
      for (int32_t u : by_row[j])
        if (std::abs(qi[u] - qi[t]) <= 2 * R) loc.push_back(u);
    bool found = false;
    int best_score = -1, bj = 0, bi = 0;
    for (int dj = -R; dj <= R; ++dj)
      for (int di = -R; di <= R; ++di) {
        const int cj = qj[t] + dj, ci = qi[t] + di;
        if (!inside_square(cj, ci)) continue;
        int score = 0;
        for (int32_t u : loc)
          if (owner[u] < 0 && std::abs(qj[u] - cj) <= R && std::abs(qi[u] - ci) <= R) ++score;
        if (!found || score > best_score || (score == best_score && (cj < bj || (cj == bj && ci < bi)))) {
          found = true;
          best_score = score;
          bj = cj;
          bi = ci;
        }
      }
    if (!found)
      return set_error(FC2D_ERR_GEOMETRY,
                       "small squares: no square inside the domain serves an interface point "
                       "(the domain is too narrow or too curved for 37-point squares)");
    std::vector<int32_t> mine;
    for (int32_t u : loc)
      if (owner[u] < 0 && std::abs(qj[u] - bj) <= R && std::abs(qi[u] - bi) <= R) {
        owner[u] = (int32_t)served.size();
        mine.push_back(u);
      }
    std::sort(mine.begin(), mine.end());
    served.push_back(mine);
    out.origin_j.push_back(bj - a);
    out.origin_i.push_back(bi - a);
  }
  out.served_off.assign(1, 0);
  for (size_t k = 0; k < served.size(); ++k) {
    for (int32_t u : served[k]) {
      out.served_lin.push_back(q[u]);
      out.served_local.push_back((qj[u] - out.origin_j[k]) * kSqP + (qi[u] - out.origin_i[k]));
    }
    out.served_off.push_back((int32_t)out.served_lin.size());
  }
  // the coarse continuation matrix A: the refined one at every n_r-th fine point
  out.A.assign((size_t)C * d, 0.0);
  for (int k = 0; k < C; ++k)
    for (int j = 0; j < d; ++j) out.A[(size_t)k * d + j] = p->Ar[(size_t)((k + 1) * n_r - 1) * d + j];
  out.Q = p->Q;
  return FC2D_OK;
}

}  // namespace fc2d
