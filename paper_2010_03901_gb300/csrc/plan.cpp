// fc2d_plan: the geometrical setup of the 2D-FC method (Section 3.5, steps 1-4) and
// the FC matrices (Section 2.2, Remark 2.2).  Host C++; the only GPU work is the
// Newton foot search (foot_newton_gpu, in extend.cu).
//
// Compiled with -ffp-contract=off: the double-double error terms and the grid
// coordinates x_i = a0 + h*i must be evaluated exactly as written.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "dd.h"
#include "fc2d_kernels.cuh"
#include "plan_internal.h"

namespace fc2d {

static thread_local std::string g_last_error;

fc2d_status set_error(fc2d_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

fc2d_status cuda_check(int err, const char* what) {
  if (err == 0) return FC2D_OK;
  return set_error(FC2D_ERR_CUDA, std::string(what) + ": " +
                                      cudaGetErrorString(static_cast<cudaError_t>(err)));
}

// ------------------------------------------------------------------------- //
// Double-double cos/sin of the rational turn 2 pi num/den
// ------------------------------------------------------------------------- //
static void dd_cos_sin_small(dd x, dd& c, dd& s) {
  // Taylor series, |x| <= pi/4
  dd x2 = x * x;
  dd tc(1.0), ts = x;
  c = dd(1.0);
  s = x;
  for (int k = 2; k < 80; k += 2) {
    tc = -(tc * x2) / dd(double((k - 1) * k));
    ts = -(ts * x2) / dd(double(k * (k + 1)));
    c += tc;
    s += ts;
    if (std::fabs(tc.hi) < 1e-34 && std::fabs(ts.hi) < 1e-34) break;
  }
}

static void dd_cos_sin_turn(long long num, long long den, dd& c, dd& s) {
  long long r = ((num % den) + den) % den;
  long long o = (8 * r) / den;  // octant
  dd phi = dd(2.0) * dd_pi() * (dd(double(8 * r - o * den)) / dd(double(8 * den)));
  dd cp, sp;
  dd_cos_sin_small(phi, cp, sp);
  dd h = dd_sqrt(dd(2.0)) * dd(0.5);
  dd cb, sb;
  switch (o % 8) {
    case 0: cb = dd(1.0); sb = dd(0.0); break;
    case 1: cb = h; sb = h; break;
    case 2: cb = dd(0.0); sb = dd(1.0); break;
    case 3: cb = -h; sb = h; break;
    case 4: cb = dd(-1.0); sb = dd(0.0); break;
    case 5: cb = -h; sb = -h; break;
    case 6: cb = dd(0.0); sb = dd(-1.0); break;
    default: cb = h; sb = -h; break;
  }
  c = cb * cp - sb * sp;
  s = sb * cp + cb * sp;
}

// ------------------------------------------------------------------------- //
// FC matrices (Section 2.2): Gram QR, oversampled Gram values, least-squares trig
// fit (Householder QR in double-double), A_r
// ------------------------------------------------------------------------- //
static void fc_matrices(int d, int C, int Z, int n_os, int n_r, int m_F,
                        std::vector<double>& Qout, std::vector<double>& Arout) {
  const int Per = d + 2 * C + Z - 1;
  // modified Gram-Schmidt on P = (i^j)
  std::vector<dd> Qc(d * d), R(d * d, dd(0.0));  // Qc column-major: Qc[j*d + i]
  for (int j = 0; j < d; ++j) {
    std::vector<dd> v(d);
    for (int i = 0; i < d; ++i) {
      dd p(1.0);
      for (int e = 0; e < j; ++e) p = p * dd(double(i));
      v[i] = p;
    }
    for (int k = 0; k < j; ++k) {
      dd r(0.0);
      for (int i = 0; i < d; ++i) r += Qc[k * d + i] * v[i];
      R[k * d + j] = r;
      for (int i = 0; i < d; ++i) v[i] -= r * Qc[k * d + i];
    }
    dd nrm(0.0);
    for (int i = 0; i < d; ++i) nrm += v[i] * v[i];
    nrm = dd_sqrt(nrm);
    R[j * d + j] = nrm;
    for (int i = 0; i < d; ++i) Qc[j * d + i] = v[i] / nrm;
  }
  // oversampled Gram values Q_os = P_os R^{-1}: rows x = i/n_os
  const int nfine = n_os * (d - 1) + 1;
  std::vector<dd> Qos(nfine * d);
  for (int i = 0; i < nfine; ++i) {
    dd x = dd(double(i)) / dd(double(n_os));
    std::vector<dd> prow(d);
    dd pw(1.0);
    for (int j = 0; j < d; ++j) {
      prow[j] = pw;
      pw = pw * x;
    }
    for (int j = 0; j < d; ++j) {
      dd s = prow[j];
      for (int k = 0; k < j; ++k) s -= Qos[i * d + k] * R[k * d + j];
      Qos[i * d + j] = s / R[j * d + j];
    }
  }
  // least-squares matrix: rows = fit points (units of 1/n_os), columns = real trig basis
  std::vector<long long> fit;
  for (int i = 0; i <= n_os * (d - 1); ++i) fit.push_back(i);
  for (int i = n_os * (d + C); i <= n_os * (d + C + Z - 1); ++i) fit.push_back(i);
  const int m = (int)fit.size();
  const int nb = 2 * m_F + 1;
  const long long den = (long long)n_os * Per;
  std::vector<dd> Bm((size_t)m * nb);  // row-major
  for (int r = 0; r < m; ++r) {
    Bm[(size_t)r * nb] = dd(1.0);
    for (int k = 1; k <= m_F; ++k) {
      dd c, s;
      dd_cos_sin_turn(k * fit[r], den, c, s);
      Bm[(size_t)r * nb + 2 * k - 1] = c;
      Bm[(size_t)r * nb + 2 * k] = s;
    }
  }
  // right-hand sides: column j of Q_os on the matching points, zero elsewhere
  std::vector<dd> rhs((size_t)m * d, dd(0.0));
  for (int i = 0; i < nfine; ++i)
    for (int j = 0; j < d; ++j) rhs[(size_t)i * d + j] = Qos[i * d + j];
  // Householder QR, applied to the right-hand sides as it goes
  for (int k = 0; k < nb; ++k) {
    dd alpha(0.0);
    for (int i = k; i < m; ++i) alpha += Bm[(size_t)i * nb + k] * Bm[(size_t)i * nb + k];
    alpha = dd_sqrt(alpha);
    if (Bm[(size_t)k * nb + k].hi > 0) alpha = -alpha;
    std::vector<dd> v(m - k);
    for (int i = k; i < m; ++i) v[i - k] = Bm[(size_t)i * nb + k];
    v[0] -= alpha;
    dd vv(0.0);
    for (auto& t : v) vv += t * t;
    dd beta = dd(2.0) / vv;
    for (int j = k; j < nb; ++j) {
      dd s(0.0);
      for (int i = k; i < m; ++i) s += v[i - k] * Bm[(size_t)i * nb + j];
      s = s * beta;
      for (int i = k; i < m; ++i) Bm[(size_t)i * nb + j] -= s * v[i - k];
    }
    for (int j = 0; j < d; ++j) {
      dd s(0.0);
      for (int i = k; i < m; ++i) s += v[i - k] * rhs[(size_t)i * d + j];
      s = s * beta;
      for (int i = k; i < m; ++i) rhs[(size_t)i * d + j] -= s * v[i - k];
    }
  }
  // back substitution R a = (Q^T b)[0:nb]
  std::vector<dd> a((size_t)nb * d);
  for (int j = 0; j < d; ++j)
    for (int r = nb - 1; r >= 0; --r) {
      dd s = rhs[(size_t)r * d + j];
      for (int c = r + 1; c < nb; ++c) s -= Bm[(size_t)r * nb + c] * a[(size_t)c * d + j];
      a[(size_t)r * d + j] = s / Bm[(size_t)r * nb + r];
    }
  // A_r[q-1][j] = g^c_j((d-1) + q/n_r), q = 1..C n_r
  const int Cr = C * n_r;
  Arout.assign((size_t)Cr * d, 0.0);
  for (int q = 1; q <= Cr; ++q) {
    long long num = (long long)(d - 1) * n_r + q;  // x = num/n_r
    std::vector<dd> row(nb);
    row[0] = dd(1.0);
    for (int k = 1; k <= m_F; ++k) {
      dd c, s;
      dd_cos_sin_turn(k * num, (long long)n_r * Per, c, s);
      row[2 * k - 1] = c;
      row[2 * k] = s;
    }
    for (int j = 0; j < d; ++j) {
      dd g(0.0);
      for (int l = 0; l < nb; ++l) g += row[l] * a[(size_t)l * d + j];
      Arout[(size_t)(q - 1) * d + j] = to_double(g);
    }
  }
  Qout.assign((size_t)d * d, 0.0);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) Qout[(size_t)i * d + j] = to_double(Qc[j * d + i]);
}

// ------------------------------------------------------------------------- //
// Curve
// ------------------------------------------------------------------------- //
void Curve::eval(double t, double& x, double& y) const { eval_d(t, 0, x, y); }

void Curve::eval_d(double t, int der, double& x, double& y) const {
  x = 0.0;
  y = 0.0;
  for (size_t k = 0; k < cx.size(); ++k) {
    if (cx[k] == 0.0 && sx[k] == 0.0 && cy[k] == 0.0 && sy[k] == 0.0) continue;
    double kt = double(k) * t;
    double c = std::cos(kt), s = std::sin(kt);
    double kk = double(k);
    switch (der) {
      case 0:
        x += cx[k] * c + sx[k] * s;
        y += cy[k] * c + sy[k] * s;
        break;
      case 1:
        x += kk * (-cx[k] * s + sx[k] * c);
        y += kk * (-cy[k] * s + sy[k] * c);
        break;
      default:
        x -= kk * kk * (cx[k] * c + sx[k] * s);
        y -= kk * kk * (cy[k] * c + sy[k] * s);
        break;
    }
  }
}

// Root of the periodic function v(t) - value in [t0, t1] (a sign change bracket) by
// Newton's method safeguarded with bisection.  which = 0: x(t), 1: y(t).
static double bracket_root(const Curve& c, int which, double value, double t0, double t1) {
  auto f = [&](double t, double& df) {
    double x, y, xd, yd;
    c.eval(t, x, y);
    c.eval_d(t, 1, xd, yd);
    df = which == 0 ? xd : yd;
    return (which == 0 ? x : y) - value;
  };
  double d0;
  double f0 = f(t0, d0);
  bool pos0 = f0 > 0;
  double lo = t0, hi = t1;
  double t = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    double df;
    double ft = f(t, df);
    if ((ft > 0) == pos0) lo = t; else hi = t;
    double tn = (df != 0.0) ? t - ft / df : 0.5 * (lo + hi);
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    if (std::fabs(tn - t) <= 4e-16 * (1.0 + std::fabs(t)) || hi - lo <= 4e-16 * (1.0 + std::fabs(t))) {
      t = tn;
      break;
    }
    t = tn;
  }
  return t;
}

// Crossings of the curve with every grid row (which = 1: y(t) = y_j, returns x's)
// or column (which = 0: x(t) = x_i, returns y's), sorted, by sign changes on n_s + 1
// uniform samples t_s = (2 pi s)/n_s.
static void line_crossings(const Curve& c, int which, int nlines, double o, double h,
                           int n_s, double tol, std::vector<std::vector<double>>& out) {
  out.assign(nlines, {});
  std::vector<double> v(n_s + 1), ts(n_s + 1);
  const double two_pi = 2.0 * M_PI;
  for (int s = 0; s < n_s; ++s) {
    ts[s] = two_pi * s / n_s;
    double x, y;
    c.eval(ts[s], x, y);
    v[s] = which == 0 ? x : y;
  }
  // the curve is closed: the sample at 2 pi is the sample at 0 (evaluated at 2 pi it
  // could round differently and hide a crossing at theta = 0 between the two)
  ts[n_s] = two_pi;
  v[n_s] = v[0];
  for (int s = 0; s < n_s; ++s) {
    double lo = std::min(v[s], v[s + 1]), hi = std::max(v[s], v[s + 1]);
    if (lo == hi) continue;
    // lines with lo <= c_l < hi change sign ((v - c_l > 0) differs at the ends)
    long long l0 = (long long)std::ceil((lo - o) / h) - 1;
    long long l1 = (long long)std::floor((hi - o) / h) + 1;
    for (long long l = std::max(0LL, l0); l <= std::min((long long)nlines - 1, l1); ++l) {
      double cl = o + h * double(l);
      bool p0 = v[s] - cl > 0, p1 = v[s + 1] - cl > 0;
      if (p0 == p1) continue;
      double t = bracket_root(c, which, cl, ts[s], ts[s + 1]);
      double x, y;
      c.eval(t, x, y);
      out[l].push_back(which == 0 ? y : x);
    }
  }
  // sort; drop pairs of consecutive crossings closer than tol (a line touching the
  // curve, seen as two roots when a sample lands on the touching point)
  for (auto& r : out) {
    std::sort(r.begin(), r.end());
    std::vector<double> kept;
    for (double x : r) {
      if (!kept.empty() && x - kept.back() < tol)
        kept.pop_back();
      else
        kept.push_back(x);
    }
    r.swap(kept);
  }
}

// ------------------------------------------------------------------------- //
// FFT axis setup
// ------------------------------------------------------------------------- //
static bool fft_axis(int n, FftAxis& ax) {
  ax.n = n;
  ax.n_radix = 0;
  int m = n;
  while (m % 5 == 0) { ax.radix[ax.n_radix++] = 5; m /= 5; }
  while (m % 3 == 0) { ax.radix[ax.n_radix++] = 3; m /= 3; }
  while (m % 8 == 0) { ax.radix[ax.n_radix++] = 8; m /= 8; }
  while (m % 4 == 0) { ax.radix[ax.n_radix++] = 4; m /= 4; }
  while (m % 2 == 0) { ax.radix[ax.n_radix++] = 2; m /= 2; }
  if (m != 1 || ax.n_radix > kMaxRadices) return false;
  ax.tw_host.assign(2 * (size_t)n, 0.0);
  for (int t = 0; t < n; ++t) {
    dd c, s;
    dd_cos_sin_turn(-(long long)t, n, c, s);
    ax.tw_host[2 * t] = to_double(c);
    ax.tw_host[2 * t + 1] = to_double(s);
  }
  return true;
}

// Twiddles of each Stockham stage after the first, for a power-of-two length N and
// radices min(E, N/Ns): block s holds w^(r k N/(Ns R)), r < R, k < Ns, stored [r][k], so
// that the lanes of a warp (consecutive k) read consecutive entries.
static std::vector<double> stage_twiddles(const FftAxis& ax, int E) {
  std::vector<double> out;
  const int N = ax.n;
  if (N <= 0 || (N & (N - 1))) return out;
  for (int ns = 1; ns < N;) {
    const int R = (N / ns >= E) ? E : N / ns;
    if (ns > 1)
      for (int r = 0; r < R; ++r)
        for (int k = 0; k < ns; ++k) {
          const long long t = ((long long)r * k * (N / (ns * R))) % N;
          out.push_back(ax.tw_host[2 * t]);
          out.push_back(ax.tw_host[2 * t + 1]);
        }
    ns *= R;
  }
  return out;
}

// ------------------------------------------------------------------------- //
// Lagrange weights
// ------------------------------------------------------------------------- //
static void lagrange(const double* nodes, int n, double t, double* w) {
  for (int k = 0; k < n; ++k) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != k) v *= (t - nodes[m]) / (nodes[k] - nodes[m]);
    w[k] = v;
  }
}

}  // namespace fc2d

using namespace fc2d;

namespace {

template <typename T>
fc2d_status upload(T** dst, const std::vector<T>& src) {
  size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  if (cudaMalloc((void**)dst, bytes) != cudaSuccess)
    return set_error(FC2D_ERR_NOMEM, "cudaMalloc of a plan table failed");
  if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T),
                                 cudaMemcpyHostToDevice) != cudaSuccess)
    return set_error(FC2D_ERR_CUDA, "cudaMemcpy of a plan table failed");
  return FC2D_OK;
}

struct Cand {
  int32_t lin;
  double seed;
};

}  // namespace

// Ownership ranges of the blend + interpolation CTAs: consecutive normal ranges
// [start_c, start_{c+1}) of at most `cap` normals covering 0..B-1, with at most n_cta
// ranges, such that the largest number of strip points owned by one range is as small
// as possible (binary search on that number; for a given bound, taking as many normals
// as fit into each range in turn uses the fewest ranges).  cnt[p]: points per normal.
static std::vector<int32_t> partition_owners(const std::vector<int64_t>& cnt, int cap, int n_cta) {
  const int B = (int)cnt.size();
  auto greedy = [&](int64_t T, std::vector<int32_t>* start) {
    int parts = 0, owned = 0;
    int64_t run = 0;
    if (start) start->assign(1, 0);
    for (int p = 0; p < B; ++p) {
      if (owned == cap || (owned > 0 && run + cnt[p] > T)) {
        ++parts;
        if (start) start->push_back(p);
        run = 0;
        owned = 0;
      }
      run += cnt[p];
      ++owned;
    }
    ++parts;
    if (start) start->push_back(B);
    return parts;
  };
  int64_t lo = 0, hi = 0;
  for (int64_t v : cnt) {
    lo = std::max(lo, v);
    hi += v;
  }
  lo = std::max(lo, (hi + n_cta - 1) / n_cta);
  hi = std::max(hi, lo);
  while (lo < hi) {  // smallest bound whose greedy partition uses <= n_cta ranges
    const int64_t mid = lo + (hi - lo) / 2;
    if (greedy(mid, nullptr) <= n_cta) hi = mid;
    else lo = mid + 1;
  }
  std::vector<int32_t> start;
  greedy(lo, &start);
  return start;
}

// Strip points grouped by the blend CTA that interpolates them (mixed form, M = 8):
// CTA c of a function computes the kTcComputed normals from start_c on (mod B) and owns
// the strip points whose first normal pb lies in [start_c, start_{c+1}), at most
// kTcOwned normals, so that pb .. pb + M - 1 are among its normals.  Two partitions:
// one CTA per SM where B allows ~48 normals each (a call of few functions then fills
// the SMs once, with the ranges balanced by their numbers of points), and the fewest
// CTAs, ceil(B / kTcOwned) (for calls of many functions, whose CTAs fill the SMs anyway
// and where extra CTAs only repeat gathers).  Within a CTA the points are ordered by
// first normal, then fine node; the weights are reordered to match.
static fc2d_status owner_set(fc2d_plan_s* p, const std::vector<int32_t>& pb,
                             const std::vector<int32_t>& sb, const std::vector<float>& w,
                             const std::vector<int64_t>& cnt, int n_cta, int M,
                             DeviceTables::Owners& out) {
  const int B = p->prm.B, ns = (int)pb.size();
  const std::vector<int32_t> start = partition_owners(cnt, kTcOwned, n_cta);
  const int n_own = (int)start.size() - 1;
  std::vector<int32_t> cta_of(B);
  for (int c = 0; c < n_own; ++c)
    for (int q = start[c]; q < start[c + 1]; ++q) cta_of[q] = c;
  std::vector<int32_t> off(n_own + 1, 0);
  for (int k = 0; k < ns; ++k) ++off[cta_of[pb[k]] + 1];
  for (int c = 0; c < n_own; ++c) off[c + 1] += off[c];
  std::vector<int32_t> fill(off.begin(), off.end() - 1), perm(ns), pack(ns);
  for (int k = 0; k < ns; ++k) {
    const int c = cta_of[pb[k]], idx = fill[c]++;
    perm[idx] = k;
    pack[idx] = (pb[k] - start[c]) | (sb[k] << 8);
  }
  // within a CTA, order the points by first normal, then first fine node: neighbouring
  // lanes then read the same or adjacent rows of the shared-memory tile
  for (int c = 0; c < n_own; ++c) {
    std::vector<int32_t> ord(off[c + 1] - off[c]);
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = off[c] + (int32_t)i;
    auto key = [&](int32_t i) { return (pack[i] & 0xFF) * 256 + (pack[i] >> 8); };
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return key(x) < key(y); });
    std::vector<int32_t> pk(ord.size()), pm(ord.size());
    for (size_t i = 0; i < ord.size(); ++i) {
      pk[i] = pack[ord[i]];
      pm[i] = perm[ord[i]];
    }
    std::copy(pk.begin(), pk.end(), pack.begin() + off[c]);
    std::copy(pm.begin(), pm.end(), perm.begin() + off[c]);
  }
  std::vector<float> wp(w.size());
  for (int idx = 0; idx < ns; ++idx)
    for (int b = 0; b < 2 * M; ++b) wp[(size_t)b * ns + idx] = w[(size_t)b * ns + perm[idx]];
  out.n = n_own;
  out.off_host = off;
  fc2d_status st;
  if ((st = upload(&out.off, off)) || (st = upload(&out.k, perm)) ||
      (st = upload(&out.pack, pack)) || (st = upload(&out.w, wp)) ||
      (st = upload(&out.start, start)))
    return st;
  return FC2D_OK;
}

static fc2d_status owner_tables(fc2d_plan_s* p, int ns, int M) {
  const int B = p->prm.B;
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
    n_sm = 0;
  p->n_sm = n_sm;
  const int n_min = (B + kTcOwned - 1) / kTcOwned;
  const int n_wide = std::max(n_min, std::min(n_sm, B / 48));
  std::vector<int32_t> pb(ns), sb(ns);
  std::vector<float> w((size_t)2 * M * ns);
  if (cudaMemcpy(pb.data(), p->dev.s_pb, (size_t)ns * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(sb.data(), p->dev.s_sb, (size_t)ns * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(w.data(), p->dev.s_w, w.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return set_error(FC2D_ERR_CUDA, "reading the interpolation tables back failed");
  std::vector<int64_t> cnt(B, 0);
  for (int k = 0; k < ns; ++k) {
    pb[k] = ((pb[k] % B) + B) % B;  // the first normal is stored unreduced near theta = 0
    if (sb[k] < 0 || sb[k] > 255)
      return set_error(FC2D_ERR_GEOMETRY, "interpolation node index out of range");
    ++cnt[pb[k]];
  }
  fc2d_status st = owner_set(p, pb, sb, w, cnt, n_wide, M, p->dev.own[0]);
  if (!st && n_wide > n_min) st = owner_set(p, pb, sb, w, cnt, n_min, M, p->dev.own[1]);
  return st;
}

extern "C" fc2d_status fc2d_plan(const fc2d_boundary* boundary, const fc2d_grid* grid,
                                 const fc2d_params* params, fc2d_plan_t* out) {
  if (!boundary || !grid || !out || boundary->n_modes < 2 || !boundary->cx ||
      !boundary->sx || !boundary->cy || !boundary->sy)
    return set_error(FC2D_ERR_ARG, "fc2d_plan: null or empty boundary/grid/out");
  *out = nullptr;
  fc2d_params P{};
  if (params) P = *params;
  if (grid->h <= 0 || grid->nx < 8 || grid->ny < 8)
    return set_error(FC2D_ERR_ARG, "fc2d_plan: grid needs h > 0 and nx, ny >= 8");
  if (grid->nx % 2 != 0)
    return set_error(FC2D_ERR_UNSUPPORTED, "fc2d_plan: nx must be even (real-to-complex DFT)");
  if (!P.d) P.d = 5;
  if (!P.C) P.C = 27;
  if (!P.Z) P.Z = 12;
  if (!P.n_os) P.n_os = 20;
  if (!P.n_r) P.n_r = 6;
  if (!P.M) P.M = P.d + 3;
  if (!P.m_F) P.m_F = 20;
  if (!P.B) P.B = (int)std::lround(2.0 * M_PI / grid->h);
  if (P.k1 <= 0) P.k1 = grid->h;
  if (P.d < 2 || P.d > 12 || P.C < 2 || P.Z < 2 || P.n_os < 1 || P.n_r < 1 || P.M < 2 ||
      P.M > kMaxM || P.B < P.M || P.m_F < 1 || P.M > P.C * P.n_r + 1 ||
      (P.precision != FC2D_FP64 && P.precision != FC2D_MIXED))
    return set_error(FC2D_ERR_ARG, "fc2d_plan: parameter out of range");
  if (P.precision == FC2D_MIXED && P.d > 8)
    return set_error(FC2D_ERR_UNSUPPORTED, "fc2d_plan: the mixed contraction handles d <= 8");

  auto* p = new fc2d_plan_s();
  auto fail = [&](fc2d_status s) {
    fc2d_destroy(p);
    return s;
  };
  cudaGetDevice(&p->device);
  p->grid = *grid;
  p->prm = P;
  p->Cr = P.C * P.n_r;
  const int nx = grid->nx, ny = grid->ny, B = P.B, M = P.M, d = P.d;
  const double a0 = grid->a0, b0 = grid->b0, h = grid->h, k1 = P.k1;

  // boundary, oriented counter-clockwise (signed area > 0)
  Curve& cv = p->curve;
  int nm = boundary->n_modes;
  cv.cx.assign(boundary->cx, boundary->cx + nm);
  cv.sx.assign(boundary->sx, boundary->sx + nm);
  cv.cy.assign(boundary->cy, boundary->cy + nm);
  cv.sy.assign(boundary->sy, boundary->sy + nm);
  double area = 0;
  for (int k = 0; k < nm; ++k) area += k * (cv.cx[k] * cv.sy[k] - cv.sx[k] * cv.cy[k]);
  if (area == 0) return fail(set_error(FC2D_ERR_GEOMETRY, "fc2d_plan: degenerate curve"));
  if (area < 0)
    for (int k = 0; k < nm; ++k) {
      cv.sx[k] = -cv.sx[k];
      cv.sy[k] = -cv.sy[k];
    }

  // FC matrices (Section 2.2, Remark 2.2)
  fc_matrices(d, P.C, P.Z, P.n_os, P.n_r, P.m_F, p->Q, p->Ar);

  // crossings of grid rows and columns with the curve
  const int n_s = 16 * B;
  std::vector<std::vector<double>> rowc, colc;
  const double tang_tol = 1e-7 * std::max(nx, ny) * h;
  line_crossings(cv, 1, ny, b0, h, n_s, tang_tol, rowc);
  line_crossings(cv, 0, nx, a0, h, n_s, tang_tol, colc);
  for (int j = 0; j < ny; ++j)
    if (rowc[j].size() % 2)
      return fail(set_error(FC2D_ERR_GEOMETRY,
                            "odd number of crossings of grid row " + std::to_string(j) +
                                " (y = " + std::to_string(b0 + h * j) + ") with the curve: " +
                                std::to_string(rowc[j].size())));
  for (int i = 0; i < nx; ++i)
    if (colc[i].size() % 2)
      return fail(set_error(FC2D_ERR_GEOMETRY,
                            "odd number of crossings of grid column " + std::to_string(i) +
                                " (x = " + std::to_string(a0 + h * i) + ") with the curve: " +
                                std::to_string(colc[i].size())));
  std::vector<double> xs(nx), ys(ny);
  for (int i = 0; i < nx; ++i) xs[i] = a0 + h * double(i);
  for (int j = 0; j < ny; ++j) ys[j] = b0 + h * double(j);

  // inside intervals per row: x_i in [X_2m, X_2m+1]
  p->row_iv_off.assign(ny + 1, 0);
  std::vector<uint8_t> inside((size_t)nx * ny, 0);
  for (int j = 0; j < ny; ++j) {
    p->row_iv_off[j] = (int32_t)(p->row_iv.size() / 2);
    const auto& X = rowc[j];
    for (size_t m = 0; m + 1 < X.size(); m += 2) {
      int il = std::max(0, (int)std::ceil((X[m] - a0) / h) - 1);
      while (il < nx && xs[il] < X[m]) ++il;
      int ih = std::min(nx - 1, (int)std::floor((X[m + 1] - a0) / h) + 1);
      while (ih >= 0 && xs[ih] > X[m + 1]) --ih;
      if (il > ih) continue;
      p->row_iv.push_back(il);
      p->row_iv.push_back(ih);
      for (int i = il; i <= ih; ++i) inside[(size_t)j * nx + i] = 1;
      p->n_inside += ih - il + 1;
    }
  }
  p->row_iv_off[ny] = (int32_t)(p->row_iv.size() / 2);
  {
    int64_t off = 0;
    p->row_iv_coff.resize(p->row_iv.size() / 2);
    for (size_t k = 0; k < p->row_iv_coff.size(); ++k) {
      p->row_iv_coff[k] = (int32_t)off;
      off += p->row_iv[2 * k + 1] - p->row_iv[2 * k] + 1;
    }
  }

  // boundary nodes and normals (eq. (3.4))
  std::vector<double> bx(B), by(B), bnx(B), bny(B), th(B);
  for (int k = 0; k < B; ++k) {
    th[k] = 2.0 * M_PI * k / B;
    cv.eval(th[k], bx[k], by[k]);
    double xd, yd;
    cv.eval_d(th[k], 1, xd, yd);
    double s = std::hypot(xd, yd);
    bnx[k] = yd / s;
    bny[k] = -xd / s;
  }

  // strip candidates: grid points in the quadrilaterals between consecutive normals,
  // widened by h/2, out to distance C k1 + h
  const double W = P.C * k1 + h;
  const double k2 = 2.0 * M_PI / B;
  std::vector<Cand> cand;
  for (int k = 0; k < B; ++k) {
    int k1i = (k + 1) % B;
    double vx[4] = {bx[k], bx[k1i], bx[k1i] + W * bnx[k1i], bx[k] + W * bnx[k]};
    double vy[4] = {by[k], by[k1i], by[k1i] + W * bny[k1i], by[k] + W * bny[k]};
    double xmin = *std::min_element(vx, vx + 4) - h, xmax = *std::max_element(vx, vx + 4) + h;
    double ymin = *std::min_element(vy, vy + 4) - h, ymax = *std::max_element(vy, vy + 4) + h;
    int i0 = std::max(0, (int)std::floor((xmin - a0) / h));
    int i1 = std::min(nx - 1, (int)std::ceil((xmax - a0) / h));
    int j0 = std::max(0, (int)std::floor((ymin - b0) / h));
    int j1 = std::min(ny - 1, (int)std::ceil((ymax - b0) / h));
    // orientation of the quad (counter-clockwise for an outward strip of a CCW curve)
    double sarea = 0;
    for (int e = 0; e < 4; ++e)
      sarea += vx[e] * vy[(e + 1) % 4] - vx[(e + 1) % 4] * vy[e];
    double sg = sarea >= 0 ? 1.0 : -1.0;
    for (int j = j0; j <= j1; ++j)
      for (int i = i0; i <= i1; ++i) {
        if (inside[(size_t)j * nx + i]) continue;
        bool ok = true;
        for (int e = 0; e < 4 && ok; ++e) {
          double ex = vx[(e + 1) % 4] - vx[e], ey = vy[(e + 1) % 4] - vy[e];
          double len = std::hypot(ex, ey);
          if (len == 0) continue;
          double cr = sg * (ex * (ys[j] - vy[e]) - ey * (xs[i] - vx[e])) / len;
          if (cr < -0.5 * h) ok = false;
        }
        if (ok) cand.push_back({j * nx + i, th[k] + 0.5 * k2});
      }
  }
  std::sort(cand.begin(), cand.end(),
            [](const Cand& a, const Cand& b) { return a.lin < b.lin; });
  cand.erase(std::unique(cand.begin(), cand.end(),
                         [](const Cand& a, const Cand& b) { return a.lin == b.lin; }),
             cand.end());
  std::vector<double> qx(cand.size()), qy(cand.size()), tq(cand.size());
  for (size_t n = 0; n < cand.size(); ++n) {
    qx[n] = xs[cand[n].lin % nx];
    qy[n] = ys[cand[n].lin / nx];
    tq[n] = cand[n].seed;
  }
  std::vector<int> conv;
  fc2d_status st = foot_newton_gpu(cv, qx, qy, tq, conv, 1.5 * k2);
  if (st != FC2D_OK) return fail(st);
  const double width = P.C * k1;
  const double two_pi = 2.0 * M_PI;
  p->row_strip_off.assign(ny + 1, 0);
  for (size_t n = 0; n < cand.size(); ++n) {
    double fx, fy;
    cv.eval(tq[n], fx, fy);
    double eta = std::hypot(qx[n] - fx, qy[n] - fy);
    if (!(eta > 0 && eta <= width)) continue;
    if (!conv[n])
      return fail(set_error(FC2D_ERR_NOT_CONVERGED, "Newton foot search did not converge"));
    double t = std::fmod(tq[n], two_pi);
    if (t < 0) t += two_pi;
    if (t >= two_pi) t = 0.0;
    p->strip_lin.push_back(cand[n].lin);
    p->strip_theta.push_back(t);
    p->strip_eta.push_back(eta);
  }
  // the strip must stay clear of the grid edge (its points are periodic neighbours)
  for (int32_t lin : p->strip_lin) {
    int i = lin % nx, j = lin / nx;
    if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1)
      return fail(set_error(FC2D_ERR_GEOMETRY, "the strip of width C*k1 reaches the grid edge"));
  }
  {
    size_t n = 0;
    for (int j = 0; j < ny; ++j) {
      p->row_strip_off[j] = (int32_t)n;
      while (n < p->strip_lin.size() && p->strip_lin[n] / nx == j) ++n;
    }
    p->row_strip_off[ny] = (int32_t)n;
  }

  // boundary data points: B nodes, column crossings, row crossings
  std::vector<int64_t> col_off(nx + 1), row_off(ny + 1);
  p->bdry_xy.clear();
  for (int k = 0; k < B; ++k) {
    p->bdry_xy.push_back(bx[k]);
    p->bdry_xy.push_back(by[k]);
  }
  int64_t off = B;
  for (int i = 0; i < nx; ++i) {
    col_off[i] = off;
    for (double y : colc[i]) {
      p->bdry_xy.push_back(xs[i]);
      p->bdry_xy.push_back(y);
    }
    off += (int64_t)colc[i].size();
  }
  col_off[nx] = off;
  for (int j = 0; j < ny; ++j) {
    row_off[j] = off;
    for (double x : rowc[j]) {
      p->bdry_xy.push_back(x);
      p->bdry_xy.push_back(ys[j]);
    }
    off += (int64_t)rowc[j].size();
  }
  row_off[ny] = off;
  p->n_bdry = off;
  p->col_off = col_off;
  p->row_off = row_off;

  // matching stencils (Section 3.2), with boundary data and (gidx_i, gw_i, wn_i) from
  // interior data only (Remark 3.2 II: stars from grid nodes alone, the foot value
  // extrapolated; wn_i has d rows and a zero weight on the boundary-datum slot)
  const int NS = M - 1;
  std::vector<int32_t> gidx((size_t)B * NS * M, 0), gidx_i((size_t)B * NS * M, 0);
  std::vector<double> gw((size_t)B * NS * M, 0.0), wn((size_t)B * (d - 1) * M, 0.0);
  std::vector<double> gw_i((size_t)B * NS * M, 0.0), wn_i((size_t)B * d * M, 0.0);
  const double tie = std::ldexp(1.0, -30), drop = 0.5;
  for (int k = 0; k < B; ++k) {
    bool vertical = std::fabs(bnx[k]) >= std::fabs(bny[k]) * (1.0 - tie);
    double base, nb, ob, on, o0;
    int nlines, nnodes;
    const std::vector<double>*line_c, *node_c;
    const std::vector<std::vector<double>>* cross;
    const std::vector<int64_t>* offs;
    if (vertical) {
      base = bx[k]; nb = bnx[k]; ob = by[k]; on = bny[k]; o0 = a0; nlines = nx; nnodes = ny;
      line_c = &xs; node_c = &ys; cross = &colc; offs = &col_off;
    } else {
      base = by[k]; nb = bny[k]; ob = bx[k]; on = bnx[k]; o0 = b0; nlines = ny; nnodes = nx;
      line_c = &ys; node_c = &xs; cross = &rowc; offs = &row_off;
    }
    int sigma = nb > 0 ? 1 : -1;
    double xi = (base - 0.5 * h * nb - o0) / h;
    long long i0 = sigma > 0 ? (long long)std::floor(xi) : (long long)std::ceil(xi);
    double tk[kMaxM];
    tk[0] = 0.0;
    for (int s = 0; s < NS; ++s) {
      long long li = i0 - (long long)sigma * s;
      if (li < 0 || li >= nlines)
        return fail(set_error(FC2D_ERR_GEOMETRY, "a matching stencil leaves the grid"));
      double t = ((*line_c)[li] - base) / nb;
      double star = ob + t * on;
      tk[s + 1] = t;
      const auto& cr = (*cross)[li];
      // inside interval of the line containing the red star
      int mpos = (int)(std::upper_bound(cr.begin(), cr.end(), star) - cr.begin()) - 1;
      if (mpos < 0 || mpos % 2 == 1 || mpos + 1 >= (int)cr.size())
        return fail(set_error(FC2D_ERR_GEOMETRY, "a red star lies outside the domain"));
      double lo = cr[mpos], hi = cr[mpos + 1];
      // nodes along the line start at the other axis origin
      double no = vertical ? b0 : a0;
      int jl = std::max(0, (int)std::ceil((lo - no) / h) - 1);
      int jh = std::min(nnodes - 1, (int)std::floor((hi - no) / h) + 1);
      while (jl <= jh && (*node_c)[jl] < lo) ++jl;
      while (jh >= jl && (*node_c)[jh] > hi) --jh;
      const size_t base_i = ((size_t)k * NS + s) * M;
      {
        // interior data only: the nodes of the inside interval, none dropped (a chord
        // without a node leaves the plan without the interior-only form)
        if (jl > jh) p->interior_ok = false;
        const int n = std::max(jh - jl + 1, 1);
        int s0 = 0, len = n;
        if (n > M) {
          int c = 0;
          for (int j = jl; j <= jh; ++j) c += ((*node_c)[j] <= star);
          s0 = std::min(std::max(c - (M + 1) / 2, 0), n - M);
          len = M;
        }
        double cn[kMaxM], w[kMaxM];
        const int jb = std::min(jl, nnodes - 1);
        for (int e = 0; e < len; ++e) cn[e] = (*node_c)[jb + s0 + e];
        lagrange(cn, len, star, w);
        for (int e = 0; e < M; ++e) {
          const int j = jb + s0 + (e < len ? e : 0);
          gidx_i[base_i + e] = vertical ? (int32_t)((int64_t)j * nx + li) : (int32_t)(li * (int64_t)nx + j);
          gw_i[base_i + e] = e < len ? w[e] : 0.0;
        }
      }
      if (jl <= jh && (*node_c)[jl] - lo < drop * h) ++jl;
      if (jl <= jh && hi - (*node_c)[jh] < drop * h) --jh;
      // candidates: lower square, nodes, upper square
      std::vector<double> cc;
      std::vector<int32_t> ci;
      cc.push_back(lo);
      ci.push_back((int32_t)(-1 - ((*offs)[li] + mpos)));
      for (int j = jl; j <= jh; ++j) {
        cc.push_back((*node_c)[j]);
        ci.push_back(vertical ? (int32_t)((int64_t)j * nx + li) : (int32_t)(li * (int64_t)nx + j));
      }
      cc.push_back(hi);
      ci.push_back((int32_t)(-1 - ((*offs)[li] + mpos + 1)));
      int n = (int)cc.size(), s0 = 0, len = n;
      if (n > M) {
        int c = 0;
        for (double v : cc) c += (v <= star);
        s0 = std::min(std::max(c - (M + 1) / 2, 0), n - M);
        len = M;
      }
      double w[kMaxM];
      lagrange(&cc[s0], len, star, w);
      for (int e = 0; e < M; ++e) {
        if (e < len) {
          gidx[base_i + e] = ci[s0 + e];
          gw[base_i + e] = w[e];
        } else {
          gidx[base_i + e] = ci[s0];
          gw[base_i + e] = 0.0;
        }
      }
    }
    for (int q = 0; q < d - 1; ++q) {
      double w[kMaxM];
      lagrange(tk, M, (q - d + 1) * k1, w);
      for (int e = 0; e < M; ++e) wn[((size_t)k * (d - 1) + q) * M + e] = w[e];
    }
    for (int q = 0; q < d; ++q) {
      double w[kMaxM];
      lagrange(tk + 1, M - 1, (q - d + 1) * k1, w);
      for (int e = 1; e < M; ++e) wn_i[((size_t)k * d + q) * M + e] = w[e - 1];
    }
  }

  // FFT axes
  if (!fft_axis(nx / 2, p->fx) || !fft_axis(ny, p->fy))
    return fail(set_error(FC2D_ERR_UNSUPPORTED, "fc2d_plan: nx/2 and ny must be 2^a 3^b 5^c"));
  p->rtw_host.assign(2 * (size_t)(nx / 2 + 1), 0.0);
  for (int t = 0; t <= nx / 2; ++t) {
    dd c, s;
    dd_cos_sin_turn(-(long long)t, nx, c, s);
    p->rtw_host[2 * t] = to_double(c);
    p->rtw_host[2 * t + 1] = to_double(s);
  }

  // upload
  std::vector<float> arh(p->Ar.size()), arl(p->Ar.size());
  for (size_t n = 0; n < p->Ar.size(); ++n) {
    // TF32 keeps 10 explicit significand bits: round the high part to 11 bits
    double v = p->Ar[n];
    int e;
    double m = std::frexp(v, &e);
    double hi = std::ldexp(std::nearbyint(std::ldexp(m, 11)), e - 11);
    arh[n] = (float)hi;
    arl[n] = (float)(v - hi);
  }
  std::vector<float> tw32x(p->fx.tw_host.begin(), p->fx.tw_host.end());
  std::vector<float> tw32y(p->fy.tw_host.begin(), p->fy.tw_host.end());
  // FP32: the table, then the same halved (exactly) for the row kernel's split
  std::vector<float> rtw32(p->rtw_host.begin(), p->rtw_host.end());
  for (size_t k = 0, n = p->rtw_host.size(); k < n; ++k) rtw32.push_back(0.5f * rtw32[k]);
  std::vector<double> tsx64 = stage_twiddles(p->fx, 8), tsy64 = stage_twiddles(p->fy, 8);
  std::vector<double> tsx16 = stage_twiddles(p->fx, 16), tsy16 = stage_twiddles(p->fy, 16);
  std::vector<float> tsx32(tsx16.begin(), tsx16.end()), tsy32(tsy16.begin(), tsy16.end());
  std::vector<int> zero_status(1, 0);
  // the stencil taps as compact indices (every grid tap is an inside point); the
  // compact form is offered when the inside points have int32 indices
  const bool compact = p->n_inside < ((int64_t)1 << 31);
  auto to_compact = [&](const std::vector<int32_t>& gi, std::vector<int32_t>& gc) {
    gc.assign(compact ? gi.size() : 0, 0);
    for (size_t e = 0; e < gc.size(); ++e) {
      const int32_t id = gi[e];
      if (id < 0) {
        gc[e] = id;
        continue;
      }
      const int jr = id / nx, ic = id - jr * nx;
      int32_t c = -1;
      for (int k = p->row_iv_off[jr]; k < p->row_iv_off[jr + 1]; ++k)
        if (ic >= p->row_iv[2 * k] && ic <= p->row_iv[2 * k + 1])
          c = p->row_iv_coff[k] + (ic - p->row_iv[2 * k]);
      if (c < 0) return false;
      gc[e] = c;
    }
    return true;
  };
  std::vector<int32_t> gidx_c, gidx_ic;
  if (!to_compact(gidx, gidx_c) || !to_compact(gidx_i, gidx_ic))
    return fail(set_error(FC2D_ERR_GEOMETRY, "a matching stencil tap is not an inside point"));
  if ((st = upload(&p->dev.Q, p->Q)) || (st = upload(&p->dev.Ar, p->Ar)) ||
      (st = upload(&p->dev.Ar_hi, arh)) || (st = upload(&p->dev.Ar_lo, arl)) ||
      (st = upload(&p->dev.gidx, gidx)) || (st = upload(&p->dev.gw, gw)) ||
      (st = upload(&p->dev.wn, wn)) || (st = upload(&p->dev.gidx_i, gidx_i)) ||
      (st = upload(&p->dev.gw_i, gw_i)) || (st = upload(&p->dev.wn_i, wn_i)) ||
      (st = upload(&p->dev.s_lin, p->strip_lin)) ||
      (st = upload(&p->dev.s_theta, p->strip_theta)) ||
      (st = upload(&p->dev.s_eta, p->strip_eta)) ||
      (st = upload(&p->dev.row_iv_off, p->row_iv_off)) ||
      (st = upload(&p->dev.row_iv, p->row_iv)) ||
      (st = upload(&p->dev.row_strip_off, p->row_strip_off)) ||
      (compact && (st = upload(&p->dev.row_iv_coff, p->row_iv_coff))) ||
      (compact && (st = upload(&p->dev.gidx_c, gidx_c))) ||
      (compact && (st = upload(&p->dev.gidx_ic, gidx_ic))) ||
      (st = upload(&p->dev.status, zero_status)) ||
      (st = upload(&p->fx.tw64, p->fx.tw_host)) || (st = upload(&p->fx.tw32, tw32x)) ||
      (st = upload(&p->fy.tw64, p->fy.tw_host)) || (st = upload(&p->fy.tw32, tw32y)) ||
      (st = upload(&p->rtw64, p->rtw_host)) || (st = upload(&p->rtw32, rtw32)) ||
      (st = upload(&p->fx.tws64, tsx64)) || (st = upload(&p->fy.tws64, tsy64)) ||
      (st = upload(&p->fx.tws32, tsx32)) || (st = upload(&p->fy.tws32, tsy32)))
    return fail(st);
  // interpolation weights (Section 3.4), computed once in FP64 on the GPU
  {
    const size_t ns = p->strip_lin.size();
    const size_t wbytes = std::max<size_t>(1, ns) * 2 * M *
                          (P.precision == FC2D_FP64 ? sizeof(double) : sizeof(float));
    if (cudaMalloc(&p->dev.s_w, wbytes) != cudaSuccess ||
        cudaMalloc((void**)&p->dev.s_pb, std::max<size_t>(1, ns) * 4) != cudaSuccess ||
        cudaMalloc((void**)&p->dev.s_sb, std::max<size_t>(1, ns) * 4) != cudaSuccess)
      return fail(set_error(FC2D_ERR_NOMEM, "cudaMalloc of the interpolation weights failed"));
    st = interp_weights_gpu((int)ns, M, p->Cr, B, k1, P.n_r, p->dev.s_theta, p->dev.s_eta,
                            P.precision == FC2D_FP64, p->dev.s_w, p->dev.s_pb, p->dev.s_sb);
    if (st) return fail(st);
    if (P.precision == FC2D_MIXED && M == 8 && ns > 0 && (st = owner_tables(p, (int)ns, M)))
      return fail(st);
  }
  if ((st = tune_plan(p))) return fail(st);
  *out = p;
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_plan_info(fc2d_plan_t p, fc2d_info* out) {
  if (!p || !out) return set_error(FC2D_ERR_ARG, "fc2d_plan_info: null argument");
  out->grid = p->grid;
  out->params = p->prm;
  out->n_strip = (int64_t)p->strip_lin.size();
  out->n_inside = p->n_inside;
  out->n_bdry = p->n_bdry;
  size_t esz = p->prm.precision == FC2D_MIXED ? 4 : 8;
  size_t F = (size_t)p->prm.B * (p->Cr + 1) * esz;
  size_t S = p->strip_lin.size() * esz;
  size_t pitch = row_pitch(p);
  size_t I = (size_t)p->grid.ny * pitch * 2 * esz;
  out->workspace_bytes_per_function = (int64_t)(F + S + I + 256 * 3);
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_boundary_points(fc2d_plan_t p, double* xy) {
  if (!p || !xy) return set_error(FC2D_ERR_ARG, "fc2d_boundary_points: null argument");
  std::memcpy(xy, p->bdry_xy.data(), p->bdry_xy.size() * sizeof(double));
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_fc_matrices(fc2d_plan_t p, double* Qh, double* Arh) {
  if (!p || !Qh || !Arh) return set_error(FC2D_ERR_ARG, "fc2d_fc_matrices: null argument");
  std::memcpy(Qh, p->Q.data(), p->Q.size() * sizeof(double));
  std::memcpy(Arh, p->Ar.data(), p->Ar.size() * sizeof(double));
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_strip_points(fc2d_plan_t p, int32_t* lin, double* theta,
                                         double* eta) {
  if (!p || !lin || !theta || !eta)
    return set_error(FC2D_ERR_ARG, "fc2d_strip_points: null argument");
  size_t n = p->strip_lin.size();
  std::memcpy(lin, p->strip_lin.data(), n * sizeof(int32_t));
  std::memcpy(theta, p->strip_theta.data(), n * sizeof(double));
  std::memcpy(eta, p->strip_eta.data(), n * sizeof(double));
  return FC2D_OK;
}

extern "C" void fc2d_destroy(fc2d_plan_t p) {
  if (!p) return;
  poisson_destroy(p);
  wave_destroy(p);
  void* ptrs[] = {p->dev.Q, p->dev.Ar, p->dev.Ar_hi, p->dev.Ar_lo, p->dev.gidx, p->dev.gw,
                  p->dev.wn, p->dev.s_lin, p->dev.s_theta, p->dev.s_eta, p->dev.s_w,
                  p->dev.s_pb, p->dev.s_sb, p->dev.own[0].off, p->dev.own[0].k,
                  p->dev.own[0].pack, p->dev.own[0].w, p->dev.own[0].start,
                  p->dev.own[1].off, p->dev.own[1].k, p->dev.own[1].pack, p->dev.own[1].w,
                  p->dev.own[1].start, p->dev.row_iv_off,
                  p->dev.row_iv, p->dev.row_strip_off, p->dev.row_iv_coff, p->dev.gidx_c,
                  p->dev.gidx_i, p->dev.gw_i, p->dev.wn_i, p->dev.gidx_ic,
                  p->dev.status, p->fx.tw64, p->fx.tw32,
                  p->fy.tw64, p->fy.tw32, p->rtw64, p->rtw32, p->ws.base,
                  p->fx.tws64, p->fx.tws32, p->fy.tws64, p->fy.tws32};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (auto& r : p->prof) {
    p->event_pool.push_back(r.start);
    p->event_pool.push_back(r.stop);
  }
  for (void* e : p->event_pool) cudaEventDestroy((cudaEvent_t)e);
  delete p;
}

extern "C" const char* fc2d_last_error(void) { return fc2d::g_last_error.c_str(); }
