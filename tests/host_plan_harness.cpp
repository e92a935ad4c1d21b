// Test harness: runs the library's host plan code (plan.cpp) on the CPU.
//
// The CUDA runtime calls the plan makes are redirected to host memory, and the plan's
// GPU Newton foot search is replaced by the same iteration on the host, so that the
// geometry, boundary points and matching stencils can be compared with the oracle
// without a GPU.  Output: binary arrays on stdout (see dump()).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

static cudaError_t h_malloc(void** p, size_t n) {
  *p = std::malloc(n ? n : 1);
  return cudaSuccess;
}
static cudaError_t h_free(void* p) {
  std::free(p);
  return cudaSuccess;
}
static cudaError_t h_memcpy(void* d, const void* s, size_t n, int) {
  std::memcpy(d, s, n);
  return cudaSuccess;
}
static cudaError_t h_getdev(int* d) {
  *d = 0;
  return cudaSuccess;
}
#define cudaMalloc(p, n) h_malloc((void**)(p), (n))
#define cudaFree(p) h_free(p)
#define cudaMemcpy(d, s, n, k) h_memcpy((d), (s), (n), (k))
#define cudaGetDevice(d) h_getdev(d)
static cudaError_t h_attr(int* v, int, int) {
  *v = 152;
  return cudaSuccess;
}
#define cudaDeviceGetAttribute(v, a, d) h_attr((v), (int)(a), (d))

#include "../paper_2010_03901_gb300/csrc/plan.cpp"
#include "../paper_2010_03901_gb300/csrc/wave_band.cpp"

namespace fc2d {
fc2d_status foot_newton_gpu(const Curve& c, const std::vector<double>& qx,
                            const std::vector<double>& qy, std::vector<double>& th,
                            std::vector<int>& conv, double window) {
  conv.assign(qx.size(), 0);
  for (size_t i = 0; i < qx.size(); ++i) {
    double t = th[i];
    {
      const double t0 = t;
      double best = 1e300;
      for (int k = -24; k <= 24; ++k) {
        double tk = t0 + window * double(k) / 24, x, y;
        c.eval(tk, x, y);
        double d2 = (x - qx[i]) * (x - qx[i]) + (y - qy[i]) * (y - qy[i]);
        if (d2 < best) {
          best = d2;
          t = tk;
        }
      }
    }
    for (int it = 0; it < 60; ++it) {
      double x, y, x1, y1, x2, y2;
      c.eval(t, x, y);
      c.eval_d(t, 1, x1, y1);
      c.eval_d(t, 2, x2, y2);
      double phi = (x - qx[i]) * x1 + (y - qy[i]) * y1;
      double dphi = x1 * x1 + y1 * y1 + (x - qx[i]) * x2 + (y - qy[i]) * y2;
      if (!(dphi > 0)) break;
      double step = phi / dphi;
      t -= step;
      if (std::fabs(step) < 1e-12) {
        c.eval(t, x, y);
        c.eval_d(t, 1, x1, y1);
        c.eval_d(t, 2, x2, y2);
        phi = (x - qx[i]) * x1 + (y - qy[i]) * y1;
        dphi = x1 * x1 + y1 * y1 + (x - qx[i]) * x2 + (y - qy[i]) * y2;
        if (dphi > 0) t -= phi / dphi;
        conv[i] = 1;
        break;
      }
    }
    th[i] = t;
  }
  return FC2D_OK;
}
void poisson_destroy(fc2d_plan_s*) {}
void wave_destroy(fc2d_plan_s*) {}
// launch-shape tuning times kernels on a GPU; the harness keeps the defaults
fc2d_status tune_plan(fc2d_plan_s*) { return FC2D_OK; }
// interpolation weights are a GPU step of the plan; the harness leaves them unset
fc2d_status interp_weights_gpu(int, int, int, int, double, int, const double*, const double*,
                               bool, void*, int32_t*, int32_t*) {
  return FC2D_OK;
}
}  // namespace fc2d

template <typename T>
static void dump(const char* name, const T* p, size_t n) {
  std::printf("%s %zu %zu\n", name, n, sizeof(T));
  std::fwrite(p, sizeof(T), n, stdout);
  std::printf("\n");
}

int main(int argc, char** argv) {
  if (argc > 1 && !std::strcmp(argv[1], "partition")) {
    // stdin: cap n_cta B cnt_0 .. cnt_{B-1}; stdout: the range starts
    int cap, n_cta, B;
    if (std::scanf("%d %d %d", &cap, &n_cta, &B) != 3) return 1;
    std::vector<int64_t> cnt(B);
    for (auto& v : cnt)
      if (std::scanf("%lld", reinterpret_cast<long long*>(&v)) != 1) return 1;
    for (int32_t v : partition_owners(cnt, cap, n_cta)) std::printf("%d ", v);
    std::printf("\n");
    return 0;
  }
  // argv: n_modes cx.. sx.. cy.. sy.. a0 b0 h nx ny d C Z n_os n_r M B m_F k1 [n_c [squares]]
  int a = 1;
  int nm = std::atoi(argv[a++]);
  std::vector<double> cx(nm), sx(nm), cy(nm), sy(nm);
  for (auto* v : {&cx, &sx, &cy, &sy})
    for (int k = 0; k < nm; ++k) (*v)[k] = std::atof(argv[a++]);
  fc2d_grid g;
  g.a0 = std::atof(argv[a++]);
  g.b0 = std::atof(argv[a++]);
  g.h = std::atof(argv[a++]);
  g.nx = std::atoi(argv[a++]);
  g.ny = std::atoi(argv[a++]);
  fc2d_params P{};
  P.d = std::atoi(argv[a++]);
  P.C = std::atoi(argv[a++]);
  P.Z = std::atoi(argv[a++]);
  P.n_os = std::atoi(argv[a++]);
  P.n_r = std::atoi(argv[a++]);
  P.M = std::atoi(argv[a++]);
  P.B = std::atoi(argv[a++]);
  P.m_F = std::atoi(argv[a++]);
  P.k1 = std::atof(argv[a++]);
  fc2d_boundary b{nm, cx.data(), sx.data(), cy.data(), sy.data()};
  fc2d_plan_t p = nullptr;
  fc2d_status st = fc2d_plan(&b, &g, &P, &p);
  std::printf("status %d %s\n", (int)st, fc2d_last_error());
  if (st) return 0;
  const size_t B = P.B, M = P.M, d = P.d;
  dump("Q", p->Q.data(), p->Q.size());
  dump("Ar", p->Ar.data(), p->Ar.size());
  dump("strip_lin", p->strip_lin.data(), p->strip_lin.size());
  dump("strip_theta", p->strip_theta.data(), p->strip_theta.size());
  dump("strip_eta", p->strip_eta.data(), p->strip_eta.size());
  dump("bdry_xy", p->bdry_xy.data(), p->bdry_xy.size());
  dump("row_iv_off", p->row_iv_off.data(), p->row_iv_off.size());
  dump("row_iv", p->row_iv.data(), p->row_iv.size());
  dump("gidx", p->dev.gidx, B * (M - 1) * M);
  dump("gidx_c", p->dev.gidx_c, B * (M - 1) * M);
  dump("row_iv_coff", p->row_iv_coff.data(), p->row_iv_coff.size());
  dump("gw", p->dev.gw, B * (M - 1) * M);
  dump("wn", p->dev.wn, B * (d - 1) * M);
  dump("gidx_i", p->dev.gidx_i, B * (M - 1) * M);
  dump("gw_i", p->dev.gw_i, B * (M - 1) * M);
  dump("wn_i", p->dev.wn_i, B * d * M);
  const int32_t ok = p->interior_ok ? 1 : 0;
  dump("interior_ok", &ok, 1);
  if (a < argc) {  // optional: the Fourier Forwarding band for n_c
    fc2d::WaveBand wb;
    const int n_c = std::atoi(argv[a++]);
    const int squares = a < argc ? std::atoi(argv[a++]) : 0;
    const int reach = squares ? (int)std::ceil(std::sqrt(2.0) * n_c) + 2 : n_c + fc2d::kUbBandExtra;
    st = fc2d::build_wave_band(p, n_c, reach, wb);
    std::printf("wave_status %d %s\n", (int)st, fc2d_last_error());
    if (st) return 0;
    dump("wb_unknown_lin", wb.unknown_lin.data(), wb.unknown_lin.size());
    dump("wb_slaved_lin", wb.slaved_lin.data(), wb.slaved_lin.size());
    dump("wb_unknown_dist", wb.unknown_dist.data(), wb.unknown_dist.size());
    dump("wb_slaved_dist", wb.slaved_dist.data(), wb.slaved_dist.size());
    dump("wb_iface_lin", wb.iface_lin.data(), wb.iface_lin.size());
    dump("wb_near_lin", wb.near_lin.data(), wb.near_lin.size());
    dump("wb_near_src", wb.near_src.data(), wb.near_src.size());
    for (auto* m : {&wb.L, &wb.D, &wb.S}) {
      const char* nm = m == &wb.L ? "L" : (m == &wb.D ? "D" : "S");
      std::string o = std::string("wb_") + nm + "_off", c = std::string("wb_") + nm + "_col",
                  w = std::string("wb_") + nm + "_w";
      dump(o.c_str(), m->off.data(), m->off.size());
      dump(c.c_str(), m->col.data(), m->col.size());
      dump(w.c_str(), m->w.data(), m->w.size());
    }
    if (squares) {
      fc2d::SquareSet sq;
      st = fc2d::build_wave_squares(p, wb, n_c, sq);
      std::printf("squares_status %d %s\n", (int)st, fc2d_last_error());
      if (st) return 0;
      dump("sq_origin_j", sq.origin_j.data(), sq.origin_j.size());
      dump("sq_origin_i", sq.origin_i.data(), sq.origin_i.size());
      dump("sq_served_off", sq.served_off.data(), sq.served_off.size());
      dump("sq_served_lin", sq.served_lin.data(), sq.served_lin.size());
      dump("sq_served_local", sq.served_local.data(), sq.served_local.size());
    }
  }
  return 0;
}
