/*
 * fc2d.h -- C ABI of the GB300 two-dimensional Fourier Continuation (2D-FC) library.
 *
 * Method: O. P. Bruno and J. Paul, "Two-dimensional Fourier Continuation and
 * applications" (arXiv 2010.03901).  A smooth f given on the Cartesian grid points
 * inside a smooth closed curve (and on a few points of the curve) is continued to a
 * bi-periodic function on the whole grid: 1D blending-to-zero along the boundary
 * normals (Section 2.2, eq. (2.6); Remark 2.2), interpolation of the normal values
 * onto the grid points of the outer strip (Sections 3.3-3.4), and a 2D DFT (eq. (3.1)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid:      x_i = a0 + i h, y_j = b0 + j h, 0 <= i < nx, 0 <= j < ny (eq. (3.7)).
 *            Grid arrays are row-major [n_f][ny][nx] (x fastest).
 * Spectrum:  fhat[f][m][l] = (1/(nx ny)) sum_{j,i} ext[f][j][i] e^{-2 pi i (l i/nx + m j/ny)},
 *            0 <= l <= nx/2, 0 <= m < ny: the half spectrum [n_f][ny][nx/2+1] of
 *            interleaved (re, im) pairs in DFT index order (m > ny/2 stands for m - ny).
 *            The phase is relative to the grid origin (a0, b0).
 * Boundary data: f_bdry[f][k] holds f at the boundary points listed by
 *            fc2d_boundary_points: first the B feet q(theta_p) of the normals
 *            (theta_p = 2 pi p/B, eq. (3.4)), then the crossings of each grid column
 *            x = x_i with the curve (i ascending, y ascending), then those of each
 *            grid row (j ascending, x ascending).
 *            f_bdry_dev may be NULL in fc2d_blend, fc2d_extend, fc2d_extend_coeffs and
 *            fc2d_extend_coeffs_compact: interior data only (Remark 3.2 II).  Each red
 *            star is then interpolated from grid nodes alone and the matching value at
 *            the foot is extrapolated from the red stars (degree M-2); it also serves
 *            as F[f][p][0].  Accuracy near the boundary is lower, as the remark says.
 *            These calls return FC2D_ERR_UNSUPPORTED with NULL boundary data when some
 *            red star's chord holds no grid node (then only the boundary form exists).
 * Memory:    pointers named *_dev are device pointers owned by the caller; *_host are
 *            host pointers owned by the caller.  The plan owns only its own tables
 *            and workspace.
 * Precision: FC2D_FP64 computes every stage in double and uses double for every
 *            array.  FC2D_MIXED reads the same double inputs (the blending matrix has
 *            entries near 4e3, so rounding the data to float first would cost ~1e-4),
 *            forms the matching values and Gram coefficients in double, runs the
 *            continuation contraction on the tensor cores in TF32 with hi/lo split
 *            operands and FP32 accumulation, and the FFT in float: ext is float and
 *            fhat is (float, float) pairs.
 * Streams:   every compute call is asynchronous on the given cudaStream_t (passed as
 *            void*; NULL = legacy default stream) and returns after launching.
 *            fc2d_plan and the host queries are synchronous.
 * Errors:    argument and geometry errors are returned synchronously; the text is in
 *            fc2d_last_error().  Device-side conditions (a Newton search that did not
 *            converge, a bounded wait that gave up) are latched in the plan and
 *            returned (once) by fc2d_sync_status.
 *            No entry point aborts, traps or exits the process.
 * Threads:   a plan may be used by one host thread at a time.
 */
#ifndef FC2D_H
#define FC2D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fc2d_plan_s* fc2d_plan_t;

typedef enum {
  FC2D_OK = 0,
  FC2D_ERR_ARG = 1,            /* bad argument (null pointer, size, parameter)        */
  FC2D_ERR_GEOMETRY = 2,       /* strip leaves the grid, stencil leaves the domain... */
  FC2D_ERR_NOT_CONVERGED = 3,  /* a Newton foot search hit its iteration cap          */
  FC2D_ERR_TIMEOUT = 4,        /* a bounded device wait gave up                       */
  FC2D_ERR_NOMEM = 5,          /* device or host allocation failed                    */
  FC2D_ERR_CUDA = 6,           /* a CUDA runtime call failed                          */
  FC2D_ERR_UNSUPPORTED = 7     /* grid size or option this build does not handle      */
} fc2d_status;

typedef enum { FC2D_FP64 = 0, FC2D_MIXED = 1 } fc2d_precision;

/* Closed curve as a trigonometric polynomial of degree n_modes-1 (eq. (3.2)):
 *   x(t) = sum_k cx[k] cos(k t) + sx[k] sin(k t),  y(t) likewise with cy, sy.
 * Either orientation; the plan re-parametrises a clockwise curve by t -> -t. */
typedef struct {
  int n_modes;
  const double *cx, *sx, *cy, *sy;  /* host arrays of length n_modes */
} fc2d_boundary;

typedef struct {
  double a0, b0, h;  /* origin and step of the grid H (eq. (3.7))  */
  int nx, ny;        /* both even, each of the form 2^a 3^b 5^c    */
} fc2d_grid;

/* Section 3.6 parameter list.  A zero field takes the paper's default (Remark 3.3):
 * d=5, C=27, Z=12, n_os=20, n_r=6, M=d+3, B=round(2 pi/h), m_F=20, k1=h.
 * Ranges: 2 <= d <= 12 (d <= 8 for FC2D_MIXED), 2 <= M <= 16, M <= C n_r + 1. */
typedef struct {
  int d, C, Z, n_os, n_r, M, B, m_F;
  double k1;      /* normal step of V-/V+ (eqs. (3.5)-(3.6)) */
  int precision;  /* fc2d_precision                          */
} fc2d_params;

typedef struct {
  fc2d_grid grid;
  fc2d_params params;  /* with defaults filled in */
  int64_t n_strip;     /* grid points in H cap V+ (continuation points)            */
  int64_t n_inside;    /* grid points in the closed domain                         */
  int64_t n_bdry;      /* boundary data points (B + column + row crossings)        */
  int64_t workspace_bytes_per_function;
} fc2d_info;

/* Geometrical setup, Section 3.5 steps 1-4: boundary grid I_B, curvilinear grids,
 * the FC matrices Q and A_r (Section 2.2, Remark 2.2; computed here in double-double
 * arithmetic), the inside test, the feet of the normals through the strip points
 * (Newton's method in FP64 on the GPU) and the matching stencils of Section 3.2.
 * Synchronous.  Uses the current CUDA device.  *out receives a new plan.
 * Returns FC2D_ERR_GEOMETRY when the strip of width C*k1 leaves the grid or a
 * stencil leaves the domain. */
fc2d_status fc2d_plan(const fc2d_boundary* boundary, const fc2d_grid* grid,
                      const fc2d_params* params, fc2d_plan_t* out);

fc2d_status fc2d_plan_info(fc2d_plan_t plan, fc2d_info* out);

/* Boundary data points (x, y), [n_bdry][2], in the order described above. */
fc2d_status fc2d_boundary_points(fc2d_plan_t plan, double* xy_host);

/* The plan's FC matrices: Q [d][d] and A_r [C n_r][d] (row-major, double). */
fc2d_status fc2d_fc_matrices(fc2d_plan_t plan, double* Q_host, double* Ar_host);

/* Strip points H cap V+: linear grid index j*nx+i (ascending), foot parameter
 * theta^Q in [0, 2 pi) and distance eta_Q (Section 3.4). */
fc2d_status fc2d_strip_points(fc2d_plan_t plan, int32_t* lin_host, double* theta_host,
                              double* eta_host);

/* Steps 5 of Section 3.5 (Section 3.2 + eq. (2.6)): matching values and blending.
 * F_dev receives [n_f][B][C n_r + 1] strip values (double for FP64, float for MIXED):
 * F[f][p][0] = f at q(theta_p) (its extrapolation with NULL boundary data),
 * F[f][p][q] = (A_r Q^T f_{D_p})_q. */
fc2d_status fc2d_blend(fc2d_plan_t plan, int n_f, const double* f_grid_dev,
                       const double* f_bdry_dev, void* F_dev, void* stream);

/* Step 6 (Section 3.4): continuation values at the strip points from F_dev.
 * vals_dev receives [n_f][n_strip] in the order of fc2d_strip_points. */
fc2d_status fc2d_interp(fc2d_plan_t plan, int n_f, const void* F_dev, void* vals_dev,
                        void* stream);

/* Steps 5-6: the extension.  ext_dev [n_f][ny][nx] receives f at the grid points in
 * the closed domain, the continuation on the strip and 0 elsewhere.  Grid values
 * outside the domain are never read.  For FP64, ext_dev may equal f_grid_dev. */
fc2d_status fc2d_extend(fc2d_plan_t plan, int n_f, const double* f_grid_dev,
                        const double* f_bdry_dev, void* ext_dev, void* stream);

/* Step 7: the 2D DFT (eq. (3.1)) of an extension, fhat_dev [n_f][ny][nx/2+1][2]. */
fc2d_status fc2d_coeffs(fc2d_plan_t plan, int n_f, const void* ext_dev, void* fhat_dev,
                        void* stream);

/* Steps 5-7 fused: the spectrum of the extension of f, without writing the extended
 * grid (the strip values go to plan workspace, the row DFT reads the domain points
 * from f_grid_dev and the strip values from the workspace).  Same result as
 * fc2d_extend followed by fc2d_coeffs. */
fc2d_status fc2d_extend_coeffs(fc2d_plan_t plan, int n_f, const double* f_grid_dev,
                               const double* f_bdry_dev, void* fhat_dev, void* stream);

/* Steps 5-7 for a complex-valued f (Section 3: f maps the domain to C).  f_grid_dev
 * [n_f][2][ny][nx] double: the real part of function f, then its imaginary part;
 * f_bdry_dev [n_f][2][n_bdry] in the same way, or NULL (interior data only).
 * fhat_dev receives the full spectrum [n_f][ny][nx][2] (re, im; double for FP64, float
 * for MIXED), fhat[f][m][l] = (1/(nx ny)) sum_{j,i} ext[f][j][i] e^{-2 pi i (l i/nx +
 * m j/ny)}, 0 <= l < nx, 0 <= m < ny, with ext = ext(Re f) + i ext(Im f) (the method is
 * linear and real).  The two parts run through the real path as functions 2f and 2f+1;
 * a last kernel assembles the full spectrum from their half spectra by Hermitian
 * symmetry.  Plan workspace: that of 2 n_f functions plus their half spectra. */
fc2d_status fc2d_extend_coeffs_complex(fc2d_plan_t plan, int n_f, const double* f_grid_dev,
                                       const double* f_bdry_dev, void* fhat_dev, void* stream);

/* The grid points of the closed domain (the points where f is given; Section 3.1) in the
 * order of the compact entry point below: row by row (y ascending), within a row by x.
 * lin_host (host memory, n_inside entries from fc2d_plan_info) receives their linear
 * indices j * nx + i.  Pure host call. */
fc2d_status fc2d_inside_points(fc2d_plan_t plan, int64_t* lin_host);

/* fc2d_extend_coeffs with f given only where the method uses it, at the grid points of
 * the closed domain (Section 3.1: the data of the 2D-FC problem are f on H ∩ Ω):
 * f_inside_dev [n_f][n_inside] in the order of fc2d_inside_points.  Same kernels and
 * arithmetic as fc2d_extend_coeffs, so the same spectrum bit for bit; the input is
 * n_inside instead of nx * ny values (about half for the kite), which halves the
 * host-to-device copy of a caller that streams f from host memory.  Returns
 * FC2D_ERR_UNSUPPORTED when n_inside exceeds 2^31 - 1. */
fc2d_status fc2d_extend_coeffs_compact(fc2d_plan_t plan, int n_f, const double* f_inside_dev,
                                       const double* f_bdry_dev, void* fhat_dev, void* stream);

/* The DFT of fc2d_coeffs for callers that cannot allocate device memory at call time.
 * The paper has no counterpart: this is a service of the library.  fc2d_coeffs grows
 * plan workspace with cudaMalloc on the first call of a new size; this entry point
 * calls no allocator (no cudaMalloc, cudaFree or allocating library routine).  It is
 * meant for callers that own all device memory through their own allocator, or that
 * run where an allocation's implicit device synchronisation is not acceptable.
 * Its scratch is one fixed device array of 64 MiB (the row-DFT intermediate,
 * n_f * ny * (nx/2+1 rounded up to 16) complex values), held by every GPU that loads
 * the library until the process exits.  Larger requests return FC2D_ERR_ARG.
 * The first call on a device looks up the array's device address for that device
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array: calls that overlap on the GPU (different streams,
 * or different plans, at the same time) race; serialise them.  Nothing in the array
 * has to start at zero.  Arguments and result as fc2d_coeffs; the plan's tables were
 * allocated by fc2d_plan. */
fc2d_status fc2d_coeffs_static(fc2d_plan_t plan, int n_f, const void* ext_dev, void* fhat_dev,
                               void* stream);

/* Poisson problem Delta u = f in the domain, u = g on the curve (Section 4.1,
 * eqs. (4.1)-(4.6)), FP64 plans (FP64 data and arithmetic, except the double-layer sums
 * on the grid: double-float, about 48 bits).  fc2d_poisson_plan builds the boundary-integral tables
 * once (synchronous): n_b equispaced parameters 2 pi k/n_b (n_b <= 0 means nx, as in
 * Section 4.1.1), the Nystrom matrix of the double-layer equation -phi/2 + K phi = g_hom,
 * the boundary interpolation stencils of u_p, and the near-boundary point lists.
 * fc2d_poisson_nodes returns n_b and, if xy_host is not NULL, the nodes [n_b][2] where
 * the Dirichlet data g are needed. */
fc2d_status fc2d_poisson_plan(fc2d_plan_t plan, int n_b);
fc2d_status fc2d_poisson_nodes(fc2d_plan_t plan, double* xy_host, int* n_b);

/* Solve: u = u_p + v.  u_p from the 2D-FC spectrum of f (multiplier of eq. (4.6), the
 * constant term + hat f_00 (x^2+y^2)/4), its values on the curve by iterated degree M-1
 * interpolation, the density by GMRES (tolerance 1e-14), v at the grid points inside by
 * the trapezoidal rule with near-boundary refinement.  f_grid_dev [n_f][ny][nx] and
 * f_bdry_dev [n_f][n_bdry] as for fc2d_extend; g_nodes_dev [n_f][n_b]; u_dev [n_f][ny][nx]
 * receives u inside the domain and 0 elsewhere; phi_dev (NULL allowed) receives the
 * density [n_f][n_b].  The GMRES iteration is driven from the host: this call waits
 * for the stream.  Returns FC2D_ERR_NOT_CONVERGED if GMRES stalls. */
fc2d_status fc2d_poisson(fc2d_plan_t plan, int n_f, const double* f_grid_dev,
                         const double* f_bdry_dev, const double* g_nodes_dev, double* u_dev,
                         double* phi_dev, void* stream);
/* Last solve: GMRES iterations and relative residual; number of near-boundary points. */
fc2d_status fc2d_poisson_info(fc2d_plan_t plan, int* gmres_iters, double* gmres_resid,
                              int64_t* n_near);

/* Fourier Forwarding interior propagator (Section 4.2, eqs. (4.8)-(4.12)), FP64 plans.
 * For n_f pairs of initial data (u, u_t), given like f in fc2d_extend (grid values
 * [n_f][ny][nx] and boundary data [n_f][n_bdry], or NULL for interior data only): the
 * 2D-FC expansions F and G, the modal
 * solutions a = hat f cos(w t) + hat g sin(w t)/w (a_00 = hat f_00 + t hat g_00),
 * w = 2 pi c sqrt((l/L_x)^2 + (m/L_y)^2), and their inverse DFTs.  u_out and ut_out
 * [n_f][ny][nx] receive U_FC(., t) and its time derivative on the whole grid; they are
 * the wave solution at the grid points farther than c t from the curve (domain of
 * dependence).  ny <= 4736. */
fc2d_status fc2d_wave_interior(fc2d_plan_t plan, int n_f, double c, double t,
                               const double* u0_grid_dev, const double* u0_bdry_dev,
                               const double* ut0_grid_dev, const double* ut0_bdry_dev,
                               double* u_out_dev, double* ut_out_dev, void* stream);

/* Kernel timing (tracing).  While enabled, every kernel the plan launches is
 * bracketed by a pair of CUDA events recorded on its launching stream.
 * fc2d_profile_read waits for those events and returns, per kernel name, the number
 * of launches and their summed device time in milliseconds, then clears the record.
 * names_host receives up to max_kernels NUL-terminated names of at most 63 chars
 * (64 bytes each).  *n_out receives the number of kernel names. */
fc2d_status fc2d_profile(fc2d_plan_t plan, int enable);
fc2d_status fc2d_profile_read(fc2d_plan_t plan, int max_kernels, char* names_host,
                              int64_t* launches_host, double* ms_host, int* n_out);

/* Waits for the stream and returns the plan's latched device status, then clears it
 * (a condition is reported once; the next call returns FC2D_OK unless a kernel latched
 * a new one). */
fc2d_status fc2d_sync_status(fc2d_plan_t plan, void* stream);

/* Failure detection check (no operation of the paper).  Runs the bounded device wait
 * of the tensor-core blend kernels on an mbarrier that nothing arrives on: after
 * 2 x polls polls the kernel latches FC2D_ERR_TIMEOUT in the plan's status word and
 * returns, so that fc2d_sync_status then returns FC2D_ERR_TIMEOUT; nothing hangs or
 * traps and the plan stays usable.  polls in 1 .. 2^22 (FC2D_ERR_ARG otherwise); one
 * block of 32 threads on `stream`, asynchronous. */
fc2d_status fc2d_wait_selftest(fc2d_plan_t plan, uint32_t polls, void* stream);

/* Fourier Forwarding solve (Section 4.2, eq. (4.9)), FP64 plans: the wave equation
 * u_tt = c^2 (u_xx + u_yy) in the domain with Dirichlet data g on the curve, advanced by
 * n_large large steps Delta T = n_c h / c from t = 0.  Each large step combines the
 * interior propagator U_FC (the 2D-FC expansions of u(T_j), u_t(T_j), eqs. (4.10)-(4.12))
 * with the near-boundary solver U_B: S = 8 n_c small steps Delta t = Delta T / S (CFL
 * c Delta t / h = 0.125, second-order Taylor, Section 4.2.1) on the grid points within
 * n_c h + 2h of the curve, Dirichlet data imposed by cubic boundary polynomials along
 * the grid lines (the embedded-boundary closure the paper cites), a fourth-difference
 * dissipation that makes the small step stable, and interface values (the band's inner
 * edge) at every small step either from U_FC by a full inverse DFT (interface_mode 0) or
 * by the paper's small-square procedure (interface_mode 1): squares of 37 x 37 grid
 * points inside the domain, each expanded by 1D-FC along rows and columns into a 64 x 64
 * periodic box once per large step, advanced modally and inverted at every small step
 * at the interface points within (18 - n_c) h of its centre; in that mode the band
 * reaches (ceil(sqrt(2) n_c) + 2) h, so that squares inside the domain reach every
 * interface point, and n_c <= 18 (FC2D_ERR_GEOMETRY if a domain is too narrow or curved
 * for the squares).  interface_mode 2: the squares of mode 1 with their every-small-step
 * evaluation (the modal advance and the two passes of inverse 64-point DFTs) in
 * double-float arithmetic, pairs of FP32 values holding about 44 significant bits (the
 * FP32 pipe issues 64 times the FP64 rate on this part); the expansions, U_B and U_FC at
 * T_{j+1} stay FP64 (fc2d_wave_band_* take mode 1 for its sets).  At T_{j+1} the grid takes U_FC where the distance to
 * the curve is >= n_c h and U_B elsewhere (eq. (4.9)); U_B continues across large steps.
 *   u_dev, ut_dev  [n_f][ny][nx] in: u and u_t at t = 0 (values inside the domain used);
 *                  out: u and u_t at t = n_large Delta T inside the domain, 0 outside.
 *   g_dir_dev      [n_large S + 1][n_f][n_bdry]: g at t = m Delta t at the plan's boundary
 *                  points (fc2d_boundary_points), or NULL for g = 0.
 *   gt_dir_dev     [n_large + 1][n_f][n_bdry]: dg/dt at t = j Delta T, or NULL for 0.
 * 1 <= n_c <= 256; ny <= 4842.  The band and its operators are built on the first call
 * for a given n_c (host, synchronous) and kept in the plan; scratch is allocated on the
 * first call for a larger n_f.  Asynchronous on `stream` otherwise. */
fc2d_status fc2d_forward_wave(fc2d_plan_t plan, int n_f, double c, int n_c, int n_large,
                              int interface_mode, double* u_dev, double* ut_dev,
                              const double* g_dir_dev, const double* gt_dir_dev, void* stream);

/* U_B's sets for large-step width n_c h and an interface mode (Section 4.2
 * near-boundary solver): counts[5] = {unknowns (stepped points), slaved points (values
 * from a boundary polynomial), interface points (U_FC values the operators read), points
 * nearer than n_c h to the curve (where U_B is the solution), squares (mode 1; else 0)}.
 * fc2d_wave_band_points copies the grid linear indices j nx + i of the first four sets,
 * ascending, into host arrays (NULL skips). */
fc2d_status fc2d_wave_band_info(fc2d_plan_t plan, int n_c, int interface_mode, int64_t* counts);
fc2d_status fc2d_wave_band_points(fc2d_plan_t plan, int n_c, int interface_mode,
                                  int32_t* unknown_lin, int32_t* slaved_lin, int32_t* iface_lin,
                                  int32_t* near_lin);

/* One U_B small step with caller data (the step fc2d_forward_wave takes with
 * interface_mode 0), for tests:
 * u, u_prev, ut and out are [n_unknown][n_f] (function-minor), grid / grid_prev the
 * U_FC grids [n_f][ny][nx] at the step's time and the one before (interface values),
 * g the Dirichlet data [n_f][n_bdry] (NULL: zero).  mode 0: out = u + dt ut + (c dt)^2/2
 * L(u); 1: out = 2u - u_prev + (c dt)^2 L(u) - 0.3 D(u - u_prev); 2: the mode-1 value v
 * stored as (v - u_prev)/(2 dt).  c dt = h/8. */
fc2d_status fc2d_wave_ub_step(fc2d_plan_t plan, int n_c, int n_f, int mode, double c,
                              const double* u_dev, const double* u_prev_dev,
                              const double* ut_dev, const double* grid_dev,
                              const double* grid_prev_dev, const double* g_dev, double* out_dev,
                              void* stream);

/* Launch shapes of the plan (no operation of the paper; each choice computes the same
 * values bit for bit).  The mixed form's 4096-point column DFT passes run in one of two
 * forms: direct (a block per tile of 64 rows x 16, 32 or 64 columns, loads straight into
 * registers) or TMA-pipelined (persistent blocks of 16 or 32 columns per tile, each
 * keeping the next tiles in flight through tensor-map copies into shared memory, every
 * wait bounded).  choice[2]: choice[0] = columns per block, choice[1] = form (0 direct,
 * 1 TMA-pipelined).  At plan time every candidate runs inside the plan's own extension
 * step (one function, synthetic inputs allocated for the purpose, 3 warm-up and 10
 * timed steps) and the fastest step is kept; us[5] (NULL allowed) receives the step
 * times in microseconds of direct 16, 32, 64, then TMA 16, 32 (0 for a candidate that
 * cannot run; all zeros when the plan has no such transform, or no memory was left
 * for the tuning inputs, which keeps {16, 0}).  Where the TMA form cannot run (an
 * intermediate not 16-byte aligned, no tensor-map encoder in the driver), a plan set to
 * it runs the direct form with the same width. */
fc2d_status fc2d_tuning(fc2d_plan_t plan, int32_t* choice, float* us);
/* Set the choice (choice[2]: columns 16, 32 or 64 with form 0, 16 or 32 with form 1;
 * FC2D_ERR_ARG otherwise), for tests and for callers that fix the launch shape; calls
 * after it use the new shape. */
fc2d_status fc2d_tuning_set(fc2d_plan_t plan, const int32_t* choice);

/* FP64 throughput probe (no operation of the paper): `blocks` blocks of 256 threads on
 * `stream`, each thread running 8 independent fused multiply-add chains of `iters`
 * steps, writing one value per thread to out_dev [blocks * 256].  *flops receives the
 * floating-point operations launched (2 per fused multiply-add); timing the launch with
 * events gives the FP64 rate the Fourier Forwarding roofline divides by. */
fc2d_status fc2d_probe_fp64(double* out_dev, int blocks, int64_t iters, double* flops,
                            void* stream);

/* Plan groups: the extension + DFT of several domains (uneven grids and function
 * counts) in one launch.  fc2d_group_create keeps the plans (not owned: destroy the
 * group before them).  fc2d_group_extend_coeffs runs fc2d_extend_coeffs of every plan
 * i on n_f[i] functions, f_grid_dev[i] / f_bdry_dev[i] (f_bdry_dev itself, or an entry,
 * may be NULL: interior data only) / fhat_dev[i] as for that call, as one CUDA graph
 * launched on `stream`, in one of two forms:
 *   branches:   every plan's whole call on its own branch, concurrently;
 *   persistent: the strip-point values (Sections 3.2-3.4) of all mixed-form members
 *               from one persistent kernel whose CTAs take work items (plan, range of
 *               normals, function) from a queue, longest first; then every plan's row
 *               and column DFTs on its own branch (FP64 members: their whole call).
 * The graph is captured on the first call, after earlier work on the device has
 * finished and the plans' workspaces are allocated.  With mixed-form members both forms
 * are captured and timed on the call's inputs (the persistent kernel's CTA shape, 256
 * threads two per SM or 512 one per SM, timed first) and the faster is kept.  The graph
 * is replayed while n_f, every pointer and every plan's workspace stay the same; a call
 * with other arguments, or after a direct call on a member plan grew that plan's
 * workspace, captures anew.  A plan may appear once in a group (FC2D_ERR_ARG
 * otherwise).  Calls on one group must not overlap in time on different streams (the
 * plans' workspaces are shared).  The result equals the separate calls bit for bit.
 * fc2d_group_tuning: choice[0] the kept form (0 branches, 1 persistent), choice[1] the
 * persistent kernel's threads per CTA (0 before the first capture or without mixed-form
 * members); us[4]: microseconds per launch of the persistent kernel with 256 and 512
 * threads, of the branches graph and of the persistent graph (0 for what was not
 * timed).  fc2d_group_tuning_set fixes the choice for later captures ({form, threads},
 * threads 256 or 512; NULL: tune again) and makes the next call capture anew. */
typedef struct fc2d_group_s* fc2d_group_t;
fc2d_status fc2d_group_create(const fc2d_plan_t* plans, int n, fc2d_group_t* out);
fc2d_status fc2d_group_extend_coeffs(fc2d_group_t group, const int* n_f,
                                     const double* const* f_grid_dev,
                                     const double* const* f_bdry_dev, void* const* fhat_dev,
                                     void* stream);
fc2d_status fc2d_group_tuning(fc2d_group_t group, int32_t* choice, float* us);
fc2d_status fc2d_group_tuning_set(fc2d_group_t group, const int32_t* choice);
void fc2d_group_destroy(fc2d_group_t group);

void fc2d_destroy(fc2d_plan_t plan);

/* Text of the last error on this host thread ("" if none). */
const char* fc2d_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FC2D_H */
