/*
 * ls.h -- C-ABI of libls, a GB300 (sm_103a) implementation of the sparsifying-preconditioned
 * iterative solve of the discretized Lippmann-Schwinger equation of
 *   L. Ying, "Sparsifying Preconditioner for the Lippmann-Schwinger Equation", arXiv:1408.4495.
 *
 * Problem (Sec. 1, eq. ls; Sec. 2.1, eqs. lsd/lso):  (I + K omega^2 m) u = g on the grid
 * (Sec. 5, ls_setup_laplace: (I + K V) u = g with the Laplace kernel; wherever omega^2 m
 * appears below, read V for such a context)
 * x_i = i h, i in {1..n}^d, h = 1/(n+1), d in {2, 3}, K(i,j) = k_{i-j} the Nystrom weights
 * of the Green's function.  Preconditioner (Sec. 2.2, eq. PC): u <= M^{-1} [A;B] g with
 * M = [A + C omega^2 m ; B], factored by nested dissection (Sec. 2.2, Sec. 3.2).
 * Iteration (Sec. 3.3): GMRES to a relative residual tolerance (1e-6 in the paper).
 *
 * Conventions shared by every entry point:
 *  - Every function returns ls_status.  None aborts, throws or exits; on failure the
 *    message is available from ls_last_error().
 *  - Arrays of complex numbers are interleaved (re, im) doubles ("double _Complex" layout),
 *    in C order over the grid (last index fastest), right-hand sides outermost: element
 *    (r, i) of an nrhs x n^d array is at [r * n^d + i].
 *  - Any array argument may be a host pointer or a device pointer of the current device;
 *    the library tells them apart with cudaPointerGetAttributes.  Host arrays are copied
 *    inside the call; device arrays are read / written in place on the context's stream.
 *    Exceptions: the host computations ls_k0_weight, ls_general_support,
 *    ls_general_boundary_stencils and ls_general_rows, and the arrays of ls_general_sketch
 *    and ls_general_setup, take host arrays only.
 *  - The caller owns every array it passes; the library keeps no pointer to them after the
 *    call returns.  The context owns all device memory it allocates.
 *  - A context is not thread-safe; distinct contexts may be used from distinct threads.
 *  - Calls are synchronous with respect to the host: when a call returns, its outputs
 *    (host or device) are complete.  The one exception is ls_factor, which only enqueues the
 *    factorization on the context's stream (see there); the calls that read the factors
 *    (ls_solve, ls_precond, ls_export_factors) wait for it and report its errors.
 */
#ifndef LS_H_
#define LS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LS_OK = 0,
  LS_EINVAL = 1,    /* invalid argument (size, dimension, NULL pointer, 1 - m <= 0, ...) */
  LS_ENOMEM = 2,    /* device or host allocation failed */
  LS_ECUDA = 3,     /* a CUDA call failed; message has the CUDA error string */
  LS_ENOCONV = 4,   /* GMRES did not reach the tolerance within max_iter; outputs are filled */
  LS_ESTATE = 5,    /* call out of order (e.g. ls_solve before ls_factor) */
  LS_ETIMEOUT = 6,  /* a bounded device wait gave up (the tensor-core front update of
                       ls_factor); the context stays usable */
  LS_EBUFFER = 7    /* m is not zero within b+1 layers of the boundary (Sec. 2.1, Sec. 3.1) */
} ls_status;

typedef enum {
  LS_PREC_FP64 = 0,  /* every step in FP64 complex ("plain" path) */
  LS_PREC_MIXED = 1, /* FP32 complex operator apply, stencil, fronts and solves; FP64 Arnoldi
                        and Hessenberg least squares; the outer residual g - A u (refinement)
                        with the operator in float-float arithmetic (LS_PREC_FF) */
  LS_PREC_FF = 2     /* ls_apply only: the FFT operator in float-float arithmetic (each real an
                        unevaluated sum of two FP32 numbers, about 48 significant bits), FP64
                        at the boundary */
} ls_prec;

typedef struct {
  int dim;       /* d: 2 or 3 */
  int n;         /* points per dimension; 2n (the FFT length) must be a power of two, 48 or 96
                    (n = 24, 48: radix-3 passes); 16 <= n <= 2048 (2D), 8 <= n <= 128 (3D) */
  int buffer_b;  /* b of Sec. 3.1: width (in grid steps) of the layer where m vanishes, >= 1;
                    0 selects the default 2 */
  int restart;   /* GMRES restart length; 0 selects 50 */
  int max_iter;  /* cap on GMRES iterations per right-hand side; 0 selects 500 */
  ls_prec prec;  /* arithmetic of the path, see ls_prec */
  int k0_rule;   /* weight k_0 of the singular point of the Nystrom table (Sec. 2.1), an
                    ls_k0_rule below: 0 = LS_K0_BALL (the default of a zero-initialised
                    struct), 1 = LS_K0_CORRECTED (fourth order up to a log); it enters the
                    operator, the symbol, C = alpha K(mu, mu) and the point sources */
  int front_fmt; /* arithmetic of the fronts' Schur products under LS_PREC_MIXED, an
                    ls_front_fmt below: 0 = LS_FRONT_3XTF32 (the default of a zero-initialised
                    struct), 1 = LS_FRONT_FP32; ignored under LS_PREC_FP64 */
} ls_grid;

/* Fronts under LS_PREC_MIXED are stored in FP32.  LS_FRONT_3XTF32: the Schur-complement
 * products with >= 64 rows and >= 16 inner columns run on the tensor cores (tcgen05
 * kind::tf32) with each operand split into two TF32 parts (hi*hi + hi*lo + lo*hi), which
 * keeps FP32 accuracy; LS_FRONT_FP32: every product on the CUDA cores.  Single-TF32 and BF16
 * fronts (LS_FRONT_TF32, LS_FRONT_BF16) are not built: their 1e-3 / 1e-2 relative error
 * would loosen the preconditioner that the iteration counts rely on; setup returns
 * LS_EINVAL for them. */
typedef enum { LS_FRONT_3XTF32 = 0, LS_FRONT_FP32 = 1, LS_FRONT_TF32 = 2, LS_FRONT_BF16 = 3 } ls_front_fmt;

typedef struct ls_ctx ls_ctx; /* opaque */

typedef struct {
  int iters;        /* GMRES iterations (one preconditioner + one operator apply each) */
  int refinements;  /* number of FP64 residual evaluations after the first cycle */
  double rel_resid; /* |g - (I + K omega^2 m) u| / |g| at the end: FP64 storage and norms; the
                       operator K inside it is the FP64 one under LS_PREC_FP64 and the
                       float-float one (about 48 significant bits) under LS_PREC_MIXED */
  int converged;    /* 1 if rel_resid <= tol */
} ls_info;

/*
 * ls_setup -- Sec. 2.1 (grid, k_t, k_0), Sec. 1 (FFT of the convolution), Sec. 3.1 (stencils).
 * Builds the Nystrom table k_t, the Fourier symbol of its (2n)^d circulant embedding, the
 * 3^d stencils alpha (eqs. Fmin, Emin, Cmin; the centre coefficient made real positive) and
 * C = alpha K(mu, mu), and the nested-dissection structure.  Tables that depend only on
 * (d, n, omega, b, k0_rule) are cached inside the library and reused by later contexts.
 *   g       grid description (copied); an unknown prec, k0_rule or front_fmt, or a front
 *           format that is not built, gives LS_EINVAL.
 *   omega   angular frequency, > 0.
 *   m       n^d real doubles, C order: the medium m(x_i) (index of refraction 1 - m).  Host or
 *           device pointer; copied.  Must vanish on the b+1 outermost layers (else LS_EBUFFER)
 *           and satisfy 1 - m > 0 (else LS_EINVAL).
 *   stream  cudaStream_t to run on, or NULL for a stream owned by the context.
 *   out     receives the context; *out is NULL on failure.
 */
ls_status ls_setup(const ls_grid* g, double omega, const double* m, void* stream, ls_ctx** out);
/*
 * ls_setup_laplace -- Sec. 5: the 3D Laplace equation with a compactly supported potential,
 * (-Delta + V) u = f, in Lippmann-Schwinger form (I + K V) u = K f with the Green's function
 * 1 / (4 pi r): k_t = h^3 / (4 pi h |t|), k_0 = a^2 / 2 (a = h (3 / (4 pi))^(1/3), the integral
 * of G over the ball of volume h^3, the omega -> 0 limit of the Helmholtz weight).  Every
 * later step is the Helmholtz one with V in place of omega^2 m: the stencils are built from
 * this kernel (Sec. 5: the preconditioner applies without modification), M = [A + C V; B],
 * and ls_solve / ls_apply / ls_precond work on (I + K V).  ls_rhs_plane_wave is refused
 * (LS_ESTATE); right-hand sides come from ls_rhs_point_source or the caller.
 *   g       grid description (copied); g->dim must be 3 (else LS_EINVAL).
 *   V       n^3 real doubles, C order: the potential V(x_i).  Host or device pointer; copied.
 *           Must be finite (else LS_EINVAL) and vanish on the b+1 outermost layers (else
 *           LS_EBUFFER); any sign (Sec. 5 takes V negative and of order 1/h^2).
 *   stream, out   as for ls_setup.
 */
ls_status ls_setup_laplace(const ls_grid* g, const double* V, void* stream, ls_ctx** out);

/*
 * ls_factor -- Sec. 2.2 eq. PC, Sec. 3.1 eq. ABop, Sec. 3.2: assembles M = [A + C omega^2 m; B]
 * into the nested-dissection fronts and computes their partial LU factorizations (pivoting
 * restricted to the fully-summed rows of each front).  FP32 fronts under LS_PREC_MIXED,
 * FP64 under LS_PREC_FP64.  May be called again (e.g. to time it); LS_ESTATE if c is NULL.
 * Asynchronous: the factorization is enqueued on the context's stream and the call returns;
 * a later ls_rhs_plane_wave overlaps it.  The next ls_solve or ls_precond waits for it and
 * reports its errors (LS_EINVAL for an exactly singular front, LS_ETIMEOUT if a bounded
 * device wait expired); after such an error the context needs ls_factor again.
 */
ls_status ls_factor(ls_ctx* c);
/*
 * ls_set_medium -- a new medium m (n^d doubles, C order, host or device; V for a Laplace
 * context) on the context's grid, frequency and kernel, with the checks of ls_setup
 * (LS_EINVAL, LS_EBUFFER; the context is unchanged on failure).  The tables that depend only
 * on (d, n, omega, b, k0_rule) -- symbol, stencils, nested-dissection structure -- and the
 * device buffers are kept, so a sequence of media on one grid costs no setup.  Drops the
 * factorization (ls_factor must run again before ls_solve) and a general-domain
 * preconditioner (ls_general_setup must run again).
 */
ls_status ls_set_medium(ls_ctx* c, const double* m);
/*
 * ls_export_factors / ls_import_factors -- checkpoint of a factorization, e.g. a serving
 * cache spilled to host memory.  The blob is a 64-byte header (grid, b, precision, k0_rule,
 * front_fmt, kernel, omega, a 64-bit hash of the FP64 potential) followed by the factored
 * fronts, the whole state the solves read.
 *   ls_export_factors: *size receives the blob's size; with out != NULL and capacity >= *size
 *     the blob is written to out (host array).  LS_ESTATE before ls_factor (or for a
 *     general-domain context), LS_EINVAL for a short capacity or a device pointer; reports
 *     the errors of a factorization still in flight.
 *   ls_import_factors: in (host array, size bytes) must come from a context with the same
 *     grid, b, precision, k0_rule, front_fmt, kernel, omega and medium (LS_EINVAL otherwise);
 *     the context is then factored, as if ls_factor had run, without repeating the work.
 */
ls_status ls_export_factors(ls_ctx* c, void* out, size_t capacity, size_t* size);
ls_status ls_import_factors(ls_ctx* c, const void* in, size_t size);

/*
 * ls_rhs_plane_wave -- Sec. 1 eq. ls, Sec. 2.1 eq. lsd: g = K(-omega^2 m u_I) with the
 * incident plane wave u_I(x) = exp(i omega x . dir), computed on the device in FP64.
 *   nrhs   number of directions, >= 1.
 *   dirs   nrhs x d doubles (unit vectors are not required), host or device.
 *   g_out  nrhs x n^d complex doubles, host or device, written.
 */
ls_status ls_rhs_plane_wave(ls_ctx* c, int nrhs, const double* dirs, double* g_out);
/*
 * ls_rhs_point_source -- Sec. 5: g = K f for delta sources, f = q delta(x - x_p) discretised
 * as q / h^d at the grid point p (unit mass on the cell), i.e. g_r(i) = q_r k_{i - p_r} / h^d,
 * computed on the device in FP64 from the kernel table.  Either kernel.
 *   nrhs       number of sources, >= 1.
 *   points     nrhs x d ints, 0-based grid indices (i_0, .., i_{d-1}) in C order, each in
 *              [0, n) (else LS_EINVAL); host or device.
 *   strengths  nrhs complex doubles q_r (interleaved re, im), host or device, or NULL for 1.
 *   g_out      nrhs x n^d complex doubles, host or device, written.
 */
ls_status ls_rhs_point_source(ls_ctx* c, int nrhs, const int* points, const double* strengths, double* g_out);

/*
 * ls_solve -- Sec. 3.3: right-preconditioned GMRES(restart) on (I + K omega^2 m) u = g with
 * the sparsifying preconditioner, all right-hand sides batched in each launch.  Under
 * LS_PREC_MIXED the inner cycles are flexible GMRES with FP32 preconditioner and operator and
 * FP64 Arnoldi, wrapped in iterative refinement whose residual g - A u is formed in FP64 with
 * the operator in float-float arithmetic; the stopping test is that relative residual.  Requires ls_factor (else LS_ESTATE).
 *   rhs    nrhs x n^d complex doubles (g), host or device.
 *   tol    relative residual tolerance, > 0.
 *   u_out  nrhs x n^d complex doubles, host or device, written (best iterate on LS_ENOCONV).
 *   info   nrhs entries, may be NULL.
 */
ls_status ls_solve(ls_ctx* c, int nrhs, const double* rhs, double tol, double* u_out, ls_info* info);

/*
 * ls_far_field -- exterior evaluation after the solve.  With u = u_I + u_s the total field
 * (u_I the plane wave of direction dir, u_s the scattered field that ls_solve returns for
 * g = ls_rhs_plane_wave(dir)), the scattered field outside the domain is
 * u_s(x) = -int G(x - y) omega^2 m(y) u(y) dy (Sec. 1, eq. ls), and as r = |x| -> infinity
 * in the direction theta, u_s(x) ~ e^{i omega r} r^{-(d-1)/2} u_inf(theta) with
 *   u_inf(theta) = -c_d h^d sum_i e^{-i omega theta . x_i} omega^2 m_i u(x_i),
 *   c_2 = e^{i pi/4} / sqrt(8 pi omega), c_3 = 1 / (4 pi)   (FP64 on the device).
 * Helmholtz contexts only (LS_ESTATE for ls_setup_laplace).
 *   nrhs   number of incident waves, >= 1.
 *   dirs   nrhs x d doubles: the incident directions the scattered fields belong to.
 *   us     nrhs x n^d complex doubles: the scattered fields (ls_solve's u_out).
 *   nobs   number of observation directions, >= 1.
 *   obs    nobs x d doubles: observation directions theta (unit vectors).
 *   out    nrhs x nobs complex doubles, written: out[r * nobs + k] = u_inf(theta_k) of wave r.
 * Host or device pointers.
 */
ls_status ls_far_field(ls_ctx* c, int nrhs, const double* dirs, const double* us, int nobs, const double* obs,
                       double* out);
/*
 * ls_k0_weight -- Sec. 2.1: the weight k_0 of the singular point of the Nystrom table, on the
 * host in FP64 (no context, no device work).
 *   rule LS_K0_BALL:      the integral of G over the disk / ball of area / volume h^d
 *                         (second-order accurate; the default of ls_grid.k0_rule).
 *   rule LS_K0_CORRECTED: the one-point correction of the trapezoidal rule (fourth order up
 *                         to a log, as Sec. 2.1 states): the weight for which the corrected
 *                         rule integrates G f exactly for a Gaussian f of width 8 h.
 *   dim 2 or 3; omega >= 0 (0 is the 3D Laplace kernel of Sec. 5; 2D needs omega > 0);
 *   h > 0.  out: 2 doubles (re, im).  LS_EINVAL on bad arguments.
 */
typedef enum { LS_K0_BALL = 0, LS_K0_CORRECTED = 1 } ls_k0_rule;
ls_status ls_k0_weight(int dim, double omega, double h, int rule, double* out);
/*
 * Sec. 4, general domains (host computations in FP64, no context, no device work).
 * ls_general_support: the unknowns of the general-domain method, the grid points within
 *   infinity distance b + 1 of supp(m) (the support with the buffer that the rectangular
 *   method keeps at the box boundary).  m: n^d doubles (C order), mask: n^d bytes written
 *   (1 = unknown).
 * ls_general_boundary_stencils: the stencils of the boundary points of the unknowns (those
 *   with a neighbour, at infinity distance 1, that is not an unknown): alpha = the unit
 *   minimiser of |alpha T(mu(i), :)|, mu(i) the neighbours among the unknowns, T the sketch
 *   (K omega^2 m) R of the rows of K omega^2 m by r >= 3^d Gaussian columns.
 *   mask: n^d bytes as written by ls_general_support; T: (number of unknowns) x r complex
 *   doubles, rows in increasing flat index of the unknowns; alpha: (number of unknowns) x 3^d
 *   complex doubles written (offset index sum_a (t_a + 1) 3^(d-1-a); zero for interior points
 *   and for offsets that are not unknowns; the coefficient at offset 0 real positive);
 *   boundary: (number of unknowns) ints written, 1 for boundary points.
 *   LS_EINVAL on bad arguments or when a smallest singular value is not simple.
 */
ls_status ls_general_support(int dim, int n, const double* m, int b, unsigned char* mask);
ls_status ls_general_boundary_stencils(int dim, int n, const unsigned char* mask, const double* T, int r,
                                       double* alpha, int* boundary);
/*
 * ls_general_sketch -- Sec. 4.1: the sketch T = (K omega^2 m) R on the unknowns of a general
 * domain, computed with the context's FP64 operator apply on the device (the potential V in
 * place of omega^2 m for a Laplace context).  Column q of R, extended by zero off the
 * unknowns, is convolved; row k of T is the result at the k-th unknown.
 *   c     a context of the full grid (ls_setup / ls_setup_laplace; no factorization needed).
 *   mask  n^d bytes (C order, nonzero = unknown), as written by ls_general_support.
 *   r     number of columns, >= 1.
 *   R     (number of unknowns) x r complex doubles (row-major, rows in increasing flat index
 *         of the unknowns), read.
 *   T     (number of unknowns) x r complex doubles, same layout, written; the input of
 *         ls_general_boundary_stencils.
 * mask, R and T are host arrays (LS_EINVAL for device pointers).  With no unknowns nothing is
 * written.  Works on the context's stream and returns when T is written.
 */
ls_status ls_general_sketch(ls_ctx* c, const unsigned char* mask, int r, const double* R, double* T);
/*
 * ls_general_setup -- Sec. 4: makes the context's preconditioner the general-domain one.
 * Rows of M and [A;B] become per point: an interior point of the unknowns (all 3^d
 * neighbours are unknowns) keeps the rectangular interior stencil and C omega^2 m; a boundary
 * point of the unknowns takes its stencil alpha_i (B(i, mu(i)), no C term); a point off the
 * unknowns takes the identity row, so the unknowns decouple from the rest of the box and the
 * nested dissection of the box factors M restricted to them.  The operator stays the box's:
 * m vanishes off the unknowns, so the box solution restricted to the unknowns is the
 * general-domain solution, and the box adds one block with identity diagonal to the
 * preconditioned operator (at most one more GMRES iteration).
 *   mask      n^d bytes (nonzero = unknown), as written by ls_general_support.
 *   alpha     (number of unknowns) x 3^d complex doubles, boundary (number of unknowns)
 *             ints: the outputs of ls_general_boundary_stencils.
 * Host arrays (LS_EINVAL for device pointers).  LS_EINVAL when a point flagged interior has a
 * neighbour off the unknowns or a boundary stencil has no positive centre.  Drops the
 * factorization: ls_factor must run again before ls_solve.  ls_stencils still reports the
 * class tables.
 */
ls_status ls_general_setup(ls_ctx* c, const unsigned char* mask, const double* alpha, const int* boundary);
/*
 * ls_general_rows -- the host step of ls_general_setup (no context, no device work): the
 * stencil of every grid point in the box embedding of Sec. 4.
 *   mask, alpha, boundary  as for ls_general_setup; alpha_interior: 3^d complex doubles, the
 *                          rectangular interior stencil (row (3^d - 1) / 2 of ls_stencils).
 *   rows      n^d x 3^d complex doubles written (offset index as for ls_stencils): e_0 off the
 *             unknowns, alpha_i at boundary points, alpha_interior at interior points.
 *   interior  n^d bytes written, 1 at interior points (the rows that carry C omega^2 m).
 * LS_EINVAL on bad arguments, when a point flagged interior has a neighbour off the unknowns
 * or off the grid, or when a boundary stencil's centre is not positive.
 */
ls_status ls_general_rows(int dim, int n, const unsigned char* mask, const double* alpha, const int* boundary,
                          const double* alpha_interior, double* rows, unsigned char* interior);
/*
 * ls_fault_alloc -- host-side fault injection for tests of the error paths (no GPU fault is
 * ever induced): the k-th device allocation of the library after this call (k >= 1,
 * process-wide, counted before the caching allocator is consulted) fails as if the device
 * were out of memory, so the call that made it returns LS_ENOMEM with the word "injected"
 * in its message.  k = 0 disarms.  LS_EINVAL for k < 0.
 */
ls_status ls_fault_alloc(long k);
/* Message of the last failed call on c (or of the last failed ls_setup when c is NULL).
 * Valid until the next call on c. */
const char* ls_last_error(const ls_ctx* c);

/* Releases every resource of c.  NULL-safe. */
void ls_free(ls_ctx* c);

/* ---------------------------------------------------------------------------------------
 * Inspection entry points: the individual steps of the path, exposed so that each can be
 * checked on its own.  Same pointer and layout conventions as above.
 * --------------------------------------------------------------------------------------- */

/* Sec. 2.1: k_t for t in [0, n]^d (the table is even in every component), (n+1)^d complex
 * doubles in C order, written to out (host or device). */
ls_status ls_kernel_table(ls_ctx* c, double* out);

/* Sec. 3.1 / Sec. 2.2: alpha for each of the 3^d point classes and C for the interior class.
 * Class index sum_a (cls_a + 1) 3^(d-1-a), cls_a = -1 on the low face of axis a, +1 on the
 * high face, 0 otherwise; coefficient index sum_a (t_a + 1) 3^(d-1-a) for offset t.
 * alpha_out: 3^d x 3^d complex doubles (zero outside mu), c_out: 3^d complex doubles.
 * Host pointers only. */
ls_status ls_stencils(ls_ctx* c, double* alpha_out, double* c_out);

/* Sec. 2.1 eq. lso: out = (I + K omega^2 m) in, nrhs vectors, in the arithmetic prec
 * (LS_PREC_MIXED = FP32 complex inside, LS_PREC_FF = float-float inside, FP64 at the
 * boundary). */
ls_status ls_apply(ls_ctx* c, int nrhs, const double* in, double* out, ls_prec prec);

/* Sec. 2.2 eq. PC, right-hand factor: out = [A;B] in (the 3^d-point stencil of each point's
 * class), in the arithmetic prec (LS_PREC_MIXED in 2D rounds in to FP32 first, as the solver's
 * vectors are). */
ls_status ls_stencil_apply(ls_ctx* c, int nrhs, const double* in, double* out, ls_prec prec);

/* Sec. 2.2 eq. PC: out = M^{-1} [A;B] in, with the factors of ls_factor (their precision).
 * With the FP32 factors and the refinement of ls_set_precond_refine on, in is rounded to
 * FP32 first (as the solver's Arnoldi vectors are) and the result carries one refinement
 * step. */
ls_status ls_precond(ls_ctx* c, int nrhs, const double* in, double* out);

/* One step of iterative refinement of the FP32 preconditioner (the paper solves eq. PC
 * exactly; its FP32 factors leave a residual that grows with the separators' conditioning):
 * z = M^{-1} r, then z += M^{-1} (r - M z) with r = [A;B] v, both solves with the FP32
 * factors and the residual in FP32.  FGMRES allows the preconditioner to change between
 * iterations.
 *   mode  1: on for every application of the mixed path; 0: off; -1: automatic (the
 *         default: the first application after each ls_factor estimates
 *         E = |[A;B] v - M z| / |[A;B] v| for its first right-hand side and refinement is on
 *         from then on while that factorization lasts when E > 0.02); -2: no change.
 *   err   when not NULL receives E of the current factorization, -1 when none was taken.
 * A forced mode (0 or 1) persists across factorizations.  No effect on the FP64 path or on
 * general domains (their stencils are per point).  LS_EINVAL for a mode outside -2..1. */
ls_status ls_set_precond_refine(ls_ctx* c, int mode, double* err);

/* Sizes of the nested-dissection factorization (Sec. 3.2). */
typedef struct {
  int levels;              /* depth of the separator tree + 1 */
  int fronts;              /* number of fronts */
  int max_front;           /* largest front order (separator + boundary) */
  int64_t factor_entries;  /* complex entries stored for all fronts (padded) */
  double factor_flops;     /* real flops of the partial factorizations (padded shapes) */
  double solve_bytes;      /* bytes of factor read by one forward + backward solve */
  /* bytes moved by one forward sweep (leaves to root) and one backward sweep of the solve,
   * split into the factor blocks read once per sweep and the vector traffic per
   * right-hand side (gathers, children's updates, front vectors), padded shapes */
  double fwd_factor_bytes, fwd_bytes_per_rhs;
  double bwd_factor_bytes, bwd_bytes_per_rhs;
} ls_nd_stats;

ls_status ls_get_nd_stats(ls_ctx* c, ls_nd_stats* out);

/* ---------------------------------------------------------------------------------------
 * Instrumentation (process-wide, for measurement; the paper has no counterpart).
 * ls_profile_start resets the per-kernel-class launch counters of the library and, when
 * timed_class is neither NULL nor empty, brackets every launch of that kernel class ("*":
 * of every class) with a pair of CUDA events recorded on the stream the kernel is launched on.
 * ls_profile_stop waits for those events and writes a NUL-terminated JSON report
 *   {"counts": {class: launches, ...}, "total": n,
 *    "timed": {"class": name, "launches": k, "ms": summed device time},
 *    "ms_by_class": {class: summed device time, ...}}
 * into report (truncated to capacity bytes; report may be NULL).  Not thread-safe with
 * respect to other calls of the library running at the same time.
 * --------------------------------------------------------------------------------------- */
ls_status ls_profile_start(const char* timed_class);
ls_status ls_profile_stop(char* report, int capacity);

/* ---------------------------------------------------------------------------------------
 * Autotuner (the paper has no counterpart: launch shapes of this implementation).
 *
 * ls_autotune -- times, on this context's factorization and solve, the alternatives of the
 * launch-shape choices that have no single best value across grids: the trailing-matrix size
 * from which the blocked front LU updates in two levels, the smallest FP32 Schur product
 * (rows) given to the tensor cores, the largest front factored Gauss-Jordan style in one CTA,
 * how many CTAs per SM the split of a solve sweep level aims at, and the smallest FP32
 * forward and backward solve levels (rows of their products, at least 32) run on the tensor
 * cores, and the largest bottom solve level (columns of its product, up to 256; rows up to
 * 64) run one CTA per front.  The last three default to -1, automatic per solve: tensor-core
 * levels from 64 rows in 3D or with more than 16 right-hand sides, none for at most 16 in
 * 2D; one-CTA-per-front levels up to 256 columns with more than 16 right-hand sides, up to
 * 64 with at most 16.  A coordinate search
 * keeps each alternative that is more than 2 % faster (the fastest of 2 factorizations / 3
 * solves of nrhs right-hand sides, CUDA events).  The choice is applied to c, kept for every
 * later context of the same (dim, n, prec, kernel) in this process, and, when the
 * environment variable LS_TUNE_FILE names a file, written there (one JSON object per line)
 * and read back by the first ls_setup of a later process.  Leaves c factored (with the
 * chosen shapes).  FFT radices (8, 4, 2, 3) and the right-hand-side batch widths (16 per
 * item, 64 per launch) are fixed.
 *   nrhs     right-hand sides of the timed solves, >= 1.
 *   report   NUL-terminated JSON: the choice and every timing (truncated to capacity bytes;
 *            may be NULL).
 * ls_tune_info -- the context's current choices as a JSON object (no device work).
 * ls_set_tune -- applies choices given as a JSON object with any of the keys of
 *   ls_tune_info (other keys are ignored; missing keys keep their values) to c only, e.g. to
 *   pin a shape or to compare two.  A factorization in flight is awaited first; the next
 *   ls_factor uses the factorization choices, the next solve the solve choices (a change of
 *   a factorization choice needs a new ls_factor to take effect).  LS_EINVAL when a value is
 *   out of range (two_level_min <= 0, tc_min_rows < 1, sweep_ctas outside 1..4,
 *   gj_max_own outside 1..32, tcs_min_rows or tcs_bwd_min_rows neither -1 nor >= 1,
 *   small_max_k outside -1..256).
 * --------------------------------------------------------------------------------------- */
ls_status ls_autotune(ls_ctx* c, int nrhs, char* report, int capacity);
ls_status ls_tune_info(const ls_ctx* c, char* report, int capacity);
ls_status ls_set_tune(ls_ctx* c, const char* json);

/* ---------------------------------------------------------------------------------------
 * Allocation-free operator apply (the paper has no counterpart: this is a deployment aid).
 *
 * Computes the same y = (I + K omega^2 m) x as ls_apply(c, nrhs, x, y, LS_PREC_FP64) but
 * allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.  It exists for
 * callers that cannot allocate device memory when they need the operator, e.g. code running
 * while another component owns the device memory pool, loops in which cudaMalloc/cudaFree
 * would synchronise the device, or deployments that forbid allocation after start-up.
 *
 *   x, y   nrhs x n^d complex doubles (interleaved), DEVICE pointers owned by the caller, on
 *          the device that was current when the context was set up; that device must be
 *          current at the call.  Host pointers, arrays of another device and a call made with
 *          another device current are rejected with LS_EINVAL.
 *
 * The FFT passes' intermediate buffer is a fixed 64 MiB array compiled into the library
 * (it occupies 64 MiB on every GPU that loads the library until the process exits).  One
 * call needs nrhs * n * 2n complex doubles in 2D (32 right-hand sides at n = 256) and
 * nrhs * (n^2 * 2n + n * (2n)^2) in 3D; larger requests return LS_EINVAL with the sizes in
 * the message.  No part of that buffer has to start at zero: every pass writes what the
 * next one reads.  All calls, on every context of the process, share the one buffer per
 * GPU, so calls whose work overlaps on the same GPU (different threads or streams) race
 * and give wrong results; serialise them.
 *
 * The first call on each device looks up the buffer's device address
 * (cudaGetSymbolAddress, which may load the library's module on that device); make that
 * first call outside any CUDA stream capture.  Synchronous like every other entry point.
 * --------------------------------------------------------------------------------------- */
ls_status ls_apply_noalloc(ls_ctx* c, int nrhs, const double* x, double* y);

#ifdef __cplusplus
}
#endif

#endif /* LS_H_ */
