/*
 * pp.h -- C ABI of a GB300 (sm_103a) library for the action of the matrix
 * inverse square root and square root, f(A) b with f(z) = z^{-1/2} or z^{1/2},
 * by polynomially preconditioned Arnoldi / Lanczos (Frommer, Ramirez-Hidalgo,
 * Schweitzer, Tsolakis, "Polynomial preconditioning for the action of the
 * matrix square root and inverse square root").
 *
 * Problem statement (Sec. 1, Sec. 2 Prop. 2.1, Sec. 3 Eq. (3.1)): given a
 * sparse A in C^{n x n} with no eigenvalue on (-inf, 0] and a vector b,
 * compute the principal A^{-1/2} b or A^{1/2} b.  A polynomial q ~ z^{-1/2}
 * (Sec. 5) turns the Krylov process onto A q(A)^2, whose spectrum clusters
 * around 1, and
 *     A^{-1/2} b = (A q(A)^2)^{-1/2} q(A) b          (left, Algorithm 1)
 *                = q(A) (A q(A)^2)^{-1/2} b          (right, Algorithm 2)
 *     A^{1/2} b  = A^{-1/2} (A b)                    (Sec. 4).
 *
 * Conventions for every entry point
 *   - Every call returns an int status: PP_OK (0) or a negative pp_status.
 *     pp_strerror() names it.  A failed call leaves the handle usable.
 *   - Pointers with suffix _d are DEVICE pointers (e.g. torch CUDA tensors'
 *     data_ptr()), owned by the caller; the library never frees them.
 *     Pointers with suffix _h are HOST pointers.
 *   - Device work is ordered on the handle's CUDA stream (the `stream`
 *     argument of pp_create_*; NULL = the legacy default stream).  A call
 *     returns after its work is queued, except where stated.  Handles are
 *     not thread-safe; distinct handles may be used from distinct threads.
 *   - Real vectors are FP64 (PP_F64) at the API; complex vectors are
 *     interleaved complex128 (PP_C128).  The arithmetic inside is chosen by
 *     pp_opts.precision.
 *   - Grid vectors are ordered with x fastest: idx = (k*Ny + j)*Nx + i.
 */
#ifndef PP_H
#define PP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pp_ctx *pp_handle;

typedef enum {
  PP_OK = 0,
  PP_ERR_INVALID_ARG = -1,   /* bad pointer, size, enum value or option         */
  PP_ERR_NOT_CONVERGED = -2, /* m_max reached; x holds the last iterate         */
  PP_ERR_NONPRIMARY = -3,    /* q <= 0 somewhere on [a,b]: the result would be a
                                non-primary root (Sec. 5, after Thm. 5.1)       */
  PP_ERR_SINGULAR = -4,      /* A^{-1/2} requested for a numerically singular A */
  PP_ERR_OOM = -5,           /* device allocation failed                        */
  PP_ERR_CUDA = -6,          /* a CUDA runtime call failed                      */
  PP_ERR_TIMEOUT = -7,       /* a bounded device wait ran out                   */
  PP_ERR_STATE = -8,         /* call out of order (e.g. pp_apply before
                                pp_build_poly)                                  */
  PP_ERR_UNSUPPORTED = -9    /* valid request this library does not implement   */
} pp_status;

typedef enum { PP_F64 = 0, PP_F32 = 1, PP_C64 = 2, PP_C128 = 3 } pp_dtype;

typedef enum {
  PP_INVSQRT = -1,
  PP_SQRT = 1,
  PP_SIGN = 2  /* sign(Q) b = Q (Q^2)^{-1/2} b for a PP_WILSON4D_Q2 handle (A = Q^2)
                  (Sec. 6, Example 2) */
} pp_func;

typedef enum {
  PP_CHEBYSHEV = 0,      /* Sec. 5.1: interpolant at deg+1 first-kind nodes of [a,b] */
  PP_RITZ_LEJA = 1,      /* Sec. 5.2: interpolant at the deg+1 Ritz values of A
                            (Newton form, Leja order)                             */
  PP_HARMONIC_RITZ = 2,  /* Sec. 5.2: same at the deg+1 harmonic Ritz values      */
  PP_LSQ_CONTOUR = 3,    /* Sec. 5.3: least-squares approximation on a contour     */
  PP_NODES = 4           /* interpolant at caller-given nodes (pp_set_poly_nodes)     */
} pp_poly_kind;

typedef enum {
  PP_LAPLACE2D5 = 0,         /* 5-point Dirichlet Laplacian, dims = {Nx, Ny}      */
  PP_LAPLACE3D7 = 1,         /* 7-point Dirichlet Laplacian, dims = {Nx, Ny, Nz}  */
  PP_CONVDIFF3D7_UPWIND = 2, /* 7-point upwind -Lap u + c.grad u, c = (c,c,c)>0,
                                params[0] = c*h; row: (6+3ch) u_c - (1+ch) (u at
                                i-1, j-1, k-1) - (u at i+1, j+1, k+1)             */
  PP_WILSON4D_DHD = 3,       /* A = D^H D of a Wilson-type operator on a periodic
                                4D lattice, dims = {L0, L1, L2, L3} (see
                                pp_create_stencil)                                */
  PP_WILSON4D_Q2 = 4         /* A = Q^2, Q = Gamma_5 D(m_w, mu), the kernel of the
                                overlap operator's sign function (Sec. 6,
                                Example 2); params = {m_w, mu}                    */
} pp_stencil_kind;

typedef enum { PP_LEFT = 0, PP_RIGHT = 1 } pp_side;

typedef enum {
  PP_PREC_F64 = 0,   /* vectors, chain and basis in IEEE FP64                    */
  PP_PREC_DW = 1,    /* vectors, chain and basis as double-word FP32 pairs
                        (hi + lo, ~48-bit significand, 8 bytes per real): FP64-
                        grade accuracy on the FP32 pipes                          */
  PP_PREC_MIXED = 2  /* double-word for the start vector, the leading basis vectors
                        and the result; FP32 chain, FP32 basis and FP32 vector
                        updates from the first stopping check at which
                        est * rho/(1-rho) * 4 u_32 * kappa_pre <= tol, where
                        est = the stopping estimate, rho = its observed
                        per-step decay, u_32 = 2^-24 and kappa_pre = the
                        ratio of the ends of the image of z q(z)^2 (FP32
                        rounding is amplified by about kappa_pre).  H_m, its
                        coefficients and the small solve stay FP64.  Single
                        applications (pp_op_apply, pp_poly_apply) run in FP32
                        under this setting.                                  */
} pp_precision;

typedef enum {
  PP_ORTH_AUTO = 0,     /* Lanczos for Hermitian A, CGS2 Arnoldi otherwise        */
  PP_ORTH_LANCZOS = 1,  /* three-term recurrence, no reorthogonalization          */
  PP_ORTH_CGS2 = 2,     /* classical Gram-Schmidt twice against the whole basis   */
  PP_ORTH_DCGS2 = 3     /* classical Gram-Schmidt twice with the second pass
                           delayed by one step: the operator is applied to the
                           candidate after its first pass, whose second pass,
                           normalization (beta^2 = ||u||^2 - ||V^T u||^2) and the
                           first pass of the next candidate are formed from one
                           sweep of inner products (V^T u, V^T y, u.u, u.y) and
                           applied in one update sweep, the new column's
                           coefficients following from linearity and the
                           Arnoldi relation of the earlier columns; two sweeps
                           over the basis per step instead of three plus a
                           normalization (a stopping check adds one inner-
                           product sweep).  Same H_m and basis as CGS2 up to
                           rounding.  Where the q(A) chain amplifies rounding
                           strongly its results level off above CGS2's (a
                           degree-15 Ritz q on a 281,903-node graph
                           Laplacian: 1.3e-8 against 2e-10 in FP64, 2.3e-7
                           against 7e-9 in double-word); with Chebyshev q on
                           convection-diffusion the two agree.  Left
                           preconditioning of real operators
                           (PP_ERR_UNSUPPORTED otherwise); batched solves use
                           CGS2.  No counterpart in the paper, which
                           reorthogonalizes without saying how (Sec. 6,
                           Example 3).                                          */
} pp_orth;

typedef struct pp_opts {
  int32_t side;         /* pp_side, default PP_LEFT                                  */
  int32_t precision;    /* pp_precision, default PP_PREC_F64                         */
  int32_t orth;         /* pp_orth, default PP_ORTH_AUTO                             */
  int32_t check_every;  /* k of the stopping rule ||f_m - f_{m+k}|| / ||f_{m+k}||
                           (Sec. 6, Example 1); 0 = max(1, floor(64/(deg+1)))      */
  int32_t profile;      /* 1: time every operator launch of the polynomial chain
                           with CUDA events (pp_stats.chain_*)                       */
  int32_t two_pass;     /* 1: two-pass Lanczos (Hermitian A, Lanczos only): the first
                           pass keeps three basis vectors and H_m, the second
                           regenerates v_1..v_m from the stored coefficients and
                           accumulates x; twice the operator work, O(n) memory
                           instead of O(m n).  mvms counts both passes.            */
  int32_t clenshaw;     /* how q(A) v is evaluated, in deg q operator steps:
                           0 (default): the Newton form of q at its Leja-ordered
                           interpolation nodes x_i by a Horner scheme (Sec. 5.2's
                           representation; for PP_CHEBYSHEV the first-kind nodes,
                           the same q), each step w <- ((A - x_i)/cap) w + a_i
                           cap^i v with cap = (max x_i - min x_i)/4: three vector
                           streams per step.  1: for PP_CHEBYSHEV the matrix
                           Clenshaw recurrence of the Chebyshev series (Sec. 5.1),
                           four streams per step (ignored for the Ritz kinds).   */
  int32_t halo;         /* 1: in the FP32 arithmetic of a solve (PP_PREC_MIXED after
                           the switch) on a 2D/3D stencil grid with nx % 4 == 0,
                           the Horner steps of q(A) after the first run two at a
                           time in one kernel: the tile of w with a two-point halo
                           and the tile of v with a one-point halo are loaded into
                           shared memory by the tensor memory accelerator, the
                           first step is evaluated on the tile plus a one-point
                           halo there and the second on the tile (three vector
                           streams per pair instead of six; the same values bit
                           for bit).  Real-node q only (Chebyshev, real Ritz
                           values); other cases run single steps.  Measured
                           slower than single steps on every workload here (the
                           pair kernel is bound by its shared-memory reads: 128^3
                           convection-diffusion 142.5 -> 129.9 solves/s, 256^3
                           11.70 -> 10.83, 2048^2 Laplacian equal).  No
                           counterpart in the paper.  0 (default): single steps.  */
  int32_t reserved[4];
} pp_opts;

typedef struct pp_stats {
  int32_t status;         /* same value pp_apply returned                           */
  int32_t iters;          /* Krylov dimension m of the returned iterate             */
  int32_t checks;         /* small f(H_m) solves performed                          */
  int32_t breakdown;      /* 1 if h_{m+1,m} vanished (Krylov space invariant)       */
  int64_t mvms;           /* products with A, counted as in Tables 1-3              */
  int64_t inner_products; /* length-n inner products and norms in the loop          */
  double est_err;         /* last ||f_m - f_{m-k}|| / ||f_m|| (inf if one check)    */
  double beta0;           /* ||q(A) b|| (left) or ||b|| (right)                     */
  double ms_total;        /* device time of the call, CUDA events                   */
  int64_t launches;       /* kernels launched by the call                           */
  int64_t chain_launches; /* operator launches (A and the Clenshaw steps of q(A))   */
  double chain_bytes;     /* their algorithmic HBM bytes: vectors read + written,
                             plus the CSR arrays for CSR handles                    */
  double chain_ms;        /* their summed device time (opts.profile = 1, else 0)    */
  int32_t switch_iter;    /* PP_PREC_MIXED: Krylov dimension at which the loop
                             moved to FP32 (-1: never); 0 for the other settings */
  int32_t reserved_i;
  double orth_ms;         /* opts.profile = 1: device time of the orthogonalization
                             (inner products, updates, norms) of every Krylov step,
                             CUDA events around each step's                       */
  double small_ms;        /* opts.profile = 1: device time of the stopping checks'
                             small projected solves, CUDA events around each     */
} pp_stats;

/* Defaults for pp_opts (all fields). */
void pp_default_opts(pp_opts *opts);

/*
 * Create a handle for a CSR matrix (Sec. 1: A sparse).  n rows/columns;
 * rowptr_d[n+1] (int64, rowptr_d[0] = 0), col_d[nnz] (int32, 0-based),
 * val_d[nnz] of dtype PP_F64 (PP_C128 is not supported).  The arrays are
 * referenced, not copied (PP_PREC_DW keeps a double-word copy of val,
 * PP_PREC_MIXED also an FP32 one), and must stay alive and unchanged for
 * the handle's lifetime.  Under PP_PREC_DW the CSR step accumulates each row
 * sum and its update in triple-float arithmetic on the FP32 pipes (about
 * 2^-72 of the summands) and rounds the result to a double-word pair, so
 * rows that cancel heavily (a graph Laplacian's) keep FP64-grade accuracy.
 * is_hermitian selects
 * Lanczos under PP_ORTH_AUTO.  Errors: PP_ERR_INVALID_ARG for n <= 0 or NULL
 * pointers, PP_ERR_UNSUPPORTED for other dtypes.
 */
int pp_create_csr(pp_handle *h, int64_t n, const int64_t *rowptr_d, const int32_t *col_d,
                  const void *val_d, int32_t dtype, int32_t is_hermitian, void *cuda_stream);

/*
 * Create a handle for a matrix-free constant-coefficient stencil on a grid
 * with Dirichlet boundary (Sec. 6, Example 1 uses the 3D Laplacian; Sec. 3.2
 * the 2D one).  dims[4] = grid points per direction (unused entries ignored);
 * params: PP_CONVDIFF3D7_UPWIND reads params[0] = c*h > 0, the others none
 * (NULL allowed).  links_d must be NULL and dtype PP_F64 for these kinds.
 *
 * PP_WILSON4D_DHD (a stand-in for the lattice QCD kernel of Sec. 6,
 * Example 2, whose configuration is not available): A = D^H D with
 *   (D psi)(x) = (4 + m0) psi(x) - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
 *                                  + (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu) ]
 * on a periodic L0 x L1 x L2 x L3 lattice, dims = {L0, L1, L2, L3}, site
 * s = ((x3 L2 + x2) L1 + x1) L0 + x0, gamma matrices of the Euclidean chiral
 * representation (gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 =
 * [[0, 1], [1, 0]]), params[0] = m0.  links_d: device array of 4 V 3 x 3
 * complex64 matrices (interleaved float re/im), U_mu(s)_{ab} at index
 * ((s * 4 + mu) * 3 + a) * 3 + b, referenced for the handle's lifetime.
 * dtype must be PP_C128: b and x are 12 V complex128 entries, 12 per site in
 * the order spin * 3 + colour.  A is Hermitian positive definite, so
 * PP_ORTH_AUTO runs Lanczos; the vector work runs on the real view (24 V
 * reals), which is exact for real recurrence coefficients.
 *
 * PP_WILSON4D_Q2 (Sec. 6, Example 2): A = Q^2 with Q = Gamma_5 D(m_w, mu),
 * D the operator above with m0 = m_w = params[0] and chemical potential
 * mu = params[1] (|mu| <= 20): the hop to x + e_3 (direction 3, gamma_4)
 * carries e^{mu}, the hop to x - e_3 carries e^{-mu}; Gamma_5 = diag(1, 1,
 * -1, -1) on spin.  Same links, dims and vector layout.  For mu != 0, Q is
 * non-Hermitian and the handle runs complex Arnoldi (classical Gram-Schmidt
 * twice with complex coefficients, complex H_m and small solve, a q with
 * complex coefficients): PP_ORTH_LANCZOS and two_pass are refused
 * (PP_ERR_INVALID_ARG), pp_build_poly's PP_LSQ_CONTOUR takes a closed
 * contour around the complex Ritz values (see pp_set_poly_lsq) and
 * PP_CHEBYSHEV needs interval_ab; under PP_PREC_MIXED the switch rule's
 * kappa_pre is estimated at each stopping check from the eigenvalues of H_m
 * (the Ritz values of A q(A)^2: ratio of the extreme moduli, times 4).  For
 * mu = 0, Q^2 = Q^H Q is Hermitian positive definite and behaves like
 * PP_WILSON4D_DHD.  pp_apply with PP_SIGN returns sign(Q) b.
 */
int pp_create_stencil(pp_handle *h, int32_t kind, const int64_t dims[4], const double *params,
                      const void *links_d, int32_t dtype, void *cuda_stream);

/* Replace the handle's options; PP_ERR_INVALID_ARG for out-of-range values. */
int pp_set_opts(pp_handle h, const pp_opts *opts);

/*
 * Build q with deg q = degree (paper: d = degree + 1 nodes) of the given kind
 * on [a,b] = interval_ab_h[0..1] (host array), the interval enclosing
 * spec(A) (Sec. 5.1).  interval_ab_h = NULL: the exact spectral interval of
 * the Laplacian and convection-diffusion stencils (Sec. 6, Example 1 formula
 * and its convection-diffusion analogue); for the other Hermitian handles
 * (Wilson, Hermitian CSR) the extreme Ritz values of 200 Lanczos steps from a
 * fixed pseudo-random start, with a lowered by 5 % and b raised by 1 %
 * (device work on the handle's stream; the call synchronises it).
 * Non-Hermitian CSR handles need an interval.  degree = 0 gives constant q,
 * i.e. plain Arnoldi/Lanczos.  The positivity of q on [a,b] is checked on a
 * dense grid (Sec. 5.1, last paragraph); PP_ERR_NONPRIMARY if it fails.
 * 0 <= degree <= 128.
 *
 * PP_RITZ_LEJA / PP_HARMONIC_RITZ (Sec. 5.2): degree + 1 Arnoldi steps on
 * A itself (classical Gram-Schmidt twice, in the handle's precision;
 * double-word for PP_PREC_MIXED) from a fixed pseudo-random start vector:
 * entry i of the real view is (s_i >> 11) 2^-52 - 1, s_i the SplitMix64
 * output for the state 0x5EED + (i + 1) 0x9E3779B97F4A7C15.  The nodes are
 * the eigenvalues of H_d, or of H_d + h_{d+1,d}^2 H_d^{-T} e_d e_d^T for
 * harmonic Ritz values.  Hermitian handles read H_d as the Lanczos matrix T
 * (diagonal and sub-diagonal; eigenvalues by bisection, harmonic ones from
 * the pencil (T^2 + h^2 e_d e_d^T, T)); other handles take the Hessenberg
 * H_d (Francis QR; complex values come in conjugate pairs).  q is then built
 * as by pp_set_poly_nodes from these nodes.  If the Krylov space of the
 * start vector is invariant earlier (small n), fewer nodes are used and
 * deg q drops accordingly (pp_get_poly reports it).  [a,b] (given, or the
 * closed form, or for Hermitian handles the extreme Ritz values lowered by
 * 5 % / raised by 1 %) only serves the positivity check and the image
 * interval.  A non-Hermitian handle without either is checked at its Ritz
 * values and the nodes only (the indication of Sec. 5.2: between them an
 * interpolant may turn negative where A has no eigenvalues); the quadrature
 * of the small solve then spans the image at those points widened by 1e6
 * both ways, and PP_PREC_MIXED stays in double-word for real handles (the
 * image does not bound the FP32 amplification; complex handles estimate it
 * from H_m, see PP_WILSON4D_Q2).
 * The node run costs degree + 1 operator applications and allocates a basis
 * of degree + 2 vectors in the workspace.
 */
int pp_build_poly(pp_handle h, int32_t degree, int32_t kind, const double *interval_ab_h);

/*
 * Autotuner (no counterpart in the paper, which fixes the degree per
 * experiment): choose deg q for a target tolerance and build q as
 * pp_build_poly would (interval from an earlier pp_build_poly, else the
 * closed form or the Lanczos estimate).  For every candidate degree up to
 * max_degree the image interval [lo, hi] of z q(z)^2 (Prop. 3.2) gives the
 * Chebyshev bound 2 ((sqrt(k)-1)/(sqrt(k)+1))^m, k = hi/lo, for the number of
 * steps m; the predicted time is m steps of (2 deg + 1) operator passes plus
 * the orthogonalization (Lanczos: constant; CGS2: growing with m), in vector
 * passes at 6 TB/s, plus 3 us per kernel launch and 40 us per stopping check,
 * and the fastest degree is taken (*degree_out).
 * For stencil handles in PP_PREC_DW / PP_PREC_MIXED it then times the
 * operator kernel with blocks of 64, 128, 256, 512 threads on the handle's stream
 * (CUDA events, synchronising) and keeps the fastest for later calls.
 * Errors: as pp_build_poly; PP_ERR_INVALID_ARG for tol outside (0, 1).
 */
int pp_autotune(pp_handle h, double tol, int32_t max_degree, int32_t *degree_out);

/*
 * Read back the polynomial: coeffs_h[0..*ncoeffs-1] (PP_CHEBYSHEV: the
 * coefficients c_i of q = sum c_i T_i((2z-a-b)/(b-a)); other kinds: the
 * coefficients of q in the real basis R_i of pp_set_poly_nodes, for real
 * nodes the Newton coefficients a_i; the nodes from pp_get_poly_nodes;
 * for the complex q of a complex operator (PP_WILSON4D_Q2 with mu != 0) the
 * real parts of its Newton coefficients), ab_h[2] = [a,b], image_h[2] =
 * [min, max] of z q(z)^2 on [a,b] (the interval of Prop. 3.2; at the
 * nodes and Ritz values where q was built from them without an interval).
 * Any output pointer may be NULL; cap = capacity of coeffs_h.  deg q =
 * *ncoeffs - 1.
 */
int pp_get_poly(pp_handle h, double *coeffs_h, int32_t cap, int32_t *ncoeffs, double *ab_h,
                double *image_h);

/*
 * q = the interpolant of z^{-1/2} (principal branch) at caller-given nodes
 * (Sec. 5.2 builds them from Ritz values; this call takes them from the
 * caller, e.g. Ritz values of an Arnoldi run started from b): deg q =
 * count - 1 <= 128.  nodes_re_h / nodes_im_h (host; nodes_im_h may be NULL
 * for real nodes): real values or complex conjugate pairs, all with Re > 0
 * (Hermitian handles: real only).  The nodes are put in Leja order (largest
 * modulus first, then each time the node farthest from the taken ones in
 * product distance; a pair is taken as its Im > 0 member followed by its
 * conjugate), and the Newton form takes them in the reverse of that order
 * (pairs kept), so that the Horner scheme, which applies the factor of the
 * last node first, applies the factors in Leja order; q is written in the
 * real basis R_0 = 1, R_{i+1} = (z - x_i)
 * R_i for a real node, R_{i+1} = (z - Re x_i) R_i, R_{i+2} = |z - x_i|^2 R_i
 * for a pair, which for real nodes is the Newton form q = sum_i a_i
 * prod_{l<i} (z - x_l), a_i the divided differences.  q(A) v is evaluated by
 * the matching backward (Horner) recurrence of deg q operator steps, each
 * scaled by cap = a quarter of the diameter of the node set.  [a,b] =
 * interval_ab_h, else the closed form of the stencils, else the extreme real
 * parts of the nodes lowered by 5 % / raised by 1 %; Re q must be positive
 * there and at the nodes (the condition of Sec. 5.2, checked on these
 * points), and the image of |z q(z)^2| over them sets the quadrature of the
 * small solve.  Host only (no device work).  Errors: PP_ERR_INVALID_ARG for
 * count out of range, non-finite nodes, a complex node without its
 * conjugate, complex nodes of a Hermitian handle, a bad interval;
 * PP_ERR_NONPRIMARY for a node with Re <= 0, coincident nodes or Re q <= 0
 * on the checked points.  The handle's kind becomes PP_NODES.
 */
int pp_set_poly_nodes(pp_handle h, const double *nodes_re_h, const double *nodes_im_h, int32_t count,
                      const double *interval_ab_h);

/*
 * q = the least-squares approximation of z^{-1/2} of degree `degree` on the
 * discretized contour z_1..z_N (Sec. 5.3): q minimizes sum_i |z_i^{-1/2} -
 * q(z_i)|^2, computed through the orthonormal basis that the Arnoldi process
 * on diag(z_1..z_N) from the vector of ones / sqrt(N) yields (alpha = P^*
 * z^{-1/2}).  pts_re_h / pts_im_h (host; pts_im_h may be NULL): N >= degree +
 * 1 points, none on (-inf, 0].  Real operators: the set must be symmetric
 * about the real axis (then q is real; PP_ERR_UNSUPPORTED otherwise: a
 * complex q of a real A would need complex vectors), real for Hermitian
 * handles.  Complex operators (PP_WILSON4D_Q2 with mu != 0): any set; q is
 * complex, its Newton form is taken at degree + 1 Leja points of the set
 * without conjugate pairing, and like a complex Ritz q it only indicates the
 * spectrum (wide quadrature; under PP_PREC_MIXED kappa_pre from H_m).
 * Re q must be positive at every point (Sec. 5.3 takes this as the
 * indication that q is in the right half-plane inside the contour;
 * PP_ERR_NONPRIMARY otherwise).  The device evaluates q in the Newton form of
 * pp_set_poly_nodes at degree + 1 Leja points chosen among the contour points
 * (q interpolates its own values there, so it is the same polynomial; the
 * call checks that the form reproduces q on all points to 1e-8 of max |q|).
 * pp_build_poly(h, degree, PP_LSQ_CONTOUR, interval) builds the contour
 * itself: the segment [a, b] when a real spectral interval is known (given,
 * closed form, or the Hermitian estimate), else around the Ritz values of
 * max(60, degree + 1) Arnoldi steps (as Example 3; Ritz values within 1e-4
 * of the largest modulus of zero, the null space of a singular A, are left
 * out): their convex hull made
 * symmetric about the real axis, the part inside |z| < r_min (half the
 * smallest Ritz modulus) replaced by the arc of that circle, max(2000,
 * 20 (degree + 1)) points at equal arc length; for a complex operator the
 * complex Arnoldi run's Ritz values and their convex hull as a closed curve
 * (no symmetrisation), kept out of |z| < r_min the same way.  Host only
 * (pp_set_poly_lsq).
 * Errors: PP_ERR_INVALID_ARG for bad points or degree.
 */
int pp_set_poly_lsq(pp_handle h, int32_t degree, const double *pts_re_h, const double *pts_im_h, int32_t npts);

/*
 * The interpolation nodes of q (host output): *kind = its pp_poly_kind,
 * nodes_re_h / nodes_im_h [0..*nnodes-1] = the nodes in the order of the
 * Newton form the device evaluates (reverse Leja order, see
 * pp_set_poly_nodes; for PP_CHEBYSHEV its deg q + 1
 * first-kind nodes of [a,b]), *scale = cap of pp_set_poly_nodes.  Any output
 * pointer may be NULL; cap = capacity of the node arrays.
 * Errors: PP_ERR_STATE before pp_build_poly.
 */
int pp_get_poly_nodes(pp_handle h, int32_t *kind, double *nodes_re_h, double *nodes_im_h, int32_t cap,
                      int32_t *nnodes, double *scale);

/*
 * x = f(A) b (Algorithm 1 or 2 by opts.side; Sec. 4 for PP_SQRT), iterating
 * until the stopping estimate is below tol or m = m_max.  b_d, x_d: device
 * vectors of n entries of the handle's vector dtype (nrhs > 1: n x nrhs,
 * column-major; stencil and CSR handles solve them as independent processes
 * in lockstep through pp_apply_batch, m_max <= 1024, a CSR handle's
 * operator steps as block SpMM; Wilson handles one after another, stats
 * summed, iters and est_err the largest); x_d must
 * not alias b_d.  On PP_ERR_NOT_CONVERGED x_d still holds the last
 * iterate.  stats (host, may be NULL) is filled on return.  Blocks the
 * calling thread at each stopping check (a few bytes read back).
 * The kernels of the steps between two stopping checks are captured once
 * as a CUDA graph per (step range, precision phase) and replayed by later
 * calls on the handle (results bitwise equal to direct launches); the
 * graphs are recorded on a private non-blocking stream the handle creates
 * on first use, launched on the handle's stream, held by the handle (freed
 * by pp_destroy) and dropped when its workspace, q, options or tol change;
 * opts.profile = 1 launches the kernels directly.
 * f = PP_SIGN (PP_WILSON4D_Q2 handles, nrhs = 1; Sec. 6, Example 2):
 * x = sign(Q) b = Q (Q^2)^{-1/2} b, the solve for (Q^2)^{-1/2} b followed by
 * one FP64 application of Q on the device (stats describe the solve).
 * Errors: PP_ERR_STATE before pp_build_poly, PP_ERR_INVALID_ARG for NULL or
 * aliasing pointers, m_max < 1 or > 4096, tol < 0, non-finite ||b||;
 * PP_ERR_UNSUPPORTED for PP_SIGN on another handle kind.
 */
int pp_apply(pp_handle h, int32_t f, const void *b_d, int64_t nrhs, int32_t m_max, double tol,
             void *x_d, pp_stats *stats);

/*
 * Same as pp_apply for HOST vectors b_h, x_h: copies b to the device, solves
 * and copies x back, all inside the call (used for end-to-end timing).
 * Returns after x_h is written.
 */
int pp_apply_host(pp_handle h, int32_t f, const double *b_h, int64_t nrhs, int32_t m_max,
                  double tol, double *x_h, pp_stats *stats);

/*
 * Batched solves: x_i = f_i(A_i) b_i for `count` handles at once, every
 * handle with nrhs[i] right-hand sides (b_d[i]: n_i x nrhs[i] FP64, column-
 * major, device; x_d[i] likewise), each right-hand side an independent
 * Krylov process (Algorithm 1 or 2 as in pp_apply).  All processes advance in
 * lockstep: every kernel launch covers the whole batch, so a batch costs the
 * launches of one solve; a process that meets its stopping estimate is masked
 * out of later launches.  Stencil handles are grouped by polynomial degree
 * and orthogonalization; the right-hand sides of a CSR handle form groups
 * of their own, up to 16 each, whose operator steps are one block SpMM
 * launch (each row's column indices and values read once for all of the
 * group's vectors; real CSR, PP_F64 values; the small solve uses the
 * handle's own quadrature rule, so each process gives pp_apply's iterate).
 * Groups run concurrently on internal streams that are
 * ordered after the work queued on cuda_stream, which waits for them before
 * the call returns (the call blocks until done).  Every handle must be a 2D
 * or 3D stencil or a CSR matrix (PP_ERR_UNSUPPORTED otherwise), have called pp_build_poly,
 * and share the precision and side options of handles[0]
 * (PP_ERR_INVALID_ARG otherwise).  With PP_PREC_MIXED a group moves to FP32
 * when the switching rule holds for all of its unconverged processes.
 * stats (host, count entries, may be NULL): per handle, iters = the largest
 * Krylov dimension over its right-hand sides, mvms / inner_products summed
 * over them, est_err the largest estimate; ms_total, launches and the
 * chain_* operator accounting of the whole batch (chain_ms with
 * handles[0]'s opts.profile = 1; the groups then run one after another
 * instead of concurrently, so that the timed launches do not overlap).  Returns
 * PP_ERR_NOT_CONVERGED if any process reached m_max (1 <= m_max <= 1024).
 */
int pp_apply_batch(const pp_handle *handles, int32_t count, const int32_t *f, const void *const *b_d,
                   const int64_t *nrhs, void *const *x_d, int32_t m_max, double tol, void *cuda_stream,
                   pp_stats *stats);

/*
 * A batch plan: the processes of pp_apply_batch (same arguments: handles,
 * f, nrhs, m_max, cuda_stream) set up once and solved by pp_batch_apply for
 * any number of right-hand-side sets.  pp_batch_create groups the processes
 * as pp_apply_batch does and allocates every group's device state (vectors
 * padded to whole reduction chunks, the growing Krylov basis, scratch,
 * tables); pp_batch_apply then launches no allocation unless a basis has to
 * grow.  The kernels of the Krylov steps between two stopping checks of a
 * group, with the check's small solve, are captured as a CUDA graph on their
 * first run and replayed by later solves (one graph launch per group and
 * check instead of a few hundred kernel launches; results bitwise equal to
 * direct launches); the host still reads each group's status records at
 * every check.  opts.profile = 1 on handles[0] launches directly.
 * No counterpart in the paper (which solves one problem at a time).
 * Errors: as pp_apply_batch; pp_batch_apply returns PP_ERR_STATE if a
 * handle's q or options changed after pp_batch_create (create a new plan).
 * The handles must outlive the plan.  pp_batch_destroy(NULL) is a no-op.
 */
typedef struct pp_batch_ctx *pp_batch;
int pp_batch_create(pp_batch *batch, const pp_handle *handles, int32_t count, const int32_t *f,
                    const int64_t *nrhs, int32_t m_max, void *cuda_stream);
/* b_d[i], x_d[i]: as pp_apply_batch, for handle i of the plan; stats as pp_apply_batch. */
int pp_batch_apply(pp_batch batch, const void *const *b_d, void *const *x_d, double tol, pp_stats *stats);
void pp_batch_destroy(pp_batch batch);

/* y_d = A x_d (one operator application in the handle's precision). */
int pp_op_apply(pp_handle h, const void *x_d, void *y_d);

/* y_d = q(A) x_d by the matrix Clenshaw recurrence (Sec. 5.1), deg q
   operator applications fused with the recurrence's vector updates.        */
int pp_poly_apply(pp_handle h, const void *x_d, void *y_d);

/*
 * y_d = q(A) x_d, the same computation as pp_poly_apply, for callers that
 * must not allocate device memory.  (The paper has no counterpart: this is a
 * deployment variant.)  Who needs it: a process whose device memory is all
 * owned by an arena or caching allocator (a framework that has reserved the
 * GPU, so a cudaMalloc from this library would fail or fragment it), and
 * latency-critical loops that forbid cudaMalloc/cudaFree after start-up
 * because those calls can block and synchronise the device.
 *
 * pp_poly_apply takes its three Clenshaw buffers (five in PP_PREC_DW, which
 * also converts x and y) from the handle's workspace, allocated on first use.
 * This variant takes them from one fixed array compiled into the library:
 * 5 * PP_STATIC_MAX_N entries of 8 bytes (10 MiB), which every GPU that
 * loads the library holds until the process exits.  It calls no cudaMalloc
 * or cudaFree and no allocating library routine.
 *
 * Arguments as pp_poly_apply: x_d, y_d are caller-owned device vectors of n
 * FP64 entries; y_d must not alias x_d.  Work is queued on the handle's
 * stream; the call returns after queueing it.
 * Limits and errors: PP_ERR_INVALID_ARG if n > PP_STATIC_MAX_N or for bad
 * pointers; PP_ERR_STATE before pp_build_poly; PP_ERR_UNSUPPORTED for CSR
 * handles in PP_PREC_DW or PP_PREC_MIXED (their converted values would need
 * an allocation) and for Wilson handles (they need a sixth vector).
 * Device: the handle's kernels use the copy of the array on the device that
 * was current when the handle was created; a call made while another device
 * is current is refused (PP_ERR_INVALID_ARG).
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current).  Make that first call
 * before any stream capture.  The call makes no other synchronising request
 * (for a CSR handle the algorithmic byte count of its statistics leaves the
 * matrix entries out until another entry point has read nnz).
 * Sharing: all calls in the process use the same array.  Every scratch entry
 * a call reads was written earlier in the same call, so nothing left by a
 * previous call affects the result; but calls whose work overlaps on the GPU
 * (other streams, other handles, other host threads) race on the array and
 * must be serialised by the caller.
 */
#define PP_STATIC_MAX_N 262144
int pp_poly_apply_static(pp_handle h, const void *x_d, void *y_d);

/*
 * Read back the quadrature rule of the small projected solve: H^{-1/2} e_1 =
 * sum_k wt_h[k] (H + sig_h[k] I)^{-1} e_1, a trapezoid rule for
 * z^{-1/2} = (2/pi) int_0^inf (t^2 + z)^{-1} dt (an integral representation
 * of the inverse square root; the paper uses a Schur square root instead,
 * Sec. 3.1), in u = log t after the substitution u = u_c + a sinh(w) whose
 * tails decay double-exponentially (the plain rule in u where that needs
 * fewer nodes).  It is built with q and checked there to a few 1e-15
 * relative on the image interval widened by 10^3 (10^6 for Ritz q without an
 * interval) and, for non-Hermitian A, on the sector |arg z| <= theta that
 * the nodes of q ask for.  *K = number of nodes; up to cap entries are
 * written.
 */
int pp_get_quadrature(pp_handle h, double *sig_h, double *wt_h, int32_t cap, int32_t *K);

/* Release the handle and its device workspace (NULL is a no-op). */
void pp_destroy(pp_handle h);

/* Static, NUL-terminated name of a status code. */
const char *pp_strerror(int32_t status);

/* Message of the last failed call on this thread ("" if none). */
const char *pp_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
int32_t pp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PP_H */
