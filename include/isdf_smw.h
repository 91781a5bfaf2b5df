/*
 * isdf_smw.h - C ABI of the GB300 (sm_103a) ISDF-SMW inverse dielectric library.
 *
 * The method (arXiv 2403.12340, "A fast low-rank inversion algorithm of
 * dielectric matrix in GW approximation"):
 *   - the orbital-pair functions M_(r; i,j) = psi_i(r) psi_j(r) (i occupied,
 *     j unoccupied; Eq. Omega text) are compressed by interpolative separable
 *     density fitting at N_mu grid points, M ~ P C with C = M[mu, :]
 *     (Eq. ISDF, Eq. MatrixExpressionISDF);
 *   - chi0 = 2 M Omega^-1 M^T and eps = I - V chi0 (Eq. matrices) are never
 *     formed; instead eps^-1 = I + V P K P^T with the N_mu x N_mu capacitance
 *     K = (1/2 (C Omega^-1 C^T)^-1 - P^T V P)^-1
 *     (Eq. epsilon_with_SMW; K of Section "Cubic scaling algorithm";
 *     Algorithm 3 steps 1-3).
 *
 * Conventions shared by every entry point
 *   - Real (Gamma-point, Eq. 8) float64 data, column-major, grid index fastest:
 *     grid point (x, y, z) is row r = x + n1 * (y + n2 * z).
 *   - Discretisation (the paper drops quadrature weights; this library's
 *     reading): orbitals are discretely orthonormal (sum_r phi_i phi_j =
 *     delta_ij) and V = F^-1 diag(v_G / dV) F with v_G = 4 pi / |G|^2,
 *     v_0 = 0, dV = L1 L2 L3 / N_r, G = 2 pi (m1/L1, m2/L2, m3/L3).
 *   - Frequencies are on the imaginary axis (Hartree); Omega(i w)^-1 =
 *     diag(D / (D^2 + w^2)), D = e_i - e_j < 0; w = 0 is the static case.
 *   - Device pointers are CUDA global-memory addresses on the context's
 *     device; host pointers are ordinary process memory.  All buffers are
 *     owned by the caller.  The context owns only its workspace.
 *   - Calls are ordered on the context's CUDA stream.  isdf_fit synchronises
 *     that stream once (it returns the numerical rank to the host); the
 *     other calls are asynchronous unless stated otherwise.  The caller must
 *     keep phi and theta alive and unmodified until the next isdf_fit or
 *     isdf_destroy, because later calls read them.
 *   - Every entry point returns ISDF_OK (0) or a negative ISDF_ERR_* code and
 *     never aborts the process; isdf_last_error() describes the last error.
 *     A failed call leaves the context usable (its fit state may be reset).
 *
 * The whitened basis.  isdf_fit factors C C^T = L L^T by Cholesky with
 * diagonal pivoting (rank r <= N_mu) and returns theta = P_r L_r, the
 * auxiliary functions of the r pivot points multiplied by their Cholesky
 * factor, i.e. theta = M C~^T with C~ = L_r^-1 C_r having orthonormal rows.
 * theta spans the same space as P, theta C~ = P C, and the operators G, D
 * and K reported below are expressed in this basis:
 *   eps^-1 = I + V theta K theta^T,  K = -D (I + G D)^-1,
 *   G = theta^T V theta,  D = -2 C~ Omega^-1 C~^T = L_r^-1 (-2 B_rr) L_r^-T.
 * Columns r..N_mu-1 of theta and rows/columns r.. of G, D, K are zero.
 */
#ifndef ISDF_SMW_H
#define ISDF_SMW_H

#include <stdint.h>

#if defined(__GNUC__)
#define ISDF_API __attribute__((visibility("default")))
#else
#define ISDF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct isdf_ctx isdf_ctx;

enum {
  ISDF_OK = 0,
  ISDF_ERR_ARG = -1,        /* null pointer, bad enum or flag */
  ISDF_ERR_SHAPE = -2,      /* non-positive or inconsistent sizes, N_mu > N_r, too large */
  ISDF_ERR_INDEX = -3,      /* interpolation index out of range or repeated */
  ISDF_ERR_NONFINITE = -4,  /* NaN or Inf in an input */
  ISDF_ERR_ORDER = -5,      /* no gap: max occupied energy >= min unoccupied energy */
  ISDF_ERR_NOT_SPD = -6,    /* a capacitance factor lost positive definiteness */
  ISDF_ERR_TIMEOUT = -7,    /* a device-side wait ran out (no hang: kernel returned) */
  ISDF_ERR_CUDA = -8,       /* a CUDA runtime call failed */
  ISDF_ERR_STATE = -9,      /* call out of order (e.g. apply before smw_inverse) */
  ISDF_ERR_NOMEM = -10      /* workspace allocation failed */
};

/* Precision of the path.  FP64: every step in float64 on the FP64 pipe.
 * MIXED: every large contraction (face-split Gram, the triangular solve of
 * the fit as a GEMM with the inverse factor, G, D, the Newton-Schulz
 * capacitance products, theta^T X and theta T) on the tensor cores with
 * operands cut into three BF16 slices and FP32 accumulation, the Coulomb
 * transform of theta in FP32; the points' C C^T, its Cholesky factorisation
 * and triangular inverse in double-float arithmetic on the FP32 pipe (float
 * pairs, about 2^-46 relative per product sum) with FP64 storage; the FFT
 * of the probe block stays in FP64.  Results agree with FP64 to about 1e-6 relative on well-conditioned
 * systems.  Both the BF16 slices and the float pairs keep FP32's exponent
 * range: entries of the matrices they carry must lie within about 1e-30 to
 * 1e30 in magnitude (or be zero); use FP64 for inputs scaled beyond it. */
enum { ISDF_PREC_FP64 = 0, ISDF_PREC_MIXED = 1, ISDF_PREC_MIXED_PAIRS = 2 };
/* MIXED whitens D as L_r^-1 (C_r Omega^-1 C_r^T) L_r^-T, which multiplies
 * the FP32-grade error of the pair products by cond(C C^T); when the fit's
 * factor shows mean(lambda) mean(1/lambda) > 4 for the eigenvalues of
 * C C^T (from ||L_r||_F and ||L_r^-1||_F; this is 1 for a perfectly
 * conditioned C C^T and grows with its condition number) it instead forms
 * S = L_r^-1 C_r diag(sqrt(-2 Omega^-1)) in pair space and D = S S^T, which
 * multiplies that error by cond(L_r) only, at the cost of one more
 * N_mu x N_pairs x N_mu tensor-core GEMM.  MIXED_PAIRS takes the pair-space
 * route always. */

/* Create a context for one periodic grid n1 x n2 x n3 with cell lengths
 * L1, L2, L3 (Bohr).  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream) on the current device, which becomes the context's device.
 * n_i in [2, 512], each a product of primes <= 13.  Allocates nothing large
 * until isdf_fit.  On error *ctx is NULL. */
ISDF_API int isdf_create(isdf_ctx** ctx, int n1, int n2, int n3, double L1, double L2, double L3,
                void* cuda_stream);

/* Free the context and its workspace (after synchronising its stream). */
ISDF_API int isdf_destroy(isdf_ctx* ctx);

/* ISDF fit (Eq. ISDF, Eq. MatrixExpressionISDF; least-squares reading of
 * M = P C): theta = M C~^T with C~ the orthonormalised C of the pivot points.
 *   phi      device, N_r x (n_v + n_c) float64, column-major (ld = N_r):
 *            orbitals, the first n_v occupied.  Read now and by
 *            build_polarizability.
 *   n_v,n_c  numbers of occupied / unoccupied orbitals (>= 1 each).
 *   mu_idx   host or device (told apart by cudaPointerGetAttributes), n_mu
 *            int64 grid indices in [0, N_r), distinct.  A device array is
 *            read after the context stream has synchronised, then copied to
 *            the host, where the indices are checked and the pivot order is
 *            kept; not a device array while a graph is captured.
 *   n_mu     number of interpolation points, 1 <= n_mu <= N_r.
 *   prec     ISDF_PREC_FP64 or ISDF_PREC_MIXED; later calls use the same mode.
 *   theta    device, N_r x n_mu float64 out (ld = N_r); must not alias phi.
 *            Later calls read it: keep it until the next fit.
 *   rank_out host int out (may be NULL): numerical rank r of C C^T.  The
 *            Cholesky stops when the largest remaining pivot falls below
 *            n_mu * 2^-52 * max diag(C C^T); r < n_mu is not an error.
 * Waits once on the host, for the Cholesky factorisation of C C^T: the FP64
 * path synchronises the context stream there; the MIXED path has queued the
 * rest of the fit for the full-rank outcome first and reads the flags
 * through a helper stream.  theta is complete once the context stream has
 * run the call's work. */
ISDF_API int isdf_fit(isdf_ctx* ctx, const double* phi, int n_v, int n_c, const int64_t* mu_idx, int n_mu,
             int prec, double* theta, int* rank_out);

/* Polarizability and Coulomb operators in the ISDF basis (Algorithm 3 steps
 * 1-2 with the direct sum over pairs, Eq. COmegaCstar):
 *   D(w) = -2 C~ Omega(i w)^-1 C~^T and G = theta^T V theta (FFT of theta).
 *   energies host, n_v + n_c float64 (Hartree); occupied ones all below the
 *            unoccupied ones (else ISDF_ERR_ORDER).
 *   omega    host, n_omega imaginary frequencies (Hartree, >= 0).
 *   n_omega  1 .. 4096; the context keeps all D(w).
 *   D_out    device, n_omega x n_mu x n_mu float64 out, or NULL.
 *   G_out    device, n_mu x n_mu float64 out, or NULL.
 * Requires a successful isdf_fit. */
ISDF_API int build_polarizability(isdf_ctx* ctx, const double* energies, const double* omega, int n_omega,
                         double* D_out, double* G_out);

/* build_polarizability for the static case (w = 0) with D computed by the
 * contour integral of Algorithm 2 instead of the sum over pairs:
 * B = C Omega^-1 C^T = (1/pi) Im of the integral of J(z) over the upper
 * half of a contour around the unoccupied energies,
 * J(z) = (Psi_v diag(1/(z - e_v)) Psi_v^T) .* (Psi_c diag(1/(z - e_c)) Psi_c^T),
 * with the conformal map of Algorithm 2 and the midpoint rule with n_nodes
 * nodes; the quadrature error falls like exp(-pi^2 n_nodes / (2 log(Q/q) + 6))
 * (Eq. rel_err_Cauchy; q the gap, Q the width from the highest occupied
 * energy to the top of the unoccupied band).  Costs 2 N_mu^2 (n_v + n_c)
 * FP64 flops per node instead of N_mu^2 n_v n_c.  energies, D_out, G_out
 * as for build_polarizability; the context then holds one frequency
 * (omega_index 0, w = 0).  ISDF_ERR_ARG unless 1 <= n_nodes <= 1024. */
ISDF_API int build_polarizability_contour(isdf_ctx* ctx, const double* energies, int n_nodes, double* D_out,
                                          double* G_out);

/* Nodes that the bound of Eq. rel_err_Cauchy asks for a relative
 * quadrature error tol (0 < tol < 1), from the energies (host, n_v + n_c);
 * negative ISDF_ERR_* on bad arguments or no gap.  The bound's constant is
 * not known, and in practice fewer nodes reach tol. */
ISDF_API int isdf_contour_nodes(const double* energies, int n_v, int n_c, double tol);

/* Host-only pieces of the MIXED capacitance route of smw_inverse, exported
 * so that they can be checked without a GPU.
 *
 * isdf_pair_weight_bounds: bounds of the pair weights 2 d / (d^2 + w^2),
 * d = e_c - e_v, over every occupied v and unoccupied c (the entries of
 * Omega(i w)^-1 in D(w) = -2 C~ Omega(i w)^-1 C~^T, Eq. COmegaCstar), from
 * the extreme energies: the weight is unimodal in d with its peak at d = w,
 * so the extremes over [gap, width] lie at the ends or at w.  In the
 * whitened basis the largest weight bounds the spectral norm of D.
 *   energies host, n_v + n_c float64, occupied first, all occupied ones
 *            below the unoccupied ones (else ISDF_ERR_ORDER).
 *   w        frequency, >= 0.
 *   wmin, wmax host out.
 * Returns ISDF_OK or a negative ISDF_ERR_*. */
ISDF_API int isdf_pair_weight_bounds(const double* energies, int n_v, int n_c, double w, double* wmin,
                                     double* wmax);

/* isdf_ns_schedule: the Newton-Schulz schedule for M = I + G D whose
 * spectrum lies in [1, kappa] (kappa = 1 + |G| |D|, the bounds above and a
 * Gershgorin bound of G): X_0 = alpha I, alpha = 2 / (1 + kappa), then
 * X <- beta_k (2 X - X (M X)) with beta_k = 2 / (2 - e_k^2), from
 * e_0 = (kappa - 1) / (kappa + 1) and e_{k+1} = e_k^2 / (2 - e_k^2), until
 * e_k < 2^-26; step k runs its products on slices[k] BF16 slices (1, 2 or 3;
 * 3 on the last two steps).
 *   kappa      >= 1 (else ISDF_ERR_ARG).
 *   max_steps  room in beta and slices (host out); 12 is always enough.
 * Returns the number of steps, or 0 when the route is not taken (it would
 * need more than 12 steps; smw_inverse then factors). */
ISDF_API int isdf_ns_schedule(double kappa, int max_steps, double* beta, int* slices);

/* SMW capacitance for frequency omega[omega_index] (K of Section "Cubic
 * scaling algorithm", Algorithm 3 step 3), in the singular-B-safe form
 * K = -D (I + G D)^-1.  FP64: K = -Q Q^T, Q = R U^-T, D = R R^T,
 * I + R^T G R = U U^T.  MIXED: X -> (I + G D)^-1 by Newton-Schulz on the
 * tensor cores, then K = -D X; the step schedule comes from rigorous
 * bounds of the spectra of G and D (one host read).  When those bounds ask
 * for more than 12 steps, or during a stream capture, the factorisation
 * route runs instead.
 *   K_out    device, n_mu x n_mu float64 out, or NULL (K is kept in the
 *            context for apply_eps_inv either way).
 * ISDF_ERR_NOT_SPD if a factorisation finds D (or I + R^T G R) not positive
 * definite in floating point. */
ISDF_API int smw_inverse(isdf_ctx* ctx, int omega_index, double* K_out);

/* smw_inverse for every frequency of the last build_polarizability at once
 * (the full-frequency form of Algorithm 3 step 3).  On a MIXED context
 * every Newton-Schulz product of all frequencies is one grouped persistent
 * launch (one schedule, from the largest spectral bound over the
 * frequencies); the batched factorisation route is the fallback.  On an
 * FP64 context the frequencies are queued one after the other.  One
 * synchronisation for the bounds (MIXED) and one at the end.
 *   K_out    device, n_omega x n_mu x n_mu float64 out, or NULL.
 * ISDF_ERR_NOT_SPD names the first frequency whose factor failed. */
ISDF_API int smw_inverse_all(isdf_ctx* ctx, double* K_out);

/* Y = eps^-1(i w) X = X + V theta K theta^T X (Eq. epsilon_with_SMW).
 *   X, Y     device, N_r x n_rhs float64 (ld = N_r); Y may equal X.
 *   n_rhs    >= 1.
 * Requires smw_inverse for the same omega_index. */
ISDF_API int apply_eps_inv(isdf_ctx* ctx, int omega_index, const double* X, int n_rhs, double* Y);

/* apply_eps_inv without any device allocation.  The paper has no
 * counterpart: this entry point is for callers that must not allocate
 * device memory when they call, such as code that runs under a fixed
 * device-memory budget, inside a latency-critical loop where a cudaMalloc or
 * cudaFree (which can synchronise the whole device) is not acceptable, or in
 * a component that is not allowed to own memory.  Everything else needed
 * (theta, K, the Coulomb tables) was allocated earlier by isdf_create,
 * isdf_fit and build_polarizability.
 *   Arguments and result: as apply_eps_inv.  The arithmetic is always FP64:
 *   on an FP64 context it is the same kernels as apply_eps_inv (same numbers
 *   up to the order of the split-K sums); on a MIXED context it applies the
 *   context's FP64 theta and K with those FP64 kernels, while apply_eps_inv
 *   there runs theta^T X and theta T on the tensor cores, so the two agree
 *   to the mixed path's accuracy (about 1e-7 relative), not bit for bit.
 *   Scratch: a file-scope device array of 8 MiB (2^20 doubles), one per GPU
 *   that loads this library, held until the process exits.  A probe column
 *   needs 2 N_mu + N_r + 2 h n2 n3 + 64 N_mu doubles (h = n1/2 + 1, each
 *   term rounded up to 256 bytes); columns are processed as many at a time
 *   as fit.  If one column does not fit the call returns ISDF_ERR_SHAPE and
 *   writes nothing (apply_eps_inv has no such limit).
 *   The first call on a device (and the first after a cudaDeviceReset, which
 *   gives the device a new CUDA context) looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Every call on a device shares the one array and leaves its contents
 *   behind; each call overwrites what it reads.  Calls whose kernels overlap
 *   on the GPU (two streams, two threads, two contexts on the same device)
 *   race on the array: order them on one stream. */
ISDF_API int apply_eps_inv_noalloc(isdf_ctx* ctx, int omega_index, const double* X, int n_rhs, double* Y);

/* ---- Adjoint (gradients through the SMW inverse) -------------------------
 * The differentiated quantity is the screened Coulomb operator in the ISDF
 * basis, W_P = P^T eps^-1 V P = G_P + G_P K_P G_P (Eq. epsilon_with_SMW times
 * V, projected on the interpolation vectors P of Eq. ISDF; G_P = P^T V P,
 * K_P the capacitance in the points basis), as a function of the orbital
 * energies and of the orbital samples at the interpolation points,
 * phi_mu = Phi[mu, :], which enter through C = M[mu, :] and Omega
 * (Eq. COmegaCstar).  The ISDF vectors (theta of the last fit) are held
 * fixed: they are the checkpoint of the forward pass.  The paper states no
 * derivative; these calls apply d(A^-1) = -A^-1 dA A^-1 to
 * K = -D (I + G D)^-1, in FP64 (on a MIXED context G and K carry the mixed
 * path's rounding). */

/* Replace the orbital samples at the interpolation points used by the next
 * build_polarizability (theta and the fit's factor stay).  phimu: device,
 * n_mu x (n_v + n_c) float64, column-major with leading dimension ldp >=
 * n_mu, rows in the order of the fit's mu_idx.  Invalidates the
 * polarizability and every K.  Synchronises the context stream (checks for
 * NaN / Inf: ISDF_ERR_NONFINITE). */
ISDF_API int isdf_set_point_orbitals(isdf_ctx* ctx, const double* phimu, long long ldp);

/* W_P for frequency omega[omega_index] in the points basis (rows and columns
 * in the order of mu_idx; those of non-pivot points, if the rank r < n_mu,
 * are zero).  W_out: device, n_mu x n_mu float64.  Requires smw_inverse for
 * that frequency.  Asynchronous. */
ISDF_API int isdf_screened_basis(isdf_ctx* ctx, int omega_index, double* W_out);

/* Reverse mode: given W_bar = dL/dW_P (device, n_mu x n_mu float64, points
 * order), writes dL/de (grad_energies, device, n_v + n_c float64) and
 * dL/dphi_mu (grad_phimu, device, n_mu x (n_v + n_c) float64, ld n_mu; zero
 * rows at non-pivot points).  Uses the state of the last build_polarizability
 * and smw_inverse for omega_index (call between the forward and any other
 * build_polarizability).  Workspace: 2 r n_v n_c + O(r^2) doubles.
 * Synchronises the context stream. */
ISDF_API int isdf_adjoint(isdf_ctx* ctx, int omega_index, const double* W_bar, double* grad_energies,
                          double* grad_phimu);

/* Reverse mode through the ISDF fit: the same loss, now with the ISDF
 * vectors P = M C^T (C C^T)^-1 a function of the orbitals on the whole grid
 * (Eq. MatrixExpressionISDF, least-squares reading), so that dL/dPhi also
 * carries the change of P, through G = P^T V P:
 *   dL/dG_P = E^T Wbar E (E = I + G_P K_P),  dL/dP = 2 V P dL/dG_P,
 *   dL/dZ = dL/dP A^-1, dL/dA = -sym(A^-1 dL/dP^T P) for Z = M C^T =
 *   (Phi_v Phi_v,mu^T) .* (Phi_c Phi_c,mu^T) and A = C C^T, and on to Phi.
 * theta and the fit's factor are the checkpoint of the forward pass: the
 * backward recomputes the face-split factors, V theta and the rest from
 * the orbitals of the fit, in FP64.
 *   W_bar         device, n_mu x n_mu float64 (points order), dL/dW_P.
 *   grad_energies device, n_v + n_c float64 out (as isdf_adjoint).
 *   grad_phi      device, N_r x (n_v + n_c) float64 out, column-major
 *                 (ld N_r): dL/dPhi on every grid point (the rows of the
 *                 interpolation points include the part through D).
 * Needs a fit of full rank (ISDF_ERR_STATE otherwise) and, like
 * isdf_adjoint, the state of the last build_polarizability and smw_inverse
 * for omega_index.  Workspace: 3 N_r n_mu + O(n_mu^2 + n_mu N_e) doubles.
 * Synchronises the context stream. */
ISDF_API int isdf_adjoint_fit(isdf_ctx* ctx, int omega_index, const double* W_bar, double* grad_energies,
                              double* grad_phi);

/* ---- Static COHSEX self-energies (Algorithm 3 steps 4-7) -------------------
 * Band self-energies of the static COHSEX approximation (Section "GW
 * approximation": Sigma_SEX_X, Sigma_X, Sigma_COH of every band n) from
 * three ISDF fits on one grid, each in its own context:
 *   ctx_vc  the dielectric fit: isdf_fit on the orbitals (n_v occupied), then
 *           build_polarizability with omega[0] = 0 and smw_inverse(0);
 *   ctx_vn  isdf_fit on [Phi_v | Phi] (N_r x (n_v + n_e), n_v "occupied"),
 *           with its own interpolation points: the occupied x all pairs;
 *   ctx_nn  isdf_fit on [Phi | Phi] (n_e "occupied"): the all x all pairs.
 * W_vn = (P_vn^T V P_vc) K (P_vc^T V P_vn), V_vn = P_vn^T V P_vn and
 * W_nn = (P_nn^T V P_vc) K (P_vc^T V P_nn), then by the Hadamard identity
 * (Eq. Hadamard) Sigma_SEX_X(n) = -psi_n^T (W_vn .* Psi_v Psi_v^T) psi_n and
 * Sigma_X(n) = -psi_n^T (V_vn .* Psi_v Psi_v^T) psi_n at the vn points,
 * Sigma_COH(n) = 1/2 psi_n^T (W_nn .* Psi Psi^T) psi_n at the nn points.
 * The quasiparticle energies of Algorithm 3 step 8 are
 * e_n + Sigma_SEX_X(n) + Sigma_X(n) + Sigma_COH(n) - (V_xc)_n.
 *   sigma  device, 3 n_e float64 out: [0, n_e) SEX_X, [n_e, 2 n_e) X,
 *          [2 n_e, 3 n_e) COH.
 * FP64 throughout, on ctx_vc's stream (the three contexts' streams are
 * synchronised first); synchronises at the end.  ISDF_ERR_STATE / _SHAPE
 * for missing steps or mismatched fits. */
ISDF_API int isdf_cohsex(isdf_ctx* ctx_vc, isdf_ctx* ctx_vn, isdf_ctx* ctx_nn, double* sigma);

/* ---- Batched full-frequency runner ----------------------------------------
 * Many systems of different sizes, every frequency of each (the
 * full-frequency form of Algorithm 3 steps 1-3 over a set of systems).
 * The paper has no counterpart: it treats one system at a time.  Each
 * system keeps its own context, CUDA stream and theta for the life of the
 * batch (repeated runs allocate nothing new once the first run has sized the
 * workspaces); a run hands the systems, largest estimated cost first, to a
 * pool of host threads that drive isdf_fit, build_polarizability and
 * smw_inverse_all of one system at a time, so that systems overlap on the
 * GPU. */
typedef struct isdf_batch isdf_batch;
typedef struct {
  int n1, n2, n3;           /* grid */
  double L1, L2, L3;        /* cell lengths (Bohr) */
  const double* phi;        /* device, N_r x (n_v + n_c), ld N_r; kept alive by the caller */
  int n_v, n_c;
  const int64_t* mu_idx;    /* host, n_mu grid indices (copied at create) */
  int n_mu;
  const double* energies;   /* host, n_v + n_c (Hartree; copied at create) */
} isdf_system;

/* Create a batch on the current device: one context, non-blocking stream and
 * theta buffer (N_r x n_mu float64) per system.  prec: ISDF_PREC_FP64 or
 * ISDF_PREC_MIXED for every system.  n_workers: host threads of a run
 * (1..64).  On error *batch is NULL and isdf_batch_last_error(NULL) says
 * why. */
ISDF_API int isdf_batch_create(isdf_batch** batch, const isdf_system* systems, int n_systems, int prec,
                               int n_workers);
ISDF_API int isdf_batch_destroy(isdf_batch* batch);

/* Fit, polarizability and SMW capacitance of every system at the n_omega
 * frequencies omega (host, Hartree, >= 0) on n_workers host threads (0: the
 * number given at create; 1 runs the systems one after the other, which
 * isolates each kernel for timing).  latency_ms (host, n_systems, or
 * NULL): time from the start of the run to the moment that system's K(w)
 * were all complete on the GPU; service_ms (host, n_systems, or NULL): time
 * from the start of that system's fit to the same moment; total_ms (host, or
 * NULL): the whole run.  Returns the first error of any system (and stops
 * handing out systems). */
ISDF_API int isdf_batch_run(isdf_batch* batch, const double* omega, int n_omega, int n_workers,
                            double* latency_ms, double* service_ms, double* total_ms);

/* CUDA-graph form of isdf_batch_run.  isdf_batch_capture first runs the
 * batch eagerly at the frequencies omega (host, n_omega), which sizes every
 * workspace and fixes each system's rank, then captures the device work of
 * all systems (fit, polarizability at every frequency, SMW) into one graph:
 * the systems run in as many parallel lanes as the batch has workers
 * (largest first, each onto the lane with the least estimated work so
 * far, like the host threads of isdf_batch_run), each system's two streams
 * forked and joined inside its branch.  Every fit must have been
 * unpivoted at full rank (else ISDF_ERR_STATE: a pivoted fit decides on the
 * host).  isdf_batch_replay launches that graph once (one cudaGraphLaunch,
 * no host work between the systems), synchronises, then checks each
 * system's device status and factorisation flags exactly as the eager calls
 * do (ISDF_ERR_NOT_SPD, ISDF_ERR_NONFINITE, ...).  The replay reads the
 * orbitals from the same device buffers at the time of the replay, so new
 * orbital values of the same shape need no recapture; the energies and
 * frequencies are those of the capture.  latency_ms (host, n_systems, or
 * NULL): time from the start of the graph to the end of each system's
 * branch, from events recorded inside the graph; total_ms (host or NULL):
 * host wall time of the launch and the synchronisation.  A new capture
 * replaces the old graph; isdf_batch_destroy frees it. */
ISDF_API int isdf_batch_capture(isdf_batch* batch, const double* omega, int n_omega);
ISDF_API int isdf_batch_replay(isdf_batch* batch, double* latency_ms, double* total_ms);

/* Tile autotuner of the tensor-core GEMMs of the mixed path (process-wide,
 * all contexts and threads).  isdf_set_autotune(1) turns it on (returns the
 * previous setting): the first call of each GEMM shape then times the
 * candidate tile widths (128 or 64 output columns per tile) and split-K
 * counts (the built-in heuristic's, twice and half of it, never below the
 * FP32 accumulation-length minimum) on the call's own operands, keeps the
 * fastest, and every later call of that shape uses it; calls recorded into a
 * CUDA graph use the table and never time.  Products that accumulate into
 * their output (beta != 0) keep the heuristic.  Tuning synchronises the
 * calling stream; a tuned choice changes results only by the FP32
 * accumulation order (split count), within the mixed path's error bound.
 * isdf_autotune_entry(i, key, choice, ms): entry i < isdf_autotune_size()
 * as key[8] = {M, N, K padded, slices, lower-only, triangular B, batch
 * count, split cap}, choice[2] = {tile width, splits}, ms[2] = {best,
 * heuristic} (ms per call when tuned); returns -1 if i is out of range.
 * isdf_autotune_clear() empties the table.  isdf_set_autotune(2) times
 * nothing and records the 64-wide tile wherever it is allowed (heuristic
 * splits), so that a workload exercises every tile path (tests). */
ISDF_API int isdf_set_autotune(int on);
ISDF_API int isdf_autotune_size(void);
ISDF_API int isdf_autotune_entry(int i, int* key, int* choice, double* ms);
ISDF_API void isdf_autotune_clear(void);

/* The context of one system (for apply_eps_inv, smw K copies, profiling)
 * and its rank after the last run. */
ISDF_API int isdf_batch_context(isdf_batch* batch, int system, isdf_ctx** ctx, int* rank);
ISDF_API const char* isdf_batch_last_error(isdf_batch* batch);

/* Split-precision DGEMM on the tensor cores, the building block of the
 * mixed-precision path (the paper has no counterpart; it is a GB300 means
 * of running FP64 contractions at tensor-core rates).
 *   C = alpha A B^T + beta C, A: M x K, B: N x K, C: M x N, all float64,
 *   column-major, device pointers (lda >= M, ldb >= N, ldc >= M).
 *   Each operand is cut into nslices (1..3) BF16 slices, x ~ x0 + x1 + x2;
 *   the products x_i y_j with i + j < nslices are accumulated in FP32 by
 *   tcgen05.mma and long K is summed in FP64 over K blocks.  nslices = 3
 *   gives errors of a few 1e-7 relative to |A| |B|.
 *   Allocates and frees its temporaries on the stream (cudaMallocAsync) and
 *   synchronises the stream before it returns.  Errors: ISDF_ERR_SHAPE,
 *   ISDF_ERR_ARG, ISDF_ERR_CUDA, ISDF_ERR_TIMEOUT; message from
 *   isdf_dgemm_split_error(). */
ISDF_API int isdf_dgemm_split(int M, int N, int K, double alpha, const double* A, long long lda, const double* B,
                              long long ldb, double beta, double* C, long long ldc, int nslices, void* cuda_stream);
ISDF_API const char* isdf_dgemm_split_error(void);

/* Pivot order and Cholesky factor of the last fit.
 *   piv_out  host, n_mu int32 out (or NULL): pivot j is point mu_idx[piv[j]];
 *            the first r are the pivot points that define theta.
 *   L_out    device, n_mu x n_mu float64 out (or NULL): L_r in its leading
 *            r x r block (lower triangular), zero elsewhere. */
ISDF_API int isdf_fit_factor(isdf_ctx* ctx, int* piv_out, double* L_out);

/* Phase timing (CUDA events on the context stream, off by default).  The
 * paper has no counterpart; it reports wall times only.  Phases:           */
enum {
  ISDF_PH_POINTS = 0,      /* C C^T of the points and its pivoted Cholesky */
  ISDF_PH_FIT_GRAM = 1,    /* face-split Gram M C_r^T over the grid */
  ISDF_PH_FIT_TRSM = 2,    /* triangular solve to the whitened basis */
  ISDF_PH_FFT = 3,         /* batched r2c FFT of theta with Coulomb weights */
  ISDF_PH_SYRK_G = 4,      /* G = S^T S over the half spectrum */
  ISDF_PH_POLAR_D = 5,     /* -2 C Omega^-1 C^T at the pivot points */
  ISDF_PH_WHITEN_D = 6,    /* D = L^-1 (.) L^-T */
  ISDF_PH_SMW = 7,         /* capacitance K */
  ISDF_PH_APPLY = 8,       /* eps^-1 X */
  ISDF_NUM_PHASES = 9
};
/* on != 0 starts recording (events are recorded around every phase of every
 * later call); on == 0 stops. */
ISDF_API int isdf_set_profiling(isdf_ctx* ctx, int on);

/* Iterative refinement of the SMW solve in apply_eps_inv (mixed precision,
 * one frequency; Eq. epsilon_with_SMW, the capacitance solve of Algorithm 3
 * step 3): after T2 = K T1 with the tensor-core K = -D X, X the
 * Newton-Schulz (I + G D)^-1, `steps` (0..8) rounds of
 * R = -D (T1 + G T2) - T2 in FP64 (the residual of (I + D G) T2 = -D T1,
 * the capacitance equation multiplied by D) and T2 <- T2 + X^T R.  Each
 * round takes the solve's error relative to the exact solve with this D and
 * G from about cond 2^-24 to its square; the error against the FP64 path
 * stays set by D, G and theta.  Other contexts (FP64, several frequencies,
 * a K from the factorisation route) ignore it.  Default 0.
 * Errors: ISDF_ERR_ARG (steps outside 0..8). */
ISDF_API int isdf_set_refinement(isdf_ctx* ctx, int steps);
/* Synchronises the device, then writes the summed milliseconds and the
 * number of recorded intervals of every phase since the last read into
 * ms[ISDF_NUM_PHASES] and counts[ISDF_NUM_PHASES] (host; either may be
 * NULL) and clears the record. */
ISDF_API int isdf_read_profile(isdf_ctx* ctx, double* ms, int* counts);
/* Short name of a phase, or NULL. */
ISDF_API const char* isdf_phase_name(int phase);
/* Kernel timing by family (recorded with the phase profile, on each
 * launch's own stream).  Families:                                         */
enum {
  ISDF_KF_TC_GEMM = 0,   /* tcgen05 split-precision GEMMs; work = BF16 MMA flops of the slice products */
  ISDF_KF_FP64_GEMM = 1, /* FP64-pipe GEMMs (tiled, batched, face-split Gram); work = flops */
  ISDF_KF_CHOL_DIAG = 2, /* 64 x 64 diagonal-block Cholesky + inverse; work = flops */
  ISDF_KF_FFT = 3,       /* batched 3-D FFTs; work = bytes (input read + output write) */
  ISDF_KF_SLICE = 4,     /* FP64 -> BF16 slicing; work = bytes */
  ISDF_KF_DF_GEMM = 5,   /* double-float trailing updates and inverse GEMMs on the FP32 pipe (mixed path); work = flops */
  ISDF_NUM_KERNEL_FAMILIES = 6
};
/* Synchronises the device, then writes per (family, phase) cell, index
 * family * ISDF_NUM_PHASES + phase, the summed milliseconds, launch count
 * and summed algorithmic work of the launches recorded since the last read
 * (host arrays of ISDF_NUM_KERNEL_FAMILIES * ISDF_NUM_PHASES, any may be
 * NULL) and clears the record.  Work counts the method's arithmetic on the
 * launch's true sizes, not tile padding. */
ISDF_API int isdf_read_kernel_profile(isdf_ctx* ctx, double* ms, int* counts, double* work);
/* The same records launch by launch (tracing): synchronises the device,
 * then writes for the first min(max, recorded) launches since the last read
 * their start and end (ms, from the earliest recorded start; CUDA events on
 * each launch's own stream, so a launch queued behind work of other
 * streams shows its wait), family, phase, work and stream (0 the context
 * stream, 1 and 2 its two helper streams, 3 another) into host arrays of
 * max entries (any may be NULL); clears the record and returns the number
 * written (negative ISDF_ERR_* on error). */
ISDF_API int isdf_read_kernel_trace(isdf_ctx* ctx, int max, double* t_start, double* t_end, int* family, int* phase,
                                    double* work, int* stream);
/* Short name of a kernel family, or NULL. */
ISDF_API const char* isdf_kernel_family_name(int family);
/* Number of kernel launches issued by this library in this process so far
 * (all contexts). */
ISDF_API long long isdf_launch_count(void);
/* Number of device allocations (cudaMalloc / cudaMallocAsync) this library
 * has made in this process so far (all contexts and threads).  The paper
 * has no counterpart; it lets a caller check that a call allocated nothing. */
ISDF_API long long isdf_device_allocations(void);

/* Diagnostic of the bounded device-side waits (the paper has no
 * counterpart).  Runs the library's grid barrier (the wait of the pivoted
 * factorisation's cooperative kernel) on the context stream with a barrier
 * that is never completed: its arrival counter is preset past the grid
 * size, so no block is the last to arrive.  Each block gives up after
 * limit_ns nanoseconds (1e3 .. 1e10), the kernel returns, and the call
 * reports ISDF_ERR_TIMEOUT as any entry point does when one of its device
 * waits runs out.  The barrier and the status word are then cleared, so the
 * context stays usable.  A return of ISDF_ERR_STATE means the barrier
 * completed, i.e. the bound failed.  Synchronises the context stream. */
ISDF_API int isdf_check_device_wait(isdf_ctx* ctx, long long limit_ns);

/* Message for the last error on this context ("" if none).  With ctx NULL,
 * the last error of isdf_create on this thread. */
ISDF_API const char* isdf_last_error(isdf_ctx* ctx);

/* Library version string. */
ISDF_API const char* isdf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ISDF_SMW_H */
