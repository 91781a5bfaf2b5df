// Adjoint of the SMW inverse in the ISDF basis (entry points declared in
// include/isdf_smw.h): the screened Coulomb operator projected on the
// interpolation vectors, W_P = P^T eps^-1 V P = G + G K G in the points
// basis, and the gradient of a scalar loss L(W_P) with respect to the
// orbital energies and the orbital samples at the interpolation points,
// with the ISDF vectors held fixed.
//
// In the whitened basis of the fit (theta = P_r L_r) every r x r operator is
// well scaled; the points basis is reached by L_r^-1:
//   W_P(pivots) = L^-T (G + G K G) L^-1.
// Reverse mode, from d(A^-1) = -A^-1 dA A^-1 applied to K = -D (I + G D)^-1:
//   Pw   = L^-1 Wbar L^-T                      (dL/dW in the whitened basis)
//   Kbar = G Pw G,  E = I + G K = (I + G D)^-1
//   Dw   = -E Kbar E^T,  Dbar = L^-T Dw L^-1   (dL/dD at the pivot points)
//   D    = sum_p d_p c_p c_p^T, d_p = -2 Omega_p(i w)^-1 (Eq. COmegaCstar)
//   Y    = sym(Dbar) C_r;  dL/dd_p = c_p . y_p;  dL/dC = 2 Y diag(d)
//   dL/de_v = sum_c dL/dd_vc dd/dDelta,  dL/de_c = -sum_v dL/dd_vc dd/dDelta,
//   dL/dphi_v(a) = sum_c dL/dC(a, vc) phi_c(a) (and v <-> c).
// Everything runs in FP64: the r^3 products and Y = Dbar C_r (2 r^2 n_v n_c
// flops, the dominant step) on the FP64 GEMM engine, the reductions in
// the small kernels below.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/isdf_smw.h"
#include "common.cuh"
#include "kernels.h"

using namespace isdf;

#include "ctx.h"

namespace {

int cuda_err(isdf_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return ctx_fail(c, ISDF_ERR_CUDA, m.c_str());
}

#define AK(expr)                                            \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return cuda_err(c, _e, #expr);   \
  } while (0)

// C_r(a, v n_c + c) = phi_mu(a, v) phi_mu(a, n_v + c): one block per pair
__global__ void k_pair_matrix(const double* __restrict__ phimu, int r, int n_v, int n_c, double* __restrict__ Cp) {
  const long long p = blockIdx.x;
  const int v = (int)(p / n_c), cc = (int)(p - (long long)v * n_c);
  const double* pv = phimu + (long long)r * v;
  const double* pc = phimu + (long long)r * (n_v + cc);
  for (int a = threadIdx.x; a < r; a += blockDim.x) Cp[a + r * p] = pv[a] * pc[a];
}

// gd[p] = sum_a C(a, p) Y(a, p), then Y(a, p) <- 2 d_p Y(a, p) with
// d_p = sw_p^2 (sw = sqrt(-2 Omega^-1) of the frequency)
__global__ void k_adj_pairs(const double* __restrict__ Cp, double* Y, int r, const double* __restrict__ sw,
                            double* __restrict__ gd) {
  __shared__ double red[128];
  const long long p = blockIdx.x;
  const double d2 = 2.0 * sw[p] * sw[p];
  double acc = 0.0;
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    const long long i = a + r * p;
    const double y = Y[i];
    acc = fma(Cp[i], y, acc);
    Y[i] = d2 * y;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) gd[p] = red[0];
}

// grad_phimu(perm[a], i) from Ybar = dL/dC (r x n_v n_c) and phi at the pivots
__global__ void k_adj_phi(const double* __restrict__ Yb, const double* __restrict__ phimu, int r, int n_v, int n_c,
                          const int* __restrict__ perm, double* __restrict__ g, long long ldg) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (a >= r) return;
  double acc = 0.0;
  if (i < n_v) {
    const double* y = Yb + a + (long long)r * ((long long)i * n_c);
    for (int cc = 0; cc < n_c; ++cc) acc = fma(y[(long long)r * cc], phimu[a + (long long)r * (n_v + cc)], acc);
  } else {
    const int j = i - n_v;
    for (int v = 0; v < n_v; ++v)
      acc = fma(Yb[a + (long long)r * ((long long)v * n_c + j)], phimu[a + (long long)r * v], acc);
  }
  g[perm[a] + ldg * i] = acc;
}

// grad_e[i]: d_p = -2 Delta / (Delta^2 + w^2), Delta = e_v - e_c
__global__ void k_adj_energy(const double* __restrict__ gd, const double* __restrict__ e, int n_v, int n_c,
                             double w, double* __restrict__ ge) {
  __shared__ double red[128];
  const int i = blockIdx.x;
  const double w2 = w * w;
  double acc = 0.0;
  const int n = i < n_v ? n_c : n_v;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int v = i < n_v ? i : t, cc = i < n_v ? t : i - n_v;
    const double dl = e[v] - e[n_v + cc];
    const double q = dl * dl + w2;
    const double dd = -2.0 * (w2 - dl * dl) / (q * q);
    const double gv = gd[(long long)v * n_c + cc] * dd;
    acc += i < n_v ? gv : -gv;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) ge[i] = red[0];
}

// dst(perm[i], perm[j]) = src(i, j), i, j < r (points order from pivot order)
__global__ void k_scatter_sym(const double* __restrict__ src, int r, const int* __restrict__ perm, double* dst,
                              long long ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i < r) dst[perm[i] + ldd * perm[j]] = src[i + (long long)r * j];
}

// dst(i, j) = src(perm[i], perm[j]), i, j < r
__global__ void k_gather_sym(const double* __restrict__ src, long long lds, int r, const int* __restrict__ perm,
                             double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i < r) dst[i + (long long)r * j] = src[perm[i] + lds * perm[j]];
}

// c = a .* b over n doubles (c may be a or b)
__global__ void k_mul_elem(const double* a, const double* b, double* c, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    c[i] = a[i] * b[i];
}

void mul_elem(const double* a, const double* b, double* c, long long n, cudaStream_t s) {
  note_launch();
  k_mul_elem<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(a, b, c, n);
}

// The rows of the points: g(idx[perm[a]], i) += gp(a, i) + gd(perm[a], i)
// (gp in pivot order, ld r; gd in points order, ld m; the points distinct)
__global__ void k_scatter_add_rows(const double* __restrict__ gp, int r, const double* __restrict__ gd, int m,
                                   const int* __restrict__ perm, const int* __restrict__ idx, double* g, long long ldg) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (a >= r) return;
  const int pt = perm[a];
  g[idx[pt] + ldg * i] += gp[a + (long long)r * i] + gd[pt + (long long)m * i];
}

// C = op(A) op(B)^T with the FP64 engine (r x r operands, ld r)
cudaError_t mm(const double* A, bool ta, const double* B, bool tb, int r, double alpha, double beta, double* C,
               cudaStream_t s) {
  return launch_gemm(A, r, ta, B, r, tb, r, r, r, alpha, beta, C, r, false, 1, nullptr, false, s);
}

int check_ready(isdf_ctx* c, int k, const char* who) {
  if (!c->polar_ready || k < 0 || k >= c->n_omega || !c->k_ready[k]) {
    std::string m = std::string(who) + ": call smw_inverse for this omega_index first";
    return ctx_fail(c, ISDF_ERR_STATE, m.c_str());
  }
  return ISDF_OK;
}

// L_r^-1 into a_linv (r x r)
int linv(isdf_ctx* c, int r) {
  const size_t rr = (size_t)r * r, wq = (size_t)(r / 2 + 64) * (r / 2 + 64);
  AK(ensure(c->a_linv, rr));
  AK(ensure(c->a_m3, std::max(rr, 5 * wq)));
  AK(launch_tri_inverse(c->Lc.p, r, r, c->a_linv.p, r, c->a_m3.p, c->a_m3.p + wq, c->stream));
  return ISDF_OK;
}

}  // namespace

extern "C" int isdf_set_point_orbitals(isdf_ctx* c, const double* phimu, long long ldp) {
  if (!c) return ISDF_ERR_ARG;
  c->err.clear();
  if (!c->fitted) return ctx_fail(c, ISDF_ERR_STATE, "isdf_set_point_orbitals: call isdf_fit first");
  if (!phimu) return ctx_fail(c, ISDF_ERR_ARG, "isdf_set_point_orbitals: null pointer argument");
  if (ldp < c->n_mu) return ctx_fail(c, ISDF_ERR_SHAPE, "isdf_set_point_orbitals: ldp < n_mu");
  const int r = c->rank, n_e = c->n_v + c->n_c;
  c->polar_ready = false;
  std::fill(c->k_ready.begin(), c->k_ready.end(), 0);
  if (r == 0) return ISDF_OK;
  AK(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream));
  AK(launch_gather_rows(phimu, ldp, c->d_perm, r, n_e, c->phimu_p.p, r, c->stream));
  AK(launch_check_finite(c->phimu_p.p, (long long)r * n_e, c->d_status, c->stream));
  unsigned st = 0;
  AK(cudaMemcpyAsync(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  AK(cudaStreamSynchronize(c->stream));
  if (st & ST_NONFINITE) return ctx_fail(c, ISDF_ERR_NONFINITE, "isdf_set_point_orbitals: NaN or Inf in phimu");
  return ISDF_OK;
}

extern "C" int isdf_screened_basis(isdf_ctx* c, int k, double* W_out) {
  if (!c) return ISDF_ERR_ARG;
  c->err.clear();
  int rc = check_ready(c, k, "isdf_screened_basis");
  if (rc != ISDF_OK) return rc;
  if (!W_out) return ctx_fail(c, ISDF_ERR_ARG, "isdf_screened_basis: null pointer argument");
  const int r = c->rank, m = c->n_mu;
  const size_t rr = (size_t)r * r;
  if (r > 65535) return ctx_fail(c, ISDF_ERR_SHAPE, "isdf_screened_basis: rank must be <= 65535");
  cudaStream_t s = c->stream;
  AK(cudaMemsetAsync(W_out, 0, (size_t)m * m * sizeof(double), s));
  if (r == 0) return ISDF_OK;
  AK(ensure(c->a_m1, rr));
  AK(ensure(c->a_m2, rr));
  AK(ensure(c->a_m4, rr));
  if ((rc = linv(c, r)) != ISDF_OK) return rc;
  const double* G = c->G.p;
  const double* K = c->K.p + rr * k;
  AK(mm(G, false, K, true, r, 1.0, 0.0, c->a_m1.p, s));            // G K
  AK(cudaMemcpyAsync(c->a_m2.p, G, rr * sizeof(double), cudaMemcpyDeviceToDevice, s));
  AK(mm(c->a_m1.p, false, G, true, r, 1.0, 1.0, c->a_m2.p, s));    // W = G + G K G
  AK(mm(c->a_m2.p, false, c->a_linv.p, true, r, 1.0, 0.0, c->a_m1.p, s));   // W L^-1
  AK(mm(c->a_linv.p, true, c->a_m1.p, true, r, 1.0, 0.0, c->a_m4.p, s));    // L^-T W L^-1
  note_launch();
  k_scatter_sym<<<dim3((r + 127) / 128, r), 128, 0, s>>>(c->a_m4.p, r, c->d_perm, W_out, m);
  AK(cudaGetLastError());
  return ISDF_OK;
}

extern "C" int isdf_adjoint(isdf_ctx* c, int k, const double* W_bar, double* grad_energies, double* grad_phimu) {
  if (!c) return ISDF_ERR_ARG;
  c->err.clear();
  int rc = check_ready(c, k, "isdf_adjoint");
  if (rc != ISDF_OK) return rc;
  if (!W_bar || !grad_energies || !grad_phimu) return ctx_fail(c, ISDF_ERR_ARG, "isdf_adjoint: null pointer argument");
  const int r = c->rank, m = c->n_mu, n_v = c->n_v, n_c = c->n_c, n_e = n_v + n_c;
  const size_t rr = (size_t)r * r, npair = (size_t)n_v * n_c;
  if (r > 65535 || n_e > 65535) return ctx_fail(c, ISDF_ERR_SHAPE, "isdf_adjoint: rank and n_e must be <= 65535");
  cudaStream_t s = c->stream;
  AK(cudaMemsetAsync(grad_phimu, 0, (size_t)m * n_e * sizeof(double), s));
  if (r == 0) {
    AK(cudaMemsetAsync(grad_energies, 0, (size_t)n_e * sizeof(double), s));
    return ISDF_OK;
  }
  if (c->a_cp.cap < (size_t)r * npair || c->a_y.cap < (size_t)r * npair) AK(cudaStreamSynchronize(s));
  AK(ensure(c->a_m1, rr));
  AK(ensure(c->a_m2, rr));
  AK(ensure(c->a_m4, rr));
  AK(ensure(c->a_cp, (size_t)r * npair));
  AK(ensure(c->a_y, (size_t)r * npair));
  AK(ensure(c->a_gd, npair));
  AK(ensure(c->a_e, n_e));
  if ((rc = linv(c, r)) != ISDF_OK) return rc;
  double* Li = c->a_linv.p;
  double *M1 = c->a_m1.p, *M2 = c->a_m2.p, *M4 = c->a_m4.p;
  const double* G = c->G.p;
  const double* K = c->K.p + rr * k;
  note_launch();
  k_gather_sym<<<dim3((r + 127) / 128, r), 128, 0, s>>>(W_bar, m, r, c->d_perm, M1);  // Wbar at the pivots
  AK(cudaGetLastError());
  AK(mm(Li, false, M1, true, r, 1.0, 0.0, M2, s));    // L^-1 Wbar
  AK(mm(M2, false, Li, false, r, 1.0, 0.0, M1, s));   // Pw = L^-1 Wbar L^-T
  AK(mm(G, false, M1, true, r, 1.0, 0.0, M2, s));     // G Pw
  AK(mm(M2, false, G, true, r, 1.0, 0.0, M1, s));     // Kbar = G Pw G
  AK(mm(G, false, K, true, r, 1.0, 0.0, M2, s));      // G K
  AK(launch_add_identity(M2, r, r, 1.0, s));          // E = I + G K
  AK(mm(M2, false, M1, true, r, 1.0, 0.0, M4, s));    // E Kbar
  AK(mm(M4, false, M2, false, r, -1.0, 0.0, M1, s));  // Dw = -E Kbar E^T
  AK(mm(M1, false, Li, true, r, 1.0, 0.0, M4, s));    // Dw L^-1
  AK(mm(Li, true, M4, true, r, 1.0, 0.0, M1, s));     // Dbar = L^-T Dw L^-1
  AK(launch_symmetrize(M1, r, r, s));
  note_launch();
  k_pair_matrix<<<(unsigned)npair, 128, 0, s>>>(c->phimu_p.p, r, n_v, n_c, c->a_cp.p);
  AK(cudaGetLastError());
  // Y = sym(Dbar) C_r  (r x n_v n_c)
  AK(launch_gemm(M1, r, false, c->a_cp.p, r, true, r, (int)npair, r, 1.0, 0.0, c->a_y.p, r, false, 1, nullptr, false,
                 s));
  note_launch();
  k_adj_pairs<<<(unsigned)npair, 128, 0, s>>>(c->a_cp.p, c->a_y.p, r, c->sw.p + npair * k, c->a_gd.p);
  AK(cudaGetLastError());
  note_launch();
  k_adj_phi<<<dim3((r + 127) / 128, n_e), 128, 0, s>>>(c->a_y.p, c->phimu_p.p, r, n_v, n_c, c->d_perm, grad_phimu, m);
  AK(cudaGetLastError());
  AK(cudaMemcpyAsync(c->a_e.p, c->energies.data(), n_e * sizeof(double), cudaMemcpyHostToDevice, s));
  note_launch();
  k_adj_energy<<<n_e, 128, 0, s>>>(c->a_gd.p, c->a_e.p, n_v, n_c, c->omega[k], grad_energies);
  AK(cudaGetLastError());
  AK(cudaStreamSynchronize(s));  // the energies were copied from a host vector that later calls may change
  return ISDF_OK;
}

// Adjoint through the fit (see include/isdf_smw.h).  With P = theta L^-1
// (points basis, full rank) and A = C C^T = L L^T, in the whitened basis:
//   Pw  = L^-1 Wbar L^-T,  E = I + G K,  Gb = E^T Pw E   (dL/dG_P = L Gb L^T)
//   dL/dZ = 2 V P dL/dG_P A^-1 = 2 V theta Gb L^-1
//   dL/dA = -sym(A^-1 (dL/dP)^T P) = -L^-T (Gb G + G Gb) L^-1
//   Z = Zv .* Zc, Zv = Phi_v Phi_v,mu^T, Zc = Phi_c Phi_c,mu^T (recomputed:
//   theta is the only checkpoint of the forward pass), A = Av .* Ac:
//   dL/dPhi_v = (dL/dZ .* Zc) Phi_v,mu,  dL/dPhi_c = (dL/dZ .* Zv) Phi_c,mu,
//   rows mu: + (dL/dZ .* Zc)^T Phi_v + 2 (dL/dA .* Ac) Phi_v,mu (and v <-> c)
//   + dL/dphi_mu through D (isdf_adjoint).
extern "C" int isdf_adjoint_fit(isdf_ctx* c, int k, const double* W_bar, double* grad_energies, double* grad_phi) {
  if (!c) return ISDF_ERR_ARG;
  c->err.clear();
  int rc = check_ready(c, k, "isdf_adjoint_fit");
  if (rc != ISDF_OK) return rc;
  if (!W_bar || !grad_energies || !grad_phi)
    return ctx_fail(c, ISDF_ERR_ARG, "isdf_adjoint_fit: null pointer argument");
  const int r = c->rank, m = c->n_mu, n_v = c->n_v, n_c = c->n_c, n_e = n_v + n_c;
  if (r != m) return ctx_fail(c, ISDF_ERR_STATE, "isdf_adjoint_fit: needs a fit of full rank (C C^T invertible)");
  if (r > 65535 || n_e > 65535) return ctx_fail(c, ISDF_ERR_SHAPE, "isdf_adjoint_fit: rank and n_e must be <= 65535");
  const long long nr = c->n_r;
  const size_t rr = (size_t)r * r, big = (size_t)nr * r;
  const long long lds = 2 * c->n_half;
  cudaStream_t s = c->stream;
  // through D at the points, theta held fixed; its point gradient goes to a_gpm
  AK(ensure(c->a_gpm, (size_t)m * n_e));
  rc = isdf_adjoint(c, k, W_bar, grad_energies, c->a_gpm.p);
  if (rc != ISDF_OK) return rc;
  AK(cudaStreamSynchronize(s));  // the buffers below may grow
  AK(ensure(c->a_z1, big));
  AK(ensure(c->a_z2, big));
  AK(ensure(c->a_z3, big));
  AK(ensure(c->spec, (size_t)lds * r));
  AK(ensure(c->a_gpp, (size_t)r * n_e));
  AK(ensure(c->a_m5, rr));
  AK(ensure(c->a_m6, rr));
  const int ks = (int)std::max<long long>(1, std::min<long long>(32, nr / 4096));
  AK(ensure(c->partial, (size_t)ks * r * n_e));
  if ((rc = linv(c, r)) != ISDF_OK) return rc;
  const double* Li = c->a_linv.p;
  double *M1 = c->a_m1.p, *M2 = c->a_m2.p, *M4 = c->a_m4.p, *M5 = c->a_m5.p, *M6 = c->a_m6.p;
  const double* G = c->G.p;
  const double* K = c->K.p + rr * k;
  const double* phv = c->phimu_p.p;                   // r x n_v, pivot order
  const double* phc = c->phimu_p.p + (size_t)r * n_v;  // r x n_c
  note_launch();
  k_gather_sym<<<dim3((r + 127) / 128, r), 128, 0, s>>>(W_bar, m, r, c->d_perm, M1);
  AK(cudaGetLastError());
  AK(mm(Li, false, M1, true, r, 1.0, 0.0, M2, s));    // L^-1 Wbar
  AK(mm(M2, false, Li, false, r, 1.0, 0.0, M1, s));   // Pw
  AK(mm(G, false, K, true, r, 1.0, 0.0, M2, s));      // G K
  AK(launch_add_identity(M2, r, r, 1.0, s));          // E
  AK(mm(M1, false, M2, true, r, 1.0, 0.0, M4, s));    // Pw E
  AK(mm(M2, true, M4, true, r, 1.0, 0.0, M5, s));     // Gb = E^T Pw E
  AK(launch_symmetrize(M5, r, r, s));
  // H = 2 Gb L^-1, then dL/dZ = V (theta H)
  AK(mm(M5, false, Li, true, r, 2.0, 0.0, M6, s));
  AK(launch_gemm(c->theta, nr, false, M6, r, true, (int)nr, r, r, 1.0, 0.0, c->a_z1.p, nr, false, 1, nullptr, false, s));
  AK(launch_fft_convolve(c->fft, c->a_z1.p, nr, r, c->spec.p, lds, c->d_wconv, nullptr, 0, c->a_z1.p, nr, c->smem_xy,
                         c->smem_z, s));
  // dL/dA = -L^-T (Gb G + G Gb) L^-1
  AK(mm(M5, false, G, true, r, 1.0, 0.0, M1, s));     // Gb G
  AK(mm(G, false, M5, true, r, 1.0, 1.0, M1, s));     // + G Gb
  AK(mm(M1, false, Li, true, r, 1.0, 0.0, M2, s));    // (.) L^-1
  AK(mm(Li, true, M2, true, r, -1.0, 0.0, M6, s));    // Abar = -L^-T (.) L^-1
  // Zv, Zc, then dL/dZ .* Zc (into Zc) and dL/dZ .* Zv (into Zv)
  AK(launch_gemm(c->phi, nr, false, phv, r, false, (int)nr, r, n_v, 1.0, 0.0, c->a_z2.p, nr, false, 1, nullptr, false,
                 s));
  AK(launch_gemm(c->phi + (size_t)nr * n_v, nr, false, phc, r, false, (int)nr, r, n_c, 1.0, 0.0, c->a_z3.p, nr, false,
                 1, nullptr, false, s));
  mul_elem(c->a_z1.p, c->a_z3.p, c->a_z3.p, (long long)big, s);  // Zbv = Zbar .* Zc
  mul_elem(c->a_z1.p, c->a_z2.p, c->a_z2.p, (long long)big, s);  // Zbc = Zbar .* Zv
  AK(cudaGetLastError());
  // grid rows: dL/dPhi_v = Zbv Phi_v,mu, dL/dPhi_c = Zbc Phi_c,mu
  AK(launch_gemm(c->a_z3.p, nr, false, phv, r, true, (int)nr, n_v, r, 1.0, 0.0, grad_phi, nr, false, 1, nullptr, false,
                 s));
  AK(launch_gemm(c->a_z2.p, nr, false, phc, r, true, (int)nr, n_c, r, 1.0, 0.0, grad_phi + (size_t)nr * n_v, nr, false,
                 1, nullptr, false, s));
  // point rows (pivot order): Zbv^T Phi_v, Zbc^T Phi_c (split over the grid)
  double* gpp = c->a_gpp.p;
  AK(launch_gemm(c->a_z3.p, nr, true, c->phi, nr, true, r, n_v, (int)nr, 1.0, 0.0, gpp, r, false, ks, c->partial.p,
                 false, s));
  AK(launch_gemm(c->a_z2.p, nr, true, c->phi + (size_t)nr * n_v, nr, true, r, n_c, (int)nr, 1.0, 0.0,
                 gpp + (size_t)r * n_v, r, false, ks, c->partial.p, false, s));
  // + 2 (Abar .* Ac) Phi_v,mu and 2 (Abar .* Av) Phi_c,mu
  AK(launch_gemm(phc, r, false, phc, r, false, r, r, n_c, 1.0, 0.0, M1, r, false, 1, nullptr, false, s));  // Ac
  AK(launch_gemm(phv, r, false, phv, r, false, r, r, n_v, 1.0, 0.0, M2, r, false, 1, nullptr, false, s));  // Av
  mul_elem(M6, M1, M1, (long long)rr, s);  // Abar .* Ac
  mul_elem(M6, M2, M2, (long long)rr, s);  // Abar .* Av
  AK(cudaGetLastError());
  AK(launch_gemm(M1, r, false, phv, r, true, r, n_v, r, 2.0, 1.0, gpp, r, false, 1, nullptr, false, s));
  AK(launch_gemm(M2, r, false, phc, r, true, r, n_c, r, 2.0, 1.0, gpp + (size_t)r * n_v, r, false, 1, nullptr, false,
                 s));
  note_launch();
  k_scatter_add_rows<<<dim3((r + 127) / 128, n_e), 128, 0, s>>>(gpp, r, c->a_gpm.p, m, c->d_perm, c->d_idx, grad_phi,
                                                               nr);
  AK(cudaGetLastError());
  AK(cudaStreamSynchronize(s));
  return ISDF_OK;
}
