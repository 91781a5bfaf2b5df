// Static COHSEX band self-energies (Algorithm 3 steps 4-7; entry point
// declared in include/isdf_smw.h).
//
// Three fits on one grid: vc (the dielectric matrix: K of Eq.
// epsilon_with_SMW at w = 0), vn (occupied x all) and nn (all x all), each
// in its own context with whitened basis theta_x = P_x L_x.  With the
// weighted half spectra S_x of theta_x (V = S^T S by Parseval, as for G):
//   A_vn = theta_vn^T V theta_vc,  A_nn = theta_nn^T V theta_vc,
//   W_vn = A_vn K A_vn^T,  W_nn = A_nn K A_nn^T,  V_vn = theta_vn^T V theta_vn,
// taken to the points basis by L_x^-T (.) L_x^-1, then the band sums by the
// Hadamard identity (Eq. Hadamard) at the points of each fit:
//   Sigma_SEX_X(n) = -psi_n^T (W_vn .* Psi_v Psi_v^T) psi_n,
//   Sigma_X(n)     = -psi_n^T (V_vn .* Psi_v Psi_v^T) psi_n,
//   Sigma_COH(n)   = 1/2 psi_n^T (W_nn .* Psi Psi^T) psi_n.
// Everything in FP64 on the context stream of the vc fit.
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/isdf_smw.h"
#include "common.cuh"
#include "kernels.h"

using namespace isdf;

#include "ctx.h"

namespace {

int cx_fail(isdf_ctx* c, int code, const std::string& m) { return ctx_fail(c, code, m.c_str()); }

#define XK(expr)                                                                                  \
  do {                                                                                            \
    cudaError_t _e = (expr);                                                                      \
    if (_e != cudaSuccess) return cx_fail(c, ISDF_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// b = a .* b, in place (a and b distinct)
__global__ void k_hadamard_in_place(const double* __restrict__ a, double* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] *= a[i];
}

// out[n] = scale * sum_a X(a, n) Y(a, n), one block per column
__global__ void k_coldot(const double* __restrict__ X, long long ldx, const double* __restrict__ Y, long long ldy,
                         int rows, double scale, double* __restrict__ out) {
  __shared__ double red[128];
  const int n = blockIdx.x;
  double acc = 0.0;
  for (int a = threadIdx.x; a < rows; a += blockDim.x) acc = fma(X[a + ldx * n], Y[a + ldy * n], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = scale * red[0];
}

// C = op(A) op(B)^T (FP64 engine), split over K when K is long
int gemm(isdf_ctx* c, const double* A, long long lda, bool ka, const double* B, long long ldb, bool kb, int M, int N,
         int K, double alpha, double beta, double* C, long long ldc, bool lower, DevBuf& part) {
  const long long tiles = (long long)((M + 63) / 64) * ((N + 63) / 64);
  int sp = (int)std::max<long long>(1, std::min<long long>(16, (2LL * c->num_sms + tiles - 1) / tiles));
  if (K < 4096) sp = 1;
  if (sp > 1) {
    if (part.cap < (size_t)sp * M * N) XK(cudaStreamSynchronize(c->stream));
    XK(ensure(part, (size_t)sp * M * N));
  }
  XK(launch_gemm(A, lda, ka, B, ldb, kb, M, N, K, alpha, beta, C, ldc, lower, sp, sp > 1 ? part.p : nullptr, false,
                 c->stream));
  return ISDF_OK;
}

// the weighted half spectrum of a context's theta (2 h n2 n3 x r)
int spectrum(isdf_ctx* c, const isdf_ctx* x, DevBuf& S) {
  const long long lds = 2 * c->n_half;
  XK(ensure(S, (size_t)lds * std::max(x->rank, 1)));
  XK(launch_fft_forward(c->fft, x->theta, c->n_r, x->rank, S.p, lds, c->d_wsyrk, c->smem_xy, c->smem_z, c->stream));
  return ISDF_OK;
}

// W <- L^-T W L^-1 for the fit of x (r x r, pivot order); scratch t, li, work
int to_points(isdf_ctx* c, const isdf_ctx* x, double* W, DevBuf& t, DevBuf& li, DevBuf& work) {
  const int r = x->rank;
  const size_t rr = (size_t)r * r, wq = (size_t)(r / 2 + 64) * (r / 2 + 64);
  XK(ensure(t, rr));
  XK(ensure(li, rr));
  XK(ensure(work, 5 * wq));
  XK(launch_tri_inverse(x->Lc.p, r, r, li.p, r, work.p, work.p + wq, c->stream));
  XK(launch_gemm(W, r, false, li.p, r, true, r, r, r, 1.0, 0.0, t.p, r, false, 1, nullptr, false, c->stream));
  XK(launch_gemm(li.p, r, true, t.p, r, true, r, r, r, 1.0, 0.0, W, r, false, 1, nullptr, false, c->stream));
  return ISDF_OK;
}

// out[n] = scale * psi_n^T (M .* Psi_o Psi_o^T) psi_n at the points of fit x:
// Psi_o = phimu_p columns [o0, o0 + no), psi_n = column a0 + n, n < nb
int band_sum(isdf_ctx* c, const isdf_ctx* x, const double* M, int o0, int no, int a0, int nb, double scale,
             double* out, DevBuf& g, DevBuf& y) {
  const int r = x->rank;
  const size_t rr = (size_t)r * r;
  const double* P = x->phimu_p.p;
  XK(ensure(g, rr));
  XK(ensure(y, (size_t)r * nb));
  XK(launch_gemm(P + (size_t)r * o0, r, false, P + (size_t)r * o0, r, false, r, r, no, 1.0, 0.0, g.p, r, true, 1,
                 nullptr, false, c->stream));
  note_launch();
  k_hadamard_in_place<<<(unsigned)std::min<size_t>((rr + 255) / 256, 4096), 256, 0, c->stream>>>(M, g.p,
                                                                                                  (long long)rr);
  XK(cudaGetLastError());
  XK(launch_gemm(g.p, r, false, P + (size_t)r * a0, r, true, r, nb, r, 1.0, 0.0, y.p, r, false, 1, nullptr, false,
                 c->stream));
  note_launch();
  k_coldot<<<nb, 128, 0, c->stream>>>(P + (size_t)r * a0, r, y.p, r, r, scale, out);
  XK(cudaGetLastError());
  return ISDF_OK;
}

bool same_grid(const isdf_ctx* a, const isdf_ctx* b) {
  for (int i = 0; i < 3; ++i)
    if (a->n[i] != b->n[i] || a->L[i] != b->L[i]) return false;
  return a->device == b->device;
}

}  // namespace

extern "C" int isdf_cohsex(isdf_ctx* c, isdf_ctx* vn, isdf_ctx* nn, double* sigma) {
  if (!c || !vn || !nn) return ISDF_ERR_ARG;
  c->err.clear();
  if (!sigma) return cx_fail(c, ISDF_ERR_ARG, "isdf_cohsex: null pointer argument");
  if (!c->polar_ready || c->n_omega < 1 || c->omega[0] != 0.0 || !c->k_ready[0])
    return cx_fail(c, ISDF_ERR_STATE, "isdf_cohsex: the vc context needs smw_inverse at omega_index 0 with w = 0");
  if (!vn->fitted || !nn->fitted) return cx_fail(c, ISDF_ERR_STATE, "isdf_cohsex: fit the vn and nn contexts first");
  if (!same_grid(c, vn) || !same_grid(c, nn)) return cx_fail(c, ISDF_ERR_SHAPE, "isdf_cohsex: the three fits need one grid");
  const int n_v = c->n_v, n_e = c->n_v + c->n_c;
  if (vn->n_v != n_v || vn->n_c != n_e || nn->n_v != n_e || nn->n_c != n_e)
    return cx_fail(c, ISDF_ERR_SHAPE,
                   "isdf_cohsex: vn must be fitted on [Phi_v | Phi] (n_v, n_e) and nn on [Phi | Phi] (n_e, n_e)");
  XK(cudaStreamSynchronize(vn->stream));
  XK(cudaStreamSynchronize(nn->stream));
  XK(cudaStreamSynchronize(c->stream));
  XK(cudaMemsetAsync(sigma, 0, 3 * (size_t)n_e * sizeof(double), c->stream));
  const int rc_ = c->rank, rv = vn->rank, rn = nn->rank;
  if (rc_ == 0 || rv == 0 || rn == 0) return ISDF_OK;
  const long long lds = 2 * c->n_half;
  DevBuf* B = c->cx;  // S_vc, S_vn, S_nn, A, T, W, scratch t, li, work, g, y, partial
  int rc;
  if ((rc = spectrum(c, c, B[0])) != ISDF_OK) return rc;
  if ((rc = spectrum(c, vn, B[1])) != ISDF_OK) return rc;
  if ((rc = spectrum(c, nn, B[2])) != ISDF_OK) return rc;
  const double* K = c->K.p;  // omega_index 0, whitened vc basis, ld rc_
  auto w_of = [&](const isdf_ctx* x, DevBuf& Sx) -> int {
    const int r = x->rank;
    int q;
    XK(ensure(B[3], (size_t)r * rc_));
    XK(ensure(B[4], (size_t)r * rc_));
    XK(ensure(B[5], (size_t)r * r));
    if ((q = gemm(c, Sx.p, lds, true, B[0].p, lds, true, r, rc_, (int)lds, 1.0, 0.0, B[3].p, r, false, B[11])) != ISDF_OK)
      return q;                                                                                  // A = S_x^T S_vc
    XK(launch_gemm(B[3].p, r, false, K, rc_, true, r, rc_, rc_, 1.0, 0.0, B[4].p, r, false, 1, nullptr, false,
                   c->stream));                                                                  // T = A K
    XK(launch_gemm(B[4].p, r, false, B[3].p, r, false, r, r, rc_, 1.0, 0.0, B[5].p, r, false, 1, nullptr, false,
                   c->stream));                                                                  // W = T A^T
    return to_points(c, x, B[5].p, B[6], B[7], B[8]);
  };
  // SEX_X and X at the vn points
  if ((rc = w_of(vn, B[1])) != ISDF_OK) return rc;
  if ((rc = band_sum(c, vn, B[5].p, 0, n_v, n_v, n_e, -1.0, sigma, B[9], B[10])) != ISDF_OK) return rc;
  XK(ensure(B[5], (size_t)rv * rv));
  if ((rc = gemm(c, B[1].p, lds, true, B[1].p, lds, true, rv, rv, (int)lds, 1.0, 0.0, B[5].p, rv, true, B[11])) != ISDF_OK)
    return rc;  // V_vn = S_vn^T S_vn
  if ((rc = to_points(c, vn, B[5].p, B[6], B[7], B[8])) != ISDF_OK) return rc;
  if ((rc = band_sum(c, vn, B[5].p, 0, n_v, n_v, n_e, -1.0, sigma + n_e, B[9], B[10])) != ISDF_OK) return rc;
  // COH at the nn points
  if ((rc = w_of(nn, B[2])) != ISDF_OK) return rc;
  if ((rc = band_sum(c, nn, B[5].p, 0, n_e, 0, n_e, 0.5, sigma + 2 * n_e, B[9], B[10])) != ISDF_OK) return rc;
  XK(cudaStreamSynchronize(c->stream));
  return ISDF_OK;
}
