// Mixed-precision ISDF-SMW (ISDF_PREC_MIXED): every large contraction runs
// on the tensor cores as a three-slice BF16 split-precision GEMM (FP32
// accumulation in TMEM, FP64 sums across K blocks); the factorisations (the
// pivoted Cholesky of C C^T, the Cholesky factors of the capacitance, the
// triangular inverses) and the small products stay in FP64.
//
//   fit   : theta = [(Phi_v Phi_v,mu^T) .* (Phi_c Phi_c,mu^T)] L^-T, the
//           face-split Gram with two TMEM accumulators, then one triangular
//           GEMM with the FP64 inverse of the Cholesky factor;
//   polar : G = S^T S with S the FP32 FFT of theta written straight into
//           BF16 slices; D = L^-1 (S_pair S_pair^T) L^-T with the pair
//           operand generated into slices;
//   smw   : K = -Q Q^T, Q = R U^-T, with R, U FP64 Cholesky factors and the
//           GEMMs around them on the tensor cores;
//   apply : theta^T X and theta T2 on the tensor cores, the Coulomb
//           convolution of the n_rhs columns in FP64.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/isdf_smw.h"
#include "ctx.h"

namespace isdf {

namespace {

constexpr int NSL = 3;  // BF16 slices per operand

inline int pad(long long x, int m) { return (int)((x + m - 1) / m * m); }

// Zero the padding of an NSL-slice stack (rows_pad x kp per slice) whose
// writer fills rows 0..R-1 at columns [0, kv) and [kvp, kend) (kv = kvp = 0:
// [0, kend)): the rows R..rows_pad-1 of every slice and, in every row, the
// columns outside those ranges.  Together with the writer this leaves the
// stack as zeroing all of it first would, but moves only the padding's bytes
// (none where the shapes are multiples of the tiles, as at 48^3 / N_mu 1536,
// where the whole-stack zeroing of the FFT's slices alone was 1 GB).
inline cudaError_t zero_padding(__nv_bfloat16* p, int R, int kend, int rows_pad, int kp, cudaStream_t st, int kv = 0,
                                int kvp = 0) {
  const size_t pitch = (size_t)kp * 2, rows = (size_t)NSL * rows_pad;
  cudaError_t e = cudaSuccess;
  if (kv < kvp) e = cudaMemset2DAsync(p + kv, pitch, 0, (size_t)(kvp - kv) * 2, rows, st);
  if (e == cudaSuccess && kend < kp) e = cudaMemset2DAsync(p + kend, pitch, 0, (size_t)(kp - kend) * 2, rows, st);
  for (int l = 0; l < NSL && e == cudaSuccess && R < rows_pad; ++l)
    e = cudaMemsetAsync(p + ((size_t)l * rows_pad + R) * kp, 0, (size_t)(rows_pad - R) * kp * 2, st);
  return e;
}

// k_slice_cm writes rows 0..R-1 at the mapped columns of 0..C-1:
// [0, kv) and [kvp, C - kv + kvp) (identity when kv = kvp = 0)
inline cudaError_t slices_cm(DevBuf& buf, const double* src, long long lds, int R, int C, int rows_pad, int kp,
                             cudaStream_t st, int kv = 0, int kvp = 0) {
  const size_t n = (size_t)NSL * rows_pad * kp;
  cudaError_t e = ensure_bf16(buf, n);
  if (e != cudaSuccess) return e;
  const int kvc = std::min(kv, C);
  e = zero_padding(buf.bf(), R, kv > 0 ? C - kvc + kvp : C, rows_pad, kp, st, kvc, kv > 0 ? kvp : 0);
  if (e != cudaSuccess) return e;
  return launch_slice_colmajor(src, lds, R, C, kv, kvp, buf.bf(), rows_pad, kp, NSL, st);
}

// k_slice_rm writes rows 0..R-1 at columns 0..K-1 (and zeros up to the next
// multiple of 8)
inline cudaError_t slices_rm(DevBuf& buf, const double* src, long long lds, int R, int K, int rows_pad, int kp,
                             cudaStream_t st) {
  const size_t n = (size_t)NSL * rows_pad * kp;
  cudaError_t e = ensure_bf16(buf, n);
  if (e != cudaSuccess) return e;
  e = zero_padding(buf.bf(), R, K, rows_pad, kp, st);
  if (e != cudaSuccess) return e;
  return launch_slice_rowmajor(src, lds, R, K, buf.bf(), rows_pad, kp, NSL, st);
}

inline TcOperand op(const DevBuf& b, int rows_pad, int kp) { return TcOperand{b.bf(), rows_pad, kp, NSL}; }
// the first s slices of the stack (products i + j < s)
inline TcOperand op_s(const DevBuf& b, int rows_pad, int kp, int s) { return TcOperand{b.bf(), rows_pad, kp, s}; }

// Slices of `count` matrices src + z sstride; problem z's slice stack starts
// at row z NSL rows_pad of buf.  buf must already hold count stacks.
inline cudaError_t slices_cm_b(DevBuf& buf, const double* src, long long lds, long long sstride, int R, int C,
                               int rows_pad, int kp, int count, cudaStream_t st) {
  const size_t per = (size_t)NSL * rows_pad * kp;
  if (buf.cap * 4 < per * count) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(buf.p, 0, per * count * 2, st);
  if (e != cudaSuccess) return e;
  return launch_slice_colmajor(src, lds, R, C, 0, 0, buf.bf(), rows_pad, kp, NSL, st, count, sstride, (long long)per);
}

inline cudaError_t slices_rm_b(DevBuf& buf, const double* src, long long lds, long long sstride, int R, int K,
                               int rows_pad, int kp, int count, cudaStream_t st) {
  const size_t per = (size_t)NSL * rows_pad * kp;
  if (buf.cap * 4 < per * count) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(buf.p, 0, per * count * 2, st);
  if (e != cudaSuccess) return e;
  return launch_slice_rowmajor(src, lds, R, K, buf.bf(), rows_pad, kp, NSL, st, count, sstride, (long long)per);
}

// byte budget of the pair-operand slices of one batch of frequencies
constexpr size_t kPairSliceBudget = size_t(4) << 30;

}  // namespace

#define MK(expr)                                        \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) return _e;                   \
  } while (0)

// Slices of M C_r^T (the face-split Gram of the fit) into c->m_zs, from the
// orbitals at the r points in pivot order (phimu_p, r x n_e, ld r).
cudaError_t mixed_fit_gram(isdf_ctx* c, const double* phi, const double* phimu_p, int n_v, int n_c, int r) {
  cudaStream_t st = c->stream;
  const long long nr = c->n_r;
  const int n_e = n_v + n_c;
  const int kvp = pad(n_v, 64), kp = kvp + pad(n_c, 64);
  const int nrp = pad(nr, 128), rp = pad(r, 128), rk = pad(r, 64);
  PhaseTimer ph(c, ISDF_PH_FIT_GRAM);
  MK(slices_cm(c->m_phis, phi, nr, (int)nr, n_e, nrp, kp, st, n_v, kvp));
  MK(slices_cm(c->m_phimus, phimu_p, r, r, n_e, rp, kp, st, n_v, kvp));
  const size_t nz = (size_t)NSL * nrp * rk;
  MK(ensure_bf16(c->m_zs, nz));
  MK(zero_padding(c->m_zs.bf(), (int)nr, r, nrp, rk, st));  // the epilogue writes rows < N_r, columns < r
  return tc_facesplit(op(c->m_phis, nrp, kp), op(c->m_phimus, rp, kp), (int)nr, r, kvp / 64, nullptr, 0,
                      c->m_zs.bf(), nrp, rk, c->d_status, st);
}

// theta (N_r x r, ld N_r) = (M C_r^T) L^-T from c->m_zs and the Cholesky
// factor c->Lc (r x r, ld r); linv_ready: c->m_linv already holds L^-1
// (built beside the factorisation).
cudaError_t mixed_fit_solve(isdf_ctx* c, double* theta, int r, bool linv_ready) {
  cudaStream_t st = c->stream;
  const long long nr = c->n_r;
  const int nrp = pad(nr, 128), rp = pad(r, 128), rk = pad(r, 64);
  PhaseTimer ph(c, ISDF_PH_FIT_TRSM);
  MK(ensure(c->m_linv, (size_t)r * r));
  const size_t wq = (size_t)(r / 2 + 64) * (r / 2 + 64);
  MK(ensure(c->m_work, 5 * wq));
  if (!linv_ready) MK(launch_tri_inverse(c->Lc.p, r, r, c->m_linv.p, r, c->m_work.p, c->m_work.p + wq, st));
  MK(slices_cm(c->m_linvs, c->m_linv.p, r, r, r, rp, rk, st));
  // theta in FP64 and, from the same epilogue, its slices for the apply:
  // K-major over mu (theta T2, m_ths) and over the grid (theta^T X, m_thetas_t)
  const int kpg = pad(nr, 64);
  const size_t nth = (size_t)NSL * nrp * rk, ntt = (size_t)NSL * rp * kpg;
  MK(ensure_bf16(c->m_ths, nth));
  MK(ensure_bf16(c->m_thetas_t, ntt));
  // the epilogue writes (m, n) of both for m < N_r, n < r
  MK(zero_padding(c->m_ths.bf(), (int)nr, r, nrp, rk, st));
  MK(zero_padding(c->m_thetas_t.bf(), r, (int)nr, rp, kpg, st));
  TcGroup whole_runs(0);
  MK(tc_gemm_f64_slices(op(c->m_zs, nrp, rk), op(c->m_linvs, rp, rk), (int)nr, r, theta, nr, true, c->m_ths.bf(), nrp,
                        rk, c->m_thetas_t.bf(), rp, kpg, c->d_status, st));
  return cudaSuccess;
}

// G = theta^T V theta (r x r) into c->G.
cudaError_t mixed_polar_G(isdf_ctx* c) {
  cudaStream_t st = c->stream;
  const int r = c->rank;
  const size_t rr = (size_t)r * r;
  const int rp = pad(r, 128);
  const long long lds32 = 2 * c->n_half;
  const int kps = pad(lds32, 64);
  const int max_split = std::max(8, tc_min_splits(kps));
  MK(ensure(c->partial, (size_t)max_split * rr));
  {
    PhaseTimer ph(c, ISDF_PH_FFT);
    MK(ensure(c->m_s32, ((size_t)lds32 * r + 1) / 2));
    const size_t ns = (size_t)NSL * rp * kps;
    MK(ensure_bf16(c->m_ss, ns));
    // the z pass writes all 2 n_half reals of each of the r rows
    MK(zero_padding(c->m_ss.bf(), r, (int)lds32, rp, kps, st));
    MK(launch_fft_forward_slices(c->fft, c->theta, c->n_r, r, (float*)c->m_s32.p, lds32, c->d_wsyrk, c->m_ss.bf(),
                                 rp, kps, NSL, c->smem_xy, c->smem_z, st));
  }
  {
    PhaseTimer ph(c, ISDF_PH_SYRK_G);
    TcGroup whole_runs(0);
    MK(tc_gemm_f64(op(c->m_ss, rp, kps), op(c->m_ss, rp, kps), r, r, 1.0, 0.0, c->G.p, r, true, false,
                   c->partial.p, max_split, c->num_sms, c->d_status, st));
  }
  return cudaSuccess;
}

// D(w_k) for all frequencies, whitened, into c->D.
cudaError_t mixed_polar_D(isdf_ctx* c, const float* swf, int n_omega) {
  cudaStream_t st = c->stream;
  const int r = c->rank, n_v = c->n_v, n_c = c->n_c;
  const size_t rr = (size_t)r * r;
  const int rp = pad(r, 128), rk = pad(r, 64);
  const int npair = n_v * n_c, kpp = pad(npair, 64);
  const int max_split = std::max(8, tc_min_splits(kpp));
  // also the split of the SYRK of G that follows on this stream: size the
  // partials once, before anything runs on the second stream
  const int max_split_g = std::max(8, tc_min_splits(pad(2 * c->n_half, 64)));
  MK(ensure(c->partial, (size_t)std::max(max_split, max_split_g) * rr));
  MK(ensure(c->tmp1, rr));
  MK(ensure(c->tmp2, rr));
  const size_t np = (size_t)NSL * rp * kpp;
  MK(ensure_bf16(c->m_pairs, np));
  for (int k = 0; k < n_omega; ++k) {
    double* Dk = c->D.p + rr * k;
    {
      PhaseTimer ph(c, ISDF_PH_POLAR_D);
      MK(launch_pair_slices(c->phimu_p.p, r, r, n_v, n_c, swf + (size_t)npair * k, c->m_pairs.bf(), rp, kpp, NSL,
                            st));
      MK(tc_gemm_f64(op(c->m_pairs, rp, kpp), op(c->m_pairs, rp, kpp), r, r, 1.0, 0.0, c->tmp1.p, r, true, false,
                     c->partial.p, max_split, c->num_sms, c->d_status, st));
    }
    MK(mixed_whiten_D(c, c->tmp1.p, Dk));
  }
  return cudaSuccess;
}

// D = L^-1 D_pp L^-T (symmetrised) on the tensor cores; D_pp may be c->tmp1.
cudaError_t mixed_whiten_D(isdf_ctx* c, const double* Dpp, double* Dk) {
  cudaStream_t st = c->stream;
  const int r = c->rank;
  const size_t rr = (size_t)r * r;
  const int rp = pad(r, 128), rk = pad(r, 64);
  MK(ensure(c->tmp2, rr));
  PhaseTimer ph(c, ISDF_PH_WHITEN_D);
  // X = L^-1 D_pp, then D = X L^-T
  MK(slices_cm(c->m_sa, Dpp, r, r, r, rp, rk, st));
  MK(tc_gemm_f64(op(c->m_linvs, rp, rk), op(c->m_sa, rp, rk), r, r, 1.0, 0.0, c->tmp2.p, r, false, false, nullptr, 1,
                 c->num_sms, c->d_status, st));
  MK(slices_cm(c->m_sa, c->tmp2.p, r, r, r, rp, rk, st));
  MK(tc_gemm_f64(op(c->m_sa, rp, rk), op(c->m_linvs, rp, rk), r, r, 1.0, 0.0, Dk, r, false, true, nullptr, 1,
                 c->num_sms, c->d_status, st));
  return launch_symmetrize(Dk, r, r, st);
}

// D(w_k) for all frequencies: the same products as mixed_polar_D, each one
// launch for a chunk of frequencies whose pair slices fit the budget.
cudaError_t mixed_polar_D_batched(isdf_ctx* c, const float* swf, int n_omega) {
  cudaStream_t st = c->stream;
  const int r = c->rank, n_v = c->n_v, n_c = c->n_c;
  const size_t rr = (size_t)r * r;
  const int rp = pad(r, 128), rk = pad(r, 64);
  const int npair = n_v * n_c, kpp = pad(npair, 64);
  const size_t per_pair = (size_t)NSL * rp * kpp, per_sq = (size_t)NSL * rp * rk;
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>(n_omega, kPairSliceBudget / (per_pair * 2)));
  const int ms = tc_min_splits(kpp);  // accumulation-length split of the long pair SYRK
  const int max_split_g = std::max(8, tc_min_splits(pad(2 * c->n_half, 64)));
  // all workspace first: a resize frees memory that queued kernels may use
  if (!tl_capture) MK(cudaStreamSynchronize(st));
  MK(ensure(c->partial, std::max((size_t)ms * chunk, (size_t)max_split_g) * rr));
  MK(ensure_bf16(c->m_pairs, per_pair * chunk));
  MK(ensure_bf16(c->b_s1, per_sq * chunk));
  MK(ensure(c->b_dtmp, 2 * rr * chunk));
  double* Dpp = c->b_dtmp.p;
  double* X = c->b_dtmp.p + rr * chunk;
  for (int k0 = 0; k0 < n_omega; k0 += chunk) {
    const int nb = std::min(chunk, n_omega - k0);
    {
      PhaseTimer ph(c, ISDF_PH_POLAR_D);
      MK(launch_pair_slices(c->phimu_p.p, r, r, n_v, n_c, swf + (size_t)npair * k0, c->m_pairs.bf(), rp, kpp, NSL,
                            st, nb, (long long)per_pair));
      const int pr = NSL * rp;
      MK(tc_gemm_f64_batched(op(c->m_pairs, rp, kpp), op(c->m_pairs, rp, kpp), r, r, 1.0, 0.0, Dpp, r, true, false,
                             ms > 1 ? c->partial.p : nullptr, ms, c->num_sms, c->d_status, st,
                             TcBatch{nb, pr, pr, (long long)rr}));
    }
    PhaseTimer ph(c, ISDF_PH_WHITEN_D);
    const int sr = NSL * rp;
    MK(slices_cm_b(c->b_s1, Dpp, r, rr, r, r, rp, rk, nb, st));
    MK(tc_gemm_f64_batched(op(c->m_linvs, rp, rk), op(c->b_s1, rp, rk), r, r, 1.0, 0.0, X, r, false, false, nullptr,
                           1, c->num_sms, c->d_status, st, TcBatch{nb, 0, sr, (long long)rr}));
    MK(slices_cm_b(c->b_s1, X, r, rr, r, r, rp, rk, nb, st));
    MK(tc_gemm_f64_batched(op(c->b_s1, rp, rk), op(c->m_linvs, rp, rk), r, r, 1.0, 0.0, c->D.p + rr * k0, r, false,
                           true, nullptr, 1, c->num_sms, c->d_status, st, TcBatch{nb, sr, 0, (long long)rr}));
    MK(launch_symmetrize(c->D.p + rr * k0, r, r, st, nb, (long long)rr));
  }
  return cudaSuccess;
}

// D(w_k) for all frequencies by whitening in pair space: S~ = L^-1 C_r
// diag(sqrt(-2 Omega^-1)) comes out of one GEMM as BF16 slices (the
// transposed pair operand is the B side, the weights scale its columns in
// the epilogue), then D = S~ S~^T.  The FP32-grade error of the pair
// operand reaches D multiplied by cond(L) instead of cond(L)^2 as in
// L^-1 (C_r diag C_r^T) L^-T, at the cost of the r x pairs x r GEMM.
cudaError_t mixed_polar_D_pairspace(isdf_ctx* c, const float* swf, int n_omega) {
  cudaStream_t st = c->stream;
  const int r = c->rank, n_v = c->n_v, n_c = c->n_c;
  const size_t rr = (size_t)r * r;
  const int rp = pad(r, 128), rk = pad(r, 64);
  const int npair = n_v * n_c, kpp = pad(npair, 64), Pp = pad(npair, 128);
  const size_t per_pair = (size_t)NSL * rp * kpp, n_t = (size_t)NSL * Pp * rk;
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>(n_omega, kPairSliceBudget / (per_pair * 2)));
  const int ms = tc_min_splits(kpp);
  const int max_split_g = std::max(8, tc_min_splits(pad(2 * c->n_half, 64)));
  if (!tl_capture) MK(cudaStreamSynchronize(st));
  MK(ensure(c->partial, std::max((size_t)std::max(ms, 8) * chunk, (size_t)max_split_g) * rr));
  MK(ensure_bf16(c->m_pairs, per_pair * chunk));
  MK(ensure_bf16(c->m_pairs_t, n_t));
  {
    PhaseTimer ph(c, ISDF_PH_POLAR_D);
    MK(cudaMemsetAsync(c->m_pairs_t.p, 0, n_t * 2, st));
    MK(launch_pair_slices_t(c->phimu_p.p, r, r, n_v, n_c, c->m_pairs_t.bf(), Pp, rk, NSL, st));
  }
  for (int k0 = 0; k0 < n_omega; k0 += chunk) {
    const int nb = std::min(chunk, n_omega - k0);
    {
      PhaseTimer ph(c, ISDF_PH_WHITEN_D);
      MK(cudaMemsetAsync(c->m_pairs.p, 0, per_pair * nb * 2, st));
      MK(tc_scaled_slices(op(c->m_linvs, rp, rk), op(c->m_pairs_t, Pp, rk), r, npair, swf + (size_t)npair * k0,
                          npair, c->m_pairs.bf(), rp, kpp, (long long)per_pair, c->d_status, st, TcBatch{nb, 0, 0, 0}));
    }
    PhaseTimer ph(c, ISDF_PH_POLAR_D);
    const int pr = NSL * rp;
    const int msb = std::max(ms, nb == 1 ? 8 : 1);
    MK(tc_gemm_f64_batched(op(c->m_pairs, rp, kpp), op(c->m_pairs, rp, kpp), r, r, 1.0, 0.0, c->D.p + rr * k0, r,
                           true, false, c->partial.p, msb, c->num_sms, c->d_status, st,
                           TcBatch{nb, pr, pr, (long long)rr}));
  }
  return cudaSuccess;
}

// K(w_k) for all frequencies from R(w_k) = c->Rw + k rr: the products of
// mixed_smw_products_T / _K and the FP64 factorisations, one launch per
// step for every frequency.
cudaError_t mixed_smw_batched(isdf_ctx* c, int nw, int* fail_T) {
  cudaStream_t st = c->stream;
  const int r = c->rank, rp = pad(r, 128), rk = pad(r, 64);
  const size_t rr = (size_t)r * r, per_sq = (size_t)NSL * rp * rk;
  const size_t wq = (size_t)(r / 2 + 64) * (r / 2 + 64);
  const long long srr = (long long)rr;
  const int sr = NSL * rp;
  if (!tl_capture) MK(cudaStreamSynchronize(st));
  MK(ensure(c->bW1, rr * nw));
  MK(ensure(c->bT, rr * nw));
  MK(ensure(c->bU, rr * nw));
  MK(ensure(c->bQ, rr * nw));
  MK(ensure_bf16(c->b_s1, per_sq * nw));
  MK(ensure_bf16(c->b_s2, per_sq * nw));
  MK(ensure_bf16(c->b_s3, per_sq));
  MK(ensure(c->b_work, wq * nw));
  MK(ensure(c->b_cb, (size_t)nw));
  MK(ensure(c->b_split, (size_t)64 * r * nw));
  const double* R = c->Rw.p;
  // T = I + R^T (G R)
  MK(slices_cm(c->b_s3, c->G.p, r, r, r, rp, rk, st));
  MK(slices_rm_b(c->b_s1, R, r, srr, r, r, rp, rk, nw, st));
  MK(tc_gemm_f64_batched(op(c->b_s3, rp, rk), op(c->b_s1, rp, rk), r, r, 1.0, 0.0, c->bW1.p, r, false, false, nullptr,
                         1, c->num_sms, c->d_status, st, TcBatch{nw, 0, sr, srr}));
  MK(slices_rm_b(c->b_s2, c->bW1.p, r, srr, r, r, rp, rk, nw, st));
  MK(cudaMemsetAsync(c->bT.p, 0, rr * nw * sizeof(double), st));
  MK(launch_add_identity(c->bT.p, r, r, 1.0, st, nw, srr));
  MK(tc_gemm_f64_batched(op(c->b_s1, rp, rk), op(c->b_s2, rp, rk), r, r, 1.0, 1.0, c->bT.p, r, false, false, nullptr,
                         1, c->num_sms, c->d_status, st, TcBatch{nw, sr, sr, srr}));
  MK(launch_symmetrize(c->bT.p, r, r, st, nw, srr));
  // T = U U^T (FP64), U^-1, Q = R U^-T, K = -Q Q^T
  MK(launch_cholesky_blocked_batched(c->bT.p, r, srr, r, nw, 0.0, c->bU.p, r, srr, c->b_cb.p, fail_T, st,
                                     reinterpret_cast<float2*>(c->b_split.p)));
  {
    DfGemm df(true);
    MK(launch_tri_inverse_batched(c->bU.p, r, srr, r, nw, c->bQ.p, r, srr, c->b_work.p, st));
  }
  MK(slices_cm_b(c->b_s1, R, r, srr, r, r, rp, rk, nw, st));
  MK(slices_cm_b(c->b_s2, c->bQ.p, r, srr, r, r, rp, rk, nw, st));
  MK(tc_gemm_f64_batched(op(c->b_s1, rp, rk), op(c->b_s2, rp, rk), r, r, 1.0, 0.0, c->bW1.p, r, false, true, nullptr,
                         1, c->num_sms, c->d_status, st, TcBatch{nw, sr, sr, srr}));
  MK(slices_cm_b(c->b_s1, c->bW1.p, r, srr, r, r, rp, rk, nw, st));
  return tc_gemm_f64_batched(op(c->b_s1, rp, rk), op(c->b_s1, rp, rk), r, r, -1.0, 0.0, c->K.p, r, true, false,
                             nullptr, 1, c->num_sms, c->d_status, st, TcBatch{nw, sr, sr, srr});
}

// K = -Q Q^T for frequency k into Kk (r x r).  Needs the unpivoted FP64
// Cholesky of the host side (passed in as a callback-free sequence: the
// caller factors D into c->R and T into c->W1).
cudaError_t mixed_smw_products_T(isdf_ctx* c) {
  // T = I + R^T (G R), T in c->T (identity already set)
  cudaStream_t st = c->stream;
  const int r = c->rank, rp = pad(r, 128), rk = pad(r, 64);
  MK(slices_cm(c->m_sa, c->G.p, r, r, r, rp, rk, st));
  MK(slices_rm(c->m_sb, c->R.p, r, r, r, rp, rk, st));  // rows = columns of R
  MK(tc_gemm_f64(op(c->m_sa, rp, rk), op(c->m_sb, rp, rk), r, r, 1.0, 0.0, c->W1.p, r, false, false, nullptr, 1,
                 c->num_sms, c->d_status, st));
  MK(slices_rm(c->m_sa, c->W1.p, r, r, r, rp, rk, st));
  MK(tc_gemm_f64(op(c->m_sb, rp, rk), op(c->m_sa, rp, rk), r, r, 1.0, 1.0, c->T.p, r, false, false, nullptr, 1,
                 c->num_sms, c->d_status, st));
  return launch_symmetrize(c->T.p, r, r, st);
}

cudaError_t mixed_smw_products_K(isdf_ctx* c, double* Kk, bool uinv_ready) {
  // U in c->W1 (and U^-1 in c->Q when uinv_ready): Q = R U^-T, K = -Q Q^T
  cudaStream_t st = c->stream;
  const int r = c->rank, rp = pad(r, 128), rk = pad(r, 64);
  const size_t rr = (size_t)r * r;
  const int max_split = 8;
  const size_t wq = (size_t)(r / 2 + 64) * (r / 2 + 64);
  MK(ensure(c->m_work, 5 * wq));
  MK(ensure(c->partial, (size_t)max_split * rr));
  if (!uinv_ready) MK(launch_tri_inverse(c->W1.p, r, r, c->Q.p, r, c->m_work.p, c->m_work.p + wq, st));  // Q <- U^-1
  MK(slices_cm(c->m_sa, c->R.p, r, r, r, rp, rk, st));
  MK(slices_cm(c->m_sb, c->Q.p, r, r, r, rp, rk, st));
  MK(tc_gemm_f64(op(c->m_sa, rp, rk), op(c->m_sb, rp, rk), r, r, 1.0, 0.0, c->Q.p, r, false, true, nullptr, 1,
                 c->num_sms, c->d_status, st));
  MK(slices_cm(c->m_sa, c->Q.p, r, r, r, rp, rk, st));
  return tc_gemm_f64(op(c->m_sa, rp, rk), op(c->m_sa, rp, rk), r, r, -1.0, 0.0, Kk, r, true, false, c->partial.p,
                     max_split, c->num_sms, c->d_status, st);
}

// The Newton-Schulz schedule for a spectrum of alpha M within [1 - e0,
// 1 + e0] (alpha = 2 / (lo + hi), e0 = (hi - lo) / (hi + lo)).  A step maps
// each eigenvalue t of M X to t (2 - t), so [1 - e, 1 + e] goes to
// [1 - e^2, 1]; the scale beta = 2 / (2 - e^2) centres it again, and
// e <- e^2 / (2 - e^2) (from e0 = 0.84, kappa 11.5: 5 steps instead of 7).
// Each step's products take the fewest BF16 slices whose rounding (about
// 2^(1 - 8 s) kappa relative, kappa = hi / lo) stays below a quarter of the
// error the step leaves; the last two take all three, so the result carries
// the three-slice rounding only (the iteration corrects the rounding of the
// earlier steps like any other error).  Stops when e < 2^-26.
bool ns_plan(double e0, NsPlan& p) {
  p.beta.clear();
  p.s.clear();
  if (!(e0 >= 0.0) || !(e0 < 1.0)) return false;
  const double kappa = (1.0 + e0) / (1.0 - e0);
  double e = e0;
  while (e > 0x1p-26) {
    if (p.steps() >= 12) return false;
    p.beta.push_back(2.0 / (2.0 - e * e));
    e = e * e / (2.0 - e * e);
    p.s.push_back(kappa * 0x1p-7 <= 0.25 * e ? 1 : (kappa * 0x1p-15 <= 0.25 * e ? 2 : NSL));
  }
  if (p.beta.empty()) {  // alpha M = I to 2^-26 already: one full step
    p.beta.push_back(1.0);
    p.s.push_back(NSL);
  }
  for (int k = std::max(0, p.steps() - 2); k < p.steps(); ++k) p.s[k] = NSL;
  return true;
}

void pair_weight_bounds(const double* energies, int n_v, int n_c, double w, double* wmin, double* wmax) {
  double emax_v = energies[0], emin_v = energies[0], emin_c = energies[n_v], emax_c = energies[n_v];
  for (int i = 0; i < n_v; ++i) {
    emax_v = std::max(emax_v, energies[i]);
    emin_v = std::min(emin_v, energies[i]);
  }
  for (int j = n_v; j < n_v + n_c; ++j) {
    emin_c = std::min(emin_c, energies[j]);
    emax_c = std::max(emax_c, energies[j]);
  }
  const double gap = emin_c - emax_v, width = emax_c - emin_v;
  auto f = [w](double d) { return 2.0 * d / (d * d + w * w); };
  *wmin = std::min(f(gap), f(width));
  *wmax = std::max(f(gap), f(width));
  if (w >= gap && w <= width) *wmax = std::max(*wmax, f(w));
}

double ns_kappa(double g_bound, double d_bound) { return 1.0 + std::max(0.0, g_bound) * std::max(0.0, d_bound); }

namespace {

// Grouped-GEMM descriptor slots of the batched capacitance: 0 the products
// G D(w), 1 the results -D(w) X(w), 2 + 2 step + kind the iteration (kind 0
// Z = M X, kind 1 X <- beta (2 X - X Z)); each has its own scale, slice
// count and operands, so its own descriptors.
inline int ns_slot(int step, int kind) { return 2 + 2 * step + kind; }
constexpr int kNsSlots = 2 + 2 * 12;

}  // namespace

// K = -D (I + G D)^-1 = -(D^-1 + G)^-1 (reading 20) on the tensor cores:
// M = I + G D, X -> M^-1 by Newton-Schulz X <- beta_k (2 X - X (M X)) from
// X = alpha I (schedule of ns_plan), then K = -D X.  G D has the spectrum of
// D^1/2 G D^1/2, so M has real eigenvalues in [1, kappa], kappa = 1 +
// |G| |D| (the bounds of ns_kappa), and alpha = 2 / (1 + kappa).  M is not
// symmetric, and the form is what keeps the iteration stable under
// rounding: a perturbation P of X enters the next iterate as 2 P - P M X -
// X M P, which vanishes at X = M^-1 whatever P is, where X (2 I - M X)
// with a rounded or symmetrised middle factor lets the modes of
// P - M^-1 P M grow once the iteration has converged.  Every product is a
// full tensor-core GEMM; K, symmetric in exact arithmetic, is the lower
// triangle of -D X, mirrored.  X stays in c->Xgd for the refinement of the
// apply.  M needs no bound, so mixed_ns_prepare builds it first, while the
// host reads the bounds; mixed_ns_iterate follows on the same stream.
cudaError_t mixed_ns_prepare(isdf_ctx* c, const double* Dk) {
  cudaStream_t st = c->stream;
  const int r = c->rank, rp = pad(r, 128), rk = pad(r, 64);
  const size_t rr = (size_t)r * r;
  double* M = c->T.p;
  MK(cudaMemsetAsync(M, 0, rr * sizeof(double), st));
  MK(launch_add_identity(M, r, r, 1.0, st));
  MK(slices_cm(c->m_sd, c->G.p, r, r, r, rp, rk, st));  // rows of G
  MK(slices_cm(c->m_sa, Dk, r, r, r, rp, rk, st));      // rows of D (= its columns)
  MK(tc_gemm_f64(op(c->m_sd, rp, rk), op(c->m_sa, rp, rk), r, r, 1.0, 1.0, M, r, false, false, nullptr, 1,
                 c->num_sms, c->d_status, st));  // M = I + G D
  return slices_cm(c->m_sd, M, r, r, r, rp, rk, st);  // rows of M, once
}

cudaError_t mixed_ns_iterate(isdf_ctx* c, const double* Dk, double* Kk, double alpha, const NsPlan& plan) {
  cudaStream_t st = c->stream;
  const int r = c->rank, rp = pad(r, 128), rk = pad(r, 64);
  const size_t rr = (size_t)r * r;
  double* X = c->Xgd.p;
  double* Z = c->R.p;
  MK(cudaMemsetAsync(X, 0, rr * sizeof(double), st));
  MK(launch_add_identity(X, r, r, alpha, st));
  for (int it = 0; it < plan.steps(); ++it) {
    const int s = plan.s[it];
    const double b = plan.beta[it];
    MK(slices_rm(c->m_sa, X, r, r, r, rp, rk, st));  // columns of X
    MK(tc_gemm_f64(op_s(c->m_sd, rp, rk, s), op_s(c->m_sa, rp, rk, s), r, r, 1.0, 0.0, Z, r, false, false, nullptr, 1,
                   c->num_sms, c->d_status, st));  // Z = M X
    MK(slices_cm(c->m_sa, X, r, r, r, rp, rk, st));  // rows of X
    MK(slices_rm(c->m_sb, Z, r, r, r, rp, rk, st));  // columns of Z
    MK(tc_gemm_f64(op_s(c->m_sa, rp, rk, s), op_s(c->m_sb, rp, rk, s), r, r, -b, 2.0 * b, X, r, false, false, nullptr,
                   1, c->num_sms, c->d_status, st));  // X <- beta (2 X - X Z), in place
  }
  MK(slices_cm(c->m_sd, Dk, r, r, r, rp, rk, st));  // rows of D
  MK(slices_rm(c->m_sa, X, r, r, r, rp, rk, st));   // columns of X
  return tc_gemm_f64(op(c->m_sd, rp, rk), op(c->m_sa, rp, rk), r, r, -1.0, 0.0, Kk, r, true, false, nullptr, 1,
                     c->num_sms, c->d_status, st);  // K = -D X
}

namespace {

void pair_weight_range(const isdf_ctx* c, int k, double* wmin, double* wmax) {
  pair_weight_bounds(c->energies.data(), c->n_v, c->n_c, c->omega[k], wmin, wmax);
}

// The capacitance of every frequency of one context (or of several, ncs >
// 1) by the steps of `plan`: each product of every context, frequency and
// tile is one work unit of a single grouped persistent launch.  Per
// context: X(w) in bW1, M(w) in bT, Z(w) in bQ; slices in b_s1, b_s2, b_s4;
// start scales in ns_alpha.  Descriptor slot q of the launch lives at
// work + q * ws, its host copy in staged[q].
cudaError_t ns_capacitance_grouped(isdf_ctx** cs, int ncs, const NsPlan& plan, cudaStream_t st, unsigned char* work,
                                   size_t ws, std::vector<std::vector<unsigned char>>& staged) {
  std::vector<TcGroupProblem> pr;
  isdf_ctx* c0 = cs[0];
  auto launch = [&](int slot) -> cudaError_t {
    return tc_gemm_f64_grouped(pr.data(), (int)pr.size(), work + slot * ws, ws, staged[slot], c0->num_sms,
                               c0->d_status, st);
  };
  // M(w) = I + G D(w)
  pr.clear();
  for (int i = 0; i < ncs; ++i) {
    isdf_ctx* c = cs[i];
    const int r = c->rank, rp = pad(r, 128), rk = pad(r, 64), nw = c->n_omega, sr = NSL * rp;
    const long long rr = (long long)r * r;
    MK(cudaMemsetAsync(c->bT.p, 0, (size_t)rr * nw * sizeof(double), st));
    MK(launch_add_identity(c->bT.p, r, r, 1.0, st, nw, rr));
    MK(slices_cm_b(c->b_s1, c->G.p, r, rr, r, r, rp, rk, 1, st));  // rows of G, shared by every frequency
    MK(slices_cm_b(c->b_s2, c->D.p, r, rr, r, r, rp, rk, nw, st));
    pr.push_back(TcGroupProblem{op(c->b_s1, rp, rk), op(c->b_s2, rp, rk), r, r, 1.0, 1.0, c->bT.p, r, false,
                                TcBatch{nw, 0, sr, rr}});
  }
  MK(launch(0));
  for (int i = 0; i < ncs; ++i) {
    isdf_ctx* c = cs[i];
    const int r = c->rank, rp = pad(r, 128), rk = pad(r, 64), nw = c->n_omega;
    const long long rr = (long long)r * r;
    MK(slices_cm_b(c->b_s1, c->bT.p, r, rr, r, r, rp, rk, nw, st));  // rows of M(w), once
    MK(launch_scaled_identity(c->bW1.p, r, nw, c->ns_alpha.p, st));
  }
  for (int it = 0; it < plan.steps(); ++it) {
    const int s = plan.s[it];
    const double b = plan.beta[it];
    pr.clear();
    for (int i = 0; i < ncs; ++i) {
      isdf_ctx* c = cs[i];
      const int r = c->rank, rp = pad(r, 128), rk = pad(r, 64), nw = c->n_omega, sr = NSL * rp;
      const long long rr = (long long)r * r;
      MK(slices_rm_b(c->b_s2, c->bW1.p, r, rr, r, r, rp, rk, nw, st));  // columns of X
      pr.push_back(TcGroupProblem{op_s(c->b_s1, rp, rk, s), op_s(c->b_s2, rp, rk, s), r, r, 1.0, 0.0, c->bQ.p, r,
                                  false, TcBatch{nw, sr, sr, rr}});
    }
    MK(launch(ns_slot(it, 0)));  // Z = M X
    pr.clear();
    for (int i = 0; i < ncs; ++i) {
      isdf_ctx* c = cs[i];
      const int r = c->rank, rp = pad(r, 128), rk = pad(r, 64), nw = c->n_omega, sr = NSL * rp;
      const long long rr = (long long)r * r;
      MK(slices_cm_b(c->b_s2, c->bW1.p, r, rr, r, r, rp, rk, nw, st));  // rows of X
      MK(slices_rm_b(c->b_s4, c->bQ.p, r, rr, r, r, rp, rk, nw, st));   // columns of Z
      pr.push_back(TcGroupProblem{op_s(c->b_s2, rp, rk, s), op_s(c->b_s4, rp, rk, s), r, r, -b, 2.0 * b, c->bW1.p, r,
                                  false, TcBatch{nw, sr, sr, rr}});
    }
    MK(launch(ns_slot(it, 1)));  // X <- beta (2 X - X Z), in place
  }
  // K(w) = -D(w) X(w), the lower triangle mirrored
  pr.clear();
  for (int i = 0; i < ncs; ++i) {
    isdf_ctx* c = cs[i];
    const int r = c->rank, rp = pad(r, 128), rk = pad(r, 64), nw = c->n_omega, sr = NSL * rp;
    const long long rr = (long long)r * r;
    MK(slices_cm_b(c->b_s1, c->D.p, r, rr, r, r, rp, rk, nw, st));
    MK(slices_rm_b(c->b_s2, c->bW1.p, r, rr, r, r, rp, rk, nw, st));
    pr.push_back(TcGroupProblem{op(c->b_s1, rp, rk), op(c->b_s2, rp, rk), r, r, -1.0, 0.0, c->K.p, r, true,
                                TcBatch{nw, sr, sr, rr}});
  }
  MK(launch(1));
  for (int i = 0; i < ncs; ++i) MK(cudaMemsetAsync(cs[i]->b_fail, 0xff, cs[i]->n_omega * sizeof(int), st));
  return cudaSuccess;
}

}  // namespace

cudaError_t mixed_smw_batched_ns(isdf_ctx* c, int nw, int* fail_T, bool* used) {
  cudaStream_t st = c->stream;
  *used = false;
  const int r = c->rank, rp = pad(r, 128), rk = pad(r, 64);
  const size_t rr = (size_t)r * r, per_sq = (size_t)NSL * rp * rk;
  const size_t ws = (tc_grouped_workspace_bytes(1) + 255) / 256 * 256;
  if (!tl_capture) {
    MK(cudaStreamSynchronize(st));  // the buffers below may grow
    MK(ensure(c->bW1, rr * nw));
    MK(ensure(c->bT, rr * nw));
    MK(ensure(c->bQ, rr * nw));
    MK(ensure_bf16(c->b_s1, per_sq * nw));
    MK(ensure_bf16(c->b_s2, per_sq * nw));
    MK(ensure_bf16(c->b_s4, per_sq * nw));
    MK(ensure(c->ns_work, (kNsSlots * ws + 7) / 8));
    if (c->ns_staged.size() < (size_t)kNsSlots) c->ns_staged.resize(kNsSlots);
    MK(ensure(c->ns_alpha, (size_t)nw));
    const size_t bw = row_abs_sum_work(r, nw);
    MK(ensure(c->ns_bound, bw + (size_t)nw + 8));
    // spectra: rigorous bounds only (Gershgorin for every D(w) and for G,
    // the pair-weight range): a schedule planned from an estimate could
    // leave a mode unconverged
    double* nb = c->ns_bound.p;
    double* lam = nb + bw;  // [nw Gershgorin of D | Gershgorin of G]
    MK(launch_row_abs_sum_max(c->D.p, r, r, lam, nb, st, nw, (long long)rr));
    MK(launch_row_abs_sum_max(c->G.p, r, r, lam + nw, nb, st));
    std::vector<double> h((size_t)nw + 1);
    MK(cudaMemcpyAsync(h.data(), lam, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    MK(cudaStreamSynchronize(st));
    std::vector<double> alpha((size_t)nw);
    double e0 = 0.0;
    for (int k = 0; k < nw; ++k) {
      double wmin = 0.0, wmax = 0.0;
      pair_weight_range(c, k, &wmin, &wmax);
      const double kappa = ns_kappa(h[nw], std::min(wmax, h[k]));
      if (!std::isfinite(kappa)) return cudaSuccess;  // not used: the caller factors
      alpha[k] = 2.0 / (1.0 + kappa);
      // one schedule for every frequency: the largest e0 (a scale sequence
      // valid for e0 keeps every smaller e0 within the same bounds)
      e0 = std::max(e0, (kappa - 1.0) / (kappa + 1.0));
    }
    NsPlan plan;
    if (!ns_plan(e0, plan)) return cudaSuccess;  // too many steps: the caller factors
    MK(cudaMemcpyAsync(c->ns_alpha.p, alpha.data(), alpha.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    MK(cudaStreamSynchronize(st));
    c->ns_e0 = e0;
    c->ns_nw = nw;
  } else if (c->ns_nw != nw || c->ns_e0 < 0.0) {
    return cudaErrorStreamCaptureUnsupported;  // a captured call needs the eager call's plan
  }
  NsPlan plan;
  ns_plan(c->ns_e0, plan);
  MK(ns_capacitance_grouped(&c, 1, plan, st, reinterpret_cast<unsigned char*>(c->ns_work.p), ws, c->ns_staged));
  (void)fail_T;  // set to "nothing failed" with the context's flags
  *used = true;
  return cudaSuccess;
}

// The capacitance stage of smw_inverse_all for several systems at once:
// every Newton-Schulz product of every system (all frequencies, all tiles)
// in one grouped persistent launch per product.  Each context must hold the
// plan of an earlier eager smw_inverse_all on the same polarizability (the
// start scales on the device, the largest e0); every system follows the
// schedule of the largest e0 over the systems (valid for all of them, and
// one slice count per launch, as the grouped kernel needs).  Descriptor
// slot q lives at work + q * ws with its host copy in staged[q];
// ns_stage_slots() slots in all.
int ns_stage_slots() { return kNsSlots; }

cudaError_t ns_stage_grouped(isdf_ctx** cs, int n, cudaStream_t st, void* work, size_t ws,
                             std::vector<std::vector<unsigned char>>& staged) {
  if (n <= 0) return cudaSuccess;
  if (n > 32) return cudaErrorInvalidValue;
  double e0 = 0.0;
  for (int i = 0; i < n; ++i) {
    isdf_ctx* c = cs[i];
    if (c->prec != ISDF_PREC_MIXED || c->rank <= 0 || c->ns_nw != c->n_omega || c->ns_e0 < 0.0)
      return cudaErrorInvalidValue;
    e0 = std::max(e0, c->ns_e0);
  }
  NsPlan plan;
  if (!ns_plan(e0, plan)) return cudaErrorInvalidValue;
  if (staged.size() < (size_t)kNsSlots) staged.resize(kNsSlots);
  return ns_capacitance_grouped(cs, n, plan, st, static_cast<unsigned char*>(work), ws, staged);
}

// Y = X + V theta K theta^T X for one chunk of nc columns.
cudaError_t mixed_apply_chunk(isdf_ctx* c, const double* Kk, const double* X, double* Y, int nc) {
  cudaStream_t st = c->stream;
  const int r = c->rank, rp = pad(r, 128), rk = pad(r, 64);
  const long long nr = c->n_r;
  const int nrp = pad(nr, 128), kpg = pad(nr, 64);
  const int ncp = pad(nc, 128);
  const int max_split = std::max(64, tc_min_splits(kpg));
  MK(ensure(c->partial, (size_t)max_split * r * nc));
  MK(ensure(c->tmp1, (size_t)r * nc));
  MK(ensure(c->tmp2, (size_t)r * nc));
  MK(ensure(c->tmp3, (size_t)nr * nc));
  // T1 = theta^T X
  MK(slices_rm(c->m_xs, X, nr, nc, (int)nr, ncp, kpg, st));
  MK(tc_gemm_f64(op(c->m_thetas_t, rp, kpg), op(c->m_xs, ncp, kpg), r, nc, 1.0, 0.0, c->tmp1.p, r, false, false,
                 c->partial.p, max_split, c->num_sms, c->d_status, st));
  // T2 = K T1 (FP64, small)
  MK(launch_gemm(Kk, r, false, c->tmp1.p, r, true, r, nc, r, 1.0, 0.0, c->tmp2.p, r, false, 16, c->partial.p, true,
                 st));
  if (c->refine > 0 && c->xgd_ready && c->ref.cap >= (size_t)2 * r * nc) {
    // iterative refinement of T2 = -(D^-1 + G)^-1 T1, i.e. of (I + D G) T2 =
    // -D T1: R = -D (T1 + G T2) - T2 in FP64, then T2 += X^T R (the error of
    // T2 solves (I + D G) E = R, and (I + D G)^-1 = ((I + G D)^-1)^T = X^T)
    const size_t blk = (size_t)r * nc, bytes = blk * sizeof(double);
    double* U = c->ref.p;
    double* R = U + blk;
    for (int it = 0; it < c->refine; ++it) {
      MK(cudaMemcpyAsync(U, c->tmp1.p, bytes, cudaMemcpyDeviceToDevice, st));
      MK(launch_gemm(c->G.p, r, false, c->tmp2.p, r, true, r, nc, r, 1.0, 1.0, U, r, false, 16, c->partial.p, true,
                     st));  // U = T1 + G T2
      MK(cudaMemcpyAsync(R, c->tmp2.p, bytes, cudaMemcpyDeviceToDevice, st));
      MK(launch_gemm(c->D.p, r, false, U, r, true, r, nc, r, -1.0, -1.0, R, r, false, 16, c->partial.p, true,
                     st));  // R = -D U - T2
      MK(launch_gemm(c->Xgd.p, r, true, R, r, true, r, nc, r, 1.0, 1.0, c->tmp2.p, r, false, 16, c->partial.p, true,
                     st));  // T2 += X^T R
    }
  }
  // T3 = theta T2
  MK(slices_rm(c->m_xs, c->tmp2.p, r, nc, r, ncp, rk, st));
  MK(tc_gemm_f64(op(c->m_ths, nrp, rk), op(c->m_xs, ncp, rk), (int)nr, nc, 1.0, 0.0, c->tmp3.p, nr, false, false,
                 nullptr, 1, c->num_sms, c->d_status, st));
  // Y = X + V T3
  const long long lds = 2 * c->n_half;
  MK(ensure(c->spec, (size_t)lds * nc));
  return launch_fft_convolve(c->fft, c->tmp3.p, nr, nc, c->spec.p, lds, c->d_wconv, X, nr, Y, nr, c->smem_xy,
                             c->smem_z, st);
}

}  // namespace isdf
