// C ABI of the ISDF-SMW library: context, argument checks and the order of
// kernel launches for isdf_fit / build_polarizability / smw_inverse /
// apply_eps_inv (declared and documented in include/isdf_smw.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/isdf_smw.h"
#include "common.cuh"
#include "kernels.h"

using namespace isdf;

#include "ctx.h"

using isdf::DevBuf;
using isdf::kMaxGrid;
using isdf::kWaitLimitNs;
using isdf::ensure;
using isdf::release;

static thread_local std::string g_create_err;

// Above this value of mean(lambda) mean(1 / lambda) of C C^T (cond(C C^T) of
// about 14 or more) the mixed path whitens D in pair space.
static constexpr double kPairWhitenMean = 4.0;

// SMs that a tensor-core GEMM leaves to the FP64 factorisations running
// beside it on the second stream (fit and polarizability) -- only where the
// factorisations' latency-bound chain of r / 64 steps (about 0.1 ms each,
// on a few SMs) is long next to the GEMM (its issued BF16 flops at about
// 0.7 PFLOP/s); their throughput-bound updates gain nothing from SMs held
// back.  Measured (ms per solve): 48^3 / N_mu = 1536 with 4, 12, 32, 64, 80,
// 100 SMs left: 25.8, 25.4, 25.0, 24.8, 25.4, 27.1; 72^3 / N_mu = 6144 (s
// per solve) with 0, 24, 64: 1.05, 1.08, 1.17.
static constexpr int kFp64Sms = 64;
static int fp64_sms_to_leave(int r, double gemm_flops) {
  const double chain_ms = std::ceil(r / 64.0) * 0.1;
  const double gemm_ms = gemm_flops / 0.7e12;
  return chain_ms > 0.5 * gemm_ms ? kFp64Sms : 0;
}

using PhaseScope = isdf::PhaseTimer;

static int fail(isdf_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

static int cuda_fail(isdf_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(c, ISDF_ERR_CUDA, m);
}

#define CK(expr)                                             \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return cuda_fail(c, _e, #expr);   \
  } while (0)

// host synchronisation, skipped while a graph is captured
#define SYNC(st)                                             \
  do {                                                       \
    if (!isdf::tl_capture) CK(cudaStreamSynchronize(st));    \
  } while (0)

thread_local bool isdf::tl_capture = false;

cudaError_t isdf::ensure(DevBuf& b, size_t n) {
  if (n <= b.cap) return cudaSuccess;
  if (tl_capture) return cudaErrorStreamCaptureUnsupported;  // sized by the eager run before the capture
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  cudaError_t e = isdf::dev_malloc(&b.p, std::max<size_t>(n, 1) * sizeof(double));
  if (e == cudaSuccess) b.cap = n;
  return e;
}

void isdf::release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

static bool factorize(int n, FftAxis& ax) {
  ax.n = n;
  ax.nf = 0;
  int m = n;
  while (m % 4 == 0 && ax.nf < FFT_MAX_FACTORS) {
    ax.f[ax.nf++] = 4;
    m /= 4;
  }
  const int primes[] = {2, 3, 5, 7, 11, 13};
  for (int p : primes)
    while (m % p == 0 && ax.nf < FFT_MAX_FACTORS) {
      ax.f[ax.nf++] = p;
      m /= p;
    }
  return m == 1;
}

static int signed_freq(int k, int n) { return (2 * k < n) ? k : (2 * k == n ? k : k - n); }

// The error a device status word reports, if any.
static int status_error(isdf_ctx* c, unsigned st, const char* where) {
  if (st & ST_TIMEOUT) return fail(c, ISDF_ERR_TIMEOUT, std::string(where) + ": device wait timed out");
  if (st & ST_NONFINITE) return fail(c, ISDF_ERR_NONFINITE, std::string(where) + ": NaN or Inf in input");
  if (st & ST_NOT_SPD)
    return fail(c, ISDF_ERR_NOT_SPD, std::string(where) + ": matrix not positive definite");
  if (st & ST_BADINDEX) return fail(c, ISDF_ERR_INDEX, std::string(where) + ": index out of range");
  return ISDF_OK;
}

// Reads back the device status word (the stream must be synchronised).
static int check_status(isdf_ctx* c, const char* where) {
  unsigned st = 0;
  cudaError_t e = cudaMemcpy(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  return status_error(c, st, where);
}

extern "C" const char* isdf_version(void) { return "isdf-smw-gb300 0.1 (fp64, sm_103a)"; }

extern "C" const char* isdf_last_error(isdf_ctx* c) {
  return c ? c->err.c_str() : g_create_err.c_str();
}

extern "C" int isdf_create(isdf_ctx** out, int n1, int n2, int n3, double L1, double L2, double L3,
                           void* stream) {
  g_create_err.clear();
  if (!out) {
    g_create_err = "isdf_create: ctx is NULL";
    return ISDF_ERR_ARG;
  }
  *out = nullptr;
  int nn[3] = {n1, n2, n3};
  double ll[3] = {L1, L2, L3};
  for (int i = 0; i < 3; ++i) {
    if (nn[i] < 2 || nn[i] > 512) {
      g_create_err = "isdf_create: grid sizes must be in [2, 512]";
      return ISDF_ERR_SHAPE;
    }
    if (!(ll[i] > 0.0) || !std::isfinite(ll[i])) {
      g_create_err = "isdf_create: cell lengths must be positive and finite";
      return ISDF_ERR_SHAPE;
    }
  }
  isdf_ctx* c = new isdf_ctx();
  c->stream = (cudaStream_t)stream;
  for (int i = 0; i < 3; ++i) {
    c->n[i] = nn[i];
    c->L[i] = ll[i];
    if (!factorize(nn[i], c->fft.ax[i])) {
      delete c;
      g_create_err = "isdf_create: grid sizes must be products of primes <= 13";
      return ISDF_ERR_SHAPE;
    }
  }
  c->fft.h = n1 / 2 + 1;
  c->n_r = (long long)n1 * n2 * n3;
  c->n_half = (long long)c->fft.h * n2 * n3;
  c->dv = L1 * L2 * L3 / (double)c->n_r;
  auto bail = [&](cudaError_t e, const char* w) {
    g_create_err = std::string("isdf_create: ") + w + ": " + cudaGetErrorString(e);
    if (c->d_tables) cudaFree(c->d_tables);
    if (c->d_status) cudaFree(c->d_status);
    delete c;
    return ISDF_ERR_CUDA;
  };
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return bail(e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) return bail(e, "cudaDeviceGetAttribute");
  int smem_optin = 0;
  e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (e != cudaSuccess) return bail(e, "cudaDeviceGetAttribute");
  c->smem_xy = fft_smem_xy(c->fft);
  c->smem_z = fft_smem_z(c->fft);
  if (c->smem_xy > (size_t)smem_optin || c->smem_z > (size_t)smem_optin) {
    delete c;
    g_create_err = "isdf_create: an xy plane or z pencil of this grid does not fit in shared memory";
    return ISDF_ERR_SHAPE;
  }
  e = fft_configure(c->smem_xy, c->smem_z);
  if (e != cudaSuccess) return bail(e, "fft_configure");
  // host tables: twiddles (float64 host cos / sin) and Coulomb weights
  size_t ntw = 2 * (size_t)(n1 + n2 + n3);
  size_t nh = (size_t)c->n_half;
  std::vector<double> tab(ntw + 2 * nh);
  size_t off = 0;
  size_t tw_off[3];
  for (int a = 0; a < 3; ++a) {
    tw_off[a] = off;
    for (int t = 0; t < nn[a]; ++t) {
      double ang = 2.0 * M_PI * (double)t / (double)nn[a];
      tab[off + 2 * t] = std::cos(ang);
      tab[off + 2 * t + 1] = -std::sin(ang);
    }
    off += 2 * (size_t)nn[a];
  }
  const int h = c->fft.h;
  for (int kz = 0; kz < n3; ++kz)
    for (int ky = 0; ky < n2; ++ky)
      for (int kx = 0; kx < h; ++kx) {
        size_t q = ((size_t)kz * n2 + ky) * h + kx;
        double g1 = 2.0 * M_PI * signed_freq(kx, n1) / L1;
        double g2 = 2.0 * M_PI * signed_freq(ky, n2) / L2;
        double g3 = 2.0 * M_PI * signed_freq(kz, n3) / L3;
        double gg = g1 * g1 + g2 * g2 + g3 * g3;
        double vg = gg > 0.0 ? 4.0 * M_PI / gg : 0.0;
        // half spectrum: kx = 0 (and kx = n1/2 for even n1) stand for themselves only
        double wx = (kx == 0 || 2 * kx == n1) ? 1.0 : 2.0;
        tab[ntw + q] = std::sqrt(wx * vg / ((double)c->n_r * c->dv));
        tab[ntw + nh + q] = vg / (c->dv * (double)c->n_r);
      }
  e = isdf::dev_malloc(&c->d_tables, tab.size() * sizeof(double));
  if (e != cudaSuccess) return bail(e, "cudaMalloc tables");
  e = cudaMemcpy(c->d_tables, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(e, "cudaMemcpy tables");
  for (int a = 0; a < 3; ++a) c->fft.ax[a].tw = c->d_tables + tw_off[a];
  c->d_wsyrk = c->d_tables + ntw;
  c->d_wconv = c->d_tables + ntw + nh;
  e = isdf::dev_malloc(&c->d_status, 64 * sizeof(unsigned));
  if (e != cudaSuccess) return bail(e, "cudaMalloc status");
  {
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->s2, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->s3, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->s4, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join3, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(e, "stream / event creation");
  }
  c->d_bar = c->d_status + 8;
  c->d_ints = (int*)(c->d_status + 16);
  e = cudaMemset(c->d_status, 0, 64 * sizeof(unsigned));
  if (e != cudaSuccess) return bail(e, "cudaMemset status");
  *out = c;
  return ISDF_OK;
}

extern "C" int isdf_destroy(isdf_ctx* c) {
  if (!c) return ISDF_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  if (c->s2) {
    cudaStreamSynchronize(c->s2);
    cudaStreamDestroy(c->s2);
  }
  if (c->s4) {
    cudaStreamSynchronize(c->s4);
    cudaStreamDestroy(c->s4);
  }
  if (c->s3) {
    cudaStreamSynchronize(c->s3);
    cudaStreamDestroy(c->s3);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_join3) cudaEventDestroy(c->ev_join3);
  for (cudaEvent_t e : c->ev_chol) cudaEventDestroy(e);
  if (c->d_fail) cudaFree(c->d_fail);
  if (c->b_fail) cudaFree(c->b_fail);
  DevBuf* bufs[] = {&c->phimu, &c->phimu_p, &c->A, &c->Lr, &c->Lc, &c->Bf, &c->chol_d, &c->chol_part,
                    &c->spec, &c->G, &c->D, &c->K, &c->R, &c->T, &c->W1, &c->Q, &c->partial,
                    &c->tmp1, &c->tmp2, &c->tmp3, &c->sw, &c->m_phis, &c->m_phimus, &c->m_zs, &c->m_linv,
                    &c->m_linvs, &c->m_work, &c->m_thetas_t, &c->m_s32, &c->m_ss, &c->m_pairs, &c->m_sa,
                    &c->m_sb, &c->m_xs, &c->cb_work, &c->Rw, &c->a_linv, &c->a_m1, &c->a_m2, &c->a_m3,
                    &c->a_m4, &c->a_cp, &c->a_y, &c->a_gd, &c->a_e, &c->a_z1, &c->a_z2, &c->a_z3, &c->a_gpm, &c->a_gpp,
                    &c->a_m5, &c->a_m6, &c->bW1, &c->bT, &c->bU, &c->bQ,
                    &c->b_s1, &c->b_s2, &c->b_s3, &c->b_work, &c->b_cb, &c->b_dtmp, &c->b_cbd, &c->ctab,
                    &c->m_pairs_t, &c->swf, &c->ew, &c->Xgd, &c->m_sd, &c->ns_bound, &c->ns_alpha, &c->ns_work,
                    &c->b_s4, &c->kappa_work, &c->inv_work, &c->m_ths, &c->cb_split, &c->b_split, &c->ref};
  for (DevBuf* b : bufs) release(*b);
  for (DevBuf& b : c->cx) release(b);
  for (auto& pe : c->prof_ev) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->d_idx) cudaFree(c->d_idx);  // d_perm and d_perm2 point into this allocation
  if (c->d_used) cudaFree(c->d_used);
  if (c->d_part_idx) cudaFree(c->d_part_idx);
  if (c->d_tables) cudaFree(c->d_tables);
  if (c->d_status) cudaFree(c->d_status);  // d_bar and d_ints point into this allocation
  delete c;
  return ISDF_OK;
}

static cudaError_t ensure_ints(int*& p, size_t& cap, size_t n) {
  if (n <= cap) return cudaSuccess;
  if (isdf::tl_capture) return cudaErrorStreamCaptureUnsupported;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = isdf::dev_malloc(&p, std::max<size_t>(n, 1) * sizeof(int));
  if (e == cudaSuccess) cap = n;
  return e;
}

// Cholesky of the n x n matrix W (ld = ldw) into the column-major factor
// Lout (ld = n); pivoted or not; rank -> c->d_ints[0], pivots -> c->d_perm.
static int cholesky(isdf_ctx* c, const double* W, long long ldw, int n, int pivot, double tol_rel,
                    double* Lout, int* d_perm) {
  CK(ensure(c->Lr, (size_t)n * n));
  CK(ensure(c->chol_d, (size_t)n));
  CK(ensure(c->chol_part, (size_t)2 * kMaxGrid));
  size_t cap_used = c->cap_used;
  CK(ensure_ints(c->d_used, cap_used, (size_t)n));
  c->cap_used = cap_used;
  if (!c->d_part_idx) CK(isdf::dev_malloc(&c->d_part_idx, 2 * kMaxGrid * sizeof(int)));
  CholWork w{c->chol_d.p, c->chol_part.p, c->d_part_idx, c->d_used, c->d_bar, kMaxGrid};
  CK(cudaMemsetAsync(c->d_ints, 0, sizeof(int), c->stream));
  CK(launch_cholesky(W, ldw, n, pivot, tol_rel, c->Lr.p, d_perm, c->d_ints, c->d_status, w,
                     std::min(c->num_sms, kMaxGrid), kWaitLimitNs, c->stream));
  CK(launch_factor_to_colmajor(c->Lr.p, n, d_perm, c->d_ints, Lout, n, n, c->stream));
  return ISDF_OK;
}

// Blocked Cholesky (no pivoting) of W into Lout (ld n); *fail (device) = -1
// on success, else the first column whose pivot fell to tol_rel * max diag.
// The mixed path's trailing updates run in double-float arithmetic from
// the split panel in cb_split (sized by the caller's workspace step).
static float2* split_panel(isdf_ctx* c, size_t need) {
  return c->prec == ISDF_PREC_MIXED && c->cb_split.cap >= need ? reinterpret_cast<float2*>(c->cb_split.p) : nullptr;
}

static int cholesky_blocked(isdf_ctx* c, const double* W, long long ldw, int n, double tol_rel, double* Lout,
                            int* fail, cudaStream_t st) {
  CK(launch_cholesky_blocked(W, ldw, n, tol_rel, Lout, n, c->cb_work.p, fail, st, split_panel(c, (size_t)64 * n)));
  return ISDF_OK;
}

// The main stream hands work to the second stream ...
static int fork_s2(isdf_ctx* c) {
  CK(cudaEventRecord(c->ev_fork, c->stream));
  CK(cudaStreamWaitEvent(c->s2, c->ev_fork, 0));
  return ISDF_OK;
}
// ... and everything queued on the main stream after this waits for it.
static int join_s2(isdf_ctx* c) {
  CK(cudaEventRecord(c->ev_join, c->s2));
  CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  return ISDF_OK;
}

// Workspace of launch_cholesky_and_inverse for an n x n factor: its step
// events and the Y / split-K buffer (sized before any fork: a resize frees).
static int chol_inverse_workspace(isdf_ctx* c, int n, bool ahead = false) {
  const size_t steps = (size_t)(n + 63) / 64 * 3;  // per step: block, panel, rest (look-ahead)
  while (c->ev_chol.size() < steps) {
    if (isdf::tl_capture) return fail(c, ISDF_ERR_STATE, "factorisation events: a captured call needs an eager call first");
    cudaEvent_t e = nullptr;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->ev_chol.push_back(e);
  }
  const size_t split = (size_t)(ahead ? 128 : 64) * n;  // two alternating split panels with look-ahead
  if (c->inv_work.cap < (size_t)9 * 64 * n || c->cb_split.cap < split) SYNC(c->stream);
  CK(ensure(c->inv_work, (size_t)9 * 64 * n));
  CK(ensure(c->cb_split, split));
  return ISDF_OK;
}

// The fit after the factorisation of C C^T: theta for the leading r pivots
// (d_perm on the device, the factor in c->Lc with ld n_mu); gram_done: the
// Gram beside the factorisation used these points in this order.
static int fit_tail(isdf_ctx* c, const double* phi, double* theta, int n_v, int n_c, int n_mu, int r, bool gram_done,
                    bool fuse_inv, int prec) {
  const int n_e = n_v + n_c;
  // Lc was written with ld = n_mu; repack the leading rank x rank block with ld = rank
  if (r > 0) {
    CK(ensure(c->Bf, (size_t)r * r));
    CK(cudaMemcpy2DAsync(c->Bf.p, r * sizeof(double), c->Lc.p, n_mu * sizeof(double), r * sizeof(double),
                         r, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->Lc.p, c->Bf.p, (size_t)r * r * sizeof(double), cudaMemcpyDeviceToDevice,
                       c->stream));
    // orbitals at the pivot points, in pivot order
    CK(ensure(c->phimu_p, (size_t)r * n_e));
    CK(launch_gather_rows(c->phimu.p, n_mu, c->d_perm, r, n_e, c->phimu_p.p, r, c->stream));
    if (prec == ISDF_PREC_MIXED) {
      if (!gram_done) CK(isdf::mixed_fit_gram(c, phi, c->phimu_p.p, n_v, n_c, r));
      // the inverse built beside the factorisation holds for the unpivoted full-rank factor
      CK(isdf::mixed_fit_solve(c, theta, r, fuse_inv && gram_done));
      // ||L||_F^2 = tr(C C^T) and ||L^-1||_F^2 = tr((C C^T)^-1), read by build_polarizability
      CK(ensure(c->kappa_work, 2 + 256));
      CK(launch_sumsq(c->Lc.p, (long long)r * r, c->kappa_work.p + 2, c->kappa_work.p, c->stream));
      CK(launch_sumsq(c->m_linv.p, (long long)r * r, c->kappa_work.p + 2, c->kappa_work.p + 1, c->stream));
    } else {
      // M C_r^T by the Hadamard identity, then theta = (M C_r^T) L_r^-T in place
      if (!gram_done) {
        PhaseScope ph(c, ISDF_PH_FIT_GRAM);
        CK(launch_facesplit_gram(phi, c->n_r, (int)c->n_r, c->phimu_p.p, r, r, n_v, n_e, theta, c->n_r,
                                 c->stream));
      }
      PhaseScope ph(c, ISDF_PH_FIT_TRSM);
      CK(launch_trsm_prep(c->Lc.p, r, r, c->Bf.p, r, c->stream));
      CK(launch_trsm_right_lt(theta, c->n_r, (int)c->n_r, c->Bf.p, r, r, c->stream));
    }
  }
  if (r < n_mu)
    CK(cudaMemsetAsync(theta + c->n_r * r, 0, (size_t)c->n_r * (n_mu - r) * sizeof(double), c->stream));
  return ISDF_OK;
}

extern "C" int isdf_fit(isdf_ctx* c, const double* phi, int n_v, int n_c, const int64_t* mu_idx,
                        int n_mu, int prec, double* theta, int* rank_out) {
  if (!c) return ISDF_ERR_ARG;
  c->err.clear();
  c->fitted = false;
  c->polar_ready = false;
  if (!phi || !theta || !mu_idx) return fail(c, ISDF_ERR_ARG, "isdf_fit: null pointer argument");
  const int mode = prec;
  if (prec == ISDF_PREC_MIXED_PAIRS) prec = ISDF_PREC_MIXED;
  if (prec != ISDF_PREC_FP64 && prec != ISDF_PREC_MIXED)
    return fail(c, ISDF_ERR_ARG, "isdf_fit: unknown precision mode");
  if (n_v < 1 || n_c < 1) return fail(c, ISDF_ERR_SHAPE, "isdf_fit: n_v and n_c must be >= 1");
  if (n_mu < 1 || (long long)n_mu > c->n_r)
    return fail(c, ISDF_ERR_SHAPE, "isdf_fit: n_mu must be in [1, N_r]");
  if ((long long)n_v * n_c > (1ll << 31) - 1 || n_mu > 65536)
    return fail(c, ISDF_ERR_SHAPE, "isdf_fit: problem too large");
  const double* tend = theta + c->n_r * n_mu;
  const double* pend = phi + c->n_r * (long long)(n_v + n_c);
  if (theta < pend && phi < tend) return fail(c, ISDF_ERR_ARG, "isdf_fit: theta overlaps phi");
  // the points may sit in host or in device memory; the checks and the pivot
  // bookkeeping below are host work, so a device array is copied over first
  // (the fit synchronises the stream once anyway)
  std::vector<int64_t> mu_host;
  {
    cudaPointerAttributes at{};
    const cudaError_t pe = cudaPointerGetAttributes(&at, mu_idx);
    if (pe != cudaSuccess) cudaGetLastError();  // an unknown host pointer on an old runtime: host memory
    if (pe == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
      if (isdf::tl_capture)
        return fail(c, ISDF_ERR_STATE, "isdf_fit: a captured fit takes its points from host memory");
      mu_host.resize(n_mu);
      CK(cudaStreamSynchronize(c->stream));  // the caller may have written the points on this stream
      CK(cudaMemcpy(mu_host.data(), mu_idx, (size_t)n_mu * sizeof(int64_t), cudaMemcpyDefault));
      mu_idx = mu_host.data();
    }
  }
  std::vector<int64_t> sorted(mu_idx, mu_idx + n_mu);
  std::sort(sorted.begin(), sorted.end());
  if (sorted.front() < 0 || sorted.back() >= c->n_r)
    return fail(c, ISDF_ERR_INDEX, "isdf_fit: interpolation index out of range");
  for (int i = 1; i < n_mu; ++i)
    if (sorted[i] == sorted[i - 1]) return fail(c, ISDF_ERR_INDEX, "isdf_fit: repeated interpolation index");
  const int n_e = n_v + n_c;
  std::vector<int> idx32(mu_idx, mu_idx + n_mu);
  if (isdf::tl_capture) {
    // a graph replays the eager fit before it: same points, same precision,
    // unpivoted at full rank (the point indices are already on the device)
    if (!c->fit_full || c->fit_idx != idx32 || c->fit_mode != mode || c->n_v != n_v || c->n_c != n_c)
      return fail(c, ISDF_ERR_STATE, "isdf_fit: a captured fit needs an eager full-rank fit of the same points first");
  }
  SYNC(c->stream);  // earlier work may still read workspace that is resized below
  CK(ensure_ints(c->d_idx, c->cap_idx, (size_t)3 * n_mu));
  c->d_perm = c->d_idx + n_mu;
  c->d_perm2 = c->d_idx + 2 * n_mu;
  if (!isdf::tl_capture)
    CK(cudaMemcpyAsync(c->d_idx, idx32.data(), n_mu * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  // mixed path: the identity order, for the rest of the fit that is queued
  // before the factorisation's flags are read (below)
  const bool tail_ahead = prec == ISDF_PREC_MIXED && !isdf::tl_capture;
  if (tail_ahead) {
    std::vector<int> ident(n_mu);
    for (int i = 0; i < n_mu; ++i) ident[i] = i;
    CK(cudaMemcpyAsync(c->d_perm, ident.data(), n_mu * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  }
  CK(cudaMemsetAsync(c->d_status, 0, 8 * sizeof(unsigned), c->stream));
  CK(launch_check_finite(phi, c->n_r * n_e, c->d_status, c->stream));
  // orbitals at the points, C C^T (face-split Gram of the point block), its pivoted Cholesky
  CK(ensure(c->phimu, (size_t)n_mu * n_e));
  CK(ensure(c->A, (size_t)n_mu * n_mu));
  CK(ensure(c->Lc, (size_t)n_mu * n_mu));
  const double tol = (double)n_mu * 2.220446049250313e-16;
  int rc0 = ISDF_OK;
  CK(ensure(c->cb_work, 1));
  {
    PhaseScope ph(c, ISDF_PH_POINTS);
    CK(launch_gather_rows(phi, c->n_r, c->d_idx, n_mu, n_e, c->phimu.p, n_mu, c->stream));
    // the mixed path sums in double-float on the FP32 pipe (about 2^-47)
    isdf::DfGemm df(prec == ISDF_PREC_MIXED);
    CK(launch_facesplit_gram(c->phimu.p, n_mu, n_mu, c->phimu.p, n_mu, n_mu, n_v, n_e, c->A.p, n_mu,
                             c->stream));
  }
  // Cholesky of C C^T in the given point order (blocked, on the second
  // stream: it is a latency-bound FP64 chain); if a pivot falls to the rank
  // threshold it is redone below with diagonal pivoting (rank-deficient C)
  // mixed path: L^-1 (for the whitened basis) is built on a third stream
  // beside the factorisation, block row by block row
  const bool fuse_inv = prec == ISDF_PREC_MIXED;
  if (fuse_inv) {
    rc0 = chol_inverse_workspace(c, n_mu, true);
    if (rc0 != ISDF_OK) return rc0;
    CK(ensure(c->m_linv, (size_t)n_mu * n_mu));
  }
  rc0 = fork_s2(c);
  if (rc0 != ISDF_OK) return rc0;
  if (fuse_inv) CK(cudaStreamWaitEvent(c->s3, c->ev_fork, 0));
  {
    PhaseScope ph(c, ISDF_PH_POINTS, c->s2);
    if (fuse_inv) {
      CK(launch_cholesky_and_inverse(c->A.p, n_mu, n_mu, tol, c->Lc.p, n_mu, c->m_linv.p, n_mu, c->cb_work.p,
                                     c->d_ints + 1, c->inv_work.p, c->s2, c->s3, c->ev_chol.data(),
                                     reinterpret_cast<float2*>(c->cb_split.p), c->s4));
    } else {
      rc0 = cholesky_blocked(c, c->A.p, n_mu, n_mu, tol, c->Lc.p, c->d_ints + 1, c->s2);
      if (rc0 != ISDF_OK) return rc0;
    }
  }
  // meanwhile, speculatively, the face-split Gram M C^T with the points in
  // the given order, which is the pivot order whenever the blocked
  // factorisation succeeds
  if (prec == ISDF_PREC_MIXED) {
    // the Cholesky on the second stream keeps some SMs (the Gram: 6 slice products, 2 N_r n_mu N_e each)
    isdf::TcSmReserve keep(fp64_sms_to_leave(n_mu, 12.0 * c->n_r * n_mu * (n_v + n_c)));
    CK(isdf::mixed_fit_gram(c, phi, c->phimu.p, n_v, n_c, n_mu));
  } else {
    PhaseScope ph(c, ISDF_PH_FIT_GRAM);
    CK(launch_facesplit_gram(phi, c->n_r, (int)c->n_r, c->phimu.p, n_mu, n_mu, n_v, n_e, theta, c->n_r,
                             c->stream));
  }
  rc0 = join_s2(c);
  if (rc0 != ISDF_OK) return rc0;
  if (fuse_inv) {
    CK(cudaEventRecord(c->ev_join3, c->s3));
    CK(cudaStreamWaitEvent(c->stream, c->ev_join3, 0));
  }
  int rc;
  int fail = -1, rank = 0;
  bool tail_queued = false;
  if (tail_ahead) {
    // mixed path: the rest of the fit is queued for the outcome the Gram
    // beside the factorisation already assumed (no failed pivot: full rank,
    // the given order), and the host reads the flags through the helper
    // stream while it runs; after a failed pivot the pivoted route below
    // redoes that work on the same stream
    CK(cudaEventRecord(c->ev_fork, c->stream));
    rc = fit_tail(c, phi, theta, n_v, n_c, n_mu, n_mu, true, fuse_inv, prec);
    if (rc != ISDF_OK) return rc;
    CK(cudaStreamWaitEvent(c->s3, c->ev_fork, 0));
    unsigned hs[32];  // the status word [0] and the flags d_ints = d_status + 16
    CK(cudaMemcpyAsync(hs, c->d_status, sizeof(hs), cudaMemcpyDeviceToHost, c->s3));
    CK(cudaStreamSynchronize(c->s3));
    rc = status_error(c, hs[0], "isdf_fit");
    if (rc != ISDF_OK) return rc;
    std::memcpy(&fail, hs + 17, sizeof(int));  // d_ints[1]
    tail_queued = fail < 0;
  } else if (!isdf::tl_capture) {  // captured: the flags are read after the replay (graph_check)
    CK(cudaStreamSynchronize(c->stream));
    rc = check_status(c, "isdf_fit");
    if (rc != ISDF_OK) return rc;
    CK(cudaMemcpy(&fail, c->d_ints + 1, sizeof(int), cudaMemcpyDeviceToHost));
  }
  c->perm.assign(n_mu, 0);
  const bool gram_done = fail < 0;
  if (fail < 0) {
    rank = n_mu;
    for (int i = 0; i < n_mu; ++i) c->perm[i] = i;
    if (!isdf::tl_capture && !tail_queued)  // captured: the identity order of the eager fit is on the device
      CK(cudaMemcpyAsync(c->d_perm, c->perm.data(), n_mu * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  } else {
    {
      PhaseScope ph(c, ISDF_PH_POINTS);
      rc0 = cholesky(c, c->A.p, n_mu, n_mu, 1, tol, c->Lc.p, c->d_perm);
      if (rc0 != ISDF_OK) return rc0;
    }
    CK(cudaStreamSynchronize(c->stream));
    rc = check_status(c, "isdf_fit");
    if (rc != ISDF_OK) return rc;
    CK(cudaMemcpy(&rank, c->d_ints, sizeof(int), cudaMemcpyDeviceToHost));
    if (rank > 0) CK(cudaMemcpy(c->perm.data(), c->d_perm, rank * sizeof(int), cudaMemcpyDeviceToHost));
  }
  {  // complete the pivot list with the unused points in increasing order
    std::vector<char> used(n_mu, 0);
    for (int j = 0; j < rank; ++j) used[c->perm[j]] = 1;
    int j = rank;
    for (int i = 0; i < n_mu; ++i)
      if (!used[i]) c->perm[j++] = i;
  }
  const int r = rank;
  if (!tail_queued) {
    int rc1 = fit_tail(c, phi, theta, n_v, n_c, n_mu, r, gram_done, fuse_inv, prec);
    if (rc1 != ISDF_OK) return rc1;
  }
  c->phi = phi;
  c->theta = theta;
  c->prec = prec;
  c->pair_mode = mode;
  c->pair_whiten = mode == ISDF_PREC_MIXED_PAIRS;
  c->n_v = n_v;
  c->n_c = n_c;
  c->n_mu = n_mu;
  c->rank = r;
  c->fitted = true;  // captured: graph_check clears it if the replay's factorisation failed
  if (!isdf::tl_capture) {
    c->fit_idx = idx32;
    c->fit_mode = mode;
    c->fit_full = gram_done;
  }
  if (rank_out) *rank_out = r;
  return ISDF_OK;
}

extern "C" int isdf_fit_factor(isdf_ctx* c, int* piv_out, double* L_out) {
  if (!c) return ISDF_ERR_ARG;
  if (!c->fitted) return fail(c, ISDF_ERR_STATE, "isdf_fit_factor: no fit");
  if (piv_out) std::memcpy(piv_out, c->perm.data(), c->n_mu * sizeof(int));
  if (L_out) {
    const int r = c->rank, m = c->n_mu;
    CK(cudaMemsetAsync(L_out, 0, (size_t)m * m * sizeof(double), c->stream));
    if (r > 0)
      CK(cudaMemcpy2DAsync(L_out, m * sizeof(double), c->Lc.p, r * sizeof(double), r * sizeof(double), r,
                           cudaMemcpyDeviceToDevice, c->stream));
  }
  return ISDF_OK;
}

// copy a dense r x r matrix (ld r) into an m x m output with zero padding
static int copy_padded(isdf_ctx* c, double* dst, const double* src, int r, int m) {
  CK(cudaMemsetAsync(dst, 0, (size_t)m * m * sizeof(double), c->stream));
  if (r > 0)
    CK(cudaMemcpy2DAsync(dst, m * sizeof(double), src, r * sizeof(double), r * sizeof(double), r,
                         cudaMemcpyDeviceToDevice, c->stream));
  return ISDF_OK;
}

static int split_for(long long tiles, long long K, int num_sms) {
  long long want = (2ll * num_sms + tiles - 1) / tiles;
  long long maxs = std::max(1ll, K / 1024);
  return (int)std::max(1ll, std::min(want, std::min(maxs, 64ll)));
}

// D(w) for every frequency and G; with n_nodes > 0 the static D by the
// contour integral of Algorithm 2 instead of the pair sum.
static int polar_impl(isdf_ctx* c, const double* energies, const double* omega, int n_omega, double* D_out,
                      double* G_out, int n_nodes) {
  if (!c) return ISDF_ERR_ARG;
  c->err.clear();
  if (!c->fitted) return fail(c, ISDF_ERR_STATE, "build_polarizability: call isdf_fit first");
  if (!energies || !omega) return fail(c, ISDF_ERR_ARG, "build_polarizability: null pointer argument");
  if (n_omega < 1 || n_omega > 4096) return fail(c, ISDF_ERR_SHAPE, "build_polarizability: n_omega in [1, 4096]");
  const int n_v = c->n_v, n_c = c->n_c, n_e = n_v + n_c, r = c->rank, m = c->n_mu;
  for (int i = 0; i < n_e; ++i)
    if (!std::isfinite(energies[i])) return fail(c, ISDF_ERR_NONFINITE, "build_polarizability: energy not finite");
  double emax_v = energies[0], emin_c = energies[n_v];
  for (int i = 0; i < n_v; ++i) emax_v = std::max(emax_v, energies[i]);
  for (int j = n_v; j < n_e; ++j) emin_c = std::min(emin_c, energies[j]);
  if (!(emax_v < emin_c)) return fail(c, ISDF_ERR_ORDER, "build_polarizability: occupied energies must lie below unoccupied ones");
  for (int k = 0; k < n_omega; ++k)
    if (!std::isfinite(omega[k]) || omega[k] < 0.0)
      return fail(c, ISDF_ERR_ARG, "build_polarizability: frequencies must be finite and >= 0");
  c->polar_ready = false;
  const size_t rr = (size_t)r * r;
  const bool cap = isdf::tl_capture;
  if (cap) {
    // a graph replays the eager call before it: the pair weights and the
    // contour tables it uploaded stay on the device, so they must not change
    if (c->n_omega != n_omega || c->omega != std::vector<double>(omega, omega + n_omega) ||
        c->energies != std::vector<double>(energies, energies + n_e) || c->polar_nodes != n_nodes)
      return fail(c, ISDF_ERR_STATE,
                  "build_polarizability: a captured call needs an eager call with the same energies and frequencies first");
    c->pair_whiten = c->polar_whiten;
  }
  SYNC(c->stream);
  if (!cap && c->prec == ISDF_PREC_MIXED && c->pair_mode == ISDF_PREC_MIXED && r > 0) {
    // mean(lambda) mean(1 / lambda) of C C^T: 1 when perfectly conditioned, at
    // most (1 + cond)^2 / (4 cond) (Kantorovich), so a large value flags a
    // large cond(C C^T)
    double fro[2] = {0.0, 0.0};
    CK(cudaMemcpy(fro, c->kappa_work.p, 2 * sizeof(double), cudaMemcpyDeviceToHost));
    c->pair_whiten = (fro[0] / r) * (fro[1] / r) > kPairWhitenMean;
  }
  CK(ensure(c->G, std::max<size_t>(rr, 1)));
  CK(ensure(c->D, std::max<size_t>(rr * n_omega, 1)));
  CK(ensure(c->K, std::max<size_t>(rr * n_omega, 1)));
  CK(ensure(c->Rw, std::max<size_t>(rr * n_omega, 1)));
  CK(ensure(c->cb_work, 1));
  if (c->cap_fail < (size_t)n_omega) {
    if (c->d_fail) cudaFree(c->d_fail);
    c->d_fail = nullptr;
    c->cap_fail = 0;
    CK(isdf::dev_malloc(&c->d_fail, n_omega * sizeof(int)));
    c->cap_fail = n_omega;
  }
  c->xgd_ready = false;
  if (r > 0) {
    // G = theta^T V theta = S^T S with S the weighted half spectrum (Parseval)
    const long long lds = 2 * c->n_half;
    const size_t npair = (size_t)n_v * n_c;
    long long tiles = (long long)((r + 63) / 64) * ((r + 63) / 64 + 1) / 2;
    int sp = split_for(tiles, lds, c->num_sms);
    int spd = split_for(tiles, (long long)npair, c->num_sms);
    // size all workspace before the first launch (a resize frees memory)
    SYNC(c->stream);
    CK(ensure(c->spec, (size_t)lds * r));
    CK(ensure(c->partial, (size_t)std::max(sp, spd) * rr));
    CK(ensure(c->sw, npair * n_omega));
    CK(ensure(c->tmp1, rr));
    if (n_omega > 1) CK(ensure(c->b_cbd, (size_t)n_omega));
    if (c->prec == ISDF_PREC_MIXED) CK(ensure(c->cb_split, (size_t)64 * r * n_omega));
    if (n_nodes > 0) CK(ensure(c->ctab, (size_t)2 * n_nodes * (n_e + 1)));
    if (c->prec == ISDF_PREC_MIXED) CK(ensure(c->swf, (npair * n_omega + 1) / 2));  // the weights in FP32
    CK(ensure(c->ew, (size_t)n_e + n_omega));
    // sqrt(-2 Omega(iw)^-1) for every pair and frequency, on the device from
    // the energies and frequencies (one small upload; a captured call reuses
    // the eager call's, which are the same)
    if (!cap) {
      c->ew_host.assign(energies, energies + n_e);
      c->ew_host.insert(c->ew_host.end(), omega, omega + n_omega);
      CK(cudaMemcpyAsync(c->ew.p, c->ew_host.data(), c->ew_host.size() * sizeof(double), cudaMemcpyHostToDevice,
                         c->stream));
    }
    CK(launch_pair_weights(c->ew.p, n_v, n_c, n_omega, c->sw.p,
                           c->prec == ISDF_PREC_MIXED ? reinterpret_cast<float*>(c->swf.p) : nullptr,
                           c->stream));
    // D(w) for every frequency (main stream)
    if (n_nodes > 0) {
      // static D by the contour integral: resolvent weights of every node
      std::vector<double> wt, wn;
      CK(contour_tables(energies, n_v, n_c, n_nodes, wt, wn));
      if (!cap) {
        CK(cudaMemcpyAsync(c->ctab.p, wt.data(), wt.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->ctab.p + wt.size(), wn.data(), wn.size() * sizeof(double), cudaMemcpyHostToDevice,
                           c->stream));
      }
      double* Dpp = c->prec == ISDF_PREC_MIXED ? c->tmp1.p : c->D.p;
      {
        PhaseScope ph(c, ISDF_PH_POLAR_D);
        CK(launch_contour_polarizability(c->phimu_p.p, r, r, n_v, n_c, c->ctab.p, c->ctab.p + wt.size(), n_nodes, Dpp,
                                         r, c->partial.p, c->partial.cap, c->num_sms, c->stream));
      }
      if (c->prec == ISDF_PREC_MIXED) {
        CK(isdf::mixed_whiten_D(c, Dpp, c->D.p));
      } else {
        PhaseScope ph(c, ISDF_PH_WHITEN_D);
        CK(launch_trsm_right_lt(c->D.p, r, r, c->Bf.p, r, r, c->stream));
        CK(launch_transpose(c->D.p, r, r, r, c->tmp1.p, r, c->stream));
        CK(launch_trsm_right_lt(c->tmp1.p, r, r, c->Bf.p, r, r, c->stream));
        CK(launch_symmetrize(c->tmp1.p, r, r, c->stream));
        CK(cudaMemcpyAsync(c->D.p, c->tmp1.p, rr * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      }
    } else if (c->prec == ISDF_PREC_MIXED && c->pair_whiten) {
      CK(isdf::mixed_polar_D_pairspace(c, reinterpret_cast<const float*>(c->swf.p), n_omega));
    } else if (c->prec == ISDF_PREC_MIXED) {
      if (n_omega > 1) {
        CK(isdf::mixed_polar_D_batched(c, reinterpret_cast<const float*>(c->swf.p), n_omega));
      } else {
        CK(isdf::mixed_polar_D(c, reinterpret_cast<const float*>(c->swf.p), n_omega));
      }
    } else {
      for (int k = 0; k < n_omega; ++k) {
        double* Dk = c->D.p + rr * k;
        {
          PhaseScope ph(c, ISDF_PH_POLAR_D);
          CK(launch_polarizability(c->phimu_p.p, r, r, n_v, n_c, c->sw.p + npair * k, Dk, r, spd, c->partial.p,
                                   c->stream));
        }
        PhaseScope ph(c, ISDF_PH_WHITEN_D);
        CK(launch_trsm_right_lt(Dk, r, r, c->Bf.p, r, r, c->stream));
        CK(launch_transpose(Dk, r, r, r, c->tmp1.p, r, c->stream));
        CK(launch_trsm_right_lt(c->tmp1.p, r, r, c->Bf.p, r, r, c->stream));
        CK(launch_symmetrize(c->tmp1.p, r, r, c->stream));
        CK(cudaMemcpyAsync(Dk, c->tmp1.p, rr * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      }
    }
    // D(w) = R R^T on the second stream, beside the Coulomb work below
    {
      int rc0 = fork_s2(c);
      if (rc0 != ISDF_OK) return rc0;
      PhaseScope ph(c, ISDF_PH_SMW, c->s2);
      if (c->prec == ISDF_PREC_MIXED) {
        // the capacitance K = -D (I + G D)^-1 comes from Newton-Schulz
        // products (smw_inverse, smw_inverse_all), which factor D only when
        // the spectral bounds do not allow that
        CK(cudaMemsetAsync(c->d_fail, 0xff, n_omega * sizeof(int), c->s2));
      } else if (n_omega > 1) {  // all frequencies in one factorisation sequence
        CK(launch_cholesky_blocked_batched(c->D.p, r, (long long)rr, r, n_omega, 0.0, c->Rw.p, r, (long long)rr,
                                           c->b_cbd.p, c->d_fail, c->s2, split_panel(c, (size_t)64 * r * n_omega)));
      } else {
        rc0 = cholesky_blocked(c, c->D.p, r, r, 0.0, c->Rw.p, c->d_fail, c->s2);
        if (rc0 != ISDF_OK) return rc0;
      }
    }
    // G = theta^T V theta (main stream)
    if (c->prec == ISDF_PREC_MIXED) {
      // nothing runs beside it on the second stream: all SMs
      CK(isdf::mixed_polar_G(c));
    } else {
      {
        PhaseScope ph(c, ISDF_PH_FFT);
        CK(launch_fft_forward(c->fft, c->theta, c->n_r, r, c->spec.p, lds, c->d_wsyrk, c->smem_xy, c->smem_z,
                              c->stream));
      }
      PhaseScope ph(c, ISDF_PH_SYRK_G);
      CK(launch_gemm(c->spec.p, lds, true, c->spec.p, lds, true, r, r, (int)lds, 1.0, 0.0, c->G.p, r, true, sp,
                     c->partial.p, false, c->stream));
    }
    {
      int rc0 = join_s2(c);
      if (rc0 != ISDF_OK) return rc0;
    }
  }
  if (G_out) {
    int rc = copy_padded(c, G_out, c->G.p, r, m);
    if (rc != ISDF_OK) return rc;
  }
  if (D_out) {
    for (int k = 0; k < n_omega; ++k) {
      int rc = copy_padded(c, D_out + (size_t)m * m * k, c->D.p + rr * k, r, m);
      if (rc != ISDF_OK) return rc;
    }
  }
  c->n_omega = n_omega;
  c->omega.assign(omega, omega + n_omega);
  c->energies.assign(energies, energies + n_e);
  c->k_ready.assign(n_omega, 0);
  c->polar_ready = true;
  // D(w) factored by the FP64 path; the mixed path factors on demand (smw_enqueue)
  c->rw_ready = c->prec != ISDF_PREC_MIXED;
  c->polar_whiten = c->pair_whiten;
  c->polar_nodes = n_nodes;
  return ISDF_OK;
}

extern "C" int build_polarizability(isdf_ctx* c, const double* energies, const double* omega, int n_omega,
                                    double* D_out, double* G_out) {
  return polar_impl(c, energies, omega, n_omega, D_out, G_out, 0);
}

extern "C" int build_polarizability_contour(isdf_ctx* c, const double* energies, int n_nodes, double* D_out,
                                            double* G_out) {
  if (!c) return ISDF_ERR_ARG;
  if (n_nodes < 1 || n_nodes > 1024) return fail(c, ISDF_ERR_ARG, "build_polarizability_contour: n_nodes in [1, 1024]");
  const double w0 = 0.0;
  return polar_impl(c, energies, &w0, 1, D_out, G_out, n_nodes);
}

extern "C" int isdf_pair_weight_bounds(const double* energies, int n_v, int n_c, double w, double* wmin,
                                       double* wmax) {
  if (!energies || !wmin || !wmax || n_v < 1 || n_c < 1 || !std::isfinite(w) || w < 0.0) return ISDF_ERR_ARG;
  double emax_v = energies[0], emin_c = energies[n_v];
  for (int i = 0; i < n_v + n_c; ++i)
    if (!std::isfinite(energies[i])) return ISDF_ERR_NONFINITE;
  for (int i = 0; i < n_v; ++i) emax_v = std::max(emax_v, energies[i]);
  for (int j = n_v; j < n_v + n_c; ++j) emin_c = std::min(emin_c, energies[j]);
  if (!(emax_v < emin_c)) return ISDF_ERR_ORDER;
  isdf::pair_weight_bounds(energies, n_v, n_c, w, wmin, wmax);
  return ISDF_OK;
}

extern "C" int isdf_ns_schedule(double kappa, int max_steps, double* beta, int* slices) {
  if (!(kappa >= 1.0) || !std::isfinite(kappa) || max_steps < 1 || !beta || !slices) return ISDF_ERR_ARG;
  isdf::NsPlan plan;
  if (!isdf::ns_plan((kappa - 1.0) / (kappa + 1.0), plan)) return 0;
  if (plan.steps() > max_steps) return ISDF_ERR_ARG;
  for (int k = 0; k < plan.steps(); ++k) {
    beta[k] = plan.beta[k];
    slices[k] = plan.s[k];
  }
  return plan.steps();
}

extern "C" int isdf_contour_nodes(const double* energies, int n_v, int n_c, double tol) {
  if (!energies || n_v < 1 || n_c < 1 || !(tol > 0.0) || !(tol < 1.0)) return ISDF_ERR_ARG;
  double e_n = energies[0], e_lo = energies[n_v], e_hi = energies[n_v];
  for (int i = 0; i < n_v; ++i) e_n = std::max(e_n, energies[i]);
  for (int i = n_v; i < n_v + n_c; ++i) {
    e_lo = std::min(e_lo, energies[i]);
    e_hi = std::max(e_hi, energies[i]);
  }
  if (!(e_lo > e_n)) return ISDF_ERR_ORDER;
  return std::max(1, contour_nodes_recommended(e_lo - e_n, e_hi - e_n, tol));
}

// Queue the SMW capacitance of frequency k (no synchronisation); the
// failure flag of the factorisation of I + R^T G R goes to failT.
static int smw_enqueue(isdf_ctx* c, int k, int* failT) {
  const int r = c->rank;
  const size_t rr = (size_t)r * r;
  double* Kk = c->K.p + rr * k;
  long long tiles = (long long)((r + 63) / 64) * ((r + 63) / 64 + 1) / 2;
  int sp = split_for(tiles, std::max(r, 1), c->num_sms);
  PhaseScope ph(c, ISDF_PH_SMW);
  if (c->prec == ISDF_PREC_MIXED && !isdf::tl_capture) {
    // K = -D (I + G D)^-1 by Newton-Schulz on the tensor cores when the
    // spectral bounds allow a few steps (rigorous bounds only, one host
    // read): I + G D has real eigenvalues in [1, 1 + |G| |D|], with |G| the
    // Gershgorin bound of G and |D| the smaller of its Gershgorin bound and
    // the largest pair weight
    const double* Dk = c->D.p + rr * k;
    double* nb = c->ns_bound.p;
    CK(launch_row_abs_sum_max(c->G.p, r, r, nb, nb + 4, c->stream));
    CK(launch_row_abs_sum_max(Dk, r, r, nb + 1, nb + 4, c->stream));
    // the host reads the bounds through the helper stream while M = I + G D,
    // which needs none, is built on this one (if the bounds then rule the
    // iteration out, the factorisation below overwrites M)
    CK(cudaEventRecord(c->ev_fork, c->stream));
    CK(isdf::mixed_ns_prepare(c, Dk));
    CK(cudaStreamWaitEvent(c->s3, c->ev_fork, 0));
    double h[2] = {0.0, 0.0};
    CK(cudaMemcpyAsync(h, nb, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->s3));
    CK(cudaStreamSynchronize(c->s3));
    double wmin = 0.0, wmax = 0.0;
    isdf::pair_weight_bounds(c->energies.data(), c->n_v, c->n_c, c->omega[k], &wmin, &wmax);
    const double kappa = isdf::ns_kappa(h[0], std::min(wmax, h[1]));
    isdf::NsPlan plan;
    if (std::isfinite(kappa) && isdf::ns_plan((kappa - 1.0) / (kappa + 1.0), plan)) {
      CK(cudaMemsetAsync(failT, 0xff, sizeof(int), c->stream));  // no factorisation to fail
      CK(isdf::mixed_ns_iterate(c, Dk, Kk, 2.0 / (1.0 + kappa), plan));
      c->xgd_ready = c->n_omega == 1;
      return ISDF_OK;
    }
  }
  c->xgd_ready = false;
  // D = R R^T: factored by build_polarizability on the second stream (FP64
  // path), or here (the mixed path leaves D(w) unfactored for its
  // Newton-Schulz route)
  if (!c->rw_ready) {
    int rc = cholesky_blocked(c, c->D.p + rr * k, r, r, 0.0, c->Rw.p + rr * k, c->d_fail + k, c->stream);
    if (rc != ISDF_OK) return rc;
  }
  CK(cudaMemcpyAsync(c->R.p, c->Rw.p + rr * k, rr * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  // T = I + R^T G R
  CK(cudaMemsetAsync(c->T.p, 0, rr * sizeof(double), c->stream));
  CK(launch_add_identity(c->T.p, r, r, 1.0, c->stream));
  if (c->prec == ISDF_PREC_MIXED) {
    CK(isdf::mixed_smw_products_T(c));
  } else {
    CK(launch_gemm(c->G.p, r, false, c->R.p, r, true, r, r, r, 1.0, 0.0, c->W1.p, r, false, 1, nullptr, false,
                   c->stream));
    CK(launch_gemm(c->R.p, r, true, c->W1.p, r, true, r, r, r, 1.0, 1.0, c->T.p, r, false, 1, nullptr, false,
                   c->stream));
    CK(launch_symmetrize(c->T.p, r, r, c->stream));
  }
  // T = U U^T; Q = R U^-T; K = -Q Q^T
  if (c->prec == ISDF_PREC_MIXED) {
    // U^-1 into Q on the second stream, block row by block row, beside the factorisation
    CK(cudaEventRecord(c->ev_fork, c->stream));
    CK(cudaStreamWaitEvent(c->s2, c->ev_fork, 0));
    CK(launch_cholesky_and_inverse(c->T.p, r, r, 0.0, c->W1.p, r, c->Q.p, r, c->cb_work.p, failT, c->inv_work.p,
                                   c->stream, c->s2, c->ev_chol.data(), reinterpret_cast<float2*>(c->cb_split.p)));
    CK(cudaEventRecord(c->ev_join, c->s2));
    CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    CK(isdf::mixed_smw_products_K(c, Kk, true));
  } else {
    int rc = cholesky_blocked(c, c->T.p, r, r, 0.0, c->W1.p, failT, c->stream);
    if (rc != ISDF_OK) return rc;
    CK(launch_trsm_prep(c->W1.p, r, r, c->Bf.p + 0, r, c->stream));
    CK(cudaMemcpyAsync(c->Q.p, c->R.p, rr * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CK(launch_trsm_right_lt(c->Q.p, r, r, c->Bf.p, r, r, c->stream));
    CK(launch_gemm(c->Q.p, r, false, c->Q.p, r, false, r, r, r, -1.0, 0.0, Kk, r, true, sp, c->partial.p, false,
                   c->stream));
    // restore the fit's TRSM table (Bf held L_r^-1 blocks for D(w) of later calls)
    CK(launch_trsm_prep(c->Lc.p, r, r, c->Bf.p, r, c->stream));
  }
  return ISDF_OK;
}

// Size the single-frequency SMW workspace (synchronising first if a buffer grows).
static int smw_workspace(isdf_ctx* c) {
  const int r = c->rank;
  const size_t rr = (size_t)r * r;
  long long tiles = (long long)((r + 63) / 64) * ((r + 63) / 64 + 1) / 2;
  int sp = split_for(tiles, std::max(r, 1), c->num_sms);
  const bool mixed = c->prec == ISDF_PREC_MIXED;
  if (c->R.cap < rr || c->T.cap < rr || c->W1.cap < rr || c->Q.cap < rr || c->partial.cap < sp * rr ||
      (mixed && c->Xgd.cap < rr))
    SYNC(c->stream);  // a resize frees memory that earlier work may read
  if (mixed) CK(ensure(c->Xgd, rr));
  CK(ensure(c->R, rr));
  CK(ensure(c->T, rr));
  CK(ensure(c->W1, rr));
  CK(ensure(c->Q, rr));
  CK(ensure(c->partial, (size_t)sp * rr));
  CK(ensure(c->ns_bound, 4 + row_abs_sum_work(r, 1)));
  if (c->prec == ISDF_PREC_MIXED) return chol_inverse_workspace(c, r);
  return ISDF_OK;
}

// Synchronise, then check the device status and the failure flags of the
// factorisations of D(w_k) (d_fail) and of I + R^T G R (failT) for k in
// [k0, k0 + nk).
static int smw_finish(isdf_ctx* c, int k0, int nk, const int* failT, const char* who) {
  if (isdf::tl_capture) return ISDF_OK;  // read by graph_check after the replay
  CK(cudaStreamSynchronize(c->stream));
  int rc = check_status(c, who);
  if (rc != ISDF_OK) return rc;
  if (c->rank > 0) {
    std::vector<int> fd(nk), ft(nk);
    CK(cudaMemcpy(fd.data(), c->d_fail + k0, nk * sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(ft.data(), failT, nk * sizeof(int), cudaMemcpyDeviceToHost));
    for (int i = 0; i < nk; ++i)
      if (fd[i] >= 0 || ft[i] >= 0)
        return fail(c, ISDF_ERR_NOT_SPD, std::string(who) + ": capacitance factor not positive definite at omega_index " +
                                             std::to_string(k0 + i));
  }
  for (int i = 0; i < nk; ++i) c->k_ready[k0 + i] = 1;
  return ISDF_OK;
}

int isdf::graph_check(isdf_ctx* c, const char* who) {
  c->err.clear();
  int rc = check_status(c, who);
  int fit_fail = -1;
  if (rc == ISDF_OK) {
    CK(cudaMemcpy(&fit_fail, c->d_ints + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (fit_fail >= 0) {
      c->fitted = false;
      c->polar_ready = false;
      return fail(c, ISDF_ERR_NOT_SPD, std::string(who) + ": the replayed fit needs pivoting (C C^T lost rank); "
                                                          "run it eagerly");
    }
  }
  if (rc != ISDF_OK) {
    c->polar_ready = false;
    return rc;
  }
  // the frequency factorisations: smw_finish's check, now on the host side
  std::fill(c->k_ready.begin(), c->k_ready.end(), 0);
  return smw_finish(c, 0, c->n_omega, c->b_fail, who);
}

extern "C" int smw_inverse(isdf_ctx* c, int k, double* K_out) {
  if (!c) return ISDF_ERR_ARG;
  c->err.clear();
  if (!c->polar_ready) return fail(c, ISDF_ERR_STATE, "smw_inverse: call build_polarizability first");
  if (k < 0 || k >= c->n_omega) return fail(c, ISDF_ERR_ARG, "smw_inverse: omega_index out of range");
  const int r = c->rank, m = c->n_mu;
  const size_t rr = (size_t)r * r;
  c->k_ready[k] = 0;
  if (r > 0) {
    int rc = smw_workspace(c);
    if (rc != ISDF_OK) return rc;
    CK(cudaMemsetAsync(c->d_status, 0, 8 * sizeof(unsigned), c->stream));
    rc = smw_enqueue(c, k, c->d_ints + 3);
    if (rc != ISDF_OK) return rc;
  }
  if (K_out) {
    int rc = copy_padded(c, K_out, c->K.p + rr * k, r, m);
    if (rc != ISDF_OK) return rc;
  }
  return smw_finish(c, k, 1, c->d_ints + 3, "smw_inverse");
}

extern "C" int smw_inverse_all(isdf_ctx* c, double* K_out) {
  if (!c) return ISDF_ERR_ARG;
  c->err.clear();
  if (!c->polar_ready) return fail(c, ISDF_ERR_STATE, "smw_inverse_all: call build_polarizability first");
  const int r = c->rank, m = c->n_mu, nw = c->n_omega;
  const size_t rr = (size_t)r * r;
  std::fill(c->k_ready.begin(), c->k_ready.end(), 0);
  if (c->cap_bfail < (size_t)nw) {
    if (isdf::tl_capture) return fail(c, ISDF_ERR_STATE, "smw_inverse_all: a captured call needs an eager call first");
    CK(cudaStreamSynchronize(c->stream));
    if (c->b_fail) cudaFree(c->b_fail);
    c->b_fail = nullptr;
    c->cap_bfail = 0;
    CK(isdf::dev_malloc(&c->b_fail, nw * sizeof(int)));
    c->cap_bfail = nw;
  }
  if (r > 0) {
    // captured: the status word keeps the fit's flags for graph_check
    if (!isdf::tl_capture) CK(cudaMemsetAsync(c->d_status, 0, 8 * sizeof(unsigned), c->stream));
    CK(cudaMemsetAsync(c->b_fail, 0xff, nw * sizeof(int), c->stream));
    if (c->prec == ISDF_PREC_MIXED && nw > 1) {
      PhaseScope ph(c, ISDF_PH_SMW);
      bool ns = false;
      CK(isdf::mixed_smw_batched_ns(c, nw, c->b_fail, &ns));
      if (!ns) {
        // the bounds ask for too many Newton-Schulz steps: factor D(w) here,
        // then the factorisation route
        if (c->b_cbd.cap < (size_t)nw || c->cb_split.cap < (size_t)64 * r * nw) {
          if (isdf::tl_capture) return fail(c, ISDF_ERR_STATE, "smw_inverse_all: a captured call needs an eager call first");
          CK(cudaStreamSynchronize(c->stream));
          CK(ensure(c->b_cbd, (size_t)nw));
          CK(ensure(c->cb_split, (size_t)64 * r * nw));
        }
        CK(launch_cholesky_blocked_batched(c->D.p, r, (long long)rr, r, nw, 0.0, c->Rw.p, r, (long long)rr, c->b_cbd.p,
                                           c->d_fail, c->stream, split_panel(c, (size_t)64 * r * nw)));
        c->rw_ready = true;
        CK(isdf::mixed_smw_batched(c, nw, c->b_fail));
      }
    } else {
      int rc = smw_workspace(c);
      if (rc != ISDF_OK) return rc;
      for (int k = 0; k < nw; ++k) {
        rc = smw_enqueue(c, k, c->b_fail + k);
        if (rc != ISDF_OK) return rc;
      }
    }
  }
  if (K_out) {
    for (int k = 0; k < nw; ++k) {
      int rc = copy_padded(c, K_out + (size_t)m * m * k, c->K.p + rr * k, r, m);
      if (rc != ISDF_OK) return rc;
    }
  }
  return smw_finish(c, 0, nw, c->b_fail, "smw_inverse_all");
}

extern "C" int apply_eps_inv(isdf_ctx* c, int k, const double* X, int n_rhs, double* Y) {
  if (!c) return ISDF_ERR_ARG;
  c->err.clear();
  if (!c->polar_ready || k < 0 || k >= c->n_omega || !c->k_ready[k])
    return fail(c, ISDF_ERR_STATE, "apply_eps_inv: call smw_inverse for this omega_index first");
  if (!X || !Y) return fail(c, ISDF_ERR_ARG, "apply_eps_inv: null pointer argument");
  if (n_rhs < 1) return fail(c, ISDF_ERR_SHAPE, "apply_eps_inv: n_rhs must be >= 1");
  const int r = c->rank;
  const long long nr = c->n_r;
  const size_t rr = (size_t)r * r;
  const double* Kk = c->K.p + rr * k;
  const int chunk = 64;
  const long long lds = 2 * c->n_half;
  const int nc0 = std::min(n_rhs, chunk);
  const long long tiles0 = (long long)((r + 127) / 128) * ((nc0 + 15) / 16);
  const int sp0 = split_for(std::max(tiles0, 1ll), nr, c->num_sms);
  if (c->tmp1.cap < (size_t)r * nc0 || c->tmp2.cap < (size_t)r * nc0 || c->tmp3.cap < (size_t)nr * nc0 ||
      c->spec.cap < (size_t)lds * nc0 || c->partial.cap < (size_t)sp0 * r * nc0)
    CK(cudaStreamSynchronize(c->stream));  // a resize frees memory that earlier work may read
  CK(ensure(c->tmp1, std::max<size_t>((size_t)r * nc0, 1)));
  CK(ensure(c->tmp2, std::max<size_t>((size_t)r * nc0, 1)));
  CK(ensure(c->tmp3, (size_t)nr * nc0));
  CK(ensure(c->spec, (size_t)lds * nc0));
  CK(ensure(c->partial, std::max<size_t>((size_t)sp0 * r * nc0, 1)));
  if (c->prec == ISDF_PREC_MIXED && c->refine > 0 && c->xgd_ready) {
    if (c->ref.cap < (size_t)2 * r * nc0) CK(cudaStreamSynchronize(c->stream));
    CK(ensure(c->ref, std::max<size_t>((size_t)2 * r * nc0, 1)));
  }
  PhaseScope ph(c, ISDF_PH_APPLY);
  for (int c0 = 0; c0 < n_rhs; c0 += chunk) {
    const int nc = std::min(chunk, n_rhs - c0);
    const double* Xc = X + nr * c0;
    double* Yc = Y + nr * c0;
    if (r == 0) {
      if (Yc != Xc) CK(cudaMemcpyAsync(Yc, Xc, (size_t)nr * nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      continue;
    }
    if (c->prec == ISDF_PREC_MIXED) {
      CK(isdf::mixed_apply_chunk(c, Kk, Xc, Yc, nc));
      continue;
    }
    // T1 = theta^T X (split over the grid), T2 = K T1, T3 = theta T2, Y = X + V T3
    int sp = sp0;  // nc <= nc0: the same split fits the partial buffer
    CK(launch_gemm(c->theta, nr, true, Xc, nr, true, r, nc, (int)nr, 1.0, 0.0, c->tmp1.p, r, false, sp,
                   c->partial.p, true, c->stream));
    CK(launch_gemm(Kk, r, false, c->tmp1.p, r, true, r, nc, r, 1.0, 0.0, c->tmp2.p, r, false,
                   std::min(sp, 16), c->partial.p, true, c->stream));
    CK(launch_gemm(c->theta, nr, false, c->tmp2.p, r, true, (int)nr, nc, r, 1.0, 0.0, c->tmp3.p, nr,
                   false, 1, nullptr, true, c->stream));
    CK(launch_fft_convolve(c->fft, c->tmp3.p, nr, nc, c->spec.p, lds, c->d_wconv, Xc, nr, Yc, nr,
                           c->smem_xy, c->smem_z, c->stream));
  }
  return ISDF_OK;
}

extern "C" int isdf_check_device_wait(isdf_ctx* c, long long limit_ns) {
  if (!c) return ISDF_ERR_ARG;
  c->err.clear();
  if (limit_ns < 1000 || limit_ns > 10000000000ll)
    return fail(c, ISDF_ERR_ARG, "isdf_check_device_wait: limit_ns must be in [1e3, 1e10]");
  if (isdf::tl_capture) return fail(c, ISDF_ERR_STATE, "isdf_check_device_wait: not while a graph is captured");
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemsetAsync(c->d_status, 0, 8 * sizeof(unsigned), c->stream));
  CK(launch_wait_check(c->d_bar, c->d_status, (uint64_t)limit_ns, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const int rc = check_status(c, "isdf_check_device_wait");
  // leave the barrier and the status word as a fresh context has them
  CK(cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), c->stream));
  CK(cudaMemsetAsync(c->d_status, 0, 8 * sizeof(unsigned), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (rc == ISDF_OK) return fail(c, ISDF_ERR_STATE, "isdf_check_device_wait: the never-completed barrier completed");
  return rc;
}

static const char* kPhaseNames[ISDF_NUM_PHASES] = {"points_chol", "fit_gram", "fit_trsm", "coulomb_fft",
                                                   "coulomb_syrk", "polar_d", "whiten_d", "smw", "apply"};

extern "C" const char* isdf_phase_name(int phase) {
  return (phase >= 0 && phase < ISDF_NUM_PHASES) ? kPhaseNames[phase] : nullptr;
}

extern "C" long long isdf_launch_count(void) { return launch_count(); }

extern "C" long long isdf_device_allocations(void) { return isdf::device_allocation_count(); }

extern "C" int isdf_set_refinement(isdf_ctx* c, int steps) {
  if (!c || steps < 0 || steps > 8) return ISDF_ERR_ARG;
  c->refine = steps;
  return ISDF_OK;
}

extern "C" int isdf_set_profiling(isdf_ctx* c, int on) {
  if (!c) return ISDF_ERR_ARG;
  c->prof_on = on != 0;
  return ISDF_OK;
}

thread_local isdf_ctx* isdf::tl_prof_ctx = nullptr;
thread_local int isdf::tl_prof_phase = -1;

isdf::KernelTimer::KernelTimer(int f, cudaStream_t s, double w) : fam(f), st(s), work(w) {
  isdf_ctx* c = tl_prof_ctx;
  if (!c || !c->prof_on) return;
  e0 = take_event(c);
  if (e0) cudaEventRecord(e0, st);
}

isdf::KernelTimer::~KernelTimer() {
  isdf_ctx* c = tl_prof_ctx;
  if (!e0 || !c) return;
  cudaEvent_t e1 = take_event(c);
  if (!e1) {
    c->ev_pool.push_back(e0);
    return;
  }
  cudaEventRecord(e1, st);
  c->kprof.push_back({fam, tl_prof_phase, e0, e1, work, st});
}

static_assert((int)KF_COUNT == (int)ISDF_NUM_KERNEL_FAMILIES, "kernel families of the header and the launchers differ");
static const char* kFamilyNames[KF_COUNT] = {"tc_gemm", "fp64_gemm", "chol_diag", "fft", "slice", "df_gemm"};

extern "C" const char* isdf_kernel_family_name(int fam) {
  return (fam >= 0 && fam < KF_COUNT) ? kFamilyNames[fam] : nullptr;
}

extern "C" int isdf_read_kernel_profile(isdf_ctx* c, double* ms, int* counts, double* work) {
  if (!c) return ISDF_ERR_ARG;
  CK(cudaDeviceSynchronize());
  const int n = ISDF_NUM_KERNEL_FAMILIES * ISDF_NUM_PHASES;
  std::vector<double> acc(n, 0.0), wk(n, 0.0);
  std::vector<int> cnt(n, 0);
  for (auto& r : c->kprof) {
    float t = 0.f;
    if (r.ph >= 0 && r.ph < ISDF_NUM_PHASES && cudaEventElapsedTime(&t, r.e0, r.e1) == cudaSuccess) {
      const int i = r.fam * ISDF_NUM_PHASES + r.ph;
      acc[i] += t;
      wk[i] += r.work;
      cnt[i] += 1;
    }
    c->ev_pool.push_back(r.e0);
    c->ev_pool.push_back(r.e1);
  }
  c->kprof.clear();
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = acc[i];
    if (counts) counts[i] = cnt[i];
    if (work) work[i] = wk[i];
  }
  return ISDF_OK;
}

extern "C" int isdf_read_kernel_trace(isdf_ctx* c, int max, double* t_start, double* t_end, int* family, int* phase,
                                      double* work, int* stream) {
  if (!c || max < 0) return ISDF_ERR_ARG;
  CK(cudaDeviceSynchronize());
  const int n = (int)std::min<size_t>(c->kprof.size(), (size_t)max);
  std::vector<double> t0(n, 0.0), t1(n, 0.0);
  double tmin = 0.0;
  for (int i = 0; i < n; ++i) {
    const auto& r = c->kprof[i];
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, c->kprof[0].e0, r.e0) != cudaSuccess) a = 0.f;
    if (cudaEventElapsedTime(&b, c->kprof[0].e0, r.e1) != cudaSuccess) b = a;
    t0[i] = a;
    t1[i] = b;
    tmin = std::min(tmin, (double)a);
  }
  for (int i = 0; i < n; ++i) {
    const auto& r = c->kprof[i];
    if (t_start) t_start[i] = t0[i] - tmin;
    if (t_end) t_end[i] = t1[i] - tmin;
    if (family) family[i] = r.fam;
    if (phase) phase[i] = r.ph;
    if (work) work[i] = r.work;
    if (stream) stream[i] = r.st == c->stream ? 0 : (r.st == c->s2 ? 1 : (r.st == c->s3 ? 2 : 3));
  }
  for (auto& r : c->kprof) {
    c->ev_pool.push_back(r.e0);
    c->ev_pool.push_back(r.e1);
  }
  c->kprof.clear();
  return n;
}

extern "C" int isdf_read_profile(isdf_ctx* c, double* ms, int* counts) {
  if (!c) return ISDF_ERR_ARG;
  CK(cudaDeviceSynchronize());
  double acc[ISDF_NUM_PHASES] = {0};
  int cnt[ISDF_NUM_PHASES] = {0};
  for (auto& pe : c->prof_ev) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pe.second.first, pe.second.second) == cudaSuccess) {
      acc[pe.first] += t;
      cnt[pe.first] += 1;
    }
    c->ev_pool.push_back(pe.second.first);
    c->ev_pool.push_back(pe.second.second);
  }
  c->prof_ev.clear();
  for (int i = 0; i < ISDF_NUM_PHASES; ++i) {
    if (ms) ms[i] = acc[i];
    if (counts) counts[i] = cnt[i];
  }
  return ISDF_OK;
}

// ---------------------------------------------------------------------------
// Read-only view of a context for the allocation-free apply (noalloc.cu).
namespace isdf {

int ctx_apply_view(isdf_ctx* c, int k, ApplyView* v) {
  if (!c || !v) return ISDF_ERR_ARG;
  c->err.clear();
  if (!c->polar_ready || k < 0 || k >= c->n_omega || !c->k_ready[k])
    return fail(c, ISDF_ERR_STATE, "apply_eps_inv_noalloc: call smw_inverse for this omega_index first");
  v->device = c->device;
  v->num_sms = c->num_sms;
  v->stream = c->stream;
  v->n_r = c->n_r;
  v->n_half = c->n_half;
  v->fft = c->fft;
  v->smem_xy = c->smem_xy;
  v->smem_z = c->smem_z;
  v->wconv = c->d_wconv;
  v->theta = c->theta;
  v->rank = c->rank;
  v->K = c->K.p + (size_t)c->rank * c->rank * k;
  return ISDF_OK;
}

int ctx_fail(isdf_ctx* c, int code, const char* msg) { return fail(c, code, msg); }

}  // namespace isdf
