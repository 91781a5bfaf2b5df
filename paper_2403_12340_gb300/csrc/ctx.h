// Internal: the ISDF-SMW context (opaque in the public header).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "kernels.h"

namespace isdf {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // bound on any device-side wait
constexpr int kMaxGrid = 512;

struct DevBuf {
  double* p = nullptr;
  size_t cap = 0;  // doubles
  __nv_bfloat16* bf() const { return reinterpret_cast<__nv_bfloat16*>(p); }
};

cudaError_t ensure(DevBuf& b, size_t n_doubles);
inline cudaError_t ensure_bf16(DevBuf& b, size_t n_elems) { return ensure(b, (n_elems + 3) / 4); }
void release(DevBuf& b);

}  // namespace isdf

using isdf::DevBuf;
using isdf::FftGrid;

struct isdf_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  int n[3] = {0, 0, 0};
  double L[3] = {0, 0, 0};
  long long n_r = 0;
  double dv = 0;
  FftGrid fft{};
  long long n_half = 0;  // h n2 n3 complex entries of a half spectrum
  size_t smem_xy = 0, smem_z = 0;
  double* d_tables = nullptr;  // twiddles x, y, z | sqrt SYRK weights | convolution weights
  const double* d_wsyrk = nullptr;
  const double* d_wconv = nullptr;
  unsigned* d_status = nullptr;
  unsigned* d_bar = nullptr;
  int* d_ints = nullptr;  // [0] rank
  std::string err;

  // fit state
  bool fitted = false;
  const double* phi = nullptr;
  double* theta = nullptr;
  int n_v = 0, n_c = 0, n_mu = 0, rank = 0;
  std::vector<int> perm;  // host copy, n_mu
  int* d_idx = nullptr;
  int* d_perm = nullptr;   // pivot order of the fit
  int* d_perm2 = nullptr;  // scratch order of the unpivoted factorisations
  size_t cap_idx = 0;
  DevBuf phimu, phimu_p, A, Lr, Lc, Bf, chol_d, chol_part, spec, G, D, K, R, T, W1, Q, partial, tmp1,
      tmp2, tmp3, sw;
  int* d_used = nullptr;
  int* d_part_idx = nullptr;
  size_t cap_used = 0;

  // mixed precision (ISDF_PREC_MIXED): BF16 slice matrices and FP64 helpers
  int prec = 0;
  // second stream for the latency-bound FP64 factorisations, run beside the
  // tensor-core / FFT work of the main stream; fork / join by events
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // a third stream that builds a triangular inverse block row by block row
  // beside the factorisation producing it (launch_cholesky_and_inverse)
  cudaStream_t s3 = nullptr;
  cudaEvent_t ev_join3 = nullptr;
  // a fourth stream for the look-ahead of the fit's factorisation (the rest
  // of each step's trailing update beside the next diagonal block)
  cudaStream_t s4 = nullptr;
  std::vector<cudaEvent_t> ev_chol;  // one per 64-wide factorisation step
  DevBuf inv_work;
  // split panels (float pairs, one per double) of the mixed path's
  // double-float trailing updates: one factorisation at a time (cb_split),
  // the batched T of smw_inverse_all (b_split)
  DevBuf cb_split, b_split;
  DevBuf m_ths;  // BF16 slices of theta (rows = grid points), written by the epilogue of the fit's TRSM
  DevBuf Rw;             // Cholesky factors of D(w), one r x r block per frequency
  int* d_fail = nullptr; // their failure flags
  size_t cap_fail = 0;
  DevBuf cb_work;  // blocked Cholesky: the max diagonal
  DevBuf m_phis, m_phimus, m_zs, m_linv, m_linvs, m_work, m_thetas_t, m_s32, m_ss, m_pairs, m_sa, m_sb, m_xs;

  // phase profiling
  bool prof_on = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
  std::vector<cudaEvent_t> ev_pool;
  struct KRec {
    int fam, ph;
    cudaEvent_t e0, e1;
    double work;
    cudaStream_t st;
  };
  std::vector<KRec> kprof;

  // all frequencies at once (mixed.cu, api.cu): per-frequency r x r stacks,
  // their slice stacks, scratch of the batched factorisations, failure flags
  DevBuf bW1, bT, bU, bQ, b_s1, b_s2, b_s3, b_work, b_cb, b_dtmp, b_cbd;
  DevBuf ctab;  // contour-integral polarizability: resolvent weights and node weights
  DevBuf cx[12];  // COHSEX (cohsex.cu): spectra, cross products, scratch
  DevBuf m_pairs_t, swf;  // pair-space whitening: transposed pair slices; the pair weights in FP32 (mixed path)
  DevBuf ew;                     // energies and frequencies of the last polarizability, on the device
  // mixed path, one frequency: R^-1 of D = R R^T, D^-1 = R^-T R^-1 and the
  // Xgd: (I + G D)^-1 of the single-frequency capacitance (kept for the
  // refinement of the apply); ns_bound: Gershgorin bounds and their workspace
  DevBuf Xgd, m_sd, ns_bound;
  // all frequencies by Newton-Schulz (mixed_smw_batched_ns): the schedule and
  // per-frequency start scales of the last eager call (a captured call
  // replays them), the grouped-GEMM descriptor slots and their host copies
  double ns_e0 = -1.0;  // the largest e0 over the frequencies (see NsPlan)
  int ns_nw = 0;
  bool rw_ready = false;  // c->Rw holds the Cholesky factors of every D(w)
  DevBuf ns_alpha, ns_work, b_s4;
  std::vector<std::vector<unsigned char>> ns_staged;
  bool xgd_ready = false;  // K of the single frequency came from Newton-Schulz: Xgd holds (I + G D)^-1
  int refine = 0;        // refinement rounds of the SMW solve in the mixed apply (isdf_set_refinement)
  DevBuf ref;            // their scratch: two r x 64 blocks
  std::vector<double> ew_host;   // their host copy (the source of the asynchronous upload)
  bool pair_whiten = false;  // mixed path: whiten D in pair space (chosen from the fit's factor)
  int pair_mode = 0;         // the precision argument of the last fit
  DevBuf kappa_work;         // [0] ||L||_F^2, [1] ||L^-1||_F^2, [2..] reduction scratch
  int* b_fail = nullptr;
  size_t cap_bfail = 0;

  // adjoint (adjoint.cu): L_r^-1, r x r products, the pair matrix at the
  // points and its gradient, device copy of the energies
  DevBuf a_linv, a_m1, a_m2, a_m3, a_m4, a_cp, a_y, a_gd, a_e;
  // adjoint through the fit: three N_r x r blocks (dL/dZ, the face-split
  // factors), point-row gradients, two more r x r products
  DevBuf a_z1, a_z2, a_z3, a_gpm, a_gpp, a_m5, a_m6;

  // polarizability / SMW state
  bool polar_ready = false;
  int n_omega = 0;
  std::vector<double> omega;
  std::vector<double> energies;  // of the last build_polarizability
  std::vector<char> k_ready;

  // what a graph capture replays (recorded by the eager calls)
  std::vector<int> fit_idx;  // points of the last fit
  int fit_mode = -1;         // its precision argument
  bool fit_full = false;     // factored unpivoted at full rank
  bool polar_whiten = false; // pair-space whitening chosen by the last build_polarizability
  int polar_nodes = 0;       // its contour node count (0: pair sum)
};

namespace isdf {

inline cudaEvent_t take_event(isdf_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Context and phase that KernelTimer records into on this thread (null
// outside a profiled phase).
extern thread_local isdf_ctx* tl_prof_ctx;
extern thread_local int tl_prof_phase;

// Records a start event now and an end event when it goes out of scope
// (only while profiling is on); launches inside the scope are timed too.
struct PhaseTimer {
  isdf_ctx* c;
  int ph;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr;
  isdf_ctx* prev_ctx = nullptr;
  int prev_ph = -1;
  bool active = false;
  PhaseTimer(isdf_ctx* ctx, int phase, cudaStream_t stream = nullptr)
      : c(ctx), ph(phase), st(stream ? stream : ctx->stream) {
    if (!c->prof_on || tl_capture) return;  // a captured graph carries no timing events
    active = true;
    prev_ctx = tl_prof_ctx;
    prev_ph = tl_prof_phase;
    tl_prof_ctx = c;
    tl_prof_phase = ph;
    e0 = take_event(c);
    if (e0) cudaEventRecord(e0, st);
  }
  ~PhaseTimer() {
    if (active) {
      tl_prof_ctx = prev_ctx;
      tl_prof_phase = prev_ph;
    }
    if (!e0) return;
    cudaEvent_t e1 = take_event(c);
    if (!e1) {
      c->ev_pool.push_back(e0);
      return;
    }
    cudaEventRecord(e1, st);
    c->prof_ev.push_back({ph, {e0, e1}});
  }
};

// mixed.cu
cudaError_t mixed_fit_gram(isdf_ctx* c, const double* phi, const double* phimu_p, int n_v, int n_c, int r);
cudaError_t mixed_fit_solve(isdf_ctx* c, double* theta, int r, bool linv_ready);
cudaError_t mixed_polar_D(isdf_ctx* c, const float* swf, int n_omega);
cudaError_t mixed_whiten_D(isdf_ctx* c, const double* Dpp, double* Dk);
cudaError_t mixed_polar_D_pairspace(isdf_ctx* c, const float* swf, int n_omega);
cudaError_t mixed_polar_G(isdf_ctx* c);
cudaError_t mixed_smw_products_T(isdf_ctx* c);
cudaError_t mixed_smw_products_K(isdf_ctx* c, double* Kk, bool uinv_ready);
cudaError_t mixed_apply_chunk(isdf_ctx* c, const double* Kk, const double* X, double* Y, int nc);
// K(w_k) = -D(w_k) (I + G D(w_k))^-1 for every frequency by Newton-Schulz,
// each product one grouped persistent GEMM over every (frequency, tile);
// *used = false if the spectral bounds ask for too many steps (the caller
// then factors).
cudaError_t mixed_smw_batched_ns(isdf_ctx* c, int nw, int* fail_T, bool* used);
// The same for n systems at once (each after an eager smw_inverse_all that
// took the Newton-Schulz route), one grouped launch per product over every
// (system, frequency, tile), on stream st; work holds ns_stage_slots()
// slots of ws bytes (tc_grouped_workspace_bytes(n), rounded up to 256).
int ns_stage_slots();  // descriptor slots of ns_stage_grouped's workspace
cudaError_t ns_stage_grouped(isdf_ctx** cs, int n, cudaStream_t st, void* work, size_t ws,
                             std::vector<std::vector<unsigned char>>& staged);
// K = -A^-1 for the SPD A in c->T by Newton-Schulz iteration on the tensor
// cores, X <- X (2 I - A X) from X = alpha I, `iters` times (the last
// product written negated into Kk)
// Newton-Schulz schedule: for each step the scale beta of
// X <- beta (2 X - X M X) and the BF16 slices of its products (ns_plan).
struct NsPlan {
  std::vector<double> beta;
  std::vector<int> s;
  int steps() const { return (int)beta.size(); }
};
// e0 = (hi - lo) / (hi + lo) for a spectrum of M within [lo, hi]; false if
// the iteration needs more than 12 steps.
bool ns_plan(double e0, NsPlan& p);
// K = -D (I + G D)^-1 for the D at Dk (r x r, ld r) and c->G, into Kk, on
// the main stream, in two parts: mixed_ns_prepare builds M = I + G D (in
// c->T, its slices in c->m_sd), then mixed_ns_iterate runs the Newton-Schulz
// steps of `plan` for M^-1 from X = alpha I and K = -D X (scratch: c->R,
// c->Xgd, which keeps X, and the slices c->m_sa, m_sb)
cudaError_t mixed_ns_prepare(isdf_ctx* c, const double* Dk);
cudaError_t mixed_ns_iterate(isdf_ctx* c, const double* Dk, double* Kk, double alpha, const NsPlan& plan);
// Upper end of the spectrum of I + G D, 1 + |G| |D| from bounds of the two
// spectra (its lower end is 1: G D has the eigenvalues of D^1/2 G D^1/2 >= 0)
double ns_kappa(double g_bound, double d_bound);
// Range [wmin, wmax] of the pair weights w = 2 |dE| / (dE^2 + w^2) over the
// valence-conduction pairs, from the band edges (the weight is unimodal in
// |dE|, peaking at |dE| = w): in the whitened basis the spectrum of D(w)
// lies within it.
void pair_weight_bounds(const double* energies, int n_v, int n_c, double w, double* wmin, double* wmax);
// All frequencies at once: D(w_k) for k < n_omega (chunked to a memory
// budget), and K(w_k) from the factors R(w_k) in c->Rw (T factors and
// their failure flags in c->bU / fail_T).
cudaError_t mixed_polar_D_batched(isdf_ctx* c, const float* swf, int n_omega);
cudaError_t mixed_smw_batched(isdf_ctx* c, int n_omega, int* fail_T);

// api.cu: after a captured graph of isdf_fit, build_polarizability and
// smw_inverse_all has run (stream synchronised), read the device status and
// failure flags that the eager calls read themselves, and set the host state
// those calls would have set.
int graph_check(isdf_ctx* c, const char* who);

}  // namespace isdf
