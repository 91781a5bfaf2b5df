// Host-side launchers of the ISDF-SMW kernels (internal C++ interface of the
// library; the public boundary is include/isdf_smw.h).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace isdf {

// Count of kernel launches issued by this library (all contexts, all threads).
void note_launch();
long long launch_count();

// Every device allocation of the library goes through these two (plain
// cudaMalloc / cudaMallocAsync), which count them (all contexts, threads).
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t s);
long long device_allocation_count();
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}
template <class T>
inline cudaError_t dev_malloc_async(T** p, size_t bytes, cudaStream_t s) {
  return dev_malloc_async(reinterpret_cast<void**>(p), bytes, s);
}

// True on a thread that is capturing a CUDA graph of the entry points
// (batch.cu): the entry points then skip their host synchronisations and
// host reads, take the shapes, rank and uploaded tables of the eager run
// before the capture, ensure() refuses to allocate and the tile autotuner
// only looks up its table.
extern thread_local bool tl_capture;

// SMs that a persistent tensor-core GEMM launched from this thread leaves
// free (0: none), so that latency-bound FP64 kernels queued on another
// stream keep running beside it (k_tc_gemm.cu; TcSmReserve sets it).
extern thread_local int tl_tc_sm_reserve;
// While a DfGemm scope with `on` is alive on this thread, the tiled GEMMs
// (launch_gemm, launch_gemm_batched, launch_gemm_batched2) run their
// products in double-float arithmetic on the FP32 pipe (about 2^-46
// relative per product sum; the mixed path's triangular inverses).
extern thread_local bool tl_gemm_df;
struct DfGemm {
  bool prev;
  explicit DfGemm(bool on) : prev(tl_gemm_df) { tl_gemm_df = on; }
  ~DfGemm() { tl_gemm_df = prev; }
};
// Chunks per FP32 accumulation run of the tensor-core GEMMs launched from
// this thread (kTcGroupChunks unless a TcGroup scope says otherwise; 0:
// one run per block's K range).
// The FP32 accumulator of a block restarts every this many chunks (512
// terms) and the runs are summed in double-float arithmetic in tensor
// memory (GEMMs with one accumulator): the tensor cores' FP32 sums of long
// same-sign runs otherwise lose about 2^-24 per term, which left D = S S^T
// (a sum over all pairs) at 5e-5 relative.  Two products skip it (TcGroup(0)):
// the fit's triangular GEMM, whose epilogue writes three outputs and whose
// error is set by the Gram it reads, and the SYRK of G, whose error is set
// by the FP32 transform of theta.
constexpr int kTcGroupChunks = 8;
extern thread_local int tl_tc_group;
struct TcGroup {
  int prev;
  explicit TcGroup(int n) : prev(tl_tc_group) { tl_tc_group = n; }
  ~TcGroup() { tl_tc_group = prev; }
};
struct TcSmReserve {
  int prev;
  explicit TcSmReserve(int n) : prev(tl_tc_sm_reserve) { tl_tc_sm_reserve = n; }
  ~TcSmReserve() { tl_tc_sm_reserve = prev; }
};

// Per-launch timing by kernel family.  While an API call on a context with
// profiling on is inside one of its phases, a KernelTimer records CUDA
// events around the launch on the launch's own stream, tagged with the
// family, the phase and the launch's algorithmic work (flops for the GEMM
// and Cholesky families, bytes for the FFT and slicing families; for
// KF_TC_GEMM the BF16 MMA flops of the slice products).
enum { KF_TC_GEMM = 0, KF_FP64_GEMM = 1, KF_CHOL_DIAG = 2, KF_FFT = 3, KF_SLICE = 4, KF_DF_GEMM = 5, KF_COUNT = 6 };
struct KernelTimer {
  KernelTimer(int fam, cudaStream_t s, double work);
  ~KernelTimer();
  KernelTimer(const KernelTimer&) = delete;
  KernelTimer& operator=(const KernelTimer&) = delete;
  int fam;
  cudaStream_t st;
  double work;
  cudaEvent_t e0 = nullptr;
};

// ---- k_dense.cu -----------------------------------------------------------
cudaError_t launch_check_finite(const double* p, long long n, unsigned* status, cudaStream_t s);
cudaError_t launch_gather_rows(const double* src, long long lds, const int* idx, int nrows, int ncols,
                               double* dst, long long ldd, cudaStream_t s);
// C (M x N) = (A_v B_v^T) .* (A_c B_c^T); A: M x n_e, B: N x n_e, both
// column-major; the first n_v columns form the v part.
cudaError_t launch_facesplit_gram(const double* A, long long lda, int M, const double* B,
                                  long long ldb, int N, int n_v, int n_e, double* C, long long ldc,
                                  cudaStream_t s);
// C = alpha * op(A) op(B)^T + beta * C with op(A)(m, k), op(B)(n, k):
// ka / kb false -> element (row, k) at p[row + ld k]; true -> p[k + ld row].
// lower_only: M == N, only lower tiles are computed and mirrored (SYRK).
// splits > 1 needs `partial` of splits * M * N doubles (deterministic reduce).
// narrow: 128 x 16 tiles (N small) instead of 64 x 64.
// tri: TRI_B_LOWER_T (op(B)(n, k) = 0 for k < n) and / or TRI_A_LOWER
// (op(A)(m, k) = 0 for k > m): the zero k blocks are skipped.
enum { TRI_B_LOWER_T = 1, TRI_A_LOWER = 2 };
cudaError_t launch_gemm(const double* A, long long lda, bool ka, const double* B, long long ldb,
                        bool kb, int M, int N, int K, double alpha, double beta, double* C,
                        long long ldc, bool lower_only, int splits, double* partial, bool narrow,
                        cudaStream_t s, int tri = 0);
// D (r x r, symmetric) = sum_{i<n_v, j<n_c} S(:, ij) S(:, ij)^T with
// S(a, ij) = phimu(a, i) phimu(a, n_v + j) sw[i n_c + j]; phimu r x n_e.
cudaError_t launch_polarizability(const double* phimu, long long ldp, int r, int n_v, int n_c,
                                  const double* sw, double* D, long long ldd, int splits,
                                  double* partial, cudaStream_t s);
// Blocked right solve X <- X L^-T in place (L lower r x r, X M x r).
// trsm_prep builds Bf: diagonal blocks L_JJ^-1, off-diagonal -L_JJ^-1 L_JI.
cudaError_t launch_trsm_prep(const double* L, long long ldl, int r, double* Bf, long long ldb,
                             cudaStream_t s);
cudaError_t launch_trsm_right_lt(double* X, long long ldx, int M, const double* Bf, long long ldb,
                                 int r, cudaStream_t s);
cudaError_t launch_transpose(const double* src, long long lds, int M, int N, double* dst,
                             long long ldd, cudaStream_t s);
// *out = sum of a[i]^2, i < n (deterministic; scratch: 256 doubles)
cudaError_t launch_sumsq(const double* a, long long n, double* scratch, double* out, cudaStream_t s);
// batch > 1: matrices A + z sA
cudaError_t launch_symmetrize(double* A, long long lda, int n, cudaStream_t s, int batch = 1, long long sA = 0);
// sqrt(-2 Omega(i w_k)^-1) of every pair (i, j) and frequency k from the
// device array ew = [energies | frequencies] into sw (and swf in FP32, if
// not null), index k n_v n_c + i n_c + j.
cudaError_t launch_pair_weights(const double* ew, int n_v, int n_c, int n_omega, double* sw, float* swf,
                                cudaStream_t s);
// out[z] (device) = max_i sum_j |A_z(i, j)|, the Gershgorin bound of a
// symmetric A_z's spectrum, for the batch matrices at A + z sA; work: at
// least row_abs_sum_work(n, batch) device doubles.  Deterministic.
size_t row_abs_sum_work(int n, int batch);
cudaError_t launch_row_abs_sum_max(const double* A, long long lda, int n, double* out, double* work, cudaStream_t s,
                                   int batch = 1, long long sA = 0);
// X_z = alpha[z] I for z < batch (n x n, ld n, matrix z at X + z n^2; alpha on the device)
cudaError_t launch_scaled_identity(double* X, int n, int batch, const double* alpha, cudaStream_t s);
// c = a + b, n doubles (c may be a or b); batch problems at + z stride
// (b at + z stride_b; stride_b < 0: the same stride)
cudaError_t launch_add(const double* a, const double* b, double* c, long long n, cudaStream_t s, int batch = 1,
                       long long stride = 0, long long stride_b = -1);
cudaError_t launch_add_identity(double* A, long long lda, int n, double v, cudaStream_t s, int batch = 1,
                                long long sA = 0);
// Two-level batch of GEMMs: problem (z1, z2), z1 < b1, z2 < b2, has
// X_z = X + z1 * sX1 + z2 * sX2 (X = A, B, C); b1 * b2 <= 65535.
struct GemmBatch {
  int b1, b2;
  long long sA1, sB1, sC1, sA2, sB2, sC2;
};
// lower: M == N, only the lower tiles are computed and mirrored (SYRK).
cudaError_t launch_gemm_batched2(const double* A, long long lda, bool ka, const double* B, long long ldb, bool kb,
                                 int M, int N, int K, double alpha, double beta, double* C, long long ldc,
                                 const GemmBatch& bt, bool lower, cudaStream_t s, int tri = 0);
// batch independent GEMMs C_z = alpha op(A_z) op(B_z)^T + beta C_z, z < batch,
// X_z = X + z * strideX (same layout conventions as launch_gemm)
cudaError_t launch_gemm_batched(const double* A, long long lda, bool ka, long long sA, const double* B,
                                long long ldb, bool kb, long long sB, int M, int N, int K, double alpha, double beta,
                                double* C, long long ldc, long long sC, int batch, cudaStream_t s, int tri = 0);
// Li = L^-1 for lower-triangular L (r x r), FP64; work >= (r/2 + 64)^2
// doubles; partial (may be null) >= 4 (r/2 + 64)^2 doubles for split-K.
cudaError_t launch_tri_inverse(const double* L, long long ldl, int r, double* Li, long long ldi, double* work,
                               double* partial, cudaStream_t s);
// Li_z = L_z^-1 for batch lower-triangular r x r matrices L + z sL ->
// Li + z sI (same merges, one launch per merge for the whole batch);
// work: batch (r/2 + 64)^2 doubles.
cudaError_t launch_tri_inverse_batched(const double* L, long long ldl, long long sL, int r, int batch, double* Li,
                                       long long ldi, long long sI, double* work, cudaStream_t s);
// L (n_full x n_full column-major) from the row-major pivoted factor Lr.
cudaError_t launch_factor_to_colmajor(const double* Lr, int n, const int* perm, const int* rank,
                                      double* L, long long ldl, int n_full, cudaStream_t s);

// C = alpha * sum_z partial[z] + beta * C (partials column-major M x N);
// lower_only: tiles above the diagonal (tile size `tile`) are read mirrored.
// batch > 1: problem z reads partial + z * splits * M * N and writes C + z * sC.
cudaError_t launch_splitk_reduce(const double* partial, int splits, int M, int N, double alpha, double beta,
                                 double* C, long long ldc, bool lower_only, int tile, cudaStream_t s, int batch = 1,
                                 long long sC = 0);

// ---- k_contour.cu: contour-integral polarizability (Algorithm 2) ----------
// Nodes from the bound of Eq. rel_err_Cauchy for a target error tol.
int contour_nodes_recommended(double gap, double width, double tol);
// Host tables of the n_nodes midpoint nodes z_j on the upper half contour:
// wtab (2 n_nodes (n_v + n_c) doubles) = 1 / (z_j - e_i) as (re, im), wnode
// (2 n_nodes) = the weights h z'(t_j).  cudaErrorInvalidValue without a gap.
cudaError_t contour_tables(const double* energies, int n_v, int n_c, int n_nodes, std::vector<double>& wtab,
                           std::vector<double>& wnode);
// D (r x r, symmetric) = -2 C_r Omega^-1 C_r^T by the contour integral over
// the orbitals at the r points (phimu, r x (n_v + n_c), ld ldp); nodes may
// be split across blocks (partial: split r^2 doubles, at most partial_cap).
cudaError_t launch_contour_polarizability(const double* phimu, long long ldp, int r, int n_v, int n_c,
                                          const double* d_wtab, const double* d_wnode, int n_nodes, double* D,
                                          long long ldd, double* partial, size_t partial_cap, int num_sms,
                                          cudaStream_t s);

// ---- k_chol_blocked.cu ----------------------------------------------------
// Blocked Cholesky without pivoting of the symmetric n x n W (column-major,
// lower part read) into L (may equal W).  *fail = -1 on success, else the
// first column whose pivot is <= tol_rel * max(diag W) (later steps are
// skipped); dmax: one double of scratch.
// split: nullptr for FP64 trailing updates, else 64 n float pairs of
// scratch for the double-float trailing updates (about 2^-46 relative per
// update instead of 2^-53; the mixed path).
cudaError_t launch_cholesky_blocked(const double* W, long long ldw, int n, double tol_rel, double* L, long long ldl,
                                    double* dmax, int* fail, cudaStream_t s, float2* split = nullptr);
// The inverse of one lower-triangular block of at most 64 x 64 (L, ld ldl)
// into Li (ld ldi; strict upper part zeroed): one thread block.
cudaError_t launch_diag_inverse_block(const double* L, long long ldl, int bs, double* Li, long long ldi,
                                      cudaStream_t s);
// launch_cholesky_blocked on stream s, and the inverse Li = L^-1 built
// block row by block row on stream aux while the factorisation proceeds:
// once the diagonal block J is factored, row block J of Li is
//   Li[J, J] = L_JJ^-1,  Li[J, 0:J] = -L_JJ^-1 (L[J, 0:J] Li[0:J, 0:J]),
// which needs only rows of L that earlier steps finished.  The caller orders
// aux after everything Li and work depend on, and joins aux before Li is
// used.  ev: at least ceil(n / 64) events (3 ceil(n / 64) with aux2);
// work: 64 n + 8 * 64 n doubles.  If the factorisation stops (fail >= 0),
// Li is undefined.
// aux2 (double-float path only): look-ahead.  Each step's trailing update
// is split: the next 64 columns on s, so the next diagonal block can start
// at once, and the rest on aux2 beside it; s waits for that rest before it
// updates the columns the rest also touches.  aux2 is joined into s before
// the function returns.
cudaError_t launch_cholesky_and_inverse(const double* W, long long ldw, int n, double tol_rel, double* L,
                                        long long ldl, double* Li, long long ldi, double* dmax, int* fail,
                                        double* work, cudaStream_t s, cudaStream_t aux, cudaEvent_t* ev,
                                        float2* split = nullptr, cudaStream_t aux2 = nullptr);
// launch_cholesky_blocked for `batch` equal-size matrices W + z sW -> L + z sL;
// dmax and fail: batch entries; split: nullptr or batch x 64 n float pairs.
cudaError_t launch_cholesky_blocked_batched(const double* W, long long ldw, long long sW, int n, int batch,
                                            double tol_rel, double* L, long long ldl, long long sL, double* dmax,
                                            int* fail, cudaStream_t s, float2* split = nullptr);

// ---- k_chol.cu ------------------------------------------------------------
struct CholWork {
  double* d;         // n
  double* part_val;  // 2 * max_blocks
  int* part_idx;     // 2 * max_blocks
  int* used;         // n
  unsigned* bar;     // 2 (count, generation)
  int max_blocks;
};
// Cholesky of the symmetric n x n matrix W (column-major, full storage):
// P^T W P = L L^T.  pivot = 1: diagonal pivoting, stops when the largest
// remaining diagonal is <= tol_rel * max(diag W); pivot = 0: natural order,
// stops (ST_NOT_SPD) at a non-positive pivot.  Writes Lr (row-major n x n,
// row index = original index), perm (n), *rank.
cudaError_t launch_cholesky(const double* W, long long ldw, int n, int pivot, double tol_rel,
                            double* Lr, int* perm, int* rank, unsigned* status, const CholWork& w,
                            int num_sms, uint64_t limit_ns, cudaStream_t s);
// Two co-resident blocks wait on a grid barrier that never completes (the
// counter at bar[0] is preset past the grid size) with the wait bound
// limit_ns: both give up, ST_TIMEOUT goes to *status.  bar: 2 words.
cudaError_t launch_wait_check(unsigned* bar, unsigned* status, uint64_t limit_ns, cudaStream_t s);

// ---- k_fft.cu -------------------------------------------------------------
constexpr int FFT_MAX_FACTORS = 16;
struct FftAxis {
  int n;
  int nf;
  int f[FFT_MAX_FACTORS];
  const double* tw;  // device, 2 n doubles: exp(-2 pi i t / n), t = 0..n-1
};
struct FftGrid {
  FftAxis ax[3];  // x, y, z
  int h;          // n1 / 2 + 1
};
// Forward real-to-complex transform of ncols real columns (each n1 n2 n3,
// ld = ldx) into the half spectrum (h n2 n3 complex per column, ld = lds
// doubles), multiplied by the real weight table wt (h n2 n3) if non-null.
cudaError_t launch_fft_forward(const FftGrid& g, const double* X, long long ldx, int ncols,
                               double* S, long long lds, const double* wt, size_t smem_xy,
                               size_t smem_z, cudaStream_t s);
// Y = Add + F^-1 diag(wt) F In for ncols columns (wt includes 1 / N_r; Add
// may be null, then Y = F^-1 diag(wt) F In); S is half-spectrum scratch
// (ncols * lds doubles).  Y may alias Add (element-wise update).
cudaError_t launch_fft_convolve(const FftGrid& g, const double* In, long long ldin, int ncols,
                                double* S, long long lds, const double* wt, const double* Add,
                                long long ldadd, double* Y, long long ldy, size_t smem_xy,
                                size_t smem_z, cudaStream_t s);
// Mixed path: forward FP32 transform of ncols float64 columns with weights
// wt, written as nsl BF16 slices (slice l at out[(l rows_pad + col) kp + k],
// k = 2 q + {0 re, 1 im}); S32 is FP32 scratch (ncols * lds32 floats,
// lds32 >= 2 h n2 n3).
cudaError_t launch_fft_forward_slices(const FftGrid& g, const double* X, long long ldx, int ncols, float* S32,
                                      long long lds32, const double* wt, __nv_bfloat16* out, int rows_pad, int kp,
                                      int nsl, size_t smem_xy, size_t smem_z, cudaStream_t s);
size_t fft_smem_xy(const FftGrid& g);
size_t fft_smem_z(const FftGrid& g);
cudaError_t fft_configure(size_t smem_xy, size_t smem_z);

// ---- k_tc_gemm.cu: split-precision GEMMs on tcgen05 -----------------------
// A "slice matrix": s BF16 slices of an R x K FP64 operand, row-major with
// K contiguous; slice l occupies rows [l rows_pad, l rows_pad + R) of a
// (s rows_pad) x kp array.  rows_pad % 128 == 0, kp % 64 == 0, zero padded.
struct TcOperand {
  const __nv_bfloat16* p;
  int rows_pad;
  int kp;
  int s;
};
// slices of a column-major FP64 matrix (R x C, element (r, c) at src[r + lds c]);
// columns c >= kv are shifted to c - kv + kvp (kv = kvp = 0: no shift)
// batch > 1: matrix z at src + z * sstride, its slices at dst + z * dstride
// (elements; dstride % 8 == 0), for all three slicing launchers.
cudaError_t launch_slice_colmajor(const double* src, long long lds, int R, int C, int kv, int kvp,
                                  __nv_bfloat16* dst, int Rp, int Kp, int s, cudaStream_t st, int batch = 1,
                                  long long sstride = 0, long long dstride = 0);
// slices of a row-major FP64 matrix (R x K, element (r, k) at src[k + lds r])
cudaError_t launch_slice_rowmajor(const double* src, long long lds, int R, int K, __nv_bfloat16* dst, int Rp,
                                  int Kp, int s, cudaStream_t st, int batch = 1, long long sstride = 0,
                                  long long dstride = 0);
// Slices of the pair operand at the points, S(a, i n_c + j) =
// phimu(a, i) phimu(a, n_v + j) swf[i n_c + j] (r rows, K = n_v n_c, FP32
// weights), zero in the padding up to Rp x Kp (Rp a multiple of 4, Kp of
// 8): the destination needs no clearing; for batch > 1, problem z uses
// swf + z n_v n_c.
cudaError_t launch_pair_slices(const double* phimu, long long ldp, int r, int n_v, int n_c, const float* swf,
                               __nv_bfloat16* dst, int Rp, int Kp, int s, cudaStream_t st, int batch = 1,
                               long long dstride = 0);
// Unscaled pair operand transposed: slices with rows p = i n_c + j (Pp rows
// per slice), K = the r points (Kp >= r, multiple of 8).
cudaError_t launch_pair_slices_t(const double* phimu, long long ldp, int r, int n_v, int n_c, __nv_bfloat16* dst,
                                 int Pp, int Kp, int s, cudaStream_t st);
// C (M x N, column-major FP64) = alpha sum_{i+j<s} A_i B_j^T + beta C.  With
// `partial` (max_split * M * N doubles) long K is split over blocks and
// reduced in FP64; pass max_split >= tc_min_splits(kp) to keep every
// accumulator within kTcMaxChunksPerSplit chunks.  lower_only: SYRK-style (M == N, mirrored).  tri_b: B is
// lower triangular as B(n, k), chunks past the tile's last n are skipped.
cudaError_t tc_gemm_f64(const TcOperand& A, const TcOperand& B, int M, int N, double alpha, double beta,
                        double* C, long long ldc, bool lower_only, bool tri_b, double* partial, int max_split,
                        int num_sms, unsigned* status, cudaStream_t st);
// A tensor-memory accumulator sums at most this many 64-wide K chunks
// (8192 terms): FP32 accumulation error grows with the number of terms
// (the long SYRKs add hundreds of thousands of same-sign products), so a
// longer K is split across blocks whose partial tiles are summed in FP64.
constexpr int kTcMaxChunksPerSplit = 128;
inline int tc_min_splits(long long kp) { return (int)((kp / 64 + kTcMaxChunksPerSplit - 1) / kTcMaxChunksPerSplit); }
// A batch of `count` problems of the same shape: problem b reads its A slice
// stack starting at row b * a_rows of A.p (a_rows = 0: one A for all), its B
// at row b * b_rows, and writes C + b * c_stride (split-K partials: b *
// splits * M * N).
struct TcBatch {
  int count;
  int a_rows, b_rows;
  long long c_stride;
};
cudaError_t tc_gemm_f64_batched(const TcOperand& A, const TcOperand& B, int M, int N, double alpha, double beta,
                                double* C, long long ldc, bool lower_only, bool tri_b, double* partial, int max_split,
                                int num_sms, unsigned* status, cudaStream_t st, const TcBatch& bt);
// Grouped persistent form (k_tc_grouped.cu): up to 32 problems, each a
// batch as tc_gemm_f64_batched takes it (no split-K; FP64 output with
// alpha / beta; lower: square problems with mirrored lower tiles), all in
// one launch whose blocks claim 128 x 128 output tiles from a device work
// queue.  dev_work: tc_grouped_workspace_bytes(n) bytes of device memory
// that holds the tensor maps, problem records and the queue counter;
// `staged` keeps the host copy of what was last uploaded there (an upload
// synchronises the stream, and none happens while a graph is captured: a
// captured call needs an eager call with the same problems first).
struct TcGroupProblem {
  TcOperand A, B;
  int M, N;
  double alpha, beta;
  double* C;
  long long ldc;
  bool lower;
  TcBatch bt;
};
size_t tc_grouped_workspace_bytes(int nprob);
cudaError_t tc_gemm_f64_grouped(const TcGroupProblem* probs, int nprob, void* dev_work, size_t work_bytes,
                                std::vector<unsigned char>& staged, int num_sms, unsigned* status, cudaStream_t st);
// C = A B^T in FP64 (M x N, column-major), and the BF16 slices of C twice:
// row-major (element (m, n) at zs[m zs_kp + n], slice stride zs_rows_pad
// zs_kp) and transposed (element (n, m) at zt[n zt_kp + m], slice stride
// zt_rows_pad zt_kp); no split-K.  Padding entries of zs / zt are not written.
cudaError_t tc_gemm_f64_slices(const TcOperand& A, const TcOperand& B, int M, int N, double* C, long long ldc,
                               bool tri_b, __nv_bfloat16* zs, int zs_rows_pad, int zs_kp, __nv_bfloat16* zt,
                               int zt_rows_pad, int zt_kp, unsigned* status, cudaStream_t st);
// Face-split Gram (A_v B_v^T) .* (A_c B_c^T): chunks [0, kv_iters) feed the
// first accumulator, the rest the second.  Output FP64 column-major (C) or,
// with zs non-null, BF16 slices (row-major M x N, zs_rows_pad x zs_kp).
// X = A B^T with column n of problem b scaled by colscale[b cs_bstride + n],
// written as BF16 slices (row-major M x N, slice stride zs_rows_pad rows of
// zs_kp; problem b at zs + b zs_bstride) instead of FP64.
cudaError_t tc_scaled_slices(const TcOperand& A, const TcOperand& B, int M, int N, const float* colscale,
                             long long cs_bstride, __nv_bfloat16* zs, int zs_rows_pad, int zs_kp, long long zs_bstride,
                             unsigned* status, cudaStream_t st, const TcBatch& bt);
cudaError_t tc_facesplit(const TcOperand& A, const TcOperand& B, int M, int N, int kv_iters, double* C,
                         long long ldc, __nv_bfloat16* zs, int zs_rows_pad, int zs_kp, unsigned* status,
                         cudaStream_t st);

}  // namespace isdf

// ---- api.cu: read-only context view for the allocation-free apply -------
struct isdf_ctx;
namespace isdf {
struct ApplyView {
  int device;
  int num_sms;
  cudaStream_t stream;
  long long n_r;
  long long n_half;
  FftGrid fft;
  size_t smem_xy, smem_z;
  const double* wconv;
  const double* theta;
  int rank;
  const double* K;
};
// Fills *v for frequency index k, or returns an ISDF_ERR_* code with the
// context's error message set.
int ctx_apply_view(isdf_ctx* c, int k, ApplyView* v);
int ctx_fail(isdf_ctx* c, int code, const char* msg);
}  // namespace isdf
