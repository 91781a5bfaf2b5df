// Dense FP64 kernels of the ISDF-SMW path: gather, face-split Gram (ISDF
// fit right-hand side M C^T), generic GEMM / SYRK with deterministic split-K,
// polarizability C Omega^-1 C^T with on-the-fly pair operands, and a blocked
// in-place right triangular solve.
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace isdf {

thread_local bool tl_gemm_df = false;


static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

static std::atomic<long long> g_allocs{0};
cudaError_t dev_malloc(void** p, size_t bytes) {
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  return cudaMalloc(p, bytes);
}
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t s) {
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  return cudaMallocAsync(p, bytes, s);
}
long long device_allocation_count() { return g_allocs.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------- utilities

__global__ void k_check_finite(const double* __restrict__ p, long long n, unsigned* status) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  bool bad = false;
  for (; i < n; i += stride) bad |= !isfinite(p[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_NONFINITE);
}

cudaError_t launch_check_finite(const double* p, long long n, unsigned* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  note_launch();
  k_check_finite<<<(int)blocks, 256, 0, s>>>(p, n, status);
  return cudaGetLastError();
}

// dst(a, e) = src(idx[a], e)
__global__ void k_gather_rows(const double* __restrict__ src, long long lds, const int* __restrict__ idx,
                              int nrows, int ncols, double* __restrict__ dst, long long ldd) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  int e = blockIdx.y;
  if (a < nrows && e < ncols) dst[a + ldd * e] = src[(long long)idx[a] + lds * e];
}

cudaError_t launch_gather_rows(const double* src, long long lds, const int* idx, int nrows, int ncols,
                               double* dst, long long ldd, cudaStream_t s) {
  if (nrows <= 0 || ncols <= 0) return cudaSuccess;
  dim3 grid((nrows + 127) / 128, ncols);
  note_launch();
  k_gather_rows<<<grid, 128, 0, s>>>(src, lds, idx, nrows, ncols, dst, ldd);
  return cudaGetLastError();
}

__global__ void k_transpose(const double* __restrict__ src, long long lds, int M, int N,
                            double* __restrict__ dst, long long ldd) {
  __shared__ double t[32][33];
  int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int i = i0 + threadIdx.x, j = j0 + k;
    if (i < M && j < N) t[k][threadIdx.x] = src[i + lds * j];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int j = j0 + threadIdx.x, i = i0 + k;
    if (i < M && j < N) dst[j + ldd * i] = t[threadIdx.x][k];
  }
}

cudaError_t launch_transpose(const double* src, long long lds, int M, int N, double* dst,
                             long long ldd, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((M + 31) / 32, (N + 31) / 32), block(32, 8);
  note_launch();
  k_transpose<<<grid, block, 0, s>>>(src, lds, M, N, dst, ldd);
  return cudaGetLastError();
}

__global__ void k_symmetrize(double* A, long long lda, int n, long long sA = 0) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  A += sA * blockIdx.z;
  if (i < n && j < i) {
    double v = 0.5 * (A[i + lda * j] + A[j + lda * i]);
    A[i + lda * j] = v;
    A[j + lda * i] = v;
  }
}

cudaError_t launch_symmetrize(double* A, long long lda, int n, cudaStream_t s, int batch, long long sA) {
  if (n <= 1 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  dim3 grid((n + 127) / 128, n, batch);
  note_launch();
  k_symmetrize<<<grid, 128, 0, s>>>(A, lda, n, sA);
  return cudaGetLastError();
}

// out[z] = max_i sum_j |A_z(i, j)| (the Gershgorin bound of the spectrum of
// a symmetric A_z) in two passes with a fixed summation order, so the bound
// is the same on every run: pass 1 sums |A(i, j)| over one of RA_CHUNKS
// column chunks per block (a thread per row, loads coalesced down the
// columns, many blocks in flight where one thread per whole row would chain
// n dependent FP64 adds); pass 2 adds the chunks of each row in order and
// takes the maximum over the rows.
constexpr int RA_CHUNKS = 16;

__global__ void k_row_abs_partial(const double* __restrict__ A, long long lda, int n, double* __restrict__ part,
                                  long long sA) {
  A += sA * blockIdx.z;
  part += (size_t)RA_CHUNKS * n * blockIdx.z;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int len = (n + RA_CHUNKS - 1) / RA_CHUNKS, j0 = blockIdx.y * len, j1 = min(n, j0 + len);
  if (i >= n) return;
  double acc = 0.0;
  for (int j = j0; j < j1; ++j) acc += fabs(A[i + lda * (long long)j]);
  part[(size_t)blockIdx.y * n + i] = acc;
}

__global__ void k_row_abs_max(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double red[256];
  part += (size_t)RA_CHUNKS * n * blockIdx.x;
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < RA_CHUNKS; ++c) s += part[(size_t)c * n + i];
    m = fmax(m, s);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

size_t row_abs_sum_work(int n, int batch) { return (size_t)RA_CHUNKS * std::max(n, 0) * std::max(batch, 0); }

cudaError_t launch_row_abs_sum_max(const double* A, long long lda, int n, double* out, double* work, cudaStream_t s,
                                   int batch, long long sA) {
  if (batch < 1 || batch > 65535) return cudaErrorInvalidValue;
  if (n <= 0) return cudaMemsetAsync(out, 0, batch * sizeof(double), s);
  note_launch();
  k_row_abs_partial<<<dim3((n + 127) / 128, RA_CHUNKS, batch), 128, 0, s>>>(A, lda, n, work, sA);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launch();
  k_row_abs_max<<<batch, 256, 0, s>>>(work, n, out);
  return cudaGetLastError();
}

// X_z = alpha[z] I (n x n, ld n, matrix z at X + z n^2)
__global__ void k_scaled_identity(double* X, int n, const double* __restrict__ alpha) {
  const long long nn = (long long)n * n;
  double* x = X + nn * blockIdx.y;
  const double a = alpha[blockIdx.y];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x)
    x[i] = (i % (n + 1) == 0) ? a : 0.0;
}

cudaError_t launch_scaled_identity(double* X, int n, int batch, const double* alpha, cudaStream_t s) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  const long long nn = (long long)n * n;
  note_launch();
  k_scaled_identity<<<dim3((unsigned)std::min<long long>((nn + 255) / 256, 1024), batch), 256, 0, s>>>(X, n, alpha);
  return cudaGetLastError();
}

// c = a + b over n contiguous doubles (problem z at + z stride)
__global__ void k_add(const double* a, const double* b, double* c, long long n,
                      long long stride, long long stride_b) {
  a += stride * blockIdx.y;
  b += stride_b * blockIdx.y;
  c += stride * blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    c[i] = a[i] + b[i];
}

cudaError_t launch_add(const double* a, const double* b, double* c, long long n, cudaStream_t s, int batch,
                       long long stride, long long stride_b) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  const long long blocks = std::min<long long>((n + 255) / 256, 1024);
  note_launch();
  k_add<<<dim3((unsigned)blocks, batch), 256, 0, s>>>(a, b, c, n, stride, stride_b < 0 ? stride : stride_b);
  return cudaGetLastError();
}

__global__ void k_add_identity(double* A, long long lda, int n, double v, long long sA = 0) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  A += sA * blockIdx.y;
  if (i < n) A[i + lda * i] += v;
}

cudaError_t launch_add_identity(double* A, long long lda, int n, double v, cudaStream_t s, int batch, long long sA) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  note_launch();
  k_add_identity<<<dim3((n + 127) / 128, batch), 128, 0, s>>>(A, lda, n, v, sA);
  return cudaGetLastError();
}

// Pair weights of the polarizability, sqrt(-2 Omega(i w_k)^-1) with
// Omega(i w)^-1 = D / (D^2 + w^2), D = e_i - e_(n_v + j) < 0 (Eq. Hedin_fourier
// on the imaginary axis): sw[k npair + i n_c + j], and the same in FP32 in
// swf when it is given.  ew = [energies (n_v + n_c) | frequencies (n_omega)].
__global__ void k_pair_weights(const double* __restrict__ ew, int n_v, int n_c, int n_omega, double* __restrict__ sw,
                               float* __restrict__ swf) {
  const long long npair = (long long)n_v * n_c;
  const long long total = npair * n_omega;
  const double* om = ew + n_v + n_c;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(idx / npair);
    const long long p = idx - (long long)k * npair;
    const int i = (int)(p / n_c), j = (int)(p - (long long)i * n_c);
    const double d = ew[i] - ew[n_v + j];
    const double v = sqrt(-2.0 * d / (d * d + om[k] * om[k]));
    sw[idx] = v;
    if (swf) swf[idx] = __double2float_rn(v);
  }
}

cudaError_t launch_pair_weights(const double* ew, int n_v, int n_c, int n_omega, double* sw, float* swf,
                                cudaStream_t s) {
  const long long total = (long long)n_v * n_c * n_omega;
  if (total <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((total + 255) / 256, 4096);
  note_launch();
  k_pair_weights<<<(unsigned)blocks, 256, 0, s>>>(ew, n_v, n_c, n_omega, sw, swf);
  return cudaGetLastError();
}

// L(a, c) = Lr[perm[a] * n + c] for c <= a < rank, zero elsewhere in n_full x n_full.
__global__ void k_factor_to_colmajor(const double* __restrict__ Lr, int n, const int* __restrict__ perm,
                                     const int* __restrict__ rank_p, double* __restrict__ L,
                                     long long ldl, int n_full) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (a >= n_full || c >= n_full) return;
  int rank = min(*rank_p, n);  // a failed factorisation may leave rank stale: never trust it past n
  double v = 0.0;
  if (a < rank && c < rank && c <= a) {
    int pa = perm[a];
    if (pa >= 0 && pa < n) v = __ldcg(&Lr[(long long)pa * n + c]);
  }
  L[a + ldl * c] = v;
}

cudaError_t launch_factor_to_colmajor(const double* Lr, int n, const int* perm, const int* rank,
                                      double* L, long long ldl, int n_full, cudaStream_t s) {
  dim3 grid((n_full + 127) / 128, n_full);
  note_launch();
  k_factor_to_colmajor<<<grid, 128, 0, s>>>(Lr, n, perm, rank, L, ldl, n_full);
  return cudaGetLastError();
}

// ------------------------------------------------- face-split Gram (ISDF fit)
// C(m, n) = (sum_{k < n_v} A(m,k) B(n,k)) * (sum_{n_v <= k < n_e} A(m,k) B(n,k)):
// with A = Phi and B = Phi at the points this is M C^T (Hadamard identity,
// Eq. Hadamard), with A = B = Phi at the points it is C C^T.
// DF: both sums in double-float on the FP32 pipe (the DfGemm scope), about
// 2^-47 relative, for the points' C C^T of the mixed path.
template <bool DF>
__global__ void __launch_bounds__(256) k_facesplit_gram(Operand<false> A, Operand<false> B, int n_v,
                                                        int n_e, double* __restrict__ C,
                                                        long long ldc, int sym) {
  using T = TileSq;
  __shared__ typename std::conditional<DF, T::SmemDf, T::Smem>::type s;
  int mt = blockIdx.x, nt = blockIdx.y;
  if (sym) lower_tile(blockIdx.x, mt, nt);  // A == B: lower tiles, mirrored
  const int m0 = mt * T::kBM, n0 = nt * T::kBN;
  double av[T::kTM][T::kTN], ac[T::kTM][T::kTN];
  zero_acc<T>(av);
  zero_acc<T>(ac);
  if constexpr (DF) {
    gemm_mainloop_df<T>(av, s, A, B, m0, n0, 0, n_v);
    gemm_mainloop_df<T>(ac, s, A, B, m0, n0, n_v, n_e);
  } else {
    gemm_mainloop<T>(av, s, A, B, m0, n0, 0, n_v);
    gemm_mainloop<T>(ac, s, A, B, m0, n0, n_v, n_e);
  }
#pragma unroll
  for (int j = 0; j < T::kTN; ++j) {
    int n = tile_col<T>(n0, j);
    if (n >= B.rows) continue;
#pragma unroll
    for (int i = 0; i < T::kTM; ++i) {
      int m = tile_row<T>(m0, i);
      if (m < A.rows) {
        const double v = av[i][j] * ac[i][j];
        C[m + ldc * n] = v;
        if (sym && mt != nt) C[n + ldc * m] = v;
      }
    }
  }
}

cudaError_t launch_facesplit_gram(const double* A, long long lda, int M, const double* B,
                                  long long ldb, int N, int n_v, int n_e, double* C, long long ldc,
                                  cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const bool sym = (A == B && lda == ldb && M == N);
  const int tm = (M + 63) / 64;
  dim3 grid = sym ? dim3(tm * (tm + 1) / 2, 1) : dim3(tm, (N + 63) / 64);
  KernelTimer kt(tl_gemm_df ? KF_DF_GEMM : KF_FP64_GEMM, s, 2.0 * n_e * (sym ? 0.5 * M * (M + 1.0) : (double)M * N));
  note_launch();
  if (tl_gemm_df)
    k_facesplit_gram<true><<<grid, 256, 0, s>>>(Operand<false>{A, lda, M}, Operand<false>{B, ldb, N}, n_v, n_e, C,
                                                ldc, sym ? 1 : 0);
  else
    k_facesplit_gram<false><<<grid, 256, 0, s>>>(Operand<false>{A, lda, M}, Operand<false>{B, ldb, N}, n_v, n_e, C,
                                                 ldc, sym ? 1 : 0);
  return cudaGetLastError();
}

// ------------------------------------------------------------ generic GEMM

template <class T>
__device__ __forceinline__ void store_tile(const double (&acc)[T::kTM][T::kTN], int m0, int n0, int M,
                                           int N, double alpha, double beta, double* C, long long ldc,
                                           bool mirror) {
#pragma unroll
  for (int j = 0; j < T::kTN; ++j) {
    int n = tile_col<T>(n0, j);
    if (n >= N) continue;
#pragma unroll
    for (int i = 0; i < T::kTM; ++i) {
      int m = tile_row<T>(m0, i);
      if (m >= M) continue;
      double v = alpha * acc[i][j];
      if (beta != 0.0) v += beta * C[m + ldc * n];
      C[m + ldc * n] = v;
      if (mirror) C[n + ldc * m] = v;
    }
  }
}

template <class T, class OpA, class OpB, bool DF>
__global__ void __launch_bounds__(T::NT) k_gemm(OpA A, OpB B, int M, int N, int K, int klen,
                                                double alpha, double beta, double* C, long long ldc,
                                                double* partial, int lower_only, int tri) {
  __shared__ typename std::conditional<DF, typename T::SmemDf, typename T::Smem>::type s;
  int mt, nt;
  if (lower_only) {
    lower_tile(blockIdx.x, mt, nt);
  } else {
    mt = blockIdx.x;
    nt = blockIdx.y;
  }
  const int m0 = mt * T::kBM, n0 = nt * T::kBN;
  int kbeg = blockIdx.z * klen;
  int kend = min(K, kbeg + klen);
  // triangular factors: op(B)(n, k) = 0 for k < n (TRI_B_LOWER_T) or
  // op(A)(m, k) = 0 for k > m (TRI_A_LOWER): skip those k
  if (tri & TRI_B_LOWER_T) kbeg = max(kbeg, n0);
  if (tri & TRI_A_LOWER) kend = min(kend, m0 + T::kBM);
  double acc[T::kTM][T::kTN];
  zero_acc<T>(acc);
  if constexpr (DF) {
    gemm_mainloop_df<T>(acc, s, A, B, m0, n0, kbeg, kend);
  } else {
    gemm_mainloop<T>(acc, s, A, B, m0, n0, kbeg, kend);
  }
  if (partial) {
    double* P = partial + (long long)blockIdx.z * M * N;
    store_tile<T>(acc, m0, n0, M, N, 1.0, 0.0, P, M, false);
  } else {
    store_tile<T>(acc, m0, n0, M, N, alpha, beta, C, ldc, lower_only && mt != nt);
  }
}

// C = alpha * sum_z partial[z] + beta * C; for lower_only (the partials hold
// the lower tiles) the upper triangle is read mirrored from the lower one,
// so C comes out exactly symmetric.
// Batched over blockIdx.z: partials of problem z start at z * splits * M * N,
// its C at C + z * sC.
__global__ void k_splitk_reduce(const double* __restrict__ partial, int splits, int M, int N,
                                double alpha, double beta, double* C, long long ldc, int lower_only,
                                int tile, long long sC = 0) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  int n = blockIdx.y;
  if (m >= M || n >= N) return;
  partial += (long long)blockIdx.z * splits * M * N;
  C += sC * blockIdx.z;
  int pm = m, pn = n;
  if (lower_only && m < n) {  // the upper triangle mirrors the lower one: C exactly symmetric
    pm = n;
    pn = m;
  }
  double v = 0.0;
  for (int z = 0; z < splits; ++z) v += partial[(long long)z * M * N + pm + (long long)M * pn];
  v *= alpha;
  if (beta != 0.0) v += beta * C[m + ldc * n];
  C[m + ldc * n] = v;
}

template <class T, class OpA, class OpB, bool DF>
__global__ void __launch_bounds__(T::NT) k_gemm_batched(OpA A, OpB B, GemmBatch bt, int M, int N, int K, double alpha,
                                                        double beta, double* C, long long ldc, int tri, int lower) {
  __shared__ typename std::conditional<DF, typename T::SmemDf, typename T::Smem>::type s;
  const int z = blockIdx.z;
  const int z1 = z % bt.b1, z2 = z / bt.b1;
  A.p += bt.sA1 * z1 + bt.sA2 * z2;
  B.p += bt.sB1 * z1 + bt.sB2 * z2;
  C += bt.sC1 * z1 + bt.sC2 * z2;
  int mt, nt;
  if (lower) {
    lower_tile(blockIdx.x, mt, nt);
  } else {
    mt = blockIdx.x;
    nt = blockIdx.y;
  }
  const int m0 = mt * T::kBM, n0 = nt * T::kBN;
  const int kbeg = (tri & TRI_B_LOWER_T) ? min(n0, K) : 0;
  const int kend = (tri & TRI_A_LOWER) ? min(K, m0 + T::kBM) : K;
  double acc[T::kTM][T::kTN];
  zero_acc<T>(acc);
  if constexpr (DF) {
    gemm_mainloop_df<T>(acc, s, A, B, m0, n0, kbeg, kend);
  } else {
    gemm_mainloop<T>(acc, s, A, B, m0, n0, kbeg, kend);
  }
  store_tile<T>(acc, m0, n0, M, N, alpha, beta, C, ldc, lower && mt != nt);
}

// Multiply-adds of C(m, n) += sum_k A(m, k) B(n, k) over the (m, n, k) the
// method needs: lower triangle only for a SYRK, k >= n / k <= m under the
// triangular flags.
static double gemm_terms(int M, int N, int K, bool lower_only, int tri) {
  double t = 0.0;
  for (int m = 0; m < M; ++m) {
    const long long nmax = lower_only ? m : N - 1;
    const long long kmax = (tri & TRI_A_LOWER) ? (m + 1 < K ? m + 1 : K) : K;
    if (tri & TRI_B_LOWER_T) {
      const long long c = nmax + 1 < kmax ? nmax + 1 : kmax;
      t += (double)(c * kmax - c * (c - 1) / 2);
    } else {
      t += (double)(nmax + 1) * (double)kmax;
    }
  }
  return t;
}

template <class T, bool KA, bool KB>
static cudaError_t gemm_batched_dispatch(const double* A, long long lda, const double* B, long long ldb, int M, int N,
                                         int K, double alpha, double beta, double* C, long long ldc,
                                         const GemmBatch& bt, bool lower, int tri, cudaStream_t s) {
  const int tm = (M + T::kBM - 1) / T::kBM;
  const int nb = bt.b1 * bt.b2;
  dim3 grid = lower ? dim3(tm * (tm + 1) / 2, 1, nb) : dim3(tm, (N + T::kBN - 1) / T::kBN, nb);
  KernelTimer kt(tl_gemm_df ? KF_DF_GEMM : KF_FP64_GEMM, s, 2.0 * nb * gemm_terms(M, N, K, lower, tri));
  note_launch();
  if (tl_gemm_df) {
    k_gemm_batched<T, Operand<KA>, Operand<KB>, true><<<grid, T::NT, 0, s>>>(
        Operand<KA>{A, lda, M}, Operand<KB>{B, ldb, N}, bt, M, N, K, alpha, beta, C, ldc, tri, lower);
  } else {
    k_gemm_batched<T, Operand<KA>, Operand<KB>, false><<<grid, T::NT, 0, s>>>(
        Operand<KA>{A, lda, M}, Operand<KB>{B, ldb, N}, bt, M, N, K, alpha, beta, C, ldc, tri, lower);
  }
  return cudaGetLastError();
}

cudaError_t launch_gemm_batched2(const double* A, long long lda, bool ka, const double* B, long long ldb, bool kb,
                                 int M, int N, int K, double alpha, double beta, double* C, long long ldc,
                                 const GemmBatch& bt, bool lower, cudaStream_t s, int tri) {
  const long long nb = (long long)bt.b1 * bt.b2;
  if (M <= 0 || N <= 0 || nb <= 0) return cudaSuccess;
  if (nb > 65535 || (lower && M != N)) return cudaErrorInvalidValue;
  const long long t64 = (long long)((M + 63) / 64) * ((N + 63) / 64) * nb / (lower ? 2 : 1);
  const bool small = t64 < 2 * 152;
#define ISDF_BGEMM_CASE(TT, a, b) \
  if (ka == a && kb == b) return gemm_batched_dispatch<TT, a, b>(A, lda, B, ldb, M, N, K, alpha, beta, C, ldc, bt, lower, tri, s);
  if (small) {
    ISDF_BGEMM_CASE(TileSm, false, false)
    ISDF_BGEMM_CASE(TileSm, false, true)
    ISDF_BGEMM_CASE(TileSm, true, false)
    ISDF_BGEMM_CASE(TileSm, true, true)
  } else {
    ISDF_BGEMM_CASE(TileSq, false, false)
    ISDF_BGEMM_CASE(TileSq, false, true)
    ISDF_BGEMM_CASE(TileSq, true, false)
    ISDF_BGEMM_CASE(TileSq, true, true)
  }
#undef ISDF_BGEMM_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_gemm_batched(const double* A, long long lda, bool ka, long long sA, const double* B,
                                long long ldb, bool kb, long long sB, int M, int N, int K, double alpha, double beta,
                                double* C, long long ldc, long long sC, int batch, cudaStream_t s, int tri) {
  GemmBatch bt{batch, 1, sA, sB, sC, 0, 0, 0};
  return launch_gemm_batched2(A, lda, ka, B, ldb, kb, M, N, K, alpha, beta, C, ldc, bt, false, s, tri);
}

cudaError_t launch_splitk_reduce(const double* partial, int splits, int M, int N, double alpha, double beta,
                                 double* C, long long ldc, bool lower_only, int tile, cudaStream_t s, int batch,
                                 long long sC) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  dim3 rg((M + 127) / 128, N, batch);
  note_launch();
  k_splitk_reduce<<<rg, 128, 0, s>>>(partial, splits, M, N, alpha, beta, C, ldc, lower_only ? 1 : 0, tile, sC);
  return cudaGetLastError();
}

template <class T, bool KA, bool KB>
static cudaError_t gemm_dispatch(const double* A, long long lda, const double* B, long long ldb, int M,
                                 int N, int K, double alpha, double beta, double* C, long long ldc,
                                 bool lower_only, int splits, double* partial, int tri, cudaStream_t s) {
  Operand<KA> oa{A, lda, M};
  Operand<KB> ob{B, ldb, N};
  int tm = (M + T::kBM - 1) / T::kBM, tn = (N + T::kBN - 1) / T::kBN;
  if (splits < 1) splits = 1;
  int klen = (K + splits - 1) / splits;
  klen = ((klen + GT_BK - 1) / GT_BK) * GT_BK;
  splits = (K + klen - 1) / klen;
  if (splits < 1) splits = 1;
  bool use_partial = splits > 1;
  dim3 grid;
  if (lower_only) {
    grid = dim3(tm * (tm + 1) / 2, 1, splits);
  } else {
    grid = dim3(tm, tn, splits);
  }
  cudaError_t e;
  {
    KernelTimer kt(tl_gemm_df ? KF_DF_GEMM : KF_FP64_GEMM, s, 2.0 * gemm_terms(M, N, K, lower_only, tri));
    note_launch();
    if (tl_gemm_df) {
      k_gemm<T, Operand<KA>, Operand<KB>, true><<<grid, T::NT, 0, s>>>(oa, ob, M, N, K, klen, alpha, beta, C, ldc,
                                                                      use_partial ? partial : nullptr,
                                                                      lower_only ? 1 : 0, tri);
    } else {
      k_gemm<T, Operand<KA>, Operand<KB>, false><<<grid, T::NT, 0, s>>>(oa, ob, M, N, K, klen, alpha, beta, C, ldc,
                                                                       use_partial ? partial : nullptr,
                                                                       lower_only ? 1 : 0, tri);
    }
    e = cudaGetLastError();
  }
  if (e != cudaSuccess || !use_partial) return e;
  dim3 rg((M + 127) / 128, N);
  note_launch();
  k_splitk_reduce<<<rg, 128, 0, s>>>(partial, splits, M, N, alpha, beta, C, ldc, lower_only ? 1 : 0,
                                     T::kBM);
  return cudaGetLastError();
}

cudaError_t launch_gemm(const double* A, long long lda, bool ka, const double* B, long long ldb,
                        bool kb, int M, int N, int K, double alpha, double beta, double* C,
                        long long ldc, bool lower_only, int splits, double* partial, bool narrow,
                        cudaStream_t s, int tri) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (splits > 1 && !partial) return cudaErrorInvalidValue;
  if (lower_only && (M != N || narrow)) return cudaErrorInvalidValue;
#define ISDF_GEMM_CASE(TT, a, b)                                                                 \
  if (ka == a && kb == b)                                                                        \
    return gemm_dispatch<TT, a, b>(A, lda, B, ldb, M, N, K, alpha, beta, C, ldc, lower_only,     \
                                   splits, partial, tri, s);
  // too few 64 x 64 tiles to fill the GPU twice: use 32 x 32 tiles (4x the blocks)
  const long long t64 = lower_only ? (long long)((M + 63) / 64) * ((M + 63) / 64 + 1) / 2
                                   : (long long)((M + 63) / 64) * ((N + 63) / 64);
  if (!narrow && t64 * (splits > 1 ? splits : 1) < 2 * 152) {
    ISDF_GEMM_CASE(TileSm, false, false)
    ISDF_GEMM_CASE(TileSm, false, true)
    ISDF_GEMM_CASE(TileSm, true, false)
    ISDF_GEMM_CASE(TileSm, true, true)
  }
  if (narrow) {
    ISDF_GEMM_CASE(TileNarrow, false, false)
    ISDF_GEMM_CASE(TileNarrow, false, true)
    ISDF_GEMM_CASE(TileNarrow, true, false)
    ISDF_GEMM_CASE(TileNarrow, true, true)
  } else {
    ISDF_GEMM_CASE(TileSq, false, false)
    ISDF_GEMM_CASE(TileSq, false, true)
    ISDF_GEMM_CASE(TileSq, true, false)
    ISDF_GEMM_CASE(TileSq, true, true)
  }
#undef ISDF_GEMM_CASE
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ polarizability
// S(a, ij) = phimu(a, i) phimu(a, n_v + j) sw[i n_c + j]: the columns of the
// pair matrix at the points (C of Eq. MatrixExpressionISDF) scaled by
// sqrt(-2 Omega^-1), generated on the fly so C (N_mu x N_v N_c) is never
// stored.  D = S S^T = -2 C Omega^-1 C^T.
struct PairOperand {
  static constexpr bool kcontig = false;
  const double* p;  // phimu, column-major r x n_e
  long long ld;
  int rows;
  int n_v, n_c;
  const double* sw;
  __device__ __forceinline__ double get(int a, int kk) const {
    int i = kk / n_c;
    int j = kk - i * n_c;
    return p[a + ld * i] * p[a + ld * (long long)(n_v + j)] * sw[kk];
  }
};

__global__ void __launch_bounds__(256) k_polarizability(PairOperand S, int K, int klen,
                                                        double* __restrict__ D, long long ldd,
                                                        double* partial) {
  using T = TileSq;
  __shared__ T::Smem s;
  int mt, nt;
  lower_tile(blockIdx.x, mt, nt);
  const int m0 = mt * T::kBM, n0 = nt * T::kBN;
  const int kbeg = blockIdx.z * klen, kend = min(K, kbeg + klen);
  double acc[T::kTM][T::kTN];
  zero_acc<T>(acc);
  gemm_mainloop<T>(acc, s, S, S, m0, n0, kbeg, kend);
  if (partial) {
    store_tile<T>(acc, m0, n0, S.rows, S.rows, 1.0, 0.0, partial + (long long)blockIdx.z * S.rows * S.rows,
                  S.rows, false);
  } else {
    store_tile<T>(acc, m0, n0, S.rows, S.rows, 1.0, 0.0, D, ldd, mt != nt);
  }
}

cudaError_t launch_polarizability(const double* phimu, long long ldp, int r, int n_v, int n_c,
                                  const double* sw, double* D, long long ldd, int splits,
                                  double* partial, cudaStream_t s) {
  if (r <= 0) return cudaSuccess;
  PairOperand S{phimu, ldp, r, n_v, n_c, sw};
  int K = n_v * n_c;
  if (splits < 1 || !partial) splits = 1;
  int klen = (K + splits - 1) / splits;
  klen = ((klen + GT_BK - 1) / GT_BK) * GT_BK;
  splits = (K + klen - 1) / klen;
  int tm = (r + 63) / 64;
  dim3 grid(tm * (tm + 1) / 2, 1, splits);
  cudaError_t e;
  {
    KernelTimer kt(KF_FP64_GEMM, s, (double)r * (r + 1) * K);
    note_launch();
    k_polarizability<<<grid, 256, 0, s>>>(S, K, klen, D, ldd, splits > 1 ? partial : nullptr);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess || splits == 1) return e;
  dim3 rg((r + 127) / 128, r);
  note_launch();
  k_splitk_reduce<<<rg, 128, 0, s>>>(partial, splits, r, r, 1.0, 0.0, D, ldd, 1, 64);
  return cudaGetLastError();
}

// ------------------------------------------------------------ triangular solve
constexpr int TRSM_NB = 64;

// sum of squares of n doubles: per-block partials, then one block sums them
// in a fixed order (deterministic)
__global__ void k_sumsq_partial(const double* __restrict__ a, long long n, double* __restrict__ part) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc = fma(a[i], a[i], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_fixed(const double* __restrict__ part, int n, double* out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

cudaError_t launch_sumsq(const double* a, long long n, double* scratch, double* out, cudaStream_t s) {
  note_launch();
  k_sumsq_partial<<<256, 256, 0, s>>>(a, n, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launch();
  k_sum_fixed<<<1, 256, 0, s>>>(scratch, 256, out);
  return cudaGetLastError();
}

// Zero an r x r block per problem (problem blockIdx.z at A + z sA).
__global__ void k_copy_zero(double* A, long long lda, long long sA, int r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i < r) A[sA * blockIdx.z + i + lda * (long long)j] = 0.0;
}

// Inverse of each 64 x 64 diagonal block of the lower-triangular L, written
// into the diagonal blocks of Bf (lower part; the strict upper part is 0).
// Forward substitution L X = I row by row, with the sums kept as running
// updates: row k of X is (e_k - acc_k) / L_kk, then every later row i adds
// L_ik X_k to its acc_i.  Row k costs one FP64 instruction on the chain and
// its update is spread over all threads (an FP64 instruction holds a warp's
// sub-partition for ~64 cycles whatever its active lanes, so one thread per
// column running its own substitution, as before, was ~7 times slower).
constexpr int DINV_THREADS = 256;
__global__ void __launch_bounds__(DINV_THREADS) k_diag_inverse(const double* __restrict__ L, long long ldl, int r,
                                                              double* __restrict__ Bf, long long ldb, long long sL = 0,
                                                              long long sB = 0) {
  __shared__ double Ls[TRSM_NB][TRSM_NB + 1];
  __shared__ double Xs[TRSM_NB][TRSM_NB + 1];  // acc, then X, row by row
  __shared__ double rinv[TRSM_NB];
  L += sL * blockIdx.y;  // matrix blockIdx.y of a batch
  Bf += sB * blockIdx.y;
  const int j0 = blockIdx.x * TRSM_NB;
  const int bs = min(TRSM_NB, r - j0);
  const int t = threadIdx.x;
  for (int idx = t; idx < TRSM_NB * TRSM_NB; idx += DINV_THREADS) {
    const int i = idx % TRSM_NB, c = idx / TRSM_NB;
    Ls[i][c] = (i < bs && c <= i) ? L[(j0 + i) + ldl * (long long)(j0 + c)] : 0.0;
    Xs[i][c] = 0.0;
  }
  __syncthreads();
  if (t < bs) rinv[t] = recip_newton(Ls[t][t]);
  __syncthreads();
  for (int k = 0; k < bs; ++k) {
    if (t <= k) Xs[k][t] = fma(-Xs[k][t], rinv[k], t == k ? rinv[k] : 0.0);
    __syncthreads();
    const int cols = k + 1, cnt = (bs - 1 - k) * cols;
    for (int idx = t; idx < cnt; idx += DINV_THREADS) {
      const int i = k + 1 + idx / cols, c = idx - (idx / cols) * cols;
      Xs[i][c] = fma(Ls[i][k], Xs[k][c], Xs[i][c]);
    }
    __syncthreads();
  }
  for (int idx = t; idx < bs * bs; idx += DINV_THREADS) {
    const int i = idx % bs, c = idx / bs;
    Bf[(j0 + i) + ldb * (long long)(j0 + c)] = (c <= i) ? Xs[i][c] : 0.0;
  }
}

// Bf[J, I] = -L_JJ^-1 L_JI for I < J (64 x 64 blocks), the diagonal
// inverses already in Bf.
__global__ void __launch_bounds__(256) k_trsm_offdiag(const double* __restrict__ L, long long ldl, int r,
                                                      double* __restrict__ Bf, long long ldb) {
  using T = TileSq;
  __shared__ T::Smem s;
  const int J = blockIdx.y + 1;
  const int It = blockIdx.x;
  if (It >= J) return;
  const int j0 = J * TRSM_NB;
  const int bs = min(TRSM_NB, r - j0);
  // A(m, k) = Dinv_J(m, k) = Bf[j0 + m, j0 + k]; B(n, k) = L[j0 + k, n] (n < j0)
  Operand<false> A{Bf + j0 + ldb * (long long)j0, ldb, bs};
  Operand<true> B{L + j0, ldl, j0};
  double acc[T::kTM][T::kTN];
  zero_acc<T>(acc);
  gemm_mainloop<T>(acc, s, A, B, 0, It * T::kBN, 0, bs);
#pragma unroll
  for (int j = 0; j < T::kTN; ++j) {
    int n = tile_col<T>(It * T::kBN, j);
    if (n >= j0) continue;
#pragma unroll
    for (int i = 0; i < T::kTM; ++i) {
      int m = tile_row<T>(0, i);
      if (m < bs) Bf[(j0 + m) + ldb * n] = -acc[i][j];
    }
  }
}

cudaError_t launch_diag_inverse_block(const double* L, long long ldl, int bs, double* Li, long long ldi,
                                      cudaStream_t s) {
  if (bs <= 0) return cudaSuccess;
  if (bs > TRSM_NB) return cudaErrorInvalidValue;
  note_launch();
  k_diag_inverse<<<1, DINV_THREADS, 0, s>>>(L, ldl, bs, Li, ldi);
  return cudaGetLastError();
}

cudaError_t launch_trsm_prep(const double* L, long long ldl, int r, double* Bf, long long ldb,
                             cudaStream_t s) {
  if (r <= 0) return cudaSuccess;
  int nb = (r + TRSM_NB - 1) / TRSM_NB;
  note_launch();
  k_diag_inverse<<<nb, DINV_THREADS, 0, s>>>(L, ldl, r, Bf, ldb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nb == 1) return e;
  dim3 grid(nb - 1, nb - 1);
  note_launch();
  k_trsm_offdiag<<<grid, 256, 0, s>>>(L, ldl, r, Bf, ldb);
  return cudaGetLastError();
}

// One block column of X <- X L^-T: X[:, J] = X[:, 0 : j0 + bs] Bf[J, 0 : j0 + bs]^T.
// Columns < j0 are already solved; columns J still hold the right-hand side.
// Each thread block owns 64 full rows of the block column, and reads all of
// them before it writes, so the update is safe in place.
__global__ void __launch_bounds__(256) k_trsm_step(double* X, long long ldx, int M,
                                                   const double* __restrict__ Bf, long long ldb, int j0,
                                                   int bs) {
  using T = TileSq;
  __shared__ T::Smem s;
  const int m0 = blockIdx.x * T::kBM;
  Operand<false> A{X, ldx, M};
  Operand<false> B{Bf + j0, ldb, bs};
  double acc[T::kTM][T::kTN];
  zero_acc<T>(acc);
  gemm_mainloop<T>(acc, s, A, B, m0, 0, 0, j0 + bs);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < T::kTN; ++j) {
    int n = tile_col<T>(0, j);
    if (n >= bs) continue;
#pragma unroll
    for (int i = 0; i < T::kTM; ++i) {
      int m = tile_row<T>(m0, i);
      if (m < M) X[m + ldx * (long long)(j0 + n)] = acc[i][j];
    }
  }
}

cudaError_t launch_trsm_right_lt(double* X, long long ldx, int M, const double* Bf, long long ldb,
                                 int r, cudaStream_t s) {
  if (M <= 0 || r <= 0) return cudaSuccess;
  for (int j0 = 0; j0 < r; j0 += TRSM_NB) {
    int bs = min(TRSM_NB, r - j0);
    KernelTimer kt(KF_FP64_GEMM, s, (double)M * bs * (2.0 * j0 + bs));
    note_launch();
    k_trsm_step<<<(M + 63) / 64, 256, 0, s>>>(X, ldx, M, Bf, ldb, j0, bs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace isdf

namespace isdf {

// Inverse of a lower-triangular r x r matrix L, in FP64: the 64 x 64
// diagonal blocks are inverted directly (k_diag_inverse), then blocks are
// merged pairwise, [[A, 0], [C, B]]^-1 = [[A^-1, 0], [-B^-1 C A^-1, B^-1]],
// for block sizes 64, 128, 256, ... (two GEMMs per merge, all merges of one
// level independent).  work: (r/2 + 64)^2 doubles.
cudaError_t launch_tri_inverse(const double* L, long long ldl, int r, double* Li, long long ldi, double* work,
                               double* partial, cudaStream_t s) {
  if (r <= 0) return cudaSuccess;
  cudaError_t e = cudaMemset2DAsync(Li, ldi * sizeof(double), 0, r * sizeof(double), r, s);
  if (e != cudaSuccess) return e;
  int nb = (r + TRSM_NB - 1) / TRSM_NB;
  note_launch();
  k_diag_inverse<<<nb, DINV_THREADS, 0, s>>>(L, ldl, r, Li, ldi);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int bs = TRSM_NB; bs < r; bs *= 2) {
    // merges of this level with a full-size lower block, batched
    const int full = r / (2 * bs);
    if (full > 0) {
      const long long sL = 2ll * bs * (1 + ldl), sI = 2ll * bs * (1 + ldi), sW = (long long)bs * bs;
      // X_z (bs x bs) = C_z A_z^-1 (A_z^-1 lower: k >= n)
      e = launch_gemm_batched(L + bs, ldl, false, sL, Li, ldi, true, sI, bs, bs, bs, 1.0, 0.0, work, bs, sW, full, s,
                              TRI_B_LOWER_T);
      if (e != cudaSuccess) return e;
      // Li[B_z, A_z] = -B_z^-1 X_z (B_z^-1 lower: k <= m)
      e = launch_gemm_batched(Li + bs + ldi * (long long)bs, ldi, false, sI, work, bs, true, sW, bs, bs, bs, -1.0,
                              0.0, Li + bs, ldi, sI, full, s, TRI_A_LOWER);
      if (e != cudaSuccess) return e;
    }
    // a ragged last merge (lower block shorter than bs)
    const int b = full * 2 * bs;
    if (b + bs < r) {
      const int sa = bs, sb = r - (b + bs);
      const int sp = partial ? 4 : 1;
      e = launch_gemm(L + (b + bs) + ldl * (long long)b, ldl, false, Li + b + ldi * (long long)b, ldi, true, sb,
                      sa, sa, 1.0, 0.0, work, sb, false, sp, partial, false, s, TRI_B_LOWER_T);
      if (e != cudaSuccess) return e;
      e = launch_gemm(Li + (b + bs) + ldi * (long long)(b + bs), ldi, false, work, sb, true, sb, sa, sb, -1.0, 0.0,
                      Li + (b + bs) + ldi * (long long)b, ldi, false, sp, partial, false, s, TRI_A_LOWER);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// Li_z = L_z^-1 for batch lower-triangular matrices L + z sL -> Li + z sI;
// work: batch * (r/2 + 64)^2 doubles.
cudaError_t launch_tri_inverse_batched(const double* L, long long ldl, long long sL, int r, int batch, double* Li,
                                       long long ldi, long long sI, double* work, cudaStream_t s) {
  if (r <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  const long long wq = (long long)(r / 2 + 64) * (r / 2 + 64);
  note_launch();
  k_copy_zero<<<dim3((r + 127) / 128, r, batch), 128, 0, s>>>(Li, ldi, sI, r);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nb = (r + TRSM_NB - 1) / TRSM_NB;
  note_launch();
  k_diag_inverse<<<dim3(nb, batch), DINV_THREADS, 0, s>>>(L, ldl, r, Li, ldi, sL, sI);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int bs = TRSM_NB; bs < r; bs *= 2) {
    const int full = r / (2 * bs);
    if (full > 0) {
      const long long sL1 = 2ll * bs * (1 + ldl), sI1 = 2ll * bs * (1 + ldi), sW1 = (long long)bs * bs;
      GemmBatch b1{full, batch, sL1, sI1, sW1, sL, sI, wq};
      e = launch_gemm_batched2(L + bs, ldl, false, Li, ldi, true, bs, bs, bs, 1.0, 0.0, work, bs, b1, false, s,
                               TRI_B_LOWER_T);
      if (e != cudaSuccess) return e;
      GemmBatch b2{full, batch, sI1, sW1, sI1, sI, wq, sI};
      e = launch_gemm_batched2(Li + bs + ldi * (long long)bs, ldi, false, work, bs, true, bs, bs, bs, -1.0, 0.0,
                               Li + bs, ldi, b2, false, s, TRI_A_LOWER);
      if (e != cudaSuccess) return e;
    }
    const int b = full * 2 * bs;
    if (b + bs < r) {
      const int sa = bs, sb = r - (b + bs);
      GemmBatch b1{batch, 1, sL, sI, wq, 0, 0, 0};
      e = launch_gemm_batched2(L + (b + bs) + ldl * (long long)b, ldl, false, Li + b + ldi * (long long)b, ldi, true,
                               sb, sa, sa, 1.0, 0.0, work, sb, b1, false, s, TRI_B_LOWER_T);
      if (e != cudaSuccess) return e;
      GemmBatch b2{batch, 1, sI, wq, sI, 0, 0, 0};
      e = launch_gemm_batched2(Li + (b + bs) + ldi * (long long)(b + bs), ldi, false, work, sb, true, sb, sa, sb,
                               -1.0, 0.0, Li + (b + bs) + ldi * (long long)b, ldi, b2, false, s, TRI_A_LOWER);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace isdf
