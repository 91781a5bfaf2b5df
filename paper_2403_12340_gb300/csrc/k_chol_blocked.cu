// Blocked right-looking Cholesky (no pivoting), FP64.
//
// For J = 0, 1, ...: the 64 x 64 diagonal block is factored in shared memory
// by one thread block; the panel below is solved in place by forward
// substitution, one warp per row over every SM; the trailing matrix gets a
// lower SYRK update, which carries nearly all of the O(n^3) work.
//
// A pivot at or below tol_rel * max(diag) stops the factorisation: the
// first failing column goes to *fail and every later kernel of the sequence
// does nothing.  The caller decides what that means (not positive definite,
// or: fall back to the pivoted factorisation for a rank-deficient C C^T).
#include "common.cuh"
#include "kernels.h"

namespace isdf {

constexpr int CB = 64;

__global__ void k_diag_max(const double* __restrict__ W, long long ldw, int n, double* out, int* fail,
                           long long sW = 0) {
  __shared__ double red[256];
  W += sW * blockIdx.x;
  out += blockIdx.x;
  fail += blockIdx.x;
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, W[i + ldw * (long long)i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out = red[0];
    *fail = -1;
  }
}

// Factor A[j0:j0+bs, j0:j0+bs] (lower part, already updated) in place; the
// strict upper part of the block is zeroed.  One thread block on one SM.
// The block is factored 8 columns at a time, so that the 64 dependent
// column steps cost 3 block barriers per 8 columns instead of one or two
// per column (barriers dominated the column-by-column version):
//   A: warp 0 factors the 8 x 8 diagonal sub-block warp-synchronously (lane i
//      holds row i; the reciprocal square root of each pivot from an FP32
//      estimate refined by two Newton steps y <- y (3 - d y^2) / 2);
//   B: the rows below solve against it (one thread per row and column of
//      the panel, forward substitution over the 8 columns);
//   C: every thread applies the rank-8 update to its share of the remaining
//      lower triangle.
// An FP64 warp instruction costs the FP64 pipe the same with one lane or
// 32, so no step runs FP64 on a single lane of many warps.
constexpr int SUB = 8;

__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);  // outside the FP32 range of the first estimate
  double y = (double)rsqrtf((float)d);
  y = y * fma(-0.5 * d * y, y, 1.5);
  return y * fma(-0.5 * d * y, y, 1.5);
}

constexpr int DIAG_THREADS = 512;

__global__ void __launch_bounds__(DIAG_THREADS) k_chol_diag(double* A, long long lda, int j0, int bs,
                                                           const double* dmax, double tol_rel, int* fail,
                                                           long long sA = 0) {
  __shared__ double Ls[CB][CB + 1];
  __shared__ double ysub[SUB];  // 1 / L(c, c) of the current sub-block
  __shared__ int s_bad;
  // problem blockIdx.x of a batch: its matrix, max and flag
  A += sA * blockIdx.x;
  dmax += blockIdx.x;
  fail += blockIdx.x;
  if (*(volatile int*)fail >= 0) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int idx = t; idx < CB * CB; idx += blockDim.x) {
    int i = idx & (CB - 1), k = idx >> 6;
    Ls[i][k] = (i < bs && k <= i) ? A[(j0 + i) + lda * (long long)(j0 + k)] : 0.0;
  }
  if (t == 0) s_bad = -1;
  const double thresh = tol_rel * (*dmax);
  __syncthreads();
  for (int jb = 0; jb < bs; jb += SUB) {
    const int w = min(SUB, bs - jb);
    // A: the w x w diagonal sub-block, warp 0, lane i <-> row jb + i
    if (warp == 0) {
      for (int c = 0; c < w; ++c) {
        __syncwarp();
        const double d = Ls[jb + c][jb + c];
        if (!(d > thresh)) {  // the same value in every lane; also catches NaN
          if (lane == 0) s_bad = jb + c;
          break;
        }
        const double y = rsqrt_newton(d);
        __syncwarp();
        if (lane == c) {
          Ls[jb + c][jb + c] = d * y;
          ysub[c] = y;
        }
        if (lane > c && lane < w) Ls[jb + lane][jb + c] *= y;
        __syncwarp();
        if (lane > c && lane < w) {
          const double lic = Ls[jb + lane][jb + c];
          for (int k = c + 1; k <= lane; ++k) Ls[jb + lane][jb + k] = fma(-lic, Ls[jb + k][jb + c], Ls[jb + lane][jb + k]);
        }
      }
    }
    __syncthreads();
    if (s_bad >= 0) break;
    const int r0 = jb + w, m = bs - r0;  // rows below the sub-block
    // B: panel rows r0.. against the sub-block: x (L_sub)^T = a, row by row
    for (int i = t; i < m; i += blockDim.x) {
      double x[SUB];
#pragma unroll
      for (int c = 0; c < SUB; ++c) {
        if (c < w) {
          double sacc = Ls[r0 + i][jb + c];
#pragma unroll
          for (int k = 0; k < SUB; ++k)
            if (k < c) sacc = fma(-x[k], Ls[jb + c][jb + k], sacc);
          x[c] = sacc * ysub[c];
          Ls[r0 + i][jb + c] = x[c];
        }
      }
    }
    __syncthreads();
    // C: rank-w update of the lower triangle of rows / columns r0..bs
    const int cnt = m * (m + 1) / 2;
    for (int idx = t; idx < cnt; idx += blockDim.x) {
      int a = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
      while ((a + 1) * (a + 2) / 2 <= idx) ++a;
      while (a * (a + 1) / 2 > idx) --a;
      const int b = idx - a * (a + 1) / 2;
      const int i = r0 + a, k = r0 + b;
      double v = Ls[i][k];
#pragma unroll
      for (int c = 0; c < SUB; ++c)
        if (c < w) v = fma(-Ls[i][jb + c], Ls[k][jb + c], v);
      Ls[i][k] = v;
    }
    __syncthreads();
  }
  if (s_bad >= 0) {
    if (t == 0) atomicCAS(fail, -1, j0 + s_bad);
    return;
  }
  for (int idx = t; idx < bs * bs; idx += blockDim.x) {
    const int i = idx % bs, k = idx / bs;
    A[(j0 + i) + lda * (long long)(j0 + k)] = (k <= i) ? Ls[i][k] : 0.0;
  }
}

// The panel below a factored diagonal block, A21 <- A21 L_jj^-T, in place:
// one warp per row, lane l holding columns l and l + 32 of the row; forward
// substitution by columns, each solved value broadcast by a shuffle.  Rows
// are independent, so every SM takes part however short the panel is.
__global__ void __launch_bounds__(256) k_panel_trsm(double* A, long long lda, int j0, int bs, int rem,
                                                   const int* fail, long long sA = 0) {
  __shared__ double Lt[CB][CB + 1];  // Lt[c][k] = L_jj(c, k), zero outside the lower triangle
  __shared__ double inv[CB];
  A += sA * blockIdx.y;  // problem blockIdx.y of a batch
  if (*(volatile const int*)(fail + blockIdx.y) >= 0) return;
  const int t = threadIdx.x;
  for (int idx = t; idx < CB * CB; idx += blockDim.x) {
    const int i = idx & (CB - 1), k = idx >> 6;
    Lt[i][k] = (i < bs && k <= i) ? A[(j0 + i) + lda * (long long)(j0 + k)] : 0.0;
  }
  __syncthreads();
  if (t < bs) inv[t] = 1.0 / Lt[t][t];
  __syncthreads();
  const int warp = t >> 5, lane = t & 31;
  for (int row = blockIdx.x * 8 + warp; row < rem; row += gridDim.x * 8) {
    double* a = A + (j0 + bs + row) + lda * (long long)j0;
    double x0 = lane < bs ? a[lda * lane] : 0.0;
    double x1 = lane + 32 < bs ? a[lda * (lane + 32)] : 0.0;
    for (int k = 0; k < bs; ++k) {
      double xk;
      if (k < 32) {
        if (lane == k) x0 *= inv[k];
        xk = __shfl_sync(0xffffffffu, x0, k);
      } else {
        if (lane == k - 32) x1 *= inv[k];
        xk = __shfl_sync(0xffffffffu, x1, k - 32);
      }
      if (lane > k) x0 = fma(-xk, Lt[lane][k], x0);
      if (lane + 32 > k) x1 = fma(-xk, Lt[lane + 32][k], x1);
    }
    if (lane < bs) a[lda * lane] = x0;
    if (lane + 32 < bs) a[lda * (lane + 32)] = x1;
  }
}

// Zero the strict upper triangle (matrix blockIdx.z at A + z sA).
__global__ void k_zero_upper(double* A, long long lda, int n, long long sA = 0) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  A += sA * blockIdx.z;
  if (i < k && k < n) A[i + lda * (long long)k] = 0.0;
}

// dst(i, j) = src(i, j) for i < rows, j < cols; problem blockIdx.z at
// dst + z sD, src + z sS
__global__ void k_copy_block(const double* __restrict__ src, long long lds, long long sS, double* __restrict__ dst,
                             long long ldd, long long sD, int rows, int cols) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i < rows && j < cols) dst[sD * blockIdx.z + i + ldd * j] = src[sS * blockIdx.z + i + lds * j];
}

static unsigned panel_blocks(int rem) {
  const int b = (rem + 7) / 8;
  return (unsigned)(b < 4 * 152 ? b : 4 * 152);
}

cudaError_t launch_cholesky_blocked(const double* W, long long ldw, int n, double tol_rel, double* L, long long ldl,
                                    double* dmax, int* fail, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e;
  if (L != W) {
    e = cudaMemcpy2DAsync(L, ldl * sizeof(double), W, ldw * sizeof(double), n * sizeof(double), n,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  note_launch();
  k_diag_max<<<1, 256, 0, s>>>(L, ldl, n, dmax, fail);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int j0 = 0; j0 < n; j0 += CB) {
    const int bs = min(CB, n - j0);
    {
      KernelTimer kt(KF_CHOL_DIAG, s, bs * (double)bs * bs / 3.0);  // bs^3 / 3 flops
      note_launch();
      k_chol_diag<<<1, DIAG_THREADS, 0, s>>>(L, ldl, j0, bs, dmax, tol_rel, fail);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int rem = n - j0 - bs;
    if (rem <= 0) break;
    {
      KernelTimer kt(KF_FP64_GEMM, s, (double)rem * bs * bs);  // triangular solve, rem bs^2 flops
      note_launch();
      k_panel_trsm<<<panel_blocks(rem), 256, 0, s>>>(L, ldl, j0, bs, rem, fail);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // trailing: A[j0+bs:, j0+bs:] -= L_panel L_panel^T (lower tiles, mirrored)
    double* Pj = L + (j0 + bs) + ldl * (long long)j0;
    e = launch_gemm(Pj, ldl, false, Pj, ldl, false, rem, rem, bs, -1.0, 1.0, L + (j0 + bs) + ldl * (long long)(j0 + bs),
                    ldl, true, 1, nullptr, false, s);
    if (e != cudaSuccess) return e;
  }
  dim3 g((n + 127) / 128, n);
  note_launch();
  k_zero_upper<<<g, 128, 0, s>>>(L, ldl, n);
  return cudaGetLastError();
}

// The same factorisation for `batch` matrices of equal size n (W_z = W + z
// sW, L_z = L + z sL): one launch per step covers every matrix.  dmax and
// fail: batch entries.
cudaError_t launch_cholesky_blocked_batched(const double* W, long long ldw, long long sW, int n, int batch,
                                            double tol_rel, double* L, long long ldl, long long sL, double* dmax,
                                            int* fail, cudaStream_t s) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  cudaError_t e;
  if (L != W || ldl != ldw || sL != sW) {
    note_launch();
    k_copy_block<<<dim3((n + 127) / 128, n, batch), 128, 0, s>>>(W, ldw, sW, L, ldl, sL, n, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  note_launch();
  k_diag_max<<<batch, 256, 0, s>>>(L, ldl, n, dmax, fail, sL);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int j0 = 0; j0 < n; j0 += CB) {
    const int bs = min(CB, n - j0);
    {
      KernelTimer kt(KF_CHOL_DIAG, s, bs * (double)bs * bs / 3.0 * batch);
      note_launch();
      k_chol_diag<<<batch, DIAG_THREADS, 0, s>>>(L, ldl, j0, bs, dmax, tol_rel, fail, sL);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int rem = n - j0 - bs;
    if (rem <= 0) break;
    {
      KernelTimer kt(KF_FP64_GEMM, s, (double)rem * bs * bs * batch);
      note_launch();
      k_panel_trsm<<<dim3(panel_blocks(rem), batch), 256, 0, s>>>(L, ldl, j0, bs, rem, fail, sL);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    double* Pj = L + (j0 + bs) + ldl * (long long)j0;
    GemmBatch tb{batch, 1, sL, sL, sL, 0, 0, 0};
    e = launch_gemm_batched2(Pj, ldl, false, Pj, ldl, false, rem, rem, bs, -1.0, 1.0,
                             L + (j0 + bs) + ldl * (long long)(j0 + bs), ldl, tb, true, s);
    if (e != cudaSuccess) return e;
  }
  note_launch();
  k_zero_upper<<<dim3((n + 127) / 128, n, batch), 128, 0, s>>>(L, ldl, n, sL);
  return cudaGetLastError();
}

}  // namespace isdf
