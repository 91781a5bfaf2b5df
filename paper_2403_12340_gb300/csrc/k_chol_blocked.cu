// Blocked right-looking Cholesky (no pivoting), FP64.
//
// For J = 0, 1, ...: the 64 x 64 diagonal block is factored in shared memory
// by one thread block, which also inverts its factor; the panel below is
// solved as one GEMM with that inverse; the trailing matrix gets a SYRK
// update.  All the O(n^3) work is in the two GEMMs, which use every SM.
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

// Factor A[j0:j0+bs, j0:j0+bs] (lower part, already updated) in place and
// write its inverse into dinv (bs x bs, ld CB).  One thread block on one
// SM, whose FP64 pipe (2 DFMA / clock) is the limit, so the kernel issues as
// few FP64 warp instructions as it can:
//  * the rank-1 update of step j touches only the m (m + 1) / 2 entries of
//    the remaining lower triangle, packed densely over the threads through a
//    table of (row, column) offsets, so no lane idles under a mask;
//  * one reciprocal square root per pivot (thread 0), columns scaled by it;
//  * the inverse by 16 x 16 blocks: the four diagonal blocks in parallel by
//    forward substitution, then the off-diagonal blocks as products
//    X_IJ = -X_II sum_{J <= K < I} L_IK X_KJ in order of I - J, which keeps
//    the dependent FMA chains 16 long instead of up to 2000.
constexpr int TRI = CB * (CB - 1) / 2;  // entries of a strictly lower 63-row triangle

__global__ void __launch_bounds__(256) k_chol_diag(double* A, long long lda, int j0, int bs, double* dinv,
                                                  const double* dmax, double tol_rel, int* fail, long long sA = 0) {
  __shared__ double Ls[CB][CB + 1];
  // problem blockIdx.x of a batch: its matrix, inverse block, max and flag
  A += sA * blockIdx.x;
  dinv += (long long)CB * CB * blockIdx.x;
  dmax += blockIdx.x;
  fail += blockIdx.x;
  __shared__ double Xs[CB][CB + 1];
  __shared__ double rdiag[CB];
  __shared__ unsigned char ta[TRI], tb[TRI];
  __shared__ int s_bad;
  if (*(volatile int*)fail >= 0) return;
  const int t = threadIdx.x;
  for (int idx = t; idx < CB * CB; idx += blockDim.x) {
    int i = idx & (CB - 1), k = idx >> 6;
    Ls[i][k] = (i < bs && k <= i) ? A[(j0 + i) + lda * (long long)(j0 + k)] : 0.0;
    Xs[i][k] = 0.0;
  }
  // (a, b) with b <= a for the packed index a (a + 1) / 2 + b
  for (int a = t; a < CB - 1; a += blockDim.x) {
    const int base = a * (a + 1) / 2;
    for (int b = 0; b <= a; ++b) {
      ta[base + b] = (unsigned char)a;
      tb[base + b] = (unsigned char)b;
    }
  }
  if (t == 0) s_bad = -1;
  const double thresh = tol_rel * (*dmax);
  __syncthreads();
  for (int j = 0; j < bs; ++j) {
    if (t == 0) {
      const double d = Ls[j][j];
      if (!(d > thresh)) {  // also catches NaN
        s_bad = j;
      } else {
        const double ri = rsqrt(d);
        Ls[j][j] = d * ri;
        rdiag[j] = ri;
      }
    }
    __syncthreads();
    if (s_bad >= 0) break;
    const double r = rdiag[j];
    for (int i = j + 1 + t; i < bs; i += blockDim.x) Ls[i][j] *= r;
    __syncthreads();
    // Ls[i][k] -= Ls[i][j] Ls[k][j] for j < k <= i < bs, packed
    const int m = bs - j - 1;
    const int cnt = m * (m + 1) / 2;
    for (int idx = t; idx < cnt; idx += blockDim.x) {
      const int i = j + 1 + ta[idx], k = j + 1 + tb[idx];
      Ls[i][k] = fma(-Ls[i][j], Ls[k][j], Ls[i][k]);
    }
    __syncthreads();
  }
  if (s_bad >= 0) {
    if (t == 0) atomicCAS(fail, -1, j0 + s_bad);
    return;
  }
  // inverse, step 1: the four diagonal 16 x 16 blocks (thread = block * 16 + column)
  if (t < CB) {
    const int o = (t >> 4) * 16, c = o + (t & 15);
    if (c < bs) {
      Xs[c][c] = rdiag[c];
      for (int i = c + 1; i < o + 16 && i < bs; ++i) {
        double acc = 0.0;
        for (int k = c; k < i; ++k) acc = fma(Ls[i][k], Xs[k][c], acc);
        Xs[i][c] = -acc * rdiag[i];
      }
    }
  }
  __syncthreads();
  // step 2: off-diagonal blocks by distance; thread (row u, col v) of a 16 x 16 block
  const int u = t & 15, v = t >> 4;
  for (int dist = 1; dist < 4; ++dist) {
    for (int J = 0; J + dist < 4; ++J) {
      const int I = J + dist;
      // W = sum_{K=J}^{I-1} L_IK X_KJ  (16 x 16), then X_IJ = -X_II W
      double w = 0.0;
      for (int K = J; K < I; ++K)
        for (int q = 0; q < 16; ++q) w = fma(Ls[I * 16 + u][K * 16 + q], Xs[K * 16 + q][J * 16 + v], w);
      __syncthreads();
      Ls[J * 16 + u][I * 16 + v] = w;  // scratch in the (unused) strict upper part
      __syncthreads();
      double x = 0.0;
      for (int q = 0; q <= u; ++q) x = fma(Xs[I * 16 + u][I * 16 + q], Ls[J * 16 + q][I * 16 + v], x);
      __syncthreads();
      Xs[I * 16 + u][J * 16 + v] = -x;
      __syncthreads();
    }
  }
  for (int idx = t; idx < bs * bs; idx += blockDim.x) {
    int i = idx % bs, k = idx / bs;
    A[(j0 + i) + lda * (long long)(j0 + k)] = (k <= i) ? Ls[i][k] : 0.0;
    dinv[i + CB * k] = (k <= i) ? Xs[i][k] : 0.0;
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

cudaError_t launch_cholesky_blocked(const double* W, long long ldw, int n, double tol_rel, double* L, long long ldl,
                                    double* dinv, double* dmax, int* fail, double* pan, cudaStream_t s) {
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
      // factor bs^3 / 3 flops and triangular inverse bs^3 / 3 flops
      KernelTimer kt(KF_CHOL_DIAG, s, 2.0 * bs * bs * bs / 3.0);
      note_launch();
      k_chol_diag<<<1, 256, 0, s>>>(L, ldl, j0, bs, dinv, dmax, tol_rel, fail);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int rem = n - j0 - bs;
    if (rem <= 0) break;
    // panel: L[j0+bs:, J] = A[j0+bs:, J] Dinv^T, computed into `pan` (rem x bs,
    // ld n) and copied back: a tile narrower than the panel must not
    // overwrite columns that another block still reads
    double* Pj = L + (j0 + bs) + ldl * (long long)j0;
    e = launch_gemm(Pj, ldl, false, dinv, CB, false, rem, bs, bs, 1.0, 0.0, pan, n, false, 1, nullptr, false, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy2DAsync(Pj, ldl * sizeof(double), pan, n * sizeof(double), rem * sizeof(double), bs,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    // trailing: A[j0+bs:, j0+bs:] -= L_panel L_panel^T (lower tiles, mirrored)
    e = launch_gemm(pan, n, false, pan, n, false, rem, rem, bs, -1.0, 1.0, L + (j0 + bs) + ldl * (long long)(j0 + bs),
                    ldl, true, 1, nullptr, false, s);
    if (e != cudaSuccess) return e;
  }
  dim3 g((n + 127) / 128, n);
  note_launch();
  k_zero_upper<<<g, 128, 0, s>>>(L, ldl, n);
  return cudaGetLastError();
}

// The same factorisation for `batch` matrices of equal size n (W_z = W + z
// sW, L_z = L + z sL): one launch per step covers every matrix.  dinv:
// batch 64 x 64 blocks, dmax / fail: batch entries, pan: batch n x 64.
cudaError_t launch_cholesky_blocked_batched(const double* W, long long ldw, long long sW, int n, int batch,
                                            double tol_rel, double* L, long long ldl, long long sL, double* dinv,
                                            double* dmax, int* fail, double* pan, cudaStream_t s) {
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
  const long long sP = (long long)n * CB;
  for (int j0 = 0; j0 < n; j0 += CB) {
    const int bs = min(CB, n - j0);
    {
      KernelTimer kt(KF_CHOL_DIAG, s, 2.0 * bs * bs * bs / 3.0 * batch);
      note_launch();
      k_chol_diag<<<batch, 256, 0, s>>>(L, ldl, j0, bs, dinv, dmax, tol_rel, fail, sL);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int rem = n - j0 - bs;
    if (rem <= 0) break;
    double* Pj = L + (j0 + bs) + ldl * (long long)j0;
    GemmBatch pb{batch, 1, sL, (long long)CB * CB, sP, 0, 0, 0};
    e = launch_gemm_batched2(Pj, ldl, false, dinv, CB, false, rem, bs, bs, 1.0, 0.0, pan, n, pb, false, s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_copy_block<<<dim3((rem + 127) / 128, bs, batch), 128, 0, s>>>(pan, n, sP, Pj, ldl, sL, rem, bs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    GemmBatch tb{batch, 1, sP, sP, sL, 0, 0, 0};
    e = launch_gemm_batched2(pan, n, false, pan, n, false, rem, rem, bs, -1.0, 1.0,
                             L + (j0 + bs) + ldl * (long long)(j0 + bs), ldl, tb, true, s);
    if (e != cudaSuccess) return e;
  }
  note_launch();
  k_zero_upper<<<dim3((n + 127) / 128, n, batch), 128, 0, s>>>(L, ldl, n, sL);
  return cudaGetLastError();
}

}  // namespace isdf
