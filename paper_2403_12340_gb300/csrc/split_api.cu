// isdf_dgemm_split: the split-precision tensor-core GEMM of the mixed path
// as a stand-alone C-ABI call (declared in include/isdf_smw.h).
#include <algorithm>
#include <string>

#include "../../include/isdf_smw.h"
#include "common.cuh"
#include "kernels.h"

using namespace isdf;

static thread_local std::string g_gemm_err;

extern "C" const char* isdf_dgemm_split_error(void) { return g_gemm_err.c_str(); }

static int gemm_fail(int code, const std::string& m) {
  g_gemm_err = m;
  return code;
}

extern "C" int isdf_dgemm_split(int M, int N, int K, double alpha, const double* A, long long lda, const double* B,
                                long long ldb, double beta, double* C, long long ldc, int nslices, void* stream) {
  g_gemm_err.clear();
  if (M < 0 || N < 0 || K < 0) return gemm_fail(ISDF_ERR_SHAPE, "isdf_dgemm_split: negative size");
  if (nslices < 1 || nslices > 3) return gemm_fail(ISDF_ERR_ARG, "isdf_dgemm_split: nslices must be 1, 2 or 3");
  if (M == 0 || N == 0) return ISDF_OK;
  if (!A || !B || !C) return gemm_fail(ISDF_ERR_ARG, "isdf_dgemm_split: null pointer");
  if (lda < M || ldb < N || ldc < M) return gemm_fail(ISDF_ERR_SHAPE, "isdf_dgemm_split: leading dimension too small");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int s = nslices;
  const int Mp = (M + 127) / 128 * 128, Np = (N + 127) / 128 * 128;
  const int Kp = (K > 0 ? (K + 63) / 64 : 1) * 64;
  const int max_split = std::max(64, tc_min_splits(Kp));
  const size_t na = (size_t)s * Mp * Kp, nb = (size_t)s * Np * Kp;
  const size_t npart = (size_t)max_split * M * N;
  __nv_bfloat16 *sa = nullptr, *sb = nullptr;
  double* part = nullptr;
  unsigned* status = nullptr;
  cudaError_t e = isdf::dev_malloc_async(&sa, na * 2, st);
  if (e == cudaSuccess) e = isdf::dev_malloc_async(&sb, nb * 2, st);
  if (e == cudaSuccess) e = isdf::dev_malloc_async(&part, npart * 8, st);
  if (e == cudaSuccess) e = isdf::dev_malloc_async(&status, 16, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sa, 0, na * 2, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sb, 0, nb * 2, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 16, st);
  if (e == cudaSuccess && K > 0) e = launch_slice_colmajor(A, lda, M, K, 0, 0, sa, Mp, Kp, s, st);
  if (e == cudaSuccess && K > 0) e = launch_slice_colmajor(B, ldb, N, K, 0, 0, sb, Np, Kp, s, st);
  if (e == cudaSuccess) {
    TcOperand oa{sa, Mp, Kp, s}, ob{sb, Np, Kp, s};
    e = tc_gemm_f64(oa, ob, M, N, alpha, beta, C, ldc, false, false, part, max_split, sms, status, st);
  }
  unsigned hst = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (sa) cudaFreeAsync(sa, st);
  if (sb) cudaFreeAsync(sb, st);
  if (part) cudaFreeAsync(part, st);
  if (status) cudaFreeAsync(status, st);
  if (e != cudaSuccess) return gemm_fail(ISDF_ERR_CUDA, std::string("isdf_dgemm_split: ") + cudaGetErrorString(e));
  if (hst & ST_TIMEOUT) return gemm_fail(ISDF_ERR_TIMEOUT, "isdf_dgemm_split: device wait timed out");
  return ISDF_OK;
}
