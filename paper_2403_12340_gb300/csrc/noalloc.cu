// apply_eps_inv_noalloc: the apply step of the ISDF-SMW inverse with all of
// its scratch in one file-scope device array, so the call itself allocates
// no device memory.  The paper has no counterpart; this exists for callers
// that must not allocate at call time (see include/isdf_smw.h).
//
// Same kernels and arithmetic as apply_eps_inv (split-K theta^T X, K T1,
// theta T2, Coulomb convolution by FFT), with its workspace carved out of
// g_apply_scratch instead of the context's lazily grown buffers.
#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/isdf_smw.h"
#include "kernels.h"

using namespace isdf;

namespace {

// 8 MiB of scratch per device that loads this library, held until exit.
constexpr size_t kPoolDoubles = (size_t)1 << 20;
static __device__ __align__(256) double g_apply_scratch[kPoolDoubles];

constexpr int kMaxDevices = 64;
constexpr int kMaxSplits = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_apply_scratch on `dev`, looked up once per device with
// that device current.  In host code the array's name is only a host-side
// stand-in; the kernels must get this address instead.
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_addr[dev]) {
    *out = g_addr[dev];
    return cudaSuccess;
  }
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return e;
  if (cur != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return e;
  double* p = nullptr;
  e = cudaGetSymbolAddress((void**)&p, g_apply_scratch);
  if (cur != dev) cudaSetDevice(cur);
  if (e != cudaSuccess) return e;
  g_addr[dev] = p;
  *out = p;
  return cudaSuccess;
}

size_t round256(size_t n_doubles) { return (n_doubles + 31) / 32 * 32; }

}  // namespace

extern "C" int apply_eps_inv_noalloc(isdf_ctx* c, int k, const double* X, int n_rhs, double* Y) {
  if (!c) return ISDF_ERR_ARG;
  ApplyView v;
  int rc = ctx_apply_view(c, k, &v);
  if (rc != ISDF_OK) return rc;
  if (!X || !Y) return ctx_fail(c, ISDF_ERR_ARG, "apply_eps_inv_noalloc: null pointer argument");
  if (n_rhs < 1) return ctx_fail(c, ISDF_ERR_SHAPE, "apply_eps_inv_noalloc: n_rhs must be >= 1");
  if (v.device < 0 || v.device >= kMaxDevices)
    return ctx_fail(c, ISDF_ERR_ARG, "apply_eps_inv_noalloc: device ordinal out of range");
  const int r = v.rank;
  const long long nr = v.n_r;
  const long long lds = 2 * v.n_half;
  if (r == 0) {
    if (Y != X) {
      cudaError_t e = cudaMemcpyAsync(Y, X, (size_t)nr * n_rhs * sizeof(double), cudaMemcpyDeviceToDevice,
                                      v.stream);
      if (e != cudaSuccess) return ctx_fail(c, ISDF_ERR_CUDA, cudaGetErrorString(e));
    }
    return ISDF_OK;
  }
  // scratch per probe column: T1 (r), T2 (r), T3 (N_r), half spectrum, split-K partials
  const size_t per_col = 2 * round256((size_t)r) + round256((size_t)nr) + round256((size_t)lds) +
                         round256((size_t)kMaxSplits * r);
  const size_t nc_fit = kPoolDoubles / per_col;
  if (nc_fit < 1) {
    std::string m = "apply_eps_inv_noalloc: one probe column needs " + std::to_string(per_col * 8) +
                    " bytes of scratch (2 N_mu + N_r + 2 h n2 n3 + 64 N_mu doubles); the static pool holds " +
                    std::to_string(kPoolDoubles * 8) + " bytes: use apply_eps_inv";
    return ctx_fail(c, ISDF_ERR_SHAPE, m.c_str());
  }
  double* base = nullptr;
  cudaError_t e = scratch_address(v.device, &base);
  if (e != cudaSuccess) return ctx_fail(c, ISDF_ERR_CUDA, cudaGetErrorString(e));
  const int nc0 = (int)std::min(std::min(nc_fit, (size_t)n_rhs), (size_t)64);
  double* T1 = base;
  double* T2 = T1 + round256((size_t)r * nc0);
  double* T3 = T2 + round256((size_t)r * nc0);
  double* S = T3 + round256((size_t)nr * nc0);
  double* P = S + round256((size_t)lds * nc0);
  const long long tiles = (long long)((r + 127) / 128) * ((nc0 + 15) / 16);
  long long want = (2ll * v.num_sms + tiles - 1) / tiles;
  const int sp = (int)std::max(1ll, std::min(want, std::min(std::max(1ll, nr / 1024), (long long)kMaxSplits)));
  for (int c0 = 0; c0 < n_rhs; c0 += nc0) {
    const int nc = std::min(nc0, n_rhs - c0);
    const double* Xc = X + nr * c0;
    double* Yc = Y + nr * c0;
    e = launch_gemm(v.theta, nr, true, Xc, nr, true, r, nc, (int)nr, 1.0, 0.0, T1, r, false, sp, P, true,
                    v.stream);
    if (e == cudaSuccess)
      e = launch_gemm(v.K, r, false, T1, r, true, r, nc, r, 1.0, 0.0, T2, r, false, 1, nullptr, true, v.stream);
    if (e == cudaSuccess)
      e = launch_gemm(v.theta, nr, false, T2, r, true, (int)nr, nc, r, 1.0, 0.0, T3, nr, false, 1, nullptr,
                      true, v.stream);
    if (e == cudaSuccess)
      e = launch_fft_convolve(v.fft, T3, nr, nc, S, lds, v.wconv, Xc, nr, Yc, nr, v.smem_xy, v.smem_z,
                              v.stream);
    if (e != cudaSuccess) return ctx_fail(c, ISDF_ERR_CUDA, cudaGetErrorString(e));
  }
  return ISDF_OK;
}
