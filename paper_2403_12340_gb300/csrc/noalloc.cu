// apply_eps_inv_noalloc: the apply step of the ISDF-SMW inverse with all of
// its scratch in one file-scope device array, so the call itself allocates
// no device memory.  The paper has no counterpart; this exists for callers
// that must not allocate at call time (see include/isdf_smw.h).
//
// The kernels and arithmetic of apply_eps_inv on an FP64 context (split-K
// theta^T X, K T1, theta T2, Coulomb convolution by FFT, all FP64), with the
// workspace carved out of g_apply_scratch instead of the context's lazily
// grown buffers.  On a mixed-precision context it runs the same FP64
// kernels on that context's theta (kept in FP64) and K: the tensor-core
// form of apply_eps_inv needs BF16 slices of the probe block padded to 128
// columns, 6 N_r bytes per padded column, far beyond a modest static pool.
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
// per device: the array's device address and the id of the CUDA context it
// was looked up in (a context id is never reused within a process)
double* g_addr[kMaxDevices] = {nullptr};
unsigned long long g_ctx_id[kMaxDevices] = {0};

// Id of the current CUDA context (the device's primary context once the
// runtime has made it current), through the driver entry points the
// runtime hands out, so that the library needs no link to the driver.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
cudaError_t current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e == cudaSuccess)
      e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return cudaErrorSymbolNotFound;
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  void* ctx = nullptr;
  if (get_current(&ctx) != 0 || !ctx) return cudaErrorDeviceUninitialized;
  return get_id(ctx, id) == 0 ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of g_apply_scratch on `dev`, looked up with that device
// current, once per device and CUDA context (after a cudaDeviceReset the
// device gets a new primary context, the library's module is loaded again
// and the array may sit elsewhere: the new context's id triggers a new
// lookup).  In host code the array's name is only a host-side stand-in;
// the kernels must get this address instead.
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return e;
  if (cur != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return e;
  // a thread that has not used the runtime yet may have no current context:
  // then the lookup itself (which binds the primary context) comes first
  unsigned long long id = 0;
  bool have_id = current_context_id(&id) == cudaSuccess;
  if (!have_id || !(g_addr[dev] && g_ctx_id[dev] == id)) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_apply_scratch);
    if (e == cudaSuccess) {
      if (!have_id) have_id = current_context_id(&id) == cudaSuccess;
      g_addr[dev] = have_id ? p : nullptr;  // without a context id: look it up on every call
      g_ctx_id[dev] = id;
      *out = p;
    }
    if (cur != dev) cudaSetDevice(cur);
    return e;
  }
  if (cur != dev) cudaSetDevice(cur);
  if (e != cudaSuccess) return e;
  *out = g_addr[dev];
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
