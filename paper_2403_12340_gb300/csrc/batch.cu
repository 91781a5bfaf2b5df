// Batched full-frequency runner (declared in include/isdf_smw.h): many
// systems of different sizes, every frequency of each, on one GPU.
//
// Two forms.  isdf_batch_run drives the entry points eagerly from host
// threads; isdf_batch_capture records the same device work of every system
// into one CUDA graph (after an eager run that sizes the workspace and fixes
// the ranks) and isdf_batch_replay launches it as a single graph.
//
// Each system owns a context, a non-blocking CUDA stream and its theta
// buffer for the life of the batch, so repeated runs allocate nothing.  A
// run hands the systems, largest estimated cost first, to a pool of host
// worker threads; a worker runs one system's fit, all-frequency
// polarizability and all-frequency SMW (smw_inverse_all) on the system's
// stream, then takes the next.  Systems on different workers overlap on the
// GPU; the largest start first, so the small ones fill the tail.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/isdf_smw.h"
#include "ctx.h"

struct isdf_batch {
  int device = 0;
  int prec = 0;
  int n_workers = 1;
  struct Sys {
    isdf_system d;
    std::vector<int64_t> mu;
    std::vector<double> energies;
    isdf_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    double* theta = nullptr;
    int rank = 0;
    double cost = 0.0;
  };
  std::vector<Sys> sys;
  std::vector<int> order;  // largest estimated cost first
  std::string err;
  // captured graph of every system's fit, polarizability and SMW
  cudaStream_t origin = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev_start = nullptr, ev_link = nullptr;
  std::vector<cudaEvent_t> ev_end;   // one per system, recorded at the end of its branch
  std::vector<cudaEvent_t> ev_lane;  // the end of the last system of each lane
  std::vector<double> g_omega;
  // the capacitance stage of every system in grouped launches (graph form)
  bool grouped_smw = false;
  void* ns_work = nullptr;
  size_t ns_ws = 0, ns_bytes = 0;
  std::vector<std::vector<unsigned char>> ns_staged;
};

namespace {

thread_local std::string g_batch_create_err;

void free_graph(isdf_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void free_batch(isdf_batch* b) {
  if (b->origin) cudaStreamSynchronize(b->origin);
  free_graph(b);
  if (b->ev_start) cudaEventDestroy(b->ev_start);
  if (b->ev_link) cudaEventDestroy(b->ev_link);
  for (cudaEvent_t e : b->ev_end) cudaEventDestroy(e);
  for (cudaEvent_t e : b->ev_lane) cudaEventDestroy(e);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->ns_work) cudaFree(b->ns_work);
  for (auto& s : b->sys) {
    if (s.ctx) isdf_destroy(s.ctx);
    if (s.theta) cudaFree(s.theta);
    if (s.stream) cudaStreamDestroy(s.stream);
  }
  delete b;
}

// flops of one system's fit, polarizability and SMW at n_omega frequencies,
// for the largest-first order
double cost_estimate(const isdf_system& d, int n_omega) {
  const double nr = (double)d.n1 * d.n2 * d.n3, m = d.n_mu, ne = d.n_v + d.n_c, np = (double)d.n_v * d.n_c;
  return nr * m * (2.0 * ne + m) + nr * m * m + n_omega * (m * m * np + 9.0 * m * m * m);
}

}  // namespace

extern "C" int isdf_batch_create(isdf_batch** out, const isdf_system* systems, int n_systems, int prec,
                                 int n_workers) {
  g_batch_create_err.clear();
  if (!out || !systems) {
    g_batch_create_err = "isdf_batch_create: null pointer argument";
    return ISDF_ERR_ARG;
  }
  *out = nullptr;
  if (n_systems < 1 || n_workers < 1 || n_workers > 64) {
    g_batch_create_err = "isdf_batch_create: need n_systems >= 1 and 1 <= n_workers <= 64";
    return ISDF_ERR_SHAPE;
  }
  if (prec != ISDF_PREC_FP64 && prec != ISDF_PREC_MIXED) {
    g_batch_create_err = "isdf_batch_create: prec must be ISDF_PREC_FP64 or ISDF_PREC_MIXED";
    return ISDF_ERR_ARG;
  }
  isdf_batch* b = new isdf_batch();
  b->prec = prec;
  b->n_workers = n_workers;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    g_batch_create_err = "isdf_batch_create: no current CUDA device";
    return ISDF_ERR_CUDA;
  }
  b->sys.resize(n_systems);
  for (int i = 0; i < n_systems; ++i) {
    const isdf_system& d = systems[i];
    auto& s = b->sys[i];
    if (!d.phi || !d.mu_idx || !d.energies || d.n_mu < 1 || d.n_v < 1 || d.n_c < 1) {
      free_batch(b);
      g_batch_create_err = "isdf_batch_create: system " + std::to_string(i) + " has a null pointer or empty size";
      return ISDF_ERR_ARG;
    }
    s.d = d;
    s.mu.assign(d.mu_idx, d.mu_idx + d.n_mu);
    s.energies.assign(d.energies, d.energies + d.n_v + d.n_c);
    s.d.mu_idx = s.mu.data();
    s.d.energies = s.energies.data();
    cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    const long long nr = (long long)d.n1 * d.n2 * d.n3;
    if (e == cudaSuccess) e = isdf::dev_malloc(&s.theta, (size_t)nr * d.n_mu * sizeof(double));
    if (e != cudaSuccess) {
      free_batch(b);
      g_batch_create_err = std::string("isdf_batch_create: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? ISDF_ERR_NOMEM : ISDF_ERR_CUDA;
    }
    int rc = isdf_create(&s.ctx, d.n1, d.n2, d.n3, d.L1, d.L2, d.L3, s.stream);
    if (rc != ISDF_OK) {
      g_batch_create_err = std::string("isdf_batch_create: system ") + std::to_string(i) + ": " +
                           isdf_last_error(nullptr);
      free_batch(b);
      return rc;
    }
  }
  b->order.resize(n_systems);
  for (int i = 0; i < n_systems; ++i) b->order[i] = i;
  *out = b;
  return ISDF_OK;
}

extern "C" int isdf_batch_destroy(isdf_batch* b) {
  if (!b) return ISDF_ERR_ARG;
  for (auto& s : b->sys)
    if (s.stream) cudaStreamSynchronize(s.stream);
  free_batch(b);
  return ISDF_OK;
}

extern "C" int isdf_batch_run(isdf_batch* b, const double* omega, int n_omega, int n_workers, double* latency_ms,
                              double* service_ms, double* total_ms) {
  if (!b) return ISDF_ERR_ARG;
  b->err.clear();
  if (!omega || n_omega < 1) {
    b->err = "isdf_batch_run: need n_omega >= 1 frequencies";
    return ISDF_ERR_ARG;
  }
  if (n_workers < 0 || n_workers > 64) {
    b->err = "isdf_batch_run: n_workers must be in [0, 64]";
    return ISDF_ERR_ARG;
  }
  const int n = (int)b->sys.size();
  for (auto& s : b->sys) s.cost = cost_estimate(s.d, n_omega);
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int x, int y) { return b->sys[x].cost > b->sys[y].cost; });
  std::vector<double> lat(n, 0.0), svc(n, 0.0);
  std::atomic<int> next{0};
  std::atomic<int> first_rc{ISDF_OK};
  std::mutex err_mu;
  const auto t0 = std::chrono::steady_clock::now();
  auto ms_since = [](std::chrono::steady_clock::time_point a) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
  };
  auto worker = [&]() {
    if (cudaSetDevice(b->device) != cudaSuccess) {
      first_rc.store(ISDF_ERR_CUDA);
      return;
    }
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n || first_rc.load() != ISDF_OK) return;
      auto& s = b->sys[b->order[i]];
      const auto ts = std::chrono::steady_clock::now();
      int rc = isdf_fit(s.ctx, s.d.phi, s.d.n_v, s.d.n_c, s.d.mu_idx, s.d.n_mu, b->prec, s.theta, &s.rank);
      if (rc == ISDF_OK) rc = build_polarizability(s.ctx, s.d.energies, omega, n_omega, nullptr, nullptr);
      if (rc == ISDF_OK) rc = smw_inverse_all(s.ctx, nullptr);
      if (rc != ISDF_OK) {
        int expect = ISDF_OK;
        if (first_rc.compare_exchange_strong(expect, rc)) {
          std::lock_guard<std::mutex> g(err_mu);
          b->err = "isdf_batch_run: system " + std::to_string(b->order[i]) + ": " + isdf_last_error(s.ctx);
        }
        return;
      }
      svc[b->order[i]] = ms_since(ts);
      lat[b->order[i]] = ms_since(t0);
    }
  };
  std::vector<std::thread> pool;
  const int nw = std::min(n_workers > 0 ? n_workers : b->n_workers, n);
  for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  if (total_ms) *total_ms = ms_since(t0);
  if (latency_ms)
    for (int i = 0; i < n; ++i) latency_ms[i] = lat[i];
  if (service_ms)
    for (int i = 0; i < n; ++i) service_ms[i] = svc[i];
  return first_rc.load();
}

extern "C" int isdf_batch_context(isdf_batch* b, int system, isdf_ctx** ctx, int* rank) {
  if (!b || !ctx) return ISDF_ERR_ARG;
  if (system < 0 || system >= (int)b->sys.size()) {
    b->err = "isdf_batch_context: system index out of range";
    return ISDF_ERR_ARG;
  }
  *ctx = b->sys[system].ctx;
  if (rank) *rank = b->sys[system].rank;
  return ISDF_OK;
}

extern "C" const char* isdf_batch_last_error(isdf_batch* b) {
  return b ? b->err.c_str() : g_batch_create_err.c_str();
}

namespace {

// Capture every system's device work into b->graph; the caller ends the
// capture on error (cudaStreamEndCapture) through end_capture below.
int capture_systems(isdf_batch* b, const double* omega, int n_omega) {
  auto cuda_err = [&](cudaError_t e, const char* what) {
    b->err = std::string("isdf_batch_capture: ") + what + ": " + cudaGetErrorString(e);
    return ISDF_ERR_CUDA;
  };
  cudaError_t e = cudaEventRecordWithFlags(b->ev_start, b->origin, cudaEventRecordExternal);
  if (e != cudaSuccess) return cuda_err(e, "start event");
  if ((e = cudaEventRecord(b->ev_link, b->origin)) != cudaSuccess) return cuda_err(e, "fork event");
  // lanes: as many systems in flight as the batch has workers; each system,
  // largest first, follows the lane with the least estimated work so far
  const int nl = (int)b->ev_lane.size();
  std::vector<double> load(nl, 0.0);
  std::vector<char> used(nl, 0);
  for (int j = 0; j < (int)b->order.size(); ++j) {
    const int i = b->order[j];
    auto& s = b->sys[i];
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    e = cudaStreamWaitEvent(s.stream, used[l] ? b->ev_lane[l] : b->ev_link, 0);
    if (e != cudaSuccess) return cuda_err(e, "fork");
    load[l] += s.cost;
    used[l] = 1;
    int rank = 0;
    int rc = isdf_fit(s.ctx, s.d.phi, s.d.n_v, s.d.n_c, s.d.mu_idx, s.d.n_mu, b->prec, s.theta, &rank);
    if (rc == ISDF_OK) rc = build_polarizability(s.ctx, s.d.energies, omega, n_omega, nullptr, nullptr);
    if (rc == ISDF_OK && !b->grouped_smw) rc = smw_inverse_all(s.ctx, nullptr);
    if (rc != ISDF_OK) {
      b->err = "isdf_batch_capture: system " + std::to_string(i) + ": " + isdf_last_error(s.ctx);
      return rc;
    }
    if ((e = cudaEventRecordWithFlags(b->ev_end[i], s.stream, cudaEventRecordExternal)) != cudaSuccess)
      return cuda_err(e, "end event");
    if ((e = cudaEventRecord(b->ev_lane[l], s.stream)) != cudaSuccess) return cuda_err(e, "lane event");
  }
  for (int l = 0; l < nl; ++l)
    if (used[l] && (e = cudaStreamWaitEvent(b->origin, b->ev_lane[l], 0)) != cudaSuccess) return cuda_err(e, "join");
  if (b->grouped_smw) {
    // every system's capacitance, all frequencies, in grouped persistent
    // launches over (system, frequency, tile): one per Newton-Schulz product
    std::vector<isdf_ctx*> cs;
    for (auto& s : b->sys) cs.push_back(s.ctx);
    e = isdf::ns_stage_grouped(cs.data(), (int)cs.size(), b->origin, b->ns_work, b->ns_ws, b->ns_staged);
    if (e != cudaSuccess) return cuda_err(e, "grouped capacitance stage");
    for (size_t i = 0; i < b->sys.size(); ++i)
      if ((e = cudaEventRecordWithFlags(b->ev_end[i], b->origin, cudaEventRecordExternal)) != cudaSuccess)
        return cuda_err(e, "end event");
  }
  return ISDF_OK;
}

// Whether the captured graph can run the capacitance stage of all systems
// together (mixed precision, several frequencies, every system's eager
// smw_inverse_all on the Newton-Schulz route, at most 32 systems); if so,
// size the descriptor workspace and run the stage once eagerly, which
// uploads the descriptors the captured launches reuse.
int prepare_grouped_smw(isdf_batch* b, int n_omega) {
  b->grouped_smw = false;
  if (b->prec != ISDF_PREC_MIXED || n_omega < 2 || b->sys.size() > 32) return ISDF_OK;
  for (auto& s : b->sys) {
    isdf_ctx* c = s.ctx;
    if (c->rank <= 0 || c->ns_nw != n_omega || c->ns_e0 < 0.0) return ISDF_OK;
  }
  const size_t ws = (isdf::tc_grouped_workspace_bytes((int)b->sys.size()) + 255) / 256 * 256;
  const size_t need = ws * (size_t)isdf::ns_stage_slots();
  if (need > b->ns_bytes) {
    if (b->ns_work) cudaFree(b->ns_work);
    b->ns_work = nullptr;
    b->ns_bytes = 0;
    b->ns_staged.clear();
    if (isdf::dev_malloc(&b->ns_work, need) != cudaSuccess) {
      b->err = "isdf_batch_capture: descriptor workspace allocation failed";
      return ISDF_ERR_NOMEM;
    }
    b->ns_bytes = need;
  }
  b->ns_ws = ws;
  std::vector<isdf_ctx*> cs;
  for (auto& s : b->sys) cs.push_back(s.ctx);
  cudaError_t e = isdf::ns_stage_grouped(cs.data(), (int)cs.size(), b->origin, b->ns_work, ws, b->ns_staged);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->origin);
  if (e != cudaSuccess) {
    b->err = std::string("isdf_batch_capture: grouped capacitance stage: ") + cudaGetErrorString(e);
    return ISDF_ERR_CUDA;
  }
  b->grouped_smw = true;
  return ISDF_OK;
}

}  // namespace

extern "C" int isdf_batch_capture(isdf_batch* b, const double* omega, int n_omega) {
  if (!b) return ISDF_ERR_ARG;
  b->err.clear();
  if (b->origin) {
    cudaError_t e = cudaStreamSynchronize(b->origin);
    if (e != cudaSuccess) {
      b->err = std::string("isdf_batch_capture: ") + cudaGetErrorString(e);
      return ISDF_ERR_CUDA;
    }
  }
  free_graph(b);
  b->g_omega.clear();
  // the eager run: workspace sizes, ranks, uploaded weights
  int rc = isdf_batch_run(b, omega, n_omega, 0, nullptr, nullptr, nullptr);
  if (rc != ISDF_OK) return rc;
  for (int i = 0; i < (int)b->sys.size(); ++i)
    if (!b->sys[i].ctx->fit_full) {
      b->err = "isdf_batch_capture: system " + std::to_string(i) +
               " needed a pivoted (rank-deficient) fit, which a captured graph cannot replay";
      return ISDF_ERR_STATE;
    }
  if (cudaSetDevice(b->device) != cudaSuccess) {
    b->err = "isdf_batch_capture: cudaSetDevice failed";
    return ISDF_ERR_CUDA;
  }
  cudaError_t e = cudaSuccess;
  if (!b->origin) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (e == cudaSuccess && !b->ev_start) e = cudaEventCreate(&b->ev_start);
  if (e == cudaSuccess && !b->ev_link) e = cudaEventCreateWithFlags(&b->ev_link, cudaEventDisableTiming);
  while (e == cudaSuccess && b->ev_end.size() < b->sys.size()) {
    cudaEvent_t x = nullptr;
    e = cudaEventCreate(&x);
    if (e == cudaSuccess) b->ev_end.push_back(x);
  }
  const size_t lanes = (size_t)std::max(1, std::min(b->n_workers, (int)b->sys.size()));
  while (e == cudaSuccess && b->ev_lane.size() < lanes) {
    cudaEvent_t x = nullptr;
    e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (e == cudaSuccess) b->ev_lane.push_back(x);
  }
  if (e != cudaSuccess) {
    b->err = std::string("isdf_batch_capture: ") + cudaGetErrorString(e);
    return ISDF_ERR_CUDA;
  }
  for (auto& s : b->sys) cudaStreamSynchronize(s.stream);
  rc = prepare_grouped_smw(b, n_omega);
  if (rc != ISDF_OK) return rc;
  // the capture itself: entry points in capture mode on this thread only
  e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    b->err = std::string("isdf_batch_capture: begin capture: ") + cudaGetErrorString(e);
    return ISDF_ERR_CUDA;
  }
  isdf::tl_capture = true;
  rc = capture_systems(b, omega, n_omega);
  isdf::tl_capture = false;
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->origin, &g);
  if (rc == ISDF_OK && e != cudaSuccess) {
    b->err = std::string("isdf_batch_capture: end capture: ") + cudaGetErrorString(e);
    rc = ISDF_ERR_CUDA;
  }
  if (rc != ISDF_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();  // clear the runtime's last-error slot after a failed capture
    return rc;
  }
  b->graph = g;
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e == cudaSuccess) e = cudaGraphUpload(b->exec, b->origin);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->origin);
  if (e != cudaSuccess) {
    free_graph(b);
    b->err = std::string("isdf_batch_capture: instantiate: ") + cudaGetErrorString(e);
    return ISDF_ERR_CUDA;
  }
  b->g_omega.assign(omega, omega + n_omega);
  return ISDF_OK;
}

extern "C" int isdf_batch_replay(isdf_batch* b, double* latency_ms, double* total_ms) {
  if (!b) return ISDF_ERR_ARG;
  b->err.clear();
  if (!b->exec) {
    b->err = "isdf_batch_replay: no captured graph (call isdf_batch_capture first)";
    return ISDF_ERR_STATE;
  }
  if (cudaSetDevice(b->device) != cudaSuccess) {
    b->err = "isdf_batch_replay: cudaSetDevice failed";
    return ISDF_ERR_CUDA;
  }
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGraphLaunch(b->exec, b->origin);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->origin);
  const double wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (e != cudaSuccess) {
    b->err = std::string("isdf_batch_replay: ") + cudaGetErrorString(e);
    return ISDF_ERR_CUDA;
  }
  if (total_ms) *total_ms = wall;
  const int n = (int)b->sys.size();
  for (int i = 0; i < n; ++i) {
    if (latency_ms) {
      float ms = -1.0f;
      if (cudaEventElapsedTime(&ms, b->ev_start, b->ev_end[i]) != cudaSuccess) ms = -1.0f;
      latency_ms[i] = ms;
    }
    const int rc = isdf::graph_check(b->sys[i].ctx, "isdf_batch_replay");
    if (rc != ISDF_OK) {
      b->err = "isdf_batch_replay: system " + std::to_string(i) + ": " + isdf_last_error(b->sys[i].ctx);
      return rc;
    }
  }
  cudaGetLastError();
  return ISDF_OK;
}
