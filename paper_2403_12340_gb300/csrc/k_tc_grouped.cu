// Grouped persistent split-precision GEMM with a device work queue.
//
// One launch computes a list of problems of different shapes -- each a
// batch of equal-shaped products C_b = alpha A_b B_b^T + beta C_b with BF16
// slice operands, as tc_gemm_f64_batched takes them -- for example the
// capacitance products of every frequency of every system of a batch.  A
// work unit is one 128 x 128 output tile of one member of one problem; the
// units of all problems form one index range, and the persistent blocks
// claim them from a global counter (atomicAdd), so blocks that draw small
// tiles of small systems simply claim more.  Inside a block the TMA
// producer claims a unit and hands its index to the MMA thread and the four
// epilogue warps through a small shared-memory ring guarded by mbarriers;
// the tiles then flow through the same stage ring, TMEM accumulators and
// double-float run sums as in k_tc_gemm.cu.  Every wait is bounded
// (tc::mbar_wait): on expiry the status word gets ST_TIMEOUT, the roles stop
// claiming, and the block waits (bounded) for its own TMA copies before it
// frees tensor memory and returns.
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "../../include/isdf_smw.h"
#include "kernels.h"
#include "tc.cuh"

namespace isdf {

namespace {

constexpr int GB_BM = 128, GB_BN = 128, GB_BK = 64;
constexpr int GB_THREADS = 192;
constexpr int GB_RING = 4;  // unit indices in flight between the producer and the other roles
constexpr int GB_SMEM_LIMIT = 227 * 1024;

struct GbProblem {
  int M, N, k_iters, tiles_m, tiles_n, lower, count, s;
  int a_rows_pad, b_rows_pad, a_brows, b_brows;
  long long c_bstride, ldc, unit_begin, units;
  double alpha, beta;
  double* C;
};

struct GbArgs {
  const GbProblem* prob;   // device, nprob entries
  const CUtensorMap* maps;  // device, 2 nprob entries (A, B of each problem), 64-byte aligned
  int nprob;
  long long units;
  unsigned long long* queue;  // device counter, zero at launch
  int group;                  // chunks per FP32 accumulation run (0: the whole K range)
  int s;                      // slices (the same for every problem)
  unsigned* status;
};

__host__ __device__ inline int gb_stage_bytes(int s) { return s * (GB_BM + GB_BN) * GB_BK * 2; }
__host__ __device__ inline int gb_stages(int s) {
  const int st = (GB_SMEM_LIMIT - 4096) / gb_stage_bytes(s);
  return st > 4 ? 4 : st;
}

struct GbUnit {
  int p, bidx, mt, nt, m0, n0;
};

__device__ __forceinline__ GbUnit gb_unit(const GbProblem* pr, int nprob, long long u) {
  int p = 0;
  while (p + 1 < nprob && u >= pr[p + 1].unit_begin) ++p;
  const GbProblem& q = pr[p];
  const long long local = u - q.unit_begin;
  const int tiles = q.lower ? q.tiles_m * (q.tiles_m + 1) / 2 : q.tiles_m * q.tiles_n;
  GbUnit w;
  w.p = p;
  w.bidx = (int)(local / tiles);
  const int tile = (int)(local - (long long)w.bidx * tiles);
  if (q.lower) {
    lower_tile(tile, w.mt, w.nt);
  } else {
    w.mt = tile / q.tiles_n;
    w.nt = tile - w.mt * q.tiles_n;
  }
  w.m0 = w.mt * GB_BM;
  w.n0 = w.nt * GB_BN;
  return w;
}

__device__ __forceinline__ int gb_groups(const GbProblem& q, int group) {
  return (group > 0 && q.k_iters > 0) ? (q.k_iters + group - 1) / group : 1;
}

}  // namespace

__global__ void __launch_bounds__(GB_THREADS, 1) k_tc_grouped(GbArgs a) {
  extern __shared__ __align__(1024) uint8_t gb_smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)gb_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ GbProblem sp[32];
  __shared__ long long uq[GB_RING];
  __shared__ int s_abort;
  const int S = gb_stages(a.s);
  const int stage_bytes = gb_stage_bytes(a.s);
  uint64_t* full = (uint64_t*)(smem + S * stage_bytes);
  uint64_t* empty = full + 4;
  uint64_t* tfull = empty + 4;
  uint64_t* tempty = tfull + 2;
  uint64_t* ufull = tempty + 2;
  uint64_t* uempty = ufull + GB_RING;
  uint32_t* tmem_slot = (uint32_t*)(uempty + GB_RING);
  constexpr uint32_t ACC = GB_BN;
  const bool grouped = a.group > 0;
  const uint32_t tcols = grouped ? 4 * ACC : 2 * ACC;
  const uint32_t df_hi = 2 * ACC, df_lo = 3 * ACC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < a.nprob; i += blockDim.x) sp[i] = a.prob[i];
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int i = 0; i < S; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&tfull[i], 1);
      tc::mbar_init(&tempty[i], 4);
    }
    for (int i = 0; i < GB_RING; ++i) {
      tc::mbar_init(&ufull[i], 1);
      tc::mbar_init(&uempty[i], 5);  // the MMA thread and the four epilogue warps
    }
    tc::fence_mbar_init();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, tcols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: claims the units
    const uint32_t bytes = (uint32_t)stage_bytes;
    uint32_t g = 0;  // stage-ring position, continuous across units
    for (uint32_t n = 0;; ++n) {
      const int slot = (int)(n % GB_RING);
      if (!tc::mbar_wait(&uempty[slot], ((n / GB_RING) & 1u) ^ 1u, a.status)) {
        s_abort = 1;
        break;
      }
      long long u = s_abort ? -1 : (long long)atomicAdd(a.queue, 1ull);
      if (u >= a.units) u = -1;
      uq[slot] = u;
      tc::mbar_arrive(&ufull[slot]);  // releases the index to the other roles
      if (u < 0) break;
      const GbUnit w = gb_unit(sp, a.nprob, u);
      const GbProblem& q = sp[w.p];
      const CUtensorMap* ma = a.maps + 2 * w.p;
      const CUtensorMap* mb = ma + 1;
      const int a_row0 = w.bidx * q.a_brows + w.m0, b_row0 = w.bidx * q.b_brows + w.n0;
      bool ok = true;
      for (int kc = 0; kc < q.k_iters; ++kc, ++g) {
        const int st = (int)(g % (uint32_t)S);
        const uint32_t ph = (g / (uint32_t)S) & 1u;
        if (!tc::mbar_wait(&empty[st], ph ^ 1u, a.status)) {
          ok = false;
          break;
        }
        tc::mbar_expect_tx(&full[st], bytes);
        uint8_t* sa = smem + st * stage_bytes;
        uint8_t* sb = sa + a.s * GB_BM * GB_BK * 2;
        for (int l = 0; l < a.s; ++l) {
          tc::tma_load_2d(sa + l * GB_BM * GB_BK * 2, ma, &full[st], kc * GB_BK, a_row0 + l * q.a_rows_pad);
          tc::tma_load_2d(sb + l * GB_BN * GB_BK * 2, mb, &full[st], kc * GB_BK, b_row0 + l * q.b_rows_pad);
        }
      }
      if (!ok) {
        s_abort = 1;
        break;
      }
    }
    // the copies this thread issued must land before the block frees its
    // shared memory: wait (bounded, 1 ms) for the last stages it filled
    const uint32_t last = g < (uint32_t)S ? g : (uint32_t)S;
    for (uint32_t i = 1; i <= last; ++i) {
      const uint32_t gg = g - i;
      const uint64_t t0 = global_ns();
      while (!tc::mbar_try_wait(&full[gg % (uint32_t)S], (gg / (uint32_t)S) & 1u) && global_ns() - t0 < 1000000ull) {
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = tc::idesc_bf16_f32(GB_BM, GB_BN);
    uint32_t g = 0, gi = 0;
    for (uint32_t n = 0;; ++n) {
      const int slot = (int)(n % GB_RING);
      if (!tc::mbar_wait(&ufull[slot], (n / GB_RING) & 1u, a.status)) {
        s_abort = 1;
        break;
      }
      const long long u = uq[slot];
      tc::mbar_arrive(&uempty[slot]);
      if (u < 0) break;
      const GbUnit w = gb_unit(sp, a.nprob, u);
      const GbProblem& q = sp[w.p];
      const int ng = gb_groups(q, a.group);
      int kc = 0;
      bool ok = true;
      for (int gr = 0; gr < ng && ok; ++gr, ++gi) {
        const int buf = (int)(gi & 1u);
        if (!tc::mbar_wait(&tempty[buf], ((gi >> 1) & 1u) ^ 1u, a.status)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)buf * ACC;
        bool first = true;
        const int kg0 = kc;
        const int kend = grouped ? min(q.k_iters, kc + a.group) : q.k_iters;
        for (; kc < kend; ++kc, ++g) {
          const int st = (int)(g % (uint32_t)S);
          if (!tc::mbar_wait(&full[st], (g / (uint32_t)S) & 1u, a.status)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + st * stage_bytes);
          const uint32_t sb = sa + (uint32_t)(a.s * GB_BM * GB_BK * 2);
#pragma unroll
          for (int kk = 0; kk < GB_BK / 16; ++kk)
            for (int i = 0; i < a.s; ++i)
              for (int j = 0; i + j < a.s; ++j) {
                const uint64_t ad = tc::desc_kmajor_sw128(sa + (uint32_t)(i * GB_BM * GB_BK * 2 + kk * 32));
                const uint64_t bd = tc::desc_kmajor_sw128(sb + (uint32_t)(j * GB_BN * GB_BK * 2 + kk * 32));
                tc::mma_bf16(d, ad, bd, idesc, first ? 0u : 1u);
                first = false;
              }
          tc::mma_commit(&empty[st]);
        }
        if (!ok) break;
        if (kend > kg0) {
          tc::mma_commit(&tfull[buf]);
        } else {
          tc::mbar_arrive(&tfull[buf]);
        }
      }
      if (!ok) {
        s_abort = 1;
        break;
      }
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: thread <-> tile row (TMEM lane)
    const int qd = warp & 3;
    const int row = qd * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(qd * 32) << 16);
    uint32_t gi = 0;
    bool stop = false;
    for (uint32_t n = 0; !stop; ++n) {
      const int slot = (int)(n % GB_RING);
      if (!tc::mbar_wait(&ufull[slot], (n / GB_RING) & 1u, a.status)) break;
      const long long u = uq[slot];
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&uempty[slot]);
      if (u < 0) break;
      const GbUnit w = gb_unit(sp, a.nprob, u);
      const GbProblem& q = sp[w.p];
      const int ng = gb_groups(q, a.group);
      double* Cb = q.C + q.c_bstride * w.bidx;
      const int m = w.m0 + row;
      for (int gr = 0; gr < ng; ++gr, ++gi) {
        const int buf = (int)(gi & 1u);
        const bool ok = tc::mbar_wait(&tfull[buf], (gi >> 1) & 1u, a.status);
        tc::fence_after_sync();
        if (!ok || s_abort) {
          stop = true;
          break;
        }
        const uint32_t acc = lane_base + (uint32_t)buf * ACC;
        const bool last = gr + 1 == ng;
        for (int c = 0; c < GB_BN; c += 16) {
          float v[16], hi[16], lo[16];
          if (q.k_iters > 0) {
            tc::tmem_ld16(acc + (uint32_t)c, v);
          } else {
            for (int i = 0; i < 16; ++i) v[i] = 0.f;
          }
          if (gr > 0) {  // (hi, lo) + v by two-sum, renormalised
            tc::tmem_ld16(lane_base + df_hi + (uint32_t)c, hi);
            tc::tmem_ld16(lane_base + df_lo + (uint32_t)c, lo);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float t = __fadd_rn(hi[i], v[i]);
              const float bv = __fsub_rn(t, hi[i]);
              const float err = __fadd_rn(__fsub_rn(hi[i], __fsub_rn(t, bv)), __fsub_rn(v[i], bv));
              const float l = __fadd_rn(lo[i], err);
              hi[i] = __fadd_rn(t, l);
              lo[i] = __fsub_rn(l, __fsub_rn(hi[i], t));
            }
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              hi[i] = v[i];
              lo[i] = 0.f;
            }
          }
          if (!last) {
            tc::tmem_st16(lane_base + df_hi + (uint32_t)c, hi);
            tc::tmem_st16(lane_base + df_lo + (uint32_t)c, lo);
            continue;
          }
          if (m >= q.M) continue;
          // beta C: the chunk's 16 loads issued together, ahead of the stores
          double cin[16];
          if (q.beta != 0.0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int nn = w.n0 + c + i;
              cin[i] = (nn < q.N && !(q.lower && nn > m)) ? Cb[m + q.ldc * nn] : 0.0;
            }
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int nn = w.n0 + c + i;
            if (nn >= q.N || (q.lower && nn > m)) break;  // lower: the lower triangle, mirrored
            const double vd = gr > 0 ? tc::f2d(hi[i]) + tc::f2d(lo[i]) : tc::f2d(hi[i]);
            double o = q.alpha == 1.0 ? vd : q.alpha * vd;
            if (q.beta != 0.0) o += q.beta * cin[i];
            Cb[m + q.ldc * nn] = o;
            if (q.lower && nn < m) Cb[nn + q.ldc * m] = o;
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&tempty[buf]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, tcols);
}

// ------------------------------------------------------------ host side

namespace {

PFN_cuTensorMapEncodeTiled_v12000 gb_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2-D map over a row-major BF16 slice array (rows x kp), box 64 x 128, 128-byte swizzle
cudaError_t gb_map(CUtensorMap* m, const __nv_bfloat16* base, int kp, long long rows) {
  auto fn = gb_encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) || (kp % 8)) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)GB_BK, (cuuint32_t)GB_BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

size_t tc_grouped_workspace_bytes(int nprob) {
  return (size_t)nprob * 2 * sizeof(CUtensorMap) + (size_t)nprob * sizeof(GbProblem) + 256;
}

cudaError_t tc_gemm_f64_grouped(const TcGroupProblem* probs, int nprob, void* dev_work, size_t work_bytes,
                                std::vector<unsigned char>& staged, int num_sms, unsigned* status, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  if (nprob > 32 || !dev_work || work_bytes < tc_grouped_workspace_bytes(nprob)) return cudaErrorInvalidValue;
  const int s = probs[0].A.s;
  // descriptors: the maps first (64-byte aligned), then the problems, then the queue counter
  std::vector<unsigned char> host(tc_grouped_workspace_bytes(nprob), 0);
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(host.data());
  GbProblem* pr = reinterpret_cast<GbProblem*>(host.data() + (size_t)nprob * 2 * sizeof(CUtensorMap));
  long long units = 0;
  double mma = 0.0;
  for (int i = 0; i < nprob; ++i) {
    const TcGroupProblem& p = probs[i];
    if (p.A.s != s || p.B.s != s || p.A.kp != p.B.kp || p.A.kp % GB_BK || p.bt.count <= 0 || p.M <= 0 || p.N <= 0 ||
        (p.lower && p.M != p.N))
      return cudaErrorInvalidValue;
    const long long arows = (long long)p.A.rows_pad * s + (long long)p.bt.a_rows * (p.bt.count - 1);
    const long long brows = (long long)p.B.rows_pad * s + (long long)p.bt.b_rows * (p.bt.count - 1);
    cudaError_t e = gb_map(&maps[2 * i], p.A.p, p.A.kp, arows);
    if (e == cudaSuccess) e = gb_map(&maps[2 * i + 1], p.B.p, p.B.kp, brows);
    if (e != cudaSuccess) return e;
    GbProblem& q = pr[i];
    q.M = p.M;
    q.N = p.N;
    q.k_iters = p.A.kp / GB_BK;
    q.tiles_m = (p.M + GB_BM - 1) / GB_BM;
    q.tiles_n = (p.N + GB_BN - 1) / GB_BN;
    q.lower = p.lower ? 1 : 0;
    q.count = p.bt.count;
    q.s = s;
    q.a_rows_pad = p.A.rows_pad;
    q.b_rows_pad = p.B.rows_pad;
    q.a_brows = p.bt.a_rows;
    q.b_brows = p.bt.b_rows;
    q.c_bstride = p.bt.c_stride;
    q.ldc = p.ldc;
    q.alpha = p.alpha;
    q.beta = p.beta;
    q.C = p.C;
    const long long tiles = q.lower ? (long long)q.tiles_m * (q.tiles_m + 1) / 2 : (long long)q.tiles_m * q.tiles_n;
    q.unit_begin = units;
    q.units = tiles * q.count;
    units += q.units;
    const double prods = 0.5 * s * (s + 1);
    mma += 2.0 * prods * (p.lower ? 0.5 * (double)p.M * (p.M + 1) : (double)p.M * p.N) * (double)p.A.kp * q.count;
  }
  const size_t qoff = tc_grouped_workspace_bytes(nprob) - 256;  // the queue counter's offset
  // upload unless the device already holds exactly these descriptors (a
  // captured graph replays the upload of the eager call before it)
  if (staged != host) {
    if (tl_capture) return cudaErrorStreamCaptureUnsupported;
    cudaError_t e = cudaMemcpyAsync(dev_work, host.data(), qoff, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);  // the host vector is a local
    if (e != cudaSuccess) return e;
    staged = host;
  }
  unsigned long long* queue = reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(dev_work) + qoff);
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  static bool configured = false;
  const int smem = gb_stages(s) * gb_stage_bytes(s) + 1024 + 256;
  if (!configured) {
    e = cudaFuncSetAttribute(k_tc_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, GB_SMEM_LIMIT - 8192);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (smem > GB_SMEM_LIMIT - 8192) return cudaErrorInvalidValue;
  GbArgs a;
  a.prob = reinterpret_cast<const GbProblem*>(static_cast<unsigned char*>(dev_work) +
                                              (size_t)nprob * 2 * sizeof(CUtensorMap));
  a.maps = reinterpret_cast<const CUtensorMap*>(dev_work);
  a.nprob = nprob;
  a.units = units;
  a.queue = queue;
  a.group = tl_tc_group;
  a.s = s;
  a.status = status;
  const int grid = (int)std::min<long long>(units, std::max(1, num_sms - std::max(0, tl_tc_sm_reserve)));
  KernelTimer kt(KF_TC_GEMM, st, mma);
  note_launch();
  k_tc_grouped<<<grid, GB_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace isdf
