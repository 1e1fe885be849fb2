// Dense filter product on the 5th-generation tensor cores (tcgen05), with the Chebyshev
// recurrence of Algorithm 3 (or Algorithm 2) fused into the epilogue:
//   out = a * (A R_Y) + b * R_Y + c * R_X + a * W diag(Lambda_Y)
//
// One CTA computes a 128 x BN output tile (BN <= 256, the whole block width when N <= 256) over a
// slice of K.  Warp roles: warp 0 issues TMA loads of 128-byte-swizzled K-major tiles of A and R_Y
// into a 4-stage shared-memory ring; warp 1 (one elected lane) issues tcgen05.mma (M = 128, N = BN,
// K = 8 for TF32 / 16 for BF16) accumulating in TMEM and releases ring slots with tcgen05.commit;
// warps 2-5 read the accumulator back with tcgen05.ld (each warp owns its 32-lane TMEM quarter, one
// output row per thread) and apply the epilogue with coalesced column-major stores.  When the
// output has fewer tiles than the GPU has SMs, K is split across CTAs (split-K) so that every SM
// streams a share of A; partial tiles go to a workspace and a second, memory-bound kernel sums them
// and applies the recurrence.  Every mbarrier wait is bounded (an error flag is raised instead of
// hanging) and TMEM is always released.
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <type_traits>

#include "tc_gemm.cuh"
#include "tc_ptx.cuh"
#include "prof.cuh"

namespace rchfsi {
namespace {

constexpr int kStages = 4;
constexpr int kThreads = 192;
constexpr int kBM = 128;
constexpr int kRowBytes = 128;  // one swizzle atom row: 32 FP32 or 64 BF16 elements

template <typename T>
struct Epi {
  float a, b, c;
  const T* Ry;
  const T* Rx;
  const T* W;
  const double* lam;
  T* out;
  int64_t ld;  // leading dimension of out / Ry / Rx / W (column-major)
};

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ void from_f(float& d, float v) { d = v; }
__device__ __forceinline__ void from_f(__nv_bfloat16& d, float v) { d = __float2bfloat16_rn(v); }

// lam_a = a lam[col] in FP32, formed once per column by the caller (an FP64 conversion per element
// would occupy the FP64 pipe).
template <typename T>
__device__ __forceinline__ void apply_epi(const Epi<T>& e, int64_t row, int64_t col, float acc, float lam_a) {
  const int64_t o = col * e.ld + row;
  float v = e.a * acc + e.b * to_f(e.Ry[o]);
  if (e.Rx) v += e.c * to_f(e.Rx[o]);
  if (e.W) v += to_f(e.W[o]) * lam_a;
  from_f(e.out[o], v);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                   int K, int BN, uint32_t tmem_cols, int kb_per_split, float* __restrict__ ws, Epi<T> ep,
                   int* __restrict__ err) {
  constexpr bool kBF16 = std::is_same<T, __nv_bfloat16>::value;
  constexpr int BK = kRowBytes / (int)sizeof(T);
  constexpr int KMMA = kBF16 ? 16 : 8;
  constexpr uint32_t kFmt = kBF16 ? 1u : 2u;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], acc_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int consumed;
  __shared__ float s_lam[256];  // a lam_j of the tile's columns (BN <= 256)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN, split = blockIdx.z;
  const int nkb_total = (K + BK - 1) / BK;
  const int kb_begin = split * kb_per_split;
  const int nkb = min(nkb_total, kb_begin + kb_per_split) - kb_begin;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t a_bytes = kBM * kRowBytes;
  const uint32_t b_bytes = (uint32_t)BN * kRowBytes;
  const uint32_t stage_bytes = a_bytes + b_bytes;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&empty_bar[s], 1);
    }
    tc::mbar_init(&acc_bar, 1);
    tc::fence_barrier_init();
    abort_flag = 0;
    consumed = 0;
    tc::prefetch_tmap(&mapA);
    tc::prefetch_tmap(&mapB);
  }
  if (ep.W && !ws)
    for (int j = threadIdx.x; j < BN; j += blockDim.x) s_lam[j] = n0 + j < N ? (float)((double)ep.a * ep.lam[n0 + j]) : 0.f;
  if (warp == 1) {
    tc::tmem_alloc(&tmem_slot, tmem_cols);
    tc::tmem_relinquish();
    tc::tc_fence_before();
  }
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* vabort = &abort_flag;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int issued = 0;
    for (int i = 0; i < nkb; ++i) {
      if (*vabort) break;
      const int s = i % kStages;
      const uint32_t ph = (uint32_t)(i / kStages) & 1u;
      if (!tc::mbar_wait(&empty_bar[s], ph ^ 1u)) {
        *vabort = 1;
        atomicExch(err, 1);
        break;
      }
      uint8_t* sa = smem + (size_t)s * stage_bytes;
      uint8_t* sb = sa + a_bytes;
      tc::mbar_arrive_expect_tx(&full_bar[s], stage_bytes);
      const int k0 = (kb_begin + i) * BK;
      tc::tma_load_2d(sa, &mapA, &full_bar[s], k0, m0);
      tc::tma_load_2d(sb, &mapB, &full_bar[s], k0, n0);
      ++issued;
    }
    if (*vabort) {
      // let the loads already in flight land before the CTA exits (bounded)
      for (int i = *(volatile int*)&consumed; i < issued; ++i)
        tc::mbar_wait(&full_bar[i % kStages], (uint32_t)(i / kStages) & 1u);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: the whole warp walks the loop with warp-uniform values, one
    // elected lane issues
    const bool leader = tc::elect_one();
    const uint32_t idesc = tc::instr_desc(kFmt, kBM, BN);
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      const uint32_t ph = (uint32_t)(i / kStages) & 1u;
      const bool w = !*vabort && tc::mbar_wait(&full_bar[s], ph);
      if (!__all_sync(0xffffffffu, w)) {
        if (leader) {
          *vabort = 1;
          atomicExch(err, 1);
        }
        ok = false;
        break;
      }
      if (leader) *(volatile int*)&consumed = i + 1;
      tc::tc_fence_after();
      const uint32_t a_base = tc::smem_u32(smem + (size_t)s * stage_bytes);
      const uint64_t a0 = tc::sw128_desc(a_base), b0 = tc::sw128_desc(a_base + a_bytes);
#pragma unroll
      for (int kk = 0; kk < BK / KMMA; ++kk) {
        const uint64_t ad = tc::desc_add(a0, kk * 32);
        const uint64_t bd = tc::desc_add(b0, kk * 32);
        if (leader) {
          if (kBF16) tc::mma_f16(tmem, ad, bd, idesc, (i > 0 || kk > 0) ? 1u : 0u);
          else tc::mma_tf32(tmem, ad, bd, idesc, (i > 0 || kk > 0) ? 1u : 0u);
        }
      }
      __syncwarp();
      if (leader) tc::mma_commit(&empty_bar[s]);
      __syncwarp();
    }
    if (ok && leader) tc::mma_commit(&acc_bar);
  } else if (warp >= 2) {
    // ---------------- epilogue: TMEM -> registers -> global
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    bool ok = tc::mbar_wait(&acc_bar, 0);
    if (!ok) {
      *vabort = 1;
      atomicExch(err, 1);
    }
    // tcgen05.ld is warp-collective: decide and proceed as a converged warp
    ok = __all_sync(0xffffffffu, ok && !*vabort);
    if (ok) {
      tc::tc_fence_after();
      const int64_t row = (int64_t)m0 + q * 32 + lane;
      const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tc::tmem_ld16(lane_addr + c0, v);
        if (row < M) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int64_t col = (int64_t)n0 + c0 + t;
            if (col < N) {
              if (ws) ws[((int64_t)split * N + col) * M + row] = v[t];
              else apply_epi(ep, row, col, v[t], ep.W ? s_lam[c0 + t] : 0.f);
            }
          }
        }
      }
    }
    tc::tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, tmem_cols);
  }
}

template <typename T>
__global__ void splitk_reduce_kernel(int M, int N, int nsplit, const float* __restrict__ ws, Epi<T> ep) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / M, row = e - col * M;
    float acc = 0.f;
    for (int s = 0; s < nsplit; ++s) acc += ws[(int64_t)s * total + e];
    apply_epi(ep, row, col, acc, ep.W ? ep.a * (float)ep.lam[col] : 0.f);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    RC_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    RC_CHECK(q == cudaDriverEntryPointSuccess && p, RCHFSI_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2D map over a matrix with `inner` contiguous elements per row (K) and `outer` rows, row pitch
// `ld` elements; box = 128 bytes x box_rows, 128-byte swizzle, zero fill out of bounds.
CUtensorMap make_map(const void* base, bool bf16, int64_t inner, int64_t outer, int64_t ld, int box_rows) {
  CUtensorMap m;
  const size_t es = bf16 ? 2 : 4;
  RC_CHECK(((uintptr_t)base & 15) == 0, RCHFSI_ERR_INVALID_ARG, "TMA base must be 16-byte aligned");
  RC_CHECK((ld * es) % 16 == 0, RCHFSI_ERR_INVALID_ARG, "TMA row pitch must be a multiple of 16 bytes");
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
  cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                           const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  RC_CHECK(r == CUDA_SUCCESS, RCHFSI_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

struct Plan {
  int BN, n_tiles, m_tiles, nsplit, kb_per_split;
  uint32_t tmem_cols;
  size_t smem;
};

Plan make_plan(int num_sms, int64_t M, int64_t N, int64_t K, int BK) {
  Plan p;
  p.n_tiles = (int)((N + 255) / 256);
  const int64_t per = (N + p.n_tiles - 1) / p.n_tiles;
  p.BN = (int)(((per + 15) / 16) * 16);
  p.m_tiles = (int)((M + kBM - 1) / kBM);
  const int tiles = p.m_tiles * p.n_tiles;
  const int nkb = (int)((K + BK - 1) / BK);
  int ns = std::max(1, num_sms / std::max(tiles, 1));
  ns = std::min(ns, nkb);
  p.kb_per_split = (nkb + ns - 1) / ns;
  p.nsplit = (nkb + p.kb_per_split - 1) / p.kb_per_split;
  uint32_t cols = 32;
  while (cols < (uint32_t)p.BN) cols <<= 1;
  p.tmem_cols = cols;
  p.smem = (size_t)kStages * (kBM * kRowBytes + (size_t)p.BN * kRowBytes) + 1024;
  return p;
}

template <typename T>
void run(cudaStream_t s, int num_sms, int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, const T* B,
         int64_t ldb, DevBuf<float>& split, const Epi<T>& ep, int* err) {
  constexpr bool bf = std::is_same<T, __nv_bfloat16>::value;
  constexpr int BK = kRowBytes / (int)sizeof(T);
  RC_CHECK(M > 0 && N > 0 && K > 0, RCHFSI_ERR_INVALID_ARG, "tensor-core GEMM with an empty dimension");
  RC_CHECK(M < (1LL << 31) && N < (1LL << 31) && K < (1LL << 31), RCHFSI_ERR_INVALID_ARG, "GEMM too large");
  const Plan p = make_plan(num_sms, M, N, K, BK);
  const CUtensorMap ma = make_map(A, bf, K, M, lda, kBM);
  const CUtensorMap mb = make_map(B, bf, K, N, ldb, p.BN);
  set_smem_limit(reinterpret_cast<const void*>(tc_gemm_kernel<T>), 232448 - 4096);
  float* ws = nullptr;
  if (p.nsplit > 1) ws = split.ensure((size_t)p.nsplit * M * N);
  dim3 grid(p.m_tiles, p.n_tiles, p.nsplit);
  const double es = sizeof(T);
  const double epi_streams = 2.0 + (ep.Rx ? 1 : 0) + (ep.W ? 1 : 0);  // Ry, out, [Rx], [W]
  {
    // algorithmic bytes: A and R_Y once, plus the epilogue streams (direct) or the partials (split-K)
    const double out_bytes = p.nsplit > 1 ? 4.0 * p.nsplit * M * N : epi_streams * es * M * N;
    prof::Scope ps(s, RCHFSI_KERNEL_FILTER_TC, 2.0 * M * N * K, es * ((double)M * K + (double)K * N) + out_bytes);
    tc_gemm_kernel<T><<<grid, kThreads, p.smem, s>>>(ma, mb, (int)M, (int)N, (int)K, p.BN, p.tmem_cols,
                                                      p.kb_per_split, ws, ep, err);
    RC_LAUNCH();
  }
  if (p.nsplit > 1) {
    const int64_t total = M * N;
    int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8);
    prof::Scope ps(s, RCHFSI_KERNEL_SPLITK_REDUCE, (double)p.nsplit * M * N,
                   4.0 * p.nsplit * M * N + epi_streams * es * M * N);
    splitk_reduce_kernel<T><<<(unsigned)blocks, 256, 0, s>>>((int)M, (int)N, p.nsplit, ws, ep);
    RC_LAUNCH();
  }
}

}  // namespace

void* tensor_map_encoder() { return reinterpret_cast<void*>(encode_fn()); }

void tc_gemm_tf32_recur(cudaStream_t s, int num_sms, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                        const float* B, int64_t ldb, DevBuf<float>& split, const TcRecur& r, int64_t ldo, int* err) {
  Epi<float> e{r.a, r.b, r.c, r.Ry, r.Rx, r.W, r.lam, r.out, ldo};
  run<float>(s, num_sms, M, N, K, A, lda, B, ldb, split, e, err);
}

void tc_gemm_bf16_recur(cudaStream_t s, int num_sms, int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A,
                        int64_t lda, const __nv_bfloat16* B, int64_t ldb, DevBuf<float>& split, const TcRecur16& r,
                        int64_t ldo, int* err) {
  Epi<__nv_bfloat16> e{r.a, r.b, r.c, r.Ry, r.Rx, r.W, r.lam, r.out, ldo};
  run<__nv_bfloat16>(s, num_sms, M, N, K, A, lda, B, ldb, split, e, err);
}

size_t tc_gemm_tf32_split_floats(int num_sms, int64_t M, int64_t N, int64_t K) {
  const Plan p = make_plan(num_sms, M, N, K, kRowBytes / 4);
  return p.nsplit > 1 ? (size_t)p.nsplit * M * N : 0;
}

void tc_gemm_tf32_recur_ws(cudaStream_t s, int num_sms, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                           const float* B, int64_t ldb, float* ws, size_t ws_floats, const TcRecur& r, int64_t ldo,
                           int* err) {
  // The launch sequence of run<float>() with caller-provided storage for the split-K partials.
  constexpr int BK = kRowBytes / 4;
  RC_CHECK(M > 0 && N > 0 && K > 0, RCHFSI_ERR_INVALID_ARG, "tensor-core GEMM with an empty dimension");
  RC_CHECK(M < (1LL << 31) && N < (1LL << 31) && K < (1LL << 31), RCHFSI_ERR_INVALID_ARG, "GEMM too large");
  const Plan p = make_plan(num_sms, M, N, K, BK);
  RC_CHECK(p.nsplit == 1 || (size_t)p.nsplit * M * N <= ws_floats, RCHFSI_ERR_INVALID_ARG,
           "split-K partials need " + std::to_string((size_t)p.nsplit * M * N) + " floats, scratch holds " +
               std::to_string(ws_floats));
  const CUtensorMap ma = make_map(A, false, K, M, lda, kBM);
  const CUtensorMap mb = make_map(B, false, K, N, ldb, p.BN);
  set_smem_limit(reinterpret_cast<const void*>(tc_gemm_kernel<float>), 232448 - 4096);
  Epi<float> ep{r.a, r.b, r.c, r.Ry, r.Rx, r.W, r.lam, r.out, ldo};
  float* w = p.nsplit > 1 ? ws : nullptr;
  dim3 grid(p.m_tiles, p.n_tiles, p.nsplit);
  tc_gemm_kernel<float><<<grid, kThreads, p.smem, s>>>(ma, mb, (int)M, (int)N, (int)K, p.BN, p.tmem_cols,
                                                        p.kb_per_split, w, ep, err);
  RC_LAUNCH();
  if (p.nsplit > 1) {
    const int64_t total = M * N;
    int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8);
    splitk_reduce_kernel<float><<<(unsigned)blocks, 256, 0, s>>>((int)M, (int)N, p.nsplit, w, ep);
    RC_LAUNCH();
  }
}

}  // namespace rchfsi
