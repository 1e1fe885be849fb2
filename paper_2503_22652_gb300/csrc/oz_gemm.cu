// FP64-accurate products from BF16 tensor-core slices (see oz_gemm.cuh for the scheme).
//
// oz_gemm_kernel<BN>: one CTA per 128 x BN output tile (BN = 32 or 64) and K range.  Warp 0 (one
// lane) streams, per 64-wide K chunk, the 7 B slices of the tile (one 28 / 56 KB stage, two stages)
// and the 7 A slices (16 KB each, a 6-deep ring) with TMA; warp 1 (the whole warp, one elected lane
// issuing) runs, for each A slice s, the products with B slices t <= 6 - s (4 x tcgen05.mma
// kind::f16, K = 16) into the TMEM accumulator of level s + t (7 levels x BN columns: two buffers
// for BN = 32, one for BN = 64, 448 columns either way), accumulating GROUP chunks per buffer;
// warps 4-11 (two per TMEM lane quarter, BN / 2 columns each) drain a finished group: tcgen05.ld of
// the 7 levels, exact scaling by 2^-8L and TwoSum into per-output float-float accumulators.  The
// final value (hi + lo) 2^(e_i + f_j - 16), formed by exponent arithmetic, is stored in FP64 (or,
// with split-K, written as a partial and summed by a second kernel).  The host picks BN and the
// split from the padded columns, the MMA rate (48 clocks per 128 x 64 x 16 MMA, 40 per 128 x 32 x
// 16) and the wave fill.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "oz_gemm.cuh"
#include "oz_digits.cuh"
#include "prof.cuh"
#include "tc_ptx.cuh"

namespace rchfsi {
namespace {

constexpr int S = kOzSlices;
constexpr int BM = 128;
constexpr int KC = 64;            // K chunk: one 128-byte row of BF16
// Chunks accumulated in TMEM before a drain: 2 x 64 = 128 K terms per exact FP32 sum (each term a
// product of two integer slices, |t_s t_r| <= 2^16, so every partial sum stays below 2^23).
constexpr int GROUP = 2;
constexpr int ASTAGES = 6;
constexpr int kThreads = 384;     // 12 warps
constexpr uint32_t kABytes = BM * 128;       // 16 KB per A slice tile
constexpr uint32_t kTmemCols = 512;          // 7 levels x 32 columns x 2 buffers, or x 64 x 1 = 448
// Output tile BM x BN: BN = 32 with two TMEM accumulator buffers (the drain of one group overlaps
// the products of the next), or BN = 64 with one (each MMA carries twice the columns for 4/3 of the
// shared-memory operand traffic; the MMAs wait for each drain).
template <int BN>
struct OzTile {
  static constexpr int NBUF = BN == 32 ? 2 : 1;
  static constexpr uint32_t kBBytes = S * BN * 128;  // all B slices of one chunk: 28 / 56 KB
};

// ---------------------------------------------------------------- slicing
// Row exponents, K-contiguous rows: one warp per (row, K slice), the K range split over
// blockIdx.y so that a few hundred rows still fill the GPU; slices meet in ex by atomicMax (ex
// preset to INT_MIN), rowexp_fix maps rows without a nonzero element to 0.
__global__ void rowexp_kcontig(int64_t R, int64_t K, const double* __restrict__ X, int64_t rs, int* ex) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (r >= R) return;
  const int64_t kb = (K + gridDim.y - 1) / gridDim.y, k0 = (int64_t)blockIdx.y * kb;
  const int64_t k1 = k0 + kb < K ? k0 + kb : K;
  int e = -100000;
  for (int64_t k = k0 + lane; k < k1; k += 32) e = max(e, exp_of(X[r * rs + k]));
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (lane == 0) atomicMax(ex + r, e);
}

// Row exponents, rows contiguous across threads (element (r, k) at X[r + k * ks]): 32 rows per
// block (coalesced), the K range split over the block's 8 warps and over blockIdx.y.  Partial maxima
// meet in ex by atomicMax (ex preset to INT_MIN); rowexp_fix then maps rows without a nonzero
// element to 0.
__global__ void __launch_bounds__(256) rowexp_rcontig(int64_t R, int64_t K, const double* __restrict__ X, int64_t ks,
                                                      int* ex) {
  __shared__ int red[8][32];
  const int64_t r = (int64_t)blockIdx.x * 32 + threadIdx.x;
  int e = -100000;
  if (r < R)
    for (int64_t k = threadIdx.y + 8 * (int64_t)blockIdx.y; k < K; k += 8 * (int64_t)gridDim.y)
      e = max(e, exp_of(X[r + k * ks]));
  red[threadIdx.y][threadIdx.x] = e;
  __syncthreads();
  if (threadIdx.y == 0 && r < R) {
#pragma unroll
    for (int y = 1; y < 8; ++y) e = max(e, red[y][threadIdx.x]);
    atomicMax(ex + r, e);
  }
}

__global__ void rowexp_fix(int64_t R, int* ex) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R && ex[r] <= -100000) ex[r] = 0;
}

// Slices of a 32-row x 64-k tile.  Block (32, 8).
__global__ void slice_kernel(int64_t R, int64_t Rp, int64_t K, int64_t Kp, const double* __restrict__ X, int64_t rs,
                             int64_t ks, const int* __restrict__ ex, __nv_bfloat16* __restrict__ out) {
  __shared__ double tile[32][KC + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t r0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * KC;
  if (ks == 1) {
    for (int rr = ty; rr < 32; rr += 8)
      for (int kk = tx; kk < KC; kk += 32) {
        const int64_t r = r0 + rr, k = k0 + kk;
        tile[rr][kk] = (r < R && k < K) ? X[r * rs + k] : 0.0;
      }
  } else {
    for (int kk = ty; kk < KC; kk += 8) {
      const int64_t r = r0 + tx, k = k0 + kk;
      tile[tx][kk] = (r < R && k < K) ? X[r * rs + k * ks] : 0.0;
    }
  }
  __syncthreads();
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t r = r0 + rr;
    if (r >= R) continue;
    const int e = ex[r];
    // digits t_s of x 2^(-e) = sum_s t_s 2^(-8(s+1)), rounded to nearest: |t_0| <= 256, |t_s| <= 128,
    // each exact in BF16; two neighbouring k per thread, stored as one 4-byte pair per slice
    long long f0 = fixed56(tile[rr][2 * tx], e), f1 = fixed56(tile[rr][2 * tx + 1], e);
    __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(out + (int64_t)r * Kp + k0 + 2 * tx);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int sh = 48 - 8 * s;
      long long t0 = f0, t1 = f1;
      if (sh > 0) {
        t0 = (f0 + (1LL << (sh - 1))) >> sh;
        t1 = (f1 + (1LL << (sh - 1))) >> sh;
        f0 -= t0 << sh;
        f1 -= t1 << sh;
      }
      // digits fit in 32 bits (|t| <= 256): an int conversion stays off the FP64 pipe, which a
      // 64-bit integer conversion occupies (a few DFMA per clock per SM on this GPU)
      o2[(int64_t)s * Rp * Kp / 2] = __floats2bfloat162_rn((float)(int)t0, (float)(int)t1);
    }
  }
}

// ---------------------------------------------------------------- the product
struct OzArgs {
  int M, N;
  int MP, NP;      // rows per slice in the A and B slice tensors
  int chunks_per_split, nchunks;
  const int* ea;
  const int* eb;
  double* C;       // final output (nsplit == 1) or partials [split][N][M]
  int64_t ldc;
  int partial;
  int upper;       // only tiles that reach the upper triangle (i <= j) are computed
  int* err;
};

__device__ __forceinline__ void two_sum(float& hi, float& lo, float b) {
  const float s = hi + b;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (b - bb);
  hi = s;
  lo += e;
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, OzArgs p) {
  constexpr int NBUF = OzTile<BN>::NBUF;
  constexpr uint32_t kBBytes = OzTile<BN>::kBBytes;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t afull[ASTAGES], aempty[ASTAGES], bfull[2], bempty[2], accfull[2], accempty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM, split = blockIdx.z;
  if (p.upper && m0 >= n0 + BN) return;  // strictly below the diagonal: mirrored afterwards
  const int c_begin = split * p.chunks_per_split;
  const int nch = min(p.nchunks, c_begin + p.chunks_per_split) - c_begin;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;                                  // ASTAGES x 16 KB
  uint8_t* sB = smem + (size_t)ASTAGES * kABytes;      // 2 x 28 KB

  if (threadIdx.x == 0) {
    for (int i = 0; i < ASTAGES; ++i) {
      tc::mbar_init(&afull[i], 1);
      tc::mbar_init(&aempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&bfull[i], 1);
      tc::mbar_init(&bempty[i], 1);
      tc::mbar_init(&accfull[i], 1);
      tc::mbar_init(&accempty[i], 256);
    }
    tc::fence_barrier_init();
    abort_flag = 0;
    tc::prefetch_tmap(&mapA);
    tc::prefetch_tmap(&mapB);
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_slot, kTmemCols);
    tc::tmem_relinquish();
    tc::tc_fence_before();
  }
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* vabort = &abort_flag;
  auto fail = [&]() {
    *vabort = 1;
    atomicExch(p.err, 1);
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      for (int ci = 0; ci < nch; ++ci) {
        const int k0 = (c_begin + ci) * KC;
        const int b = ci & 1;
        if (*vabort || !tc::mbar_wait(&bempty[b], (uint32_t)((ci >> 1) & 1) ^ 1u)) {
          fail();
          break;
        }
        tc::mbar_arrive_expect_tx(&bfull[b], kBBytes);
        for (int t = 0; t < S; ++t)
          tc::tma_load_2d(sB + (size_t)b * kBBytes + (size_t)t * BN * 128, &mapB, &bfull[b], k0, t * p.NP + n0);
        bool ok = true;
        for (int s = 0; s < S; ++s) {
          const int j = ci * S + s;
          const int q = j % ASTAGES;
          if (*vabort || !tc::mbar_wait(&aempty[q], (uint32_t)((j / ASTAGES) & 1) ^ 1u)) {
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&afull[q], kABytes);
          tc::tma_load_2d(sA + (size_t)q * kABytes, &mapA, &afull[q], k0, s * p.MP + m0);
        }
        if (!ok) {
          fail();
          break;
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: the whole warp walks the fully unrolled (s, t, k) sequence with
    // warp-uniform values, one elected lane issues
    const bool leader = tc::elect_one();
    const uint32_t idesc = tc::instr_desc(1u, BM, BN);  // BF16 x BF16 -> FP32, M = 128
    bool ok = true;
    for (int ci = 0; ci < nch && ok; ++ci) {
      const int b = ci & 1;
      const int g = ci / GROUP, xb = g % NBUF;  // accumulation group and its TMEM buffer
      const bool first = (ci % GROUP) == 0, last = (ci % GROUP) == GROUP - 1 || ci == nch - 1;
      bool w = !*vabort && tc::mbar_wait(&bfull[b], (uint32_t)((ci >> 1) & 1));
      if (w && first) w = tc::mbar_wait(&accempty[xb], (uint32_t)((g / NBUF) & 1) ^ 1u);
      ok = __all_sync(0xffffffffu, w);
      if (!ok) break;
      const uint64_t b_desc = tc::sw128_desc(tc::smem_u32(sB + (size_t)b * kBBytes));
      const uint32_t d_base = tmem + (uint32_t)(xb * S * BN);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int j = ci * S + s;
        const int q = j % ASTAGES;
        w = !*vabort && tc::mbar_wait(&afull[q], (uint32_t)((j / ASTAGES) & 1));
        ok = __all_sync(0xffffffffu, w);
        if (!ok) break;
        tc::tc_fence_after();
        // base descriptors plus compile-time offsets: a few integer adds per MMA
        const uint64_t a0 = tc::sw128_desc(tc::smem_u32(sA + (size_t)q * kABytes));
#pragma unroll
        for (int t = 0; t < S - s; ++t) {
          const uint32_t d = d_base + (uint32_t)((s + t) * BN);
          const uint64_t b0 = tc::desc_add(b_desc, (uint32_t)(t * BN * 128));
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            if (leader)
              tc::mma_f16(d, tc::desc_add(a0, kk * 32), tc::desc_add(b0, kk * 32), idesc,
                          (first && s == 0 && kk == 0) ? 0u : 1u);
        }
        __syncwarp();
        if (leader) tc::mma_commit(&aempty[q]);
        __syncwarp();
      }
      if (!ok) break;
      if (leader) {
        tc::mma_commit(&bempty[b]);
        if (last) tc::mma_commit(&accfull[xb]);
      }
      __syncwarp();
    }
    if (!ok && leader) fail();
  } else if (warp >= 4) {
    // ---------------- epilogue: 8 warps, lane quarter q, column half h (BN / 2 columns each)
    constexpr int HC = BN / 2;
    const int q = warp & 3, h = (warp - 4) >> 2;
    float hi[HC], lo[HC];
#pragma unroll
    for (int u = 0; u < HC; ++u) hi[u] = lo[u] = 0.f;
    bool ok = true;
    const int ngroups = (nch + GROUP - 1) / GROUP;
    for (int g = 0; g < ngroups; ++g) {
      const int b = g % NBUF;
      bool w = !*vabort && tc::mbar_wait(&accfull[b], (uint32_t)((g / NBUF) & 1));
      if (!w) fail();
      if (!__all_sync(0xffffffffu, w && !*vabort)) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * S * BN + h * HC);
      float scale = 1.f;
#pragma unroll 1
      for (int L = 0; L < S; ++L) {
#pragma unroll
        for (int c = 0; c < HC / 16; ++c) {
          float v[16];
          tc::tmem_ld16(base + (uint32_t)(L * BN + c * 16), v);
#pragma unroll
          for (int u = 0; u < 16; ++u) two_sum(hi[c * 16 + u], lo[c * 16 + u], v[u] * scale);
        }
        scale *= 0.00390625f;  // 2^-8
      }
      tc::tc_fence_before();
      tc::mbar_arrive(&accempty[b]);
    }
    if (ok) {
      const int64_t i = (int64_t)m0 + q * 32 + lane;
      if (i < p.M) {
        const int ei = p.ea[i];
#pragma unroll
        for (int u = 0; u < HC; ++u) {
          const int64_t jcol = (int64_t)n0 + h * HC + u;
          if (jcol < p.N) {
            // (hi + lo) 2^(e_i + f_j - 16): exact conversions by exponent arithmetic and one FP64 add
            const int pw = ei + p.eb[jcol] - 16;
            const double v = f32_scaled(hi[u], pw) + f32_scaled(lo[u], pw);
            if (p.partial) p.C[((int64_t)split * p.N + jcol) * p.M + i] = v;
            else p.C[jcol * p.ldc + i] = v;
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

__global__ void oz_sum_kernel(int64_t M, int64_t N, int nsplit, const double* __restrict__ part, double* C,
                              int64_t ldc) {
  const int64_t total = M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / M, i = e - j * M;
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += part[(int64_t)s * total + e];
    C[j * ldc + i] = acc;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    RC_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q));
    RC_CHECK(q == cudaDriverEntryPointSuccess && ptr, RCHFSI_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

// All slices of an operand as one 2D BF16 tensor: S*R rows of Kp elements.
CUtensorMap slice_map(const OzOperand& op, int box_rows) {
  CUtensorMap m;
  RC_CHECK(((uintptr_t)op.sl.p & 15) == 0 && (op.Kp * 2) % 16 == 0, RCHFSI_ERR_INVALID_ARG, "slice alignment");
  cuuint64_t dims[2] = {(cuuint64_t)op.Kp, (cuuint64_t)(S * op.Rp)};
  cuuint64_t strides[1] = {(cuuint64_t)(op.Kp * 2)};
  cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)op.sl.p, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  RC_CHECK(r == CUDA_SUCCESS, RCHFSI_ERR_CUDA, "cuTensorMapEncodeTiled failed for a slice tensor");
  return m;
}

}  // namespace

namespace {
int sm_count() {
  static const int n = [] {
    int d = 0, c = 152;
    if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, d) != cudaSuccess)
      c = 152;
    return c;
  }();
  return n;
}
}  // namespace

void oz_slice(cudaStream_t s, int64_t R, int64_t K, const double* X, int64_t rs, int64_t ks, OzOperand& op) {
  RC_CHECK(R > 0 && K > 0, RCHFSI_ERR_INVALID_ARG, "oz_slice: empty operand");
  RC_CHECK(ks == 1 || rs == 1, RCHFSI_ERR_INVALID_ARG, "oz_slice: one of the strides must be 1");
  op.R = R;
  op.Rp = std::max<int64_t>(R, 32);  // the 128-row TMA box must fit in the S * Rp rows of the tensor
  op.K = K;
  op.Kp = (K + KC - 1) / KC * KC;
  op.sl.ensure((size_t)S * op.Rp * op.Kp);
  op.ex.ensure((size_t)R);
  prof::Scope ps(s, RCHFSI_KERNEL_RR_AUX, 0.0, 8.0 * R * K + 2.0 * S * op.Rp * op.Kp);
  if (op.Rp > R) RC_CUDA(cudaMemsetAsync(op.sl.p, 0, sizeof(__nv_bfloat16) * S * op.Rp * op.Kp, s));
  if (ks == 1) {
    // K slices of >= 256 elements, enough (row, slice) warps for ~16 per SM
    const unsigned rb = cdiv(R, 8);
    const unsigned kb = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(cdiv(K, 256), (int64_t)(sm_count() * 16 * 8) / std::max<int64_t>(R, 1)));
    RC_CUDA(cudaMemsetAsync(op.ex.p, 0x80, sizeof(int) * R, s));  // 0x80808080: below every exponent
    rowexp_kcontig<<<dim3(rb, kb), 256, 0, s>>>(R, K, X, rs, op.ex.p);
    RC_LAUNCH();
    rowexp_fix<<<cdiv(R, 256), 256, 0, s>>>(R, op.ex.p);
  } else {
    // enough blocks to fill the GPU a few times over, each warp walking at least 8 k
    const unsigned rb = cdiv(R, 32);
    const unsigned kb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(K, 64), (int64_t)(sm_count() * 16) / rb));
    RC_CUDA(cudaMemsetAsync(op.ex.p, 0x80, sizeof(int) * R, s));  // 0x80808080: below every exponent
    rowexp_rcontig<<<dim3(rb, kb), dim3(32, 8), 0, s>>>(R, K, X, ks, op.ex.p);
    RC_LAUNCH();
    rowexp_fix<<<cdiv(R, 256), 256, 0, s>>>(R, op.ex.p);
  }
  RC_LAUNCH();
  RC_CHECK(cdiv(R, 32) <= 65535u, RCHFSI_ERR_INVALID_ARG, "oz_slice: too many rows");
  dim3 grid((unsigned)(op.Kp / KC), cdiv(R, 32));
  slice_kernel<<<grid, dim3(32, 8), 0, s>>>(R, op.Rp, K, op.Kp, X, rs, ks, op.ex.p, op.sl.p);
  RC_LAUNCH();
}

namespace {

// Split-K count: the smallest with which the CTAs fill whole waves of one CTA per SM to >= 90%
// (else the best found), each split keeping >= 4 chunks so that its TMEM drains stay amortised.
int choose_split(int tiles, int nchunks, int num_sms, double* eff_out) {
  const int max_split = std::max(1, std::min(64, nchunks / 4));
  double best = -1.0;
  int nsplit = 1;
  for (int ns = 1; ns <= max_split; ++ns) {
    const int64_t ctas = (int64_t)tiles * ns;
    const int64_t waves = (ctas + num_sms - 1) / num_sms;
    const double eff = (double)ctas / (double)(waves * num_sms);
    if (eff > best + 1e-9) {
      best = eff;
      nsplit = ns;
    }
    if (eff >= 0.9) break;
  }
  *eff_out = best;
  return nsplit;
}

// C(i, j) = C(j, i) for i > j (column-major n x n)
__global__ void mirror_upper_kernel(int n, double* C, int64_t ldc) {
  const int64_t tot = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / n), i = (int)(t - (int64_t)j * n);
    if (i > j) C[(int64_t)j * ldc + i] = C[(int64_t)i * ldc + j];
  }
}

// Output tiles of a product that reach the upper triangle (all of them unless `upper`).
int kept_tiles(int m_tiles, int n_tiles, int BN, bool upper) {
  if (!upper) return m_tiles * n_tiles;
  int t = 0;
  for (int bm = 0; bm < m_tiles; ++bm)
    for (int bn = 0; bn < n_tiles; ++bn) t += (bm * BM < bn * BN + BN) ? 1 : 0;
  return t;
}

template <int BN>
void oz_gemm_launch(cudaStream_t s, int num_sms, const OzOperand& A, const OzOperand& B, double* C, int64_t ldc,
                    DevBuf<double>& ws, int* err, int nsplit_in, bool upper) {
  const int64_t M = A.R, N = B.R;
  const int m_tiles = (int)((M + BM - 1) / BM), n_tiles = (int)((N + BN - 1) / BN);
  const int nchunks = (int)(A.Kp / KC);
  int nsplit = nsplit_in;
  const int per = (nchunks + nsplit - 1) / nsplit;
  nsplit = (nchunks + per - 1) / per;
  RC_CHECK(m_tiles <= 65535 && nsplit <= 65535, RCHFSI_ERR_INVALID_ARG, "oz_gemm: grid too large");
  const CUtensorMap ma = slice_map(A, BM);
  const CUtensorMap mb = slice_map(B, BN);
  const size_t smem = (size_t)ASTAGES * kABytes + 2 * (size_t)OzTile<BN>::kBBytes + 1024;
  set_smem_limit(reinterpret_cast<const void*>(oz_gemm_kernel<BN>), (int)smem);
  OzArgs p;
  p.M = (int)M;
  p.N = (int)N;
  p.MP = (int)A.Rp;
  p.NP = (int)B.Rp;
  p.chunks_per_split = per;
  p.nchunks = nchunks;
  p.ea = A.ex.p;
  p.eb = B.ex.p;
  p.err = err;
  p.partial = nsplit > 1;
  p.upper = upper ? 1 : 0;
  if (nsplit > 1) {
    p.C = ws.ensure((size_t)nsplit * M * N);
    p.ldc = M;
  } else {
    p.C = C;
    p.ldc = ldc;
  }
  dim3 grid(n_tiles, m_tiles, nsplit);
  {
    // tensor-core flops of the 28 slice products; bytes: the slices once and the FP64 output
    // (a symmetric product computes the kept tiles only: the flops of those tiles)
    const double frac = (double)kept_tiles(m_tiles, n_tiles, BN, upper) / ((double)m_tiles * n_tiles);
    prof::Scope ps(s, RCHFSI_KERNEL_GEMM_F64_EMU, 2.0 * M * N * A.Kp * (S * (S + 1) / 2) * frac,
                   2.0 * S * (double)(M + N) * A.Kp + 8.0 * M * N);
    oz_gemm_kernel<BN><<<grid, kThreads, smem, s>>>(ma, mb, p);
    RC_LAUNCH();
  }
  if (nsplit > 1) {
    const int64_t total = M * N;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8);
    oz_sum_kernel<<<blocks, 256, 0, s>>>(M, N, nsplit, p.C, C, ldc);
    RC_LAUNCH();
  }
  if (upper) {
    const unsigned blocks = (unsigned)std::min<int64_t>((M * N + 255) / 256, (int64_t)num_sms * 4);
    mirror_upper_kernel<<<blocks, 256, 0, s>>>((int)M, C, ldc);
    RC_LAUNCH();
  }
}

}  // namespace

void oz_gemm(cudaStream_t s, int num_sms, const OzOperand& A, const OzOperand& B, double* C, int64_t ldc,
             DevBuf<double>& ws, int* err, bool symmetric) {
  RC_CHECK(A.K == B.K && A.Kp == B.Kp, RCHFSI_ERR_INVALID_ARG, "oz_gemm: K mismatch");
  const int64_t M = A.R, N = B.R;
  RC_CHECK(!symmetric || M == N, RCHFSI_ERR_INVALID_ARG, "oz_gemm: a symmetric product is square");
  RC_CHECK(M < (1LL << 31) && N < (1LL << 31), RCHFSI_ERR_INVALID_ARG, "oz_gemm: too large");
  const int m_tiles = (int)((M + BM - 1) / BM);
  const int nchunks = (int)(A.Kp / KC);
  // tile width: 64 unless its padded columns or its worse wave fill cost more than the wider MMAs
  // save (a 128 x 64 x 16 MMA takes 48 clocks, a 128 x 32 x 16 one 40: 1.67x the columns per clock)
  double e32 = 0.0, e64 = 0.0;
  const int t32 = kept_tiles(m_tiles, (int)((N + 31) / 32), 32, symmetric);
  const int t64 = kept_tiles(m_tiles, (int)((N + 63) / 64), 64, symmetric);
  const int s32 = choose_split(t32, nchunks, num_sms, &e32);
  const int s64 = choose_split(t64, nchunks, num_sms, &e64);
  const double c32 = (double)((N + 31) / 32 * 32) / 1.0 / std::max(e32, 1e-3);
  const double c64 = (double)((N + 63) / 64 * 64) / 1.67 / std::max(e64, 1e-3);
  if (c64 < c32)
    oz_gemm_launch<64>(s, num_sms, A, B, C, ldc, ws, err, s64, symmetric);
  else
    oz_gemm_launch<32>(s, num_sms, A, B, C, ldc, ws, err, s32, symmetric);
}

}  // namespace rchfsi
