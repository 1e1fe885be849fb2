// FP64-accurate products from BF16 tensor-core slices (see oz_gemm.cuh for the scheme).
//
// oz_gemm_kernel: persistent CTAs (one per SM) walking (128 x 64 output tile, K range) items.
// Warp 0 (one lane) streams, per 32-wide K chunk, the 7 A and the 7 B slices of the tile (8 KB and
// 4 KB each, 64-byte swizzle) into one 84 KB stage with TMA, two stages, one barrier per stage;
// warp 1 (the whole warp, one elected lane issuing) runs, for each A slice s, the products with B
// slices t <= 6 - s (2 x tcgen05.mma kind::f16, K = 16) into the TMEM accumulator of level s + t,
// GROUP chunks (128 K terms) per exact accumulation group.  TMEM holds 8 level blocks of 64 columns,
// 7 for the group and one spare, rotated so that the next group's first writes go to blocks in the
// order they are freed; warps 2-17 (four per TMEM lane quarter, 16 columns each) fold level L of a
// group as soon as the group's pass L is done: tcgen05.ld, exact scaling by 2^-8L and TwoSum into
// per-output float-float accumulators.  The final value (hi + lo) 2^(e_i + f_j - 16), formed by
// exponent arithmetic, is stored in FP64 (or, with split-K, written as a partial and summed by a
// second kernel) while the next item's MMAs run.  The host splits K only as far as the items fill the
// CTAs.
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
constexpr int KC = 64;            // K tile of the slicing kernel (K is padded to a multiple of it)
// Chunks accumulated in TMEM before a drain: 2 x 64 = 128 K terms per exact FP32 sum (each term a
// product of two integer slices, |t_s t_r| <= 2^16, so every partial sum stays below 2^23).
constexpr int KCH = 32;           // K chunk of the products: one 64-byte row of BF16 per slice
constexpr int GROUP = 4;          // chunks per exact accumulation group (4 x 32 = 128 K terms)
constexpr int NSTAGE = 2;
constexpr int BN = 64;            // output tile columns
constexpr int kThreads = 576;     // 18 warps: TMA producer, MMA issuer, 16 epilogue warps
constexpr int kEpiThreads = 512;
constexpr uint32_t kASlice = BM * 64;        // 8 KB per A slice of a chunk
constexpr uint32_t kBSlice = BN * 64;        // 4 KB per B slice of a chunk
constexpr uint32_t kStage = S * (kASlice + kBSlice);  // all 14 slices of one chunk: 84 KB
constexpr uint32_t kTmemCols = 512;          // 8 level blocks x 64 columns

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
  int n_tiles;     // column tiles
  int kept;        // output tiles computed (all, or those reaching the upper triangle)
  int64_t items;   // kept x splits
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

// Level blocks in TMEM: 8 blocks of 64 columns, 7 holding the levels of the current accumulation
// group and one spare.  perm packs, per level L = 0..6, its block (4 bits each; bits 28-31: the
// spare).  The next group puts level 0 in the spare and levels 6, 5, .., 1 in the blocks of levels
// 0, 1, .., 5, the order in which the epilogue frees them, so its MMAs start before this group is
// fully drained.
__device__ __forceinline__ uint32_t perm_block(uint32_t perm, int L) { return (perm >> (4 * L)) & 7u; }
__device__ __forceinline__ uint32_t perm_next(uint32_t perm) {
  uint32_t n = perm_block(perm, 7);
  for (int L = 1; L < S; ++L) n |= perm_block(perm, S - 1 - L) << (4 * L);
  return n | (perm_block(perm, 6) << 28);
}
constexpr uint32_t kPerm0 = 0x76543210u;

// Shared-memory descriptor of a K-major tile with 64-byte rows and 64-byte swizzle (the layout the
// TMA's 64-byte swizzle writes: 16-byte chunk c of row r at chunk c ^ ((r >> 1) & 3)), 8-row atoms
// 512 bytes apart; layout type 4 of the descriptor (checked on the GPU against a plain product).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t smem_addr) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_addr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Work item -> (row tile, column tile, K split).  Items run split-major, column tile fastest, so
// CTAs working at the same time share the row tile's A slices and the split's K range in L2.  With
// `upper`, row tile tm keeps only the column tiles tn >= tm BM / BN (those reaching i <= j).
struct OzItem {
  int tm, tn, split;
};
__device__ __forceinline__ OzItem oz_item(const OzArgs& p, int64_t it) {
  OzItem r;
  r.split = (int)(it / p.kept);
  int t = (int)(it - (int64_t)r.split * p.kept);
  if (!p.upper) {
    r.tm = t / p.n_tiles;
    r.tn = t - r.tm * p.n_tiles;
    return r;
  }
  int tm = 0;
  for (;; ++tm) {
    const int row = p.n_tiles - (tm * BM) / BN;
    if (t < row) break;
    t -= row;
  }
  r.tm = tm;
  r.tn = (tm * BM) / BN + t;
  return r;
}

__global__ void __launch_bounds__(kThreads, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, OzArgs p) {
  extern __shared__ uint8_t smem_raw[];
  // lev[g & 1][L]: level L of accumulation group g has all its products (two sets, so that the next
  // group's levels never complete a phase that the epilogue is still waiting for)
  __shared__ __align__(8) uint64_t sfull[NSTAGE], sempty[NSTAGE], lev[2][S], bfree[8], mdone;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // stage b: A slices at b * kStage + s * kASlice, B slices after them (K-major, 64-byte swizzle)

  if (threadIdx.x == 0) {
    for (int i = 0; i < NSTAGE; ++i) {
      tc::mbar_init(&sfull[i], 1);
      tc::mbar_init(&sempty[i], 1);
    }
    for (int L = 0; L < S; ++L) {
      tc::mbar_init(&lev[0][L], 1);
      tc::mbar_init(&lev[1][L], 1);
    }
    for (int b = 0; b < 8; ++b) tc::mbar_init(&bfree[b], kEpiThreads);
    tc::mbar_init(&mdone, 1);
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
  const int64_t G = gridDim.x;
  auto chunks_of = [&](int split) {
    const int c0 = split * p.chunks_per_split;
    return min(p.nchunks, c0 + p.chunks_per_split) - c0;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: per K chunk, the 7 A and 7 B slices into one stage
      int64_t cg = 0;  // chunks issued so far
      bool ok = true;
      for (int64_t it = blockIdx.x; it < p.items && ok; it += G) {
        const OzItem w = oz_item(p, it);
        const int nch = chunks_of(w.split), c_begin = w.split * p.chunks_per_split;
        for (int ci = 0; ci < nch; ++ci, ++cg) {
          const int k0 = (c_begin + ci) * KCH;
          const int b = (int)(cg % NSTAGE);
          if (*vabort || !tc::mbar_wait(&sempty[b], (uint32_t)((cg / NSTAGE) & 1) ^ 1u)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + (size_t)b * kStage;
          tc::mbar_arrive_expect_tx(&sfull[b], kStage);
          for (int t = 0; t < S; ++t) {
            tc::tma_load_2d(st + (size_t)t * kASlice, &mapA, &sfull[b], k0, t * p.MP + w.tm * BM);
            tc::tma_load_2d(st + (size_t)S * kASlice + (size_t)t * kBSlice, &mapB, &sfull[b], k0, t * p.NP + w.tn * BN);
          }
        }
      }
      if (!ok) {
        fail();
        // wait (bounded) for copies that may still be landing in this CTA's shared memory
        for (int64_t c = (cg > NSTAGE ? cg - NSTAGE : 0); c < cg; ++c)
          tc::mbar_wait(&sfull[c % NSTAGE], (uint32_t)((c / NSTAGE) & 1));
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: the whole warp walks the unrolled (s, t, k) sequence with
    // warp-uniform values, one elected lane issues
    const bool leader = tc::elect_one();
    const uint32_t idesc = tc::instr_desc(1u, BM, BN);  // BF16 x BF16 -> FP32, M = 128
    uint32_t perm = kPerm0, use_par = 0;  // use_par bit b: parity of the uses of level block b so far
    int64_t cg = 0, gidx = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < p.items && ok; it += G) {
      const OzItem wi = oz_item(p, it);
      const int nch = chunks_of(wi.split);
      for (int ci = 0; ci < nch && ok; ++ci, ++cg) {
        const int b = (int)(cg % NSTAGE);
        const bool first = (ci % GROUP) == 0, last = (ci % GROUP) == GROUP - 1 || ci == nch - 1;
        bool w = !*vabort && tc::mbar_wait(&sfull[b], (uint32_t)((cg / NSTAGE) & 1));
        ok = __all_sync(0xffffffffu, w);
        if (!ok) break;
        const uint32_t st = tc::smem_u32(smem + (size_t)b * kStage);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const uint64_t a0 = sw64_desc(st + (uint32_t)s * kASlice);
#pragma unroll
          for (int u = 0; u < S - s; ++u) {
            // the group's first pass makes the first write of each level, into a block the
            // epilogue has released, in the order they are released (spare first, then 6, .., 1)
            const bool fresh = first && s == 0;
            const int t = fresh ? (u == 0 ? 0 : S - u) : u;
            const uint32_t blk = perm_block(perm, s + t);
            if (fresh) {
              w = !*vabort && tc::mbar_wait(&bfree[blk], ((use_par >> blk) & 1u) ^ 1u);
              ok = __all_sync(0xffffffffu, w);
              if (!ok) break;
              use_par ^= 1u << blk;
              tc::tc_fence_after();
            }
            const uint32_t d = tmem + blk * (uint32_t)BN;
            const uint64_t b0 = sw64_desc(st + (uint32_t)S * kASlice + (uint32_t)t * kBSlice);
#pragma unroll
            for (int kk = 0; kk < KCH / 16; ++kk)
              if (leader)
                tc::mma_f16(d, tc::desc_add(a0, kk * 32), tc::desc_add(b0, kk * 32), idesc,
                            (fresh && kk == 0) ? 0u : 1u);
          }
          if (!ok) break;
          if (last) {
            __syncwarp();
            if (leader) tc::mma_commit(&lev[gidx & 1][s]);  // level s of the group has all its products
            __syncwarp();
          }
        }
        if (!ok) break;
        __syncwarp();
        if (leader) tc::mma_commit(&sempty[b]);
        __syncwarp();
        if (last) {
          perm = perm_next(perm);
          ++gidx;
        }
      }
    }
    if (!ok && leader) fail();
    // every issued MMA completes (bounded wait) before the TMEM is released
    __syncwarp();
    if (leader) tc::mma_commit(&mdone);
    __syncwarp();
    tc::mbar_wait(&mdone, 0);
  } else {
    // ---------------- epilogue: 16 warps, lane quarter q, 16 columns each.  Level L of a group is
    // folded (exact scaling by 2^-8L, TwoSum into per-output float-float accumulators) as soon as
    // the group's pass L is done, and its block released; the final value of an item is stored while
    // the next item's MMAs run.
    const int q = warp & 3, hq = (warp - 2) >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hq * 16);
    uint32_t perm = kPerm0;
    int64_t gidx = 0;  // accumulation groups drained so far
    bool ok = true;
    for (int64_t it = blockIdx.x; it < p.items && ok; it += G) {
      const OzItem wi = oz_item(p, it);
      const int ngroups = (chunks_of(wi.split) + GROUP - 1) / GROUP;
      float hi[16], lo[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) hi[u] = lo[u] = 0.f;
      for (int g = 0; g < ngroups && ok; ++g, ++gidx) {
        uint64_t* lv = lev[gidx & 1];
        const uint32_t par = (uint32_t)((gidx >> 1) & 1);
        float scale = 1.f;
#pragma unroll 1
        for (int L = 0; L < S; ++L) {
          const bool w = !*vabort && tc::mbar_wait(&lv[L], par);
          ok = __all_sync(0xffffffffu, w);
          if (!ok) break;
          tc::tc_fence_after();
          const uint32_t blk = perm_block(perm, L);
          float v[16];
          tc::tmem_ld16(lane_base + blk * (uint32_t)BN, v);
          tc::tc_fence_before();
          tc::mbar_arrive(&bfree[blk]);
#pragma unroll
          for (int u = 0; u < 16; ++u) two_sum(hi[u], lo[u], v[u] * scale);
          scale *= 0.00390625f;  // 2^-8
        }
        perm = perm_next(perm);
      }
      if (!ok) {
        fail();
        break;
      }
      const int64_t i = (int64_t)wi.tm * BM + q * 32 + lane;
      if (i < p.M) {
        const int ei = p.ea[i];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int64_t jcol = (int64_t)wi.tn * BN + hq * 16 + u;
          if (jcol < p.N) {
            // (hi + lo) 2^(e_i + f_j - 16): exact conversions by exponent arithmetic and one FP64 add
            const int pw = ei + p.eb[jcol] - 16;
            const double v = f32_scaled(hi[u], pw) + f32_scaled(lo[u], pw);
            if (p.partial) p.C[((int64_t)wi.split * p.N + jcol) * p.M + i] = v;
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
  cuuint32_t box[2] = {(cuuint32_t)KCH, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)op.sl.p, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
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

// Split-K count: the smallest with which the (tile, split) items fill whole rounds of one item per
// persistent CTA to >= 90% (else the best found), each split keeping >= 4 chunks so that its
// drains and final store stay amortised.
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
int kept_tiles(int m_tiles, int n_tiles, bool upper) {
  if (!upper) return m_tiles * n_tiles;
  int t = 0;
  for (int bm = 0; bm < m_tiles; ++bm) t += std::max(0, n_tiles - (bm * BM) / BN);
  return t;
}

}  // namespace

void oz_gemm(cudaStream_t s, int num_sms, const OzOperand& A, const OzOperand& B, double* C, int64_t ldc,
             DevBuf<double>& ws, int* err, bool symmetric) {
  RC_CHECK(A.K == B.K && A.Kp == B.Kp, RCHFSI_ERR_INVALID_ARG, "oz_gemm: K mismatch");
  const int64_t M = A.R, N = B.R;
  RC_CHECK(!symmetric || M == N, RCHFSI_ERR_INVALID_ARG, "oz_gemm: a symmetric product is square");
  RC_CHECK(M < (1LL << 31) && N < (1LL << 31), RCHFSI_ERR_INVALID_ARG, "oz_gemm: too large");
  const int m_tiles = (int)((M + BM - 1) / BM), n_tiles = (int)((N + BN - 1) / BN);
  const int nchunks = (int)(A.Kp / KCH);
  const int kept = kept_tiles(m_tiles, n_tiles, symmetric);
  // persistent CTAs over (tile, K split) items: split K only as far as the items then fill the CTAs
  double eff = 0.0;
  int nsplit = choose_split(kept, nchunks, num_sms, &eff);
  const int per = (nchunks + nsplit - 1) / nsplit;
  nsplit = (nchunks + per - 1) / per;
  const CUtensorMap ma = slice_map(A, BM);
  const CUtensorMap mb = slice_map(B, BN);
  constexpr size_t smem = (size_t)NSTAGE * kStage + 1024;
  set_smem_limit(reinterpret_cast<const void*>(oz_gemm_kernel), (int)smem);
  OzArgs p;
  p.M = (int)M;
  p.N = (int)N;
  p.MP = (int)A.Rp;
  p.NP = (int)B.Rp;
  p.chunks_per_split = per;
  p.nchunks = nchunks;
  p.n_tiles = n_tiles;
  p.kept = kept;
  p.items = (int64_t)kept * nsplit;
  p.ea = A.ex.p;
  p.eb = B.ex.p;
  p.err = err;
  p.partial = nsplit > 1;
  p.upper = symmetric ? 1 : 0;
  if (nsplit > 1) {
    p.C = ws.ensure((size_t)nsplit * M * N);
    p.ldc = M;
  } else {
    p.C = C;
    p.ldc = ldc;
  }
  const unsigned grid = (unsigned)std::min<int64_t>(p.items, num_sms);
  {
    // tensor-core flops of the 28 slice products; bytes: the slices once and the FP64 output
    // (a symmetric product computes the kept tiles only: the flops of those tiles)
    const double frac = (double)kept / ((double)m_tiles * n_tiles);
    prof::Scope ps(s, RCHFSI_KERNEL_GEMM_F64_EMU, 2.0 * M * N * A.Kp * (S * (S + 1) / 2) * frac,
                   2.0 * S * (double)(M + N) * A.Kp + 8.0 * M * N);
    oz_gemm_kernel<<<grid, kThreads, smem, s>>>(ma, mb, p);
    RC_LAUNCH();
  }
  if (nsplit > 1) {
    const int64_t total = M * N;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8);
    oz_sum_kernel<<<blocks, 256, 0, s>>>(M, N, nsplit, p.C, C, ldc);
    RC_LAUNCH();
  }
  if (symmetric) {
    const unsigned blocks = (unsigned)std::min<int64_t>((M * N + 255) / 256, (int64_t)num_sms * 4);
    mirror_upper_kernel<<<blocks, 256, 0, s>>>((int)M, C, ldc);
    RC_LAUNCH();
  }
}

}  // namespace rchfsi
