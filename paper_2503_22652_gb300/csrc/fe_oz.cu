// FP64-accurate finite-element cell products on the BF16 tensor cores (the FP64 operator products
// of the residual and Rayleigh-Ritz steps, Algorithm 1): Y[dofs(c), :] += A_c X[dofs(c), :].
//
// The cell matrices and the block are split exactly into 7 BF16 slices of base-256 digits (the
// scheme of oz_gemm.cuh): A_c(r, k) = 2^ea(c,r) sum_s t_s 2^-8(s+1) with one exponent per cell row,
// X(i, j) = 2^ex(j) sum_t u_t 2^-8(t+1) with one exponent per block column (the column's maximum
// over all dofs, so the error of a product is bounded normwise, as for an FP64 GEMM).  A cell
// product is then 28 slice products A_c^(s) X_c^(t), s + t <= 6, each a 128 x BN x 128 tcgen05 MMA;
// the products of one level L = s + t sum to an integer that FP32 holds exactly (levels <= 5; the
// last level, weight 2^-48, at most one unit off), so the 7 level accumulators live in TMEM and are
// folded once per tile, in float-float (a 2^-48 relative rounding per cell contribution, the order
// of an FP64 dot product's own rounding over the 125 terms of a cell row).
//
// The cell contributions are summed in 64-bit fixed point: entry (d, j) holds V with value
// V 2^(E_d + ex_j + H - 62), E_d the largest row exponent of the cell rows that reach dof d and H
// headroom bits for the cells that share it (|V| < 2^61).  A contribution is rounded once to that
// grid (its last place is 2^-58 of the contribution's bound for the largest row, below the FP64
// rounding of the sum) and added with an integer atomic: no FP64 instruction on the SMs (this GPU's
// FP64 rate is ~1/2000 of its BF16 tensor rate), and a sum that does not depend on the order of
// the cells.  One pass converts the integers to FP64 at the end.
//
// fe_oz_kernel, one persistent CTA per SM walking (cell, 64-column tile) items, 640 threads:
//   warp 0     cell-slice loader (one lane): cp.async.bulk of the 32 KB A_c^(s) images into a
//              3-deep ring;
//   warp 1     MMA issuer (the whole warp over an unrolled sequence, one elected lane issuing):
//              pass s = 0..6 multiplies A_c^(s) with X_c^(t), t <= 6 - s, into the TMEM
//              accumulator of level s + t.  Level s is complete after pass s and X_c^(6-s) is no
//              longer read, so each pass ends with two commits: "level s done" and "slice 6-s free".
//              TMEM holds 8 level blocks of 64 columns: 7 for the item, one spare, rotated so that
//              the next item's first writes go to blocks in the order the epilogue frees them;
//   warps 2-3  gather (two dof rows each): 16-byte cp.async of the rows' 64 columns of each slice
//              plane into the MN-major 128-byte-swizzled image X_c^(t), slice by slice as the
//              previous item releases them (slice 0, freed last, alternates between two images);
//   warps 4-19 epilogue (four per TMEM lane quarter, 16 columns each): folds level L into a
//              float-float (hi, lo) pair as soon as pass L is done and frees its block, then
//              converts to the fixed-point grid by integer arithmetic and scatters with 64-bit
//              integer atomics while the next item's MMAs run.
// Every mbarrier wait is bounded; on a timeout the kernel raises the error flag and unwinds.
#include "fe.cuh"
#include "oz_digits.cuh"
#include "prof.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace rchfsi {
namespace {

constexpr int S = 7;               // slices per operand
constexpr int kNCP = 128;          // padded cell size (M and K)
constexpr int kThreads = 640;      // 20 warps
constexpr int kBN = 64;            // column tile: one 128-byte swizzle row of BF16 per dof
constexpr uint32_t kASlice = kNCP * kNCP * 2;  // 32 KB per A slice image
constexpr uint32_t kXSlice = kNCP * kBN * 2;   // 16 KB per X slice image
constexpr int kRowBytes = 128;
constexpr int kARing = 3;          // cell-slice images in flight (the issuer runs up to two passes ahead)

__device__ __forceinline__ uint32_t sw_off2(int r, int k, int rows) {
  // byte offset of BF16 element (row r, k) in a K-major 128B-swizzled image with `rows` rows
  const int kb = k >> 6;
  const int byte = (k & 63) * 2;
  const int chunk = (byte >> 4) ^ (r & 7);
  return (uint32_t)kb * rows * kRowBytes + (uint32_t)r * kRowBytes + (chunk << 4) + (byte & 15);
}

// Byte offset of the 16-byte chunk c (columns 8c .. 8c+7) of dof row k in an MN-major
// 128B-swizzled X slice image: one 128-byte row per dof, 8-row atoms of 1024 bytes.
__device__ __forceinline__ uint32_t mn_chunk_off(int k, int c) {
  return (uint32_t)(k >> 3) * 1024u + (uint32_t)(k & 7) * kRowBytes + ((uint32_t)(c ^ (k & 7)) << 4);
}

// Shared-memory descriptor of an MN-major 128B-swizzled BF16 operand whose MN extent is one
// 64-element swizzle row: 8-row K groups 1024 bytes apart (stride byte offset); the leading byte
// offset (distance between 64-element MN groups) is not used at this width.
__device__ __forceinline__ uint64_t mn_sw128_desc(uint32_t smem_addr) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_addr >> 4) & 0x3FFF);
  d |= (uint64_t)(1024 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Pack cell matrices (n_cells x nc x nc FP64 row-major) into per-cell images of the 7 BF16 slices,
// [cell][s][128 x 128 K-major swizzled], and the per-row exponents [cell][128]: first the row
// exponents, one warp per padded row (-100000 for a zero or padding row: it adds nothing, so it
// sets no scale), then the digits, one thread per (row, k) element.
__global__ void slice_rowexp_kernel(int64_t n_cells, int nc, const double* __restrict__ A, int* __restrict__ rexp) {
  const int64_t rows = n_cells * kNCP;
  const int lane = threadIdx.x & 31;
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < rows;
       e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t c = e / kNCP;
    const int r = (int)(e % kNCP);
    int ea = -100000;
    if (r < nc) {
      const double* row = A + (c * nc + r) * nc;
      for (int k = lane; k < nc; k += 32) ea = max(ea, exp_of(row[k]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, o));
    if (lane == 0) rexp[e] = ea;
  }
}

__global__ void pack_slices_kernel(int64_t n_cells, int nc, const double* __restrict__ A, const int* __restrict__ rexp,
                                   uint8_t* __restrict__ img) {
  const int64_t total = n_cells * kNCP * kNCP;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / (kNCP * kNCP);
    const int r = (int)((e / kNCP) % kNCP), k = (int)(e % kNCP);
    int ea = rexp[c * kNCP + r];
    if (ea == -100000) ea = 0;
    long long f = (r < nc && k < nc) ? fixed56(A[(c * nc + r) * nc + k], ea) : 0;
    uint8_t* base = img + c * (int64_t)S * kASlice + sw_off2(r, k, kNCP);
#pragma unroll
    for (int s = 0; s < S; ++s)
      *reinterpret_cast<__nv_bfloat16*>(base + (size_t)s * kASlice) = __float2bfloat16_rn((float)(int)next_digit(f, s));
  }
}

// Column exponents of a column-major m x n block X (leading dimension m): one block per column,
// cexp[j] = the largest exponent in column j (-100000 for a zero column).
__global__ void __launch_bounds__(256) colexp_cols_kernel(int64_t m, const double* __restrict__ X, int* cexp) {
  __shared__ int red[8];
  const double* col = X + (int64_t)blockIdx.x * m;
  int e = -100000;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) e = max(e, exp_of(col[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) e = max(e, red[w]);
    cexp[blockIdx.x] = e;
  }
}

// Per dof, the largest row exponent of the cell rows that reach it (rowexp initialised to -100000).
__global__ void rowexp_kernel(int64_t n_cells, int nc, const int* __restrict__ dofs, const int* __restrict__ aexp,
                              int64_t e_stride, int* rowexp) {
  const int64_t total = n_cells * nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / nc;
    const int i = (int)(e % nc);
    const int ea = aexp[c * e_stride + i];
    if (ea > -100000) atomicMax(rowexp + dofs[e], ea);
  }
}

// Value of accumulator entry (row i, column j): V 2^(rowexp(dof) + cexp(j) + H - 62), with
// dof = i mod mrow (the two halves of a complex embedding share the dof's scale; m <= 2 mrow).  An exponent
// above the FP64 range marks a non-finite input in that row of a cell matrix or column of X.
__device__ __forceinline__ double fixed_value(long long V, int er, int ec, int H) {
  if (er > 1024 || ec > 1024) return __longlong_as_double(0x7ff8000000000000LL);
  if (V == 0) return 0.0;
  return fixed_to_f64(V, er + ec + H - 62);
}

// Fixed-point accumulator (row-major m x n) -> FP64 column-major Ycol (leading dimension m), through
// 32 x 32 shared-memory tiles (coalesced reads along rows, writes along columns).
__global__ void __launch_bounds__(256) fixed_to_cols_kernel(int64_t m, int n, int64_t mrow,
                                                            const long long* __restrict__ V,
                                                            const int* __restrict__ rowexp,
                                                            const int* __restrict__ cexp, int H,
                                                            double* __restrict__ Ycol) {
  __shared__ double tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int j = j0 + tx;
  const int ec = (j < n) ? cexp[j] : 0;
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r;
    double v = 0.0;
    if (i < m && j < n) v = fixed_value(V[i * n + j], rowexp[i < mrow ? i : i - mrow], ec, H);
    tile[r][tx] = v;
  }
  __syncthreads();
  const int64_t i = i0 + tx;
  for (int c = ty; c < 32; c += 8) {
    const int jj = j0 + c;
    if (i < m && jj < n) Ycol[(int64_t)jj * m + i] = tile[tx][c];
  }
}

// The 7 slice planes of a column-major m x n block X (leading dimension m): plane t holds the
// digits u_t as BF16, row-major with np >= n columns (np a multiple of 64, columns n .. np-1 zero),
// so that every dof row of a column tile is one aligned 128-byte run.  32 x 32 tiles through shared
// memory: reads coalesced along the rows of X, writes along the columns of the planes.
__global__ void __launch_bounds__(256) xslice_cols_kernel(int64_t m, int n, int np, const double* __restrict__ X,
                                                          const int* __restrict__ cexp,
                                                          __nv_bfloat16* __restrict__ planes) {
  __shared__ double tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int c = ty; c < 32; c += 8) {
    const int j = j0 + c;
    const int64_t i = i0 + tx;
    tile[c][tx] = (j < n && i < m) ? X[(int64_t)j * m + i] : 0.0;
  }
  __syncthreads();
  const int j = j0 + tx;
  int e = (j < n) ? cexp[j] : 0;
  if (e == -100000) e = 0;
  const int64_t pstride = m * (int64_t)np;
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r;
    if (i >= m) break;
    long long f = fixed56(tile[tx][r], e);
    __nv_bfloat16* dst = planes + i * np + j;
#pragma unroll
    for (int t = 0; t < S; ++t) {
      // |digit| <= 256: converted through int (a 64-bit integer conversion uses the FP64 pipe)
      dst[(int64_t)t * pstride] = __float2bfloat16_rn((float)(int)next_digit(f, t));
    }
  }
}

struct FeOzArgs {
  int64_t n_cells;
  int nc, n, np, ntiles;
  const int* dofs;
  const uint8_t* aimg;    // slice images; cell stride a_stride bytes (0: one matrix shared by all cells)
  int64_t a_stride;
  const int* aexp;        // row exponents; cell stride e_stride ints
  int64_t e_stride;
  const __nv_bfloat16* planes;  // 7 planes of rows x np
  int64_t plane_stride;         // elements between planes
  const int* rowexp;            // per dof: the scale exponent of its accumulator rows
  int H;                        // headroom bits of the accumulator
  long long* Y;                 // fixed-point accumulator, row-major, n columns
  int neg;      // subtract instead of add (the -Ai X_i part of a complex product)
  int* err;
};

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(tc::smem_u32(bar))
               : "memory");
}

// 16-byte asynchronous copy global -> shared (L2 only); `in` = false writes 16 zero bytes instead
// (no bytes are read from src then).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool in) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(reinterpret_cast<uint64_t>(src)),
               "r"(in ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void red_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void two_sum(float& hi, float& lo, float b) {
  const float s = hi + b;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (b - bb);
  hi = s;
  lo += e;
}


// Level buffers in TMEM: 8 blocks of 64 columns, 7 holding the levels of the current item and one
// spare.  perm packs, per level L = 0..6, its block (4 bits each; bits 28-31: the spare).  The next
// item puts level 0 in the spare and levels 6, 5, .., 1 in the blocks of levels 0, 1, .., 5, the
// order in which the epilogue frees them, so its MMAs start before this item is fully folded.
__device__ __forceinline__ uint32_t perm_block(uint32_t perm, int L) { return (perm >> (4 * L)) & 7u; }
__device__ __forceinline__ uint32_t perm_next(uint32_t perm) {
  uint32_t n = perm_block(perm, 7);                                   // level 0 <- spare
  for (int L = 1; L < S; ++L) n |= perm_block(perm, S - 1 - L) << (4 * L);  // level L <- old level 6 - L
  return n | (perm_block(perm, 6) << 28);                             // spare <- old level 6
}

// X slice images: slices 1..6 in blocks 1..6, slice 0 in block 0 or 7 by item parity (its block
// is freed last, so the next item's copy goes to the other one).
__device__ __forceinline__ int x_block(int t, int64_t j) { return t ? t : ((j & 1) ? 7 : 0); }
// parity of the phase of the block's barriers that item j uses (blocks 0 and 7 serve every other item)
__device__ __forceinline__ uint32_t x_par(int t, int64_t j) { return (uint32_t)(t ? (j & 1) : ((j >> 1) & 1)); }

__global__ void __launch_bounds__(kThreads, 1) fe_oz_kernel(const __grid_constant__ FeOzArgs p) {
  extern __shared__ uint8_t smem_raw[];
  // lev[j & 1][L]: level L of item j has all its products (two sets, so that the next item's levels
  // never complete a phase that the epilogue is still waiting for)
  __shared__ __align__(8) uint64_t afull[kARing], aempty[kARing], xfull[8], xempty[8], lev[2][S], bfree[8], mdone;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;                          // kARing x 32 KB, K-major cell slices
  uint8_t* sX = smem + kARing * kASlice;       // 8 x 16 KB, MN-major X slices
  if (threadIdx.x == 0) {
    for (int i = 0; i < kARing; ++i) {
      tc::mbar_init(&afull[i], 1);
      tc::mbar_init(&aempty[i], 1);
    }
    for (int b = 0; b < 8; ++b) {
      tc::mbar_init(&xfull[b], 64);  // every gathering thread, once its copies of the slice have landed
      tc::mbar_init(&xempty[b], 1);
      tc::mbar_init(&bfree[b], 512);  // every epilogue thread, once it has read the block
    }
    for (int t = 0; t < S; ++t) {
      tc::mbar_init(&lev[0][t], 1);
      tc::mbar_init(&lev[1][t], 1);
    }
    tc::mbar_init(&mdone, 1);
    tc::fence_barrier_init();
    abort_flag = 0;
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_slot, 512);
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
  const int64_t my_cells = (p.n_cells > (int64_t)blockIdx.x) ? (p.n_cells - 1 - blockIdx.x) / G + 1 : 0;
  const int64_t items = my_cells * p.ntiles;
  constexpr uint32_t kPerm0 = 0x76543210u;

  if (warp == 0) {
    // ---------------- cell-slice loader (one lane)
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t j = 0; j < items && !*vabort; ++j) {
        const int64_t cell = blockIdx.x + (j / p.ntiles) * G;
        const uint8_t* src = p.aimg + cell * p.a_stride;
        bool ok = true;
        for (int s = 0; s < S; ++s) {
          const int64_t a = j * S + s;
          const int q = (int)(a % kARing);
          if (*vabort || !tc::mbar_wait(&aempty[q], (uint32_t)((a / kARing) & 1) ^ 1u)) {
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&afull[q], kASlice);
          bulk_g2s(sA + (size_t)q * kASlice, src + (size_t)s * kASlice, kASlice, &afull[q]);
          ++issued;
        }
        if (!ok) {
          fail();
          break;
        }
      }
      if (*vabort) {
        // wait (bounded) for copies that may still be landing in this CTA's shared memory
        for (int64_t a = (issued > kARing ? issued - kARing : 0); a < issued; ++a)
          tc::mbar_wait(&afull[a % kARing], (uint32_t)((a / kARing) & 1));
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: the whole warp walks the unrolled (s, t, k) sequence with
    // warp-uniform values, one elected lane issues
    const bool leader = tc::elect_one();
    const uint32_t idesc = tc::instr_desc(1u, kNCP, kBN) | (1u << 16);  // BF16 -> FP32, B (X) MN-major
    const uint64_t x_desc = mn_sw128_desc(tc::smem_u32(sX));
    uint32_t perm = kPerm0, use_par = 0;  // use_par bit b: parity of the uses of level block b so far
    int q = 0;                            // ring slot of the next cell slice and its phase parity
    uint32_t qpar = 0;
    bool ok = true;
    for (int64_t j = 0; j < items && ok; ++j) {
#pragma unroll
      for (int s = 0; s < S; ++s) {
        bool w = !*vabort && tc::mbar_wait(&afull[q], qpar);
        ok = __all_sync(0xffffffffu, w);
        if (!ok) break;
        tc::tc_fence_after();
        const uint64_t a0 = tc::sw128_desc(tc::smem_u32(sA + (size_t)q * kASlice));
#pragma unroll
        for (int u = 0; u < S - s; ++u) {
          // pass 0 takes the X slices in the order the gather refills them (0, 6, 5, .., 1) and
          // makes the first write of each level, into a block the epilogue has released
          const int t = (s == 0) ? (u == 0 ? 0 : S - u) : u;
          const uint32_t blk = perm_block(perm, s + t);
          if (s == 0) {
            w = !*vabort && tc::mbar_wait(&xfull[x_block(t, j)], x_par(t, j));
            if (w) w = tc::mbar_wait(&bfree[blk], ((use_par >> blk) & 1u) ^ 1u);
            ok = __all_sync(0xffffffffu, w);
            if (!ok) break;
            use_par ^= 1u << blk;
            tc::tc_fence_after();
          }
          const uint32_t d = tmem + blk * (uint32_t)kBN;
          const uint64_t x0 = tc::desc_add(x_desc, (uint32_t)x_block(t, j) * kXSlice);
#pragma unroll
          for (int kk = 0; kk < kNCP / 16; ++kk) {
            const int kel = kk * 16;
            const uint32_t aoff = (uint32_t)(kel >> 6) * kNCP * kRowBytes + (uint32_t)((kel & 63) * 2);
            // MN-major X: 16 K rows (two 1024-byte atoms) per MMA
            if (leader)
              tc::mma_f16(d, tc::desc_add(a0, aoff), tc::desc_add(x0, (uint32_t)kk * 2048u), idesc,
                          (s == 0 && kk == 0) ? 0u : 1u);
          }
        }
        if (!ok) break;
        __syncwarp();
        if (leader) {
          tc::mma_commit(&aempty[q]);
          // level s has all its products, and X slice 6 - s is not read again (for slices 1..6
          // the gather waits on lev[] itself)
          tc::mma_commit(&lev[j & 1][s]);
          if (s == S - 1) tc::mma_commit(&xempty[x_block(0, j)]);
        }
        __syncwarp();
        if (++q == kARing) {
          q = 0;
          qpar ^= 1u;
        }
      }
      perm = perm_next(perm);
    }
    if (!ok && leader) fail();
    // every issued MMA completes (bounded wait) before the TMEM is released
    __syncwarp();
    if (leader) tc::mma_commit(&mdone);
    __syncwarp();
    tc::mbar_wait(&mdone, 0);
  } else if (warp < 4) {
    // ---------------- gather: thread k copies dofs k and k + 64, 64 columns of every slice plane
    // (zeros for the padding rows >= n_c), slice 0 first (its block was freed two items ago), then
    // 6, 5, .., 1 as the previous item releases them.  A slice is signalled once its copies have
    // landed: wait for all but the newest group, make the writes visible to the tensor cores, arrive.
    const int k = threadIdx.x - 64;  // 0 .. 63
    const uint32_t xs = tc::smem_u32(sX);
    for (int64_t j = 0; j < items; ++j) {
      const int64_t cell = blockIdx.x + (j / p.ntiles) * G;
      const int tile = (int)(j % p.ntiles);
      const __nv_bfloat16* src0[2];
      bool in[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int kr = k + 64 * r;
        const int g = (kr < p.nc) ? __ldg(p.dofs + cell * p.nc + kr) : -1;
        in[r] = g >= 0;
        src0[r] = p.planes + (in[r] ? (int64_t)g * p.np + (int64_t)tile * kBN : 0);
      }
      bool ok = true;
      int prev = -1;
      for (int u = 0; u < S; ++u) {
        const int t = (u == 0) ? 0 : S - u;
        const int b = x_block(t, j);
        // slice t >= 1 is free once pass 6 - t of the previous item is done; slice 0's block once
        // the item before that is done
        const bool freed = t ? (j == 0 || tc::mbar_wait(&lev[(j - 1) & 1][S - 1 - t], (uint32_t)(((j - 1) >> 1) & 1)))
                             : tc::mbar_wait(&xempty[b], x_par(0, j) ^ 1u);
        if (*vabort || !freed) {
          ok = false;
          break;
        }
        const uint32_t dst = xs + (uint32_t)b * kXSlice;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const __nv_bfloat16* src = src0[r] + (int64_t)t * p.plane_stride;
#pragma unroll
          for (int c = 0; c < kBN / 8; ++c) cp_async16(dst + mn_chunk_off(k + 64 * r, c), src + 8 * c, in[r]);
        }
        cp_async_commit();
        if (prev >= 0) {
          cp_async_wait<1>();
          fence_proxy_async();
          tc::mbar_arrive(&xfull[prev]);
        }
        prev = b;
      }
      cp_async_wait<0>();
      if (!ok) {
        fail();
        break;
      }
      fence_proxy_async();
      tc::mbar_arrive(&xfull[prev]);
    }
  } else {
    // ---------------- epilogue: fold level L as soon as pass L is done and release its block,
    // then convert and scatter-add while the next item's MMAs run; four warps per TMEM lane
    // quarter, 16 columns each
    const int q = warp & 3, hq = (warp - 4) >> 2;
    const int i = q * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hq * 16);
    uint32_t perm = kPerm0;
    for (int64_t j = 0; j < items; ++j) {
      const int64_t cell = blockIdx.x + (j / p.ntiles) * G;
      const int tile = (int)(j % p.ntiles);
      uint64_t* lv = lev[j & 1];
      const uint32_t par = (uint32_t)((j >> 1) & 1);
      int g = -1, qs = 0;
      if (i < p.nc) {
        g = __ldg(p.dofs + cell * p.nc + i);
        // the contribution (hi + lo) 2^(ea + ex - 16) in units of the accumulator's last place
        // 2^(rowexp + ex + H - 62): the column exponent ex cancels
        const int ea = __ldg(p.aexp + cell * p.e_stride + i);
        qs = ea == -100000 ? 0 : max(46 - p.H + ea - __ldg(p.rowexp + g), -200);
      }
      float hi[16], lo[16];
      bool ok = true;
      float scale = 1.f;
#pragma unroll 1
      for (int L = 0; L < S; ++L) {
        const bool w = !*vabort && tc::mbar_wait(&lv[L], par);
        ok = __all_sync(0xffffffffu, w);
        if (!ok) break;
        tc::tc_fence_after();
        const uint32_t blk = perm_block(perm, L);
        float v[16];
        tc::tmem_ld16(lane_base + blk * (uint32_t)kBN, v);
        tc::tc_fence_before();
        tc::mbar_arrive(&bfree[blk]);
        if (L == 0) {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            hi[u] = v[u];
            lo[u] = 0.f;
          }
        } else {
#pragma unroll
          for (int u = 0; u < 16; ++u) two_sum(hi[u], lo[u], v[u] * scale);
        }
        scale *= 0.00390625f;  // 2^-8 per level
      }
      if (!ok) {
        fail();
        break;
      }
      perm = perm_next(perm);
      if (g >= 0) {
        // integer adds: exact, so the sum does not depend on the order of the cells
        unsigned long long* out = reinterpret_cast<unsigned long long*>(p.Y + (int64_t)g * p.n);
        const int c0 = tile * kBN + hq * 16;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int col = c0 + u;
          if (col < p.n) {
            const long long v = f32_to_fixed(hi[u], qs) + f32_to_fixed(lo[u], qs);
            red_add_u64(out + col, (unsigned long long)(p.neg ? -v : v));
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

}  // namespace

namespace {

void fill_int(cudaStream_t s, int* p, int n, int v);

__global__ void fill_int_kernel(int* p, int n, int v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

void fill_int(cudaStream_t s, int* p, int n, int v) {
  fill_int_kernel<<<cdiv(n, 256) < 64 ? cdiv(n, 256) : 64, 256, 0, s>>>(p, n, v);
  RC_LAUNCH();
}

// Slice images and row exponents of an operator's cell matrices (made on first use).
void ensure_slices(cudaStream_t s, const FeOp& op, bool useB) {
  DevBuf<uint8_t>& img = useB ? op.ozB : op.ozA;
  DevBuf<int>& ex = useB ? op.ozBe : op.ozAe;
  if (img.p && op.oz_packed[useB]) return;
  const int64_t cells = (useB && op.B_shared) ? 1 : op.n_cells;
  img.ensure((size_t)cells * S * kASlice);
  ex.ensure((size_t)cells * kNCP);
  const double* src = useB ? op.B64.p : op.A64.p;
  const int64_t rows = cells * kNCP;
  slice_rowexp_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((rows * 32 + 255) / 256, 152 * 32)), 256, 0,
                        s>>>(cells, op.nc, src, ex.p);
  RC_LAUNCH();
  const int64_t total = rows * kNCP;
  pack_slices_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 32)), 256, 0,
                       s>>>(cells, op.nc, src, ex.p, img.p);
  RC_LAUNCH();
  op.oz_packed[useB] = true;
}

// Per-dof scale exponents of the accumulator for op (and, for the A product of a complex operator,
// its imaginary part, which adds into the same rows); made on first use.
const int* ensure_rowexp(cudaStream_t s, const FeOp& op, bool useB) {
  DevBuf<int>& rx = useB ? op.ozBrow : op.ozArow;
  if (rx.p && op.rowexp_packed[useB]) return rx.p;
  const int64_t nd = op.cplx ? op.mc : op.m;
  rx.ensure((size_t)nd);
  fill_int(s, rx.p, (int)nd, -100000);
  auto add = [&](const FeOp& o) {
    const bool shared = useB && o.B_shared;
    const int64_t total = o.n_cells * o.nc;
    rowexp_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8)), 256, 0, s>>>(
        o.n_cells, o.nc, o.dofs.p, useB ? o.ozBe.p : o.ozAe.p, shared ? 0 : kNCP, rx.p);
    RC_LAUNCH();
  };
  ensure_slices(s, op, useB);
  add(op);
  if (op.cplx && !useB) {
    ensure_slices(s, *op.imag, false);
    add(*op.imag);
  }
  op.rowexp_packed[useB] = true;
  return rx.p;
}

// Headroom bits of the accumulator: a cell product row adds at most 2^(ea + ex + 7) (n_c <= 128
// terms of |digit products| <= 2^16), max_mult cells (twice that for a complex A) add into one entry.
int headroom(const FeOp& op, bool useB) {
  int mult = std::max(1, op.max_mult) * ((op.cplx && !useB) ? 2 : 1);
  int b = 0;
  while ((1 << b) < mult) ++b;
  return 8 + b;
}

void launch_oz(cudaStream_t s, int num_sms, const FeOp& op, bool useB, const __nv_bfloat16* planes,
               int64_t plane_stride, int np, const int* rowexp, int H, long long* Y, int n, bool neg) {
  constexpr size_t smem = kARing * kASlice + 8 * (size_t)kXSlice + 1024;
  set_smem_limit(reinterpret_cast<const void*>(fe_oz_kernel), (int)smem);
  ensure_slices(s, op, useB);
  const bool shared = useB && op.B_shared;
  FeOzArgs a{};
  a.n_cells = op.n_cells;
  a.nc = op.nc;
  a.n = n;
  a.np = np;
  a.ntiles = np / kBN;
  a.dofs = op.dofs.p;
  a.aimg = useB ? op.ozB.p : op.ozA.p;
  a.a_stride = shared ? 0 : (int64_t)S * kASlice;
  a.aexp = useB ? op.ozBe.p : op.ozAe.p;
  a.e_stride = shared ? 0 : kNCP;
  a.planes = planes;
  a.plane_stride = plane_stride;
  a.rowexp = rowexp;
  a.H = H;
  a.Y = Y;
  a.neg = neg ? 1 : 0;
  a.err = op.err;
  const unsigned grid = (unsigned)std::min<int64_t>(op.n_cells, num_sms);
  const double nc = op.nc, C = (double)op.n_cells;
  prof::Scope ps(s, RCHFSI_KERNEL_FE_CELL_F64, 2.0 * nc * nc * C * n,
                 14.0 * (double)C * nc * n + 8.0 * 2.0 * (double)C * nc * n + (shared ? 1.0 : C) * S * kASlice);
  if (grid == 0) return;
  fe_oz_kernel<<<grid, kThreads, smem, s>>>(a);
  RC_LAUNCH();
}

}  // namespace

void fe_apply_f64_cols_tc(cudaStream_t s, const FeOp& op, const double* X, double* AX, double* BX, int n,
                          int num_sms, double* accA, double* accB) {
  RC_CHECK(op.nc <= kNCP, RCHFSI_ERR_INVALID_ARG, "n_c larger than 128");
  RC_CHECK((!AX || accA) && (!BX || accB), RCHFSI_ERR_INVALID_ARG, "fixed-point accumulator missing");
  const int64_t m = op.m;
  if (n <= 0 || m <= 0 || (!AX && !BX)) return;
  // column exponents over every row (both halves of a complex block), then the slice planes of
  // X, rows padded to np columns: made once for both products
  int* cexp = op.ozcexp.ensure(n);
  const int np = (int)cdiv(n, kBN) * kBN;
  const int64_t total = m * (int64_t)np;
  __nv_bfloat16* planes = op.ozplanes.ensure((size_t)S * total);
  {
    prof::Scope ps(s, RCHFSI_KERNEL_RR_AUX, 0.0, 16.0 * m * n + 14.0 * (double)total);
    colexp_cols_kernel<<<(unsigned)n, 256, 0, s>>>(m, X, cexp);
    RC_LAUNCH();
    xslice_cols_kernel<<<dim3(cdiv(m, 32), (unsigned)(np / 32)), 256, 0, s>>>(m, n, np, X, cexp, planes);
    RC_LAUNCH();
  }
  const int64_t mrow = op.cplx ? op.mc : m;
  for (int which = 0; which < 2; ++which) {
    const bool useB = which == 1;
    double* out = useB ? BX : AX;
    if (!out) continue;
    // fixed-point accumulator (64-bit integers in the scratch block), zero
    long long* V = reinterpret_cast<long long*>(useB ? accB : accA);
    RC_CUDA(cudaMemsetAsync(V, 0, sizeof(long long) * m * n, s));
    const int* rowexp = ensure_rowexp(s, op, useB);
    const int H = headroom(op, useB);
    if (!op.cplx) {
      launch_oz(s, num_sms, op, useB, planes, total, np, rowexp, H, V, n, false);
    } else {
      // complex operator on the real embedding (rows [0, mc) real parts, [mc, 2 mc) imaginary
      // parts): Y_r = Ar X_r - Ai X_i,  Y_i = Ai X_r + Ar X_i;  the real B acts on each half
      const int64_t poff = op.mc * (int64_t)np, yoff = op.mc * (int64_t)n;
      if (useB) {
        launch_oz(s, num_sms, op, true, planes, total, np, rowexp, H, V, n, false);
        launch_oz(s, num_sms, op, true, planes + poff, total, np, rowexp, H, V + yoff, n, false);
      } else {
        const FeOp& im = *op.imag;
        launch_oz(s, num_sms, op, false, planes, total, np, rowexp, H, V, n, false);
        launch_oz(s, num_sms, im, false, planes + poff, total, np, rowexp, H, V, n, true);
        launch_oz(s, num_sms, im, false, planes, total, np, rowexp, H, V + yoff, n, false);
        launch_oz(s, num_sms, op, false, planes + poff, total, np, rowexp, H, V + yoff, n, false);
      }
    }
    prof::Scope ps(s, RCHFSI_KERNEL_RR_AUX, 0.0, 16.0 * m * n);
    fixed_to_cols_kernel<<<dim3(cdiv(m, 32), cdiv(n, 32)), 256, 0, s>>>(m, n, mrow, V, rowexp, cexp, H, out);
    RC_LAUNCH();
  }
}

}  // namespace rchfsi
