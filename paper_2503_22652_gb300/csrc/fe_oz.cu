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
// fe_oz_kernel, one persistent CTA per SM walking (cell, column tile) items, 576 threads:
//   warps 0-7  gather: thread (k, h) copies its dof k's row, columns h*BN/2.., of the 7 X slice
//              planes (sliced once per product by xslice_kernel) into the K-major 128-byte-swizzled
//              shared images X_c^(t);
//   warp 8     MMA issuer (the whole warp over an unrolled sequence, one elected lane issuing):
//              for each A slice s (streamed through a 2-deep ring) the products with X_c^(t),
//              t <= 6 - s, into the TMEM accumulator of level s + t;
//   warps 9-16 epilogue (two per TMEM lane quarter, alternate 16 columns): tcgen05.ld of the 7
//              levels, float-float fold, exact conversion and exponent scaling by integer
//              arithmetic, one FP64 add, FP64 atomic scatter-add;
//   warp 17    cell-slice loader (one lane): cp.async.bulk of the 32 KB A_c^(s) images.
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
constexpr int kThreads = 576;      // 18 warps
constexpr int kMaxBN = 64;
constexpr uint32_t kASlice = kNCP * kNCP * 2;  // 32 KB per A slice image
constexpr int kRowBytes = 128;

__device__ __forceinline__ uint32_t sw_off2(int r, int k, int rows) {
  // byte offset of BF16 element (row r, k) in a K-major 128B-swizzled image with `rows` rows
  const int kb = k >> 6;
  const int byte = (k & 63) * 2;
  const int chunk = (byte >> 4) ^ (r & 7);
  return (uint32_t)kb * rows * kRowBytes + (uint32_t)r * kRowBytes + (chunk << 4) + (byte & 15);
}

// Pack cell matrices (n_cells x nc x nc FP64 row-major) into per-cell images of the 7 BF16 slices,
// [cell][s][128 x 128 K-major swizzled], and the per-row exponents [cell][128].
__global__ void pack_slices_kernel(int64_t n_cells, int nc, const double* __restrict__ A, uint8_t* __restrict__ img,
                                   int* __restrict__ rexp) {
  const int64_t rows = n_cells * kNCP;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / kNCP;
    const int r = (int)(e % kNCP);
    const double* row = A + (c * nc + r) * nc;
    int ea = -100000;
    if (r < nc)
      for (int k = 0; k < nc; ++k) ea = max(ea, exp_of(row[k]));
    if (ea == -100000) ea = 0;
    rexp[e] = ea;
    uint8_t* base = img + c * (int64_t)S * kASlice;
    for (int k = 0; k < kNCP; ++k) {
      long long f = (r < nc && k < nc) ? fixed56(row[k], ea) : 0;
      for (int s = 0; s < S; ++s) {
        const int t = (int)next_digit(f, s);
        *reinterpret_cast<__nv_bfloat16*>(base + (size_t)s * kASlice + sw_off2(r, k, kNCP)) =
            __float2bfloat16_rn((float)t);
      }
    }
  }
}

// Column exponents of a row-major m x n block (max over rows), into cexp (initialised to -100000).
__global__ void colexp_kernel(int64_t m, int n, const double* __restrict__ X, int* cexp) {
  for (int j0 = threadIdx.x; j0 < n; j0 += blockDim.x) {
    int e = -100000;
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) e = max(e, exp_of(X[i * n + j0]));
    if (e > -100000) atomicMax(cexp + j0, e);
  }
}

// The 7 slice planes of X (row-major m x n): plane t holds the digits u_t, as BF16, row-major.
// Thread (x, y): column pair 2 x of rows y, y + gridDim.y blockDim.y, ... (the column exponents are
// loaded once; two columns per thread give 16-byte loads and 4-byte stores).  n even.
__global__ void __launch_bounds__(256) xslice_kernel(int64_t m, int n, const double* __restrict__ X,
                                                     const int* __restrict__ cexp,
                                                     __nv_bfloat16* __restrict__ planes) {
  const int j = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (j >= n) return;
  int e0 = cexp[j], e1 = cexp[j + 1];
  if (e0 == -100000) e0 = 0;
  if (e1 == -100000) e1 = 0;
  const int64_t total = m * n;
  for (int64_t i = blockIdx.y * (int64_t)blockDim.y + threadIdx.y; i < m; i += (int64_t)gridDim.y * blockDim.y) {
    const int64_t e = i * n + j;
    const double2 x = *reinterpret_cast<const double2*>(X + e);
    long long f0 = fixed56(x.x, e0), f1 = fixed56(x.y, e1);
#pragma unroll
    for (int t = 0; t < S; ++t) {
      // |digit| <= 256: converted through int (a 64-bit integer conversion uses the FP64 pipe)
      const float d0 = (float)(int)next_digit(f0, t), d1 = (float)(int)next_digit(f1, t);
      *reinterpret_cast<__nv_bfloat162*>(planes + (int64_t)t * total + e) = __floats2bfloat162_rn(d0, d1);
    }
  }
}

// Odd n: one column per thread.
__global__ void xslice1_kernel(int64_t total, int n, const double* __restrict__ X, const int* __restrict__ cexp,
                               __nv_bfloat16* __restrict__ planes) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int ex = cexp[e % n];
    if (ex == -100000) ex = 0;
    long long f = fixed56(X[e], ex);
#pragma unroll
    for (int t = 0; t < S; ++t) planes[(int64_t)t * total + e] = __float2bfloat16_rn((float)(int)next_digit(f, t));
  }
}

struct FeOzArgs {
  int64_t n_cells;
  int nc, n, BN, ntiles;
  const int* dofs;
  const uint8_t* aimg;    // slice images; cell stride a_stride bytes (0: one matrix shared by all cells)
  int64_t a_stride;
  const int* aexp;        // row exponents; cell stride e_stride ints
  int64_t e_stride;
  const __nv_bfloat16* planes;  // 7 x m x n
  int64_t plane_stride;         // m * n
  const int* cexp;
  double* Y;
  int neg;      // subtract instead of add (the -Ai X_i part of a complex product)
  int vec;      // n % 8 == 0: 16-byte gathers
  int* err;
};

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(tc::smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// OR of v over the 256 epilogue threads (named barrier 1); every epilogue warp must call it.
__device__ __forceinline__ bool epi_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.or.pred po, 1, 256, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void two_sum(float& hi, float& lo, float b) {
  const float s = hi + b;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (b - bb);
  hi = s;
  lo += e;
}


__global__ void __launch_bounds__(kThreads, 1) fe_oz_kernel(const __grid_constant__ FeOzArgs p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t afull[2], aempty[2], xfull, xempty, accfull, accempty;
  __shared__ int s_cexp[kMaxBN];  // column exponents of the current tile (epilogue)
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int BN = p.BN;
  const uint32_t x_bytes = (uint32_t)BN * kNCP * 2;  // one X slice image
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;                 // 2 x 32 KB
  uint8_t* sX = smem + 2 * kASlice;   // 7 x BN x 128 x 2
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&afull[i], 1);
      tc::mbar_init(&aempty[i], 1);
    }
    tc::mbar_init(&xfull, 256);
    tc::mbar_init(&xempty, 1);
    tc::mbar_init(&accfull, 1);
    tc::mbar_init(&accempty, 256);
    tc::fence_barrier_init();
    abort_flag = 0;
  }
  if (warp == 8) {
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

  if (warp < 8) {
    // ---------------- gather of the X slice planes
    const int k = threadIdx.x & 127, h = threadIdx.x >> 7;
    const int half = BN / 2;
    for (int64_t j = 0; j < items; ++j) {
      const int64_t cell = blockIdx.x + (j / p.ntiles) * G;
      const int t = (int)(j % p.ntiles);
      if (*vabort || !tc::mbar_wait(&xempty, (uint32_t)(j & 1) ^ 1u)) {
        fail();
        break;
      }
      const int g = (k < p.nc) ? p.dofs[cell * p.nc + k] : -1;
      const int c0 = t * BN + h * half;
      if (p.vec) {
        // two planes at a time, each thread's 32 columns as four 16-byte loads per plane: eight
        // loads in flight before any is stored (rows start on 16-byte boundaries when n % 8 == 0)
        for (int s0 = 0; s0 < S; s0 += 2) {
          uint4 q[2][4];
#pragma unroll
          for (int d = 0; d < 2; ++d) {
            const int s = s0 + d;
            const __nv_bfloat16* row =
                (g >= 0 && s < S) ? p.planes + (int64_t)s * p.plane_stride + (int64_t)g * p.n : nullptr;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int cc = 8 * u, col = c0 + cc;
              q[d][u] = make_uint4(0u, 0u, 0u, 0u);
              if (row && cc < half) {
                if (col + 7 < p.n) {
                  q[d][u] = __ldg(reinterpret_cast<const uint4*>(row + col));
                } else {
                  __nv_bfloat16* t8 = reinterpret_cast<__nv_bfloat16*>(&q[d][u]);
                  for (int w = 0; w < 8; ++w) t8[w] = (col + w < p.n) ? row[col + w] : __float2bfloat16_rn(0.f);
                }
              }
            }
          }
#pragma unroll
          for (int d = 0; d < 2; ++d) {
            const int s = s0 + d;
            if (s >= S) break;
            uint8_t* img = sX + (size_t)s * x_bytes;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int cc = 8 * u;
              if (cc >= half) break;
              const __nv_bfloat16* v8 = reinterpret_cast<const __nv_bfloat16*>(&q[d][u]);
#pragma unroll
              for (int w = 0; w < 8; ++w)
                *reinterpret_cast<__nv_bfloat16*>(img + sw_off2(h * half + cc + w, k, BN)) = v8[w];
            }
          }
        }
      } else {
        for (int s = 0; s < S; ++s) {
          const __nv_bfloat16* row = (g >= 0) ? p.planes + (int64_t)s * p.plane_stride + (int64_t)g * p.n : nullptr;
          uint8_t* img = sX + (size_t)s * x_bytes;
          for (int u = 0; u < half; ++u) {
            const int col = c0 + u;
            __nv_bfloat16 v = __float2bfloat16_rn(0.f);
            if (row && col < p.n) v = row[col];
            *reinterpret_cast<__nv_bfloat16*>(img + sw_off2(h * half + u, k, BN)) = v;
          }
        }
      }
      fence_proxy_async();
      tc::mbar_arrive(&xfull);
    }
  } else if (warp == 8) {
    // ---------------- MMA issuer: the whole warp walks the fully unrolled (s, t, k) sequence with
    // warp-uniform values, one elected lane issues (a runtime loop issued from one divergent lane
    // ran the tensor pipe at about two thirds of this rate)
    const bool leader = tc::elect_one();
    const uint32_t idesc = tc::instr_desc(1u, kNCP, BN);  // BF16 x BF16 -> FP32
    const uint64_t x_desc = tc::sw128_desc(tc::smem_u32(sX));
    const uint32_t x_khalf = (uint32_t)BN * kRowBytes;     // second 64-element K half of an X image
    bool ok = true;
    for (int64_t j = 0; j < items && ok; ++j) {
      bool w = !*vabort && tc::mbar_wait(&xfull, (uint32_t)(j & 1));
      if (w) w = tc::mbar_wait(&accempty, (uint32_t)(j & 1) ^ 1u);
      ok = __all_sync(0xffffffffu, w);
      if (!ok) break;
      tc::tc_fence_after();
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int64_t a = j * S + s;
        const int q = (int)(a & 1);
        w = !*vabort && tc::mbar_wait(&afull[q], (uint32_t)((a >> 1) & 1));
        ok = __all_sync(0xffffffffu, w);
        if (!ok) break;
        tc::tc_fence_after();
        // base descriptors plus compile-time offsets: a few integer adds per MMA
        const uint64_t a0 = tc::sw128_desc(tc::smem_u32(sA + (size_t)q * kASlice));
#pragma unroll
        for (int t = 0; t < S - s; ++t) {
          const uint32_t d = tmem + (uint32_t)((s + t) * BN);
          const uint64_t x0 = tc::desc_add(x_desc, (uint32_t)t * x_bytes);
          const uint64_t x1 = tc::desc_add(x0, x_khalf);
#pragma unroll
          for (int kk = 0; kk < kNCP / 16; ++kk) {
            const int kel = kk * 16;
            const uint32_t aoff = (uint32_t)(kel >> 6) * kNCP * kRowBytes + (uint32_t)((kel & 63) * 2);
            const uint32_t boff = (uint32_t)((kel & 63) * 2);
            if (leader)
              tc::mma_f16(d, tc::desc_add(a0, aoff), tc::desc_add(kel < 64 ? x0 : x1, boff), idesc,
                          (s == 0 && kk == 0) ? 0u : 1u);
          }
        }
        __syncwarp();
        if (leader) tc::mma_commit(&aempty[q]);
        __syncwarp();
      }
      if (!ok) break;
      if (leader) {
        tc::mma_commit(&xempty);
        tc::mma_commit(&accfull);
      }
      __syncwarp();
    }
    if (!ok && leader) fail();
  } else if (warp < 17) {
    // ---------------- epilogue: fold the 7 levels, scale, FP64 scatter-add; two warps per TMEM
    // lane quarter, alternate 16-column chunks each
    const int q = warp & 3, hh = (warp - 9) >> 2;
    const int i = q * 32 + lane;
    const int etid = (warp - 9) * 32 + lane;  // 0 .. 255
    for (int64_t j = 0; j < items; ++j) {
      const int64_t cell = blockIdx.x + (j / p.ntiles) * G;
      const int t = (int)(j % p.ntiles);
      bool ok = !*vabort && tc::mbar_wait(&accfull, (uint32_t)(j & 1));
      if (!ok) fail();
      // column exponents of this tile, shared by the 8 epilogue warps
      if (etid < BN) {
        const int col = t * BN + etid;
        int ex = col < p.n ? __ldg(p.cexp + col) : 0;
        s_cexp[etid] = ex == -100000 ? 0 : ex;
      }
      // one decision for all 8 warps (named barrier 1 also publishes the exponents)
      if (epi_any(!ok || *vabort)) break;
      tc::tc_fence_after();
      int g = -1, ea = 0;
      if (i < p.nc) {
        g = p.dofs[cell * p.nc + i];
        ea = p.aexp[cell * p.e_stride + i];
      }
      double* out = (g >= 0) ? p.Y + (int64_t)g * p.n : nullptr;
      const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
      for (int c0 = hh * 16; c0 < BN; c0 += 32) {
        float hi[16], lo[16];
        tc::tmem_ld16(lane_addr + (uint32_t)c0, hi);
#pragma unroll
        for (int u = 0; u < 16; ++u) lo[u] = 0.f;
        float scale = 0.00390625f;  // 2^-8
#pragma unroll 1
        for (int L = 1; L < S; ++L) {
          float v[16];
          tc::tmem_ld16(lane_addr + (uint32_t)(L * BN + c0), v);
#pragma unroll
          for (int u = 0; u < 16; ++u) two_sum(hi[u], lo[u], v[u] * scale);
          scale *= 0.00390625f;
        }
        if (out) {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int col = t * BN + c0 + u;
            if (col < p.n) {
              // (hi + lo) 2^(ea + ex - 16): two exact conversions by integer arithmetic, one FP64 add
              const int pw = ea + s_cexp[c0 + u] - 16;
              const double v = f32_scaled(hi[u], pw) + f32_scaled(lo[u], pw);
              atomicAdd(out + col, p.neg ? -v : v);
            }
          }
        }
      }
      // the tile's exponents may be overwritten only after every epilogue warp is done with them
      asm volatile("bar.sync 1, 256;" ::: "memory");
      tc::tc_fence_before();
      tc::mbar_arrive(&accempty);
    }
  } else {
    // ---------------- cell-slice loader (warp 17, one lane)
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t j = 0; j < items && !*vabort; ++j) {
        const int64_t cell = blockIdx.x + (j / p.ntiles) * G;
        const uint8_t* src = p.aimg + cell * p.a_stride;
        bool ok = true;
        for (int s = 0; s < S; ++s) {
          const int64_t a = j * S + s;
          const int q = (int)(a & 1);
          if (*vabort || !tc::mbar_wait(&aempty[q], (uint32_t)((a >> 1) & 1) ^ 1u)) {
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
        for (int64_t a = (issued > 2 ? issued - 2 : 0); a < issued; ++a)
          tc::mbar_wait(&afull[a & 1], (uint32_t)((a >> 1) & 1));
      }
    }
  }
  __syncthreads();
  if (warp == 8) {
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
  if (img.p) return;
  const int64_t cells = (useB && op.B_shared) ? 1 : op.n_cells;
  img.ensure((size_t)cells * S * kASlice);
  ex.ensure((size_t)cells * kNCP);
  const double* src = useB ? op.B64.p : op.A64.p;
  RC_CUDA(cudaMemsetAsync(img.p, 0, (size_t)cells * S * kASlice, s));
  const int64_t rows = cells * kNCP;
  pack_slices_kernel<<<(unsigned)std::min<int64_t>((rows + 127) / 128, 152 * 8), 128, 0, s>>>(cells, op.nc, src,
                                                                                            img.p, ex.p);
  RC_LAUNCH();
}

void launch_oz(cudaStream_t s, int num_sms, const FeOp& op, bool useB, const __nv_bfloat16* planes,
               int64_t plane_stride, const int* cexp, double* Y, int n, bool neg) {
  set_smem_limit(reinterpret_cast<const void*>(fe_oz_kernel), 232448 - 1024);
  ensure_slices(s, op, useB);
  const bool shared = useB && op.B_shared;
  FeOzArgs a{};
  a.n_cells = op.n_cells;
  a.nc = op.nc;
  a.n = n;
  a.BN = std::min(kMaxBN, std::max(16, (n + 15) / 16 * 16));
  a.ntiles = (n + a.BN - 1) / a.BN;
  a.dofs = op.dofs.p;
  a.aimg = useB ? op.ozB.p : op.ozA.p;
  a.a_stride = shared ? 0 : (int64_t)S * kASlice;
  a.aexp = useB ? op.ozBe.p : op.ozAe.p;
  a.e_stride = shared ? 0 : kNCP;
  a.planes = planes;
  a.plane_stride = plane_stride;
  a.cexp = cexp;
  a.Y = Y;
  a.neg = neg ? 1 : 0;
  a.vec = (n % 8) == 0;
  a.err = op.err;
  const size_t smem = 2 * kASlice + (size_t)S * a.BN * kNCP * 2 + 1024;
  const unsigned grid = (unsigned)std::min<int64_t>(op.n_cells, num_sms);
  const double nc = op.nc, C = (double)op.n_cells;
  prof::Scope ps(s, RCHFSI_KERNEL_FE_CELL_F64, 2.0 * nc * nc * C * n,
                 14.0 * (double)C * nc * n + 8.0 * 2.0 * (double)C * nc * n + (shared ? 1.0 : C) * S * kASlice);
  fe_oz_kernel<<<grid, kThreads, smem, s>>>(a);
  RC_LAUNCH();
}

}  // namespace

void fe_apply_f64_rows_tc(cudaStream_t s, const FeOp& op, bool useB, const double* X, double* Y, int n,
                          int num_sms) {
  RC_CHECK(op.nc <= kNCP, RCHFSI_ERR_INVALID_ARG, "n_c larger than 128");
  const int64_t m = op.m;
  RC_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * m * n, s));
  // column exponents over every row (both halves of a complex block), then the slice planes
  int* cexp = op.ozcexp.ensure(n);
  fill_int(s, cexp, n, -100000);
  colexp_kernel<<<(unsigned)std::min<int64_t>(m, 152 * 8), 256, 0, s>>>(m, n, X, cexp);
  RC_LAUNCH();
  const int64_t total = m * n;
  __nv_bfloat16* planes = op.ozplanes.ensure((size_t)S * total);
  if (n % 2 == 0) {
    // 32 column pairs x 8 rows per block; enough row blocks for ~16 blocks per SM
    const unsigned gx = cdiv(n / 2, 32);
    const unsigned gy = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(m, 8), (int64_t)num_sms * 16 / gx + 1));
    xslice_kernel<<<dim3(gx, gy), dim3(32, 8), 0, s>>>(m, n, X, cexp, planes);
  } else {
    xslice1_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16), 256, 0, s>>>(total, n, X, cexp,
                                                                                               planes);
  }
  RC_LAUNCH();
  if (!op.cplx) {
    launch_oz(s, num_sms, op, useB, planes, total, cexp, Y, n, false);
    return;
  }
  // complex operator on the real embedding (rows [0, mc) real parts, [mc, 2 mc) imaginary parts):
  //   Y_r = Ar X_r - Ai X_i,  Y_i = Ai X_r + Ar X_i;  the real B acts on each half
  const int64_t off = op.mc * (int64_t)n;
  if (useB) {
    launch_oz(s, num_sms, op, true, planes, total, cexp, Y, n, false);
    launch_oz(s, num_sms, op, true, planes + off, total, cexp, Y + off, n, false);
    return;
  }
  const FeOp& im = *op.imag;
  launch_oz(s, num_sms, op, false, planes, total, cexp, Y, n, false);
  launch_oz(s, num_sms, im, false, planes + off, total, cexp, Y, n, true);
  launch_oz(s, num_sms, im, false, planes, total, cexp, Y + off, n, false);
  launch_oz(s, num_sms, op, false, planes + off, total, cexp, Y + off, n, false);
}

}  // namespace rchfsi
