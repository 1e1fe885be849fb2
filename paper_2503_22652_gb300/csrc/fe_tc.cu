// Finite-element filter product on the tcgen05 tensor cores:
//   Rx[dofs(c), :] += a * A_c (D^-1 Ry)[dofs(c), :]      for every cell c     (dmode 1)
// (dmode 2: the D^-1 scaling is applied to the output rows instead; dmode 0: none).
//
// Per (cell, column tile) work item: D (128 x BN, FP32 in TMEM) = A_c (128 x 128, cell matrix padded
// from n_c <= 128) x X_c (128 x BN, the cell's rows of the block).  A persistent CTA per SM walks its
// cells; for each cell it streams the column tiles.  Warp roles:
//   warps 0-7  gather: thread (k, h) reads half of row dofs(c)[k] of the tile of R_Y (eight 16-byte
//              loads in flight), scales by D^-1, rounds to the operand type and writes it transposed
//              into the K-major 128-byte-swizzled shared-memory image of X_c (two stages), then
//              fence.proxy.async + mbarrier arrive;
//   warp 8     MMA issuer (the whole warp, one elected lane issuing): tcgen05.mma kind::tf32
//              (K = 8) or kind::f16 (BF16, K = 16) into one of two TMEM accumulators,
//              tcgen05.commit to release stages / buffers;
//   warps 9-12 epilogue: tcgen05.ld of the accumulator rows (thread = cell-local dof), scaling, and
//              vectorised float4 atomic scatter-add into R_X (dofs shared by neighbouring cells get
//              one add per cell);
//   warp 13    cell-matrix loader: one cp.async.bulk of the pre-swizzled cell-matrix image (two
//              buffers, so the next cell's matrix streams in while the current one is in use).
// The cell-matrix images are built once per operator and precision by a packing kernel.  Every
// mbarrier wait is bounded; on a timeout the kernel raises the error flag and unwinds.
//
// One launch takes a list of "parts" (up to kMaxParts): each part is one real cell-matrix product
// (its own cells, images, input and output blocks, width n, tile width BN and scalar a), so the four
// real products of a complex operator, or the products of many problems (a batch of k-points),
// run as a single persistent launch over the concatenated cell list.  The scalar a may be read
// from device memory (a coefficient table), so a captured CUDA graph of the filter loop stays valid
// when the Chebyshev coefficients change.
#include "fe_tc.cuh"
#include "prof.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace rchfsi {
namespace {

constexpr int kNCP = 128;         // padded cell size (MMA M and K)
constexpr int kThreads = 448;     // 14 warps
constexpr int kRowBytes = 128;

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row r, k) in a K-major 128B-swizzled image with `rows` rows per k-block.
template <int ES>
__device__ __forceinline__ uint32_t sw_off(int r, int k, int rows) {
  constexpr int per = kRowBytes / ES;  // elements per 128-byte row
  const int kb = k / per;
  const int byte = (k % per) * ES;
  const int chunk = (byte >> 4) ^ (r & 7);
  return (uint32_t)kb * rows * kRowBytes + (uint32_t)r * kRowBytes + (chunk << 4) + (byte & 15);
}

// Pack cell matrices (n_cells x nc x nc, FP64, row-major) into per-cell 128 x 128 swizzled images.
template <bool BF16>
__global__ void pack_cells_kernel(int64_t n_cells, int nc, const double* __restrict__ A, uint8_t* __restrict__ img) {
  constexpr int ES = BF16 ? 2 : 4;
  const int64_t per_cell = (int64_t)kNCP * kNCP;
  const int64_t total = n_cells * per_cell;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / per_cell;
    const int r = (int)((e % per_cell) / kNCP), k = (int)(e % kNCP);
    const double v = (r < nc && k < nc) ? A[(c * nc + r) * nc + k] : 0.0;
    uint8_t* base = img + c * per_cell * ES + sw_off<ES>(r, k, kNCP);
    if (BF16) *reinterpret_cast<__nv_bfloat16*>(base) = __float2bfloat16_rn((float)v);
    else *reinterpret_cast<float*>(base) = tf32_rna((float)v);
  }
}

constexpr int kMaxParts = 64;

struct FePart {
  int64_t n_cells, cell_off;  // cells of this part, and their offset in the concatenated list
  const int* dofs;
  const uint8_t* img;         // packed cell images
  const float* Ry;
  float* Rx;
  const double* dinv;
  const double* coef;         // if set, a = sign * *coef (read by the kernel), else a = a_val
  float a_val, sign;
  int nc, n, BN, ntiles, dmode, vec;
};

struct FeBatch {
  int nparts;
  int64_t total_cells;
  uint32_t tmem_cols;
  int maxBN;
  int* err;
  FePart part[kMaxParts];
};

// Part holding the global cell g (parts are few: a linear scan).
__device__ __forceinline__ int part_of(const FeBatch& p, int64_t g) {
  int q = 0;
  while (q + 1 < p.nparts && g >= p.part[q + 1].cell_off) ++q;
  return q;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(tc::smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1) fe_tc_kernel(const __grid_constant__ FeBatch p) {
  constexpr int ES = BF16 ? 2 : 4;
  constexpr int KMMA = BF16 ? 16 : 8;
  constexpr uint32_t kFmt = BF16 ? 1u : 2u;
  constexpr uint32_t kABytes = kNCP * kNCP * ES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t afull[2], aempty[2], bfull[2], bempty[2], accfull[2], accempty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t b_bytes = (uint32_t)p.maxBN * kNCP * ES;  // one operand stage at the widest tile
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA[2] = {smem, smem + kABytes};
  uint8_t* sB[2] = {smem + 2 * kABytes, smem + 2 * kABytes + b_bytes};

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&afull[i], 1);
      tc::mbar_init(&aempty[i], 1);
      tc::mbar_init(&bfull[i], 256);
      tc::mbar_init(&bempty[i], 1);
      tc::mbar_init(&accfull[i], 1);
      tc::mbar_init(&accempty[i], 128);
    }
    tc::fence_barrier_init();
    abort_flag = 0;
  }
  if (warp == 8) {
    tc::tmem_alloc(&tmem_slot, p.tmem_cols);
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

  if (warp < 8) {
    // ---------------- gather: thread (k, h) owns cell-local dof k, columns h*BN/2 .. of the tile;
    // eight 16-byte loads are issued before any is used, to keep enough bytes in flight
    const int k = threadIdx.x & 127, h = threadIdx.x >> 7;
    int64_t j = 0;
    bool stop = false;
    for (int64_t g = blockIdx.x; g < p.total_cells && !stop; g += G) {
      const FePart& P = p.part[part_of(p, g)];
      const int64_t cell = g - P.cell_off;
      const int BN = P.BN, half = BN / 2;
      int gi = -1;
      float sc = 0.f;
      if (k < P.nc) {
        gi = P.dofs[cell * P.nc + k];
        sc = (P.dmode == 1) ? (float)P.dinv[gi] : 1.f;
      }
      const float* row = (gi >= 0) ? P.Ry + (int64_t)gi * P.n : nullptr;
      for (int t = 0; t < P.ntiles; ++t, ++j) {
        const int bs = (int)(j & 1);
        if (*vabort || !tc::mbar_wait(&bempty[bs], (uint32_t)((j >> 1) & 1) ^ 1u)) {
          fail();
          stop = true;
          break;
        }
        uint8_t* img = sB[bs];
        const int c0 = t * BN + h * half;  // first column of this thread
        for (int nn = 0; nn < half; nn += 32) {
          float4 q[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int cc = nn + 4 * u, col = c0 + cc;
            q[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row && cc < half) {
              if (P.vec && col + 3 < P.n) {
                q[u] = __ldg(reinterpret_cast<const float4*>(row + col));
              } else {
                float* f = reinterpret_cast<float*>(&q[u]);
                for (int w = 0; w < 4; ++w)
                  if (col + w < P.n) f[w] = __ldg(row + col + w);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int cc = nn + 4 * u;
            if (cc >= half) break;
            const float* f = reinterpret_cast<const float*>(&q[u]);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              const float x = f[w] * sc;
              uint8_t* dst = img + sw_off<ES>(h * half + cc + w, k, BN);
              if (BF16) *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(x);
              else *reinterpret_cast<float*>(dst) = tf32_rna(x);
            }
          }
        }
        fence_proxy_async();
        tc::mbar_arrive(&bfull[bs]);
      }
    }
  } else if (warp == 8) {
    // ---------------- MMA issuer: the whole warp walks the loops with warp-uniform values, one
    // elected lane issues
    const bool leader = tc::elect_one();
    int64_t j = 0, cl = 0;
    bool stop = false;
    for (int64_t g = blockIdx.x; g < p.total_cells && !stop; g += G, ++cl) {
      const FePart& P = p.part[part_of(p, g)];
      const int BN = P.BN;
      const uint32_t idesc = tc::instr_desc(kFmt, kNCP, BN);
      const int ab = (int)(cl & 1);
      for (int t = 0; t < P.ntiles; ++t, ++j) {
        const int bs = (int)(j & 1), xb = (int)(j & 1);
        bool ok = !*vabort;
        if (ok && t == 0) ok = tc::mbar_wait(&afull[ab], (uint32_t)((cl >> 1) & 1));
        if (ok) ok = tc::mbar_wait(&bfull[bs], (uint32_t)((j >> 1) & 1));
        if (ok) ok = tc::mbar_wait(&accempty[xb], (uint32_t)((j >> 1) & 1) ^ 1u);
        if (!__all_sync(0xffffffffu, ok)) {
          if (leader) fail();
          stop = true;
          break;
        }
        tc::tc_fence_after();
        // base descriptors plus compile-time offsets (one more add per 128-byte K block of B)
        const uint64_t a0 = tc::sw128_desc(tc::smem_u32(sA[ab]));
        const uint64_t b0 = tc::sw128_desc(tc::smem_u32(sB[bs]));
        const uint32_t bblk = (uint32_t)BN * kRowBytes;
        const uint32_t d = tmem + (uint32_t)(xb * p.maxBN);
        constexpr int per = kRowBytes / ES;
#pragma unroll
        for (int kk = 0; kk < kNCP / KMMA; ++kk) {
          const int kel = kk * KMMA;
          const uint32_t aoff = (uint32_t)(kel / per) * kNCP * kRowBytes + (uint32_t)((kel % per) * ES);
          const uint64_t ad = tc::desc_add(a0, aoff);
          const uint64_t bd = tc::desc_add(b0, (uint32_t)(kel / per) * bblk + (uint32_t)((kel % per) * ES));
          if (leader) {
            if (BF16) tc::mma_f16(d, ad, bd, idesc, kk > 0 ? 1u : 0u);
            else tc::mma_tf32(d, ad, bd, idesc, kk > 0 ? 1u : 0u);
          }
        }
        __syncwarp();
        if (leader) {
          tc::mma_commit(&bempty[bs]);
          tc::mma_commit(&accfull[xb]);
          if (t == P.ntiles - 1) tc::mma_commit(&aempty[ab]);
        }
        __syncwarp();
      }
    }
  } else if (warp < 13) {
    // ---------------- epilogue: TMEM -> scatter-add
    const int q = warp & 3;
    const int i = q * 32 + lane;  // cell-local dof of this thread's accumulator row
    int64_t j = 0;
    bool stop = false;
    for (int64_t g = blockIdx.x; g < p.total_cells && !stop; g += G) {
      const FePart& P = p.part[part_of(p, g)];
      const int64_t cell = g - P.cell_off;
      const int BN = P.BN;
      const float a = P.sign * (P.coef ? (float)__ldg(P.coef) : P.a_val);
      int gi = -1;
      float sc = 0.f;
      if (i < P.nc) {
        gi = P.dofs[cell * P.nc + i];
        sc = a * ((P.dmode == 2) ? (float)P.dinv[gi] : 1.f);
      }
      float* out = (gi >= 0) ? P.Rx + (int64_t)gi * P.n : nullptr;
      for (int t = 0; t < P.ntiles; ++t, ++j) {
        const int xb = (int)(j & 1);
        bool ok = !*vabort && tc::mbar_wait(&accfull[xb], (uint32_t)((j >> 1) & 1));
        if (!ok) fail();
        if (!__all_sync(0xffffffffu, ok && !*vabort)) {
          stop = true;
          break;
        }
        tc::tc_fence_after();
        const int n0 = t * BN;
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(xb * p.maxBN);
        for (int c0 = 0; c0 < BN; c0 += 16) {
          float v[16];
          tc::tmem_ld16(lane_addr + c0, v);
          if (out) {
#pragma unroll
            for (int u = 0; u < 16; u += 4) {
              const int col = n0 + c0 + u;
              if (P.vec && col + 3 < P.n) {
                atomicAdd(reinterpret_cast<float4*>(out + col),
                          make_float4(sc * v[u], sc * v[u + 1], sc * v[u + 2], sc * v[u + 3]));
              } else {
#pragma unroll
                for (int w = 0; w < 4; ++w)
                  if (col + w < P.n) atomicAdd(out + col + w, sc * v[u + w]);
              }
            }
          }
        }
        tc::tc_fence_before();
        tc::mbar_arrive(&accempty[xb]);
      }
    }
  } else {
    // ---------------- cell-matrix loader (warp 13, one lane)
    if (lane == 0) {
      int64_t issued = 0, cl = 0;
      for (int64_t g = blockIdx.x; g < p.total_cells; g += G, ++cl) {
        const int ab = (int)(cl & 1);
        if (*vabort || !tc::mbar_wait(&aempty[ab], (uint32_t)((cl >> 1) & 1) ^ 1u)) {
          fail();
          break;
        }
        const FePart& P = p.part[part_of(p, g)];
        const int64_t cell = g - P.cell_off;
        tc::mbar_arrive_expect_tx(&afull[ab], kABytes);
        bulk_g2s(sA[ab], P.img + cell * (int64_t)kABytes, kABytes, &afull[ab]);
        ++issued;
      }
      if (*vabort) {
        // wait (bounded) for copies that may still be landing in this CTA's shared memory
        for (int64_t c2 = (issued > 2 ? issued - 2 : 0); c2 < issued; ++c2)
          tc::mbar_wait(&afull[c2 & 1], (uint32_t)((c2 >> 1) & 1));
      }
    }
  }
  __syncthreads();
  if (warp == 8) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, p.tmem_cols);
  }
}

}  // namespace

namespace {

// Widest column tile (multiple of 16) that keeps two cell-matrix buffers and two operand stages in
// shared memory and two accumulators in TMEM, split evenly over the block width n.
int default_bn(int n, bool bf) {
  const int bn_max = bf ? 208 : 96;
  const int ntiles = (n + bn_max - 1) / bn_max;
  int BN = (((n + ntiles - 1) / ntiles) + 15) / 16 * 16;
  return BN < 16 ? 16 : BN;
}

const uint8_t* ensure_images(cudaStream_t s, FeOp& op, bool bf) {
  const int ES = bf ? 2 : 4;
  DevBuf<uint8_t>& img = bf ? op.img16 : op.imgtf;
  if (!img.p) {
    const size_t per_cell = (size_t)kNCP * kNCP * ES;
    img.ensure(per_cell * op.n_cells);
    const int64_t total = op.n_cells * (int64_t)kNCP * kNCP;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
    if (bf) pack_cells_kernel<true><<<blocks, 256, 0, s>>>(op.n_cells, op.nc, op.A64.p, img.p);
    else pack_cells_kernel<false><<<blocks, 256, 0, s>>>(op.n_cells, op.nc, op.A64.p, img.p);
    RC_LAUNCH();
  }
  return img.p;
}

}  // namespace

int fe_tc_bn_max(int precision) { return precision == RCHFSI_BF16 ? 208 : 96; }

void fe_tc_parts_prepare(cudaStream_t s, FeOp& op, int precision) {
  const bool bf = precision == RCHFSI_BF16;
  ensure_images(s, op, bf);
  if (op.cplx) ensure_images(s, *op.imag, bf);
}

void fe_tc_batch(cudaStream_t s, int precision, const FeTcPart* parts, int nparts, int num_sms) {
  RC_CHECK(precision == RCHFSI_TF32 || precision == RCHFSI_BF16, RCHFSI_ERR_INVALID_ARG, "FE tensor path: TF32/BF16");
  RC_CHECK(nparts >= 1 && nparts <= kMaxParts, RCHFSI_ERR_INVALID_ARG, "FE tensor path: 1..64 parts per launch");
  const bool bf = precision == RCHFSI_BF16;
  const int ES = bf ? 2 : 4;
  FeBatch b{};
  b.nparts = nparts;
  b.maxBN = 16;
  int64_t off = 0;
  double flops = 0.0, bytes = 0.0;
  for (int q = 0; q < nparts; ++q) {
    const FeTcPart& t = parts[q];
    FeOp& op = *t.op;
    RC_CHECK(op.nc <= kNCP, RCHFSI_ERR_INVALID_ARG, "n_c larger than 128");
    RC_CHECK(t.n >= 1, RCHFSI_ERR_INVALID_ARG, "FE tensor path: empty block");
    FePart& P = b.part[q];
    P.n_cells = op.n_cells;
    P.cell_off = off;
    P.dofs = op.dofs.p;
    P.img = ensure_images(s, op, bf);
    P.Ry = t.Ry;
    P.Rx = t.Rx;
    P.dinv = op.Dinv.p;
    P.coef = t.coef;
    P.a_val = t.a;
    P.sign = t.sign;
    P.nc = op.nc;
    P.n = t.n;
    P.BN = t.BN > 0 ? t.BN : default_bn(t.n, bf);
    RC_CHECK(P.BN % 16 == 0 && P.BN >= 16 && P.BN <= fe_tc_bn_max(precision), RCHFSI_ERR_INVALID_ARG,
             "FE tensor path: tile width must be a multiple of 16 up to the precision's maximum");
    P.ntiles = (t.n + P.BN - 1) / P.BN;
    P.dmode = t.dmode;
    P.vec = (t.n % 4) == 0;
    b.maxBN = std::max(b.maxBN, P.BN);
    off += op.n_cells;
    const double nc = op.nc, C = (double)op.n_cells, rows = (double)(op.cplx ? op.mc : op.m);
    flops += 2.0 * nc * nc * C * t.n;
    bytes += 4.0 * 3.0 * rows * t.n + (double)ES * nc * nc * C;
  }
  b.total_cells = off;
  b.err = parts[0].op->err;
  uint32_t cols = 32;
  while (cols < (uint32_t)(2 * b.maxBN)) cols <<= 1;
  b.tmem_cols = cols;
  const size_t per_cell = (size_t)kNCP * kNCP * ES;
  const size_t smem = 2 * per_cell + 2 * (size_t)b.maxBN * kNCP * ES + 1024;
  RC_CHECK(smem <= 232448 - 1024, RCHFSI_ERR_INVALID_ARG, "FE tensor path: shared memory plan too large");
  auto kern = bf ? fe_tc_kernel<true> : fe_tc_kernel<false>;
  // one limit for every plan (a per-launch value would race with a concurrent launch of a wider plan)
  set_smem_limit(reinterpret_cast<const void*>(kern), 232448 - 1024);
  const unsigned grid = (unsigned)std::min<int64_t>(b.total_cells, (int64_t)num_sms);
  prof::Scope ps(s, RCHFSI_KERNEL_FE_CELL, flops, bytes);
  kern<<<grid, kThreads, smem, s>>>(b);
  RC_LAUNCH();
}

void fe_tc_product(cudaStream_t s, FeOp& op, int precision, const float* Ry, float* Rx, int n, float a, int dmode) {
  int dev = 0, sms = 152;
  RC_CUDA(cudaGetDevice(&dev));
  RC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  FeTcPart parts[4];
  const int np = fe_tc_parts(op, Ry, Rx, n, a, nullptr, dmode, 0, parts);
  fe_tc_batch(s, precision, parts, np, sms);
}

int fe_tc_parts(FeOp& op, const float* Ry, float* Rx, int n, float a, const double* coef, int dmode, int BN,
                FeTcPart* out) {
  if (!op.cplx) {
    out[0] = FeTcPart{&op, Ry, Rx, n, a, coef, 1.f, dmode, BN};
    return 1;
  }
  // complex operator on the real embedding: rows [0, mc) real parts, [mc, 2 mc) imaginary parts
  //   Y_r += a (Ar X_r - Ai X_i),   Y_i += a (Ai X_r + Ar X_i)
  const int64_t off = op.mc * (int64_t)n;
  FeOp& im = *op.imag;
  out[0] = FeTcPart{&op, Ry, Rx, n, a, coef, 1.f, dmode, BN};
  out[1] = FeTcPart{&im, Ry + off, Rx, n, a, coef, -1.f, dmode, BN};
  out[2] = FeTcPart{&im, Ry, Rx + off, n, a, coef, 1.f, dmode, BN};
  out[3] = FeTcPart{&op, Ry + off, Rx + off, n, a, coef, 1.f, dmode, BN};
  return 4;
}

}  // namespace rchfsi
