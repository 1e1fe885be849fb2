// Fused degree step of the finite-element R-ChFSI filter (the loop body of Algorithm 3) on the
// tcgen05 tensor cores, in one pass over the block.
//
// The recurrence R_k = a_k A D^-1 R_{k-1} + b_k R_{k-1} + c_k R_{k-2} + a_k W Lambda_{k-1} runs on
// scaled iterates S_j = s_j R_j, with s_k = s_{k-2} / c_k chosen on the host, so that
//   S_k = S_{k-2} + alpha A D^-1 S_{k-1} + beta S_{k-1} + omega W Lambda_{k-1},
//   alpha = s_k a_k / s_{k-1},  beta = s_k b_k / s_{k-1},  omega = s_k a_k:
// the old iterate enters with coefficient 1, so the whole step is additions into the buffer that
// holds S_{k-2}.  The cell products are added with vector atomics (a dof shared by several cells
// receives one add per cell); beta S_{k-1} + omega W Lambda is added once per dof, by the cell that
// owns it (the first cell, in cell order, that contains it).  Each of S_{k-1}, S_{k-2} and W is
// then read once and S_k written once per step, the four block streams of the algorithm, plus
// the cell matrices.
//
// Per (cell, column tile): D (128 x BN, FP32 in TMEM) = T + (A_c D_c^-1) V_c, where A_c D_c^-1 is the
// cell matrix with its columns scaled by D^-1 at the cell's dofs (padded from n_c <= 128 to 128 x
// 128, packed once per operator as a K-major 128-byte-swizzled TF32 image), V_c (128 x BN) the
// cell's rows of S_{k-1}, and T the owner terms of the cell's owned rows divided by alpha, so that
// alpha D is the whole contribution of the cell.  The rows of V_c and the owned rows of W are
// gathered from the row-major blocks with 16-byte cp.async copies by 256 threads (a warp
// instruction copies whole 256-byte row segments) into a ring of 128-byte-swizzled stages, up to
// two tiles ahead of the tile being converted.  (A single loader warp issuing the copies, or TMA
// tile::gather4 copies of four 128-byte rows, moved only ~6 bytes per clock per SM.)  The same
// threads then convert: each (one cell node, half of the columns) reads its row, stores T into the
// accumulator with tcgen05.st and, after a barrier among the converters, rewrites the stage in
// place as the K-major TF32 operand of the MMA (the swizzled reads and the operand writes are both
// free of shared-memory bank conflicts).
//
// Warp roles (448 threads):
//   warp 0     cell images: one bulk copy per cell (nA buffers);
//   warp 1     MMA issuer (the whole warp walks the loop, one elected lane issues), accumulating
//              onto the owner terms in one of two TMEM accumulators of BN columns;
//   warps 2-9  gather + convert (warp w: nodes 32 (w % 4).., the TMEM lanes it may access, and
//              half of the tile's columns);
//   warps 10-13 epilogue: TMEM lanes 32 (w % 4).. (one cell node per thread); alpha scaling and
//              red.global.add.v4.f32 into the output rows.
// Every mbarrier wait is bounded; on a timeout the kernel raises the error flag, waits (bounded)
// for its copies and MMAs in flight, releases TMEM and returns.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fe_step.cuh"
#include "prof.cuh"
#include "tc_ptx.cuh"

namespace rchfsi {
namespace {

constexpr int kNCP = 128;                       // padded cell size (MMA M and K)
constexpr int kThreads = 448;                   // 14 warps
constexpr uint32_t kABytes = kNCP * kNCP * 4;   // TF32 cell image
constexpr uint32_t kChunkBytes = kNCP * 128;    // 32 columns of V_c: 128 rows of 128 bytes
constexpr int kWRows = 80;                      // owned rows of W staged per cell (at most)
constexpr uint32_t kWChunkBytes = kWRows * 128;
constexpr int kMaxParts = 64;
constexpr int kMaxStages = 6;
constexpr int kSmemMax = 232448;                // dynamic + static shared memory per CTA

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row r, k) of a 128 x 128 K-major 128-byte-swizzled FP32 image.
__device__ __forceinline__ uint32_t sw_off4(int r, int k) {
  const int kb = k >> 5, byte = (k & 31) * 4;
  const int chunk = (byte >> 4) ^ (r & 7);
  return (uint32_t)kb * kNCP * 128 + (uint32_t)r * 128 + (chunk << 4) + (byte & 15);
}

// (A_c D_c^-1) images: column k of cell c scaled by dinv[dofs(c, k)], rounded to TF32.
__global__ void pack_scaled_kernel(int64_t n_cells, int nc, const double* __restrict__ A, const int* __restrict__ dofs,
                                   const double* __restrict__ dinv, uint8_t* __restrict__ img) {
  const int64_t per_cell = (int64_t)kNCP * kNCP;
  const int64_t total = n_cells * per_cell;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / per_cell;
    const int r = (int)((e % per_cell) / kNCP), k = (int)(e % kNCP);
    const double v = (r < nc && k < nc) ? A[(c * nc + r) * nc + k] * dinv[dofs[c * nc + k]] : 0.0;
    *reinterpret_cast<float*>(img + c * per_cell * 4 + sw_off4(r, k)) = tf32_rna((float)v);
  }
}

struct StepPartDev {
  const int* dofs;
  const int8_t* own_pos;  // per cell 128 entries: >= 0 when the cell owns its node k
  const uint8_t* img;
  const float* V;
  const float* W;
  float* U;
  const float* lam;
  const double* coef;
  int64_t n_cells, cell_off;
  float alpha, beta, omega, sign;
  int nc, n, ntiles, owner;  // owner = 0: no owner terms in this part
};

struct StepBatch {
  StepPartDev part[kMaxParts];
  int64_t total_cells;
  int nparts, nA, nslots;
  uint32_t tmem_cols;
  int* err;
};

__device__ __forceinline__ int part_of(const StepBatch& p, int64_t g) {
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

// 16-byte asynchronous copy global -> shared (L2 only); `in` = false writes 16 zero bytes instead.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool in) {
  // no memory clobber: the copy is ordered by the mbarrier that completes with it, and loads that
  // feed later copies may be scheduled ahead of it
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(in ? 16 : 0));
}

// Arrive on `bar` once every cp.async this thread issued before has completed (the barrier's count
// includes this arrival).
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// Byte offset of element (row r, k) of a K-major 128-byte-swizzled FP32 operand with `rows` rows
// per 32-element K block.
__device__ __forceinline__ uint32_t img_off(int r, int k, int rows) {
  const int kb = k >> 5, byte = (k & 31) * 4;
  return (uint32_t)kb * rows * 128 + (uint32_t)r * 128 + ((((byte >> 4) ^ (r & 7))) << 4) + (byte & 15);
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1) fe_step_kernel(const __grid_constant__ StepBatch p) {
  constexpr int NCH = BN / 32;
  constexpr int CPR = BN / 4;                     // 16-byte chunks per row of a tile
  constexpr int HB = BN / 2;                      // columns of one converter thread per tile
  constexpr uint32_t kHalf = NCH * kChunkBytes;   // 128 rows of BN FP32 values
  constexpr uint32_t kSlotBytes = kHalf + NCH * kWChunkBytes;  // V rows (then the operand), owned W rows
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t afull[2], aempty[2], bfull[kMaxStages], bempty[kMaxStages], ifull[kMaxStages],
      accfull[2], accempty[2], cvt_read, mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + (size_t)p.nA * kABytes;
  float* sL = reinterpret_cast<float*>(sB + (size_t)p.nslots * kSlotBytes);  // Lambda of each stage's columns

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&afull[i], 1);
      tc::mbar_init(&aempty[i], 1);
      tc::mbar_init(&accfull[i], 1);
      tc::mbar_init(&accempty[i], 128);
    }
    for (int i = 0; i < kMaxStages; ++i) {
      tc::mbar_init(&bfull[i], 256);  // every gathering thread, once its copies have landed
      tc::mbar_init(&bempty[i], 1);
      tc::mbar_init(&ifull[i], 256);
    }
    tc::mbar_init(&cvt_read, 256);
    tc::mbar_init(&mma_done, 1);
    tc::fence_barrier_init();
    abort_flag = 0;
  }
  if (warp == 1) {
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
  const int nA = p.nA, nS = p.nslots;

  if (warp == 0) {
    // ---------------- cell images: one bulk copy per cell into nA buffers
    if (lane == 0) {
      int64_t cl = 0;
      for (int64_t g = blockIdx.x; g < p.total_cells; g += G, ++cl) {
        const int ab = (int)(cl % nA);
        if (*vabort || !tc::mbar_wait(&aempty[ab], (uint32_t)((cl / nA) & 1) ^ 1u)) {
          fail();
          break;
        }
        const StepPartDev& P = p.part[part_of(p, g)];
        tc::mbar_arrive_expect_tx(&afull[ab], kABytes);
        bulk_g2s(sA + (size_t)ab * kABytes, P.img + (g - P.cell_off) * (int64_t)kABytes, kABytes, &afull[ab]);
      }
      if (*vabort)  // let the copies already issued land before the shared memory is released (bounded)
        for (int64_t c2 = (cl > nA ? cl - nA : 0); c2 < cl; ++c2) tc::mbar_wait(&afull[c2 % nA], (uint32_t)((c2 / nA) & 1));
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: accumulates onto the owner terms the converters stored
    const bool leader = tc::elect_one();
    constexpr uint32_t idesc = tc::instr_desc(2u, kNCP, BN);  // TF32, both operands K-major
    int64_t j = 0, cl = 0;
    bool stop = false;
    for (int64_t g = blockIdx.x; g < p.total_cells && !stop; g += G, ++cl) {
      const StepPartDev& P = p.part[part_of(p, g)];
      const int ab = (int)(cl % nA);
      for (int t = 0; t < P.ntiles; ++t, ++j) {
        const int s = (int)(j % nS), xb = (int)(j & 1);
        bool ok = !*vabort;
        if (ok && t == 0) ok = tc::mbar_wait(&afull[ab], (uint32_t)((cl / nA) & 1));
        if (ok) ok = tc::mbar_wait(&ifull[s], (uint32_t)((j / nS) & 1));
        if (!__all_sync(0xffffffffu, ok)) {
          if (leader) fail();
          stop = true;
          break;
        }
        tc::tc_fence_after();
        const uint64_t a0 = tc::sw128_desc(tc::smem_u32(sA + (size_t)ab * kABytes));
        const uint64_t b0 = tc::sw128_desc(tc::smem_u32(sB + (size_t)s * kSlotBytes));
        const uint32_t d = tmem + (uint32_t)(xb * BN);
#pragma unroll
        for (int kk = 0; kk < kNCP / 8; ++kk) {
          const int kel = kk * 8;
          const uint32_t aoff = (uint32_t)(kel >> 5) * kNCP * 128 + (uint32_t)((kel & 31) * 4);
          const uint32_t boff = (uint32_t)(kel >> 5) * BN * 128 + (uint32_t)((kel & 31) * 4);
          if (leader) tc::mma_tf32(d, tc::desc_add(a0, aoff), tc::desc_add(b0, boff), idesc, 1u);
        }
        __syncwarp();
        if (leader) {
          tc::mma_commit(&bempty[s]);
          tc::mma_commit(&accfull[xb]);
          if (t == P.ntiles - 1) tc::mma_commit(&aempty[ab]);
        }
        __syncwarp();
      }
    }
    // every MMA issued has completed before TMEM is released
    if (leader) {
      tc::mma_commit(&mma_done);
      tc::mbar_wait(&mma_done, 0u);
    }
    __syncwarp();
  } else if (warp < 10) {
    // ---------------- gather + convert (256 threads)
    // Gather (all 256 threads, coalesced: a warp instruction copies whole 256-byte row segments):
    // the tile's rows of V and owned rows of W as 16-byte cp.async copies into the 128-byte-swizzled
    // stage, and the tile's Lambda values; each thread arrives on the stage's barrier once its copies
    // have landed.  Tiles are gathered `ahead` tiles ahead of the one being converted.
    // Convert (thread (k, h): cell node k = TMEM lane k, half h of the columns): the owner terms
    // into the accumulator (tcgen05.st), then, once all threads have read the stage, the stage
    // rewritten in place as the K-major TF32 operand.
    const int gt = threadIdx.x - 64;         // 0..255
    const int k = (warp & 3) * 32 + lane;
    const int h = (warp - 2) >> 2;
    const int ahead = nS - 1;  // tiles gathered ahead: tile j + ahead reuses the stage of tile j - 1
    // gather cursor (the tile `ahead` tiles ahead of the one converted): this thread copies the rows
    // kr = (it * 256 + gt) / CPR of every tile, the same for all tiles of a cell, so their offsets
    // and owner flags are loaded once per cell
    constexpr int kIt = kNCP * CPR / 256;
    int64_t gg = blockIdx.x, jg = 0;
    int tg = 0;
    int64_t rowoff[kIt];
    int ownpos[kIt];
    auto gather = [&]() -> bool {
      if (gg >= p.total_cells) return true;
      const StepPartDev& P = p.part[part_of(p, gg)];
      const int s = (int)(jg % nS);
      const int64_t cell = gg - P.cell_off;
      if (tg == 0) {
#pragma unroll
        for (int it = 0; it < kIt; ++it) {
          const int kr = (it * 256 + gt) / CPR;
          rowoff[it] = (int64_t)__ldg(P.dofs + cell * P.nc + min(kr, P.nc - 1)) * P.n;  // padding rows repeat
          ownpos[it] = (P.owner && kr < P.nc) ? (int)__ldg(P.own_pos + cell * kNCP + kr) : -1;
        }
      }
      if (!tc::mbar_wait(&bempty[s], (uint32_t)((jg / nS) & 1) ^ 1u)) return false;
      const int c0 = tg * BN;
      uint8_t* slot = sB + (size_t)s * kSlotBytes;
#pragma unroll
      for (int it = 0; it < kIt; ++it) {
        const int e = it * 256 + gt;
        const int kr = e / CPR, ch = e % CPR, col = c0 + 4 * ch;
        const bool in = col < P.n;
        const uint32_t off = (uint32_t)(ch >> 3) * kChunkBytes + (uint32_t)kr * 128 + (uint32_t)(((ch & 7) ^ (kr & 7)) << 4);
        cp_async16(slot + off, P.V + rowoff[it] + (in ? col : 0), in);
        if (ownpos[it] >= 0) {  // owned row: W row into position ownpos of the compact W area
          const int o = ownpos[it];
          const uint32_t woff = (uint32_t)(ch >> 3) * kWChunkBytes + (uint32_t)o * 128 + (uint32_t)(((ch & 7) ^ (o & 7)) << 4);
          cp_async16(slot + kHalf + woff, P.W + rowoff[it] + (in ? col : 0), in);
        }
      }
      for (int e = gt; e < BN / 4; e += 256) {
        const int col = c0 + 4 * e;
        const bool in = col < P.n;
        cp_async16(sL + (size_t)s * BN + 4 * e, P.lam + (in ? col : 0), in);
      }
      cp_async_arrive_noinc(&bfull[s]);
      ++jg;
      if (++tg == P.ntiles) {
        tg = 0;
        gg += G;
      }
      return true;
    };
    bool stop = false;
    for (int a = 0; a < ahead && !stop; ++a)
      if (!gather()) {
        fail();
        stop = true;
      }
    int64_t j = 0;
    for (int64_t g = blockIdx.x; g < p.total_cells && !stop; g += G) {
      const StepPartDev& P = p.part[part_of(p, g)];
      const int64_t cell = g - P.cell_off;
      const bool real = k < P.nc;
      const int o = (real && P.owner) ? (int)__ldg(P.own_pos + cell * kNCP + k) : -1;  // compact W row
      const bool own = o >= 0;
      float al = P.alpha, be = P.beta, om = P.omega;
      if (P.coef) {
        al = (float)__ldg(P.coef);
        be = (float)__ldg(P.coef + 1);
        om = (float)__ldg(P.coef + 2);
      }
      al *= P.sign;
      const float rbe = be / al, rom = om / al;  // owner terms divided by alpha
      for (int t = 0; t < P.ntiles; ++t, ++j) {
        const int s = (int)(j % nS), xb = (int)(j & 1);
        bool ok = !*vabort && tc::mbar_wait(&bfull[s], (uint32_t)((j / nS) & 1));
        if (ok) ok = tc::mbar_wait(&accempty[xb], (uint32_t)((j >> 1) & 1) ^ 1u);
        if (!ok) fail();
        if (!__all_sync(0xffffffffu, ok && !*vabort)) {
          stop = true;
          break;
        }
        tc::tc_fence_after();
        uint8_t* slot = sB + (size_t)s * kSlotBytes;
        const uint8_t* vrow = slot + (size_t)k * 128;
        const uint8_t* wrow = slot + kHalf + (size_t)(own ? o : 0) * 128;
        const float* lam = sL + (size_t)s * BN;
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(xb * BN + h * HB);
        float4 v[HB / 4];
#pragma unroll
        for (int c16 = 0; c16 < HB / 16; ++c16) {
          float tv[16];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int col = h * HB + c16 * 16 + 4 * u;      // column within the tile
            const int c = col >> 5, qd = (col & 31) >> 2;  // 32-column chunk, 16-byte chunk in the row
            // 16-byte chunk qd of staged row k sits at chunk qd ^ (k % 8) (the 128-byte swizzle)
            const uint32_t off = (uint32_t)c * kChunkBytes + (uint32_t)((qd ^ (k & 7)) << 4);
            float4 x = *reinterpret_cast<const float4*>(vrow + off);
            const uint32_t woff = (uint32_t)c * kWChunkBytes + (uint32_t)((qd ^ (o & 7)) << 4);
            if (!real) x = make_float4(0.f, 0.f, 0.f, 0.f);
            v[c16 * 4 + u] = x;
            float4 tq = make_float4(0.f, 0.f, 0.f, 0.f);
            if (own) {
              // (FP32 Lambda: a conversion from FP64 would hold the SM's FP64 pipe ~16 clocks per warp)
              const float4 wv = *reinterpret_cast<const float4*>(wrow + woff);
              const float4 lv = *reinterpret_cast<const float4*>(lam + col);
              tq.x = rbe * x.x + rom * lv.x * wv.x;
              tq.y = rbe * x.y + rom * lv.y * wv.y;
              tq.z = rbe * x.z + rom * lv.z * wv.z;
              tq.w = rbe * x.w + rom * lv.w * wv.w;
            }
            tv[4 * u] = tq.x;
            tv[4 * u + 1] = tq.y;
            tv[4 * u + 2] = tq.z;
            tv[4 * u + 3] = tq.w;
          }
          tc::tmem_st16(taddr + c16 * 16, tv);
        }
        tc::tmem_wait_st();
        // once every converter has read its part of the stage (a bounded wait on a barrier that
        // completes one phase per tile), rewrite the stage as the K-major operand
        tc::mbar_arrive(&cvt_read);
        ok = tc::mbar_wait(&cvt_read, (uint32_t)(j & 1));
        if (!ok) fail();
        if (!__all_sync(0xffffffffu, ok && !*vabort)) {
          stop = true;
          break;
        }
#pragma unroll
        for (int u = 0; u < HB / 4; ++u) {
          const int col = h * HB + 4 * u;
          const float4 x = v[u];
          *reinterpret_cast<float*>(slot + img_off(col, k, BN)) = tf32_rna(x.x);
          *reinterpret_cast<float*>(slot + img_off(col + 1, k, BN)) = tf32_rna(x.y);
          *reinterpret_cast<float*>(slot + img_off(col + 2, k, BN)) = tf32_rna(x.z);
          *reinterpret_cast<float*>(slot + img_off(col + 3, k, BN)) = tf32_rna(x.w);
        }
        fence_proxy_async();  // the generic-proxy writes, before the MMA reads them
        tc::tc_fence_before();
        tc::mbar_arrive(&ifull[s]);
        // the tile `ahead` further on, into the stage of tile j - 1 (free once its MMA is done)
        if (!gather()) {
          fail();
          stop = true;
        }
      }
    }
    // copies still in flight land before the shared memory is released
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else {
    // ---------------- epilogue
    const int q = warp & 3;              // TMEM lane quarter this warp may access
    const int i = q * 32 + lane;         // cell-local node of this thread's accumulator row
    int64_t j = 0;
    bool stop = false;
    for (int64_t g = blockIdx.x; g < p.total_cells && !stop; g += G) {
      const StepPartDev& P = p.part[part_of(p, g)];
      const int64_t cell = g - P.cell_off;
      float al = P.coef ? (float)__ldg(P.coef) : P.alpha;
      al *= P.sign;
      const int64_t row = (i < P.nc) ? (int64_t)__ldg(P.dofs + cell * P.nc + i) * P.n : -1;
      for (int t = 0; t < P.ntiles; ++t, ++j) {
        const int xb = (int)(j & 1);
        const int c0 = t * BN;
        bool ok = !*vabort && tc::mbar_wait(&accfull[xb], (uint32_t)((j >> 1) & 1));
        if (!ok) fail();
        if (!__all_sync(0xffffffffu, ok && !*vabort)) {
          stop = true;
          break;
        }
        tc::tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(xb * BN);
#pragma unroll
        for (int cc = 0; cc < BN; cc += 16) {
          float v[16];
          tc::tmem_ld16(taddr + cc, v);
          if (row >= 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int col = c0 + cc + 4 * u;
              if (col < P.n)
                red_add_v4(P.U + row + col, al * v[4 * u], al * v[4 * u + 1], al * v[4 * u + 2], al * v[4 * u + 3]);
            }
          }
        }
        tc::tc_fence_before();
        tc::mbar_arrive(&accempty[xb]);
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, p.tmem_cols);
  }
}

// Shared-memory plan of a tile width: cell-image buffers and stages (V rows, owned W rows) that fit.
struct Plan {
  int nA, nslots;
  size_t smem;
};

Plan make_plan(int BN) {
  // the deepest ring of stages that fits beside one cell image (the gathers run nslots - 1 tiles
  // ahead); a second image buffer only when it leaves at least three stages
  const size_t stage = (size_t)(BN / 32) * (kChunkBytes + kWChunkBytes) + (size_t)BN * 4;
  const size_t cap = kSmemMax - 1024 - 512;  // alignment slack and the kernel's static shared memory
  for (int nA : {1, 2}) {
    for (int ns = kMaxStages; ns >= (nA == 2 ? 3 : 2); --ns) {
      const size_t need = (size_t)nA * kABytes + (size_t)ns * stage;
      if (need <= cap) return Plan{nA, ns, need + 1024};
    }
  }
  return Plan{0, 0, 0};
}

const uint8_t* scaled_images(cudaStream_t s, FeOp& op, const double* dinv) {
  if (!op.imgADtf.p || !op.imgAD_packed) {
    op.imgADtf.ensure((size_t)kABytes * op.n_cells);
    const int64_t total = op.n_cells * (int64_t)kNCP * kNCP;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
    pack_scaled_kernel<<<blocks, 256, 0, s>>>(op.n_cells, op.nc, op.A64.p, op.dofs.p, dinv, op.imgADtf.p);
    op.imgAD_packed = true;
    RC_LAUNCH();
  }
  return op.imgADtf.p;
}

template <int BN>
void launch(cudaStream_t s, const StepBatch& b, const Plan& pl, unsigned grid) {
  set_smem_limit(reinterpret_cast<const void*>(fe_step_kernel<BN>), kSmemMax - 512);
  fe_step_kernel<BN><<<grid, kThreads, pl.smem, s>>>(b);
  RC_LAUNCH();
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int64_t, int, int>, int> g_tune;

}  // namespace

bool fe_step_supported(const FeOp& op, int n, int precision) {
  return precision == RCHFSI_TF32 && n % 4 == 0 && n >= 4 && op.nc <= kNCP && op.own_pos.p != nullptr &&
         op.own_max <= kWRows;
}

void fe_step_prepare(cudaStream_t s, FeOp& op) {
  scaled_images(s, op, op.Dinv.p);
  if (op.cplx) scaled_images(s, *op.imag, op.Dinv.p);
}

int fe_step_parts(FeOp& op, const float* V, const float* W, float* U, const float* lam, int n, float alpha,
                  float beta, float omega, const double* coef, FeStepPart* out) {
  if (!op.cplx) {
    out[0] = FeStepPart{&op, V, W, U, lam, coef, op.m, n, alpha, beta, omega, 1.f, true};
    return 1;
  }
  // complex operator on the real embedding: rows [0, mc) real parts, [mc, 2 mc) imaginary parts
  //   U_r += alpha (Ar V_r - Ai V_i),   U_i += alpha (Ai V_r + Ar V_i)
  // and the owner terms of each half once (with the Ar part of that half)
  const int64_t mc = op.mc, off = mc * (int64_t)n;
  FeOp& im = *op.imag;
  out[0] = FeStepPart{&op, V, W, U, lam, coef, mc, n, alpha, beta, omega, 1.f, true};
  out[1] = FeStepPart{&im, V + off, W, U, lam, coef, mc, n, alpha, beta, omega, -1.f, false};
  out[2] = FeStepPart{&im, V, W, U + off, lam, coef, mc, n, alpha, beta, omega, 1.f, false};
  out[3] = FeStepPart{&op, V + off, W + off, U + off, lam, coef, mc, n, alpha, beta, omega, 1.f, true};
  return 4;
}

void fe_step_batch(cudaStream_t s, const FeStepPart* parts, int nparts, int BN, int num_sms) {
  RC_CHECK(nparts >= 1 && nparts <= kMaxParts, RCHFSI_ERR_INVALID_ARG, "fused FE step: 1..64 parts per launch");
  RC_CHECK(BN == 32 || BN == 64 || BN == 96, RCHFSI_ERR_INVALID_ARG, "fused FE step: column tile of 32, 64 or 96");
  const Plan pl = make_plan(BN);
  RC_CHECK(pl.nA > 0, RCHFSI_ERR_INVALID_ARG, "fused FE step: no shared-memory plan for this tile");
  StepBatch b{};
  b.nparts = nparts;
  b.nA = pl.nA;
  b.nslots = pl.nslots;
  int64_t off = 0;
  double flops = 0.0, bytes = 0.0;
  for (int q = 0; q < nparts; ++q) {
    const FeStepPart& t = parts[q];
    FeOp& op = *t.op;
    RC_CHECK(op.nc <= kNCP && t.n % 4 == 0 && op.own_pos.p && op.own_max <= kWRows, RCHFSI_ERR_INVALID_ARG,
             "fused FE step: n_c <= 128, n a multiple of 4, owner positions and at most 80 owned dofs per cell");
    StepPartDev& P = b.part[q];
    RC_CHECK(((uintptr_t)t.V & 15) == 0 && ((uintptr_t)t.W & 15) == 0 && ((uintptr_t)t.U & 15) == 0,
             RCHFSI_ERR_INVALID_ARG, "fused FE step: blocks must start on 16-byte boundaries");
    P.dofs = op.dofs.p;
    P.own_pos = op.own_pos.p;
    P.owner = t.owner ? 1 : 0;
    // the scaled images use the D^-1 of the rows the part reads (both halves share it)
    P.img = scaled_images(s, op, op.Dinv.p);
    P.V = t.V;
    P.W = t.W;
    P.U = t.U;
    P.lam = t.lam;
    P.coef = t.coef;
    P.n_cells = op.n_cells;
    P.cell_off = off;
    P.alpha = t.alpha;
    P.beta = t.beta;
    P.omega = t.omega;
    P.sign = t.sign;
    P.nc = op.nc;
    P.n = t.n;
    P.ntiles = (t.n + BN - 1) / BN;
    off += op.n_cells;
    const double nc = op.nc, C = (double)op.n_cells;
    flops += 2.0 * nc * nc * C * t.n;
    // algorithmic bytes: the cell images, and for the owner part of each row half the four block
    // streams (V read, U read and written, W read); a complex operator's cross parts re-read V
    bytes += 4.0 * nc * nc * C + (t.owner ? 16.0 * (double)t.rows * t.n : 0.0);
  }
  b.total_cells = off;
  b.err = parts[0].op->err;
  uint32_t cols = 32;
  while (cols < (uint32_t)(2 * BN)) cols <<= 1;
  b.tmem_cols = cols;
  const unsigned grid = (unsigned)std::min<int64_t>(b.total_cells, (int64_t)num_sms);
  prof::Scope ps(s, RCHFSI_KERNEL_FE_CELL, flops, bytes);
  switch (BN) {
    case 32: launch<32>(s, b, pl, grid); break;
    case 64: launch<64>(s, b, pl, grid); break;
    default: launch<96>(s, b, pl, grid); break;
  }
}

int fe_step_tune(cudaStream_t s, int num_sms, FeOp& op, int n, const float* V, const float* W, const float* lam) {
  const auto key = std::make_tuple(op.nc, (int64_t)op.n_cells, n, op.cplx ? 1 : 0);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  std::vector<int> cand;
  for (int bn : {32, 64, 96})
    if (bn <= std::max(32, (n + 31) / 32 * 32) && make_plan(bn).nA > 0) cand.push_back(bn);
  DevBuf<float> scratch;
  float* out = scratch.ensure((size_t)op.m * n);
  cudaEvent_t e0, e1;
  RC_CUDA(cudaEventCreate(&e0));
  RC_CUDA(cudaEventCreate(&e1));
  int best = cand[0];
  float best_ms = 1e30f;
  for (int bn : cand) {
    FeStepPart parts[4];
    const int np = fe_step_parts(op, V, W, out, lam, n, 1.f, 0.5f, 0.25f, nullptr, parts);
    fe_step_batch(s, parts, np, bn, num_sms);  // warm-up
    RC_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 2; ++r) fe_step_batch(s, parts, np, bn, num_sms);
    RC_CUDA(cudaEventRecord(e1, s));
    RC_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    RC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best = bn;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return best;
}

}  // namespace rchfsi
