// Tensor-core path for the dense pairwise steps (sm_103a), BF16x3 forms: planar complex
// GEMM
//   C[b] = A[b] (m x k) . B[b] (n x k)^T      (complex, 4M or 3M real decomposition)
// with both operands K-major, written through the separable row/column offset maps (the
// TF32 and 3xTF32 forms, complex and real, are in gemm_tf32.cu; the shared pieces in
// tc_common.cuh). The kernels compute 128 x 128 output tiles per SM (256 x 128 per pair of
// SMs in the cta_group::2 forms) with one elected thread issuing tcgen05.mma from
// shared-memory descriptors, operands brought by TMA into a ring of stages (mbarrier
// transaction counts), accumulators in tensor memory:
//   contract_tcb_kernel            BF16x3 form: operands already split into BF16 hi/lo
//                                  planes by their producers, kind::f16, 256-term chunks;
//   contract_tcb2_kernel           BF16x3 on paired SMs (m >= 256, k > 2048): one two-CTA
//                                  cluster per 256 x 128 tile, M = 256 MMAs;
//   contract_tcb2p_kernel          the same, persistent clusters (256 < k <= 2048);
//   contract_tcb3m_kernel          BF16x3 with the 3M complex product;
//   contract_tcb_persistent_kernel BF16x3 for shallow steps (k <= 256): one CTA per SM over
//                                  the tiles, stores of a tile overlapping the next tile;
//   contract_tcb_shallow_kernel    the same for k <= 64 with sixteen epilogue warps.
// The epilogues store each 32 x 32 block in address order (store_block). Every mbarrier
// wait is bounded by wall time; on expiry the CTA records an error code, drains its
// copies, frees its tensor memory and returns.
#include <cstdint>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "mbarrier.cuh"
#include "split_bf16.cuh"
#include "tc_common.cuh"

namespace tn {
namespace {

// Self-test of the bounded wait: one thread waits on an mbarrier that is completed only
// if `arrive` is set. Without the arrival the wait runs out after limit_ns, the kernel
// records code 99 in the error word and returns normally.
__global__ void bounded_wait_selftest_kernel(int arrive, uint64_t limit_ns, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (arrive) mbar_arrive(&bar);
  if (!mbar_wait(&bar, 0, limit_ns)) atomicExch(err, 99);
}

// ---------------------------------------------------------------------------------
// BF16x3 (split-BF16) form, kind::f16 with BF16 operands.
//
// Both operands arrive in the split-BF16 form (split_bf16.cuh), written by the kernels
// that produced them, so this kernel does no conversion: per k-block one TMA box of
// (32 k) x (128 rows) x (4 planes) per operand lands as the tiles
//   [re_hi | im_hi | re_lo | im_lo], 128 rows of 64 bytes each, 64-byte swizzle,
// and [B_re | B_im] of either precision is one 256-row operand. Per 16-deep k-atom:
//   hi:  D_hi(Re|Im) += A_re_h.[B_re_h|B_im_h];  D_hi.Re -= A_im_h.B_im_h;  D_hi.Im += A_im_h.B_re_h
//   lo:  the same three with (A_lo, B_hi) and with (A_hi, B_lo), into D_lo
// (the A_lo.B_lo term, <= 2^-16 relative, is dropped). -A_im uses the instruction's
// negate-A bit. D_lo spans all of k; D_hi is folded into round-to-nearest register
// totals every CK k-blocks (256 terms) as in the 3xTF32 kernel, and the lo MMAs of a
// chunk's first k-block are issued before the wait for that fold, so the fold overlaps
// tensor-core work. Warps: 0 TMA, 1 MMA + TMEM, 2-9 fold / epilogue (320 threads).
struct CB {
  static constexpr int BK = 32, ROWB = 64, CK = 8;
  static constexpr int PLANE = BM * ROWB;                   // 8 KiB: one plane of one operand
  static constexpr int OFF_B = 4 * PLANE;
  static constexpr int STAGE = 8 * PLANE;                   // 64 KiB: A and B, 4 planes each
  static constexpr int STAGES = 3;
  static constexpr int THREADS = 320;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 1024;
  static constexpr uint32_t COLS = 512;  // hi: re @0, im @128; lo: re @256, im @384
};
static_assert(BM == BN, "the split-BF16 tiles share one plane size");

// Instruction descriptor, kind::f16: D f32, A/B bf16, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}
constexpr uint32_t kNegateA = 1u << 13;
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// SCALED: exponent scaling (a.recs): the epilogue applies the operands' scales and records
// the result's exponent (tc_scale); every scaled BF16x3 4M step runs this kernel.
template <bool SCALED>
__global__ void __launch_bounds__(CB::THREADS, 1)
    contract_tcb_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        StepArgs a, int64_t t_first, int* err) {
  constexpr int STAGES = CB::STAGES, BK = CB::BK, ROWB = CB::ROWB, CK = CB::CK;
  constexpr int PLANE = CB::PLANE, STAGE = CB::STAGE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
  uint64_t* full = bars;                 // [STAGES]
  uint64_t* empty = bars + STAGES;       // [STAGES]
  uint64_t* acc_full = bars + 2 * STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles_m = (a.m + BM - 1) / BM, tiles_n = (a.n + BN - 1) / BN;
  const int64_t t = t_first + blockIdx.x;  // this launch's tiles start at t_first
  const int64_t per_group = GROUP_M * tiles_n;
  const int64_t first_m = (t / per_group) * GROUP_M;
  const int64_t gm = tiles_m - first_m < GROUP_M ? tiles_m - first_m : GROUP_M;
  const int64_t tm = first_m + (t % per_group) % gm, tn = (t % per_group) / gm;
  const int m0 = static_cast<int>(tm * BM), n0 = static_cast<int>(tn * BN);
  const int b = blockIdx.y;
  const int num_kb = static_cast<int>((a.k + BK - 1) / BK);
  const int n_chunks = (num_kb + CK - 1) / CK;
  const int pa = a.a_bstride ? 4 * b : 0, pb = a.b_bstride ? 4 * b : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(CB::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < num_kb; ++kb) {
        const int s = kb % STAGES;
        if (!mbar_wait(&empty[s], ((kb / STAGES) & 1) ^ 1)) {
          atomicExch(err, 21);
          break;
        }
        mbar_expect_tx(&full[s], STAGE);
        uint8_t* st = smem + s * STAGE;
        const int k0 = kb * BK;
        tma_load_3d(st, &tmA, &full[s], k0, m0, pa);
        tma_load_3d(st + CB::OFF_B, &tmB, &full[s], k0, n0, pb);
        issued = kb + 1;
      }
      for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
        if (!mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1)) atomicExch(err, 22);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t id_w = idesc_bf16(BM, 2 * BN);   // A . [B_re | B_im] -> (Re | Im)
      constexpr uint32_t id_n = idesc_bf16(BM, BN);
      const uint32_t d_hi = tmem, d_lo = tmem + 256;
      bool ok = true;
      for (int c = 0; c < n_chunks && ok; ++c) {
        const int kb_end = min(num_kb, (c + 1) * CK);
        for (int kb = c * CK; kb < kb_end; ++kb) {
          const int s = kb % STAGES;
          if (!mbar_wait(&full[s], (kb / STAGES) & 1)) {
            atomicExch(err, 23);
            ok = false;
            break;
          }
          fence_after();
          const uint32_t sa = su32(smem + s * STAGE), sb = sa + CB::OFF_B;
#pragma unroll
          for (int j = 0; j < BK / 16; ++j) {
            const uint32_t o = j * 32;
            const uint64_t ar_l = smem_desc<ROWB>(sa + 2 * PLANE + o), ai_l = smem_desc<ROWB>(sa + 3 * PLANE + o);
            const uint64_t ar_h = smem_desc<ROWB>(sa + o), ai_h = smem_desc<ROWB>(sa + PLANE + o);
            const uint64_t b_h = smem_desc<ROWB>(sb + o), bi_h = smem_desc<ROWB>(sb + PLANE + o);
            const uint64_t b_l = smem_desc<ROWB>(sb + 2 * PLANE + o), bi_l = smem_desc<ROWB>(sb + 3 * PLANE + o);
            const uint32_t first = (kb > 0 || j > 0) ? 1u : 0u;
            mma_bf16(d_lo, ar_l, b_h, id_w, first);              // A_re_lo . [B_re_h | B_im_h]
            mma_bf16(d_lo, ai_l, bi_h, id_n | kNegateA, 1u);     // Re -= A_im_lo . B_im_h
            mma_bf16(d_lo + 128, ai_l, b_h, id_n, 1u);           // Im += A_im_lo . B_re_h
            mma_bf16(d_lo, ar_h, b_l, id_w, 1u);                 // A_re_h . [B_re_lo | B_im_lo]
            mma_bf16(d_lo, ai_h, bi_l, id_n | kNegateA, 1u);
            mma_bf16(d_lo + 128, ai_h, b_l, id_n, 1u);
          }
          if (kb == c * CK) {
            // the chunk accumulator must have been folded before the hi MMAs reuse it
            if (!mbar_wait(acc_empty, (c & 1) ^ 1)) {
              atomicExch(err, 24);
              ok = false;
              mma_commit(&empty[s]);
              break;
            }
            fence_after();
          }
#pragma unroll
          for (int j = 0; j < BK / 16; ++j) {
            const uint32_t o = j * 32;
            const uint64_t ar_h = smem_desc<ROWB>(sa + o), ai_h = smem_desc<ROWB>(sa + PLANE + o);
            const uint64_t b_h = smem_desc<ROWB>(sb + o), bi_h = smem_desc<ROWB>(sb + PLANE + o);
            const uint32_t acc = (kb > c * CK || j > 0) ? 1u : 0u;
            mma_bf16(d_hi, ar_h, b_h, id_w, acc);
            mma_bf16(d_hi, ai_h, bi_h, id_n | kNegateA, 1u);
            mma_bf16(d_hi + 128, ai_h, b_h, id_n, 1u);
          }
          mma_commit(&empty[s]);
        }
        mma_commit(acc_full);  // also on error, so the fold sees issued MMAs retire
      }
    }
  } else {
    const int q = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
    float run_re[64], run_im[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) run_re[i] = run_im[i] = 0.f;
    bool ok = true;
    for (int c = 0; c < n_chunks && ok; ++c) {
      if (!mbar_wait(acc_full, c & 1)) {
        atomicExch(err, 25);
        ok = false;
        break;
      }
      fence_after();
      float v[32];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const uint32_t col = lane_base + half * 64 + p * 32;
        tmem_ld32(tmem + col, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) run_re[p * 32 + i] += v[i];
        tmem_ld32(tmem + 128 + col, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) run_im[p * 32 + i] += v[i];
        if (c == n_chunks - 1) {  // after the last chunk: the cross terms too
          tmem_ld32(tmem + 256 + col, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) run_re[p * 32 + i] += v[i];
          tmem_ld32(tmem + 384 + col, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) run_im[p * 32 + i] += v[i];
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
    }
    // epilogue: thread = TMEM lane (row); this warp's 64 columns
    const int row = q * 32 + lane;
    const int64_t m = static_cast<int64_t>(m0) + row;
    const bool row_ok = ok && m < a.m;
    const int64_t ro = row_ok ? map_offset(a.rows, m) : 0;
    float* C = a.C + static_cast<int64_t>(b) * a.c_bstride;
    const int split = a.c_split;
    // The stage buffers are free here: the last fold waited for the final MMA, which
    // consumed every staged tile; no TMA load is outstanding.
    // this warp's 32 x 64 results, Re then Im, rows of 65 floats: the registers are free
    // before the stores begin
    float* tr = reinterpret_cast<float*>(smem) + (warp - 2) * 2 * 32 * 65;
    if constexpr (SCALED) {
      // (rows past m and columns past n hold zeros: their operands were zero-filled by TMA)
      const TcScale sc = tc_scale(a, b);
      int lmax = -127;
#pragma unroll
      for (int j = 0; j < 64; ++j) {
        run_re[j] = run_re[j] * sc.sa * sc.sb;
        run_im[j] = run_im[j] * sc.sa * sc.sb;
        lmax = max(lmax, exp_of(fmaxf(fabsf(run_re[j]), fabsf(run_im[j]))));
      }
      tc_scale_finish(a, b, lmax, t == 0 && threadIdx.x == 64);
    }
#pragma unroll
    for (int j = 0; j < 64; ++j) {
      tr[lane * 65 + j] = run_re[j];
      tr[32 * 65 + lane * 65 + j] = run_im[j];
    }
    __syncwarp();
    for (int cb = 0; cb < 2; ++cb) {
      const int64_t n = static_cast<int64_t>(n0) + half * 64 + cb * 32 + lane;
      const bool col_ok = ok && n < a.n;
      store_block(C, a.c_plane, split, tr + cb * 32, 65, 32 * 65, ro, col_ok ? map_offset(a.cols, n) : 0, row_ok,
                  col_ok, lane);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CB::COLS));
  }
}

// ---------------------------------------------------------------------------------
// BF16x3 4M on paired SMs (tcgen05 cta_group::2). A cluster of two CTAs computes one
// 256 x 128 output tile: CTA r (rank in the pair) loads A rows m0 + 128 r .. + 127 and B
// rows n0 + 64 r .. + 63 (all four split planes, 32 deep per k-block) into its own shared
// memory by TMA, and CTA 0 issues M = 256, N = 128 MMAs that read A and B from both. Per
// SM and 16-deep atom TMA writes 24 KiB instead of 32 KiB and each SM fetches half of its B
// panel, so the L2 and DRAM operand traffic per output halves; the data moved per flop, and
// with it the power drawn, drops, which under the power limit buys clock. The accumulation is that of
// contract_tcb_kernel term for term (hi.hi chunk accumulator folded into round-to-nearest
// registers every 256 terms, the cross terms over all of k), with the four real products of
// each complex product as separate N = 128 MMAs in the same order per accumulator, so each
// output row gets the same bits as there. Each CTA's tensor memory holds its 128 rows.
// Protocol: CTA 1's loads complete on its own barriers; one of its threads forwards each
// completed stage to CTA 0 (remote mbarrier arrive); CTA 0's commits arrive on both CTAs'
// barriers (multicast); the fold warps of both CTAs release the accumulators to CTA 0.
// Every wait is bounded; after an expired wait the CTA records a code (51-59), stops
// issuing and reaches the common teardown (cluster barriers, the pair's collective TMEM
// release), which every thread of both CTAs always executes. A pair started after an
// error skips its work (the leader's reading of the error word is shared with its peer).
struct CB2 {
  static constexpr int BK = 32, ROWB = 64, CK = 8;
  static constexpr int PLANE_A = 128 * ROWB;               // 8 KiB: one plane of this CTA's A rows
  static constexpr int PLANE_B = 64 * ROWB;                // 4 KiB: one plane of this CTA's B rows
  static constexpr int OFF_B = 4 * PLANE_A;
  static constexpr int STAGE = 4 * PLANE_A + 4 * PLANE_B;  // 48 KiB
  static constexpr int STAGES = 4;
  static constexpr int THREADS = 320;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 1024;
  static constexpr uint32_t COLS = 512;                    // hi: re @0, im @128; lo: re @256, im @384
  static constexpr int GROUP = 8;                          // raster: pair tiles grouped along M
};

__device__ __forceinline__ void mma_bf16_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// arrive on `bar` of both CTAs of the pair when the MMAs issued so far complete
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          su32(bar)),
      "h"(static_cast<uint16_t>(3))
      : "memory");
}
// arrive on the barrier at the same offset in CTA 0 of the cluster
__device__ __forceinline__ void mbar_arrive_leader(uint64_t* bar) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(su32(bar)), "r"(0));
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}
__device__ __forceinline__ uint32_t ld_leader_u32(const uint32_t* p) {
  uint32_t remote, v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(su32(p)), "r"(0));
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(remote) : "memory");
  return v;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(CB2::THREADS, 1)
    contract_tcb2_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                         StepArgs a, int64_t t_first, int* err) {
  constexpr int STAGES = CB2::STAGES, BK = CB2::BK, ROWB = CB2::ROWB, CK = CB2::CK;
  constexpr int PA = CB2::PLANE_A, PB = CB2::PLANE_B, STAGE = CB2::STAGE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
  uint64_t* full = bars;                  // [STAGES] this CTA's loads landed
  uint64_t* ready = bars + STAGES;        // [STAGES] (CTA 0) CTA 1's loads landed
  uint64_t* empty = bars + 2 * STAGES;    // [STAGES] the stage's MMAs completed
  uint64_t* acc_full = bars + 3 * STAGES;
  uint64_t* acc_empty = acc_full + 1;     // (CTA 0) both CTAs' fold warps read the chunk
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);
  uint32_t* skip_slot = tmem_slot + 1;

  uint32_t rank;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles_m = (a.m + 2 * BM - 1) / (2 * BM), tiles_n = (a.n + BN - 1) / BN;
  const int64_t t = t_first + (blockIdx.x >> 1);  // this launch's tiles start at t_first
  const int64_t per_group = CB2::GROUP * tiles_n;
  const int64_t first_m = (t / per_group) * CB2::GROUP;
  const int64_t gm = tiles_m - first_m < CB2::GROUP ? tiles_m - first_m : CB2::GROUP;
  const int64_t tm = first_m + (t % per_group) % gm, tn = (t % per_group) / gm;
  const int m0 = static_cast<int>(tm * 2 * BM), n0 = static_cast<int>(tn * BN);
  const int b = blockIdx.y;
  const int num_kb = static_cast<int>((a.k + BK - 1) / BK);
  const int n_chunks = (num_kb + CK - 1) / CK;
  const int pa = a.a_bstride ? 4 * b : 0, pb = a.b_bstride ? 4 * b : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 16);
    *skip_slot = *reinterpret_cast<volatile int*>(err) != 0 ? 1u : 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(CB2::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  cluster_sync_all();  // both CTAs' barriers initialised and the pair's TMEM allocated
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const bool skip = ld_leader_u32(skip_slot) != 0;  // one decision for the pair

  if (skip) {
    // an earlier CTA gave up a wait: no work, only the common teardown
  } else if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < num_kb; ++kb) {
        const int s = kb % STAGES;
        if (!mbar_wait(&empty[s], ((kb / STAGES) & 1) ^ 1)) {
          atomicExch(err, 51);
          break;
        }
        mbar_expect_tx(&full[s], STAGE);
        uint8_t* st = smem + s * STAGE;
        const int k0 = kb * BK;
        tma_load_3d(st, &tmA, &full[s], k0, m0 + 128 * static_cast<int>(rank), pa);
        tma_load_3d(st + CB2::OFF_B, &tmB, &full[s], k0, n0 + 64 * static_cast<int>(rank), pb);
        issued = kb + 1;
      }
      // before exit: every load landed, and every commit of CTA 0 for them arrived here
      for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb) {
        if (!mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1)) atomicExch(err, 52);
        if (!mbar_wait(&empty[kb % STAGES], (kb / STAGES) & 1)) atomicExch(err, 53);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 1) {
      // forward each landed stage to CTA 0, in order
      for (int kb = 0; kb < num_kb; ++kb) {
        if (!mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1)) {
          atomicExch(err, 54);
          break;
        }
        mbar_arrive_leader(&ready[kb % STAGES]);
      }
    } else if (lane == 0) {
      constexpr uint32_t id = idesc_bf16(2 * BM, BN);
      const uint32_t d_hi = tmem, d_lo = tmem + 256;
      // the cross terms (into D_lo) of one k-block: 8 MMAs per 16-deep atom
      auto cross = [&](uint32_t sa, uint32_t sb, bool first_kb) {
#pragma unroll
        for (int j = 0; j < BK / 16; ++j) {
          const uint32_t o = j * 32;
          const uint64_t ar_h = smem_desc<ROWB>(sa + o), ai_h = smem_desc<ROWB>(sa + PA + o);
          const uint64_t ar_l = smem_desc<ROWB>(sa + 2 * PA + o), ai_l = smem_desc<ROWB>(sa + 3 * PA + o);
          const uint64_t br_h = smem_desc<ROWB>(sb + o), bi_h = smem_desc<ROWB>(sb + PB + o);
          const uint64_t br_l = smem_desc<ROWB>(sb + 2 * PB + o), bi_l = smem_desc<ROWB>(sb + 3 * PB + o);
          const uint32_t first = (!first_kb || j > 0) ? 1u : 0u;
          mma_bf16_pair(d_lo, ar_l, br_h, id, first);           // Re += A_re_lo . B_re_h
          mma_bf16_pair(d_lo, ai_l, bi_h, id | kNegateA, 1u);   // Re -= A_im_lo . B_im_h
          mma_bf16_pair(d_lo + 128, ar_l, bi_h, id, first);     // Im += A_re_lo . B_im_h
          mma_bf16_pair(d_lo + 128, ai_l, br_h, id, 1u);        // Im += A_im_lo . B_re_h
          mma_bf16_pair(d_lo, ar_h, br_l, id, 1u);
          mma_bf16_pair(d_lo, ai_h, bi_l, id | kNegateA, 1u);
          mma_bf16_pair(d_lo + 128, ar_h, bi_l, id, 1u);
          mma_bf16_pair(d_lo + 128, ai_h, br_l, id, 1u);
        }
      };
      // hi . hi of one k-block into the chunk accumulator D_hi: 4 MMAs per atom
      auto hihi = [&](uint32_t sa, uint32_t sb, bool first_kb) {
#pragma unroll
        for (int j = 0; j < BK / 16; ++j) {
          const uint32_t o = j * 32;
          const uint64_t ar_h = smem_desc<ROWB>(sa + o), ai_h = smem_desc<ROWB>(sa + PA + o);
          const uint64_t br_h = smem_desc<ROWB>(sb + o), bi_h = smem_desc<ROWB>(sb + PB + o);
          const uint32_t acc = (!first_kb || j > 0) ? 1u : 0u;
          mma_bf16_pair(d_hi, ar_h, br_h, id, acc);
          mma_bf16_pair(d_hi, ai_h, bi_h, id | kNegateA, 1u);
          mma_bf16_pair(d_hi + 128, ar_h, bi_h, id, acc);
          mma_bf16_pair(d_hi + 128, ai_h, br_h, id, 1u);
        }
      };
      auto stage_a = [&](int kb) { return su32(smem + (kb % STAGES) * STAGE); };
      auto landed = [&](int kb) {
        return mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1) && mbar_wait(&ready[kb % STAGES], (kb / STAGES) & 1);
      };
      // Per chunk: the cross terms of its first LEAD k-blocks are issued before the wait for
      // the previous chunk's fold (which both CTAs' warps must report, one of them across
      // the pair), so the fold and its remote release overlap tensor work; then the hi.hi
      // MMAs of those k-blocks, and the rest of the chunk k-block by k-block. Each
      // accumulator receives its MMAs in k order either way.
      constexpr int LEAD = 2;
      bool ok = true;
      for (int c = 0; c < n_chunks && ok; ++c) {
        const int kb0 = c * CK, kb_end = min(num_kb, (c + 1) * CK);
        const int lead_end = min(kb_end, kb0 + LEAD);
        for (int kb = kb0; kb < lead_end && ok; ++kb) {
          if (!landed(kb)) {
            atomicExch(err, 55);
            ok = false;
            break;
          }
          fence_after();
          cross(stage_a(kb), stage_a(kb) + CB2::OFF_B, kb == 0);
        }
        if (ok && !mbar_wait(acc_empty, (c & 1) ^ 1)) {  // the chunk accumulator is free
          atomicExch(err, 56);
          ok = false;
        }
        if (!ok) {
          mma_commit_pair(acc_full);  // let the fold see the issued MMAs retire
          break;
        }
        fence_after();
        for (int kb = kb0; kb < lead_end; ++kb) {
          hihi(stage_a(kb), stage_a(kb) + CB2::OFF_B, kb == kb0);
          mma_commit_pair(&empty[kb % STAGES]);
        }
        for (int kb = lead_end; kb < kb_end; ++kb) {
          if (!landed(kb)) {
            atomicExch(err, 55);
            ok = false;
            break;
          }
          fence_after();
          cross(stage_a(kb), stage_a(kb) + CB2::OFF_B, false);
          hihi(stage_a(kb), stage_a(kb) + CB2::OFF_B, false);
          mma_commit_pair(&empty[kb % STAGES]);
        }
        mma_commit_pair(acc_full);  // also on error, so the fold sees issued MMAs retire
      }
    }
  } else {
    const int q = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
    float run_re[64], run_im[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) run_re[i] = run_im[i] = 0.f;
    bool ok = true;
    for (int c = 0; c < n_chunks && ok; ++c) {
      if (!mbar_wait(acc_full, c & 1)) {
        atomicExch(err, 57);
        ok = false;
        break;
      }
      fence_after();
      float v[32];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const uint32_t col = lane_base + half * 64 + p * 32;
        tmem_ld32(tmem + col, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) run_re[p * 32 + i] += v[i];
        tmem_ld32(tmem + 128 + col, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) run_im[p * 32 + i] += v[i];
        if (c == n_chunks - 1) {
          tmem_ld32(tmem + 256 + col, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) run_re[p * 32 + i] += v[i];
          tmem_ld32(tmem + 384 + col, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) run_im[p * 32 + i] += v[i];
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) {
        if (rank == 0) mbar_arrive(acc_empty);
        else mbar_arrive_leader(acc_empty);
      }
    }
    // epilogue: thread = TMEM lane = row m0 + 128 rank + 32 q + lane; this warp's 64 columns
    const int row = q * 32 + lane;
    const int64_t m = static_cast<int64_t>(m0) + 128 * static_cast<int64_t>(rank) + row;
    const bool row_ok = ok && m < a.m;
    const int64_t ro = row_ok ? map_offset(a.rows, m) : 0;
    float* C = a.C + static_cast<int64_t>(b) * a.c_bstride;
    const int split = a.c_split;
    // the stage buffers are free: the last fold waited for the final MMA, which read every
    // staged tile of both CTAs (the producer's tail waits keep its copies from landing later)
    float* tr = reinterpret_cast<float*>(smem) + (warp - 2) * 2 * 32 * 65;
    if (ok) {
#pragma unroll
      for (int j = 0; j < 64; ++j) {
        tr[lane * 65 + j] = run_re[j];
        tr[32 * 65 + lane * 65 + j] = run_im[j];
      }
    }
    __syncwarp();
    if (ok) {
      for (int cb = 0; cb < 2; ++cb) {
        const int64_t n = static_cast<int64_t>(n0) + half * 64 + cb * 32 + lane;
        const bool col_ok = n < a.n;
        store_block(C, a.c_plane, split, tr + cb * 32, 65, 32 * 65, ro, col_ok ? map_offset(a.cols, n) : 0, row_ok,
                    col_ok, lane);
      }
    }
  }
  // common teardown: every thread of both CTAs
  fence_before();
  __syncthreads();
  cluster_sync_all();  // both CTAs done with TMEM and with each other's barriers
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CB2::COLS));
  __syncthreads();
  cluster_sync_all();
}

// ---------------------------------------------------------------------------------
// The paired-SM BF16x3 kernel in persistent form: each cluster of two CTAs walks the
// (batch entry, 256 x 128 tile) items c, c + G, ... (G clusters, as many as are resident).
// The k-block ring runs on across items, and after the last fold of an item the fold warps
// release the accumulators before storing the item from registers (through their own
// shared-memory blocks, not the ring), so the next item's MMAs overlap the epilogue and no
// CTA is started or torn down per tile: what a one-tile-per-cluster launch pays per tile
// (TMEM allocation, pipeline fill, epilogue) is paid once. The arithmetic, the roles and the
// protocol are those of contract_tcb2_kernel; barrier phases count k-blocks and chunks over
// all items of the cluster. A new item's cross-term MMAs (which restart D_lo) wait for the
// previous item's last fold.
// Paired-SM steps with k up to this run the persistent kernel; deeper ones one cluster per
// tile. Measured on the 14- and 13-cycle circuits: at k = 512 and 1024 the persistent form
// is 1.5x and 1.15x faster (no per-tile start-up and epilogue); at k = 4096 the two are
// within 1.5 % (the per-tile form ahead), at k >= 16384 the per-tile form is 4-8 % faster
// (four ring stages instead of three, the per-tile cost being small there).
constexpr int64_t kPairsPersistentMaxK = 2048;
// steps with k <= 64 run contract_tcb_shallow_kernel
constexpr bool kShallowKernel = true;
struct CB2P {
  static constexpr int STAGES = 3;
  // per fold warp: Re and Im of one 32 x 32 block, then the fold warps' block orders
  static constexpr int EPI = 8 * 2 * 32 * 33 * 4 + 8 * 128;
  static constexpr int SMEM = STAGES * CB2::STAGE + EPI + 1024 + 1024;
};
static_assert(CB2P::SMEM <= 232448, "shared memory per CTA");

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(CB2::THREADS, 1)
    contract_tcb2p_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                          StepArgs a, int32_t nb, int* err) {
  constexpr int STAGES = CB2P::STAGES, BK = CB2::BK, ROWB = CB2::ROWB, CK = CB2::CK;
  constexpr int PA = CB2::PLANE_A, PB = CB2::PLANE_B, STAGE = CB2::STAGE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* epi = reinterpret_cast<float*>(smem + STAGES * STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE + CB2P::EPI);
  uint64_t* full = bars;                  // [STAGES] this CTA's loads landed
  uint64_t* ready = bars + STAGES;        // [STAGES] (CTA 0) CTA 1's loads landed
  uint64_t* empty = bars + 2 * STAGES;    // [STAGES] the stage's MMAs completed
  uint64_t* acc_full = bars + 3 * STAGES;
  uint64_t* acc_empty = acc_full + 1;     // (CTA 0) both CTAs' fold warps read the chunk
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);
  uint32_t* skip_slot = tmem_slot + 1;

  uint32_t rank;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles_m = (a.m + 2 * BM - 1) / (2 * BM), tiles_n = (a.n + BN - 1) / BN;
  const int64_t tiles = tiles_m * tiles_n, total = tiles * nb;
  const int64_t cluster = blockIdx.x >> 1, n_clusters = gridDim.x >> 1;
  const int num_kb = static_cast<int>((a.k + BK - 1) / BK);
  const int n_chunks = (num_kb + CK - 1) / CK;
  // item w -> batch entry and the tile's first row and column (grouped raster per entry)
  auto item = [&](int64_t w, int& b, int& m0, int& n0) {
    const int64_t t = w % tiles;
    const int64_t per_group = CB2::GROUP * tiles_n;
    const int64_t first_m = (t / per_group) * CB2::GROUP;
    const int64_t gm = tiles_m - first_m < CB2::GROUP ? tiles_m - first_m : CB2::GROUP;
    const int64_t tm = first_m + (t % per_group) % gm, tn = (t % per_group) / gm;
    b = static_cast<int>(w / tiles);
    m0 = static_cast<int>(tm * 2 * BM);
    n0 = static_cast<int>(tn * BN);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 16);
    *skip_slot = *reinterpret_cast<volatile int*>(err) != 0 ? 1u : 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(CB2::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  cluster_sync_all();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const bool skip = ld_leader_u32(skip_slot) != 0;

  if (skip) {
    // an earlier CTA gave up a wait: no work, only the common teardown
  } else if (warp == 0) {
    if (lane == 0) {
      int64_t g = 0;  // k-blocks issued by this CTA over all its items
      bool ok = true;
      for (int64_t w = cluster; w < total && ok; w += n_clusters) {
        int b, m0, n0;
        item(w, b, m0, n0);
        const int pa = a.a_bstride ? 4 * b : 0, pb = a.b_bstride ? 4 * b : 0;
        for (int kb = 0; kb < num_kb; ++kb, ++g) {
          const int s = static_cast<int>(g % STAGES);
          if (!mbar_wait(&empty[s], static_cast<uint32_t>((g / STAGES) & 1) ^ 1)) {
            atomicExch(err, 51);
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], STAGE);
          uint8_t* st = smem + s * STAGE;
          tma_load_3d(st, &tmA, &full[s], kb * BK, m0 + 128 * static_cast<int>(rank), pa);
          tma_load_3d(st + CB2::OFF_B, &tmB, &full[s], kb * BK, n0 + 64 * static_cast<int>(rank), pb);
        }
      }
      // before exit: every load landed, and every commit of CTA 0 for them arrived here
      for (int64_t j = g > STAGES ? g - STAGES : 0; j < g; ++j) {
        if (!mbar_wait(&full[j % STAGES], static_cast<uint32_t>((j / STAGES) & 1))) atomicExch(err, 52);
        if (!mbar_wait(&empty[j % STAGES], static_cast<uint32_t>((j / STAGES) & 1))) atomicExch(err, 53);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 1) {
      // forward each landed stage to CTA 0, in order
      const int64_t mine = total > cluster ? (total - cluster + n_clusters - 1) / n_clusters : 0;
      const int64_t blocks = mine * num_kb;
      for (int64_t g = 0; g < blocks; ++g) {
        if (!mbar_wait(&full[g % STAGES], static_cast<uint32_t>((g / STAGES) & 1))) {
          atomicExch(err, 54);
          break;
        }
        mbar_arrive_leader(&ready[g % STAGES]);
      }
    } else if (lane == 0) {
      constexpr uint32_t id = idesc_bf16(2 * BM, BN);
      const uint32_t d_hi = tmem, d_lo = tmem + 256;
      auto cross = [&](uint32_t sa, uint32_t sb, bool first_kb) {
#pragma unroll
        for (int j = 0; j < BK / 16; ++j) {
          const uint32_t o = j * 32;
          const uint64_t ar_h = smem_desc<ROWB>(sa + o), ai_h = smem_desc<ROWB>(sa + PA + o);
          const uint64_t ar_l = smem_desc<ROWB>(sa + 2 * PA + o), ai_l = smem_desc<ROWB>(sa + 3 * PA + o);
          const uint64_t br_h = smem_desc<ROWB>(sb + o), bi_h = smem_desc<ROWB>(sb + PB + o);
          const uint64_t br_l = smem_desc<ROWB>(sb + 2 * PB + o), bi_l = smem_desc<ROWB>(sb + 3 * PB + o);
          const uint32_t first = (!first_kb || j > 0) ? 1u : 0u;
          mma_bf16_pair(d_lo, ar_l, br_h, id, first);
          mma_bf16_pair(d_lo, ai_l, bi_h, id | kNegateA, 1u);
          mma_bf16_pair(d_lo + 128, ar_l, bi_h, id, first);
          mma_bf16_pair(d_lo + 128, ai_l, br_h, id, 1u);
          mma_bf16_pair(d_lo, ar_h, br_l, id, 1u);
          mma_bf16_pair(d_lo, ai_h, bi_l, id | kNegateA, 1u);
          mma_bf16_pair(d_lo + 128, ar_h, bi_l, id, 1u);
          mma_bf16_pair(d_lo + 128, ai_h, br_l, id, 1u);
        }
      };
      auto hihi = [&](uint32_t sa, uint32_t sb, bool first_kb) {
#pragma unroll
        for (int j = 0; j < BK / 16; ++j) {
          const uint32_t o = j * 32;
          const uint64_t ar_h = smem_desc<ROWB>(sa + o), ai_h = smem_desc<ROWB>(sa + PA + o);
          const uint64_t br_h = smem_desc<ROWB>(sb + o), bi_h = smem_desc<ROWB>(sb + PB + o);
          const uint32_t acc = (!first_kb || j > 0) ? 1u : 0u;
          mma_bf16_pair(d_hi, ar_h, br_h, id, acc);
          mma_bf16_pair(d_hi, ai_h, bi_h, id | kNegateA, 1u);
          mma_bf16_pair(d_hi + 128, ar_h, bi_h, id, acc);
          mma_bf16_pair(d_hi + 128, ai_h, br_h, id, 1u);
        }
      };
      int64_t g = 0;   // k-blocks consumed over all items
      int64_t G = 0;   // chunks over all items
      auto stage_of = [&](int64_t gg) { return su32(smem + (gg % STAGES) * STAGE); };
      auto landed = [&](int64_t gg) {
        const uint32_t ph = static_cast<uint32_t>((gg / STAGES) & 1);
        return mbar_wait(&full[gg % STAGES], ph) && mbar_wait(&ready[gg % STAGES], ph);
      };
      constexpr int LEAD = 2;
      bool ok = true;
      for (int64_t w = cluster; w < total && ok; w += n_clusters) {
        for (int c = 0; c < n_chunks && ok; ++c, ++G) {
          const int kb0 = c * CK, kb_end = min(num_kb, (c + 1) * CK);
          // a new item restarts D_lo: its cross terms wait for the previous item's last fold
          const int lead_end = c == 0 ? kb0 : min(kb_end, kb0 + LEAD);
          for (int kb = kb0; kb < lead_end && ok; ++kb) {
            if (!landed(g + (kb - kb0))) {
              atomicExch(err, 55);
              ok = false;
              break;
            }
            fence_after();
            cross(stage_of(g + (kb - kb0)), stage_of(g + (kb - kb0)) + CB2::OFF_B, false);
          }
          if (ok && !mbar_wait(acc_empty, static_cast<uint32_t>(G & 1) ^ 1)) {
            atomicExch(err, 56);
            ok = false;
          }
          if (!ok) {
            mma_commit_pair(acc_full);
            break;
          }
          fence_after();
          for (int kb = kb0; kb < lead_end; ++kb) {
            hihi(stage_of(g), stage_of(g) + CB2::OFF_B, kb == kb0);
            mma_commit_pair(&empty[g % STAGES]);
            ++g;
          }
          for (int kb = lead_end; kb < kb_end; ++kb) {
            if (!landed(g)) {
              atomicExch(err, 55);
              ok = false;
              break;
            }
            fence_after();
            cross(stage_of(g), stage_of(g) + CB2::OFF_B, kb == 0);
            hihi(stage_of(g), stage_of(g) + CB2::OFF_B, kb == kb0);
            mma_commit_pair(&empty[g % STAGES]);
            ++g;
          }
          mma_commit_pair(acc_full);  // also on error, so the fold sees issued MMAs retire
        }
      }
    }
  } else {
    const int q = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
    float* tr = epi + (warp - 2) * 2 * 32 * 33;  // this warp's Re and Im transpose blocks
    const int split = a.c_split;
    bool pow2 = a.m >= 32 && a.n >= 32;
    for (int d = 0; d < a.rows.n; ++d) pow2 = pow2 && (a.rows.ext[d] & (a.rows.ext[d] - 1u)) == 0u;
    for (int d = 0; d < a.cols.n; ++d) pow2 = pow2 && (a.cols.ext[d] & (a.cols.ext[d] - 1u)) == 0u;
    // kept in shared memory (the same for every lane), not in registers
    BlockOrder& ord = reinterpret_cast<BlockOrder*>(epi + 8 * 2 * 32 * 33)[warp - 2];
    {
      const BlockOrder o = block_order(pow2 ? map_offset(a.rows, lane) : 0, pow2 ? map_offset(a.cols, lane) : 0,
                                       pow2, lane);
      if (lane == 0) ord = o;
      __syncwarp();
    }
    int64_t G = 0;  // chunks folded over all items
    bool ok = true;
    for (int64_t w = cluster; w < total && ok; w += n_clusters) {
      int b, m0, n0;
      item(w, b, m0, n0);
      float run_re[64], run_im[64];
#pragma unroll
      for (int i = 0; i < 64; ++i) run_re[i] = run_im[i] = 0.f;
      for (int c = 0; c < n_chunks; ++c, ++G) {
        if (!mbar_wait(acc_full, static_cast<uint32_t>(G & 1))) {
          atomicExch(err, 57);
          ok = false;
          break;
        }
        fence_after();
        float v[32];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const uint32_t col = lane_base + half * 64 + p * 32;
          tmem_ld32(tmem + col, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) run_re[p * 32 + i] += v[i];
          tmem_ld32(tmem + 128 + col, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) run_im[p * 32 + i] += v[i];
          if (c == n_chunks - 1) {
            tmem_ld32(tmem + 256 + col, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) run_re[p * 32 + i] += v[i];
            tmem_ld32(tmem + 384 + col, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) run_im[p * 32 + i] += v[i];
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) {
          if (rank == 0) mbar_arrive(acc_empty);
          else mbar_arrive_leader(acc_empty);
        }
      }
      if (!ok) break;
      // epilogue from registers while the next item's MMAs run: thread = row
      // m0 + 128 rank + 32 q + lane; this warp's 64 columns, one 32 x 32 block at a time
      const int64_t m = static_cast<int64_t>(m0) + 128 * static_cast<int64_t>(rank) + q * 32 + lane;
      const bool row_ok = m < a.m;
      const int64_t ro = row_ok ? map_offset(a.rows, m) : 0;
      float* C = a.C + static_cast<int64_t>(b) * a.c_bstride;
#pragma unroll
      for (int cb = 0; cb < 2; ++cb) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          tr[lane * 33 + j] = run_re[cb * 32 + j];
          tr[32 * 33 + lane * 33 + j] = run_im[cb * 32 + j];
        }
        __syncwarp();
        const int64_t n = static_cast<int64_t>(n0) + half * 64 + cb * 32 + lane;
        const bool col_ok = n < a.n;
        const int64_t co = col_ok ? map_offset(a.cols, n) : 0;
        if (ord.ok && __all_sync(0xffffffffu, row_ok && col_ok)) {
          const int64_t base = __shfl_sync(0xffffffffu, ro, 0) + __shfl_sync(0xffffffffu, co, 0);
          store_ordered(C, a.c_plane, split, tr, 33, 32 * 33, base, ord, lane);
        } else {
          store_block(C, a.c_plane, split, tr, 33, 32 * 33, ro, co, row_ok, col_ok, lane);
        }
        __syncwarp();
      }
    }
  }
  // common teardown: every thread of both CTAs
  fence_before();
  __syncthreads();
  cluster_sync_all();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CB2::COLS));
  __syncthreads();
  cluster_sync_all();
}

// ---------------------------------------------------------------------------------
// BF16x3 form with the 3M complex product (Gauss): with s = a_re + a_im and t = b_re + b_im,
//   P1 = a_re.b_re,  P2 = a_im.b_im,  P3 = s.t;   Re = P1 - P2,  Im = P3 - P1 - P2,
// three real products per complex MAC instead of four, each as hi.hi + hi.lo + lo.hi of
// the BF16 halves: 9 MMAs (128 x 128 x 16) per 16-deep k-atom instead of 12. The operands
// arrive in the 3M split form (split_bf16.cuh: [re_h | re_l | im_h | im_l | s_h | s_l], the
// sums written by the producers), so one product's two planes of one operand are one TMA
// box. The ring holds (k-block, product) slots of [A_h | A_l | B_h | B_l] (32 deep, 32 KiB);
// product j accumulates in tensor-memory columns 128 j. The three accumulators are
// folded into round-to-nearest register totals of Re and Im every CK k-blocks (256 terms),
// as in contract_tcb_kernel; the MMAs of the next chunk wait for the fold. Warps: 0 TMA,
// 1 MMA + TMEM, 2-9 fold / epilogue (320 threads).
struct CB3 {
  static constexpr int BK = 32, ROWB = 64, CK = 8;
  static constexpr int PLANE = BM * ROWB;                   // 8 KiB
  static constexpr int OFF_B = 2 * PLANE;
  static constexpr int SLOT = 4 * PLANE;                    // 32 KiB: [A_h | A_l | B_h | B_l]
  static constexpr int SLOTS = 6;                           // two k-blocks of three products
  static constexpr int THREADS = 320;
  static constexpr int SMEM = SLOTS * SLOT + 1024 + 1024;
  static constexpr uint32_t COLS = 512;                     // P1 @0, P2 @128, P3 @256
};
static_assert(CB3::SMEM <= 232448, "shared memory per CTA");
static_assert(8 * 2 * 32 * 65 * 4 <= CB3::SLOTS * CB3::SLOT, "epilogue transposes fit the ring");

// 16 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(CB3::THREADS, 1)
    contract_tcb3m_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                          StepArgs a, int64_t t_first, int* err) {
  constexpr int SLOTS = CB3::SLOTS, BK = CB3::BK, ROWB = CB3::ROWB, CK = CB3::CK;
  constexpr int PLANE = CB3::PLANE, SLOT = CB3::SLOT;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SLOTS * SLOT);
  uint64_t* full = bars;                 // [SLOTS]
  uint64_t* empty = bars + SLOTS;        // [SLOTS]
  uint64_t* acc_full = bars + 2 * SLOTS;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles_m = (a.m + BM - 1) / BM, tiles_n = (a.n + BN - 1) / BN;
  const int64_t t = t_first + blockIdx.x;  // this launch's tiles start at t_first
  const int64_t per_group = GROUP_M * tiles_n;
  const int64_t first_m = (t / per_group) * GROUP_M;
  const int64_t gm = tiles_m - first_m < GROUP_M ? tiles_m - first_m : GROUP_M;
  const int64_t tm = first_m + (t % per_group) % gm, tn = (t % per_group) / gm;
  const int m0 = static_cast<int>(tm * BM), n0 = static_cast<int>(tn * BN);
  const int b = blockIdx.y;
  const int num_kb = static_cast<int>((a.k + BK - 1) / BK);
  const int n_chunks = (num_kb + CK - 1) / CK;
  const int pa = a.a_bstride ? 6 * b : 0, pb = a.b_bstride ? 6 * b : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SLOTS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(CB3::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const int n_items = 3 * num_kb;  // (k-block, product) slots in order

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < n_items; ++it) {
        const int s = it % SLOTS;
        if (!mbar_wait(&empty[s], ((it / SLOTS) & 1) ^ 1)) {
          atomicExch(err, 31);
          break;
        }
        mbar_expect_tx(&full[s], SLOT);
        uint8_t* st = smem + s * SLOT;
        const int k0 = (it / 3) * BK, j = it % 3;
        tma_load_3d(st, &tmA, &full[s], k0, m0, pa + 2 * j);
        tma_load_3d(st + CB3::OFF_B, &tmB, &full[s], k0, n0, pb + 2 * j);
        issued = it + 1;
      }
      for (int it = issued > SLOTS ? issued - SLOTS : 0; it < issued; ++it)
        if (!mbar_wait(&full[it % SLOTS], (it / SLOTS) & 1)) atomicExch(err, 32);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t id_n = idesc_bf16(BM, BN);
      bool ok = true;
      for (int c = 0; c < n_chunks && ok; ++c) {
        const int kb_end = min(num_kb, (c + 1) * CK);
        for (int kb = c * CK; kb < kb_end && ok; ++kb) {
          for (int j = 0; j < 3; ++j) {
            const int it = 3 * kb + j, s = it % SLOTS;
            if (!mbar_wait(&full[s], (it / SLOTS) & 1)) {
              atomicExch(err, 33);
              ok = false;
              break;
            }
            if (kb == c * CK && j == 0) {
              // the accumulators must have been folded before this chunk overwrites them
              if (!mbar_wait(acc_empty, (c & 1) ^ 1)) {
                atomicExch(err, 34);
                ok = false;
                mma_commit(&empty[s]);
                break;
              }
            }
            fence_after();
            const uint32_t sa = su32(smem + s * SLOT), sb = sa + CB3::OFF_B;
            const uint32_t d = tmem + 128 * j;
#pragma unroll
            for (int q = 0; q < BK / 16; ++q) {
              const uint32_t o = q * 32;
              const uint64_t ah = smem_desc<ROWB>(sa + o), al = smem_desc<ROWB>(sa + PLANE + o);
              const uint64_t bh = smem_desc<ROWB>(sb + o), bl = smem_desc<ROWB>(sb + PLANE + o);
              const uint32_t acc = (kb > c * CK || q > 0) ? 1u : 0u;
              mma_bf16(d, ah, bh, id_n, acc);   // hi.hi
              mma_bf16(d, ah, bl, id_n, 1u);    // hi.lo
              mma_bf16(d, al, bh, id_n, 1u);    // lo.hi
            }
            mma_commit(&empty[s]);
          }
        }
        mma_commit(acc_full);  // also on error, so the fold sees issued MMAs retire
      }
    }
  } else {
    const int q = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
    float run_re[64], run_im[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) run_re[i] = run_im[i] = 0.f;
    bool ok = true;
    for (int c = 0; c < n_chunks && ok; ++c) {
      if (!mbar_wait(acc_full, c & 1)) {
        atomicExch(err, 35);
        ok = false;
        break;
      }
      fence_after();
      float v1[16], v2[16];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const uint32_t col = lane_base + half * 64 + p * 16;
        tmem_ld16(tmem + col, v1);
        tmem_ld16(tmem + 128 + col, v2);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          run_re[p * 16 + i] += v1[i] - v2[i];
          v1[i] += v2[i];  // P1 + P2
        }
        tmem_ld16(tmem + 256 + col, v2);
#pragma unroll
        for (int i = 0; i < 16; ++i) run_im[p * 16 + i] += v2[i] - v1[i];
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
    }
    // epilogue: thread = TMEM lane (row); this warp's 64 columns
    const int row = q * 32 + lane;
    const int64_t m = static_cast<int64_t>(m0) + row;
    const bool row_ok = ok && m < a.m;
    const int64_t ro = row_ok ? map_offset(a.rows, m) : 0;
    float* C = a.C + static_cast<int64_t>(b) * a.c_bstride;
    const int split = a.c_split;
    // The ring is free here: the last fold waited for the final MMA, which consumed every
    // staged slot; no TMA load is outstanding.
    float* tr = reinterpret_cast<float*>(smem) + (warp - 2) * 2 * 32 * 65;
#pragma unroll
    for (int j = 0; j < 64; ++j) {
      tr[lane * 65 + j] = run_re[j];
      tr[32 * 65 + lane * 65 + j] = run_im[j];
    }
    __syncwarp();
    for (int cb = 0; cb < 2; ++cb) {
      const int64_t n = static_cast<int64_t>(n0) + half * 64 + cb * 32 + lane;
      const bool col_ok = ok && n < a.n;
      store_block(C, a.c_plane, split, tr + cb * 32, 65, 32 * 65, ro, col_ok ? map_offset(a.cols, n) : 0, row_ok,
                  col_ok, lane);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CB3::COLS));
  }
}

// ---------------------------------------------------------------------------------
// BF16x3, persistent, for shallow steps (k <= 256: at most one fold chunk per tile, so the
// numerics are those of contract_tcb_kernel). Such a step is bound by its output stores,
// not by the tensor core; with one tile per CTA most
// of a CTA's life is set-up, pipeline fill and the epilogue, serialised. Here one CTA per
// SM walks the (batch entry, tile) items with a stride of the grid; the stage ring,
// barrier phases and tensor memory carry over, and the fold warps release the
// accumulators before storing a tile, so the stores of one tile overlap the loads and
// MMAs of the next. (For deep steps the same structure keeps the tensor core busier but,
// measured, draws the clock down under the power cap: those keep one tile per CTA.) Same
// MMA sequence and numerics as contract_tcb_kernel; 2 stages, and a 32 x 33 transpose
// block per fold warp for the epilogue.
struct CBP {
  static constexpr int STAGES = 2;
  // per fold warp: Re and Im of one 32 x 32 block, then the fold warps' block orders
  static constexpr int EPI = 8 * 2 * 32 * 33 * 4 + 8 * 128;
  static constexpr int BARS = 256;
  static constexpr int SMEM = STAGES * CB::STAGE + EPI + BARS + 1024 /*align*/;
  static constexpr int MAX_K = CB::CK * CB::BK;            // used for k <= 256: one fold chunk per tile
};
static_assert(CBP::SMEM <= 232448, "shared memory per CTA");

// Work item w -> batch entry and the output tile's first row and column (the grouped
// raster of contract_tcb_kernel within each batch entry).
struct TileCoord {
  int b, m0, n0;
};
__device__ __forceinline__ TileCoord tile_of(int64_t w, int64_t tiles_m, int64_t tiles_n) {
  const int64_t tiles = tiles_m * tiles_n;
  const int64_t t = w % tiles;
  const int64_t per_group = GROUP_M * tiles_n;
  const int64_t first_m = (t / per_group) * GROUP_M;
  const int64_t gm = tiles_m - first_m < GROUP_M ? tiles_m - first_m : GROUP_M;
  const int64_t tm = first_m + (t % per_group) % gm, tn = (t % per_group) / gm;
  return TileCoord{static_cast<int>(w / tiles), static_cast<int>(tm * BM), static_cast<int>(tn * BN)};
}

__global__ void __launch_bounds__(CB::THREADS, 1)
    contract_tcb_persistent_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                                   StepArgs a, int32_t nb, int* err) {
  constexpr int STAGES = CBP::STAGES, BK = CB::BK, ROWB = CB::ROWB;
  constexpr int PLANE = CB::PLANE, STAGE = CB::STAGE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* epi = reinterpret_cast<float*>(smem + STAGES * STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE + CBP::EPI);
  uint64_t* full = bars;                 // [STAGES]
  uint64_t* empty = bars + STAGES;       // [STAGES]
  uint64_t* acc_full = bars + 2 * STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles_m = (a.m + BM - 1) / BM, tiles_n = (a.n + BN - 1) / BN;
  const int64_t total = tiles_m * tiles_n * nb;
  const int num_kb = static_cast<int>((a.k + BK - 1) / BK);  // <= CK: one fold chunk per tile

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(CB::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int64_t g = 0;  // k-blocks issued by this CTA: stage g % STAGES, phase g / STAGES
      bool ok = true;
      for (int64_t w = blockIdx.x; w < total && ok; w += gridDim.x) {
        const TileCoord tc = tile_of(w, tiles_m, tiles_n);
        const int pa = a.a_bstride ? 4 * tc.b : 0, pb = a.b_bstride ? 4 * tc.b : 0;
        for (int kb = 0; kb < num_kb; ++kb, ++g) {
          const int s = static_cast<int>(g % STAGES);
          if (!mbar_wait(&empty[s], static_cast<uint32_t>((g / STAGES) & 1) ^ 1)) {
            atomicExch(err, 31);
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], STAGE);
          uint8_t* st = smem + s * STAGE;
          tma_load_3d(st, &tmA, &full[s], kb * BK, tc.m0, pa);
          tma_load_3d(st + CB::OFF_B, &tmB, &full[s], kb * BK, tc.n0, pb);
        }
      }
      // every issued load has landed before the CTA can exit
      for (int64_t j = g > STAGES ? g - STAGES : 0; j < g; ++j)
        if (!mbar_wait(&full[j % STAGES], static_cast<uint32_t>((j / STAGES) & 1))) atomicExch(err, 32);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t id_w = idesc_bf16(BM, 2 * BN);
      constexpr uint32_t id_n = idesc_bf16(BM, BN);
      const uint32_t d_hi = tmem, d_lo = tmem + 256;
      int64_t g = 0, q = 0;  // k-blocks consumed, tiles committed
      bool ok = true;
      for (int64_t w = blockIdx.x; w < total && ok; w += gridDim.x, ++q) {
        // the previous tile's accumulators must have been read
        if (!mbar_wait(acc_empty, static_cast<uint32_t>(q & 1) ^ 1)) {
          atomicExch(err, 33);
          break;
        }
        fence_after();
        for (int kb = 0; kb < num_kb; ++kb, ++g) {
          const int s = static_cast<int>(g % STAGES);
          if (!mbar_wait(&full[s], static_cast<uint32_t>((g / STAGES) & 1))) {
            atomicExch(err, 34);
            ok = false;
            break;
          }
          fence_after();
          const uint32_t sa = su32(smem + s * STAGE), sb = sa + CB::OFF_B;
#pragma unroll
          for (int j = 0; j < BK / 16; ++j) {
            const uint32_t o = j * 32;
            const uint64_t ar_l = smem_desc<ROWB>(sa + 2 * PLANE + o), ai_l = smem_desc<ROWB>(sa + 3 * PLANE + o);
            const uint64_t ar_h = smem_desc<ROWB>(sa + o), ai_h = smem_desc<ROWB>(sa + PLANE + o);
            const uint64_t b_h = smem_desc<ROWB>(sb + o), bi_h = smem_desc<ROWB>(sb + PLANE + o);
            const uint64_t b_l = smem_desc<ROWB>(sb + 2 * PLANE + o), bi_l = smem_desc<ROWB>(sb + 3 * PLANE + o);
            const uint32_t acc = (kb > 0 || j > 0) ? 1u : 0u;
            mma_bf16(d_lo, ar_l, b_h, id_w, acc);
            mma_bf16(d_lo, ai_l, bi_h, id_n | kNegateA, 1u);
            mma_bf16(d_lo + 128, ai_l, b_h, id_n, 1u);
            mma_bf16(d_lo, ar_h, b_l, id_w, 1u);
            mma_bf16(d_lo, ai_h, bi_l, id_n | kNegateA, 1u);
            mma_bf16(d_lo + 128, ai_h, b_l, id_n, 1u);
            mma_bf16(d_hi, ar_h, b_h, id_w, acc);
            mma_bf16(d_hi, ai_h, bi_h, id_n | kNegateA, 1u);
            mma_bf16(d_hi + 128, ai_h, b_h, id_n, 1u);
          }
          mma_commit(&empty[s]);
        }
        mma_commit(acc_full);  // also on error, so the fold sees issued MMAs retire
      }
    }
  } else {
    const int q4 = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(q4 * 32) << 16;
    float* tr = epi + (warp - 2) * 2 * 32 * 33;  // this warp's Re and Im transpose blocks
    const int split = a.c_split;
    // When every extent of the offset maps is a power of two, every full 32 x 32 block of
    // the step has the address order of the first one: it is computed once here, and a
    // full block only adds its base offset (the other blocks take store_block's checks).
    bool pow2 = a.m >= 32 && a.n >= 32;
    for (int d = 0; d < a.rows.n; ++d) pow2 = pow2 && (a.rows.ext[d] & (a.rows.ext[d] - 1u)) == 0u;
    for (int d = 0; d < a.cols.n; ++d) pow2 = pow2 && (a.cols.ext[d] & (a.cols.ext[d] - 1u)) == 0u;
    // kept in shared memory (the same for every lane), not in registers
    BlockOrder& ord = reinterpret_cast<BlockOrder*>(epi + 8 * 2 * 32 * 33)[warp - 2];
    {
      const BlockOrder o = block_order(pow2 ? map_offset(a.rows, lane) : 0, pow2 ? map_offset(a.cols, lane) : 0,
                                       pow2, lane);
      if (lane == 0) ord = o;
      __syncwarp();
    }
    int64_t q = 0;  // tiles folded
    for (int64_t w = blockIdx.x; w < total; w += gridDim.x, ++q) {
      const TileCoord tc = tile_of(w, tiles_m, tiles_n);
      if (!mbar_wait(acc_full, static_cast<uint32_t>(q & 1))) {
        atomicExch(err, 35);
        break;
      }
      fence_after();
      float run_re[64], run_im[64], v[32];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const uint32_t col = lane_base + half * 64 + p * 32;
        tmem_ld32(tmem + col, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) run_re[p * 32 + i] = v[i];
        tmem_ld32(tmem + 128 + col, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) run_im[p * 32 + i] = v[i];
        tmem_ld32(tmem + 256 + col, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) run_re[p * 32 + i] += v[i];
        tmem_ld32(tmem + 384 + col, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) run_im[p * 32 + i] += v[i];
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);  // the accumulators are free for the next tile
      // epilogue from registers: thread = TMEM lane (row); this warp's 64 columns
      const int64_t m = static_cast<int64_t>(tc.m0) + q4 * 32 + lane;
      const bool row_ok = m < a.m;
      const int64_t ro = row_ok ? map_offset(a.rows, m) : 0;
      float* C = a.C + static_cast<int64_t>(tc.b) * a.c_bstride;
#pragma unroll
      for (int cb = 0; cb < 2; ++cb) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          tr[lane * 33 + j] = run_re[cb * 32 + j];
          tr[32 * 33 + lane * 33 + j] = run_im[cb * 32 + j];
        }
        __syncwarp();
        const int64_t n = static_cast<int64_t>(tc.n0) + half * 64 + cb * 32 + lane;
        const bool col_ok = n < a.n;
        const int64_t co = col_ok ? map_offset(a.cols, n) : 0;
        if (ord.ok && __all_sync(0xffffffffu, row_ok && col_ok)) {
          const int64_t base = __shfl_sync(0xffffffffu, ro, 0) + __shfl_sync(0xffffffffu, co, 0);
          store_ordered(C, a.c_plane, split, tr, 33, 32 * 33, base, ord, lane);
        } else {
          store_block(C, a.c_plane, split, tr, 33, 32 * 33, ro, co, row_ok, col_ok, lane);
        }
        __syncwarp();
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CB::COLS));
  }
}

// ---------------------------------------------------------------------------------
// Shallow steps (k <= 64, BF16x3 4M): the result tile is stored for every one or two
// k-blocks of MMA work, so the epilogue sets the pace. Persistent like
// contract_tcb_persistent_kernel, but with sixteen fold/epilogue warps (a 32 x 32 block each
// per tile: twice the warps to hide the transpose, split and store latencies) and a single
// ring stage (its 64 KiB pay for the warps' transpose blocks); loading and the MMAs of the
// next tile run while the previous tile is stored. Warps: 0 TMA, 1 MMA + TMEM, 2-17 fold and
// epilogue. Bounded waits as in the other kernels (codes 61-65).
struct CBS {
  static constexpr int EPI_WARPS = 16;
  static constexpr int THREADS = 32 * (2 + EPI_WARPS);
  static constexpr int MAX_K = 2 * CB::BK;                 // two k-blocks per tile at most
  static constexpr int EPI = EPI_WARPS * 2 * 32 * 33 * 4 + EPI_WARPS * 128;
  static constexpr int SMEM = CB::STAGE + EPI + 256 + 1024;
};
static_assert(CBS::SMEM <= 232448, "shared memory per CTA");

__global__ void __launch_bounds__(CBS::THREADS, 1)
    contract_tcb_shallow_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                                StepArgs a, int32_t nb, int* err) {
  constexpr int BK = CB::BK, ROWB = CB::ROWB, PLANE = CB::PLANE, STAGE = CB::STAGE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* epi = reinterpret_cast<float*>(smem + STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGE + CBS::EPI);
  uint64_t* full = bars;
  uint64_t* empty = bars + 1;
  uint64_t* acc_full = bars + 2;
  uint64_t* acc_empty = bars + 3;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles_m = (a.m + BM - 1) / BM, tiles_n = (a.n + BN - 1) / BN;
  const int64_t total = tiles_m * tiles_n * nb;
  const int num_kb = static_cast<int>((a.k + BK - 1) / BK);  // 1 or 2

  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_init(empty, 1);
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, CBS::EPI_WARPS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(CB::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int64_t g = 0;  // k-blocks issued: phase g of the one stage
      bool ok = true;
      for (int64_t w = blockIdx.x; w < total && ok; w += gridDim.x) {
        const TileCoord tc = tile_of(w, tiles_m, tiles_n);
        const int pa = a.a_bstride ? 4 * tc.b : 0, pb = a.b_bstride ? 4 * tc.b : 0;
        for (int kb = 0; kb < num_kb; ++kb, ++g) {
          if (!mbar_wait(empty, static_cast<uint32_t>(g & 1) ^ 1)) {
            atomicExch(err, 61);
            ok = false;
            break;
          }
          mbar_expect_tx(full, STAGE);
          tma_load_3d(smem, &tmA, full, kb * BK, tc.m0, pa);
          tma_load_3d(smem + CB::OFF_B, &tmB, full, kb * BK, tc.n0, pb);
        }
      }
      // every issued load has landed before the CTA can exit
      if (g > 0 && !mbar_wait(full, static_cast<uint32_t>((g - 1) & 1))) atomicExch(err, 62);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t id_w = idesc_bf16(BM, 2 * BN);
      constexpr uint32_t id_n = idesc_bf16(BM, BN);
      const uint32_t d_hi = tmem, d_lo = tmem + 256;
      int64_t g = 0, q = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; w < total && ok; w += gridDim.x, ++q) {
        if (!mbar_wait(acc_empty, static_cast<uint32_t>(q & 1) ^ 1)) {  // the previous tile was read
          atomicExch(err, 63);
          break;
        }
        fence_after();
        for (int kb = 0; kb < num_kb; ++kb, ++g) {
          if (!mbar_wait(full, static_cast<uint32_t>(g & 1))) {
            atomicExch(err, 64);
            ok = false;
            break;
          }
          fence_after();
          const uint32_t sa = su32(smem), sb = sa + CB::OFF_B;
#pragma unroll
          for (int j = 0; j < BK / 16; ++j) {
            const uint32_t o = j * 32;
            const uint64_t ar_l = smem_desc<ROWB>(sa + 2 * PLANE + o), ai_l = smem_desc<ROWB>(sa + 3 * PLANE + o);
            const uint64_t ar_h = smem_desc<ROWB>(sa + o), ai_h = smem_desc<ROWB>(sa + PLANE + o);
            const uint64_t b_h = smem_desc<ROWB>(sb + o), bi_h = smem_desc<ROWB>(sb + PLANE + o);
            const uint64_t b_l = smem_desc<ROWB>(sb + 2 * PLANE + o), bi_l = smem_desc<ROWB>(sb + 3 * PLANE + o);
            const uint32_t acc = (kb > 0 || j > 0) ? 1u : 0u;
            mma_bf16(d_lo, ar_l, b_h, id_w, acc);
            mma_bf16(d_lo, ai_l, bi_h, id_n | kNegateA, 1u);
            mma_bf16(d_lo + 128, ai_l, b_h, id_n, 1u);
            mma_bf16(d_lo, ar_h, b_l, id_w, 1u);
            mma_bf16(d_lo, ai_h, bi_l, id_n | kNegateA, 1u);
            mma_bf16(d_lo + 128, ai_h, b_l, id_n, 1u);
            mma_bf16(d_hi, ar_h, b_h, id_w, acc);
            mma_bf16(d_hi, ai_h, bi_h, id_n | kNegateA, 1u);
            mma_bf16(d_hi + 128, ai_h, b_h, id_n, 1u);
          }
          mma_commit(empty);
        }
        mma_commit(acc_full);  // also on error, so the fold sees issued MMAs retire
      }
    }
  } else {
    const int e = warp - 2;                        // 0..15
    const int q4 = warp & 3, cq = e >> 2;          // TMEM lane quarter; 32-column group
    const uint32_t lane_base = static_cast<uint32_t>(q4 * 32) << 16;
    float* tr = epi + e * 2 * 32 * 33;             // this warp's Re and Im transpose block
    const int split = a.c_split;
    bool pow2 = a.m >= 32 && a.n >= 32;
    for (int d = 0; d < a.rows.n; ++d) pow2 = pow2 && (a.rows.ext[d] & (a.rows.ext[d] - 1u)) == 0u;
    for (int d = 0; d < a.cols.n; ++d) pow2 = pow2 && (a.cols.ext[d] & (a.cols.ext[d] - 1u)) == 0u;
    BlockOrder& ord = reinterpret_cast<BlockOrder*>(epi + CBS::EPI_WARPS * 2 * 32 * 33)[e];
    {
      const BlockOrder o = block_order(pow2 ? map_offset(a.rows, lane) : 0, pow2 ? map_offset(a.cols, lane) : 0,
                                       pow2, lane);
      if (lane == 0) ord = o;
      __syncwarp();
    }
    int64_t q = 0;
    for (int64_t w = blockIdx.x; w < total; w += gridDim.x, ++q) {
      const TileCoord tc = tile_of(w, tiles_m, tiles_n);
      if (!mbar_wait(acc_full, static_cast<uint32_t>(q & 1))) {
        atomicExch(err, 65);
        break;
      }
      fence_after();
      // this warp's 32 columns: hi + lo of Re, then of Im, into the transpose block
      float v[32], u[32];
      const uint32_t col = lane_base + cq * 32;
      tmem_ld32(tmem + col, v);
      tmem_ld32(tmem + 256 + col, u);
#pragma unroll
      for (int j = 0; j < 32; ++j) tr[lane * 33 + j] = v[j] + u[j];
      tmem_ld32(tmem + 128 + col, v);
      tmem_ld32(tmem + 384 + col, u);
#pragma unroll
      for (int j = 0; j < 32; ++j) tr[32 * 33 + lane * 33 + j] = v[j] + u[j];
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);  // the accumulators are free for the next tile
      const int64_t m = static_cast<int64_t>(tc.m0) + q4 * 32 + lane;
      const bool row_ok = m < a.m;
      const int64_t ro = row_ok ? map_offset(a.rows, m) : 0;
      float* C = a.C + static_cast<int64_t>(tc.b) * a.c_bstride;
      const int64_t n = static_cast<int64_t>(tc.n0) + cq * 32 + lane;
      const bool col_ok = n < a.n;
      const int64_t co = col_ok ? map_offset(a.cols, n) : 0;
      if (ord.ok && __all_sync(0xffffffffu, row_ok && col_ok)) {
        const int64_t base = __shfl_sync(0xffffffffu, ro, 0) + __shfl_sync(0xffffffffu, co, 0);
        store_ordered(C, a.c_plane, split, tr, 33, 32 * 33, base, ord, lane);
      } else {
        store_block(C, a.c_plane, split, tr, 33, 32 * 33, ro, co, row_ok, col_ok, lane);
      }
      __syncwarp();
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CB::COLS));
  }
}

// 3-D map over a split-BF16 operand: (k, rows, plane), plane = 4*copy + {re_hi, im_hi,
// re_lo, im_lo}; box 32 x rows x 4 planes, 64-byte swizzle.
bool make_map_split(CUtensorMap* map, const float* base, int64_t rows, int64_t k, int64_t copies,
                    int64_t plane_elems, int box_rows) {
  auto enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(k), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(4 * copies)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(k * 2), static_cast<cuuint64_t>(plane_elems * 2)};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(CB::BK), static_cast<cuuint32_t>(box_rows), 4};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<float*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 3-D map over a 3M split-BF16 operand: (k, rows, plane), plane = 6*copy + {re_h, re_l,
// im_h, im_l, s_h, s_l}; box 32 x rows x 2 planes (one product's hi and lo), 64-byte swizzle.
bool make_map_split3m(CUtensorMap* map, const float* base, int64_t rows, int64_t k, int64_t copies,
                      int64_t plane_elems, int box_rows) {
  auto enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(k), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(6 * copies)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(k * 2), static_cast<cuuint64_t>(plane_elems * 2)};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(CB3::BK), static_cast<cuuint32_t>(box_rows), 2};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<float*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

cudaError_t launch_tcb3m(const StepArgs& a, int32_t nb, int* err, cudaStream_t st) {
  // the shared-memory opt-in, once per process (thread-safe static initialisation)
  static const cudaError_t configured =
      cudaFuncSetAttribute(contract_tcb3m_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CB3::SMEM);
  if (configured != cudaSuccess) return configured;
  CUtensorMap ta, tb;
  const int64_t ca = a.a_bstride ? static_cast<int64_t>(nb) : 1;
  const int64_t cb = a.b_bstride ? static_cast<int64_t>(nb) : 1;
  if (!make_map_split3m(&ta, a.A, a.m, a.k, ca, a.a_plane, BM) ||
      !make_map_split3m(&tb, a.B, a.n, a.k, cb, a.b_plane, BN))
    return cudaErrorInvalidValue;
  const int64_t tiles = ((a.m + BM - 1) / BM) * ((a.n + BN - 1) / BN);
  return launch_bands(contract_tcb3m_kernel, tiles, nb, CB3::THREADS, CB3::SMEM, st, ta, tb, a, err);
}

// Tiles per batch entry in one launch of the per-tile paired kernel: about kBandWaves waves
// of the clusters that can be resident at once. The clusters of a launch start together and
// stay near each other in k, so the panels they share come from DRAM about once per wave
// (one launch for a whole deep step let them drift apart: 2.4x the DRAM traffic).
int64_t pair_band_tiles(int64_t pair_tiles, int32_t nb) {
  static const int clusters = [] {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(CB2::THREADS, 1, 1);
    cfg.dynamicSmemBytes = CB2::SMEM;
    cudaFuncSetAttribute(contract_tcb2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CB2::SMEM);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, contract_tcb2_kernel, &cfg) != cudaSuccess || n <= 0) n = 0;
    return n;
  }();
  if (kBandWaves <= 0 || clusters <= 0 || nb <= 0) return pair_tiles;
  const int64_t want = (int64_t(clusters) * kBandWaves + nb - 1) / nb;
  return want < pair_tiles ? want : pair_tiles;
}

cudaError_t launch_tcb(const StepArgs& a, int32_t nb, int* err, cudaStream_t st, bool pairs) {
  static const cudaError_t configured = [] {
    cudaError_t e =
        cudaFuncSetAttribute(contract_tcb_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, CB::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(contract_tcb_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, CB::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(contract_tcb_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               CBP::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(contract_tcb2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CB2::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(contract_tcb2p_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CB2P::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(contract_tcb_shallow_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CBS::SMEM);
    return e;
  }();
  if (configured != cudaSuccess) return configured;
  CUtensorMap ta, tb;
  const int64_t ca = a.a_bstride ? static_cast<int64_t>(nb) : 1;
  const int64_t cb = a.b_bstride ? static_cast<int64_t>(nb) : 1;
  if (a.recs) {
    // exponent scaling: one SM per tile, launched in bands, for every k
    if (!make_map_split(&ta, a.A, a.m, a.k, ca, a.a_plane, BM) ||
        !make_map_split(&tb, a.B, a.n, a.k, cb, a.b_plane, BN))
      return cudaErrorInvalidValue;
    const int64_t tiles = ((a.m + BM - 1) / BM) * ((a.n + BN - 1) / BN);
    return launch_bands(contract_tcb_kernel<true>, tiles, nb, CB::THREADS, CB::SMEM, st, ta, tb, a, err);
  }
  if (pairs && a.k > CBP::MAX_K && a.m >= 2 * BM) {
    // paired SMs: this CTA's 128 rows of A and 64 rows of B per box
    if (!make_map_split(&ta, a.A, a.m, a.k, ca, a.a_plane, BM) ||
        !make_map_split(&tb, a.B, a.n, a.k, cb, a.b_plane, BN / 2))
      return cudaErrorInvalidValue;
    const int64_t pair_tiles = ((a.m + 2 * BM - 1) / (2 * BM)) * ((a.n + BN - 1) / BN);
    if (a.k <= kPairsPersistentMaxK) {
      // persistent: as many clusters as are resident at once, each walking its items
      static const int clusters = [] {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2, 1, 1);
        cfg.blockDim = dim3(CB2::THREADS, 1, 1);
        cfg.dynamicSmemBytes = CB2P::SMEM;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, contract_tcb2p_kernel, &cfg) != cudaSuccess || n <= 0) n = 0;
        return n;
      }();
      if (clusters > 0) {
        const int64_t items = pair_tiles * static_cast<int64_t>(nb);
        const int64_t g = items < clusters ? items : clusters;
        contract_tcb2p_kernel<<<static_cast<unsigned>(2 * g), CB2::THREADS, CB2P::SMEM, st>>>(ta, tb, a, nb, err);
        return cudaGetLastError();
      }
    }
    const int64_t per_launch = pair_band_tiles(pair_tiles, nb);
    for (int64_t t0 = 0; t0 < pair_tiles; t0 += per_launch) {
      const int64_t cnt = pair_tiles - t0 < per_launch ? pair_tiles - t0 : per_launch;
      dim3 grid(static_cast<unsigned>(2 * cnt), static_cast<unsigned>(nb));
      contract_tcb2_kernel<<<grid, CB2::THREADS, CB2::SMEM, st>>>(ta, tb, a, t0, err);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (!make_map_split(&ta, a.A, a.m, a.k, ca, a.a_plane, BM) || !make_map_split(&tb, a.B, a.n, a.k, cb, a.b_plane, BN))
    return cudaErrorInvalidValue;
  const int64_t tiles = ((a.m + BM - 1) / BM) * ((a.n + BN - 1) / BN);
  if (a.k <= CBS::MAX_K && kShallowKernel) {
    // shallowest steps: persistent, sixteen epilogue warps, one CTA per SM
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t items = tiles * static_cast<int64_t>(nb);
    const unsigned grid = static_cast<unsigned>(items < sms ? items : sms);
    contract_tcb_shallow_kernel<<<grid, CBS::THREADS, CBS::SMEM, st>>>(ta, tb, a, nb, err);
    return cudaGetLastError();
  }
  if (a.k <= CBP::MAX_K) {
    // shallow step: persistent, one CTA per SM (the shared memory admits one)
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t items = tiles * static_cast<int64_t>(nb);
    const unsigned grid = static_cast<unsigned>(items < sms ? items : sms);
    contract_tcb_persistent_kernel<<<grid, CB::THREADS, CBP::SMEM, st>>>(ta, tb, a, nb, err);
    return cudaGetLastError();
  }
  return launch_bands(contract_tcb_kernel<false>, tiles, nb, CB::THREADS, CB::SMEM, st, ta, tb, a, err);
}

}  // namespace

bool tc_supported() { return true; }

cudaError_t launch_bounded_wait_selftest(int arrive, uint64_t limit_ns, int* err, cudaStream_t st) {
  bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(arrive, limit_ns, err);
  return cudaGetLastError();
}

bool tc_step_ok(int64_t m, int64_t n, int64_t k, int32_t prec) {
  // TMA rows are k * element bytes and must be whole 16-byte units: k % 4 for the FP32
  // operands, k % 8 for the split-BF16 ones
  const int64_t kq = prec == TN_C64_BF16X3 ? 8 : 4;
  // n below the 128-column tile is allowed (the B box is zero-filled past n, the epilogue
  // masks the columns): a quarter-filled tile still beats the CUDA cores several-fold
  return m >= BM && n >= 16 && k >= 8 && k % kq == 0 && k <= (int64_t(1) << 30) && m < (int64_t(1) << 31) &&
         n < (int64_t(1) << 31);
}

int64_t tc_launches(int64_t m, int64_t n, int64_t k, int32_t nb, int32_t prec, bool pairs, bool scaled) {
  if (prec == TN_C64_BF16X3 && !scaled) {
    if (k <= CBP::MAX_K) return 1;  // persistent kernels
    if (pairs && m >= 2 * BM) {
      if (k <= kPairsPersistentMaxK) return 1;
      const int64_t pair_tiles = ((m + 2 * BM - 1) / (2 * BM)) * ((n + BN - 1) / BN);
      const int64_t per = pair_band_tiles(pair_tiles, nb);
      return (pair_tiles + per - 1) / per;
    }
  }
  if (prec != TN_C64_BF16X3 && prec != kPrecBF16x3M)
    return tf32_launches(m, n, nb, prec == TN_R32_TF32 || prec == TN_R32_3XTF32);
  const int64_t tiles = ((m + BM - 1) / BM) * ((n + BN - 1) / BN);
  const int64_t per = sm_band_tiles(tiles, nb);
  return (tiles + per - 1) / per;
}

cudaError_t launch_contract_tc(const StepArgs& a, int32_t nb, int32_t prec, bool cplx, int* err,
                               cudaStream_t st, bool pairs) {
  if (a.maxplus) return cudaErrorNotSupported;
  if (!cplx || prec == TN_C64_TF32 || prec == TN_C64_3XTF32) return launch_contract_tf32(a, nb, prec, cplx, err, st);
  if (prec == kPrecBF16x3M) return a.recs ? cudaErrorNotSupported : launch_tcb3m(a, nb, err, st);
  if (prec == TN_C64_BF16X3) return launch_tcb(a, nb, err, st, pairs);
  return cudaErrorNotSupported;
}

}  // namespace tn
