// TF32-family tensor-core kernels (sm_103a): the TF32 and 3xTF32 forms of the pairwise
// GEMM C[b] = A[b] (m x k) . B[b] (n x k)^T, complex (4M) and real, with or without
// exponent scaling:
//   contract_tc_kernel<REAL, SCALED>   TF32: A_re, A_im, B_re, B_im fp32 tiles, 32-deep
//                                      k-blocks, 3 stages, D_rr / D_ii / D_x accumulators
//                                      (Re C = D_rr - D_ii, Im C = D_x); 192 threads (real
//                                      tiles: 2 stages, 320 threads, two CTAs per SM);
//   contract_tc3_kernel<REAL, SCALED>  3xTF32: eight warps split each staged tile into
//                                      hi = RN_tf32(v) and lo = v - hi, hi.hi in 32-term
//                                      chunks folded into round-to-nearest registers, cross
//                                      terms in their own accumulator; 320 threads.
// Real steps take 128 x 256 output tiles (two B tiles read as one 256-row operand).
// Every mbarrier wait is bounded by wall time; on expiry the CTA records an error code,
// drains its copies, frees its tensor memory and returns.
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "mbarrier.cuh"
#include "scale.cuh"
#include "split_bf16.cuh"
#include "tc_common.cuh"

namespace tn {
namespace {

// TF32 form (contract_tc_kernel). A complex stage holds A_re A_im B_re B_im (3 stages, one
// CTA per SM; tensor memory D_rr @0, D_ii @128, D_x @256; warps 0 TMA, 1 MMA, 2-5 epilogue).
// A real one holds A B_0 B_1, the two B tiles of a 256-column tile, in 2 stages, and its
// accumulator takes 256 columns: two CTAs fit on an SM, so one's epilogue overlaps the
// other's MMAs; eight epilogue warps (2-9: warp w drains TMEM lane quarter w % 4, columns
// 128 ((w - 2) / 4) .. + 127) store its 32K results.
template <bool REAL>
struct Cfg {
  static constexpr int BK = 32;                             // fp32 elements per k-block
  static constexpr int ROWB = BK * 4;                       // bytes per tile row (= swizzle span)
  static constexpr int TILE_A = BM * ROWB;
  static constexpr int TILE_B = BN * ROWB;
  static constexpr int OFF_B = REAL ? TILE_A : 2 * TILE_A;  // first B tile
  static constexpr int STAGE = REAL ? TILE_A + 2 * TILE_B : 2 * TILE_A + 2 * TILE_B;
  static constexpr int STAGES = REAL ? 2 : 3;
  static constexpr int THREADS = REAL ? 320 : 192;
  static constexpr uint32_t TMEM_COLS = REAL ? 256 : 512;
  static constexpr int SMEM = STAGES * STAGE + 1024 /*barriers*/ + 1024 /*align*/;
  static_assert(SMEM <= 232448 && STAGE % 1024 == 0 && OFF_B % 1024 == 0, "stages fit, swizzle-aligned tiles");
  static_assert((THREADS / 32 - 2) * 2 * 32 * 33 * 4 <= STAGES * STAGE, "epilogue transposes fit the stages");
};

// v rounded to the nearest value with 10 fraction bits (ties away from zero): half a unit in
// the 10th fraction bit is added to the magnitude and the low 13 bits cleared (finite v
// below the largest TF32-representable value; an overflow would carry into the exponent).
__device__ __forceinline__ float tf32_rn(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xffffe000u);
}

// REAL: a real step. Its tile is 128 x 256: the stage holds A and the B tiles of columns
// n0 .. n0 + 127 and n0 + 128 .. n0 + 255 side by side, one 128 x 256 MMA per k-atom reads
// the two as one operand, and the accumulator's 256 columns are the tile's output columns
// in order. SCALED: exponent scaling (a.recs).
template <bool REAL, bool SCALED>
__global__ void __launch_bounds__(Cfg<REAL>::THREADS, 1)
    contract_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       StepArgs a, int64_t t_first, int* err) {
  using G = Cfg<REAL>;
  constexpr int STAGES = G::STAGES, BK = G::BK, ROWB = G::ROWB;
  constexpr int TILE_A = G::TILE_A, TILE_B = G::TILE_B, STAGE = G::STAGE, OFF_B = G::OFF_B;
  constexpr int TN = REAL ? 2 * BN : BN;            // output columns per tile
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
  uint64_t* full = bars;                     // [STAGES]
  uint64_t* empty = bars + STAGES;           // [STAGES]
  uint64_t* acc_full = bars + 2 * STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped raster over output tiles for L2 reuse of A and B tiles
  const int64_t tiles_m = (a.m + BM - 1) / BM, tiles_n = (a.n + TN - 1) / TN;
  const int64_t t = t_first + blockIdx.x;  // this launch's tiles start at t_first
  const int64_t per_group = GROUP_M * tiles_n;
  const int64_t first_m = (t / per_group) * GROUP_M;
  const int64_t gm = tiles_m - first_m < GROUP_M ? tiles_m - first_m : GROUP_M;
  const int64_t tm = first_m + (t % per_group) % gm, tn = (t % per_group) / gm;
  const int m0 = static_cast<int>(tm * BM), n0 = static_cast<int>(tn * TN);
  const int b = blockIdx.y;
  const int num_kb = static_cast<int>((a.k + BK - 1) / BK);
  // plane of this batch entry's copy in the TMA maps: 2b + {re, im} complex, b real
  const int pa = a.a_bstride ? (REAL ? b : 2 * b) : 0, pb = a.b_bstride ? (REAL ? b : 2 * b) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(G::TMEM_COLS));
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
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1)) {
          atomicExch(err, 1);
          break;
        }
        mbar_expect_tx(&full[s], STAGE);
        uint8_t* st = smem + s * STAGE;
        const int k0 = kb * BK;
        tma_load_3d(st, &tmA, &full[s], k0, m0, pa);
        if constexpr (REAL) {
          // the second B tile may lie wholly past n: the box is then zero-filled
          tma_load_3d(st + OFF_B, &tmB, &full[s], k0, n0, pb);
          tma_load_3d(st + OFF_B + TILE_B, &tmB, &full[s], k0, n0 + BN, pb);
        } else {
          tma_load_3d(st + TILE_A, &tmA, &full[s], k0, m0, pa + 1);
          tma_load_3d(st + 2 * TILE_A, &tmB, &full[s], k0, n0, pb);
          tma_load_3d(st + 2 * TILE_A + TILE_B, &tmB, &full[s], k0, n0, pb + 1);
        }
        issued = kb + 1;
      }
      // drain: every stage's last issued load has landed before the CTA can exit
      for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
        if (!mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1)) atomicExch(err, 2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(BM, TN);
      const uint32_t d_rr = tmem, d_ii = tmem + 128, d_x = tmem + 256;
      for (int kb = 0; kb < num_kb; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait(&full[s], ph)) {
          atomicExch(err, 3);
          break;
        }
        fence_after();
        const uint32_t st = su32(smem + s * STAGE);
#pragma unroll
        for (int j = 0; j < BK / 8; ++j) {
          const uint32_t acc = (kb > 0 || j > 0) ? 1u : 0u;
          const uint64_t ar = smem_desc<ROWB>(st + j * 32), ai = smem_desc<ROWB>(st + TILE_A + j * 32);
          const uint64_t br = smem_desc<ROWB>(st + OFF_B + j * 32);
          const uint64_t bi = smem_desc<ROWB>(st + OFF_B + TILE_B + j * 32);
          if constexpr (REAL) {
            mma_tf32(tmem, ar, br, idesc, acc);  // br: the 256 B rows of both tiles
          } else {
            mma_tf32(d_rr, ar, br, idesc, acc);
            mma_tf32(d_ii, ai, bi, idesc, acc);
            mma_tf32(d_x, ar, bi, idesc, acc);
            mma_tf32(d_x, ai, br, idesc, 1u);
          }
        }
        mma_commit(&empty[s]);
      }
      mma_commit(acc_full);  // also on error: lets the epilogue see in-flight MMAs retire
    }
  } else {
    // epilogue: TMEM lane quarter of this warp = warp % 4
    const bool ok = mbar_wait(acc_full, 0);
    if (!ok) atomicExch(err, 6);
    fence_after();
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const int64_t m = static_cast<int64_t>(m0) + row;
    const bool row_ok = ok && m < a.m;
    const int64_t ro = row_ok ? map_offset(a.rows, m) : 0;
    float* C = a.C + static_cast<int64_t>(b) * a.c_bstride;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
    // Each 32 x 32 block goes through shared memory (the drained stage buffers) and is
    // stored in address order (store_block): 32 consecutive elements per warp store for
    // the usual layouts.
    float* tr = reinterpret_cast<float*>(smem) + (warp - 2) * 2 * 32 * 33;  // [2][32][33]
    const TcScale sc = tc_scale(a, b);
    int lmax = -127;
    // this warp's 32-column blocks: all of a complex tile's, half of a real tile's
    constexpr int NCB = REAL ? TN / 64 : TN / 32;
    const int c_first = REAL ? ((warp - 2) >> 2) * NCB : 0;
    for (int c = c_first; c < c_first + NCB; ++c) {
      const int64_t nb0 = static_cast<int64_t>(n0) + c * 32;
      if constexpr (REAL) {
        float v[32];
        tmem_ld32(tmem + lane_base + c * 32, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if constexpr (SCALED) {
            v[j] = v[j] * sc.sa * sc.sb;
            if (row_ok && nb0 + j < a.n) lmax = max(lmax, exp_of(fabsf(v[j])));
          }
          tr[lane * 33 + j] = v[j];
        }
      } else {
        float rr[32], ii[32], xx[32];
        tmem_ld32(tmem + lane_base + c * 32, rr);
        tmem_ld32(tmem + lane_base + 128 + c * 32, ii);
        tmem_ld32(tmem + lane_base + 256 + c * 32, xx);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          float re = rr[j] - ii[j], im = xx[j];
          if constexpr (SCALED) {
            re = re * sc.sa * sc.sb;
            im = im * sc.sa * sc.sb;
            if (row_ok && nb0 + j < a.n) lmax = max(lmax, exp_of(fmaxf(fabsf(re), fabsf(im))));
          }
          tr[lane * 33 + j] = re;
          tr[32 * 33 + lane * 33 + j] = im;
        }
      }
      __syncwarp();
      const int64_t n = nb0 + lane;
      const bool col_ok = ok && n < a.n;
      store_block<REAL>(C, a.c_plane, kFmtPlanar, tr, 33, 32 * 33, ro, col_ok ? map_offset(a.cols, n) : 0, row_ok,
                        col_ok, lane);
      __syncwarp();
    }
    if constexpr (SCALED) tc_scale_finish(a, b, lmax, t == 0 && threadIdx.x == 64);
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::TMEM_COLS));
  }
}

// ---------------------------------------------------------------------------------
// 3xTF32 with round-to-nearest accumulation across k.
//
// The tensor core's FP32 accumulator truncates each addition, so a long TMEM
// accumulation drifts toward zero by ~k * 2^-25 relative (measured). Here the MMAs
// accumulate only CK k-blocks (CK * 16 terms) into the TMEM chunk accumulator
// (re @0, im @128; Re uses the instruction's negate-A bit for -A_im.B_im); eight
// warps then add the chunk into running totals held in their registers with ordinary
// round-to-nearest FP32 additions, and release the accumulator for the next chunk.
// The same eight warps split every staged tile into hi/lo (so the MMA pipe waits only
// for the short drain), and finally write the totals out. 128 x 128 tiles: the kernel is
// bound by shared-memory operand reads (each 3xTF32 MMA re-reads its tiles), so the
// wide tile keeps reads per flop low.
// Warps: 0 TMA, 1 MMA + TMEM, 2-9 split / drain / epilogue (320 threads); warp w of
// 2-9 drains TMEM lane quarter w % 4, columns 64 * ((w - 2) / 4) .. +63.

// Stage layout (raw values and, in the lo buffers, their lo parts), 8 KiB tiles:
//   A_re | A_im | -B_im | B_re | B_im
// so that [B_re | B_im] and [-B_im | B_re] are each one 256-row operand: per k-atom
// A_re.[B_re|B_im] and A_im.[-B_im|B_re] add into (Re, Im) with one 128 x 256 MMA each.
// A real step (REAL) uses the A_re, B_re and B_im slots for A and the B tiles of columns
// n0 .. n0 + 127 and n0 + 128 .. n0 + 255: a 128 x 256 tile, A.[B_0|B_1] per k-atom.
struct C3 {
  // CK = 2: 32-term chunks. Each truncating addition loses up to an ulp of the running chunk
  // sum, so the error grows with the chunk; 64-term chunks were 5 % faster but left the
  // FP32-accurate form at twice plain FP32's error on long paths of small steps.
  static constexpr int BK = 16, ROWB = 64, CK = 2;
  static constexpr int TILE_A = BM * ROWB;                  // 8 KiB
  static constexpr int TILE_B = BN * ROWB;                  // 8 KiB
  static constexpr int OFF_AI = TILE_A, OFF_BNEG = 2 * TILE_A;
  static constexpr int OFF_BR = 2 * TILE_A + TILE_B, OFF_BI = 2 * TILE_A + 2 * TILE_B;
  static constexpr int TMA_BYTES = 2 * TILE_A + 2 * TILE_B; // 32 KiB per stage by TMA
  static constexpr int STAGE = 2 * TILE_A + 3 * TILE_B;     // 40 KiB
  static constexpr int STAGES = 3, LO = 2;
  static constexpr int THREADS = 320;
  static constexpr int SMEM = (STAGES + LO) * STAGE + 1024 + 1024;
  static constexpr uint32_t COLS = 512;  // re @0, im @128, re_lo @256, im_lo @384
};

// 32 columns nb0 .. nb0 + 31 of this thread's row of a real result, v[OFF .. OFF + 31]: one
// column of the warp's 32 rows per warp store when the rows are the unit-stride side, else
// through shared memory (tr, this warp's 32 x 33 floats) one row per warp store. The lanes
// compute the 32 column offsets once and pass them round by shuffles.
template <int OFF>
__device__ __forceinline__ void store_real_cols(float* C, const StepArgs& a, const float (&v)[64], int64_t nb0,
                                                int64_t ro, bool row_ok, bool ok, bool rows_unit, float* tr,
                                                int lane) {
  const int64_t n = nb0 + lane;
  const bool col_ok = ok && n < a.n;
  const int64_t co = col_ok ? map_offset(a.cols, n) : 0;  // lane j: column nb0 + j
  if (rows_unit) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t co_j = __shfl_sync(0xffffffffu, co, j);
      if (row_ok && nb0 + j < a.n) C[ro + co_j] = v[OFF + j];
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) tr[lane * 33 + j] = v[OFF + j];
  __syncwarp();
  for (int r = 0; r < 32; ++r) {
    const int64_t ro_r = __shfl_sync(0xffffffffu, ro, r);
    const bool ok_r = __shfl_sync(0xffffffffu, row_ok ? 1 : 0, r) != 0;
    if (ok_r && col_ok) C[ro_r + co] = tr[r * 33 + lane];
  }
  __syncwarp();
}

template <bool REAL, bool SCALED>
__global__ void __launch_bounds__(C3::THREADS, 1)
    contract_tc3_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        StepArgs a, int64_t t_first, int* err) {
  constexpr int STAGES = C3::STAGES, BK = C3::BK, ROWB = C3::ROWB, CK = C3::CK;
  constexpr int TILE_A = C3::TILE_A, TILE_B = C3::TILE_B, STAGE = C3::STAGE;
  constexpr int TN = REAL ? 2 * BN : BN;                                    // output columns per tile
  constexpr int LOADED = REAL ? TILE_A + 2 * TILE_B : C3::TMA_BYTES;        // TMA bytes per stage
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* lo_base = smem + STAGES * STAGE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(lo_base + C3::LO * STAGE);
  uint64_t* full = bars;                     // [STAGES]
  uint64_t* empty = bars + STAGES;           // [STAGES]
  uint64_t* conv_full = bars + 2 * STAGES;   // [2]
  uint64_t* lo_empty = conv_full + 2;        // [2]
  uint64_t* acc_full = lo_empty + 2;         // chunk accumulated
  uint64_t* acc_empty = acc_full + 1;        // chunk drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles_m = (a.m + BM - 1) / BM, tiles_n = (a.n + TN - 1) / TN;
  const int64_t t = t_first + blockIdx.x;  // this launch's tiles start at t_first
  const int64_t per_group = GROUP_M * tiles_n;
  const int64_t first_m = (t / per_group) * GROUP_M;
  const int64_t gm = tiles_m - first_m < GROUP_M ? tiles_m - first_m : GROUP_M;
  const int64_t tm = first_m + (t % per_group) % gm, tn = (t % per_group) / gm;
  const int m0 = static_cast<int>(tm * BM), n0 = static_cast<int>(tn * TN);
  const int b = blockIdx.y;
  const int num_kb = static_cast<int>((a.k + BK - 1) / BK);
  const int n_chunks = (num_kb + CK - 1) / CK;
  const int pa = a.a_bstride ? (REAL ? b : 2 * b) : 0, pb = a.b_bstride ? (REAL ? b : 2 * b) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&conv_full[i], 256);
      mbar_init(&lo_empty[i], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(C3::COLS));
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
          atomicExch(err, 11);
          break;
        }
        mbar_expect_tx(&full[s], LOADED);
        uint8_t* st = smem + s * STAGE;
        const int k0 = kb * BK;
        tma_load_3d(st, &tmA, &full[s], k0, m0, pa);
        if constexpr (REAL) {
          // the second B tile may lie wholly past n: the box is then zero-filled
          tma_load_3d(st + C3::OFF_BR, &tmB, &full[s], k0, n0, pb);
          tma_load_3d(st + C3::OFF_BI, &tmB, &full[s], k0, n0 + BN, pb);
        } else {
          tma_load_3d(st + C3::OFF_AI, &tmA, &full[s], k0, m0, pa + 1);
          tma_load_3d(st + C3::OFF_BR, &tmB, &full[s], k0, n0, pb);
          tma_load_3d(st + C3::OFF_BI, &tmB, &full[s], k0, n0, pb + 1);
        }
        issued = kb + 1;
      }
      for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
        if (!mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1)) atomicExch(err, 12);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(BM, 2 * BN);  // 128 x 256: (Re | Im) at once
      const uint32_t d_hi = tmem, d_lo = tmem + 256;
      bool ok = true;
      for (int c = 0; c < n_chunks && ok; ++c) {
        const int kb_end = min(num_kb, (c + 1) * CK);
        for (int kb = c * CK; kb < kb_end; ++kb) {
          const int s = kb % STAGES;
          if (!mbar_wait(&full[s], (kb / STAGES) & 1) || !mbar_wait(&conv_full[kb & 1], (kb >> 1) & 1)) {
            atomicExch(err, 14);
            ok = false;
            break;
          }
          fence_after();
          const uint32_t st = su32(smem + s * STAGE);
          const uint32_t lo = su32(lo_base + (kb & 1) * STAGE);
          // the cross terms first: their accumulator runs over all of k (it is ~2^-11 of the
          // result, so its own truncation is negligible) and is read once, after the last
          // chunk, so a chunk's first k-block issues them before the wait for the previous
          // chunk's fold, which then overlaps tensor-core work
#pragma unroll
          for (int j = 0; j < BK / 8; ++j) {
            const uint64_t ar = smem_desc<ROWB>(st + j * 32), ai = smem_desc<ROWB>(st + C3::OFF_AI + j * 32);
            const uint64_t b_ri = smem_desc<ROWB>(st + C3::OFF_BR + j * 32);    // [B_re | B_im]
            const uint64_t b_nr = smem_desc<ROWB>(st + C3::OFF_BNEG + j * 32);  // [-B_im | B_re]
            const uint64_t arl = smem_desc<ROWB>(lo + j * 32), ail = smem_desc<ROWB>(lo + C3::OFF_AI + j * 32);
            const uint64_t bl_ri = smem_desc<ROWB>(lo + C3::OFF_BR + j * 32);
            const uint64_t bl_nr = smem_desc<ROWB>(lo + C3::OFF_BNEG + j * 32);
            mma_tf32(d_lo, arl, b_ri, idesc, (kb > 0 || j > 0) ? 1u : 0u);
            if constexpr (!REAL) mma_tf32(d_lo, ail, b_nr, idesc, 1u);
            mma_tf32(d_lo, ar, bl_ri, idesc, 1u);
            if constexpr (!REAL) mma_tf32(d_lo, ai, bl_nr, idesc, 1u);
          }
          if (kb == c * CK) {
            // the chunk accumulator must have been folded before the hi MMAs reuse it
            if (!mbar_wait(acc_empty, (c & 1) ^ 1)) {
              atomicExch(err, 13);
              ok = false;
              mma_commit(&empty[s]);
              mma_commit(&lo_empty[kb & 1]);
              break;
            }
            fence_after();
          }
          // hi.hi products into the main accumulators (Re | Im), so the main sums take only
          // two truncating additions per 8 terms (one for a real step: its 256 columns are
          // all hi.hi)
#pragma unroll
          for (int j = 0; j < BK / 8; ++j) {
            const uint32_t acc = (kb > c * CK || j > 0) ? 1u : 0u;
            const uint64_t ar = smem_desc<ROWB>(st + j * 32), ai = smem_desc<ROWB>(st + C3::OFF_AI + j * 32);
            const uint64_t b_ri = smem_desc<ROWB>(st + C3::OFF_BR + j * 32);
            const uint64_t b_nr = smem_desc<ROWB>(st + C3::OFF_BNEG + j * 32);
            mma_tf32(d_hi, ar, b_ri, idesc, acc);
            if constexpr (!REAL) mma_tf32(d_hi, ai, b_nr, idesc, 1u);
          }
          mma_commit(&empty[s]);
          mma_commit(&lo_empty[kb & 1]);
        }
        mma_commit(acc_full);  // also on error, so the drain sees issued MMAs retire
      }
    }
  } else {
    const int et = threadIdx.x - 64;  // 0..255
    const int q = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
    float run_re[64], run_im[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) run_re[i] = run_im[i] = 0.f;
    bool ok = true;
    for (int kb = 0; kb <= num_kb; ++kb) {
      // Fold chunk dc of the TMEM accumulators into the register totals and release
      // them: once one k-block into the next chunk is split (so the MMA pipe restarts at
      // once), and after the last k-block.
      const int dc = kb == num_kb ? n_chunks - 1 : (kb % CK == 0 && kb > 0 ? kb / CK - 1 : -1);
      if (kb < num_kb) {
        const int s = kb % STAGES;
        if (ok && (!mbar_wait(&full[s], (kb / STAGES) & 1) || !mbar_wait(&lo_empty[kb & 1], ((kb >> 1) & 1) ^ 1))) {
          atomicExch(err, 15);
          ok = false;
        }
      }
      if (kb < num_kb && ok) {
        const int s = kb % STAGES;
        float4* src = reinterpret_cast<float4*>(smem + s * STAGE);
        float4* dst = reinterpret_cast<float4*>(lo_base + (kb & 1) * STAGE);
        // hi = value rounded to the nearest TF32 (written back in place), lo = value - hi
        // (exact); for B_im also -hi and -lo. kind::tf32 reads an FP32 operand by dropping
        // its low 13 mantissa bits (tests/test_gpu_tc.py::test_tf32_operand_rounding), so hi
        // is read exactly and only lo is truncated -- by at most 2^-10 of |lo|, with the
        // sign of lo, i.e. without a bias. (Using the staged value itself as hi would have
        // the hardware truncate it: a bias toward zero in every product.)
        // float4s of A (A_re, A_im; a real step's A alone), then of the two B slots
        constexpr int NA = (REAL ? TILE_A : 2 * TILE_A) / 16;
        constexpr int SKIP = (C3::OFF_BR - (REAL ? TILE_A : 2 * TILE_A)) / 16;
#pragma unroll 4
        for (int i = et; i < LOADED / 16; i += 256) {
          const int f = i < NA ? i : i + SKIP;  // skip the -B_im slot (and a real step's A_im)
          const float4 v = src[f];
          float4 h, l;
          h.x = tf32_rn(v.x);
          h.y = tf32_rn(v.y);
          h.z = tf32_rn(v.z);
          h.w = tf32_rn(v.w);
          l.x = v.x - h.x;
          l.y = v.y - h.y;
          l.z = v.z - h.z;
          l.w = v.w - h.w;
          src[f] = h;
          dst[f] = l;
          if (!REAL && f >= C3::OFF_BI / 16) {
            const int g = f - (C3::OFF_BI - C3::OFF_BNEG) / 16;
            src[g] = make_float4(-h.x, -h.y, -h.z, -h.w);
            dst[g] = make_float4(-l.x, -l.y, -l.z, -l.w);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&conv_full[kb & 1]);
      }
      if (dc >= 0 && ok) {
        if (!mbar_wait(acc_full, dc & 1)) {
          atomicExch(err, 16);
          ok = false;
        } else {
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
            if (dc == n_chunks - 1) {  // last chunk: the cross terms too
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
      }
    }
    // epilogue: thread = TMEM lane (row); this warp's 64 columns
    const int row = q * 32 + lane;
    const int64_t m = static_cast<int64_t>(m0) + row;
    const bool row_ok = ok && m < a.m;
    const int64_t ro = row_ok ? map_offset(a.rows, m) : 0;
    float* C = a.C + static_cast<int64_t>(b) * a.c_bstride;
    // The stage buffers are free here: this warp's last drain waited for the final MMA,
    // which waited for every warp's last split; no TMA load is outstanding.
    // Row-by-row stores (one row per warp store, through shared memory when the columns
    // are the unit-stride side): the address-ordered block store costs this kernel
    // registers its split loop needs.
    const bool rows_unit = a.rows.n > 0 && a.rows.stride[a.rows.n - 1] == 1;
    float* tr = reinterpret_cast<float*>(smem) + (warp - 2) * 2 * 32 * 33;  // [2][32][33]
    if constexpr (SCALED) {
      const TcScale sc = tc_scale(a, b);
      int lmax = -127;
      // (rows past m and columns past n hold zeros: their operands were zero-filled by TMA,
      // as the k tail is)
#pragma unroll
      for (int i = 0; i < 64; ++i) {
        run_re[i] = run_re[i] * sc.sa * sc.sb;
        run_im[i] = run_im[i] * sc.sa * sc.sb;
        lmax = max(lmax, REAL ? max(exp_of(fabsf(run_re[i])), exp_of(fabsf(run_im[i])))
                              : exp_of(fmaxf(fabsf(run_re[i]), fabsf(run_im[i]))));
      }
      tc_scale_finish(a, b, lmax, t == 0 && threadIdx.x == 64);
    }
    if constexpr (REAL) {
      // run_re: columns n0 + half * 64 + (0 .. 63), run_im: the same + 128; one row per
      // warp store (through shared memory when the columns are the unit-stride side)
      const int64_t c0 = static_cast<int64_t>(n0) + half * 64;
      store_real_cols<0>(C, a, run_re, c0, ro, row_ok, ok, rows_unit, tr, lane);
      store_real_cols<32>(C, a, run_re, c0 + 32, ro, row_ok, ok, rows_unit, tr, lane);
      store_real_cols<0>(C, a, run_im, c0 + 128, ro, row_ok, ok, rows_unit, tr, lane);
      store_real_cols<32>(C, a, run_im, c0 + 160, ro, row_ok, ok, rows_unit, tr, lane);
    } else {
#pragma unroll
      for (int cb = 0; cb < 2; ++cb) {
        const int64_t nb0 = static_cast<int64_t>(n0) + half * 64 + cb * 32;
        const int64_t n = nb0 + lane;
        const bool col_ok = ok && n < a.n;
        const int64_t co = col_ok ? map_offset(a.cols, n) : 0;  // lane j: column nb0 + j
        if (rows_unit) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int64_t co_j = __shfl_sync(0xffffffffu, co, j);
            if (row_ok && nb0 + j < a.n) {
              C[ro + co_j] = run_re[cb * 32 + j];
              C[a.c_plane + ro + co_j] = run_im[cb * 32 + j];
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            tr[lane * 33 + j] = run_re[cb * 32 + j];
            tr[32 * 33 + lane * 33 + j] = run_im[cb * 32 + j];
          }
          __syncwarp();
          for (int r = 0; r < 32; ++r) {
            const int64_t ro_r = __shfl_sync(0xffffffffu, ro, r);
            const bool ok_r = __shfl_sync(0xffffffffu, row_ok ? 1 : 0, r) != 0;
            if (ok_r && col_ok) {
              C[ro_r + co] = tr[r * 33 + lane];
              C[a.c_plane + ro_r + co] = tr[32 * 33 + r * 33 + lane];
            }
          }
          __syncwarp();
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C3::COLS));
  }
}

// Planes of an operand's TMA map: 2 per stored copy (re, im) for a complex step, 1 for a
// real one (plane p of a real batched operand starts at p * its batch stride, which equals
// its plane size); one copy unless the operand is batched.
int64_t map_planes(bool batched, int32_t nb, bool real) {
  return (batched ? static_cast<int64_t>(nb) : 1) * (real ? 1 : 2);
}
// Output columns per tile of the TF32-family kernels: real steps take 128 x 256 tiles.
int64_t tf32_tiles(int64_t m, int64_t n, bool real) {
  const int64_t tn = real ? 2 * BN : BN;
  return ((m + BM - 1) / BM) * ((n + tn - 1) / tn);
}

template <bool REAL, bool SCALED>
cudaError_t launch_tf32(const StepArgs& a, int32_t nb, int* err, cudaStream_t st) {
  using G = Cfg<REAL>;
  static const cudaError_t configured = cudaFuncSetAttribute(
      contract_tc_kernel<REAL, SCALED>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  if (configured != cudaSuccess) return configured;
  CUtensorMap ta, tb;
  if (!make_map(&ta, a.A, a.m, a.k, map_planes(a.a_bstride != 0, nb, REAL), a.a_plane, BM, G::BK) ||
      !make_map(&tb, a.B, a.n, a.k, map_planes(a.b_bstride != 0, nb, REAL), a.b_plane, BN, G::BK))
    return cudaErrorInvalidValue;
  return launch_bands(contract_tc_kernel<REAL, SCALED>, tf32_tiles(a.m, a.n, REAL), nb, G::THREADS, G::SMEM, st, ta,
                      tb, a, err);
}

template <bool REAL, bool SCALED>
cudaError_t launch_tc3(const StepArgs& a, int32_t nb, int* err, cudaStream_t st) {
  static const cudaError_t configured = cudaFuncSetAttribute(
      contract_tc3_kernel<REAL, SCALED>, cudaFuncAttributeMaxDynamicSharedMemorySize, C3::SMEM);
  if (configured != cudaSuccess) return configured;
  CUtensorMap ta, tb;
  if (!make_map(&ta, a.A, a.m, a.k, map_planes(a.a_bstride != 0, nb, REAL), a.a_plane, BM, C3::BK) ||
      !make_map(&tb, a.B, a.n, a.k, map_planes(a.b_bstride != 0, nb, REAL), a.b_plane, BN, C3::BK))
    return cudaErrorInvalidValue;
  return launch_bands(contract_tc3_kernel<REAL, SCALED>, tf32_tiles(a.m, a.n, REAL), nb, C3::THREADS, C3::SMEM, st,
                      ta, tb, a, err);
}

}  // namespace

cudaError_t launch_contract_tf32(const StepArgs& a, int32_t nb, int32_t prec, bool cplx, int* err,
                                 cudaStream_t st) {
  const bool sc = a.recs != nullptr;
  if (!cplx) {
    if (prec == TN_R32_TF32) return sc ? launch_tf32<true, true>(a, nb, err, st) : launch_tf32<true, false>(a, nb, err, st);
    if (prec == TN_R32_3XTF32) return sc ? launch_tc3<true, true>(a, nb, err, st) : launch_tc3<true, false>(a, nb, err, st);
    return cudaErrorNotSupported;
  }
  if (prec == TN_C64_TF32) return sc ? launch_tf32<false, true>(a, nb, err, st) : launch_tf32<false, false>(a, nb, err, st);
  if (prec == TN_C64_3XTF32) return sc ? launch_tc3<false, true>(a, nb, err, st) : launch_tc3<false, false>(a, nb, err, st);
  return cudaErrorNotSupported;
}

int64_t tf32_launches(int64_t m, int64_t n, int32_t nb, bool real) {
  const int64_t tiles = tf32_tiles(m, n, real);
  const int64_t per = sm_band_tiles(tiles, nb);
  return (tiles + per - 1) / per;
}

}  // namespace tn
