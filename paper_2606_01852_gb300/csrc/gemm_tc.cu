// Tensor-core path for the dense pairwise steps (sm_103a): planar complex GEMM
//   C[b] = A[b] (m x k) . B[b] (n x k)^T      (complex, 4M real decomposition)
// with both operands K-major, written through the separable row/column offset maps.
// The kernels compute 128 x 128 output tiles per SM (256 x 128 per pair of SMs in the
// cta_group::2 forms) with one elected thread issuing tcgen05.mma from shared-memory
// descriptors, operands brought by TMA into a ring of stages (mbarrier transaction counts),
// accumulators in tensor memory:
//   contract_tc_kernel<1>          TF32 form: A_re, A_im, B_re, B_im fp32 tiles, 32-deep
//                                  k-blocks, 3 stages, D_rr / D_ii / D_x accumulators
//                                  (Re C = D_rr - D_ii, Im C = D_x); 192 threads;
//   contract_tc3_kernel            3xTF32 form: eight warps split each staged tile into
//                                  hi = RN_tf32(v) and lo = v - hi, hi.hi in 64-term chunks
//                                  folded into round-to-nearest registers, cross terms in
//                                  their own accumulator; 320 threads;
//   contract_tcb_kernel            BF16x3 form: operands already split into BF16 hi/lo
//                                  planes by their producers, kind::f16, 256-term chunks;
//   contract_tcb2_kernel           BF16x3 on paired SMs (m >= 256, k > 4096): one two-CTA
//                                  cluster per 256 x 128 tile, M = 256 MMAs;
//   contract_tcb2p_kernel          the same, persistent clusters (256 < k <= 4096);
//   contract_tcb3m_kernel          BF16x3 with the 3M complex product;
//   contract_tcb_persistent_kernel BF16x3 for shallow steps (k <= 256): one CTA per SM over
//                                  the tiles, stores of a tile overlapping the next tile;
//   contract_tcb_shallow_kernel    the same for k <= 64 with sixteen epilogue warps.
// The epilogues of the TF32 and BF16x3 kernels store each 32 x 32 block in address order
// (store_block). Every mbarrier wait is bounded by wall time; on expiry the CTA records an
// error code, drains its copies, frees its tensor memory and returns.
#include <cstdint>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "mbarrier.cuh"
#include "split_bf16.cuh"

namespace tn {
namespace {

constexpr int BM = 128, BN = 128;
constexpr int NTHREADS = 192;
constexpr uint32_t TMEM_COLS = 512;                         // D_rr @0, D_ii @128, D_x @256
constexpr int GROUP_M = 16;                                 // raster: tiles grouped along M

template <int SPLIT>
struct Cfg {
  static constexpr int BK = SPLIT == 1 ? 32 : 16;           // fp32 elements per k-block
  static constexpr int ROWB = BK * 4;                       // bytes per tile row (= swizzle span)
  static constexpr int TILE_A = BM * ROWB;
  static constexpr int TILE_B = BN * ROWB;
  static constexpr int STAGE = 2 * TILE_A + 2 * TILE_B;     // A_re A_im B_re B_im
  static constexpr int STAGES = SPLIT == 1 ? 3 : 4;
  static constexpr int LO = SPLIT == 1 ? 0 : 2;             // lo buffers
  static constexpr int SMEM = (STAGES + LO) * STAGE + 1024 /*barriers*/ + 1024 /*align*/;
};

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
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
// Shared-memory matrix descriptor of a K-major tile whose rows are ROWB bytes with the
// matching swizzle (128 B -> mode 2, 64 B -> mode 4); 8-row groups 8*ROWB bytes apart.
template <int ROWB>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFF) >> 4);
  d |= static_cast<uint64_t>(1) << 16;                 // leading byte offset (unused here)
  d |= static_cast<uint64_t>((8 * ROWB) >> 4) << 32;   // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                 // descriptor version
  d |= static_cast<uint64_t>(ROWB == 128 ? 2 : 4) << 61;
  return d;
}
// Instruction descriptor, kind::tf32: D f32, A/B tf32, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

#define TN_R8(i) "=r"(r[i + 0]), "=r"(r[i + 1]), "=r"(r[i + 2]), "=r"(r[i + 3]), "=r"(r[i + 4]), \
                 "=r"(r[i + 5]), "=r"(r[i + 6]), "=r"(r[i + 7])
// 32 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : TN_R8(0), TN_R8(8), TN_R8(16), TN_R8(24)
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
#undef TN_R8

__device__ __forceinline__ float tf32_trunc(float v) { return __uint_as_float(__float_as_uint(v) & 0xffffe000u); }
// v rounded to the nearest value with 10 fraction bits (ties away from zero): half a unit in
// the 10th fraction bit is added to the magnitude and the low 13 bits cleared (finite v
// below the largest TF32-representable value; an overflow would carry into the exponent).
__device__ __forceinline__ float tf32_rn(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xffffe000u);
}

// V consecutive 16-bit values (the low halves of x[]) as one store of 2V bytes.
template <int V>
__device__ __forceinline__ void store_halves(uint16_t* d, const uint32_t (&x)[V]) {
  if constexpr (V == 1) {
    d[0] = static_cast<uint16_t>(x[0]);
  } else if constexpr (V == 2) {
    *reinterpret_cast<uint32_t*>(d) = x[0] | (x[1] << 16);
  } else if constexpr (V == 4) {
    *reinterpret_cast<uint2*>(d) = make_uint2(x[0] | (x[1] << 16), x[2] | (x[3] << 16));
  } else {
    *reinterpret_cast<uint4*>(d) =
        make_uint4(x[0] | (x[1] << 16), x[2] | (x[3] << 16), x[4] | (x[5] << 16), x[6] | (x[7] << 16));
  }
}

// V consecutive elements (V = 1, 2, 4, 8) of an address-ordered run: Re values re[],
// Im values im[], stored at element `off` of a tensor copy that starts at C, in storage
// mode fmt (planar FP32, split BF16, or split BF16 with the 3M sum planes), one vector
// store per plane (off and the planes are V-aligned).
template <int V>
__device__ __forceinline__ void store_run(float* C, int64_t plane, int64_t off, const float* re, const float* im,
                                          int fmt) {
  if (fmt == kFmtPlanar) {
    if constexpr (V == 1) {
      C[off] = re[0];
      C[plane + off] = im[0];
    } else if constexpr (V == 2) {
      *reinterpret_cast<float2*>(C + off) = make_float2(re[0], re[1]);
      *reinterpret_cast<float2*>(C + plane + off) = make_float2(im[0], im[1]);
    } else {
#pragma unroll
      for (int h = 0; h < V; h += 4) {
        *reinterpret_cast<float4*>(C + off + h) = make_float4(re[h], re[h + 1], re[h + 2], re[h + 3]);
        *reinterpret_cast<float4*>(C + plane + off + h) = make_float4(im[h], im[h + 1], im[h + 2], im[h + 3]);
      }
    }
    return;
  }
  if constexpr (V >= 2) {
    if (fmt == kFmtSplit) {
      // hi = RN_bf16(v), lo = RN_bf16(v - hi), two values per conversion (the same values
      // as split_pair's one at a time); 32-bit word w holds elements 2w (low) and 2w + 1
      constexpr int W = V / 2;
      uint32_t hr[W], hi_[W], lr[W], li[W];
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(re[2 * w], re[2 * w + 1]);
        const __nv_bfloat162 b = __floats2bfloat162_rn(im[2 * w], im[2 * w + 1]);
        const __nv_bfloat162 c =
            __floats2bfloat162_rn(re[2 * w] - __low2float(a), re[2 * w + 1] - __high2float(a));
        const __nv_bfloat162 d =
            __floats2bfloat162_rn(im[2 * w] - __low2float(b), im[2 * w + 1] - __high2float(b));
        hr[w] = uint32_t(__bfloat16_as_ushort(a.x)) | (uint32_t(__bfloat16_as_ushort(a.y)) << 16);
        hi_[w] = uint32_t(__bfloat16_as_ushort(b.x)) | (uint32_t(__bfloat16_as_ushort(b.y)) << 16);
        lr[w] = uint32_t(__bfloat16_as_ushort(c.x)) | (uint32_t(__bfloat16_as_ushort(c.y)) << 16);
        li[w] = uint32_t(__bfloat16_as_ushort(d.x)) | (uint32_t(__bfloat16_as_ushort(d.y)) << 16);
      }
      uint16_t* S = reinterpret_cast<uint16_t*>(C) + off;
      if constexpr (W == 1) {
        *reinterpret_cast<uint32_t*>(S) = hr[0];
        *reinterpret_cast<uint32_t*>(S + plane) = hi_[0];
        *reinterpret_cast<uint32_t*>(S + 2 * plane) = lr[0];
        *reinterpret_cast<uint32_t*>(S + 3 * plane) = li[0];
      } else if constexpr (W == 2) {
        *reinterpret_cast<uint2*>(S) = make_uint2(hr[0], hr[1]);
        *reinterpret_cast<uint2*>(S + plane) = make_uint2(hi_[0], hi_[1]);
        *reinterpret_cast<uint2*>(S + 2 * plane) = make_uint2(lr[0], lr[1]);
        *reinterpret_cast<uint2*>(S + 3 * plane) = make_uint2(li[0], li[1]);
      } else {
        *reinterpret_cast<uint4*>(S) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
        *reinterpret_cast<uint4*>(S + plane) = make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
        *reinterpret_cast<uint4*>(S + 2 * plane) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
        *reinterpret_cast<uint4*>(S + 3 * plane) = make_uint4(li[0], li[1], li[2], li[3]);
      }
      return;
    }
  }
  // hi = RN_bf16(v), lo = RN_bf16(v - hi) of re, im (and s = re + im in the 3M form)
  uint32_t hr[V], hi_[V], lr[V], li[V];
#pragma unroll
  for (int u = 0; u < V; ++u) {
    __nv_bfloat16 a, b, c, d;
    split_pair(re[u], a, c);
    split_pair(im[u], b, d);
    hr[u] = __bfloat16_as_ushort(a);
    hi_[u] = __bfloat16_as_ushort(b);
    lr[u] = __bfloat16_as_ushort(c);
    li[u] = __bfloat16_as_ushort(d);
  }
  uint16_t* S = reinterpret_cast<uint16_t*>(C) + off;
  if (fmt == kFmtSplit) {
    store_halves<V>(S, hr);
    store_halves<V>(S + plane, hi_);
    store_halves<V>(S + 2 * plane, lr);
    store_halves<V>(S + 3 * plane, li);
    return;
  }
  uint32_t hs[V], ls[V];
#pragma unroll
  for (int u = 0; u < V; ++u) {
    __nv_bfloat16 a, c;
    split_pair(re[u] + im[u], a, c);
    hs[u] = __bfloat16_as_ushort(a);
    ls[u] = __bfloat16_as_ushort(c);
  }
  store_halves<V>(S, hr);
  store_halves<V>(S + plane, lr);
  store_halves<V>(S + 2 * plane, hi_);
  store_halves<V>(S + 3 * plane, li);
  store_halves<V>(S + 4 * plane, hs);
  store_halves<V>(S + 5 * plane, ls);
}

// The address-ordered stores of one block, lanes taking V = 2^VB consecutive addresses.
// e[k], src[k]: the k-th smallest bit weight (log2) and which bit of r (0-4) or c (5-9)
// carries it; the VB smallest weights are 1, 2, ..., 2^(VB-1).
template <int VB>
__device__ __forceinline__ void store_sorted(float* C, int64_t plane, int split, const float* t, int pitch, int cs,
                                             int64_t base, const int* e, const int* src, int lane) {
  constexpr int V = 1 << VB;
  // r and c take disjoint bits, so t's index r * pitch + c is a sum of one increment per
  // set bit: the lane's part, the store's part and, per element of the run, du[u]
  auto step = [&](int k) { return src[k] < 5 ? pitch << src[k] : 1 << (src[k] - 5); };
  int du[V];
#pragma unroll
  for (int u = 0; u < V; ++u) {
    du[u] = 0;
#pragma unroll
    for (int k = 0; k < VB; ++k)
      if ((u >> k) & 1) du[u] += step(k);
  }
  int il = 0;
  int64_t al = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k)
    if ((lane >> k) & 1) {
      il += step(VB + k);
      al += int64_t(1) << e[VB + k];
    }
  for (int s = 0; s < (32 >> VB); ++s) {
    int is = il;
    int64_t ah = 0;
#pragma unroll
    for (int k = 0; k < 5 - VB; ++k)
      if ((s >> k) & 1) {
        is += step(VB + 5 + k);
        ah += int64_t(1) << e[VB + 5 + k];
      }
    float re[V], im[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      re[u] = t[is + du[u]];
      im[u] = t[cs + is + du[u]];
    }
    store_run<V>(C, plane, base + al + ah, re, im, split);
  }
}

// Store one 32 x 32 block of a result tile from shared memory (t[r * pitch + c] = Re,
// t[cs + r * pitch + c] = Im; row r is lane r's row, column c lane c's column) in the
// order of its addresses. When the block's offsets are linear in the bits of (r, c) with
// power-of-two weights -- every row and column extent of the offset maps a power of two,
// as in every network with extent-2 modes -- off(r, c) = off(0, 0) + sum of per-bit
// weights, and the ten weights sorted ascending give the block's elements in address
// order. Each lane then writes V consecutive addresses with one vector store per plane
// (V up to 4 FP32 or 8 BF16 values, 16 bytes, as far as the smallest weights are 1, 2, 4,
// ... and the block is aligned), and a warp store covers 32 V consecutive elements when
// the following weights continue the sequence (interleaved row/column layouts included).
// Otherwise (ragged block, other extents) it falls back to one row per store. ro / co:
// this lane's row / column offset; row_ok / col_ok: in range.
// The address order of a 32 x 32 block: the ten bit weights (log2; bits 0-4 of the row,
// 5-9 of the column index) sorted ascending, with the bit each comes from; ok when the
// block's offsets are linear in those bits with power-of-two weights. ro_rel / co_rel: this
// lane's row / column offset relative to the block's first row / column.
struct BlockOrder {
  int e[10], src[10];
  bool ok;
};
static_assert(sizeof(BlockOrder) <= 128, "a fold warp's block order slot");
__device__ __forceinline__ BlockOrder block_order(int64_t ro_rel, int64_t co_rel, bool in_range, int lane) {
  BlockOrder o;
  bool lin = in_range;
  int64_t pr = 0, pc = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int64_t wr = __shfl_sync(0xffffffffu, ro_rel, 1 << i);
    const int64_t wc = __shfl_sync(0xffffffffu, co_rel, 1 << i);
    o.e[i] = (wr > 0 && (wr & (wr - 1)) == 0) ? 63 - __clzll(wr) : -1;
    o.e[5 + i] = (wc > 0 && (wc & (wc - 1)) == 0) ? 63 - __clzll(wc) : -1;
    lin = lin && o.e[i] >= 0 && o.e[5 + i] >= 0;
    pr += ((lane >> i) & 1) * wr;
    pc += ((lane >> i) & 1) * wc;
  }
  lin = lin && pr == ro_rel && pc == co_rel;
  o.ok = __all_sync(0xffffffffu, lin);
#pragma unroll
  for (int i = 0; i < 10; ++i) o.src[i] = i;
  if (o.ok) {
#pragma unroll
    for (int i = 1; i < 10; ++i)
#pragma unroll
      for (int j = i; j > 0; --j)
        if (o.e[j] < o.e[j - 1]) {
          const int te = o.e[j];
          o.e[j] = o.e[j - 1];
          o.e[j - 1] = te;
          const int ts = o.src[j];
          o.src[j] = o.src[j - 1];
          o.src[j - 1] = ts;
        }
  }
  return o;
}

// The address-ordered stores of a block whose order is `o` (o.ok) and whose first element
// is at `base`: each lane writes V consecutive addresses with one vector store per plane
// (V as far as the smallest weights are 1, 2, 4, ... and base and the plane size are
// V-aligned; 16 bytes at most).
__device__ __forceinline__ void store_ordered(float* C, int64_t plane, int split, const float* t, int pitch, int cs,
                                              int64_t base, const BlockOrder& o, int lane) {
  int vb = 0;
  while (vb < (split ? 3 : 2) && o.e[vb] == vb) ++vb;
  while (vb > 0 && ((base | plane) & ((int64_t(1) << vb) - 1)) != 0) --vb;
  if (vb == 3) store_sorted<3>(C, plane, split, t, pitch, cs, base, o.e, o.src, lane);
  else if (vb == 2) store_sorted<2>(C, plane, split, t, pitch, cs, base, o.e, o.src, lane);
  else if (vb == 1) store_sorted<1>(C, plane, split, t, pitch, cs, base, o.e, o.src, lane);
  else store_sorted<0>(C, plane, split, t, pitch, cs, base, o.e, o.src, lane);
}

// Store one 32 x 32 block of a result tile from shared memory (t[r * pitch + c] = Re,
// t[cs + r * pitch + c] = Im; row r is lane r's row, column c lane c's column) in the
// order of its addresses. When the block's offsets are linear in the bits of (r, c) with
// power-of-two weights -- every row and column extent of the offset maps a power of two,
// as in every network with extent-2 modes -- off(r, c) = off(0, 0) + sum of per-bit
// weights, and the ten weights sorted ascending give the block's elements in address
// order (block_order); a warp store then covers 32 V consecutive elements when the
// following weights continue the sequence (interleaved row/column layouts included).
// Otherwise (ragged block, other extents) it falls back to one row per store. ro / co:
// this lane's row / column offset; row_ok / col_ok: in range.
__device__ __forceinline__ void store_block(float* C, int64_t plane, int split, const float* t, int pitch,
                                            int cs, int64_t ro, int64_t co, bool row_ok, bool col_ok, int lane) {
  const int64_t ro0 = __shfl_sync(0xffffffffu, ro, 0), co0 = __shfl_sync(0xffffffffu, co, 0);
  const BlockOrder o = block_order(ro - ro0, co - co0, row_ok && col_ok, lane);
  if (o.ok) {
    store_ordered(C, plane, split, t, pitch, cs, ro0 + co0, o, lane);
    return;
  }
  for (int r = 0; r < 32; ++r) {
    const int64_t ro_r = __shfl_sync(0xffffffffu, ro, r);
    const bool ok_r = __shfl_sync(0xffffffffu, row_ok ? 1 : 0, r) != 0;
    if (ok_r && col_ok) store_cplx(C, plane, ro_r + co, t[r * pitch + lane], t[cs + r * pitch + lane], split);
  }
}

template <int SPLIT>
__global__ void __launch_bounds__(NTHREADS, 1)
    contract_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       StepArgs a, int64_t t_first, int* err) {
  using G = Cfg<SPLIT>;
  constexpr int STAGES = G::STAGES, BK = G::BK, ROWB = G::ROWB;
  constexpr int TILE_A = G::TILE_A, TILE_B = G::TILE_B, STAGE = G::STAGE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* lo_base = smem + STAGES * STAGE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(lo_base + G::LO * STAGE);
  uint64_t* full = bars;                     // [STAGES]
  uint64_t* empty = bars + STAGES;           // [STAGES]
  uint64_t* conv_full = bars + 2 * STAGES;   // [2]
  uint64_t* lo_empty = conv_full + 2;        // [2]
  uint64_t* acc_full = lo_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped raster over output tiles for L2 reuse of A and B tiles
  const int64_t tiles_m = (a.m + BM - 1) / BM, tiles_n = (a.n + BN - 1) / BN;
  const int64_t t = t_first + blockIdx.x;  // this launch's tiles start at t_first
  const int64_t per_group = GROUP_M * tiles_n;
  const int64_t first_m = (t / per_group) * GROUP_M;
  const int64_t gm = tiles_m - first_m < GROUP_M ? tiles_m - first_m : GROUP_M;
  const int64_t tm = first_m + (t % per_group) % gm, tn = (t % per_group) / gm;
  const int m0 = static_cast<int>(tm * BM), n0 = static_cast<int>(tn * BN);
  const int b = blockIdx.y;
  const int num_kb = static_cast<int>((a.k + BK - 1) / BK);
  const int pa = a.a_bstride ? 2 * b : 0, pb = a.b_bstride ? 2 * b : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&conv_full[i], 128);
      mbar_init(&lo_empty[i], 1);
    }
    mbar_init(acc_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(TMEM_COLS));
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
        tma_load_3d(st + TILE_A, &tmA, &full[s], k0, m0, pa + 1);
        tma_load_3d(st + 2 * TILE_A, &tmB, &full[s], k0, n0, pb);
        tma_load_3d(st + 2 * TILE_A + TILE_B, &tmB, &full[s], k0, n0, pb + 1);
        issued = kb + 1;
      }
      // drain: every stage's last issued load has landed before the CTA can exit
      for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
        if (!mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1)) atomicExch(err, 2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(BM, BN);
      const uint32_t d_rr = tmem, d_ii = tmem + 128, d_x = tmem + 256;
      for (int kb = 0; kb < num_kb; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait(&full[s], ph)) {
          atomicExch(err, 3);
          break;
        }
        if (SPLIT == 3 && !mbar_wait(&conv_full[kb & 1], (kb >> 1) & 1)) {
          atomicExch(err, 4);
          break;
        }
        fence_after();
        const uint32_t st = su32(smem + s * STAGE);
        const uint32_t lo = su32(lo_base + (kb & 1) * STAGE);
#pragma unroll
        for (int j = 0; j < BK / 8; ++j) {
          const uint32_t acc = (kb > 0 || j > 0) ? 1u : 0u;
          const uint64_t ar = smem_desc<ROWB>(st + j * 32), ai = smem_desc<ROWB>(st + TILE_A + j * 32);
          const uint64_t br = smem_desc<ROWB>(st + 2 * TILE_A + j * 32);
          const uint64_t bi = smem_desc<ROWB>(st + 2 * TILE_A + TILE_B + j * 32);
          mma_tf32(d_rr, ar, br, idesc, acc);
          mma_tf32(d_ii, ai, bi, idesc, acc);
          mma_tf32(d_x, ar, bi, idesc, acc);
          mma_tf32(d_x, ai, br, idesc, 1u);
          if (SPLIT == 3) {
            const uint64_t arl = smem_desc<ROWB>(lo + j * 32), ail = smem_desc<ROWB>(lo + TILE_A + j * 32);
            const uint64_t brl = smem_desc<ROWB>(lo + 2 * TILE_A + j * 32);
            const uint64_t bil = smem_desc<ROWB>(lo + 2 * TILE_A + TILE_B + j * 32);
            mma_tf32(d_rr, arl, br, idesc, 1u);
            mma_tf32(d_rr, ar, brl, idesc, 1u);
            mma_tf32(d_ii, ail, bi, idesc, 1u);
            mma_tf32(d_ii, ai, bil, idesc, 1u);
            mma_tf32(d_x, arl, bi, idesc, 1u);
            mma_tf32(d_x, ar, bil, idesc, 1u);
            mma_tf32(d_x, ail, br, idesc, 1u);
            mma_tf32(d_x, ai, brl, idesc, 1u);
          }
        }
        mma_commit(&empty[s]);
        if (SPLIT == 3) mma_commit(&lo_empty[kb & 1]);
      }
      mma_commit(acc_full);  // also on error: lets the epilogue see in-flight MMAs retire
    }
  } else {
    const int et = threadIdx.x - 64;  // 0..127
    if (SPLIT == 3) {
      for (int kb = 0; kb < num_kb; ++kb) {
        const int s = kb % STAGES;
        if (!mbar_wait(&full[s], (kb / STAGES) & 1) || !mbar_wait(&lo_empty[kb & 1], ((kb >> 1) & 1) ^ 1)) {
          atomicExch(err, 5);
          break;
        }
        float4* src = reinterpret_cast<float4*>(smem + s * STAGE);
        float4* dst = reinterpret_cast<float4*>(lo_base + (kb & 1) * STAGE);
#pragma unroll 4
        for (int i = et; i < STAGE / 16; i += 128) {
          const float4 v = src[i];
          float4 h, l;
          h.x = tf32_trunc(v.x);
          h.y = tf32_trunc(v.y);
          h.z = tf32_trunc(v.z);
          h.w = tf32_trunc(v.w);
          l.x = v.x - h.x;
          l.y = v.y - h.y;
          l.z = v.z - h.z;
          l.w = v.w - h.w;
          src[i] = h;
          dst[i] = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&conv_full[kb & 1]);
      }
    }
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
    for (int c = 0; c < BN / 32; ++c) {
      float rr[32], ii[32], xx[32];
      tmem_ld32(tmem + lane_base + c * 32, rr);
      tmem_ld32(tmem + lane_base + 128 + c * 32, ii);
      tmem_ld32(tmem + lane_base + 256 + c * 32, xx);
      const int64_t nb0 = static_cast<int64_t>(n0) + c * 32;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        tr[lane * 33 + j] = rr[j] - ii[j];
        tr[32 * 33 + lane * 33 + j] = xx[j];
      }
      __syncwarp();
      const int64_t n = nb0 + lane;
      const bool col_ok = ok && n < a.n;
      store_block(C, a.c_plane, kFmtPlanar, tr, 33, 32 * 33, ro, col_ok ? map_offset(a.cols, n) : 0, row_ok, col_ok,
                  lane);
      __syncwarp();
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
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
struct C3 {
  static constexpr int BK = 16, ROWB = 64, CK = 4;
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

__global__ void __launch_bounds__(C3::THREADS, 1)
    contract_tc3_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        StepArgs a, int64_t t_first, int* err) {
  constexpr int STAGES = C3::STAGES, BK = C3::BK, ROWB = C3::ROWB, CK = C3::CK;
  constexpr int TILE_A = C3::TILE_A, TILE_B = C3::TILE_B, STAGE = C3::STAGE;
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
  const int pa = a.a_bstride ? 2 * b : 0, pb = a.b_bstride ? 2 * b : 0;

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
        mbar_expect_tx(&full[s], C3::TMA_BYTES);
        uint8_t* st = smem + s * STAGE;
        const int k0 = kb * BK;
        tma_load_3d(st, &tmA, &full[s], k0, m0, pa);
        tma_load_3d(st + C3::OFF_AI, &tmA, &full[s], k0, m0, pa + 1);
        tma_load_3d(st + C3::OFF_BR, &tmB, &full[s], k0, n0, pb);
        tma_load_3d(st + C3::OFF_BI, &tmB, &full[s], k0, n0, pb + 1);
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
        if (!mbar_wait(acc_empty, (c & 1) ^ 1)) {
          atomicExch(err, 13);
          break;
        }
        fence_after();
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
#pragma unroll
          for (int j = 0; j < BK / 8; ++j) {
            const uint32_t acc = (kb > c * CK || j > 0) ? 1u : 0u;
            const uint64_t ar = smem_desc<ROWB>(st + j * 32), ai = smem_desc<ROWB>(st + C3::OFF_AI + j * 32);
            const uint64_t b_ri = smem_desc<ROWB>(st + C3::OFF_BR + j * 32);    // [B_re | B_im]
            const uint64_t b_nr = smem_desc<ROWB>(st + C3::OFF_BNEG + j * 32);  // [-B_im | B_re]
            const uint64_t arl = smem_desc<ROWB>(lo + j * 32), ail = smem_desc<ROWB>(lo + C3::OFF_AI + j * 32);
            const uint64_t bl_ri = smem_desc<ROWB>(lo + C3::OFF_BR + j * 32);
            const uint64_t bl_nr = smem_desc<ROWB>(lo + C3::OFF_BNEG + j * 32);
            // hi.hi products into the main accumulators (Re | Im); the small cross terms into
            // their own, so the main sums take only two truncating additions per 8 terms
            mma_tf32(d_hi, ar, b_ri, idesc, acc);
            mma_tf32(d_hi, ai, b_nr, idesc, 1u);
            // the cross-term accumulator runs over all of k (it is ~2^-11 of the result,
            // so its own truncation is negligible) and is read once, after the last chunk
            mma_tf32(d_lo, arl, b_ri, idesc, (kb > 0 || j > 0) ? 1u : 0u);
            mma_tf32(d_lo, ail, b_nr, idesc, 1u);
            mma_tf32(d_lo, ar, bl_ri, idesc, 1u);
            mma_tf32(d_lo, ai, bl_nr, idesc, 1u);
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
        constexpr int NA = 2 * TILE_A / 16;  // float4s of A_re, A_im
#pragma unroll 4
        for (int i = et; i < C3::TMA_BYTES / 16; i += 256) {
          const int f = i < NA ? i : i + TILE_B / 16;  // skip the -B_im slot
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
          if (f >= C3::OFF_BI / 16) {
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
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
      const int64_t nb0 = static_cast<int64_t>(n0) + half * 64 + cb * 32;
      if (rows_unit) {
        if (row_ok) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int64_t n = nb0 + j;
            if (n < a.n) {
              const int64_t off = ro + map_offset(a.cols, n);
              C[off] = run_re[cb * 32 + j];
              C[a.c_plane + off] = run_im[cb * 32 + j];
            }
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          tr[lane * 33 + j] = run_re[cb * 32 + j];
          tr[32 * 33 + lane * 33 + j] = run_im[cb * 32 + j];
        }
        __syncwarp();
        const int64_t n = nb0 + lane;
        const bool col_ok = ok && n < a.n;
        const int64_t co = col_ok ? map_offset(a.cols, n) : 0;
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
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C3::COLS));
  }
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
// waves of resident CTAs (or CTA pairs) per launch of the one-tile-per-CTA kernels, which
// launch a deep step in bands of tiles (0: one launch for the step)
constexpr int kBandWaves = 8;
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

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 3-D map over one operand: (k, rows, plane), plane = 2*batch + {re, im}; box BK x rows.
bool make_map(CUtensorMap* map, const float* base, int64_t rows, int64_t k, int64_t planes, int64_t plane_elems,
              int box_rows, int bk) {
  auto enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(k), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(planes)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(k * 4), static_cast<cuuint64_t>(plane_elems * 4)};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(bk), static_cast<cuuint32_t>(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapSwizzle sw = bk * 4 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
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

// Tiles per batch entry in one launch of a one-tile-per-CTA kernel (one CTA per SM by its
// shared memory): about kBandWaves waves of the SMs, for the reason given at
// pair_band_tiles.
int64_t sm_band_tiles(int64_t tiles, int32_t nb) {
  static const int sms = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
      n = 0;
    return n;
  }();
  if (kBandWaves <= 0 || sms <= 0 || nb <= 0) return tiles;
  const int64_t want = (int64_t(sms) * kBandWaves + nb - 1) / nb;
  return want < tiles ? want : tiles;
}

// Launch kern over `tiles` tiles x nb batch entries in bands of sm_band_tiles.
template <typename Kern, typename... Args>
cudaError_t launch_bands(Kern kern, int64_t tiles, int32_t nb, int threads, int smem, cudaStream_t st,
                         const CUtensorMap& ta, const CUtensorMap& tb, const StepArgs& a, int* err) {
  const int64_t per = sm_band_tiles(tiles, nb);
  for (int64_t t0 = 0; t0 < tiles; t0 += per) {
    const int64_t cnt = tiles - t0 < per ? tiles - t0 : per;
    kern<<<dim3(static_cast<unsigned>(cnt), static_cast<unsigned>(nb)), threads, smem, st>>>(ta, tb, a, t0, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
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

template <int SPLIT>
cudaError_t launch_split(const StepArgs& a, int32_t nb, int* err, cudaStream_t st) {
  static const cudaError_t configured =
      cudaFuncSetAttribute(contract_tc_kernel<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<SPLIT>::SMEM);
  if (configured != cudaSuccess) return configured;
  CUtensorMap ta, tb;
  const int64_t pa = a.a_bstride ? 2 * static_cast<int64_t>(nb) : 2;
  const int64_t pb = a.b_bstride ? 2 * static_cast<int64_t>(nb) : 2;
  constexpr int bk = Cfg<SPLIT>::BK;
  if (!make_map(&ta, a.A, a.m, a.k, pa, a.a_plane, BM, bk) || !make_map(&tb, a.B, a.n, a.k, pb, a.b_plane, BN, bk))
    return cudaErrorInvalidValue;
  const int64_t tiles = ((a.m + BM - 1) / BM) * ((a.n + BN - 1) / BN);
  return launch_bands(contract_tc_kernel<SPLIT>, tiles, nb, NTHREADS, Cfg<SPLIT>::SMEM, st, ta, tb, a, err);
}

cudaError_t launch_tc3(const StepArgs& a, int32_t nb, int* err, cudaStream_t st) {
  static const cudaError_t configured =
      cudaFuncSetAttribute(contract_tc3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, C3::SMEM);
  if (configured != cudaSuccess) return configured;
  CUtensorMap ta, tb;
  const int64_t pa = a.a_bstride ? 2 * static_cast<int64_t>(nb) : 2;
  const int64_t pb = a.b_bstride ? 2 * static_cast<int64_t>(nb) : 2;
  if (!make_map(&ta, a.A, a.m, a.k, pa, a.a_plane, BM, C3::BK) ||
      !make_map(&tb, a.B, a.n, a.k, pb, a.b_plane, BN, C3::BK))
    return cudaErrorInvalidValue;
  const int64_t tiles = ((a.m + BM - 1) / BM) * ((a.n + BN - 1) / BN);
  return launch_bands(contract_tc3_kernel, tiles, nb, C3::THREADS, C3::SMEM, st, ta, tb, a, err);
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
    cudaError_t e = cudaFuncSetAttribute(contract_tcb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CB::SMEM);
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
  return launch_bands(contract_tcb_kernel, tiles, nb, CB::THREADS, CB::SMEM, st, ta, tb, a, err);
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

int64_t tc_launches(int64_t m, int64_t n, int64_t k, int32_t nb, int32_t prec, bool pairs) {
  if (prec == TN_C64_BF16X3) {
    if (k <= CBP::MAX_K) return 1;  // persistent kernels
    if (pairs && m >= 2 * BM) {
      if (k <= kPairsPersistentMaxK) return 1;
      const int64_t pair_tiles = ((m + 2 * BM - 1) / (2 * BM)) * ((n + BN - 1) / BN);
      const int64_t per = pair_band_tiles(pair_tiles, nb);
      return (pair_tiles + per - 1) / per;
    }
  }
  const int64_t tiles = ((m + BM - 1) / BM) * ((n + BN - 1) / BN);
  const int64_t per = sm_band_tiles(tiles, nb);
  return (tiles + per - 1) / per;
}

cudaError_t launch_contract_tc(const StepArgs& a, int32_t nb, int32_t prec, bool cplx, int* err,
                               cudaStream_t st, bool pairs) {
  if (!cplx || a.recs) return cudaErrorNotSupported;
  if (prec == kPrecBF16x3M) return launch_tcb3m(a, nb, err, st);
  if (prec == TN_C64_TF32) return launch_split<1>(a, nb, err, st);
  if (prec == TN_C64_3XTF32) return launch_tc3(a, nb, err, st);
  if (prec == TN_C64_BF16X3) return launch_tcb(a, nb, err, st, pairs);
  return cudaErrorNotSupported;
}

}  // namespace tn
