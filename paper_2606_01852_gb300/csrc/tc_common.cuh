// Shared pieces of the tcgen05 GEMM kernels (device side and their launch helpers):
// TMA loads, shared-memory and instruction descriptors, MMA issue and tensor-memory
// loads, the address-ordered epilogue stores, tensor-map encoding and banded launches.
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "mbarrier.cuh"
#include "scale.cuh"
#include "split_bf16.cuh"

namespace tn {
namespace {

constexpr int BM = 128, BN = 128;
constexpr int GROUP_M = 16;                                 // raster: tiles grouped along M
// waves of resident CTAs (or CTA pairs) per launch of the one-tile-per-CTA kernels, which
// launch a deep step in bands of tiles (0: one launch for the step)
constexpr int kBandWaves = 8;

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

// V consecutive FP32 values (V = 1, 2, 4) of a real result at element `off`.
template <int V>
__device__ __forceinline__ void store_run_real(float* C, int64_t off, const float* v) {
  if constexpr (V == 1) {
    C[off] = v[0];
  } else if constexpr (V == 2) {
    *reinterpret_cast<float2*>(C + off) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int h = 0; h < V; h += 4)
      *reinterpret_cast<float4*>(C + off + h) = make_float4(v[h], v[h + 1], v[h + 2], v[h + 3]);
  }
}

// The address-ordered stores of one block, lanes taking V = 2^VB consecutive addresses.
// e[k], src[k]: the k-th smallest bit weight (log2) and which bit of r (0-4) or c (5-9)
// carries it; the VB smallest weights are 1, 2, ..., 2^(VB-1).
// REAL: a real result, t holds the one plane and C is FP32.
template <int VB, bool REAL = false>
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
    if constexpr (REAL) {
      float v[V];
#pragma unroll
      for (int u = 0; u < V; ++u) v[u] = t[is + du[u]];
      store_run_real<V>(C, base + al + ah, v);
    } else {
      float re[V], im[V];
#pragma unroll
      for (int u = 0; u < V; ++u) {
        re[u] = t[is + du[u]];
        im[u] = t[cs + is + du[u]];
      }
      store_run<V>(C, plane, base + al + ah, re, im, split);
    }
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
template <bool REAL = false>
__device__ __forceinline__ void store_ordered(float* C, int64_t plane, int split, const float* t, int pitch, int cs,
                                              int64_t base, const BlockOrder& o, int lane) {
  int vb = 0;
  while (vb < (!REAL && split ? 3 : 2) && o.e[vb] == vb) ++vb;
  while (vb > 0 && ((base | plane) & ((int64_t(1) << vb) - 1)) != 0) --vb;
  if constexpr (!REAL) {
    if (vb == 3) {
      store_sorted<3>(C, plane, split, t, pitch, cs, base, o.e, o.src, lane);
      return;
    }
  }
  if (vb == 2) store_sorted<2, REAL>(C, plane, split, t, pitch, cs, base, o.e, o.src, lane);
  else if (vb == 1) store_sorted<1, REAL>(C, plane, split, t, pitch, cs, base, o.e, o.src, lane);
  else store_sorted<0, REAL>(C, plane, split, t, pitch, cs, base, o.e, o.src, lane);
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
// this lane's row / column offset; row_ok / col_ok: in range. REAL: a real FP32 result
// (one plane in t; plane, split and cs unused).
template <bool REAL = false>
__device__ __forceinline__ void store_block(float* C, int64_t plane, int split, const float* t, int pitch,
                                            int cs, int64_t ro, int64_t co, bool row_ok, bool col_ok, int lane) {
  const int64_t ro0 = __shfl_sync(0xffffffffu, ro, 0), co0 = __shfl_sync(0xffffffffu, co, 0);
  const BlockOrder o = block_order(ro - ro0, co - co0, row_ok && col_ok, lane);
  if (o.ok) {
    store_ordered<REAL>(C, plane, split, t, pitch, cs, ro0 + co0, o, lane);
    return;
  }
  for (int r = 0; r < 32; ++r) {
    const int64_t ro_r = __shfl_sync(0xffffffffu, ro, r);
    const bool ok_r = __shfl_sync(0xffffffffu, row_ok ? 1 : 0, r) != 0;
    if (ok_r && col_ok) {
      if constexpr (REAL) C[ro_r + co] = t[r * pitch + lane];
      else store_cplx(C, plane, ro_r + co, t[r * pitch + lane], t[cs + r * pitch + lane], split);
    }
  }
}

// Exponent scaling on a tensor-core step. The operands are read as stored, so their
// scales 2^-e_A and 2^-e_B multiply the accumulated result instead of each operand: the
// same values as scaling on load, as a power of two commutes with every rounding in
// between (the operands' TF32 truncation or hi/lo split, the products and the sums) as long
// as no value leaves FP32's normal range. Stored intermediates are sums of products of renormalised
// operands (a small multiple of k in magnitude), so their unscaled products stay far inside
// it; leaves are read as given, so a leaf's entries times its partner's must stay inside it.
struct TcScale {
  float sa, sb;
};
__device__ __forceinline__ TcScale tc_scale(const StepArgs& a, int b) {
  TcScale s{1.f, 1.f};
  if (a.recs) {
    s.sa = pow2_neg(scale_exp(a.recs + a.rec_a + (a.a_bstride ? b : 0)));
    s.sb = pow2_neg(scale_exp(a.recs + a.rec_b + (a.b_bstride ? b : 0)));
  }
  return s;
}
// After a warp's stores (all 32 lanes): the warp's largest exponent into C's record, and
// from one thread per batch entry C's log scale (its operands' log scales and exponents).
__device__ __forceinline__ void tc_scale_finish(const StepArgs& a, int b, int lmax, bool log_thread) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  ScaleRec* rc = a.recs + a.rec_c + (a.c_bstride ? b : 0);
  if ((threadIdx.x & 31) == 0) atomicMax(&rc->emax, lmax);
  if (log_thread) {
    const ScaleRec* ra = a.recs + a.rec_a + (a.a_bstride ? b : 0);
    const ScaleRec* rb = a.recs + a.rec_b + (a.b_bstride ? b : 0);
    rc->log2 = ra->log2 + rb->log2 + scale_exp(ra) + scale_exp(rb);
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

}  // namespace
}  // namespace tn
