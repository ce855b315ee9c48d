// CUDA-core kernels of the contraction engine (sm_103a):
//   stage_leaves      : leaf staging and slicing (declared order -> planned order,
//                       sliced labels fixed per batch entry, complex64 -> planar fp32
//                       or, for operands of BF16x3 steps, split BF16)
//   contract_simt     : any pairwise step C[b] = A[b](m x k) . B[b](n x k)^T, FP32 FMA,
//                       written through the separable row/column offset maps
//   contract_stream   : big x small steps (n*k tiny), one pass over the big operand
//   accumulate_root   : compensated FP64 sum of the root over the slice batch; the last
//                       pass writes the FP64 result and its log scale
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "kernels.h"
#include "mbarrier.cuh"
#include "scale.cuh"
#include "split_bf16.cuh"
#include "staging.cuh"

namespace tn {

// ---------------------------------------------------------------------------------
// leaf staging (a4)

__global__ void stage_leaves_kernel(const LeafDesc* __restrict__ descs, char* __restrict__ ws,
                                    int64_t slice_begin, int32_t nb, int32_t only_batched,
                                    int32_t is_complex, ScaleRec* recs, const int32_t* rec_index,
                                    int32_t rec_batched_base) {
  const LeafDesc& d = descs[blockIdx.x];
  if (d.tiled || (only_batched && !d.batched)) return;
  const int32_t copies = d.batched ? nb : 1;
  const int64_t total = d.size * copies;
  int lmax = -127;
  for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
    const int64_t b = i / d.size;
    int64_t e = i - b * d.size;
    int64_t src = 0;
    for (int r = d.rank - 1; r >= 0; --r) {
      const uint32_t x = d.ext[r];
      src += (e % x) * d.sstride[r];
      e /= x;
    }
    const int64_t sid = slice_begin + b;
    for (int q = 0; q < d.n_sl; ++q) src += ((sid / d.sl_div[q]) % d.sl_ext[q]) * d.sl_stride[q];
    const int64_t el = i - b * d.size;
    if (is_complex) {
      const float2 v = reinterpret_cast<const float2*>(d.src)[src];
      float* dst = reinterpret_cast<float*>(ws + d.dst) + b * cplx_floats(d.split) * d.size;
      store_cplx(dst, d.size, el, v.x, v.y, d.split);
      if (recs) lmax = max(lmax, exp_of(fmaxf(fabsf(v.x), fabsf(v.y))));
    } else {
      const float v = reinterpret_cast<const float*>(d.src)[src];
      float* dst = reinterpret_cast<float*>(ws + d.dst) + b * d.size;
      dst[el] = v;
      if (recs) lmax = max(lmax, exp_of(fabsf(v)));
    }
  }
  if (recs) {
    // one block per leaf: the leaf's copies share a record per batch entry; a leaf
    // copy is tiny, so take the block-wide max over all copies (same for every b).
    __shared__ int smax;
    if (threadIdx.x == 0) smax = -127;
    __syncthreads();
    atomicMax(&smax, lmax);
    __syncthreads();
    for (int q = threadIdx.x; q < copies; q += blockDim.x) {
      ScaleRec* r = recs + rec_index[blockIdx.x] + (d.batched ? q : 0);
      r->emax = smax;
      r->log2 = 0;
    }
  }
}

// Tiled permutation of one large leaf (K-PERM): one CTA per (rest index, 32 x 32 tile of
// output-group index x input-group index), blockIdx.y = batch copy. Loads run along the
// input group (its fastest position is the declared order's innermost, so a warp reads
// contiguous source addresses; two complex64 elements per 16-byte load where the stride
// is 1 and the extent even), the tile goes through shared memory, and stores run along
// the output group (contiguous in the staged copy: four FP32 values per 16-byte store and
// plane, or eight BF16 values per plane in the split form). When the declared innermost
// position is itself in the output group, loads run along the output group instead.
template <bool CPLX>
__global__ void __launch_bounds__(256, 5) stage_leaf_tiled_kernel(const LeafDesc* __restrict__ descs, int32_t leaf,
                                                               char* __restrict__ ws, int64_t slice_begin,
                                                               ScaleRec* recs, const int32_t* rec_index) {
  constexpr int TT = kTilesInFlight;  // tiles per CTA iteration (loads of all before any store)
  const LeafDesc& d = descs[leaf];
  __shared__ float tre[TT][32][33];
  __shared__ float tim[TT][CPLX ? 32 : 1][33];
  // per-tile offset tables (table_entry): rebuilt only when a slot's chunk indices change
  // (never, when each group fits one 32-wide chunk)
  __shared__ int64_t s_isrc[TT][32], s_osrc[TT][32], s_irow[TT][32];
  __shared__ TileCursor s_cur[TT];
  __shared__ int s_rebuild[TT];
  __shared__ int64_t s_built[TT][2];
  __shared__ int s_nt;
  const int tid = threadIdx.x;
  const int b = blockIdx.y;
  const int64_t tiles = d.Pr * ((d.Po + 31) / 32) * ((d.Pi + 31) / 32);
  const int64_t blk0 = int64_t(blockIdx.x) * kTilesPerCta;
  const int64_t blk1 = blk0 + kTilesPerCta < tiles ? blk0 + kTilesPerCta : tiles;
  const int64_t Pi = d.Pi, Po = d.Po;
  const bool vec = CPLX && d.vec_load && (reinterpret_cast<uintptr_t>(d.src) & 15) == 0;
  const int64_t np = CPLX ? cplx_floats(d.split) : 1;
  float* base = reinterpret_cast<float*>(ws + d.dst) + int64_t(b) * np * d.size;
  if (tid < TT) s_built[tid][0] = s_built[tid][1] = -1;
  int lmax = -127;
  for (int64_t blk = blk0; blk < blk1; blk += TT) {
    __syncthreads();  // slot state of the previous iteration is no longer read
    if (tid == 0) s_nt = iteration_tiles(d, blk, blk0, blk1, slice_begin + b, s_cur, s_built, s_rebuild);
    __syncthreads();
    const int nt = s_nt;
    bool any = false;
    for (int u = 0; u < nt; ++u) any = any || s_rebuild[u];
    if (any) {
      const int u = tid >> 5, r = tid & 31;
      if (u < nt && s_rebuild[u])
        table_entry(d, s_cur[u].co * 32, s_cur[u].ci * 32, r, s_isrc[u][r], s_osrc[u][r], s_irow[u][r]);
      __syncthreads();
    }
    // ---- load the tiles: tre[u][ti][to] = element (output-group go0 + to, input-group gi0 + ti)
    if (vec) {
      const float4* src4 = reinterpret_cast<const float4*>(d.src);
      const int ti = 2 * (tid & 15);
      float4 v[TT][2];
#pragma unroll
      for (int u = 0; u < TT; ++u)
#pragma unroll
        for (int rep = 0; rep < 2; ++rep) {
          const int to = (tid >> 4) + 16 * rep;
          const int64_t gi = s_cur[u].ci * 32 + ti, go = s_cur[u].co * 32 + to;
          v[u][rep] = make_float4(0.f, 0.f, 0.f, 0.f);
          // elements gi and gi + 1 differ in the fastest position only (gi even, extent even)
          if (u < nt && gi < Pi && go < Po)
            v[u][rep] = __ldg(src4 + ((s_cur[u].src0 + s_isrc[u][ti] + s_osrc[u][to]) >> 1));
        }
#pragma unroll
      for (int u = 0; u < TT; ++u)
#pragma unroll
        for (int rep = 0; rep < 2; ++rep) {
          const int to = (tid >> 4) + 16 * rep;
          const float4 w = v[u][rep];
          tre[u][ti][to] = w.x;
          tim[u][ti][to] = w.y;
          tre[u][ti + 1][to] = w.z;
          tim[u][ti + 1][to] = w.w;
          lmax = max(lmax, exp_of(fmaxf(fmaxf(fabsf(w.x), fabsf(w.y)), fmaxf(fabsf(w.z), fabsf(w.w)))));
        }
    } else {
      // one element per load; lanes along the input group, or along the output group when
      // the declared innermost position is there
      for (int u = 0; u < nt; ++u)
        for (int rep = 0; rep < 4; ++rep) {
          const int a0 = tid & 31, a1 = (tid >> 5) + 8 * rep;
          const int ti = d.load_o ? a1 : a0, to = d.load_o ? a0 : a1;
          const int64_t gi = s_cur[u].ci * 32 + ti, go = s_cur[u].co * 32 + to;
          if (gi < Pi && go < Po) {
            const int64_t so = s_cur[u].src0 + s_isrc[u][ti] + s_osrc[u][to];
            if (CPLX) {
              const float2 w = __ldg(reinterpret_cast<const float2*>(d.src) + so);
              tre[u][ti][to] = w.x;
              tim[u][ti][to] = w.y;
              lmax = max(lmax, exp_of(fmaxf(fabsf(w.x), fabsf(w.y))));
            } else {
              const float w = __ldg(reinterpret_cast<const float*>(d.src) + so);
              tre[u][ti][to] = w;
              lmax = max(lmax, exp_of(fabsf(w)));
            }
          }
        }
    }
    __syncthreads();
    // ---- store: a row of a tile (fixed input-group index) is contiguous in the staged copy
    for (int u = 0; u < nt; ++u) {
      const int64_t go0 = s_cur[u].co * 32, gi0 = s_cur[u].ci * 32, dst0 = s_cur[u].dst0;
      if (CPLX && d.split) {
        // eight consecutive elements per thread and plane: 16-byte stores of BF16
        const int q = tid & 3, ti = tid >> 2;
        const int64_t gi = gi0 + ti;
        if (ti < 32 && gi < Pi) {
          const int64_t row = dst0 + s_irow[u][ti];
          const int to = 8 * q;
          if (go0 + to + 7 < Po && ((row + to) & 7) == 0 && (d.size & 7) == 0) {
            // planes in storage order: split form [rh | ih | rl | il], 3M form [rh | rl | ih | il | sh | sl]
            uint32_t pl[6][8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float vr = tre[u][ti][to + e], vi = tim[u][ti][to + e];
              __nv_bfloat16 rh, rl, ih, il, sh, sl;
              split_pair(vr, rh, rl);
              split_pair(vi, ih, il);
              split_pair(vr + vi, sh, sl);
              const bool m3 = d.split == kFmtSplit3M;
              pl[0][e] = __bfloat16_as_ushort(rh);
              pl[1][e] = __bfloat16_as_ushort(m3 ? rl : ih);
              pl[2][e] = __bfloat16_as_ushort(m3 ? ih : rl);
              pl[3][e] = __bfloat16_as_ushort(il);
              pl[4][e] = __bfloat16_as_ushort(sh);
              pl[5][e] = __bfloat16_as_ushort(sl);
            }
            uint16_t* S = reinterpret_cast<uint16_t*>(base) + row + to;
            auto pack = [](const uint32_t* x) {
              return make_uint4(x[0] | (x[1] << 16), x[2] | (x[3] << 16), x[4] | (x[5] << 16), x[6] | (x[7] << 16));
            };
            const int planes = d.split == kFmtSplit3M ? 6 : 4;
            for (int p = 0; p < planes; ++p) *reinterpret_cast<uint4*>(S + p * d.size) = pack(pl[p]);
          } else {
            for (int e = 0; e < 8; ++e)
              if (go0 + to + e < Po)
                store_cplx(base, d.size, row + to + e, tre[u][ti][to + e], tim[u][ti][to + e], d.split);
          }
        }
      } else {
        // four consecutive FP32 values per thread and plane: 16-byte stores
        const int q = tid & 7, ti = tid >> 3;
        const int64_t gi = gi0 + ti;
        if (gi < Pi) {
          const int64_t row = dst0 + s_irow[u][ti];
          const int to = 4 * q;
          if (go0 + to + 3 < Po && ((row + to) & 3) == 0 && (d.size & 3) == 0) {
            *reinterpret_cast<float4*>(base + row + to) =
                make_float4(tre[u][ti][to], tre[u][ti][to + 1], tre[u][ti][to + 2], tre[u][ti][to + 3]);
            if (CPLX)
              *reinterpret_cast<float4*>(base + d.size + row + to) =
                  make_float4(tim[u][ti][to], tim[u][ti][to + 1], tim[u][ti][to + 2], tim[u][ti][to + 3]);
          } else {
            for (int e = 0; e < 4; ++e)
              if (go0 + to + e < Po) {
                base[row + to + e] = tre[u][ti][to + e];
                if (CPLX) base[d.size + row + to + e] = tim[u][ti][to + e];
              }
          }
        }
      }
    }
  }
  if (recs) {
    // exponent record of this copy: the largest exponent over the tiles (the records
    // start at the atomicMax identity every pass)
    for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    ScaleRec* rec = recs + rec_index[leaf] + (d.batched ? b : 0);
    if ((tid & 31) == 0) atomicMax(&rec->emax, lmax);
    if (blockIdx.x == 0 && tid == 0) rec->log2 = 0;
  }
}

// Pipelined form of the tiled staging kernel (LeafDesc::fast: each group one 32-wide chunk,
// 16-byte loads, the CTA's 16 tiles spanning the rest index's fastest positions): the
// offset tables and the tiles' rest offsets are built once per CTA, and the loads of tile
// i + 1 are in flight while tile i is stored (two tile buffers, one barrier per tile).
template <int SPLIT>
__device__ __forceinline__ void store_tile_row(float* base, int64_t size, int64_t row, int tid, const float (*tre)[33],
                                               const float (*tim)[33]) {
  if (SPLIT) {
    const int q = tid & 3, ti = tid >> 2, to = 8 * q;
    if (ti >= 32) return;
    uint32_t pl[6][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float vr = tre[ti][to + e], vi = tim[ti][to + e];
      __nv_bfloat16 rh, rl, ih, il, sh, sl;
      split_pair(vr, rh, rl);
      split_pair(vi, ih, il);
      split_pair(vr + vi, sh, sl);
      pl[0][e] = __bfloat16_as_ushort(rh);
      pl[1][e] = __bfloat16_as_ushort(SPLIT == kFmtSplit3M ? rl : ih);
      pl[2][e] = __bfloat16_as_ushort(SPLIT == kFmtSplit3M ? ih : rl);
      pl[3][e] = __bfloat16_as_ushort(il);
      pl[4][e] = __bfloat16_as_ushort(sh);
      pl[5][e] = __bfloat16_as_ushort(sl);
    }
    uint16_t* S = reinterpret_cast<uint16_t*>(base) + row + to;
    constexpr int planes = SPLIT == kFmtSplit3M ? 6 : 4;
#pragma unroll
    for (int p = 0; p < planes; ++p)
      *reinterpret_cast<uint4*>(S + p * size) =
          make_uint4(pl[p][0] | (pl[p][1] << 16), pl[p][2] | (pl[p][3] << 16), pl[p][4] | (pl[p][5] << 16),
                     pl[p][6] | (pl[p][7] << 16));
  } else {
    const int q = tid & 7, ti = tid >> 3, to = 4 * q;
    *reinterpret_cast<float4*>(base + row + to) =
        make_float4(tre[ti][to], tre[ti][to + 1], tre[ti][to + 2], tre[ti][to + 3]);
    *reinterpret_cast<float4*>(base + size + row + to) =
        make_float4(tim[ti][to], tim[ti][to + 1], tim[ti][to + 2], tim[ti][to + 3]);
  }
}

template <int SPLIT>
__global__ void __launch_bounds__(256, 4) stage_leaf_fast_kernel(const LeafDesc* __restrict__ descs, int32_t leaf,
                                                                 char* __restrict__ ws, int64_t slice_begin,
                                                                 ScaleRec* recs, const int32_t* rec_index) {
  const LeafDesc& d = descs[leaf];
  __shared__ float tre[2][32][33], tim[2][32][33];
  __shared__ int64_t s_isrc[32], s_osrc[32], s_irow[32], s_lsrc[kTilesPerCta], s_ldst[kTilesPerCta];
  __shared__ int64_t s_hi[2];
  const int tid = threadIdx.x, b = blockIdx.y;
  if (tid < 32) {
    int64_t osrc, irow;
    table_entry(d, 0, 0, tid, s_isrc[tid], osrc, irow);
    s_osrc[tid] = osrc;
    s_irow[tid] = irow;
  } else if (tid < 32 + kTilesPerCta) {
    rest_lo_offsets(d, tid - 32, s_lsrc[tid - 32], s_ldst[tid - 32]);
  } else if (tid == 64) {
    rest_hi_offsets(d, blockIdx.x, slice_begin + b, s_hi[0], s_hi[1]);
  }
  __syncthreads();
  const int64_t hsrc = s_hi[0], hdst = s_hi[1];
  const float4* src4 = reinterpret_cast<const float4*>(d.src);
  float* base = reinterpret_cast<float*>(ws + d.dst) + int64_t(b) * cplx_floats(d.split) * d.size;
  const int ti = 2 * (tid & 15), to0 = tid >> 4;
  const int64_t sa = s_isrc[ti] + s_osrc[to0], sb = s_isrc[ti] + s_osrc[to0 + 16];
  int lmax = -127;
  float4 v0 = __ldg(src4 + ((hsrc + s_lsrc[0] + sa) >> 1)), v1 = __ldg(src4 + ((hsrc + s_lsrc[0] + sb) >> 1));
  for (int i = 0; i < kTilesPerCta; ++i) {
    float (*br)[33] = tre[i & 1];
    float (*bi)[33] = tim[i & 1];
    br[ti][to0] = v0.x;
    bi[ti][to0] = v0.y;
    br[ti + 1][to0] = v0.z;
    bi[ti + 1][to0] = v0.w;
    br[ti][to0 + 16] = v1.x;
    bi[ti][to0 + 16] = v1.y;
    br[ti + 1][to0 + 16] = v1.z;
    bi[ti + 1][to0 + 16] = v1.w;
    lmax = max(lmax, exp_of(fmaxf(fmaxf(fmaxf(fabsf(v0.x), fabsf(v0.y)), fmaxf(fabsf(v0.z), fabsf(v0.w))),
                                  fmaxf(fmaxf(fabsf(v1.x), fabsf(v1.y)), fmaxf(fabsf(v1.z), fabsf(v1.w))))));
    __syncthreads();  // tile i is in shared memory; the stores of tile i - 1 are done
    if (i + 1 < kTilesPerCta) {
      v0 = __ldg(src4 + ((hsrc + s_lsrc[i + 1] + sa) >> 1));
      v1 = __ldg(src4 + ((hsrc + s_lsrc[i + 1] + sb) >> 1));
    }
    const int rti = SPLIT ? (tid >> 2) : (tid >> 3);
    if (rti < 32) store_tile_row<SPLIT>(base, d.size, hdst + s_ldst[i] + s_irow[rti], tid, br, bi);
  }
  if (recs) {
    for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    ScaleRec* rec = recs + rec_index[leaf] + (d.batched ? b : 0);
    if ((tid & 31) == 0) atomicMax(&rec->emax, lmax);
    if (blockIdx.x == 0 && tid == 0) rec->log2 = 0;
  }
}

void launch_stage_leaves(const LeafDesc* descs, const LeafDesc* host_descs, int32_t n_leaves, char* ws,
                         int64_t slice_begin, int32_t nb, bool only_batched, bool is_complex, ScaleRec* recs,
                         const int32_t* rec_index, cudaStream_t st) {
  if (n_leaves <= 0) return;
  stage_leaves_kernel<<<n_leaves, 128, 0, st>>>(descs, ws, slice_begin, nb, only_batched ? 1 : 0,
                                                is_complex ? 1 : 0, recs, rec_index, 0);
  for (int32_t t = 0; t < n_leaves; ++t) {
    const LeafDesc& h = host_descs[t];
    if (!h.tiled || (only_batched && !h.batched)) continue;
    const int64_t tiles = h.Pr * ((h.Po + 31) / 32) * ((h.Pi + 31) / 32);
    const int64_t ctas = (tiles + kTilesPerCta - 1) / kTilesPerCta;
    dim3 grid(static_cast<unsigned>(ctas), static_cast<unsigned>(h.batched ? nb : 1));
    if (h.fast && (reinterpret_cast<uintptr_t>(h.src) & 15) == 0) {  // 16-byte loads need an aligned source
      if (h.split == kFmtSplit3M)
        stage_leaf_fast_kernel<kFmtSplit3M><<<grid, 256, 0, st>>>(descs, t, ws, slice_begin, recs, rec_index);
      else if (h.split == kFmtSplit)
        stage_leaf_fast_kernel<kFmtSplit><<<grid, 256, 0, st>>>(descs, t, ws, slice_begin, recs, rec_index);
      else
        stage_leaf_fast_kernel<kFmtPlanar><<<grid, 256, 0, st>>>(descs, t, ws, slice_begin, recs, rec_index);
      continue;
    }
    if (is_complex)
      stage_leaf_tiled_kernel<true><<<grid, 256, 0, st>>>(descs, t, ws, slice_begin, recs, rec_index);
    else
      stage_leaf_tiled_kernel<false><<<grid, 256, 0, st>>>(descs, t, ws, slice_begin, recs, rec_index);
  }
}

// ---------------------------------------------------------------------------------
// generic step kernel: 64 x 64 output tile, 16-deep k slices, 256 threads, 4 x 4
// outputs per thread (rows ty*4.., columns tx + 16j so a half-warp stores 16
// consecutive columns). MAXPLUS (real only): C = max_k (A + B), -inf padding.

template <bool CPLX, bool MAXPLUS = false>
__global__ void __launch_bounds__(256) contract_simt_kernel(StepArgs a) {
  static_assert(!(CPLX && MAXPLUS), "the max-plus semiring is real");
  const float kZero = MAXPLUS ? __int_as_float(0xff800000) : 0.f;  // the semiring's zero (-inf)
  constexpr int BM = 64, BN = 64, BK = 16, NP = CPLX ? 2 : 1;
  __shared__ float As[NP][BK][BM + 4];
  __shared__ float Bs[NP][BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t tiles_n = (a.n + BN - 1) / BN;
  const int64_t tile = blockIdx.x;
  const int64_t m0 = (tile / tiles_n) * BM, n0 = (tile % tiles_n) * BN;
  const int b = blockIdx.y;
  const float* A = a.A + b * a.a_bstride;
  const float* B = a.B + b * a.b_bstride;
  float* C = a.C + b * a.c_bstride;
  // this CTA's part of k (all of it unless the step is split, blockIdx.z = part)
  const int64_t kc = a.ksplit > 1 ? ((a.k + a.ksplit - 1) / a.ksplit + BK - 1) / BK * BK : a.k;
  const int64_t kbeg = blockIdx.z * kc, kend = kbeg + kc < a.k ? kbeg + kc : a.k;
  float sa = 1.f, sb = 1.f;
  if (a.recs) {
    const ScaleRec* ra = a.recs + a.rec_a + (a.a_bstride ? b : 0);
    const ScaleRec* rb = a.recs + a.rec_b + (a.b_bstride ? b : 0);
    sa = pow2_neg(scale_exp(ra));
    sb = pow2_neg(scale_exp(rb));
  }
  float accr[4][4], acci[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = kZero;

  const int lr = tid >> 2, lk = (tid & 3) * 4;  // loader: row lr, k lk..lk+3
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t kk = k0 + lk + q;
        const int64_t ra = m0 + lr, rb = n0 + lr;
        float va = kZero, vb = kZero;
        if (ra < a.m && kk < kend) va = A[p * a.a_plane + ra * a.k + kk] * sa;
        if (rb < a.n && kk < kend) vb = B[p * a.b_plane + rb * a.k + kk] * sb;
        As[p][lk + q][lr] = va;
        Bs[p][lk + q][lr] = vb;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float ar[4], br[4], ai[4], bi[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ar[i] = As[0][kk][ty * 4 + i];
        br[i] = Bs[0][kk][tx + 16 * i];
        if (CPLX) {
          ai[i] = As[1][kk][ty * 4 + i];
          bi[i] = Bs[1][kk][tx + 16 * i];
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (CPLX) {
            accr[i][j] = fmaf(ar[i], br[j], accr[i][j]);
            accr[i][j] = fmaf(-ai[i], bi[j], accr[i][j]);
            acci[i][j] = fmaf(ar[i], bi[j], acci[i][j]);
            acci[i][j] = fmaf(ai[i], br[j], acci[i][j]);
          } else if (MAXPLUS) {
            accr[i][j] = fmaxf(accr[i][j], ar[i] + br[j]);
          } else {
            accr[i][j] = fmaf(ar[i], br[j], accr[i][j]);
          }
        }
    }
    __syncthreads();
  }
  if (a.ksplit > 1) {
    // partial tile of this part of k, dense [part][b][plane][m][n]; combined and written
    // through the offset maps by simt_combine_kernel
    float* P0 = a.part + ((int64_t(blockIdx.z) * gridDim.y + b) * NP) * a.m * a.n;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t m = m0 + ty * 4 + i;
      if (m >= a.m) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t n = n0 + tx + 16 * j;
        if (n >= a.n) continue;
        P0[m * a.n + n] = accr[i][j];
        if (CPLX) P0[a.m * a.n + m * a.n + n] = acci[i][j];
      }
    }
    return;
  }
  // epilogue through the offset maps
  int64_t coff[4];
  bool cok[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t n = n0 + tx + 16 * j;
    cok[j] = n < a.n;
    coff[j] = cok[j] ? map_offset(a.cols, n) : 0;
  }
  int lmax = -127;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + ty * 4 + i;
    if (m >= a.m) continue;
    const int64_t ro = map_offset(a.rows, m);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!cok[j]) continue;
      if (CPLX) store_cplx(C, a.c_plane, ro + coff[j], accr[i][j], acci[i][j], a.c_split);
      else C[ro + coff[j]] = accr[i][j];
      if (a.recs) lmax = max(lmax, exp_of(CPLX ? fmaxf(fabsf(accr[i][j]), fabsf(acci[i][j]))
                                               : fabsf(accr[i][j])));
    }
  }
  if (a.recs) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    ScaleRec* rc = a.recs + a.rec_c + (a.c_bstride ? b : 0);
    if ((tid & 31) == 0) atomicMax(&rc->emax, lmax);
    if (tile == 0 && tid == 0) {
      const ScaleRec* ra = a.recs + a.rec_a + (a.a_bstride ? b : 0);
      const ScaleRec* rb = a.recs + a.rec_b + (a.b_bstride ? b : 0);
      rc->log2 = ra->log2 + rb->log2 + scale_exp(ra) + scale_exp(rb);
    }
  }
}

// ---------------------------------------------------------------------------------
// step chains: a run of tiny steps in one CTA. Each step's outputs are spread over the
// threads (thread = output element, batch entry by batch entry), each summed over k in
// order with the FMAs of contract_simt_kernel (the same bits); the CTA barrier between
// steps orders a step's stores, and its scale record, before the next step's loads.

template <bool CPLX, bool MAXPLUS>
__global__ void __launch_bounds__(512) contract_chain_kernel(const ChainStep* __restrict__ steps, int32_t n_steps,
                                                             int32_t nb, int32_t skip_unbatched) {
  static_assert(!(CPLX && MAXPLUS), "the max-plus semiring is real");
  static_assert(sizeof(ChainStep) % 4 == 0, "ChainStep copied as 32-bit words");
  constexpr int kWords = sizeof(ChainStep) / 4;
  const float kZero = MAXPLUS ? __int_as_float(0xff800000) : 0.f;
  // the step descriptors pass through shared memory, the next one fetched while the current
  // step runs (double buffer)
  __shared__ ChainStep cur[2];
  auto fetch = [&](int32_t i) {
    const int* src = reinterpret_cast<const int*>(steps + i);
    int* dst = reinterpret_cast<int*>(&cur[i & 1]);
    for (int w = threadIdx.x; w < kWords; w += blockDim.x) dst[w] = src[w];
  };
  if (n_steps > 0) fetch(0);
  __syncthreads();
  for (int32_t i = 0; i < n_steps; ++i) {
    if (i + 1 < n_steps) fetch(i + 1);  // the buffer step i - 1 used: free since its barrier
    const StepArgs& a = cur[i & 1].a;
    const bool batched = cur[i & 1].batched != 0;
    if (!(skip_unbatched && !batched)) {  // (uniform over the CTA)
      const int32_t nbs = batched ? nb : 1;
      const int64_t mn = a.m * a.n;
      for (int32_t b = 0; b < nbs; ++b) {
        float sa = 1.f, sb = 1.f;
        if (a.recs) {
          sa = pow2_neg(scale_exp(a.recs + a.rec_a + (a.a_bstride ? b : 0)));
          sb = pow2_neg(scale_exp(a.recs + a.rec_b + (a.b_bstride ? b : 0)));
        }
        const float* A = a.A + b * a.a_bstride;
        const float* B = a.B + b * a.b_bstride;
        float* C = a.C + b * a.c_bstride;
        int lmax = -127;
        for (int64_t idx = threadIdx.x; idx < mn; idx += blockDim.x) {
          const int64_t r = idx / a.n, c = idx - r * a.n;
          const float* ar = A + r * a.k;
          const float* br = B + c * a.k;
          float accr = kZero, acci = kZero;
          for (int64_t kk = 0; kk < a.k; ++kk) {
            const float xr = ar[kk] * sa, yr = br[kk] * sb;
            if (CPLX) {
              const float xi = ar[a.a_plane + kk] * sa, yi = br[a.b_plane + kk] * sb;
              accr = fmaf(xr, yr, accr);
              accr = fmaf(-xi, yi, accr);
              acci = fmaf(xr, yi, acci);
              acci = fmaf(xi, yr, acci);
            } else if (MAXPLUS) {
              accr = fmaxf(accr, xr + yr);
            } else {
              accr = fmaf(xr, yr, accr);
            }
          }
          const int64_t off = map_offset(a.rows, r) + map_offset(a.cols, c);
          if (CPLX) store_cplx(C, a.c_plane, off, accr, acci, a.c_split);
          else C[off] = accr;
          if (a.recs) lmax = max(lmax, exp_of(CPLX ? fmaxf(fabsf(accr), fabsf(acci)) : fabsf(accr)));
        }
        if (a.recs) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
          ScaleRec* rc = a.recs + a.rec_c + (a.c_bstride ? b : 0);
          if ((threadIdx.x & 31) == 0) atomicMax(&rc->emax, lmax);
          if (threadIdx.x == 0) {
            const ScaleRec* ra = a.recs + a.rec_a + (a.a_bstride ? b : 0);
            const ScaleRec* rb = a.recs + a.rec_b + (a.b_bstride ? b : 0);
            rc->log2 = ra->log2 + rb->log2 + scale_exp(ra) + scale_exp(rb);
          }
        }
      }
    }
    __syncthreads();  // this step's stores and scale record before the next step's loads
  }
}

void launch_contract_chain(const ChainStep* steps, int32_t n, int32_t nb, bool skip_unbatched, bool cplx,
                           bool maxplus, cudaStream_t st) {
  if (cplx) contract_chain_kernel<true, false><<<1, 512, 0, st>>>(steps, n, nb, skip_unbatched ? 1 : 0);
  else if (maxplus) contract_chain_kernel<false, true><<<1, 512, 0, st>>>(steps, n, nb, skip_unbatched ? 1 : 0);
  else contract_chain_kernel<false, false><<<1, 512, 0, st>>>(steps, n, nb, skip_unbatched ? 1 : 0);
}

// ---------------------------------------------------------------------------------
// big x small steps (n*k <= 256, n <= 16): the small operand sits in shared memory
// and every thread streams rows of the big one; one HBM pass over A and C. A warp's 32
// rows are 32 * k consecutive floats of each plane: read as float4 (one 16-byte load per
// lane per four k, so a warp load covers whole 128-byte lines) when k is a multiple of 4
// and the planes are 16-byte aligned, else one float at a time.

template <bool CPLX, int NMAX>
__global__ void __launch_bounds__(256) contract_stream_kernel(StepArgs a) {
  __shared__ float Bs[2][256];
  const int b = blockIdx.y;
  const float* __restrict__ A = a.A + b * a.a_bstride;
  const float* Bp = a.B + b * a.b_bstride;
  float* C = a.C + b * a.c_bstride;
  float sa = 1.f, sb = 1.f;
  if (a.recs) {
    sa = pow2_neg(scale_exp(a.recs + a.rec_a + (a.a_bstride ? b : 0)));
    sb = pow2_neg(scale_exp(a.recs + a.rec_b + (a.b_bstride ? b : 0)));
  }
  const int nk = (int)(a.n * a.k);
  for (int i = threadIdx.x; i < nk; i += blockDim.x) {
    Bs[0][i] = Bp[i] * sb;
    if (CPLX) Bs[1][i] = Bp[a.b_plane + i] * sb;
  }
  __syncthreads();
  const int n = (int)a.n, k = (int)a.k;
  int64_t coff[NMAX];
#pragma unroll
  for (int j = 0; j < NMAX; ++j) coff[j] = j < n ? map_offset(a.cols, j) : 0;
  const bool v4 = (k & 3) == 0 &&
                  ((reinterpret_cast<uintptr_t>(A) | static_cast<uintptr_t>(CPLX ? a.a_plane * 4 : 0)) & 15) == 0;
  int lmax = -127;
  // ROWS rows per thread per iteration (r0 + i * G): their loads are issued together, so
  // more bytes are in flight per SM at the occupancy the registers allow
  constexpr int ROWS = NMAX <= 4 ? 2 : 1;
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r0 < a.m; r0 += ROWS * G) {
    float cr[ROWS][NMAX], ci[ROWS][NMAX];
    bool live[ROWS];
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
      live[i] = r0 + i * G < a.m;
#pragma unroll
      for (int j = 0; j < NMAX; ++j) cr[i][j] = ci[i][j] = 0.f;
    }
    // one term of row i: x (scaled) times column kk of the small operand
    auto mac = [&](int i, float xr, float xi, int kk) {
      xr *= sa;
      xi *= sa;
#pragma unroll
      for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
          const float yr = Bs[0][j * k + kk];
          if (CPLX) {
            const float yi = Bs[1][j * k + kk];
            cr[i][j] = fmaf(xr, yr, cr[i][j]);
            cr[i][j] = fmaf(-xi, yi, cr[i][j]);
            ci[i][j] = fmaf(xr, yi, ci[i][j]);
            ci[i][j] = fmaf(xi, yr, ci[i][j]);
          } else {
            cr[i][j] = fmaf(xr, yr, cr[i][j]);
          }
        }
      }
    };
    if (v4) {
      for (int kk = 0; kk < k; kk += 4) {
        float4 xr[ROWS], xi[ROWS];
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
          xr[i] = xi[i] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (live[i]) {
            const float* arow = A + (r0 + i * G) * k + kk;
            xr[i] = __ldg(reinterpret_cast<const float4*>(arow));
            if (CPLX) xi[i] = __ldg(reinterpret_cast<const float4*>(arow + a.a_plane));
          }
        }
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
          mac(i, xr[i].x, xi[i].x, kk);
          mac(i, xr[i].y, xi[i].y, kk + 1);
          mac(i, xr[i].z, xi[i].z, kk + 2);
          mac(i, xr[i].w, xi[i].w, kk + 3);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < ROWS; ++i) {
        if (!live[i]) continue;
        const float* arow = A + (r0 + i * G) * k;
        for (int kk = 0; kk < k; ++kk) mac(i, __ldg(arow + kk), CPLX ? __ldg(arow + a.a_plane + kk) : 0.f, kk);
      }
    }
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
      if (!live[i]) continue;
      const int64_t ro = map_offset(a.rows, r0 + i * G);
#pragma unroll
      for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
          if (CPLX) store_cplx(C, a.c_plane, ro + coff[j], cr[i][j], ci[i][j], a.c_split);
          else C[ro + coff[j]] = cr[i][j];
          if (a.recs)
            lmax = max(lmax, exp_of(CPLX ? fmaxf(fabsf(cr[i][j]), fabsf(ci[i][j])) : fabsf(cr[i][j])));
        }
      }
    }
  }
  if (a.recs) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    ScaleRec* rc = a.recs + a.rec_c + (a.c_bstride ? b : 0);
    if ((threadIdx.x & 31) == 0) atomicMax(&rc->emax, lmax);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const ScaleRec* ra = a.recs + a.rec_a + (a.a_bstride ? b : 0);
      const ScaleRec* rb = a.recs + a.rec_b + (a.b_bstride ? b : 0);
      rc->log2 = ra->log2 + rb->log2 + scale_exp(ra) + scale_exp(rb);
    }
  }
}

// Big x small steps with k = 4, 8 or 16 and a 16-byte-aligned big operand: its rows reach
// shared memory by bulk copies (cp.async.bulk, one per plane per 256-row tile) through a
// ring of S tiles per CTA, so the bytes in flight per SM are set by the ring, not by the
// registers of the threads; each thread then computes one row of a tile and stores its n
// outputs. Persistent: CTA c takes tiles c, c + gridDim.x, ...; thread 0 issues the copies,
// refilling a tile's slot once every thread has read it. The waits are bounded: an expired
// one records code 41 in err, and the CTA waits (bounded) for its copies in flight and
// stops.
template <int K, bool CPLX>
struct StreamTma {
  static constexpr int TR = 256;                     // rows per tile (one per thread)
  static constexpr int PL = CPLX ? 2 : 1;
  static constexpr int TILE = TR * K;                // floats of one plane of one tile
  static constexpr int S = K <= 4 ? 6 : (K <= 8 ? 4 : 3);
  static constexpr int SMEM = S * PL * TILE * 4 + 2 * 256 * 4 + S * 8;
};

template <bool CPLX, int NMAX, int K>
__global__ void __launch_bounds__(256) contract_stream_tma_kernel(StepArgs a, int* err) {
  using G = StreamTma<K, CPLX>;
  constexpr int TR = G::TR, TILE = G::TILE, S = G::S, PL = G::PL;
  extern __shared__ __align__(128) float sm[];
  float* ring = sm;                                  // [S][PL][TR * K]
  float* Bs = sm + S * PL * TILE;                    // [2][256]
  uint64_t* full = reinterpret_cast<uint64_t*>(Bs + 2 * 256);
  const int tid = threadIdx.x;
  const int b = blockIdx.y;
  const float* A = a.A + b * a.a_bstride;
  const float* Bp = a.B + b * a.b_bstride;
  float* C = a.C + b * a.c_bstride;
  float sa = 1.f, sb = 1.f;
  if (a.recs) {
    sa = pow2_neg(scale_exp(a.recs + a.rec_a + (a.a_bstride ? b : 0)));
    sb = pow2_neg(scale_exp(a.recs + a.rec_b + (a.b_bstride ? b : 0)));
  }
  const int n = (int)a.n;
  for (int i = tid; i < n * K; i += blockDim.x) {
    Bs[i] = Bp[i] * sb;
    if (CPLX) Bs[256 + i] = Bp[a.b_plane + i] * sb;
  }
  const int64_t tiles = (a.m + TR - 1) / TR;
  const int64_t mine = tiles > blockIdx.x ? (tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  auto issue = [&](int64_t i) {  // local tile i into slot i % S (thread 0)
    const int slot = static_cast<int>(i % S);
    const int64_t r0 = (blockIdx.x + i * gridDim.x) * TR;
    const int64_t rows = a.m - r0 < TR ? a.m - r0 : TR;
    const uint32_t bytes = static_cast<uint32_t>(rows * K * 4);
    float* dst = ring + slot * PL * TILE;
    mbar_expect_tx(&full[slot], PL * bytes);
    bulk_load(dst, A + r0 * K, bytes, &full[slot]);
    if (CPLX) bulk_load(dst + TILE, A + a.a_plane + r0 * K, bytes, &full[slot]);
  };
  int64_t issued = 0;
  if (tid == 0) {
    for (int i = 0; i < S; ++i) mbar_init(&full[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (; issued < S && issued < mine; ++issued) issue(issued);
  }
  __syncthreads();
  int64_t coff[NMAX];
#pragma unroll
  for (int j = 0; j < NMAX; ++j) coff[j] = j < n ? map_offset(a.cols, j) : 0;
  int lmax = -127;
  int64_t i = 0;
  for (; i < mine; ++i) {
    const int slot = static_cast<int>(i % S);
    const bool ok = __syncthreads_and(mbar_wait(&full[slot], static_cast<uint32_t>((i / S) & 1)) ? 1 : 0);
    if (!ok) {
      if (tid == 0) atomicExch(err, 41);
      break;
    }
    const int64_t r = (blockIdx.x + i * gridDim.x) * TR + tid;
    if (r < a.m) {
      const float* xr_s = ring + slot * PL * TILE + tid * K;
      float cr[NMAX], ci[NMAX];
#pragma unroll
      for (int j = 0; j < NMAX; ++j) cr[j] = ci[j] = 0.f;
#pragma unroll
      for (int k4 = 0; k4 < K; k4 += 4) {
        const float4 xr = *reinterpret_cast<const float4*>(xr_s + k4);
        const float4 xi = CPLX ? *reinterpret_cast<const float4*>(xr_s + TILE + k4) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float vr[4] = {xr.x * sa, xr.y * sa, xr.z * sa, xr.w * sa};
        const float vi[4] = {xi.x * sa, xi.y * sa, xi.z * sa, xi.w * sa};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
          for (int j = 0; j < NMAX; ++j) {
            if (j < n) {
              const float yr = Bs[j * K + k4 + q];
              if (CPLX) {
                const float yi = Bs[256 + j * K + k4 + q];
                cr[j] = fmaf(vr[q], yr, cr[j]);
                cr[j] = fmaf(-vi[q], yi, cr[j]);
                ci[j] = fmaf(vr[q], yi, ci[j]);
                ci[j] = fmaf(vi[q], yr, ci[j]);
              } else {
                cr[j] = fmaf(vr[q], yr, cr[j]);
              }
            }
          }
        }
      }
      const int64_t ro = map_offset(a.rows, r);
#pragma unroll
      for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
          if (CPLX) store_cplx(C, a.c_plane, ro + coff[j], cr[j], ci[j], a.c_split);
          else C[ro + coff[j]] = cr[j];
          if (a.recs) lmax = max(lmax, exp_of(CPLX ? fmaxf(fabsf(cr[j]), fabsf(ci[j])) : fabsf(cr[j])));
        }
      }
    }
    __syncthreads();  // every thread has read the slot: refill it
    if (tid == 0 && issued < mine) issue(issued++);
  }
  if (tid == 0) {  // after an expired wait: let the copies in flight land before exiting
    for (int64_t j = i; j < issued; ++j)
      if (!mbar_wait(&full[j % S], static_cast<uint32_t>((j / S) & 1))) break;
  }
  if (a.recs) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    ScaleRec* rc = a.recs + a.rec_c + (a.c_bstride ? b : 0);
    if ((tid & 31) == 0) atomicMax(&rc->emax, lmax);
    if (blockIdx.x == 0 && tid == 0) {
      const ScaleRec* ra = a.recs + a.rec_a + (a.a_bstride ? b : 0);
      const ScaleRec* rb = a.recs + a.rec_b + (a.b_bstride ? b : 0);
      rc->log2 = ra->log2 + rb->log2 + scale_exp(ra) + scale_exp(rb);
    }
  }
}

template <bool CPLX, int NMAX, int K>
void launch_stream_tma(const StepArgs& a, int32_t nb, int num_sms, int* err, cudaStream_t st) {
  constexpr int smem = StreamTma<K, CPLX>::SMEM;
  // resident CTAs per SM, looked up once per form (thread-safe static initialisation)
  static const int per_sm = [] {
    cudaFuncSetAttribute(contract_stream_tma_kernel<CPLX, NMAX, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, contract_stream_tma_kernel<CPLX, NMAX, K>, 256, smem);
    return occ > 0 ? occ : 1;
  }();
  const int64_t tiles = (a.m + 255) / 256;
  int64_t gx = (int64_t(num_sms) * per_sm + nb - 1) / nb;
  gx = std::max<int64_t>(1, std::min<int64_t>(gx, tiles));
  contract_stream_tma_kernel<CPLX, NMAX, K><<<dim3((unsigned)gx, (unsigned)nb), 256, smem, st>>>(a, err);
}

// Combine the k parts of a split SIMT step in part order (sum, or max for max-plus) and
// write C through the offset maps. One thread per output element of every batch entry.
__global__ void simt_combine_kernel(StepArgs a, int32_t nb, int32_t cplx) {
  const int64_t mn = a.m * a.n, np = cplx ? 2 : 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nb * mn;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / mn, o = e - b * mn;
    const float* P0 = a.part + b * np * mn + o;
    const int64_t pstride = (int64_t)nb * np * mn;  // one part to the next
    float vr = P0[0], vi = cplx ? P0[mn] : 0.f;
    for (int s = 1; s < a.ksplit; ++s) {
      const float xr = P0[s * pstride];
      if (a.maxplus) {
        vr = fmaxf(vr, xr);
      } else {
        vr += xr;
        if (cplx) vi += P0[s * pstride + mn];
      }
    }
    const int64_t i = o / a.n, j = o - i * a.n;
    const int64_t off = map_offset(a.rows, i) + map_offset(a.cols, j);
    float* C = a.C + b * a.c_bstride;
    if (cplx) store_cplx(C, a.c_plane, off, vr, vi, a.c_split);
    else C[off] = vr;
  }
}

int32_t simt_ksplit(int64_t m, int64_t n, int64_t k, int64_t copies, int num_sms, bool scaled) {
  if (scaled || k < 2048) return 1;
  // aim at four 256-thread CTAs per SM (the kernel's blocks are short-lived)
  const int64_t tiles = ((m + 63) / 64) * ((n + 63) / 64) * copies;
  if (tiles >= 2 * int64_t(num_sms)) return 1;
  int64_t s = (4 * int64_t(num_sms) + tiles - 1) / tiles;
  s = std::min<int64_t>(s, k / 1024);
  s = std::min<int64_t>(s, 32);
  return s > 1 ? int32_t(s) : 1;
}

void launch_contract_simt(const StepArgs& a, int32_t nb, bool cplx, cudaStream_t st) {
  const int64_t tiles = ((a.m + 63) / 64) * ((a.n + 63) / 64);
  dim3 grid((unsigned)tiles, (unsigned)nb, (unsigned)(a.ksplit > 1 ? a.ksplit : 1));
  if (cplx) contract_simt_kernel<true><<<grid, 256, 0, st>>>(a);
  else if (a.maxplus) contract_simt_kernel<false, true><<<grid, 256, 0, st>>>(a);
  else contract_simt_kernel<false><<<grid, 256, 0, st>>>(a);
  if (a.ksplit > 1) {
    const int64_t total = int64_t(nb) * a.m * a.n;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
    simt_combine_kernel<<<blocks, 256, 0, st>>>(a, nb, cplx ? 1 : 0);
  }
}

// The bulk-copy form takes k = 4, 8, 16 with the big operand's planes and batch entries
// 16-byte aligned and at least 32 tiles of rows; the register form everything else.
bool stream_tma_ok(const StepArgs& a) {
  const bool kk = a.k == 4 || a.k == 8 || a.k == 16;
  const bool al = (reinterpret_cast<uintptr_t>(a.A) & 15) == 0 && (a.a_plane & 3) == 0 && (a.a_bstride & 3) == 0;
  return kk && al && a.n <= 16 && a.m >= 32 * 256;
}

void launch_contract_stream(const StepArgs& a, int32_t nb, bool cplx, int num_sms, int* err, cudaStream_t st) {
  if (stream_tma_ok(a)) {
#define TN_STREAM_TMA(KK)                                                                   \
  if (a.k == KK) {                                                                          \
    if (a.n <= 4) {                                                                         \
      if (cplx) launch_stream_tma<true, 4, KK>(a, nb, num_sms, err, st);                    \
      else launch_stream_tma<false, 4, KK>(a, nb, num_sms, err, st);                        \
    } else {                                                                                \
      if (cplx) launch_stream_tma<true, 16, KK>(a, nb, num_sms, err, st);                   \
      else launch_stream_tma<false, 16, KK>(a, nb, num_sms, err, st);                       \
    }                                                                                       \
    return;                                                                                 \
  }
    TN_STREAM_TMA(4)
    TN_STREAM_TMA(8)
    TN_STREAM_TMA(16)
#undef TN_STREAM_TMA
  }
  int64_t blocks = (a.m + 255) / 256;
  const int64_t cap = (int64_t)num_sms * 8;
  if (blocks > cap) blocks = cap;
  dim3 grid((unsigned)blocks, (unsigned)nb);
#define TN_STREAM_CASE(NM)                                                            \
  if (a.n <= NM) {                                                                     \
    if (cplx) contract_stream_kernel<true, NM><<<grid, 256, 0, st>>>(a);               \
    else contract_stream_kernel<false, NM><<<grid, 256, 0, st>>>(a);                   \
    return;                                                                            \
  }
  TN_STREAM_CASE(2)
  TN_STREAM_CASE(4)
  TN_STREAM_CASE(8)
  TN_STREAM_CASE(16)
#undef TN_STREAM_CASE
}

// ---------------------------------------------------------------------------------
// cross-slice accumulation (a7) and output (a8): per output element, add the nb slice
// results of this pass in slice order with Neumaier compensation; with exponent scaling
// each slice's value is brought to the reference exponent of the first slice ever added.
// Passes before the last keep [sum re, sum im, comp re, comp im] in FP64 per element; the
// last pass writes sum + comp straight to the caller's output (and the log scale), so a
// one-pass call never touches the accumulator, and a one-slice call (widen_root_kernel)
// does no FP64 arithmetic at all.

// The binary64 value of a binary32 value, exactly, from the two formats' fields with integer
// operations only (this GPU's FP64 pipe is narrow; a conversion per output element would
// bound a one-slice open output): the exponent is rebiased from 127 to 1023 and the 23
// fraction bits move to the top of the 52; subnormal inputs are normalised; zeros and
// infinities keep their sign, and a NaN its sign and payload with the quiet bit set (as an
// IEEE 754 conversion returns a signaling NaN quieted).
__device__ __forceinline__ double f64_of_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = static_cast<uint64_t>(u >> 31) << 63;
  const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  uint64_t bits;
  if (e == 0xffu) {
    bits = sign | (uint64_t(0x7ff) << 52) | (uint64_t(m) << 29) | (m ? uint64_t(1) << 51 : 0);
  } else if (e != 0u) {
    bits = sign | (uint64_t(e + (1023 - 127)) << 52) | (uint64_t(m) << 29);
  } else if (m == 0u) {
    bits = sign;
  } else {  // m * 2^-149 with the leading one at bit p: exponent p - 149, fraction below it
    const int p = 31 - __clz(static_cast<int>(m));
    bits = sign | (uint64_t(p - 149 + 1023) << 52) | ((uint64_t(m) << (52 - p)) & ((uint64_t(1) << 52) - 1));
  }
  return __longlong_as_double(static_cast<long long>(bits));
}

__global__ void accumulate_root_kernel(const float* __restrict__ root, int64_t size, int32_t nb,
                                       int64_t bstride, int64_t plane, int32_t cplx, double* acc,
                                       const ScaleRec* recs, int32_t rec_root, int32_t root_batched,
                                       int64_t* ref_exp, int32_t first, int32_t last, int32_t maxplus,
                                       void* out, double* log_scale) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= size) return;
  double* s = acc + e * 4;
  if (maxplus) {  // slices combine by maximum (real, unscaled)
    double best = first ? __longlong_as_double(static_cast<long long>(0xfff0000000000000ull)) : s[0];
    for (int b = 0; b < nb; ++b) best = fmax(best, (double)root[b * bstride + e]);
    if (last) {
      reinterpret_cast<double*>(out)[e] = best;
      if (e == 0 && log_scale) *log_scale = 0.0;
    } else {
      s[0] = best;
    }
    return;
  }
  double sr = first ? 0.0 : s[0], si = first ? 0.0 : s[1];
  double cr = first ? 0.0 : s[2], ci = first ? 0.0 : s[3];
  int64_t ref = 0;
  if (recs) {
    const ScaleRec* r0 = recs + rec_root;
    ref = first ? r0->log2 : *ref_exp;
  }
  for (int b = 0; b < nb; ++b) {
    double vr = root[b * bstride + e];
    double vi = cplx ? root[b * bstride + plane + e] : 0.0;
    if (recs) {
      const ScaleRec* r = recs + rec_root + (root_batched ? b : 0);
      // stored values are unscaled outputs of the last step: true = v * 2^log2
      const int64_t sh = r->log2 - ref;
      vr = ldexp(vr, (int)sh);
      vi = ldexp(vi, (int)sh);
    }
    double t = sr + vr;
    cr += fabs(sr) >= fabs(vr) ? (sr - t) + vr : (vr - t) + sr;
    sr = t;
    t = si + vi;
    ci += fabs(si) >= fabs(vi) ? (si - t) + vi : (vi - t) + si;
    si = t;
  }
  if (last) {
    if (cplx) reinterpret_cast<double2*>(out)[e] = make_double2(sr + cr, si + ci);
    else reinterpret_cast<double*>(out)[e] = sr + cr;
    if (e == 0 && log_scale) *log_scale = recs ? double(ref) * 0.69314718055994530942 : 0.0;
    return;
  }
  s[0] = sr;
  s[1] = si;
  s[2] = cr;
  s[3] = ci;
  if (recs && first && e == 0) *ref_exp = ref;
}

// One slice in one pass: the output is that slice's value, widened exactly; no FP64
// arithmetic. Grid-stride, two elements (e, e + G) per thread per iteration.
__global__ void __launch_bounds__(256) widen_root_kernel(const float* __restrict__ root, int64_t size,
                                                         int64_t plane, int32_t cplx, void* out,
                                                         const ScaleRec* rec, double* log_scale) {
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e0 < size; e0 += 2 * G) {
    float re[2], im[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int64_t e = e0 + i * G;
      re[i] = e < size ? __ldg(root + e) : 0.f;
      im[i] = cplx && e < size ? __ldg(root + plane + e) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int64_t e = e0 + i * G;
      if (e >= size) continue;
      if (cplx) reinterpret_cast<double2*>(out)[e] = make_double2(f64_of_f32(re[i]), f64_of_f32(im[i]));
      else reinterpret_cast<double*>(out)[e] = f64_of_f32(re[i]);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && log_scale)
    *log_scale = rec ? double(rec->log2) * 0.69314718055994530942 : 0.0;
}

void launch_accumulate_root(const float* root, int64_t size, int32_t nb, int64_t bstride,
                            int64_t plane, bool cplx, double* acc, const ScaleRec* recs,
                            int32_t rec_root, bool root_batched, int64_t* ref_exp, bool first, bool last,
                            bool maxplus, void* out, double* log_scale, int num_sms, cudaStream_t st) {
  if (first && last && nb == 1) {
    const int64_t want = (size + 511) / 512;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, int64_t(num_sms) * 8));
    widen_root_kernel<<<blocks, 256, 0, st>>>(root, size, plane, cplx ? 1 : 0, out,
                                              recs && !maxplus ? recs + rec_root : nullptr, log_scale);
    return;
  }
  const int threads = 128;
  const unsigned blocks = (unsigned)((size + threads - 1) / threads);
  accumulate_root_kernel<<<blocks, threads, 0, st>>>(root, size, nb, bstride, plane, cplx ? 1 : 0, acc,
                                                     recs, rec_root, root_batched ? 1 : 0, ref_exp,
                                                     first ? 1 : 0, last ? 1 : 0, maxplus ? 1 : 0, out,
                                                     log_scale);
}

// ---------------------------------------------------------------------------------
// split-K steps (m*n <= kSplitMaxOut outputs, very long k; e.g. the final scalar of a
// closed network, a dot product of two large tensors). Pass 1: CTA (chunk, b) sums
// its k-range for every output -- FP32 over the few terms each thread owns, FP64
// across threads -- and writes one FP64 partial per output to scratch[b][chunk].
// Pass 2: per (b, output), the partials are added in chunk order in FP64 and the
// result stored through the offset maps. Deterministic: no atomics.

template <bool CPLX, bool MAXPLUS = false>
__global__ void __launch_bounds__(256) splitk_partial_kernel(StepArgs a, double* scratch, int64_t kc,
                                                             int32_t chunks) {
  static_assert(!(CPLX && MAXPLUS), "the max-plus semiring is real");
  const int chunk = blockIdx.x, b = blockIdx.y;
  const int m = (int)a.m, n = (int)a.n, mn = m * n;
  const float* A = a.A + b * a.a_bstride;
  const float* B = a.B + b * a.b_bstride;
  float sa = 1.f, sb = 1.f;
  if (a.recs) {
    sa = pow2_neg(scale_exp(a.recs + a.rec_a + (a.a_bstride ? b : 0)));
    sb = pow2_neg(scale_exp(a.recs + a.rec_b + (a.b_bstride ? b : 0)));
  }
  float accr[kSplitMaxOut], acci[kSplitMaxOut];
  const float zero = MAXPLUS ? __int_as_float(0xff800000) : 0.f;  // the semiring's zero
#pragma unroll
  for (int o = 0; o < kSplitMaxOut; ++o) accr[o] = acci[o] = zero;
  const int64_t k0 = (int64_t)chunk * kc;
  const int64_t k1 = min(a.k, k0 + kc);
  if (MAXPLUS) {
    for (int64_t kk = k0 + threadIdx.x; kk < k1; kk += blockDim.x) {
#pragma unroll
      for (int o = 0; o < kSplitMaxOut; ++o) {
        if (o < mn) {
          const int i = o / n, j = o - (o / n) * n;
          accr[o] = fmaxf(accr[o], A[i * a.k + kk] + B[j * a.k + kk]);
        }
      }
    }
  }
  // the output index o is a compile-time constant in every unrolled iteration, so the
  // accumulators stay in registers
  const bool vec = !MAXPLUS && (a.k & 3) == 0 && (a.a_plane & 3) == 0 && (a.b_plane & 3) == 0 &&
                   ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) == 0;
  if (vec) {
    // 16-byte loads, four k-steps of the block unrolled: every thread has all of its
    // loads of the chunk in flight before its first FMA (the step is HBM-bound)
#pragma unroll 4
    for (int64_t kk = k0 + 4 * threadIdx.x; kk < k1; kk += 4 * blockDim.x) {
#pragma unroll
      for (int o = 0; o < kSplitMaxOut; ++o) {
        if (o < mn) {
          const int i = o / n, j = o - (o / n) * n;
          const float4 xr = *reinterpret_cast<const float4*>(A + i * a.k + kk);
          const float4 yr = *reinterpret_cast<const float4*>(B + j * a.k + kk);
          if (CPLX) {
            const float4 xi = *reinterpret_cast<const float4*>(A + a.a_plane + i * a.k + kk);
            const float4 yi = *reinterpret_cast<const float4*>(B + a.b_plane + j * a.k + kk);
            const float ar[4] = {xr.x * sa, xr.y * sa, xr.z * sa, xr.w * sa};
            const float ai[4] = {xi.x * sa, xi.y * sa, xi.z * sa, xi.w * sa};
            const float br[4] = {yr.x * sb, yr.y * sb, yr.z * sb, yr.w * sb};
            const float bi[4] = {yi.x * sb, yi.y * sb, yi.z * sb, yi.w * sb};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              accr[o] = fmaf(ar[e], br[e], fmaf(-ai[e], bi[e], accr[o]));
              acci[o] = fmaf(ar[e], bi[e], fmaf(ai[e], br[e], acci[o]));
            }
          } else {
            accr[o] = fmaf(xr.x * sa, yr.x * sb, accr[o]);
            accr[o] = fmaf(xr.y * sa, yr.y * sb, accr[o]);
            accr[o] = fmaf(xr.z * sa, yr.z * sb, accr[o]);
            accr[o] = fmaf(xr.w * sa, yr.w * sb, accr[o]);
          }
        }
      }
    }
  }
  for (int64_t kk = k0 + threadIdx.x; !MAXPLUS && !vec && kk < k1; kk += blockDim.x) {
#pragma unroll
    for (int o = 0; o < kSplitMaxOut; ++o) {
      if (o < mn) {
        const int i = o / n, j = o - (o / n) * n;
        const float xr = A[i * a.k + kk] * sa;
        const float yr = B[j * a.k + kk] * sb;
        if (CPLX) {
          const float xi = A[a.a_plane + i * a.k + kk] * sa;
          const float yi = B[a.b_plane + j * a.k + kk] * sb;
          accr[o] = fmaf(xr, yr, fmaf(-xi, yi, accr[o]));
          acci[o] = fmaf(xr, yi, fmaf(xi, yr, acci[o]));
        } else {
          accr[o] = fmaf(xr, yr, accr[o]);
        }
      }
    }
  }
  __shared__ double red[2][kSplitMaxOut][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 0; o < kSplitMaxOut; ++o) {
    if (o >= mn) break;
    double vr = accr[o], vi = acci[o];
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      if (MAXPLUS) {
        vr = fmax(vr, __shfl_xor_sync(0xffffffffu, vr, s));
      } else {
        vr += __shfl_xor_sync(0xffffffffu, vr, s);
        vi += __shfl_xor_sync(0xffffffffu, vi, s);
      }
    }
    if (lane == 0) {
      red[0][o][warp] = vr;
      red[1][o][warp] = vi;
    }
  }
  __syncthreads();
  if (threadIdx.x < mn) {
    const int o = threadIdx.x;
    double vr = MAXPLUS ? (double)zero : 0.0, vi = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (MAXPLUS) {
        vr = fmax(vr, red[0][o][w]);
      } else {
        vr += red[0][o][w];
        vi += red[1][o][w];
      }
    }
    double* dst = scratch + (((int64_t)b * chunks + chunk) * mn + o) * 2;
    dst[0] = vr;
    dst[1] = vi;
  }
}

constexpr int kFinalThreads = 128;

__global__ void __launch_bounds__(kFinalThreads) splitk_final_kernel(StepArgs a, const double* scratch,
                                                                    int32_t chunks, int32_t cplx) {
  const int b = blockIdx.x;
  const int m = (int)a.m, n = (int)a.n, mn = m * n;
  float* C = a.C + b * a.c_bstride;
  __shared__ double part[2][kFinalThreads];
  int lmax = -127;
  // thread t adds the partials of a contiguous run of chunks in order; thread 0 then adds
  // the runs in order: a fixed association for a given chunk count (deterministic)
  const int per = (chunks + kFinalThreads - 1) / kFinalThreads;
  const double zero = a.maxplus ? __longlong_as_double(static_cast<long long>(0xfff0000000000000ull)) : 0.0;
  for (int o = 0; o < mn; ++o) {
    double sr = zero, si = 0.0;
    const int c0 = threadIdx.x * per, c1 = min(chunks, c0 + per);
    for (int c = c0; c < c1; ++c) {
      const double* p = scratch + (((int64_t)b * chunks + c) * mn + o) * 2;
      if (a.maxplus) {
        sr = fmax(sr, p[0]);
      } else {
        sr += p[0];
        si += p[1];
      }
    }
    part[0][threadIdx.x] = sr;
    part[1][threadIdx.x] = si;
    __syncthreads();
    double vr = zero, vi = 0.0;
    if (threadIdx.x == 0)
      for (int t = 0; t < kFinalThreads; ++t) {
        if (a.maxplus) {
          vr = fmax(vr, part[0][t]);
        } else {
          vr += part[0][t];
          vi += part[1][t];
        }
      }
    __syncthreads();  // every thread, every o: part is rewritten next iteration
    if (threadIdx.x == 0) {
      const int i = o / n, j = o % n;
      const int64_t off = map_offset(a.rows, i) + map_offset(a.cols, j);
      if (cplx) store_cplx(C, a.c_plane, off, (float)vr, (float)vi, a.c_split);
      else C[off] = (float)vr;
      if (a.recs) lmax = max(lmax, exp_of(cplx ? fmaxf(fabsf((float)vr), fabsf((float)vi)) : fabsf((float)vr)));
    }
  }
  if (a.recs) {
    ScaleRec* rc = a.recs + a.rec_c + (a.c_bstride ? b : 0);
    atomicMax(&rc->emax, lmax);
    if (threadIdx.x == 0) {
      const ScaleRec* ra = a.recs + a.rec_a + (a.a_bstride ? b : 0);
      const ScaleRec* rb = a.recs + a.rec_b + (a.b_bstride ? b : 0);
      rc->log2 = ra->log2 + rb->log2 + scale_exp(ra) + scale_exp(rb);
    }
  }
}

int32_t splitk_chunks(int64_t k) { return (int32_t)((k + kSplitChunk - 1) / kSplitChunk); }

void launch_contract_splitk(const StepArgs& a, int32_t nb, bool cplx, double* scratch, cudaStream_t st) {
  const int32_t chunks = splitk_chunks(a.k);
  dim3 grid((unsigned)chunks, (unsigned)nb);
  if (cplx) splitk_partial_kernel<true><<<grid, 256, 0, st>>>(a, scratch, kSplitChunk, chunks);
  else if (a.maxplus) splitk_partial_kernel<false, true><<<grid, 256, 0, st>>>(a, scratch, kSplitChunk, chunks);
  else splitk_partial_kernel<false><<<grid, 256, 0, st>>>(a, scratch, kSplitChunk, chunks);
  splitk_final_kernel<<<(unsigned)nb, kFinalThreads, 0, st>>>(a, scratch, chunks, cplx ? 1 : 0);
}

}  // namespace tn
