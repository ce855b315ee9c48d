// Index arithmetic of the tiled leaf-permutation kernel (K-PERM), shared by the kernel
// and by the host-side replay that checks it (tn_plan_check_staging).
#pragma once

#include <cstdint>

#include "tn_internal.h"

namespace tn {

// offset of index g over the positions pos[0..n-1] (mixed radix, last fastest) under `stride`
__host__ __device__ inline int64_t group_offset(int64_t g, const int8_t* pos, int32_t n, const uint32_t* ext,
                                                const int64_t* stride) {
  int64_t off = 0;
  if (g >= 0 && g < (int64_t(1) << 32)) {  // 32-bit digits (the same values, fewer instructions)
    uint32_t h = static_cast<uint32_t>(g);
    for (int q = n - 1; q >= 0; --q) {
      const uint32_t e = ext[pos[q]];
      off += int64_t(h % e) * stride[pos[q]];
      h /= e;
    }
    return off;
  }
  for (int q = n - 1; q >= 0; --q) {
    const uint32_t e = ext[pos[q]];
    off += (g % e) * stride[pos[q]];
    g /= e;
  }
  return off;
}

// offset of output-group index g (the trailing `no` planned positions) under `stride`
__host__ __device__ inline int64_t tail_offset(int64_t g, int32_t rank, int32_t no, const uint32_t* ext,
                                               const int64_t* stride) {
  int64_t off = 0;
  if (g >= 0 && g < (int64_t(1) << 32)) {
    uint32_t h = static_cast<uint32_t>(g);
    for (int i = rank - 1; i >= rank - no; --i) {
      const uint32_t e = ext[i];
      off += int64_t(h % e) * stride[i];
      h /= e;
    }
    return off;
  }
  for (int i = rank - 1; i >= rank - no; --i) {
    const uint32_t e = ext[i];
    off += (g % e) * stride[i];
    g /= e;
  }
  return off;
}

// A tile of the tiled staging kernel: its first output-group and input-group indices, and
// the source (rest index + slice) and staged (rest index) offsets they add to.
struct TileBase {
  int64_t go0, gi0, src0, dst0;
};

// Tile `blk` (0 .. Pr * ceil(Po/32) * ceil(Pi/32) - 1) of leaf d for slice `sid`.
__host__ __device__ inline TileBase tile_base(const LeafDesc& d, int64_t blk, int64_t sid) {
  const int64_t co = (d.Po + 31) / 32, ci = (d.Pi + 31) / 32;
  TileBase t;
  t.go0 = (blk % co) * 32;
  blk /= co;
  t.gi0 = (blk % ci) * 32;
  const int64_t r = blk / ci;
  t.src0 = group_offset(r, d.rpos, d.nr, d.ext, d.sstride);
  t.dst0 = group_offset(r, d.rpos, d.nr, d.ext, d.dstride);
  for (int q = 0; q < d.n_sl; ++q) t.src0 += ((sid / d.sl_div[q]) % d.sl_ext[q]) * d.sl_stride[q];
  return t;
}

// Source element (declared order) and staged element of tile entry (ti, to).
__host__ __device__ inline int64_t tile_src(const LeafDesc& d, const TileBase& t, int64_t gi, int64_t go) {
  return t.src0 + group_offset(gi, d.ipos, d.ni, d.ext, d.sstride) + tail_offset(go, d.rank, d.no, d.ext, d.sstride);
}
__host__ __device__ inline int64_t tile_dst_row(const LeafDesc& d, const TileBase& t, int64_t gi) {
  return t.dst0 + group_offset(gi, d.ipos, d.ni, d.ext, d.dstride) + t.go0;
}

}  // namespace tn
