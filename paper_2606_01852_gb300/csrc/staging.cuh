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

// A CTA of the tiled kernel walks consecutive tiles: the cursor holds the chunk indices and
// the digits of the rest index, and advancing it updates the offsets by the stride of the
// digits that change (amortised one digit per tile), equal to tile_base of the next tile.
struct TileCursor {
  int64_t co, ci;                  // output-group and input-group chunk of the tile
  int64_t src0, dst0;              // offsets of the rest index (src0 with the slice's)
  uint32_t dig[kMaxLeafRank];      // digits of the rest index over rpos, last fastest
};

__host__ __device__ inline void cursor_start(const LeafDesc& d, int64_t blk, int64_t sid, TileCursor& c) {
  const int64_t nco = (d.Po + 31) / 32, nci = (d.Pi + 31) / 32;
  c.co = blk % nco;
  blk /= nco;
  c.ci = blk % nci;
  int64_t r = blk / nci;
  c.src0 = 0;
  c.dst0 = 0;
  for (int q = d.nr - 1; q >= 0; --q) {
    const int p = d.rpos[q];
    c.dig[q] = static_cast<uint32_t>(r % d.ext[p]);
    r /= d.ext[p];
    c.src0 += int64_t(c.dig[q]) * d.sstride[p];
    c.dst0 += int64_t(c.dig[q]) * d.dstride[p];
  }
  for (int q = 0; q < d.n_sl; ++q) c.src0 += ((sid / d.sl_div[q]) % d.sl_ext[q]) * d.sl_stride[q];
}

__host__ __device__ inline void cursor_next(const LeafDesc& d, TileCursor& c) {
  if (++c.co < (d.Po + 31) / 32) return;
  c.co = 0;
  if (++c.ci < (d.Pi + 31) / 32) return;
  c.ci = 0;
  for (int q = d.nr - 1; q >= 0; --q) {
    const int p = d.rpos[q];
    c.src0 += d.sstride[p];
    c.dst0 += d.dstride[p];
    if (++c.dig[q] < d.ext[p]) return;
    c.src0 -= int64_t(d.ext[p]) * d.sstride[p];
    c.dst0 -= int64_t(d.ext[p]) * d.dstride[p];
    c.dig[q] = 0;
  }
}

// tiles one CTA of the tiled kernel walks, and tiles it holds in flight per iteration
constexpr int kTilesPerCta = 16;
constexpr int kTilesInFlight = 4;

// One iteration of a CTA at tile blk (its tiles blk0 .. blk1-1): advance the cursors of
// the iteration's tiles (slot u holds tile blk + u) and decide which slots' offset tables
// must be rebuilt -- those whose chunk indices differ from the ones the slot's table was
// last built for (built[u], -1 before the first build). Returns the number of tiles.
__host__ __device__ inline int iteration_tiles(const LeafDesc& d, int64_t blk, int64_t blk0, int64_t blk1,
                                               int64_t sid, TileCursor* cur, int64_t (*built)[2], int* rebuild) {
  const int nt = blk1 - blk < kTilesInFlight ? static_cast<int>(blk1 - blk) : kTilesInFlight;
  for (int u = 0; u < nt; ++u) {
    if (u == 0 && blk == blk0) {
      cursor_start(d, blk, sid, cur[0]);
    } else {
      cur[u] = cur[u == 0 ? kTilesInFlight - 1 : u - 1];
      cursor_next(d, cur[u]);
    }
    rebuild[u] = (cur[u].co != built[u][0] || cur[u].ci != built[u][1]) ? 1 : 0;
    built[u][0] = cur[u].co;
    built[u][1] = cur[u].ci;
  }
  return nt;
}

// Entry r (0..31) of a tile's offset tables: source offset of input-group index gi0 + r and
// of output-group index go0 + r (both without the rest index), and staged offset of the
// row of input-group index gi0 + r (0 past the group's end).
__host__ __device__ inline void table_entry(const LeafDesc& d, int64_t go0, int64_t gi0, int r, int64_t& isrc,
                                            int64_t& osrc, int64_t& irow) {
  const int64_t gi = gi0 + r, go = go0 + r;
  isrc = gi < d.Pi ? group_offset(gi, d.ipos, d.ni, d.ext, d.sstride) : 0;
  osrc = go < d.Po ? tail_offset(go, d.rank, d.no, d.ext, d.sstride) : 0;
  irow = gi < d.Pi ? group_offset(gi, d.ipos, d.ni, d.ext, d.dstride) + go0 : 0;
}

// Pipelined form (LeafDesc::fast): CTA c walks tiles 16 c .. 16 c + 15, whose rest index is
// 16 c + i; its offsets split into the low part (i over the last nlo rest positions, the
// same for every CTA) and the high part (c over the others, plus the slice's offset).
__host__ __device__ inline void rest_lo_offsets(const LeafDesc& d, int64_t lo, int64_t& src, int64_t& dst) {
  src = dst = 0;
  for (int q = d.nr - 1; q >= d.nr - d.nlo; --q) {
    const int p = d.rpos[q];
    const int64_t g = lo % d.ext[p];
    lo /= d.ext[p];
    src += g * d.sstride[p];
    dst += g * d.dstride[p];
  }
}
__host__ __device__ inline void rest_hi_offsets(const LeafDesc& d, int64_t hi, int64_t sid, int64_t& src, int64_t& dst) {
  src = dst = 0;
  for (int q = d.nr - d.nlo - 1; q >= 0; --q) {
    const int p = d.rpos[q];
    const int64_t g = hi % d.ext[p];
    hi /= d.ext[p];
    src += g * d.sstride[p];
    dst += g * d.dstride[p];
  }
  for (int q = 0; q < d.n_sl; ++q) src += ((sid / d.sl_div[q]) % d.sl_ext[q]) * d.sl_stride[q];
}

// Source element (declared order) and staged element of tile entry (ti, to).
__host__ __device__ inline int64_t tile_src(const LeafDesc& d, const TileBase& t, int64_t gi, int64_t go) {
  return t.src0 + group_offset(gi, d.ipos, d.ni, d.ext, d.sstride) + tail_offset(go, d.rank, d.no, d.ext, d.sstride);
}
__host__ __device__ inline int64_t tile_dst_row(const LeafDesc& d, const TileBase& t, int64_t gi) {
  return t.dst0 + group_offset(gi, d.ipos, d.ni, d.ext, d.dstride) + t.go0;
}

}  // namespace tn
