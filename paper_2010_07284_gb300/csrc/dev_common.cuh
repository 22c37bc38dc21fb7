// Small device helpers shared by every kernel of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "vl_internal.h"

#define VL_DEV __device__ __forceinline__

namespace vl {

// Bits of word w (of a row of width W) that are real pixels.
VL_DEV uint32_t vmask(int w, int W) {
  int n = W - 32 * w;
  return n >= 32 ? 0xFFFFFFFFu : (n <= 0 ? 0u : ((1u << n) - 1u));
}

// Mask of bits 0..b inclusive.
VL_DEV uint32_t le_mask(int b) { return b >= 31 ? 0xFFFFFFFFu : ((2u << b) - 1u); }

// Loads that bypass L1: data written by other CTAs of the same launch.
// Row and column of element i of a row-major grid of `cols` columns: a
// 32-bit division while i < 2^32 (every word index, and every pixel index
// of a grid under 2^32 pixels), else a 64-bit one.
VL_DEV void split_index(long long i, int cols, int& row, int& col) {
  if (i < (1LL << 32)) {
    const unsigned u = (unsigned)i, c = (unsigned)cols, r = u / c;
    row = (int)r;
    col = (int)(u - r * c);
  } else {
    row = (int)(i / cols);
    col = (int)(i - (long long)row * cols);
  }
}

VL_DEV uint32_t ldcg(const uint32_t* p) { return __ldcg(p); }
VL_DEV int32_t ldcg(const int32_t* p) { return __ldcg(p); }
VL_DEV float ldcg(const float* p) { return __ldcg(p); }
VL_DEV uint8_t ldcg(const uint8_t* p) {
  return (uint8_t)__ldcg((const unsigned char*)p);
}

// First error wins.
VL_DEV void set_status(int32_t* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Horizontal dilation of word c given its left/right neighbour words.
VL_DEV uint32_t hdil(uint32_t l, uint32_t c, uint32_t r) {
  return c | (c << 1) | (l >> 31) | (c >> 1) | (r << 31);
}

// Dilated word from a 3x3 neighbourhood of words (rows u, m, d; columns
// left, centre, right).  conn 8: square; conn 4: cross.
VL_DEV uint32_t near_word(uint32_t ul, uint32_t uc, uint32_t ur, uint32_t ml,
                          uint32_t mc, uint32_t mr, uint32_t dl, uint32_t dc,
                          uint32_t dr, int conn) {
  if (conn == 8) return hdil(ul, uc, ur) | hdil(ml, mc, mr) | hdil(dl, dc, dr);
  return uc | dc | hdil(ml, mc, mr);
}

// Order-preserving map float -> uint32 (for selects on float keys); every
// NaN maps to the largest key, after +infinity.
VL_DEV uint32_t f2key(float f) {
  if (f != f) return 0xFFFFFFFFu;
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
VL_DEV float key2f(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(u);
}

// ---- number images: float or uint16 planes of H x pitch elements
// (a uint16 pixel is its integer value, exact in float)

// Channel ch of image im; plane_elems = H * pitch.
VL_DEV const void* chan_ptr(const DevImage& im, int ch, size_t plane_elems) {
  const size_t esz = im.format == PX_U16 ? 2 : 4;
  return static_cast<const char*>(im.data) + (size_t)ch * plane_elems * esz;
}

// Element i of a channel plane.  `nc`: the read-only path may be used (the
// image is not written during the launch).
VL_DEV float ld_px(const void* p, int format, bool nc, size_t i) {
  if (format == PX_U16) return (float)__ldg(static_cast<const unsigned short*>(p) + i);
  const float* f = static_cast<const float*>(p) + i;
  return nc ? __ldg(f) : __ldcg(f);
}

// Elements i .. i+3 (i a multiple of 4: 16- or 8-byte aligned).
VL_DEV float4 ld_px4(const void* p, int format, bool nc, size_t i) {
  if (format == PX_U16) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(static_cast<const unsigned short*>(p) + i));
    return make_float4((float)(u.x & 0xFFFFu), (float)(u.x >> 16), (float)(u.y & 0xFFFFu),
                       (float)(u.y >> 16));
  }
  const float4* f = reinterpret_cast<const float4*>(static_cast<const float*>(p) + i);
  return nc ? __ldg(f) : __ldcg(f);
}

}  // namespace vl
