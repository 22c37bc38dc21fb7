// Fused evaluation of a group of pointwise and N operators on one tile.
//
// A group is a sub-DAG of threshold atoms, not/and/or and N (Sec. 2) whose
// inputs are image channels or masks materialised by earlier steps.  Every
// value lives in a shared-memory buffer of (th + 2*halo) rows x (tww + 2)
// words: the core tile plus `halo` rows above and below and one 32-px word
// left and right.  A node whose value is needed `h` pixels beyond the core
// is computed over rows [halo - h, halo + th + h); N consumes one pixel of
// halo, so a chain of k N operators inside a group needs halo >= k (the
// compiler caps it at 31, inside the one-word horizontal margin).  Pixels
// outside the image are stored as 0, which is exactly the clipping of the
// neighbourhood at the image border.
#pragma once
#include "dev_common.cuh"

namespace vl {

struct GroupCtx {
  int H, W, Wp, pitch;
  int r0, w0, th, tww;  // core tile: image row, image word, rows, words
  int halo;
  int bh, bw;           // buffer rows (stride), buffer words
  int conn;
  uint32_t* buf;        // shared memory: buffers of bh * bw words
  const DevImage* images;
  uint32_t* const* slots;
  const float* pct_val;
};

VL_DEV uint32_t* gbuf(const GroupCtx& c, int b) { return c.buf + (size_t)b * c.bh * c.bw; }

VL_DEV void group_tile(const GroupCtx& c, const Insn* insns, int n_insn) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const int bw = c.bw;
  for (int k = 0; k < n_insn; ++k) {
    const Insn I = insns[k];
    const int h = I.h;
    const int i_lo = c.halo - h, i_hi = c.halo + c.th + h;  // buffer rows
    const int rows = i_hi - i_lo;
    if (I.op == I_THR) {
      const DevImage im = c.images[I.img];
      const float* plane = im.data + (size_t)I.ch * c.H * c.pitch;
      const float t = (I.slot >= 0) ? c.pct_val[I.slot] : I.t;
      const bool lt = (I.b & 1);
      uint32_t* d = gbuf(c, I.dst);
      const int nwords = rows * bw;
      for (int idx = warp; idx < nwords; idx += nw) {
        int i = i_lo + idx / bw, j = idx - (idx / bw) * bw;
        int y = c.r0 - c.halo + i, wg = c.w0 - 1 + j;
        uint32_t word = 0;
        if (y >= 0 && y < c.H && wg >= 0 && wg < c.Wp) {
          float v = __ldg(plane + (size_t)y * c.pitch + 32 * wg + lane);
          bool p = lt ? (v < t) : (v > t);
          word = __ballot_sync(0xFFFFFFFFu, p) & vmask(wg, c.W);
        }
        if (lane == 0) d[i * bw + j] = word;
      }
    } else if (I.op == I_STORE) {
      const uint32_t* a = gbuf(c, I.a);
      uint32_t* g = c.slots[I.slot];
      const int nwords = c.th * c.tww;
      for (int idx = tid; idx < nwords; idx += nthr) {
        int r = idx / c.tww, w = idx - r * c.tww;
        g[(size_t)(c.r0 + r) * c.Wp + c.w0 + w] = a[(c.halo + r) * bw + 1 + w];
      }
    } else {
      uint32_t* d = gbuf(c, I.dst);
      const uint32_t* a = gbuf(c, I.a);
      const uint32_t* b = gbuf(c, I.b);
      const uint32_t* g = (I.op == I_LOAD) ? c.slots[I.slot] : nullptr;
      const int nwords = rows * bw;
      for (int idx = tid; idx < nwords; idx += nthr) {
        int i = i_lo + idx / bw, j = idx - (idx / bw) * bw;
        int y = c.r0 - c.halo + i, wg = c.w0 - 1 + j;
        uint32_t word = 0;
        if (y >= 0 && y < c.H && wg >= 0 && wg < c.Wp) {
          const int o = i * bw + j;
          switch (I.op) {
            case I_LOAD: word = ldcg(&g[(size_t)y * c.Wp + wg]); break;
            case I_NOT: word = ~a[o] & vmask(wg, c.W); break;
            case I_AND: word = a[o] & b[o]; break;
            case I_OR: word = a[o] | b[o]; break;
            case I_ANDNOT: word = a[o] & ~b[o]; break;
            case I_CONST: word = I.b ? vmask(wg, c.W) : 0u; break;
            case I_NEAR: {
              uint32_t ul = 0, uc = a[o - bw], ur = 0, ml = 0, mc = a[o], mr = 0,
                       dl = 0, dc = a[o + bw], dr = 0;
              if (j > 0) { ul = a[o - bw - 1]; ml = a[o - 1]; dl = a[o + bw - 1]; }
              if (j + 1 < bw) { ur = a[o - bw + 1]; mr = a[o + 1]; dr = a[o + bw + 1]; }
              word = near_word(ul, uc, ur, ml, mc, mr, dl, dc, dr, c.conn) & vmask(wg, c.W);
              break;
            }
            default: break;
          }
        }
        d[i * bw + j] = word;
      }
    }
    __syncthreads();
  }
}

}  // namespace vl
