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
  // rank codes (I_RTHR): tables, the job's planes, and a shared-memory
  // stage beside the buffers for the planes of the group's tables
  const RankTab* rtab;
  const uint32_t* planes;
  size_t pstride;       // words per plane (H * Wp)
  uint32_t* stage;
  int stage_cap;        // words
  int rank_mask, rank_halo;
};

VL_DEV void cp_async4(uint32_t* smem_dst, const uint32_t* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
VL_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
VL_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Words of the stage that the planes of the group's rank tables take (rows
// of the core tile plus rank_halo above and below, all buffer words).
VL_DEV int rank_stage_words(const GroupCtx& c, int upto_table) {
  const int per_plane = (c.th + 2 * c.rank_halo) * c.bw;
  int n = 0;
  for (unsigned m = (unsigned)c.rank_mask; m; m &= m - 1) {
    const int t = __ffs(m) - 1;
    if (t >= upto_table) break;
    n += (c.rtab[t].nbits + 1) * per_plane;
  }
  return n;
}

// Start copying the planes of the group's rank tables into the stage (each
// thread its share of words, asynchronously); returns whether they fit.
VL_DEV bool rank_stage_begin(const GroupCtx& c) {
  if (!c.rank_mask || rank_stage_words(c, 32) > c.stage_cap) return false;
  const int rows_s = c.th + 2 * c.rank_halo;
  const int per_plane = rows_s * c.bw;
  uint32_t* dst = c.stage;
  for (unsigned m = (unsigned)c.rank_mask; m; m &= m - 1) {
    const RankTab T = c.rtab[__ffs(m) - 1];
    for (int p = 0; p <= T.nbits; ++p, dst += per_plane) {
      const uint32_t* src = c.planes + (size_t)(T.plane0 + p) * c.pstride;
      for (int idx = threadIdx.x; idx < per_plane; idx += blockDim.x) {
        const int i = idx / c.bw, j = idx - (idx / c.bw) * c.bw;
        const int y = c.r0 - c.rank_halo + i, wg = c.w0 - 1 + j;
        if (y >= 0 && y < c.H && wg >= 0 && wg < c.Wp) cp_async4(dst + idx, src + (size_t)y * c.Wp + wg);
      }
    }
  }
  cp_async_commit();
  return true;
}

// Most code bits of a rank table (values <= 8191: codes < 2^14).
constexpr int kRankMaxBits = 14;

// The instruction stream and the slot table are read-only for the whole
// launch: both go through the read-only data cache, so that every tile of a
// step after the first on an SM finds them in L1 instead of L2.
VL_DEV Insn ld_insn(const Insn* p) {
  const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
  Insn I;
  memcpy(&I, &v, sizeof(Insn));
  return I;
}
VL_DEV uint32_t* ld_slot(uint32_t* const* slots, int k) {
  return reinterpret_cast<uint32_t*>(
      __ldg(reinterpret_cast<const unsigned long long*>(slots + k)));
}


// Word ownership: buffer word idx (row-major, idx = row * bw + word) is
// always read and written by thread idx mod EXEC_THREADS, by every
// instruction except the float threshold, so that the compiler needs a
// block barrier (I_SYNC) only where a thread touches a word another thread
// touched since the previous one.  First word of [lo, ...) this thread owns.
VL_DEV int own_first(int lo, int tid) {
  return lo <= tid ? tid : tid + ((lo - tid + EXEC_THREADS - 1) / EXEC_THREADS) * EXEC_THREADS;
}

// BW > 0: the buffer row length as a compile-time constant (index
// arithmetic and divisions by the row length fold into multiplies); 0: read
// from c.  The number of buffer rows is only a stride between buffers and
// stays a run-time value, so that any tile height runs the fast path.
// Launched with EXEC_THREADS threads.
template <int BW>
VL_DEV void group_tile_t(const GroupCtx& c, const Insn* insns, int n_insn) {
  const int tid = threadIdx.x, nthr = EXEC_THREADS;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const int bw = BW > 0 ? BW : c.bw;
  const int bhbw = c.bh * bw;
  auto gbuf = [&](int b) { return c.buf + (size_t)b * bhbw; };
  // 0: planes read from global memory; 1: being staged; 2: staged
  int stage = rank_stage_begin(c) ? 1 : 0;
  for (int k = 0; k < n_insn; ++k) {
    const Insn I = ld_insn(insns + k);
    if (I.op & I_SYNC) __syncthreads();  // uniform: one instruction stream per CTA
    const int op = I.op & ~I_SYNC;
    const int h = I.h;
    const int i_lo = c.halo - h, i_hi = c.halo + c.th + h;  // buffer rows
    const int rows = i_hi - i_lo;
    const int w_lo = i_lo * bw, w_hi = i_hi * bw;           // buffer words
    if (op == I_RTHR) {
      if (stage == 1) {  // uniform: every thread waits for its copies, then all
        cp_async_wait_all();
        __syncthreads();
        stage = 2;
      }
      const int nb = I.ch;
      const unsigned K = (uint16_t)I.img;
      const bool lt = I.b & 1;
      const int per_plane = (c.th + 2 * c.rank_halo) * bw;
      const uint32_t* sp = c.stage + rank_stage_words(c, I.a);
      const int s_row0 = c.halo - c.rank_halo;  // buffer row of stage row 0
      uint32_t* d = gbuf(I.dst);
      for (int idx = own_first(w_lo, tid); idx < w_hi; idx += nthr) {
        const int i = idx / bw, j = idx - (idx / bw) * bw;
        const int y = c.r0 - c.halo + i, wg = c.w0 - 1 + j;
        uint32_t word = 0;
        if (y >= 0 && y < c.H && wg >= 0 && wg < c.Wp) {
          // bit-sliced code >= K: the subtraction code - K must not borrow.
          // Bit b passes the borrow on as ~x_b | borrow where K_b = 1 and
          // as ~x_b & borrow where K_b = 0, i.e. the majority of (~x_b,
          // borrow, K_b) -- one logic op per plane.  Below K's lowest set
          // bit no borrow starts, so the chain begins there (K = 0: code
          // >= K everywhere).  K's bits are the same for every thread.
          // (two separate loops: a select between a shared and a global load
          // inside one loop made every word wait for global memory)
          uint32_t borrow = 0, nan = 0;
          const int b0 = K ? __ffs(K) - 1 : nb;
          if (stage) {
            const uint32_t* s0 = sp + (size_t)(i - s_row0) * bw + j;
#pragma unroll 4
            for (int b = 0; b < kRankMaxBits; ++b) {
              if (b < b0 || b >= nb) continue;
              const uint32_t x = s0[b * per_plane], km = 0u - ((K >> b) & 1u);
              borrow = (~x & borrow) | (~x & km) | (borrow & km);
            }
            if (lt) nan = s0[nb * per_plane];
          } else {
            const uint32_t* g0 = c.planes + (size_t)I.slot * c.pstride + (size_t)y * c.Wp + wg;
            for (int b = b0; b < nb; ++b) {
              const uint32_t x = ldcg(g0 + (size_t)b * c.pstride), km = 0u - ((K >> b) & 1u);
              borrow = (~x & borrow) | (~x & km) | (borrow & km);
            }
            if (lt) nan = ldcg(g0 + (size_t)nb * c.pstride);
          }
          const uint32_t ge = ~borrow;
          word = lt ? (~ge & ~nan) : ge;
          word &= vmask(wg, c.W);
        }
        d[idx] = word;
      }
    } else if (op == I_THR) {
      const DevImage im = c.images[I.img];
      const void* plane = chan_ptr(im, I.ch, (size_t)c.H * c.pitch);
      const int fmt = im.format;
      const bool nc = !im.written;
      const float t = (I.slot >= 0) ? c.pct_val[I.slot] : I.t;
      const bool lt = (I.b & 1);
      uint32_t* d = gbuf(I.dst);
      const int nwords = rows * bw;
      // one 16-byte load per lane covers 4 pixels: a warp reads 4 words
      // (512 bytes) per load and keeps UNR loads in flight; the 8 lanes of a
      // word merge their 4-bit pieces with three shuffles
      constexpr int UNR = 2;
      const int sub = lane & 7;
      if (fmt == PX_U16) {
        // uint16 planes: 8-byte loads of 4 pixels per lane, UNR16 in flight
        constexpr int UNR16 = 2;
        const unsigned short* p16 = static_cast<const unsigned short*>(plane);
        for (int base = warp * 4 * UNR16; base < nwords; base += nw * 4 * UNR16) {
          uint2 q[UNR16];
#pragma unroll
          for (int u = 0; u < UNR16; ++u) {
            const int idx = base + 4 * u + (lane >> 3);
            const int i = i_lo + idx / bw, wg = c.w0 - 1 + (idx - (idx / bw) * bw);
            const int y = c.r0 - c.halo + i;
            const bool in = idx < nwords && y >= 0 && y < c.H && wg >= 0 && wg < c.Wp;
            q[u] = in ? __ldg(reinterpret_cast<const uint2*>(p16 + (size_t)y * c.pitch + 32 * wg + 4 * sub))
                      : make_uint2(0u, 0u);
          }
#pragma unroll
          for (int u = 0; u < UNR16; ++u) {
            const int idx = base + 4 * u + (lane >> 3);
            const int i = i_lo + idx / bw, j = idx - (idx / bw) * bw, wg = c.w0 - 1 + j;
            const int y = c.r0 - c.halo + i;
            const bool in = idx < nwords && y >= 0 && y < c.H && wg >= 0 && wg < c.Wp;
            const float v0 = (float)(q[u].x & 0xFFFFu), v1 = (float)(q[u].x >> 16);
            const float v2 = (float)(q[u].y & 0xFFFFu), v3 = (float)(q[u].y >> 16);
            const uint32_t nib = lt ? ((v0 < t) | ((v1 < t) << 1) | ((v2 < t) << 2) | ((v3 < t) << 3))
                                    : ((v0 > t) | ((v1 > t) << 1) | ((v2 > t) << 2) | ((v3 > t) << 3));
            uint32_t word = nib << (4 * sub);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
            if (sub == 0 && idx < nwords) d[i * bw + j] = in ? (word & vmask(wg, c.W)) : 0u;
          }
        }
      } else
      for (int base = warp * 4 * UNR; base < nwords; base += nw * 4 * UNR) {
        float4 v[UNR];
        uint32_t inm = 0;
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int idx = base + 4 * u + (lane >> 3);
          const int i = i_lo + idx / bw, wg = c.w0 - 1 + (idx - (idx / bw) * bw);
          const int y = c.r0 - c.halo + i;
          const bool in = idx < nwords && y >= 0 && y < c.H && wg >= 0 && wg < c.Wp;
          const float4* p4 = reinterpret_cast<const float4*>(
              static_cast<const float*>(plane) + (size_t)y * c.pitch + 32 * wg) + sub;
          v[u] = in ? (nc ? __ldg(p4) : __ldcg(p4)) : make_float4(0.f, 0.f, 0.f, 0.f);
          inm |= (in ? 1u : 0u) << u;
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          uint32_t nib;
          if (lt) nib = (v[u].x < t) | ((v[u].y < t) << 1) | ((v[u].z < t) << 2) | ((v[u].w < t) << 3);
          else nib = (v[u].x > t) | ((v[u].y > t) << 1) | ((v[u].z > t) << 2) | ((v[u].w > t) << 3);
          uint32_t word = nib << (4 * sub);
          word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
          word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
          word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
          const int idx = base + 4 * u + (lane >> 3);
          if (sub == 0 && idx < nwords) {
            const int i = i_lo + idx / bw, j = idx - (idx / bw) * bw;
            d[i * bw + j] = ((inm >> u) & 1u) ? (word & vmask(c.w0 - 1 + j, c.W)) : 0u;
          }
        }
      }
    } else if (op == I_STORE) {
      // the core words, each from the thread that owns it in the buffer
      const uint32_t* a = gbuf(I.a);
      uint32_t* g = ld_slot(c.slots, I.slot);
      const int s_hi = (c.halo + c.th) * bw;
      for (int idx = own_first(c.halo * bw, tid); idx < s_hi; idx += nthr) {
        const int i = idx / bw, j = idx - (idx / bw) * bw;
        if (j >= 1 && j <= c.tww) g[(size_t)(c.r0 + i - c.halo) * c.Wp + c.w0 + j - 1] = a[idx];
      }
    } else if (op == I_AND || op == I_OR || op == I_ANDNOT) {
      // every buffer holds 0 outside the image, and so does the result of
      // these three: no bounds to check
      uint32_t* d = gbuf(I.dst);
      const uint32_t* a = gbuf(I.a);
      const uint32_t* b = gbuf(I.b);
      const int first = own_first(w_lo, tid);
      if (op == I_AND) {
        for (int idx = first; idx < w_hi; idx += nthr) d[idx] = a[idx] & b[idx];
      } else if (op == I_OR) {
        for (int idx = first; idx < w_hi; idx += nthr) d[idx] = a[idx] | b[idx];
      } else {
        for (int idx = first; idx < w_hi; idx += nthr) d[idx] = a[idx] & ~b[idx];
      }
    } else {
      uint32_t* d = gbuf(I.dst);
      const uint32_t* a = gbuf(I.a);
      const uint32_t* b = gbuf(I.b);
      const uint32_t* g = (op == I_LOAD) ? ld_slot(c.slots, I.slot) : nullptr;
      for (int idx = own_first(w_lo, tid); idx < w_hi; idx += nthr) {
        const int i = idx / bw, j = idx - (idx / bw) * bw;
        const int y = c.r0 - c.halo + i, wg = c.w0 - 1 + j;
        uint32_t word = 0;
        if (y >= 0 && y < c.H && wg >= 0 && wg < c.Wp) {
          const int o = idx;
          switch (op) {
            case I_LOAD: word = ldcg(&g[(size_t)y * c.Wp + wg]); break;
            case I_NOT: word = ~a[o] & vmask(wg, c.W); break;
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
        d[idx] = word;
      }
    }
  }
  if (stage == 1) cp_async_wait_all();  // no copy may outlive the tile
}

// The group interpreter for the tile widths the autotuner tries (buffer
// words = tile words + 2: 32, 16 and 8-word tiles), generic otherwise.
VL_DEV void group_tile(const GroupCtx& c, const Insn* insns, int n_insn) {
  switch (c.bw) {
    case 34: group_tile_t<34>(c, insns, n_insn); break;
    case 18: group_tile_t<18>(c, insns, n_insn); break;
    case 10: group_tile_t<10>(c, insns, n_insn); break;
    default: group_tile_t<0>(c, insns, n_insn); break;
  }
}

}  // namespace vl
